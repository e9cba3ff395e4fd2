"""Host build of the tridiagonal QR chain the MinSR cutoff route runs on one GPU thread
(paper_2503_12557_gb300/csrc/peps_tdql.cuh, plain scalar code): compiled with the host C++
compiler and checked against numpy's symmetric eigensolver on random tridiagonal matrices.

td_ql turns y into Z^T y and d into the eigenvalues, recording every rotation in one double;
td_replay applies Z.  So Z f(Lambda) Z^T y must equal V f(Lambda) V^T y from eigh for any f, the
eigenvalues must agree, the rotation encoding must round-trip, and the two failure exits (the
record's capacity, the iteration limit on non-finite input) must be reported, not overrun.
"""
import os
import shutil
import struct
import subprocess

import numpy as np
import pytest

HDR = os.path.join(os.path.dirname(__file__), "..", "paper_2503_12557_gb300", "csrc", "peps_tdql.cuh")

DRIVER = r"""
#define __host__
#define __device__
#define __forceinline__ inline
#include <cstdio>
#include <cstdlib>
#include <vector>
#include "peps_tdql.cuh"
// stdin: N, cap, mode, d[N], e[N], y[N], f[?]   mode 0: u = f(Lambda) Z^T y, then Z u
// stdout: status, steps, len, d[N], y[N]
int main() {
  int N, mode; long long cap;
  if (fread(&N, 4, 1, stdin) != 1 || fread(&cap, 8, 1, stdin) != 1 || fread(&mode, 4, 1, stdin) != 1) return 2;
  std::vector<double> d(N + 1), e(N + 1), y(N + 1);
  if (fread(d.data(), 8, N, stdin) != (size_t)N || fread(e.data(), 8, N, stdin) != (size_t)N ||
      fread(y.data(), 8, N, stdin) != (size_t)N) return 2;
  const size_t cap0 = (size_t)cap / 2, cap1 = (size_t)cap - cap0;
  std::vector<double> r0(cap0 + 1), r1(cap1 + 1);
  long long steps = 0; size_t len = 0;
  int st = peps::td_ql(d.data(), e.data(), y.data(), N, r0.data(), cap0, r1.data(), cap1, 60, &steps, &len);
  if (st == 0 && mode == 0) {
    for (int i = 0; i < N; ++i) y[i] = y[i] / (1.0 + d[i] * d[i]);   // f(Lambda) = 1 / (1 + Lambda^2)
    peps::td_replay(y.data(), r0.data(), cap0, r1.data(), len);
  }
  fwrite(&st, 4, 1, stdout); fwrite(&steps, 8, 1, stdout); long long l = (long long)len; fwrite(&l, 8, 1, stdout);
  fwrite(d.data(), 8, N, stdout); fwrite(y.data(), 8, N, stdout);
  if (mode == 1) {  // encoding round trip over the angles in y
    for (int i = 0; i < N; ++i) {
      double c = cos(y[i]), s = sin(y[i]);
      if (c < 0) { c = -c; s = -s; }
      double c2, s2; peps::td_dec(peps::td_enc(c, s), c2, s2);
      double err = fmax(fabs(c2 - c), fabs(s2 - s)); fwrite(&err, 8, 1, stdout);
    }
  }
  return 0;
}
"""


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    d = tmp_path_factory.mktemp("tdql")
    src = d / "drv.cpp"
    src.write_text(DRIVER)
    exe = d / "drv"
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", os.path.dirname(os.path.abspath(HDR)), str(src), "-o", str(exe)],
                   check=True, capture_output=True)
    return str(exe)


def _run(exe, d, e, y, cap=None, mode=0):
    N = len(d)
    cap = 2 * max(N * N, 4096) if cap is None else cap
    inp = struct.pack("<iqi", N, cap, mode) + np.asarray(d, float).tobytes() + np.asarray(e, float).tobytes() \
        + np.asarray(y, float).tobytes()
    out = subprocess.run([exe], input=inp, capture_output=True, check=True).stdout
    st, steps, ln = struct.unpack("<iqq", out[:20])
    arr = np.frombuffer(out[20:], dtype=np.float64)
    return st, steps, ln, arr[:N].copy(), arr[N:2 * N].copy(), arr[2 * N:].copy()


@pytest.mark.parametrize("N,seed", [(1, 0), (2, 1), (3, 2), (17, 3), (64, 4), (200, 5)])
def test_qr_chain_applies_f_of_the_tridiagonal(driver, N, seed):
    rng = np.random.default_rng(seed)
    d = rng.standard_normal(N) * 3.0
    e = np.zeros(N)
    e[:N - 1] = rng.standard_normal(N - 1)
    y = rng.standard_normal(N)
    st, steps, ln, lam, u, _ = _run(driver, d, e, y)
    assert st == 0
    Tri = np.diag(d) + np.diag(e[:N - 1], 1) + np.diag(e[:N - 1], -1)
    w, V = np.linalg.eigh(Tri)
    assert np.allclose(np.sort(lam), w, rtol=0, atol=1e-13 * max(1.0, np.abs(w).max()))
    ref = V @ ((V.T @ y) / (1.0 + w * w))
    assert np.linalg.norm(u - ref) <= 1e-13 * np.linalg.norm(ref)
    assert ln <= 2 * max(N * N, 4096)


def test_qr_chain_graded_and_clustered_spectra(driver):
    # the spectra MinSR meets: eigenvalues spread over many decades, exact pairs (the real
    # embedding of a complex T), a zero block
    rng = np.random.default_rng(7)
    Q, _ = np.linalg.qr(rng.standard_normal((60, 60)))
    lam = np.concatenate([10.0 ** rng.uniform(-8, 3, 40), np.repeat(rng.uniform(0.5, 2.0, 5), 2), np.zeros(10)])
    A = (Q * lam) @ Q.T
    # Householder tridiagonal form of A (numpy, the test's own reduction)
    n = len(lam)
    T = A.copy()
    for k in range(n - 2):
        x = T[k + 1:, k].copy()
        a = -np.copysign(np.linalg.norm(x), x[0])
        v = x.copy()
        v[0] -= a
        nv = np.linalg.norm(v)
        if nv == 0:
            continue
        v /= nv
        H = np.eye(n - k - 1) - 2 * np.outer(v, v)
        T[k + 1:, :] = H @ T[k + 1:, :]
        T[:, k + 1:] = T[:, k + 1:] @ H
    d = np.diag(T).copy()
    e = np.zeros(n)
    e[:n - 1] = np.diag(T, 1)
    y = rng.standard_normal(n)
    st, steps, ln, ev, u, _ = _run(driver, d, e, y)
    assert st == 0
    Tri = np.diag(d) + np.diag(e[:n - 1], 1) + np.diag(e[:n - 1], -1)
    w, V = np.linalg.eigh(Tri)
    assert np.allclose(np.sort(ev), w, rtol=0, atol=1e-13 * np.abs(w).max())
    ref = V @ ((V.T @ y) / (1.0 + w * w))
    assert np.linalg.norm(u - ref) <= 1e-12 * np.linalg.norm(ref)


def test_rotation_encoding_round_trip(driver):
    ang = np.concatenate([np.linspace(-np.pi, np.pi, 2001), [0.0, np.pi / 2, -np.pi / 2, np.pi / 4, -np.pi / 4,
                                                             np.pi / 4 + 1e-15, 1e-300, np.pi / 2 - 1e-12]])
    st, steps, ln, _, _, err = _run(driver, np.zeros(len(ang)), np.zeros(len(ang)), ang, mode=1)
    assert st == 0 and len(err) == len(ang)
    assert err.max() <= 1e-15


def test_record_capacity_and_iteration_limit_are_reported(driver):
    rng = np.random.default_rng(11)
    N = 50
    d, e, y = rng.standard_normal(N), rng.standard_normal(N), rng.standard_normal(N)
    st, *_ = _run(driver, d, e, y, cap=100)
    assert st == 2  # the record would pass its capacity: stopped before writing past it
    d2 = d.copy()
    d2[10] = np.nan
    st, steps, *_ = _run(driver, d2, e, y)
    assert st == 1 and steps <= 61  # a non-finite entry never deflates: the iteration limit ends it

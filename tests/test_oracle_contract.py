"""Pins of the oracle's boundary-MPS contraction against exact contractions and closed facts.

* Two exact routes (dense row transfer, one einsum over the whole network) agree.
* Boundary MPS with chi at the exact rank equals the exact amplitude (truncation is the only
  approximation, Sec. "On the boundary MPS method").
* psi_x and psi_{x,x+1} equal psi_top at exact chi (Eq. (boundary_MPS_approx) holds for every i).
* The truncation equals the sequence of full-vector Schmidt projections (brute force) and the
  independent density-matrix form.
"""
import math

import numpy as np
import pytest

from paper_2503_12557_gb300.inputs import (Lattice, peps_random, configs_uniform_sz0, configs_uniform,
                                           theta_to_tensors)
from oracle import tn, exact


def test_exact_routes_agree():
    for (Lx, Ly, D, cplx) in [(2, 2, 2, False), (2, 3, 2, False), (3, 3, 2, True), (3, 2, 3, False)]:
        lat = Lattice(Lx, Ly, 2, D)
        th = peps_random(lat, 11 + Lx * Ly, complex_=cplx)
        for S in configs_uniform(lat, 5, 3):
            a = exact.amplitude_rowtransfer(th, S, lat)
            b = exact.amplitude_fullnet(th, S, lat)
            assert abs(a - b) <= 1e-12 * abs(b)


def test_state_vector_matches_rowtransfer():
    lat = Lattice(3, 3, 2, 2)
    th = peps_random(lat, 5)
    psi = exact.state_vector(th, lat)
    for S in configs_uniform(lat, 6, 1):
        assert abs(psi[exact.config_index(S, 2)] - exact.amplitude_rowtransfer(th, S, lat)) < 1e-12 * abs(psi).max()


@pytest.mark.parametrize("cplx", [False, True])
def test_boundary_mps_exact_chi_4x4(cplx):
    # 4x4, D=2: chi = 4 = D^2 is exact (the exact boundary bond is at most D^floor(Ly/2) = 4)
    lat = Lattice(4, 4, 2, 2)
    th = peps_random(lat, 1001, complex_=cplx)
    for S in configs_uniform_sz0(lat, 12, 2001):
        la, ph, st = tn.log_amplitude(th, S, lat, 4)
        ex = exact.amplitude_rowtransfer(th, S, lat)
        assert st == 0
        assert abs(la - math.log(abs(ex))) < 1e-12
        assert abs(np.exp(1j * ph) - ex / abs(ex)) < 1e-12


def test_psi_rows_equal_at_exact_chi():
    lat = Lattice(4, 5, 2, 2)
    th = peps_random(lat, 77)
    T = theta_to_tensors(lat, th)
    for S in configs_uniform(lat, 4, 9):
        env, Ap = tn.environments(T, S, lat, 64)
        ex = exact.amplitude_rowtransfer(th, S, lat)
        for x in range(lat.Lx):
            l, p = tn.log_psi_row(env, Ap, x)
            assert abs(l - math.log(abs(ex))) < 1e-11
            assert abs(math.cos(p) - np.sign(ex)) < 1e-12
        for x in range(lat.Lx - 1):
            l, p = tn.log_psi_pair(env, Ap, x)
            assert abs(l - math.log(abs(ex))) < 1e-11


def test_truncated_rows_differ_but_close():
    # below the exact rank psi_x depends on x (the fast estimator's non-variational spread)
    lat = Lattice(6, 6, 2, 3)
    th = peps_random(lat, 3, scale=0.3, bias=1.0)
    T = theta_to_tensors(lat, th)
    S = configs_uniform_sz0(lat, 1, 4)[0]
    env, Ap = tn.environments(T, S, lat, 4)
    ls = [tn.log_psi_row(env, Ap, x)[0] for x in range(lat.Lx)]
    assert max(ls) - min(ls) > 1e-8
    env9, Ap9 = tn.environments(T, S, lat, 27)
    ex = math.log(abs(exact.amplitude_rowtransfer(th, S, lat)))
    assert abs(tn.log_psi_row(env9, Ap9, lat.Lx - 1)[0] - ex) < 1e-11


def _random_mps(n, p, bond, seed, decay=0.6):
    rng = np.random.default_rng(seed)
    out = []
    dims = [1] + [bond] * (n - 1) + [1]
    for k in range(n):
        t = rng.standard_normal((dims[k], p, dims[k + 1]))
        # spread the spectrum so that cuts are gapped
        t = t * (decay ** np.arange(dims[k + 1]))[None, None, :]
        out.append(t)
    return out


def _bruteforce_truncate(vec, n, p, chi):
    """Sequential Schmidt projections on the full vector, cut (n-1 | 1) first, then leftwards."""
    v = vec.copy()
    for k in range(n - 1, 0, -1):
        M = v.reshape(p ** k, p ** (n - k))
        U, s, Vh = np.linalg.svd(M, full_matrices=False)
        keep = min(chi, len(s))
        P = np.conj(Vh[:keep].T) @ Vh[:keep]
        v = (M @ P).reshape(-1)
    return v


@pytest.mark.parametrize("n,p,bond,chi", [(5, 2, 6, 3), (6, 3, 8, 4), (4, 4, 9, 5)])
def test_truncate_svd_equals_bruteforce(n, p, bond, chi):
    mps = _random_mps(n, p, bond, seed=n * 100 + chi)
    vec = tn.mps_to_vector(mps)
    ref = _bruteforce_truncate(vec, n, p, chi)
    got, st, w = tn.truncate_svd(mps, chi)
    gv = tn.mps_to_vector(got)
    assert max(e.shape[0] for e in got[1:]) <= chi
    assert np.linalg.norm(gv - ref) <= 1e-10 * np.linalg.norm(ref)
    # discarded weight is reported and the truncation is not trivial here
    assert 0 < w < 1


@pytest.mark.parametrize("n,p,bond,chi", [(5, 2, 6, 3), (6, 4, 8, 5)])
def test_truncate_dm_equals_svd(n, p, bond, chi):
    mps = _random_mps(n, p, bond, seed=7 * n + chi)
    a, _, _ = tn.truncate_svd(mps, chi)
    b = tn.truncate_dm(mps, chi)
    va, vb = tn.mps_to_vector(a), tn.mps_to_vector(b)
    assert np.linalg.norm(va - vb) <= 1e-9 * np.linalg.norm(va)


def _bruteforce_truncate_cut(vec, n, p, chi, cut):
    """As _bruteforce_truncate with the truncated-weight rule: at every cut keep the fewest
    Schmidt values (at most chi) whose discarded share of sum s^2 is at most cut."""
    v = vec.copy()
    kept = []
    for k in range(n - 1, 0, -1):
        M = v.reshape(p ** k, p ** (n - k))
        U, s, Vh = np.linalg.svd(M, full_matrices=False)
        tot = float(np.sum(s ** 2))
        keep = 1
        while keep < len(s) and float(np.sum(s[keep:] ** 2)) / tot > cut:
            keep += 1
        keep = min(keep, chi)
        kept.append(keep)
        P = np.conj(Vh[:keep].T) @ Vh[:keep]
        v = (M @ P).reshape(-1)
    return v, kept


@pytest.mark.parametrize("n,p,bond,chi,cut", [(6, 2, 8, 8, 1e-2), (5, 3, 9, 9, 5e-3), (6, 2, 8, 3, 1e-4)])
def test_truncate_cutoff_equals_bruteforce(n, p, bond, chi, cut):
    # decaying spectra, so that the cutoff, not chi, sets most bond dimensions
    mps = _random_mps(n, p, bond, seed=31 * n + bond)
    for k, e in enumerate(mps):
        mps[k] = e * (0.45 ** np.arange(e.shape[2]))[None, None, :]
    vec = tn.mps_to_vector(mps)
    ref, kept = _bruteforce_truncate_cut(vec, n, p, chi, cut)
    got, st, w = tn.truncate_svd(mps, (chi, cut))
    assert st == 0
    assert [e.shape[0] for e in got[1:]][::-1] == kept
    assert min(kept) < min(chi, bond)  # the cutoff, not the cap, sets some bond
    assert np.linalg.norm(tn.mps_to_vector(got) - ref) <= 1e-10 * np.linalg.norm(ref)
    assert w <= cut
    # the density-matrix form applies the same rule
    b = tn.truncate_dm(mps, (chi, cut))
    assert np.linalg.norm(tn.mps_to_vector(b) - ref) <= 1e-9 * np.linalg.norm(ref)


def test_truncate_cutoff_zero_is_fixed_chi():
    mps = _random_mps(5, 2, 6, seed=8)
    a, _, _ = tn.truncate_svd(mps, 3)
    b, _, _ = tn.truncate_svd(mps, (3, 0.0))
    assert all(np.array_equal(x, y) for x, y in zip(a, b))


def test_cut_margin_hand_computed():
    # s^2 = (0.9, 0.08, 0.015, 0.005), cutoff 0.01: tails 0.1, 0.02, 0.005 -> three kept; the
    # comparisons that decide it sit 9, 1 and 0.5 cutoffs away from it (0.5 the smallest)
    s = np.sqrt([0.9, 0.08, 0.015, 0.005])
    assert tn.keep_count(s, 4, 0.01) == (3, 0)
    assert abs(tn.cut_margin(s, 4, 0.01) - 0.5) < 1e-12
    assert abs(tn.cut_margin(s, 2, 0.01) - 1.0) < 1e-12      # chi = 2 caps it: only k = 1, 2 decide
    assert tn.cut_margin(s, 4, 0.0) == math.inf
    # a tail sitting on the cutoff (up to rounding): zero margin and the near-cutoff flag
    s2 = np.sqrt([0.97, 0.02, 0.01, 0.0])
    assert tn.cut_margin(s2, 4, 0.01) < 1e-12
    assert tn.keep_count(s2, 4, 0.01)[1] == tn.NEAR_DEGENERATE


def test_truncate_at_full_rank_is_identity():
    mps = _random_mps(5, 2, 4, seed=3)
    got, st, w = tn.truncate_svd(mps, 64)
    assert np.allclose(tn.mps_to_vector(got), tn.mps_to_vector(mps), rtol=0, atol=1e-12)
    assert w < 1e-28


def test_normalisation_is_bookkeeping():
    mps = _random_mps(4, 3, 5, seed=1)
    scaled = [e * 10.0 ** (k + 3) for k, e in enumerate(mps)]
    nm, lg, st = tn.normalize(scaled)
    assert st == 0
    for e in nm:
        assert abs(np.max(np.abs(e)) - 1.0) < 1e-15
    v = tn.mps_to_vector(nm) * math.exp(lg)
    assert np.allclose(v, tn.mps_to_vector(scaled), rtol=1e-12)


def test_zero_normaliser_flag():
    mps = _random_mps(3, 2, 2, seed=1)
    mps[1] = np.zeros_like(mps[1])
    _, lg, st = tn.normalize(mps)
    assert st & tn.ZERO_NORM and lg == -math.inf


def test_near_degenerate_flag():
    s = np.array([1.0, 0.5, 0.5, 0.1])
    assert tn._cut_flags(s, 2) == tn.NEAR_DEGENERATE
    assert tn._cut_flags(s, 1) == 0
    assert tn._cut_flags(np.array([1.0, 0.5, 1e-13, 1e-13]), 2) == 0

"""The variational-bound local energy (oracle, FP64; test infrastructure only).

Paper: Sec. "On Variational Upper Bound to the Ground State Energy" and the appendix on
variational upper bounds.  The fast estimator (energy.local_energy) takes each ratio
psi(S')/psi(S) from whichever boundary-MPS pair lies next to the term, so different terms see
different approximations of psi.  Fixing one cut i for every amplitude,

    psi_i(S) = E^u[i](S) . E^l[i+1](S)

(the upper boundary MPS of the first i rows overlapped with the lower boundary MPS of the
remaining rows; the paper numbers rows from 1, so i = 1 .. Lx-1), makes the estimator

    E_loc^bound(S) = sum_S' <S|H|S'> psi_i(S') / psi_i(S)

the local energy of one fixed state |psi_i>: its |psi_i|^2-weighted mean is
<psi_i|H|psi_i> / <psi_i|psi_i>, an upper bound of the ground-state energy.

Everything here is computed from scratch for every configuration (no environment reuse):
psi_i(S') builds the environments of S' itself.  Readings: the overlap is the plain contraction
(no complex conjugation, like psi); <S|h|S'> in the matrix-element order of energy.py; the
status of E_loc^bound ORs the status of S's full environment pass with that of every S'
amplitude.
"""
from __future__ import annotations

import math

import numpy as np

from paper_2503_12557_gb300.inputs import Lattice, theta_to_tensors
from . import tn


def _overlap(eu, el):
    """Plain contraction of two boundary MPS over their shared physical legs,
    sum E^u[a_0 p_0 a_1] E^l[b_0 p_0 b_1] E^u[a_1 p_1 a_2] E^l[b_1 p_1 b_2] ...,
    column by column from the left, each partial divided by its largest modulus.
    Returns (normalised scalar, log scale)."""
    L = np.ones((1, 1), dtype=np.result_type(eu[0], el[0]))
    logs = 0.0
    for y in range(len(eu)):
        L = np.einsum("ab,apx,bpz->xz", L, eu[y], el[y])
        m = float(np.max(np.abs(L)))
        if m == 0.0 or not np.isfinite(m):
            return 0.0, -math.inf
        L = L / m
        logs += math.log(m)
    return L[0, 0], logs


def psi_cut(T, S, lat: Lattice, chi, i: int):
    """(ln|psi_i(S)|, phase, status): upper boundary MPS through row i-1 (0-based rows
    0 .. i-1), lower boundary MPS from row Lx-1 up to row i, and their overlap.  Each
    environment row is truncated and normalised as in tn.environments."""
    if not 1 <= i <= lat.Lx - 1:
        raise ValueError("cut i must lie in 1 .. Lx-1")
    Ap = tn.project(T, S, lat)
    st = 0
    eu, lu, s0 = tn.normalize(tn.top_row_mps(Ap[0]))
    st |= s0
    for x in range(1, i):
        tr, s1, _ = tn.truncate_svd(tn.apply_down(eu, Ap[x]), chi)
        eu, lg, s2 = tn.normalize(tr)
        st |= s1 | s2
        lu += lg
    el, ll, s0 = tn.normalize(tn.bottom_row_mps(Ap[lat.Lx - 1]))
    st |= s0
    for x in range(lat.Lx - 2, i - 1, -1):
        tr, s1, _ = tn.truncate_svd(tn.apply_up(el, Ap[x]), chi)
        el, lg, s2 = tn.normalize(tr)
        st |= s1 | s2
        ll += lg
    v, lo = _overlap(eu, el)
    if v == 0:
        return -math.inf, 0.0, st
    return math.log(abs(v)) + lo + lu + ll, float(np.angle(v)), st


def local_energy_bound(theta, S, lat: Lattice, chi, H, i: int, T=None):
    """E_loc^bound(S) (complex), ln|psi_i(S)|, its phase and the status bits."""
    T = theta_to_tensors(lat, theta) if T is None else T
    S = np.asarray(S)
    env, _ = tn.environments(T, S, lat, chi)
    l0, p0, st = psi_cut(T, S, lat, chi, i)
    st |= env.status
    d = lat.d
    e = 0.0 + 0.0j
    for (a_, b_, v) in H["pairs"]:
        e += v * int(S[a_]) * int(S[b_])
    for s in range(lat.nsites):
        e += H["onsite"][s][int(S[s])]
    for sites, h in H["terms"]:
        k = len(sites)
        a = 0
        for s in sites:
            a = a * d + int(S[s])
        for b in range(d ** k):
            hab = h[a, b]
            if hab == 0:
                continue
            if b == a:
                e += hab
                continue
            S2 = S.copy()
            for t, s in enumerate(sites):
                S2[s] = (b // d ** (k - 1 - t)) % d
            l1, p1, s1 = psi_cut(T, S2, lat, chi, i)
            st |= s1
            if np.isfinite(l1):
                e += hab * math.exp(l1 - l0) * complex(math.cos(p1 - p0), math.sin(p1 - p0))
    return e, l0, p0, st


def evaluate_bound(theta, S_batch, lat: Lattice, chi, H, i: int):
    """E_loc^bound, ln|psi_i|, phase and status for a batch of configurations."""
    T = theta_to_tensors(lat, theta)
    ns = len(S_batch)
    el = np.zeros(ns, dtype=np.complex128)
    la = np.zeros(ns)
    ph = np.zeros(ns)
    st = np.zeros(ns, dtype=np.int32)
    for n, S in enumerate(S_batch):
        el[n], la[n], ph[n], st[n] = local_energy_bound(theta, S, lat, chi, H, i, T=T)
    return dict(eloc=el, logabs=la, phase=ph, status=st)

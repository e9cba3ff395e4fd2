"""Local energy and log-derivatives from the boundary-MPS sandwiches (oracle, FP64).

Paper: Eq. (local_estimator) and Eq. (local_obs) (E_loc(S) = sum_S' <S|H|S'> psi(S')/psi(S),
restricted to S' that differ from S inside a term's support, environments outside the support
reused); Sec. "On reusing environments": diagonal terms need no amplitude; Sec. "On Numerical
Stability": ratios as exp(ln psi(S') - ln psi(S)); Sec. "Reformulation ...": O_{S,k} =
(d psi(S)/d theta_k) / psi(S), computed from the same environments (Sec. "On the boundary MPS
method", last paragraph).

Readings:
  * Matrix element order: <S|h|S'> (the paper's O_{S'S} read as an index-order slip; only this
    order reproduces <psi|H|psi> for a complex Hermitian H).
  * A term whose support lies in one row x uses psi_x for both S and S'; a term whose support
    spans rows x, x+1 uses psi_{x,x+1}; O for a site in row x uses psi_x.
"""
from __future__ import annotations

import math

import numpy as np

from paper_2503_12557_gb300.inputs import Lattice, theta_to_tensors, site_offsets
from . import tn


def _ratio(l1, p1, l0, p0):
    """psi'/psi from (ln|psi'|, phase') and (ln|psi|, phase)."""
    if not np.isfinite(l1):
        return 0.0
    return math.exp(l1 - l0) * complex(math.cos(p1 - p0), math.sin(p1 - p0))


def local_energy(theta, S, lat: Lattice, chi: int, H, env_ap=None):
    """E_loc(S) (complex) and the environment status bits."""
    T = theta_to_tensors(lat, theta)
    env, Ap = env_ap if env_ap is not None else tn.environments(T, S, lat, chi)
    Ly, d = lat.Ly, lat.d
    S = np.asarray(S)
    e = 0.0 + 0.0j
    for (i, j, v) in H["pairs"]:
        e += v * int(S[i]) * int(S[j])
    for i in range(lat.nsites):
        e += H["onsite"][i][int(S[i])]
    cache = {}
    for sites, h in H["terms"]:
        k = len(sites)
        rows = sorted({s // Ly for s in sites})
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
            Ap2 = tn.project(T, S2, lat)
            if len(rows) == 1:
                x = rows[0]
                if ("r", x) not in cache:
                    cache[("r", x)] = tn.log_psi_row(env, Ap, x)
                l0, p0 = cache[("r", x)]
                l1, p1 = tn.log_psi_row(env, Ap2, x)
            elif len(rows) == 2 and rows[1] == rows[0] + 1:
                x = rows[0]
                if ("p", x) not in cache:
                    cache[("p", x)] = tn.log_psi_pair(env, Ap, x)
                l0, p0 = cache[("p", x)]
                l1, p1 = tn.log_psi_pair(env, Ap2, x)
            else:
                raise ValueError("term support must lie in one row or two adjacent rows")
            e += hab * _ratio(l1, p1, l0, p0)
    return e, env.status


def log_derivative(theta, S, lat: Lattice, chi: int, env_ap=None):
    """O_{S,k} for all k (length N_p): delta_{s, s_xy} Env_xy[l,u,r,d] / psi_x(S)."""
    T = theta_to_tensors(lat, theta)
    env, Ap = env_ap if env_ap is not None else tn.environments(T, S, lat, chi)
    Lx, Ly = lat.Lx, lat.Ly
    offs = site_offsets(lat)
    dt = np.result_type(theta.dtype, np.float64)
    O = np.zeros(offs[-1], dtype=dt)
    for x in range(Lx):
        eu, el, A = env.Eu[x - 1], env.El[x + 1], Ap[x]
        L = [np.ones((1, 1, 1), dtype=dt)]
        lL = [0.0]
        for y in range(Ly):
            nL = tn.absorb1(L[y], eu[y], A[y], el[y])
            m = float(np.max(np.abs(nL)))
            L.append(nL / m)
            lL.append(lL[y] + math.log(m))
        R = [None] * (Ly + 1)
        lR = [0.0] * (Ly + 1)
        R[Ly] = np.ones((1, 1, 1), dtype=dt)
        for y in range(Ly - 1, -1, -1):
            nR = tn.absorb1_right(R[y + 1], eu[y], A[y], el[y])
            m = float(np.max(np.abs(nR)))
            R[y] = nR / m
            lR[y] = lR[y + 1] + math.log(m)
        val = L[Ly][0, 0, 0]
        for y in range(Ly):
            # Env[l,u,r,d] = sum L[a,l,b] eu[a,u,x] el[b,d,z] R[x,r,z]
            t = np.einsum("alb,aux->lbux", L[y], eu[y])
            t = np.einsum("lbux,xrz->lburz", t, R[y + 1])
            envt = np.einsum("lburz,bdz->lurd", t, el[y])
            o = envt / val * math.exp(lL[y] + lR[y + 1] - lL[Ly])
            i = x * Ly + y
            s = int(S[i])
            blk = O[offs[i]:offs[i + 1]].reshape(T[x][y].shape)
            blk[s] = o
    return O


def evaluate(theta, S_batch, lat: Lattice, chi: int, H=None, want_O=True):
    """ln|psi_top|, phase, E_loc, O, status and the smallest cutoff-decision margin
    (tn.cut_margin; inf at fixed chi) for a batch of configurations."""
    T = theta_to_tensors(lat, theta)
    ns = len(S_batch)
    margin = np.full(ns, math.inf)
    la = np.zeros(ns)
    ph = np.zeros(ns)
    el = np.zeros(ns, dtype=np.complex128)
    st = np.zeros(ns, dtype=np.int32)
    O = None
    if want_O:
        O = np.zeros((ns, len(theta)), dtype=np.result_type(theta.dtype, np.float64))
    for i, S in enumerate(S_batch):
        env_ap = tn.environments(T, S, lat, chi)
        env, Ap = env_ap
        la[i], ph[i] = tn.log_psi_row(env, Ap, lat.Lx - 1)
        st[i] = env.status
        margin[i] = env.cut_margin
        if H is not None:
            el[i], _ = local_energy(theta, S, lat, chi, H, env_ap=env_ap)
        if want_O:
            O[i] = log_derivative(theta, S, lat, chi, env_ap=env_ap)
    return dict(logabs=la, phase=ph, eloc=el, O=O, status=st, cut_margin=margin)

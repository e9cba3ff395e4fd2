"""Direct (row-by-row conditional) sampling of a finite PEPS (oracle, FP64; test infrastructure only).

Paper: Sec. "On Direct Sampling" and the appendix "Direct sampling of PEPS" (Eq.
(prob_from_cond_prob), Eq. (rho), Alg. `sampling`).  A configuration is drawn with probability

    p(S) = p(S_1) prod_i p(S_{i+1} | S_<i+1),

row by row from the top.  The conditional distribution of row i comes from the reduced
density matrix of row i with the rows above fixed to the drawn configuration and the rows
below traced out:

    rho_{S<i}[i] = T^u_{S<i}[i] . D^l[i+1] . (T^u_{S<i}[i])^*,

  * D^l[i+1]: the double-layer boundary MPS of rows i+1 .. Lx with the physical legs traced
    (site tensors D[c][(d, d')][e], (d, d') the up legs of row i+1 in the ket and the bra),
    built from the bottom by the exact double-layer MPO product and an SVD compression to
    chi_d, each site divided by its largest modulus;
  * T^u_{S<i}[i] = E^u[i-1](S) . T[i]: the single-layer upper environment of the drawn rows
    applied to row i with its physical legs open (kept exact: the bond D_s of the paper is
    read as chi D, no second truncation);
  * inside the row, the sites are drawn left to right from the one-dimensional structure
    (MPS sampling): p(s_y | s_<y) is proportional to the contraction of the left partial
    with site y fixed to s_y, the right partial with sites > y traced (s = s'), and D^l.

After a row is drawn, E^u[i] = truncate_chi(E^u[i-1] . T_proj[i]) exactly as tn.environments.
Readings: a conditional weight below zero (possible once D^l is truncated) counts as zero; the
draw for site (x, y) of chain c in draw round t takes u = uniform53(Philox4x32-10(counter =
(x Ly + y, t, c, 2), key = seed)) and picks the smallest s whose cumulative normalised
probability exceeds u; log p(S) sums the logs of the drawn conditionals.
"""
from __future__ import annotations

import math

import numpy as np

from paper_2503_12557_gb300.inputs import Lattice, theta_to_tensors
from . import tn
from .philox import key_of_seed, uniform53


def double_layer_row(Trow):
    """Double-layer MPO of one row: M[y][(l,l'), (u,u'), (r,r'), (d,d')] =
    sum_s T[s, l, u, r, d] conj(T[s, l', u', r', d'])."""
    out = []
    for T in Trow:
        _, l, u, r, d = T.shape
        M = np.einsum("slurd,sLURE->lLuUrRdE", T, np.conj(T))
        out.append(M.reshape(l * l, u * u, r * r, d * d))
    return out


def lower_double_envs(T, lat: Lattice, chi_d):
    """D^l[x] for x = 1 .. Lx (0-based: rows x .. Lx-1 traced; D^l[Lx] trivial) as lists of
    site tensors [c][(u, u')][e]; each row compressed to chi_d and normalised."""
    Dl = {lat.Lx: [np.ones((1, 1, 1), dtype=np.result_type(T[0][0].dtype, np.float64)) for _ in range(lat.Ly)]}
    for x in range(lat.Lx - 1, 0, -1):
        M = double_layer_row(T[x])
        # exact double-layer product: site [(c, L)][U][(f, R)] = sum_p D^l[c][p][f] M[L][U][R][p]
        prod = []
        for e, m in zip(Dl[x + 1], M):
            c, _, f = e.shape
            L, U, R, _ = m.shape
            prod.append(np.einsum("cpf,LURp->cLUfR", e, m).reshape(c * L, U, f * R))
        tr, _, _ = tn.truncate_svd(prod, chi_d)
        Dl[x], _, _ = tn.normalize(tr)
    return Dl


def _row_walk(Trow, eu, dl, Srow=None, key=None, ctr=None):
    """Draw (or, with Srow given, evaluate) one row.  Trow: site tensors (d, Dl, Du, Dr, Dd);
    eu: E^u of the rows above ([a][u][b]); dl: D^l of the rows below ([c][(d,d')][e]).
    key: Philox key; ctr(y): the counter of site y's uniform.
    Returns (row states, sum of log conditionals, zero-weight flag)."""
    Ly = len(Trow)
    # ket sites of T^u: K[(a,l), s, dd, (b,r)]
    K = []
    for e, A in zip(eu, Trow):
        a, _, b = e.shape
        s, l, _, r, dd = A.shape
        K.append(np.einsum("aub,slurd->alsdbr", e, A).reshape(a * l, s, dd, b * r))
    Dg = []
    for e, k in zip(dl, K):
        c, _, f = e.shape
        dd = k.shape[2]
        Dg.append(e.reshape(c, dd, dd, f))
    # right partials with the physical legs traced: R[y][B, e, B']
    R = [None] * (Ly + 1)
    R[Ly] = np.ones((1, 1, 1), dtype=np.result_type(K[0], Dg[0]))
    for y in range(Ly - 1, -1, -1):
        t = np.einsum("AsdB,Beb->Asdeb", K[y], R[y + 1])          # pairwise stages: a
        t = np.einsum("Asdeb,cdDe->AscDb", t, Dg[y])               # contraction order chosen
        t = np.einsum("AscDb,asDb->Aca", t, np.conj(K[y]))         # for small intermediates
        m = float(np.max(np.abs(t)))
        R[y] = t / m if m > 0 else t
    L = np.ones((1, 1, 1), dtype=R[Ly].dtype)
    states, logp, zero = [], 0.0, False
    for y in range(Ly):
        t = np.einsum("Aca,AsdB->casdB", L, K[y])
        t = np.einsum("casdB,cdDe->asDeB", t, Dg[y])
        cand = np.einsum("asDeB,asDb->sBeb", t, np.conj(K[y]))
        w = np.array([max(0.0, float(np.real(np.sum(cand[s] * R[y + 1])))) for s in range(cand.shape[0])])
        tot = float(np.sum(w))
        if not tot > 0.0:
            zero = True
            w = np.ones_like(w)
            tot = float(np.sum(w))
        p = w / tot
        if Srow is not None:
            s = int(Srow[y])
        else:
            u = uniform53(ctr(y), key)
            s = int(np.searchsorted(np.cumsum(p), u, side="right"))
            s = min(s, len(p) - 1)
        logp += math.log(p[s]) if p[s] > 0 else -math.inf
        states.append(s)
        Ln = cand[s]
        m = float(np.max(np.abs(Ln)))
        L = Ln / m if m > 0 else Ln
    return states, logp, zero


def walk(theta, lat: Lattice, chi, chi_d, S=None, seed=0, chain=0, draw=0, Dl=None):
    """Draw one configuration (S None) or evaluate log p(S) of a given one.
    Returns (S, log p(S), status bits)."""
    T = theta_to_tensors(lat, theta)
    Dl = lower_double_envs(T, lat, chi_d) if Dl is None else Dl
    key = key_of_seed(seed)
    Ly = lat.Ly
    out = np.zeros(lat.nsites, dtype=np.uint8)
    dt = np.result_type(T[0][0].dtype, np.float64)
    eu = [np.ones((1, 1, 1), dtype=dt) for _ in range(Ly)]
    logp, st = 0.0, 0
    for x in range(lat.Lx):
        Srow = None if S is None else np.asarray(S)[x * Ly:(x + 1) * Ly]
        row, lp, zero = _row_walk(T[x], eu, Dl[x + 1], Srow, key, lambda y: (x * Ly + y, draw, chain, 2))
        if zero:
            st |= tn.ZERO_NORM
        logp += lp
        out[x * Ly:(x + 1) * Ly] = row
        if x < lat.Lx - 1:
            Ap = [T[x][y][row[y]] for y in range(Ly)]
            if x == 0:
                e, _, s0 = tn.normalize(tn.top_row_mps(Ap))
            else:
                tr, s1, _ = tn.truncate_svd(tn.apply_down(eu, Ap), chi)
                e, _, s0 = tn.normalize(tr)
                s0 |= s1
            st |= s0
            eu = e
    return out, logp, st


def sample(theta, lat: Lattice, chi, chi_d, n, seed, draw=0):
    """n configurations (chains 0 .. n-1 of draw round `draw`) with their log p and status."""
    T = theta_to_tensors(lat, theta)
    Dl = lower_double_envs(T, lat, chi_d)
    S = np.zeros((n, lat.nsites), dtype=np.uint8)
    lp = np.zeros(n)
    st = np.zeros(n, dtype=np.int32)
    for c in range(n):
        S[c], lp[c], st[c] = walk(theta, lat, chi, chi_d, seed=seed, chain=c, draw=draw, Dl=Dl)
    return S, lp, st

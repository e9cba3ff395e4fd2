"""Boundary-MPS contraction of a PEPS projected on one configuration (oracle, FP64).

Paper: Sec. "On the boundary MPS method" (boundary environments E^u[i], E^l[j], truncation of
the MPS-MPO product from bond D_c D back to D_c, Eq. (boundary_MPS_approx)); Sec. "On Numerical
Stability" (every environment tensor divided by its largest entry, logarithms accumulated);
Eq. (PsiS) for the amplitude.

Index conventions (shared with the inputs module):
  projected site tensor  A[l, u, r, d] = T[x, y][s_xy, l, u, r, d]
  upper environment site e[a, d, b]   (left bond, open down leg of the rows above, right bond)
  lower environment site e[a, u, b]   (left bond, open up leg of the rows below, right bond)
  Eu[x] approximates rows 0..x, El[x] approximates rows x..Lx-1; Eu[-1] and El[Lx] are the
  trivial one-site-per-column environments with all bonds of dimension 1.

Readings of the paper used here (the paper prints no truncation steps):
  * Truncation = sequential SVD compression: left-canonicalise the exact product with QR, then
    sweep right to left, keeping at every bond the min(chi, rank-bound) largest singular values.
    The density-matrix algorithm the paper names gives the same truncated state when it sweeps
    in the same direction (truncate_dm below implements that form independently).
  * Normalisation: after every row step each site tensor is divided by its largest modulus.
  * psi_top := Eu[Lx-2] . T_proj[Lx-1]; psi_x := Eu[x-1] . T_proj[x] . El[x+1] (one-row
    sandwich); psi_{x,x+1} := Eu[x-1] . T_proj[x] . T_proj[x+1] . El[x+2] (two-row sandwich).
"""
from __future__ import annotations

import math

import numpy as np

from paper_2503_12557_gb300.inputs import Lattice, theta_to_tensors

NEAR_DEGENERATE = 1 << 0
ZERO_NORM = 1 << 1
NONFINITE = 1 << 2


class Env:
    """Normalised boundary-MPS rows with their accumulated log scales and status bits."""

    def __init__(self, Lx):
        self.Eu = {}
        self.El = {}
        self.logu = {}
        self.logl = {}
        self.status = 0
        self.max_discarded = 0.0
        self.cut_margin = math.inf


def project(T, S, lat: Lattice):
    """T_proj[x][y] = T[x][y][s_xy] (Alg. `sampling`, proj)."""
    return [[T[x][y][int(S[x * lat.Ly + y])] for y in range(lat.Ly)] for x in range(lat.Lx)]


def trivial_row(Ly, dtype):
    return [np.ones((1, 1, 1), dtype=dtype) for _ in range(Ly)]


def top_row_mps(Arow):
    """Row 0 read as an MPS: e[a=l, d, b=r] (its up legs have dimension 1)."""
    return [np.transpose(A[:, 0, :, :], (0, 2, 1)).copy() for A in Arow]


def bottom_row_mps(Arow):
    """Row Lx-1 read as an MPS: e[a=l, u, b=r] (its down legs have dimension 1)."""
    return [A[:, :, :, 0].copy() for A in Arow]


def apply_down(mps, Arow):
    """Exact MPS-MPO product for the upper environment: new[(a,l), d, (b,r)] = sum_u e[a,u,b] A[l,u,r,d]."""
    out = []
    for e, A in zip(mps, Arow):
        a, _, b = e.shape
        l, _, r, d = A.shape
        out.append(np.einsum("aub,lurd->aldbr", e, A).reshape(a * l, d, b * r))
    return out


def apply_up(mps, Arow):
    """Exact MPS-MPO product for the lower environment: new[(a,l), u, (b,r)] = sum_d A[l,u,r,d] e[a,d,b]."""
    out = []
    for e, A in zip(mps, Arow):
        a, _, b = e.shape
        l, u, r, _ = A.shape
        out.append(np.einsum("adb,lurd->alubr", e, A).reshape(a * l, u, b * r))
    return out


def normalize(mps):
    """Divide every site tensor by its largest modulus; return (tensors, sum of logs, status)."""
    out, logsum, st = [], 0.0, 0
    for e in mps:
        f = float(np.max(np.abs(e))) if e.size else 0.0
        if not np.isfinite(f):
            st |= NONFINITE
            out.append(e)
            continue
        if f == 0.0:
            st |= ZERO_NORM
            out.append(e)
            logsum = -math.inf
            continue
        out.append(e / f)
        logsum += math.log(f)
    return out, logsum, st


def _cut_flags(s, keep):
    """Near-degenerate cut: kept and discarded singular values closer than 1e-8 sigma_1 while the
    first discarded one is not negligible (1e-12 sigma_1)."""
    if keep >= len(s) or s[0] == 0.0:
        return 0
    if (s[keep - 1] - s[keep]) < 1e-8 * s[0] and s[keep] > 1e-12 * s[0]:
        return NEAR_DEGENERATE
    return 0


def chi_cut(chi):
    """chi as an int (fixed bond dimension) or a pair (chi_max, cutoff) for the truncated-weight
    rule of Sec. "On the boundary MPS method" (the paper truncates at a discarded weight 1e-4)."""
    if np.isscalar(chi):
        return int(chi), 0.0
    return int(chi[0]), float(chi[1])


def keep_count(s, chi, cut):
    """Number of singular values kept at one bond (s sorted descending): min(chi, len(s)), and
    with cut > 0 at most the smallest k >= 1 whose relative discarded weight
    sum_{i >= k} s_i^2 / sum_i s_i^2 is at most cut.  Also returns NEAR_DEGENERATE when that
    weight comparison is within 1e-9 (relative) of the cutoff at the chosen boundary, where the
    decision is not stable under rounding."""
    keep = min(chi, len(s))
    if cut <= 0.0:
        return keep, 0
    w = np.asarray(s, dtype=float) ** 2
    tot = float(np.sum(w))
    if tot <= 0.0:
        return keep, 0
    tail = np.concatenate([np.cumsum(w[::-1])[::-1], [0.0]]) / tot  # tail[k] = sum_{i>=k} w_i / tot
    kcut = next(k for k in range(1, len(s) + 1) if tail[k] <= cut)
    flag = 0
    for k in (kcut - 1, kcut):
        if 1 <= k <= len(s) and abs(tail[k] - cut) <= 1e-9 * cut:
            flag = NEAR_DEGENERATE
    if kcut >= keep:
        return keep, 0
    return kcut, flag


def cut_margin(s, chi, cut):
    """How far the cutoff decision of keep_count is from changing: the smallest relative
    distance |tail[k] - cut| / cut over the comparisons k = 1 .. min(chi, kcut) (a superset of
    those that decide the kept count; inf without a cutoff).  A computation whose tails carry a
    relative rounding error below this margin keeps the same number of singular values."""
    if cut <= 0.0:
        return math.inf
    w = np.asarray(s, dtype=float) ** 2
    tot = float(np.sum(w))
    if tot <= 0.0:
        return math.inf
    tail = np.concatenate([np.cumsum(w[::-1])[::-1], [0.0]]) / tot
    kcut = next(k for k in range(1, len(s) + 1) if tail[k] <= cut)
    last = min(chi, kcut, len(s))
    return float(min(abs(tail[k] - cut) for k in range(1, last + 1)) / cut)


def truncate_svd(mps, chi, stats=None):
    """Sequential SVD compression to bond dimension chi (QR left-canonicalisation, then
    right-to-left SVDs); chi may be (chi_max, cutoff), see keep_count.  Returns (mps, status,
    max discarded weight); a dict passed as stats receives the smallest cut_margin."""
    chi, cut = chi_cut(chi)
    A = [e.copy() for e in mps]
    n = len(A)
    for k in range(n - 1):
        a, p, b = A[k].shape
        Q, R = np.linalg.qr(A[k].reshape(a * p, b))
        A[k] = Q.reshape(a, p, Q.shape[1])
        A[k + 1] = np.einsum("ij,jpk->ipk", R, A[k + 1])
    st, wmax = 0, 0.0
    for k in range(n - 1, 0, -1):
        a, p, b = A[k].shape
        U, s, Vh = np.linalg.svd(A[k].reshape(a, p * b), full_matrices=False)
        keep, fl = keep_count(s, chi, cut)
        st |= _cut_flags(s, keep) | fl
        if stats is not None:
            stats["cut_margin"] = min(stats.get("cut_margin", math.inf), cut_margin(s, chi, cut))
        tot = float(np.sum(s ** 2))
        if tot > 0.0:
            wmax = max(wmax, float(np.sum(s[keep:] ** 2)) / tot)
        A[k] = Vh[:keep].reshape(keep, p, b)
        A[k - 1] = np.einsum("ipj,jk->ipk", A[k - 1], U[:, :keep] * s[:keep])
    return A, st, wmax


def truncate_dm(mps, chi):
    """The same truncation in density-matrix form: exact left Gram environments G, then from
    the right: Y = M C, rho = Y^dag G Y, keep the top-chi eigenvectors.  Independent cross-check
    of truncate_svd (the two agree whenever the kept subspace is separated by a gap)."""
    chi, cut = chi_cut(chi)
    n = len(mps)
    G = [np.ones((1, 1), dtype=mps[0].dtype)]
    for k in range(n - 1):
        G.append(np.einsum("ij,ipa,jpb->ab", G[k], np.conj(mps[k]), mps[k], optimize=True))
    C = np.ones((1, 1), dtype=mps[0].dtype)
    out = [None] * n
    for k in range(n - 1, 0, -1):
        Y = np.einsum("apb,bc->apc", mps[k], C)
        a, p, c = Y.shape
        rho = np.einsum("ij,ipc,jqd->pcqd", G[k], np.conj(Y), Y, optimize=True).reshape(p * c, p * c)
        w, V = np.linalg.eigh(rho)
        order = np.argsort(-w, kind="stable")
        keep = min(chi, p * c, a)
        if cut > 0.0:
            ev = np.sqrt(np.clip(w[order], 0.0, None))
            keep = min(keep, keep_count(ev, p * c, cut)[0])
        Vk = V[:, order[:keep]]
        out[k] = np.conj(Vk.T).reshape(keep, p, c)
        C = Y.reshape(a, p * c) @ Vk
    out[0] = np.einsum("apb,bc->apc", mps[0], C)
    return out


def environments(T, S, lat: Lattice, chi: int, sides=("u", "l"), trunc=truncate_svd):
    """All normalised upper (Eu[-1..Lx-2]) and lower (El[1..Lx]) environments of configuration S."""
    Ap = project(T, S, lat)
    dt = np.result_type(*[A.dtype for A in Ap[0]])
    env = Env(lat.Lx)
    env.Eu[-1], env.logu[-1] = trivial_row(lat.Ly, dt), 0.0
    env.El[lat.Lx], env.logl[lat.Lx] = trivial_row(lat.Ly, dt), 0.0
    if "u" in sides:
        e, lg, st = normalize(top_row_mps(Ap[0]))
        env.status |= st
        env.Eu[0], env.logu[0] = e, lg
        for x in range(1, lat.Lx - 1):
            prod = apply_down(env.Eu[x - 1], Ap[x])
            if trunc is truncate_svd:
                stats = {}
                tr, st, w = trunc(prod, chi, stats)
                env.status |= st
                env.max_discarded = max(env.max_discarded, w)
                env.cut_margin = min(env.cut_margin, stats.get("cut_margin", math.inf))
            else:
                tr = trunc(prod, chi)
            e, lg, st = normalize(tr)
            env.status |= st
            env.Eu[x], env.logu[x] = e, env.logu[x - 1] + lg
    if "l" in sides:
        e, lg, st = normalize(bottom_row_mps(Ap[lat.Lx - 1]))
        env.status |= st
        env.El[lat.Lx - 1], env.logl[lat.Lx - 1] = e, lg
        for x in range(lat.Lx - 2, 0, -1):
            prod = apply_up(env.El[x + 1], Ap[x])
            if trunc is truncate_svd:
                stats = {}
                tr, st, w = trunc(prod, chi, stats)
                env.status |= st
                env.max_discarded = max(env.max_discarded, w)
                env.cut_margin = min(env.cut_margin, stats.get("cut_margin", math.inf))
            else:
                tr = trunc(prod, chi)
            e, lg, st = normalize(tr)
            env.status |= st
            env.El[x], env.logl[x] = e, env.logl[x + 1] + lg
    return env, Ap


def _log_of(val, logscale):
    """(ln|psi|, phase) of psi = val * exp(logscale)."""
    if val == 0:
        return -math.inf, 0.0
    return math.log(abs(val)) + logscale, float(np.angle(val))


def absorb1(L, eu, A, el):
    """Left partial of a one-row sandwich moved over one column:
    L'[x, r, z] = sum L[a, l, b] eu[a, u, x] A[l, u, r, d] el[b, d, z]."""
    t = np.einsum("alb,aux->lbux", L, eu)
    t = np.einsum("lbux,lurd->bxrd", t, A)
    return np.einsum("bxrd,bdz->xrz", t, el)


def absorb1_right(R, eu, A, el):
    """Right partial of a one-row sandwich moved over one column:
    R'[a, l, b] = sum eu[a, u, x] A[l, u, r, d] el[b, d, z] R[x, r, z]."""
    t = np.einsum("aux,xrz->aurz", eu, R)
    t = np.einsum("aurz,lurd->alzd", t, A)
    return np.einsum("alzd,bdz->alb", t, el)


def sandwich1(eu, Arow, el):
    """One-row sandwich eu . Arow . el contracted column by column from the left, each partial
    divided by its largest modulus.  Returns (value of the normalised scalar, log scale)."""
    L = np.ones((1, 1, 1), dtype=np.result_type(eu[0], Arow[0], el[0]))
    logs = 0.0
    for y in range(len(Arow)):
        L = absorb1(L, eu[y], Arow[y], el[y])
        m = float(np.max(np.abs(L)))
        if m == 0.0 or not np.isfinite(m):
            return 0.0, -math.inf
        L = L / m
        logs += math.log(m)
    return L[0, 0, 0], logs


def sandwich2(eu, A1, A2, el):
    """Two-row sandwich eu . A1 . A2 . el (rows x and x+1), same bookkeeping as sandwich1."""
    L = np.ones((1, 1, 1, 1), dtype=np.result_type(eu[0], A1[0], A2[0], el[0]))
    logs = 0.0
    for y in range(len(A1)):
        t = np.einsum("aijb,aux->ijbux", L, eu[y])
        t = np.einsum("ijbux,iurv->jbxrv", t, A1[y])
        t = np.einsum("jbxrv,jvsd->bxrsd", t, A2[y])
        L = np.einsum("bxrsd,bdz->xrsz", t, el[y])
        m = float(np.max(np.abs(L)))
        if m == 0.0 or not np.isfinite(m):
            return 0.0, -math.inf
        L = L / m
        logs += math.log(m)
    return L[0, 0, 0, 0], logs


def log_psi_row(env, Ap, x):
    """(ln|psi_x|, phase) of the one-row sandwich at row x."""
    v, lg = sandwich1(env.Eu[x - 1], Ap[x], env.El[x + 1])
    return _log_of(v, lg + env.logu[x - 1] + env.logl[x + 1])


def log_psi_pair(env, Ap, x):
    """(ln|psi_{x,x+1}|, phase) of the two-row sandwich at rows x, x+1."""
    v, lg = sandwich2(env.Eu[x - 1], Ap[x], Ap[x + 1], env.El[x + 2])
    return _log_of(v, lg + env.logu[x - 1] + env.logl[x + 2])


def log_amplitude(theta, S, lat: Lattice, chi: int, trunc=truncate_svd):
    """(ln|psi_top(S)|, phase, status) with psi_top = Eu[Lx-2] . T_proj[Lx-1]."""
    T = theta_to_tensors(lat, theta)
    env, Ap = environments(T, S, lat, chi, sides=("u",), trunc=trunc)
    la, ph = log_psi_row(env, Ap, lat.Lx - 1)
    st = env.status | (NONFINITE if not np.isfinite(la) else 0)
    return la, ph, st


def mps_to_vector(mps):
    """Dense vector of an open MPS (first site's left bond and last site's right bond of dim 1)."""
    v = mps[0]
    for e in mps[1:]:
        v = np.einsum("...a,apb->...pb", v, e)
    return v.reshape(-1)

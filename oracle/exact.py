"""Exact references for tiny lattices (oracle side): no truncation anywhere.

* amplitude_rowtransfer: psi(S) of Eq. (PsiS) by a dense row-transfer contraction (a vector over
  all down legs of the rows done so far); exact for any chi because nothing is truncated.
* amplitude_fullnet: psi(S) of Eq. (PsiS) by one einsum over the whole network (a different
  contraction route, for lattices with a handful of sites).
* state_vector: all d^N amplitudes with the physical legs left open, basis index
  sum_i s_i d^(N-1-i).
* hamiltonian_sparse: <S|H|S'> of a term list as a sparse matrix, so that (H psi)(S) gives the
  exact local energy E_loc(S) = (H psi)(S) / psi(S) of Eq. (local_obs).
"""
from __future__ import annotations

import string

import numpy as np
import scipy.sparse as sp

from paper_2503_12557_gb300.inputs import Lattice, theta_to_tensors


def _letters():
    return string.ascii_letters


def amplitude_rowtransfer(theta, S, lat: Lattice):
    T = theta_to_tensors(lat, theta)
    Ly = lat.Ly
    L = _letters()
    v = np.ones([1] * Ly, dtype=theta.dtype)
    for x in range(lat.Lx):
        u = L[0:Ly]
        h = L[Ly:2 * Ly + 1]
        d = L[2 * Ly + 1:3 * Ly + 1]
        ops = [u]
        args = [v]
        for y in range(Ly):
            ops.append(h[y] + u[y] + h[y + 1] + d[y])
            args.append(T[x][y][int(S[x * Ly + y])])
        v = np.einsum(",".join(ops) + "->" + d, *args, optimize="greedy")
    return v.reshape(-1)[0]


def amplitude_fullnet(theta, S, lat: Lattice):
    """One einsum over all Lx*Ly tensors (bond letters assigned per edge)."""
    T = theta_to_tensors(lat, theta)
    Lx, Ly = lat.Lx, lat.Ly
    letters = iter(_letters())
    hb = {}
    vb = {}
    for x in range(Lx):
        for y in range(Ly + 1):
            hb[(x, y)] = next(letters)
    for x in range(Lx + 1):
        for y in range(Ly):
            vb[(x, y)] = next(letters)
    ops, args = [], []
    for x in range(Lx):
        for y in range(Ly):
            ops.append(hb[(x, y)] + vb[(x, y)] + hb[(x, y + 1)] + vb[(x + 1, y)])
            args.append(T[x][y][int(S[x * Ly + y])])
    return np.einsum(",".join(ops) + "->", *args, optimize="greedy")


def state_vector(theta, lat: Lattice):
    """psi(S) for all S; index of S is sum_i s_i d^(N-1-i)."""
    T = theta_to_tensors(lat, theta)
    Ly, d = lat.Ly, lat.d
    L = _letters()
    v = np.ones([1] + [1] * Ly, dtype=theta.dtype)  # (P, down legs...)
    for x in range(lat.Lx):
        P = "Z"
        u = L[0:Ly]
        h = L[Ly:2 * Ly + 1]
        dd = L[2 * Ly + 1:3 * Ly + 1]
        s = L[3 * Ly + 1:4 * Ly + 1]
        ops = [P + u]
        args = [v]
        for y in range(Ly):
            ops.append(s[y] + h[y] + u[y] + h[y + 1] + dd[y])
            args.append(T[x][y])
        v = np.einsum(",".join(ops) + "->" + P + s + dd, *args, optimize="greedy")
        shp = v.shape
        v = v.reshape((shp[0] * d ** Ly,) + shp[1 + Ly:])
    return v.reshape(-1)


def config_index(S, d):
    idx = 0
    for s in S:
        idx = idx * d + int(s)
    return idx


def index_configs(N, d):
    """All configurations in basis order, shape (d^N, N)."""
    idx = np.arange(d ** N)
    out = np.zeros((d ** N, N), dtype=np.int64)
    for i in range(N - 1, -1, -1):
        out[:, i] = idx % d
        idx //= d
    return out


def hamiltonian_sparse(H, lat: Lattice):
    N, d = lat.nsites, lat.d
    dim = d ** N
    Sall = index_configs(N, d)
    pw = d ** np.arange(N - 1, -1, -1)
    rows, cols, vals = [], [], []
    diag = np.zeros(dim, dtype=np.complex128)
    for (i, j, v) in H["pairs"]:
        diag += v * Sall[:, i] * Sall[:, j]
    for i in range(N):
        diag += H["onsite"][i][Sall[:, i]]
    for sites, h in H["terms"]:
        k = len(sites)
        a = np.zeros(dim, dtype=np.int64)
        for s in sites:
            a = a * d + Sall[:, s]
        base = np.arange(dim) - sum(Sall[:, s] * pw[s] for s in sites)
        for b in range(d ** k):
            digits = [(b // d ** (k - 1 - t)) % d for t in range(k)]
            col = base + sum(digits[t] * pw[sites[t]] for t in range(k))
            hv = h[a, b]
            nz = hv != 0
            rows.append(np.arange(dim)[nz])
            cols.append(col[nz])
            vals.append(hv[nz])
    rows.append(np.arange(dim))
    cols.append(np.arange(dim))
    vals.append(diag)
    Hm = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                       shape=(dim, dim)).tocsr()
    return Hm


def exact_local_energy(psi, Hm):
    """E_loc(S) = (H psi)(S) / psi(S) for every basis state."""
    return (Hm @ psi) / psi


def exact_energy(psi, Hm):
    return complex(np.vdot(psi, Hm @ psi) / np.vdot(psi, psi))

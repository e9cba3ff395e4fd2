"""Metropolis sweeps with environment reuse (oracle, FP64).

The paper samples directly from double-layer environments (Sec. "On Direct Sampling",
App. B); these Markov chains are the local-update alternative it contrasts that scheme with.
Environment reuse inside a sweep follows Sec. "On reusing environments": a move inside row x
only needs E^u[x-1], the rows it touches and E^l below them.

Readings (the paper prints no Markov-chain update scheme):
  Sweeps alternate direction: an even sweep id runs down the rows, an odd one up, so that every
  sweep starts from the environments the previous one left behind.
  One downward sweep (even sweep id) of one chain:
    El[x] for the current S (all rows, bottom up);  Eu[-1] trivial;  slot = 0
    for x = 0 .. Lx-1:
      row moves, y in order:  exchange: (x,y)<->(x,y+1) for y = 0..Ly-2;  flip: (x,y) for y = 0..Ly-1
          ratio = psi_x(S')/psi_x(S) with Eu[x-1] and El[x+1]
      vertical moves (exchange only, x < Lx-1): (x,y)<->(x+1,y) for y = 0..Ly-1
          ratio = psi_{x,x+1}(S')/psi_{x,x+1}(S) with Eu[x-1] and El[x+2]
      if x < Lx-1: Eu[x] = normalise(truncate(Eu[x-1] o T_proj[x]))  (with the updated S)
  One upward sweep (odd sweep id), the mirror image:
    Eu[x] for the current S (all rows, top down);  El[Lx] trivial;  slot = 0
    for x = Lx-1 .. 0:
      row moves as above, ratio psi_x with Eu[x-1] and El[x+1]
      vertical moves (exchange only, x > 0): (x-1,y)<->(x,y) for y = 0..Ly-1,
          ratio psi_{x-1,x} with Eu[x-2] and El[x+1]
      if x > 0: El[x] = normalise(truncate(El[x+1] o T_proj[x]))  (with the updated S)
  Every move slot draws u = uniform53(counter=(slot, sweep, chain, 0), key=seed) and then
  slot += 1, whether or not a move is possible (an exchange of equal spins is skipped).
  Accept iff u < |psi'/psi|^2, evaluated as u < exp(2 (ln|psi'| - ln|psi|)).
"""
from __future__ import annotations

import math

import numpy as np

from paper_2503_12557_gb300.inputs import Lattice, theta_to_tensors
from . import tn
from .philox import uniform53, key_of_seed


def _accept(u, l1, l0):
    if not np.isfinite(l1):
        return False
    return u < math.exp(2.0 * (l1 - l0))


def sweep(theta, S, lat: Lattice, chi: int, move: str, seed: int, chain: int, sweep_id: int):
    """One sweep of one chain (downward for an even sweep id, upward for an odd one); returns
    (new S, accepted moves, attempted moves)."""
    if sweep_id % 2 == 1:
        return _sweep_up(theta, S, lat, chi, move, seed, chain, sweep_id)
    T = theta_to_tensors(lat, theta)
    S = np.array(S, dtype=np.uint8)
    Lx, Ly = lat.Lx, lat.Ly
    env, _ = tn.environments(T, S, lat, chi, sides=("l",))
    key = key_of_seed(seed)
    slot = 0
    acc = att = 0
    eu_prev, logu_prev = env.Eu[-1], 0.0
    for x in range(Lx):
        # horizontal / single-site moves inside row x
        moves = [(x * Ly + y, x * Ly + y + 1) for y in range(Ly - 1)] if move == "exchange" \
            else [(x * Ly + y,) for y in range(Ly)]
        for m in moves:
            u = uniform53((slot, sweep_id, chain, 0), key)
            slot += 1
            if move == "exchange" and S[m[0]] == S[m[1]]:
                continue
            S2 = S.copy()
            if move == "exchange":
                S2[m[0]], S2[m[1]] = S[m[1]], S[m[0]]
            else:
                S2[m[0]] = lat.d - 1 - S[m[0]]
            A0 = tn.project(T, S, lat)[x]
            A1 = tn.project(T, S2, lat)[x]
            v0, g0 = tn.sandwich1(eu_prev, A0, env.El[x + 1])
            v1, g1 = tn.sandwich1(eu_prev, A1, env.El[x + 1])
            l0 = math.log(abs(v0)) + g0 if v0 != 0 else -math.inf
            l1 = math.log(abs(v1)) + g1 if v1 != 0 else -math.inf
            att += 1
            if _accept(u, l1, l0):
                S = S2
                acc += 1
        if move == "exchange" and x < Lx - 1:
            for y in range(Ly):
                i, j = x * Ly + y, (x + 1) * Ly + y
                u = uniform53((slot, sweep_id, chain, 0), key)
                slot += 1
                if S[i] == S[j]:
                    continue
                S2 = S.copy()
                S2[i], S2[j] = S[j], S[i]
                P0 = tn.project(T, S, lat)
                P1 = tn.project(T, S2, lat)
                v0, g0 = tn.sandwich2(eu_prev, P0[x], P0[x + 1], env.El[x + 2])
                v1, g1 = tn.sandwich2(eu_prev, P1[x], P1[x + 1], env.El[x + 2])
                l0 = math.log(abs(v0)) + g0 if v0 != 0 else -math.inf
                l1 = math.log(abs(v1)) + g1 if v1 != 0 else -math.inf
                att += 1
                if _accept(u, l1, l0):
                    S = S2
                    acc += 1
        if x < Lx - 1:
            A = tn.project(T, S, lat)[x]
            if x == 0:
                prod = tn.top_row_mps(A)
            else:
                prod, _, _ = tn.truncate_svd(tn.apply_down(eu_prev, A), chi)
            eu_prev, lg, _ = tn.normalize(prod)
            logu_prev += lg
    return S, acc, att


def _sweep_up(theta, S, lat: Lattice, chi: int, move: str, seed: int, chain: int, sweep_id: int):
    """The upward sweep: rows Lx-1 .. 0 with the upper environments of the sweep's start and the
    lower ones built from the updated rows."""
    T = theta_to_tensors(lat, theta)
    S = np.array(S, dtype=np.uint8)
    Lx, Ly = lat.Lx, lat.Ly
    env, _ = tn.environments(T, S, lat, chi, sides=("u",))
    key = key_of_seed(seed)
    slot = 0
    acc = att = 0
    el_prev = env.El[Lx]
    for x in range(Lx - 1, -1, -1):
        moves = [(x * Ly + y, x * Ly + y + 1) for y in range(Ly - 1)] if move == "exchange" \
            else [(x * Ly + y,) for y in range(Ly)]
        for m in moves:
            u = uniform53((slot, sweep_id, chain, 0), key)
            slot += 1
            if move == "exchange" and S[m[0]] == S[m[1]]:
                continue
            S2 = S.copy()
            if move == "exchange":
                S2[m[0]], S2[m[1]] = S[m[1]], S[m[0]]
            else:
                S2[m[0]] = lat.d - 1 - S[m[0]]
            v0, g0 = tn.sandwich1(env.Eu[x - 1], tn.project(T, S, lat)[x], el_prev)
            v1, g1 = tn.sandwich1(env.Eu[x - 1], tn.project(T, S2, lat)[x], el_prev)
            l0 = math.log(abs(v0)) + g0 if v0 != 0 else -math.inf
            l1 = math.log(abs(v1)) + g1 if v1 != 0 else -math.inf
            att += 1
            if _accept(u, l1, l0):
                S = S2
                acc += 1
        if move == "exchange" and x > 0:
            for y in range(Ly):
                i, j = (x - 1) * Ly + y, x * Ly + y
                u = uniform53((slot, sweep_id, chain, 0), key)
                slot += 1
                if S[i] == S[j]:
                    continue
                S2 = S.copy()
                S2[i], S2[j] = S[j], S[i]
                P0 = tn.project(T, S, lat)
                P1 = tn.project(T, S2, lat)
                v0, g0 = tn.sandwich2(env.Eu[x - 2], P0[x - 1], P0[x], el_prev)
                v1, g1 = tn.sandwich2(env.Eu[x - 2], P1[x - 1], P1[x], el_prev)
                l0 = math.log(abs(v0)) + g0 if v0 != 0 else -math.inf
                l1 = math.log(abs(v1)) + g1 if v1 != 0 else -math.inf
                att += 1
                if _accept(u, l1, l0):
                    S = S2
                    acc += 1
        if x > 0:
            A = tn.project(T, S, lat)[x]
            if x == Lx - 1:
                prod = tn.bottom_row_mps(A)
            else:
                prod, _, _ = tn.truncate_svd(tn.apply_up(el_prev, A), chi)
            el_prev, _, _ = tn.normalize(prod)
    return S, acc, att


def run_chains(theta, S0, lat: Lattice, chi: int, move: str, seed: int, nsweeps: int, sweep0: int = 0):
    """nsweeps sweeps for every chain (row of S0); sweep ids sweep0 .. sweep0+nsweeps-1."""
    S = np.array(S0, dtype=np.uint8)
    acc = np.zeros(len(S), dtype=np.int64)
    att = np.zeros(len(S), dtype=np.int64)
    for c in range(len(S)):
        for k in range(nsweeps):
            S[c], a, t = sweep(theta, S[c], lat, chi, move, seed, c, sweep0 + k)
            acc[c] += a
            att[c] += t
    return S, acc, att


def transition_matrix_exact(psi, lat: Lattice, move: str, up: bool = False):
    """Full transition matrix of one sweep (downward, or upward with up=True) on a tiny lattice
    with exact amplitudes psi (basis index sum s_i d^(N-1-i)), built as the product of the
    single-move kernels in sweep order.  Returns (P_sweep, list of single-move kernels)."""
    N, d, Ly, Lx = lat.nsites, lat.d, lat.Ly, lat.Lx
    dim = d ** N
    p = np.abs(psi) ** 2
    from .exact import index_configs
    Sall = index_configs(N, d)
    pw = d ** np.arange(N - 1, -1, -1)
    kernels = []
    order = []
    for x in (range(Lx - 1, -1, -1) if up else range(Lx)):
        if move == "exchange":
            order += [(x * Ly + y, x * Ly + y + 1) for y in range(Ly - 1)]
            if up and x > 0:
                order += [((x - 1) * Ly + y, x * Ly + y) for y in range(Ly)]
            if not up and x < Lx - 1:
                order += [(x * Ly + y, (x + 1) * Ly + y) for y in range(Ly)]
        else:
            order += [(x * Ly + y,) for y in range(Ly)]
    for m in order:
        K = np.zeros((dim, dim))
        for a in range(dim):
            if len(m) == 2:
                i, j = m
                if Sall[a, i] == Sall[a, j]:
                    K[a, a] = 1.0
                    continue
                b = a + (Sall[a, j] - Sall[a, i]) * pw[i] + (Sall[a, i] - Sall[a, j]) * pw[j]
            else:
                i = m[0]
                b = a + ((d - 1 - Sall[a, i]) - Sall[a, i]) * pw[i]
            r = min(1.0, p[b] / p[a]) if p[a] > 0 else 1.0
            K[a, b] += r
            K[a, a] += 1.0 - r
        kernels.append(K)
    P = np.eye(dim)
    for K in kernels:
        P = P @ K
    return P, kernels

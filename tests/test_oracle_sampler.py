"""Pins of the oracle's Metropolis sweep.

* On 3x3 lattices the full transition matrix built from exact amplitudes, for the downward and
  the upward sweep: every single-move kernel satisfies detailed balance with respect to |psi|^2
  and the sweep leaves |psi|^2 stationary (exchange moves also keep S^z).
* At exact chi the oracle's sweep (environment reuse, running E^u updates) makes the same
  accept/reject decisions as a brute-force sweep that reads ratios off the exact state vector
  with the same Philox uniforms.
"""
import numpy as np
import pytest

from paper_2503_12557_gb300.inputs import Lattice, peps_random, configs_neel, configs_uniform
from oracle import sampler, exact
from oracle.philox import uniform53, key_of_seed


@pytest.mark.parametrize("move,up", [("exchange", False), ("flip", False), ("exchange", True), ("flip", True)])
def test_detailed_balance_and_stationarity(move, up):
    lat = Lattice(3, 3, 2, 2)
    th = peps_random(lat, 5, scale=0.5, bias=1.0)
    psi = exact.state_vector(th, lat)
    p = np.abs(psi) ** 2
    p = p / p.sum()
    P, kernels = sampler.transition_matrix_exact(psi, lat, move, up=up)
    for K in kernels:
        assert np.allclose(K.sum(1), 1.0, atol=1e-13)
        F = p[:, None] * K
        assert np.max(np.abs(F - F.T)) < 1e-13
    assert np.max(np.abs(p @ P - p)) < 1e-12
    if move == "exchange":
        Sall = exact.index_configs(9, 2)
        sz = Sall.sum(1)
        nz = np.argwhere(P > 0)
        assert np.all(sz[nz[:, 0]] == sz[nz[:, 1]])


def _bruteforce_sweep(psi, S, lat, move, seed, chain, sweep_id):
    Lx, Ly, d = lat.Lx, lat.Ly, lat.d
    key = key_of_seed(seed)
    slot = 0
    S = S.copy()

    def lnp(s):
        return np.log(abs(psi[exact.config_index(s, d)]))

    up = sweep_id % 2 == 1      # odd sweeps run up the rows, vertical bonds to the row above
    for x in (range(Lx - 1, -1, -1) if up else range(Lx)):
        moves = [(x * Ly + y, x * Ly + y + 1) for y in range(Ly - 1)] if move == "exchange" \
            else [(x * Ly + y,) for y in range(Ly)]
        if move == "exchange" and not up and x < Lx - 1:
            moves += [(x * Ly + y, (x + 1) * Ly + y) for y in range(Ly)]
        if move == "exchange" and up and x > 0:
            moves += [((x - 1) * Ly + y, x * Ly + y) for y in range(Ly)]
        for m in moves:
            u = uniform53((slot, sweep_id, chain, 0), key)
            slot += 1
            S2 = S.copy()
            if len(m) == 2:
                if S[m[0]] == S[m[1]]:
                    continue
                S2[m[0]], S2[m[1]] = S[m[1]], S[m[0]]
            else:
                S2[m[0]] = d - 1 - S[m[0]]
            if u < np.exp(2 * (lnp(S2) - lnp(S))):
                S = S2
    return S


@pytest.mark.parametrize("move,lat", [("exchange", Lattice(3, 4, 2, 2)), ("flip", Lattice(4, 3, 2, 2))])
def test_sweep_matches_bruteforce_at_exact_chi(move, lat):
    th = peps_random(lat, 17, scale=0.5, bias=1.0)
    psi = exact.state_vector(th, lat)
    S0 = configs_neel(lat, 3) if move == "exchange" else configs_uniform(lat, 3, 2)
    acc_total = 0
    for c in range(3):
        a = S0[c].copy()
        b = S0[c].copy()
        for k in range(3):
            a, acc, att = sampler.sweep(th, a, lat, 16, move, seed=99, chain=c, sweep_id=k)
            b = _bruteforce_sweep(psi, b, lat, move, 99, c, k)
            assert np.array_equal(a, b)
            acc_total += acc
            assert acc <= att
    assert acc_total > 0

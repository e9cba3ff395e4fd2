"""Pins of the oracle's local energy and log-derivatives.

* E_loc(S) = (H psi)(S)/psi(S) per configuration at exact chi (Eq. (local_obs)), for the
  Heisenberg, J1-J2-chiral (complex PEPS) and Rydberg Hamiltonians; the mean of E_loc under
  |psi|^2 equals <psi|H|psi>/<psi|psi> (Eq. (local_estimator)).
* A planted mistake (the transposed matrix element order) fails the chiral check.
* O: Euler identity sum_k T_k O_k = 1 per site (exact even below the exact chi: psi_x is
  linear in every tensor of row x), and central finite differences of the exact ln psi.
"""
import math

import numpy as np
import pytest

from paper_2503_12557_gb300.inputs import (Lattice, csl, peps_random, configs_uniform_sz0, configs_uniform,
                                           heisenberg, j1j2_chiral, rydberg, site_offsets, theta_to_tensors)
from oracle import energy, exact, tn


def _check_eloc_exact(lat, th, H, chi, configs, tol=1e-10):
    psi = exact.state_vector(th, lat)
    Hm = exact.hamiltonian_sparse(H, lat)
    ex = exact.exact_local_energy(psi, Hm)
    for S in configs:
        e, st = energy.local_energy(th, S, lat, chi, H)
        ref = ex[exact.config_index(S, lat.d)]
        assert abs(e - ref) <= tol * max(1.0, abs(ref)), (e, ref)


def test_eloc_heisenberg_4x4():
    lat = Lattice(4, 4, 2, 2)
    th = peps_random(lat, 1001)
    _check_eloc_exact(lat, th, heisenberg(lat), 4, configs_uniform_sz0(lat, 10, 2001))


def test_eloc_chiral_complex_3x3():
    lat = Lattice(3, 3, 2, 2)
    th = peps_random(lat, 21, complex_=True)
    H = j1j2_chiral(lat)
    _check_eloc_exact(lat, th, H, 8, configs_uniform(lat, 8, 4))


def test_eloc_rydberg_3x3():
    lat = Lattice(3, 3, 2, 2)
    th = peps_random(lat, 31, scale=0.5, bias=1.0)
    H = rydberg(lat, delta=1.0)
    _check_eloc_exact(lat, th, H, 8, configs_uniform(lat, 8, 5))


@pytest.mark.parametrize("model", ["j1j2_chiral", "csl"])
def test_energy_average_equals_expectation_complex(model):
    lat = Lattice(2, 3, 2, 2)
    th = peps_random(lat, 41, complex_=True)
    H = j1j2_chiral(lat) if model == "j1j2_chiral" else csl(lat)
    psi = exact.state_vector(th, lat)
    Hm = exact.hamiltonian_sparse(H, lat)
    Sall = exact.index_configs(lat.nsites, 2).astype(np.uint8)
    el = np.array([energy.local_energy(th, S, lat, 8, H)[0] for S in Sall])
    p = np.abs(psi) ** 2
    avg = np.sum(p * el) / np.sum(p)
    assert abs(avg - exact.exact_energy(psi, Hm)) < 1e-12
    # planted mistake: the transposed matrix element order <S'|h|S> gives a different energy
    Ht = dict(H)
    Ht["terms"] = [(s, h.T.copy()) for s, h in H["terms"]]
    elt = np.array([energy.local_energy(th, S, lat, 8, Ht)[0] for S in Sall])
    assert abs(np.sum(p * elt) / np.sum(p) - avg) > 1e-3


def test_diagonal_terms_need_no_amplitude():
    # a Hamiltonian of only diagonal parts gives the same E_loc for any PEPS
    lat = Lattice(3, 3, 2, 2)
    H = rydberg(lat, delta=2.0)
    H["terms"] = []
    S = configs_uniform(lat, 1, 2)[0]
    e1, _ = energy.local_energy(peps_random(lat, 1), S, lat, 4, H)
    e2, _ = energy.local_energy(peps_random(lat, 2), S, lat, 4, H)
    ref = sum(v * S[i] * S[j] for i, j, v in H["pairs"]) - 2.0 * S.sum()
    assert abs(e1 - ref) < 1e-12 and abs(e2 - ref) < 1e-12


@pytest.mark.parametrize("lat,chi,init", [
    (Lattice(4, 4, 2, 2), 2, dict()),                       # truncated: Euler still exact
    (Lattice(5, 4, 2, 3), 5, dict(scale=0.5, bias=1.0)),
])
def test_logderiv_euler_identity(lat, chi, init):
    th = peps_random(lat, 8, **init)
    offs = site_offsets(lat)
    for S in configs_uniform(lat, 3, 1):
        O = energy.log_derivative(th, S, lat, chi)
        for i in range(lat.nsites):
            assert abs(np.dot(th[offs[i]:offs[i + 1]], O[offs[i]:offs[i + 1]]) - 1.0) < 1e-11


def test_logderiv_zero_off_slice():
    lat = Lattice(3, 3, 2, 2)
    th = peps_random(lat, 9)
    T = theta_to_tensors(lat, th)
    offs = site_offsets(lat)
    S = configs_uniform(lat, 1, 3)[0]
    O = energy.log_derivative(th, S, lat, 4)
    for i in range(lat.nsites):
        blk = O[offs[i]:offs[i + 1]].reshape(T[i // 3][i % 3].shape)
        assert np.all(blk[1 - S[i]] == 0)


@pytest.mark.parametrize("cplx", [False, True])
def test_logderiv_finite_difference(cplx):
    lat = Lattice(3, 3, 2, 2)
    th = peps_random(lat, 12, complex_=cplx)
    S = configs_uniform(lat, 1, 7)[0]
    O = energy.log_derivative(th, S, lat, 4)
    psi0 = exact.amplitude_rowtransfer(th, S, lat)
    rng = np.random.default_rng(0)
    idx = np.flatnonzero(O != 0)
    h = 1e-6
    for k in rng.choice(idx, 12, replace=False):
        tp, tm = th.copy(), th.copy()
        tp[k] += h
        tm[k] -= h
        fd = (exact.amplitude_rowtransfer(tp, S, lat) - exact.amplitude_rowtransfer(tm, S, lat)) / (2 * h) / psi0
        assert abs(fd - O[k]) <= 1e-7 * max(1.0, abs(O[k]))

"""Pins of the oracle's variational-bound estimator (oracle/bound.py).

* With one fixed cut i, the |psi_i|^2-weighted mean of E_loc^bound over a whole magnetisation
  sector equals <psi_i|H|psi_i> / <psi_i|psi_i> from a sparse H built independently, at a
  truncating chi, for real and complex PEPS (a term taken from another cut's amplitude, a
  transposed matrix element or a dropped conjugate breaks it), and it is above the ground
  state.  The fast estimator, which mixes cuts, does not satisfy the identity there.
* At the two ends the cut amplitude is a one-row sandwich (i = 1: exact top row against the
  truncated lower environment; i = Lx-1: psi_top).
* At exact chi, psi_i is the exact amplitude and E_loc^bound the exact (H psi)(S) / psi(S).
"""
import math

import numpy as np
import pytest

from paper_2503_12557_gb300 import inputs as I
from oracle import bound, energy, exact, tn


def _sector(lat, n_up):
    allS = exact.index_configs(lat.nsites, lat.d)
    return allS[allS.sum(axis=1) == n_up]


def _sector_vectors(th, lat, chi, H, i, Ssec):
    T = I.theta_to_tensors(lat, th)
    dim = lat.d ** lat.nsites
    psi = np.zeros(dim, dtype=np.complex128)
    el = np.zeros(len(Ssec), dtype=np.complex128)
    for n, S in enumerate(Ssec):
        e, l0, p0, st = bound.local_energy_bound(th, S, lat, chi, H, i, T=T)
        assert st & tn.NEAR_DEGENERATE == 0
        psi[exact.config_index(S, lat.d)] = math.exp(l0) * complex(math.cos(p0), math.sin(p0))
        el[n] = e
    return psi, el


@pytest.mark.parametrize("cplx,i", [(False, 1), (False, 2), (True, 1)])
def test_bound_is_the_energy_of_one_fixed_state(cplx, i):
    lat = I.Lattice(3, 3, 2, 3)
    chi = 2                                               # Schmidt rank up to 3 across a 3-site row: truncating
    th = I.peps_random(lat, 5 + i, scale=0.6, bias=1.0, complex_=cplx)
    H = I.j1j2_chiral(lat, J1=1.0, J2=0.5, Jchi=0.4 if cplx else 0.0)
    if not cplx:
        H["terms"] = [t for t in H["terms"] if len(t[0]) == 2]
    Hm = exact.hamiltonian_sparse(H, lat)
    Ssec = _sector(lat, 4)                                # S^z conserved: 126 configurations
    psi, el = _sector_vectors(th, lat, chi, H, i, Ssec)
    w = np.abs(psi[[exact.config_index(S, 2) for S in Ssec]]) ** 2
    mean = np.sum(w * el) / np.sum(w)
    ref = np.vdot(psi, Hm @ psi) / np.vdot(psi, psi)
    assert abs(mean - ref) <= 1e-11 * max(1.0, abs(ref)), (mean, ref)
    assert abs(ref.imag) < 1e-12
    # variational: above the lowest energy of the sector's Hamiltonian
    idx = [exact.config_index(S, 2) for S in Ssec]
    e0 = np.linalg.eigvalsh(Hm[idx][:, idx].toarray())[0]
    assert mean.real >= e0 - 1e-12
    # the same identity fails for the fast estimator (amplitudes from several cuts): the
    # truncation is strong enough here for the pin to see a mixed-cut mistake
    fast = energy.evaluate(th, Ssec, lat, chi, H=H, want_O=False)
    ptop = np.zeros_like(psi)
    ptop[idx] = np.exp(fast["logabs"] + 1j * fast["phase"])
    wf = np.abs(ptop[idx]) ** 2
    mf = np.sum(wf * fast["eloc"]) / np.sum(wf)
    rf = np.vdot(ptop, Hm @ ptop) / np.vdot(ptop, ptop)
    assert abs(mf - rf) > 1e-6 * max(1.0, abs(rf))


def test_cut_at_the_ends_is_a_row_sandwich():
    lat = I.Lattice(4, 3, 2, 3)
    th = I.peps_random(lat, 17, scale=0.5, bias=1.0)
    T = I.theta_to_tensors(lat, th)
    for S in I.configs_uniform(lat, 4, 18):
        env, Ap = tn.environments(T, S, lat, 2)
        for i, x in ((1, 0), (lat.Lx - 1, lat.Lx - 1)):
            l1, p1, _ = bound.psi_cut(T, S, lat, 2, i)
            l2, p2 = tn.log_psi_row(env, Ap, x)
            assert abs(l1 - l2) < 1e-12 and abs(np.angle(np.exp(1j * (p1 - p2)))) < 1e-12
        # an interior cut is a different approximation at this chi
        lm, _, _ = bound.psi_cut(T, S, lat, 2, 2)
        assert abs(lm - tn.log_psi_row(env, Ap, lat.Lx - 1)[0]) > 1e-9


def test_exact_chi_gives_exact_amplitudes_and_local_energy():
    lat = I.Lattice(3, 3, 2, 2)
    th = I.peps_random(lat, 23)
    H = I.heisenberg(lat)
    psi = exact.state_vector(th, lat)
    Hm = exact.hamiltonian_sparse(H, lat)
    ex = exact.exact_local_energy(psi, Hm)
    T = I.theta_to_tensors(lat, th)
    for S in I.configs_uniform(lat, 5, 24):
        k = exact.config_index(S, 2)
        for i in (1, 2):
            l0, p0, st = bound.psi_cut(T, S, lat, 4, i)
            assert abs(l0 - math.log(abs(psi[k]))) < 1e-11
            assert abs(np.angle(np.exp(1j * p0) / np.sign(psi[k]))) < 1e-11
            e, _, _, _ = bound.local_energy_bound(th, S, lat, 4, H, i, T=T)
            assert abs(e - ex[k]) <= 1e-10 * max(1.0, abs(ex[k]))


def test_bad_cut_rejected():
    lat = I.Lattice(3, 3, 2, 2)
    T = I.theta_to_tensors(lat, I.peps_random(lat, 1))
    S = np.zeros(9, dtype=np.uint8)
    for i in (0, 3):
        with pytest.raises(ValueError):
            bound.psi_cut(T, S, lat, 2, i)

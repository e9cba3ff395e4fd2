"""Model Hamiltonians against closed-form spectra (pins the term lists shared by both paths)."""
import math

import numpy as np

from paper_2503_12557_gb300.inputs import Lattice, csl, heisenberg, j1j2_chiral, rydberg
from oracle import exact


def _dense(H, lat):
    return exact.hamiltonian_sparse(H, lat).toarray()


def test_heisenberg_dimer():
    # one bond: singlet -3/4 J, triplet +1/4 J
    ev = np.linalg.eigvalsh(_dense(heisenberg(Lattice(1, 2, 2, 1), J=1.0), Lattice(1, 2, 2, 1)))
    assert np.allclose(sorted(ev), [-0.75, 0.25, 0.25, 0.25])


def test_heisenberg_2x2_is_four_site_ring():
    lat = Lattice(2, 2, 2, 1)
    ev = np.linalg.eigvalsh(_dense(heisenberg(lat), lat))
    assert abs(ev[0] - (-2.0)) < 1e-12  # 4-site Heisenberg ring ground energy -2J
    assert len(heisenberg(lat)["terms"]) == 4


def test_heisenberg_bond_count():
    for L in (4, 8, 12):
        assert len(heisenberg(Lattice(L, L, 2, 1))["terms"]) == 2 * L * (L - 1)


def test_chirality_spectrum():
    # S1.(S2 x S3) on three spin-1/2: eigenvalues 0 (x4, the S=3/2 quartet) and +-sqrt(3)/4 (x2 each)
    H = j1j2_chiral(Lattice(2, 2, 2, 1), J1=0.0, J2=0.0, Jchi=1.0)
    h = H["terms"][-1][1]
    ev = np.sort(np.linalg.eigvalsh(h))
    s = math.sqrt(3) / 4
    assert np.allclose(ev, [-s, -s, 0, 0, 0, 0, s, s])
    assert np.allclose(h, h.conj().T)
    # purely imaginary, antisymmetric matrix (time-reversal odd)
    assert np.allclose(h.real, 0)


def test_j1j2_chiral_counts():
    lat = Lattice(10, 10, 2, 1)
    H = j1j2_chiral(lat)
    n2 = sum(1 for s, _ in H["terms"] if len(s) == 2)
    n3 = sum(1 for s, _ in H["terms"] if len(s) == 3)
    assert n2 == 180 + 162 and n3 == 324


def test_rydberg_single_atom():
    lat = Lattice(1, 1, 2, 1)
    for delta in (0.0, 1.0, 3.0):
        ev = np.linalg.eigvalsh(_dense(rydberg(lat, delta=delta), lat))
        # H = 1/2 sigma^x - delta n : eigenvalues -delta/2 -+ sqrt(delta^2 + 1)/2
        ref = sorted([-delta / 2 - math.sqrt(delta ** 2 + 1) / 2, -delta / 2 + math.sqrt(delta ** 2 + 1) / 2])
        assert np.allclose(ev, ref)


def test_rydberg_pairs():
    H = rydberg(Lattice(12, 12, 2, 1))
    assert len(H["pairs"]) == 2550
    # nearest-neighbour coupling V0 / 1 = Rb^6
    i, j, v01 = H["pairs"][0]
    assert (i, j) == (0, 1) and abs(v01 - 1.7 ** 6) < 1e-12


def test_csl_ring_term_spectrum_and_action():
    # i(P - P^-1) with P the cyclic shift of four spin-1/2: P has eigenvalues +-i three times each
    # (one per orbit of four basis states), so the ring term has eigenvalues +-2 lam (x3) and 0 (x10)
    lam = 0.37
    H = csl(Lattice(2, 2, 2, 1), J1=0.0, J2=0.0, lam=lam)
    ring = [h for s, h in H["terms"] if len(s) == 4]
    assert len(ring) == 1
    h = ring[0]
    ev = np.sort(np.linalg.eigvalsh(h))
    assert np.allclose(ev, [-2 * lam] * 3 + [0.0] * 10 + [2 * lam] * 3)
    assert np.allclose(h, h.conj().T) and np.allclose(h.real, 0)
    # P|s1 s2 s3 s4> = |s4 s1 s2 s3> and P^-1|s1 s2 s3 s4> = |s2 s3 s4 s1>, checked on a basis state
    e = np.zeros(16)
    e[0b0100] = 1.0
    out = (h / (1j * lam)) @ e  # (P - P^-1) |0100> = |0010> - |1000>
    ref = np.zeros(16)
    ref[0b0010], ref[0b1000] = 1.0, -1.0
    assert np.allclose(out, ref)


def test_csl_commutes_with_total_spin_and_counts():
    lat = Lattice(2, 3, 2, 1)
    Hm = _dense(csl(lat), lat)
    # SU(2) invariance: [H, S^z_total] = 0 and [H, (S^x_total)] = 0
    n = lat.nsites
    sx = np.array([[0, 0.5], [0.5, 0]])
    sz = np.diag([0.5, -0.5])
    def total(op):
        tot = np.zeros((2 ** n, 2 ** n), dtype=complex)
        for i in range(n):
            m = np.array([[1.0]])
            for j in range(n):
                m = np.kron(m, op if j == i else np.eye(2))
            tot += m
        return tot
    for op in (sx, sz):
        T = total(op)
        assert np.allclose(Hm @ T - T @ Hm, 0, atol=1e-12)
    H = csl(Lattice(16, 16, 2, 1))
    assert sum(1 for s, _ in H["terms"] if len(s) == 4) == 15 * 15
    assert sum(1 for s, _ in H["terms"] if len(s) == 2) == 2 * 16 * 15 + 2 * 15 * 15

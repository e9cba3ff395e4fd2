"""Model Hamiltonians against closed-form spectra (pins the term lists shared by both paths)."""
import math

import numpy as np

from paper_2503_12557_gb300.inputs import Lattice, heisenberg, j1j2_chiral, rydberg
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

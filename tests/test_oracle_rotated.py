"""Pins of the rotated-basis estimator's inputs and oracle (inputs.axis_parts, oracle/rotated.py).

* The three diagonal parts, rotated back with V_alpha^{(x)N}, sum to the Heisenberg-type H
  (J1 and J2 bonds) on a 2 x 3 lattice.
* The rotated PEPS contracted exactly equals the rotated state vector (V^dagger)^{(x)N} psi.
* The per-basis energies of the rotated PEPS sum to <psi|H|psi> / <psi|psi> of the unrotated one.
"""
import numpy as np

from paper_2503_12557_gb300 import inputs as I
from oracle import exact, rotated


def _kron_n(V, n):
    out = np.array([[1.0 + 0j]])
    for _ in range(n):
        out = np.kron(out, V)
    return out


def test_parts_rotate_back_to_h():
    lat = I.Lattice(2, 3, 2, 1)
    bonds = I.spin_bonds(lat, J1=1.0, J2=0.45)
    H = I.j1j2_chiral(lat, J1=1.0, J2=0.45, Jchi=0.0)
    H["terms"] = [t for t in H["terms"] if len(t[0]) == 2]
    Hm = exact.hamiltonian_sparse(H, lat).toarray()
    tot = np.zeros_like(Hm)
    for V, Hd in I.axis_parts(lat, bonds):
        Dg = exact.hamiltonian_sparse(Hd, lat).toarray()
        assert np.allclose(Dg, np.diag(np.diag(Dg)))        # diagonal in its own basis
        U = _kron_n(V, lat.nsites)
        tot += U @ Dg @ U.conj().T
    assert np.allclose(tot, Hm, atol=1e-12)
    # the bases: columns are sigma^alpha eigenvectors with eigenvalues +1, -1
    for V, P in zip(I.axis_bases(), I.pauli()):
        assert np.allclose(P @ V, V @ np.diag([1.0, -1.0]))
        assert np.allclose(V.conj().T @ V, np.eye(2))


def test_rotated_peps_is_rotated_state_vector():
    lat = I.Lattice(3, 3, 2, 2)
    th = I.peps_random(lat, 3, scale=0.6, bias=1.0)
    psi = exact.state_vector(th, lat)
    for V in I.axis_bases():
        M = V.conj().T
        th2 = rotated.rotate_theta(th, lat, M)
        psi2 = exact.state_vector(th2, lat)
        ref = _kron_n(M, lat.nsites) @ psi
        assert np.allclose(psi2, ref, atol=1e-12 * np.max(np.abs(ref)))


def test_energy_from_rotated_bases_is_the_energy():
    lat = I.Lattice(3, 3, 2, 2)
    for seed, cplx in ((5, False), (6, True)):
        th = I.peps_random(lat, seed, scale=0.6, bias=1.0, complex_=cplx)
        bonds = I.spin_bonds(lat, J1=1.0, J2=0.5)
        H = I.j1j2_chiral(lat, J1=1.0, J2=0.5, Jchi=0.0)
        H["terms"] = [t for t in H["terms"] if len(t[0]) == 2]
        e_ref = exact.exact_energy(exact.state_vector(th, lat), exact.hamiltonian_sparse(H, lat)).real
        e, per = rotated.energy_exact(th, lat, I.axis_parts(lat, bonds))
        assert abs(e - e_ref) < 1e-11 * max(1.0, abs(e_ref))
        assert len(per) == 3 and all(np.isfinite(per))

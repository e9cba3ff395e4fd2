"""Pins of the oracle's MinSR solve (Eq. (tdvp_fast)) against the SR forms it replaces
(Eq. (tdvp_slow)) and against the exact energy."""
import numpy as np

from paper_2503_12557_gb300.inputs import Lattice, peps_random, configs_uniform_sz0, heisenberg
from oracle import minsr, energy, exact


def _problem(ns=64, npar=200, seed=0, cplx=False):
    rng = np.random.default_rng(seed)
    O = rng.standard_normal((ns, npar)) + 0.3
    e = rng.standard_normal(ns) - 2.0
    if cplx:
        O = O + 1j * rng.standard_normal((ns, npar))
        e = e + 0.1j * rng.standard_normal(ns)
    return O, e


def test_pushthrough_identity():
    for cplx in (False, True):
        O, e = _problem(cplx=cplx)
        a, _ = minsr.minsr(O, e, lam=1e-3, tau=0.1)
        b = minsr.sr_pushthrough(O, e, lam=1e-3, tau=0.1)
        assert np.linalg.norm(a - b) <= 1e-10 * np.linalg.norm(b)


def test_weighted_pushthrough():
    O, e = _problem(seed=3)
    w = np.random.default_rng(1).uniform(0.2, 2.0, O.shape[0])
    a, _ = minsr.minsr(O, e, w=w, lam=1e-2)
    b = minsr.sr_pushthrough(O, e, w=w, lam=1e-2)
    assert np.linalg.norm(a - b) <= 1e-10 * np.linalg.norm(b)


def test_pinv_identity_and_min_norm():
    O, e = _problem(ns=50, npar=120, seed=4)
    rc = 1e-10
    a, info = minsr.minsr(O, e, lam=0.0, rcond=rc, tau=1.0)
    b = minsr.sr_pinv(O, e, tau=1.0, rcond=np.sqrt(rc))
    assert info["rank"] == 49  # centring removes one direction
    assert np.linalg.norm(a - b) <= 1e-9 * np.linalg.norm(b)
    # exact solve on the sampled space: Obar (-dtheta) = ebar when Obar has full row rank after centring
    Ob, eb = minsr.centred(O, e)
    assert np.linalg.norm(Ob @ (-a) - eb) <= 1e-9 * np.linalg.norm(eb)
    # minimum norm: adding a null-space component only increases the norm
    null = np.linalg.svd(Ob)[2][-1]
    assert np.linalg.norm(-a + 0.1 * null) > np.linalg.norm(a)


def test_energy_decreases_with_exact_weights():
    # all Sz=0 configurations weighted by |psi|^2: a small MinSR step lowers the exact energy
    lat = Lattice(3, 4, 2, 2)
    th = peps_random(lat, 1001)
    H = heisenberg(lat)
    psi = exact.state_vector(th, lat)
    Hm = exact.hamiltonian_sparse(H, lat)
    Sall = exact.index_configs(12, 2)
    sz0 = Sall.sum(1) == 6
    S = Sall[sz0].astype(np.uint8)
    p = np.abs(psi[sz0]) ** 2
    res = energy.evaluate(th, S, lat, 4, H=H)
    dth, _ = minsr.minsr(res["O"], res["eloc"].real, w=p, lam=1e-6, tau=0.02)
    E0 = exact.exact_energy(psi, Hm).real
    E1 = exact.exact_energy(exact.state_vector(th + dth.real, lat), Hm).real
    assert E1 < E0 - 1e-4

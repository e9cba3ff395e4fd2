"""MinSR with a pseudo-inverse cutoff through the tridiagonal form (Eq. (tdvp_fast)): Householder
reduction, implicit QR on the tridiagonal form applied to the transformed ebar, rotations
replayed, reflectors applied back.  Taken with cfg.solve = 3 (the default cutoff route is the
cyclic Jacobi); compared with the oracle's MinSR (eigendecomposition of T, cutoff, dtheta) on
the same inputs.

Gate: dtheta to 1e-9 in relative 2-norm, as the cyclic Jacobi route's parity tests.  Both sides
are backward-stable FP64 eigensolvers whose eigenvalues carry absolute errors of order
eps max(Lambda); the cases keep no eigenvalue closer to zero than about 1e-3 max(Lambda), so the
kept components agree far inside the gate.  The rank kept is compared exactly: the cut
eigenvalues (the centring's null vector, the zero eigenvalues of a rank-deficient O) lie many
orders of magnitude below the cutoff.
"""
import numpy as np
import pytest
import torch

from paper_2503_12557_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    from paper_2503_12557_gb300 import build, peps
    build.build()
    return peps


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a)).cuda()


def _minsr_raw(P, O, e, lam, rc, tau, solve):
    """minsr_step on a handle whose N_p covers O's column count (zero-padded columns change no
    MinSR value)."""
    ns, npar = O.shape
    for Ly in range(2, 33):
        for D in range(1, 9):
            lat = I.Lattice(2, Ly, 2, D)
            if I.num_params(lat) >= npar:
                break
        if I.num_params(lat) >= npar:
            break
    h = P.PEPS(lat.Lx, lat.Ly, 2, lat.D, lat.D, max_samples=2, solve=solve)
    Op = np.zeros((ns, h.Np))
    Op[:, :npar] = O
    dth, info = h.minsr_step(_dev(Op), _dev(np.stack([e, np.zeros(ns)], 1)), lam=lam, rcond=rc, tau=tau)
    word = h.last_status()
    h.close()
    return dth.cpu().numpy()[:npar], info.cpu().numpy(), word


@pytest.mark.parametrize("ns,npar,lam,rc,solve", [
    (333, 500, 1e-4, 1e-9, 3),    # forced at a small size, odd Ns (padding row)
    (64, 40, 1e-3, 1e-8, 3),      # rank-deficient O: 24 zero eigenvalues cut
    (2, 3, 1e-3, 1e-8, 3),        # the smallest problem: no Householder step
    (3, 5, 1e-3, 1e-8, 3),        # one Householder step
    (1030, 1200, 1e-4, 1e-8, 3),  # above 1024 rows
    (1031, 900, 1e-3, 1e-10, 3),  # above 1024 rows, rank-deficient, odd Ns
])
def test_minsr_tridiagonal_route_vs_oracle(P, ns, npar, lam, rc, solve):
    from oracle import minsr
    rng = np.random.default_rng(ns + 17)
    O = rng.standard_normal((ns, npar)) + 0.1 * rng.standard_normal(npar)
    e = rng.standard_normal(ns) - 3.0
    d_ref, inf_ref = minsr.minsr(O, e, lam=lam, rcond=rc, tau=0.1)
    dth, info, word = _minsr_raw(P, O, e, lam, rc, 0.1, solve)
    assert word == 0
    assert np.linalg.norm(dth - d_ref) <= 1e-9 * np.linalg.norm(d_ref)
    assert int(info[0]) == inf_ref["rank"]
    assert abs(info[2] - inf_ref["lmax"]) <= 1e-10 * inf_ref["lmax"]
    assert info[3] >= 1  # QR steps


def test_minsr_tridiagonal_route_matches_jacobi_route(P):
    # the two cutoff routes of the library on the same inputs (the Jacobi one is the default):
    # the same rank and dtheta up to rounding
    rng = np.random.default_rng(99)
    O = rng.standard_normal((200, 260)) + 0.1 * rng.standard_normal(260)
    e = rng.standard_normal(200)
    d3, i3, _ = _minsr_raw(P, O, e, 1e-3, 1e-8, 0.05, 3)
    d0, i0, _ = _minsr_raw(P, O, e, 1e-3, 1e-8, 0.05, 0)
    assert int(i3[0]) == int(i0[0])
    assert np.linalg.norm(d3 - d0) <= 1e-10 * np.linalg.norm(d0)


def test_complex_minsr_tridiagonal_route_vs_oracle(P):
    # complex PEPS: the real embedding repeats every eigenvalue; the rank is reported once each
    from oracle import energy, minsr
    lat = I.Lattice(3, 3, 2, 2)
    th = I.peps_random(lat, 4, scale=0.6, bias=1.0, complex_=True)
    S = I.configs_uniform_sz0(lat, 48, 5)
    ref = energy.evaluate(th, S, lat, 4, H=I.j1j2_chiral(lat), want_O=True)
    h = P.PEPS(lat.Lx, lat.Ly, lat.d, lat.D, 4, max_samples=len(S), cplx=True, solve=3)
    Od = torch.as_tensor(ref["O"]).cuda()
    ed = torch.as_tensor(np.stack([ref["eloc"].real, ref["eloc"].imag], 1)).cuda()
    dth, info = h.minsr_step(Od, ed, lam=1e-3, rcond=1e-10, tau=0.07)
    torch.cuda.synchronize()
    d_ref, inf_ref = minsr.minsr(ref["O"], ref["eloc"], lam=1e-3, rcond=1e-10, tau=0.07)
    d = dth.cpu().numpy()
    assert np.linalg.norm(d - d_ref) <= 1e-9 * np.linalg.norm(d_ref)
    assert int(info[0].item()) == inf_ref["rank"]
    h.close()

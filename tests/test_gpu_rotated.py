"""The rotated-basis estimator through the C ABI: the device rotation of the physical index
(peps_rotate_params) against the oracle's, amplitudes of the rotated (complex) PEPS against the
oracle's contraction, the diagonal-only energy path against the oracle's diagonal value, and
the sampled three-basis energy against the exact energy of the same PEPS."""
import numpy as np
import pytest
import torch

from paper_2503_12557_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2503_12557_gb300 import build, peps
    build.build()
    return peps


@pytest.mark.parametrize("cplx_in", [False, True])
def test_rotate_params_vs_oracle(P, cplx_in):
    from oracle import rotated
    lat = I.Lattice(4, 5, 2, 3)
    th = I.peps_random(lat, 71, scale=0.6, bias=1.0, complex_=cplx_in)
    h = P.PEPS(4, 5, 2, 3, 9, max_samples=1, cplx=True)
    for V in I.axis_bases():
        M = V.conj().T
        out = h.rotate_params(M, torch.as_tensor(th).cuda())
        torch.cuda.synchronize()
        ref = rotated.rotate_theta(th, lat, M)
        assert np.max(np.abs(out.cpu().numpy() - ref)) <= 1e-15 * max(1.0, np.max(np.abs(ref)))


def test_rotated_amplitudes_and_diagonal_energy_vs_oracle(P):
    from oracle import energy, rotated
    lat = I.Lattice(4, 4, 2, 2)
    th = I.peps_random(lat, 73, scale=0.5, bias=1.0)
    S = I.configs_uniform(lat, 12, 74)
    parts = I.axis_parts(lat, I.spin_bonds(lat, J1=1.0, J2=0.5))
    h = P.PEPS(4, 4, 2, 2, 3, max_samples=len(S), cplx=True)
    Sd = torch.as_tensor(S).cuda()
    for V, Hd in parts:
        M = V.conj().T
        h.set_params(h.rotate_params(M, torch.as_tensor(th).cuda()))
        r = h.evaluate(None, Sd, want_eloc=False, want_O=False)
        e = h.evaluate(Hd, Sd, want_logpsi=False, want_eloc=True, want_O=False)
        torch.cuda.synchronize()
        ref = energy.evaluate(rotated.rotate_theta(th, lat, M), S, lat, 3, H=None, want_O=False)
        ok = (ref["status"] & 1) == 0
        assert np.max(np.abs(r["logabs"].cpu().numpy() - ref["logabs"])[ok]) <= 1e-10
        dph = np.angle(np.exp(1j * (r["phase"].cpu().numpy() - ref["phase"])))
        assert np.max(np.abs(dph)[ok]) <= 1e-9
        dv = np.array([rotated.diagonal_value(Hd, s) for s in S])
        assert np.max(np.abs(e["eloc"].cpu().numpy()[:, 0] - dv)) <= 1e-12
        assert np.all(e["eloc"].cpu().numpy()[:, 1] == 0.0)


def test_sampled_rotated_energy_matches_exact(P):
    # 4 x 4 at exact chi: flip chains on each rotated PEPS, diagonal energies averaged; the
    # sum against the exact <H> of the unrotated PEPS (oracle state vector), within 5 sigma
    from oracle import rotated
    from paper_2503_12557_gb300 import estimators
    lat = I.Lattice(4, 4, 2, 2)
    th = I.peps_random(lat, 75, scale=0.5, bias=1.0)
    bonds = I.spin_bonds(lat, J1=1.0, J2=0.5)
    e_ex, per_ex = rotated.energy_exact(th, lat, I.axis_parts(lat, bonds))
    S0 = I.configs_uniform(lat, 4096, 76)
    e, se, per = estimators.rotated_basis_energy(4, 4, 2, 4, torch.as_tensor(th).cuda(), bonds, S0,
                                                 burn_in=30, seed=77)
    print(f"rotated-basis energy {e:.5f} +- {se:.5f}, exact {e_ex:.5f}; per basis "
          + ", ".join(f"{m:.4f}+-{s:.4f} (exact {x:.4f}, acc {a:.2f})" for (m, s, a), x in zip(per, per_ex)))
    for (m, s, a), x in zip(per, per_ex):
        assert abs(m - x) <= 5 * s + 1e-9
        assert 0.0 < a < 1.0
    assert abs(e - e_ex) <= 5 * se

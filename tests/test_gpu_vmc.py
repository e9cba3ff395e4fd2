"""The whole optimisation loop on the GPU (sample -> psi / E_loc / O -> MinSR -> update) on the
4x4 open Heisenberg model: the exact energy of the optimised PEPS (from the oracle's full state
vector, no sampling noise) falls toward the exact ground-state energy, and a run resumed from a
checkpoint repeats the uninterrupted run bit for bit."""
import json

import numpy as np
import pytest
import torch

from paper_2503_12557_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def V():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2503_12557_gb300 import build, peps, vmc
    build.build()
    return peps, vmc


def _exact(th, lat, H):
    from oracle import exact
    psi = exact.state_vector(th, lat)
    Hm = exact.hamiltonian_sparse(H, lat)
    return exact.exact_energy(psi, Hm).real / lat.nsites


def test_vmc_energy_decreases_toward_ground_state(V):
    import scipy.sparse.linalg as sla
    from oracle import exact
    P, vmc = V
    lat = I.Lattice(4, 4, 2, 2)
    H = I.heisenberg(lat)
    e0 = float(sla.eigsh(exact.hamiltonian_sparse(H, lat), k=1, which="SA")[0][0]) / lat.nsites
    th0 = I.peps_random(lat, 21, scale=0.5, bias=1.0)
    run = vmc.VMC(4, 4, 2, 2, 4, H, th0, I.configs_neel(lat, 512), seed=5, lam=1e-3, tau=0.1)
    run.burn_in(10)
    hist = run.run(40)
    th1 = run.theta.cpu().numpy()
    ea, eb = _exact(th0, lat, H), _exact(th1, lat, H)
    print(f"exact E/N: start {ea:.5f}, after 40 steps {eb:.5f}, ground state {e0:.5f}; "
          f"sampled {hist[-1]['energy_per_site']:.5f} +- {hist[-1]['stderr_per_site']:.5f}")
    assert eb < ea - 0.25 * (ea - e0)        # a quarter of the way to the ground state at least
    assert eb >= e0 - 1e-9                   # variational
    assert all(m["status_nonzero"] == 0 for m in hist)
    assert 0.05 < hist[-1]["acceptance"] < 1.0
    run.close()


def test_checkpoint_resume_repeats_the_run(V, tmp_path):
    P, vmc = V
    lat = I.Lattice(4, 4, 2, 2)
    H = I.heisenberg(lat)
    th0 = I.peps_random(lat, 22, scale=0.5, bias=1.0)
    a = vmc.VMC(4, 4, 2, 2, 3, H, th0, I.configs_neel(lat, 96), seed=9, lam=1e-3, tau=0.05)
    a.burn_in(4)
    a.run(3)
    ck = str(tmp_path / "ck")
    a.save(ck)
    log_a = str(tmp_path / "a.jsonl")
    a.run(3, log_path=log_a)
    b = vmc.VMC.load(ck, H)
    log_b = str(tmp_path / "b.jsonl")
    b.run(3, log_path=log_b)
    torch.cuda.synchronize()
    assert torch.equal(a.theta, b.theta) and torch.equal(a.S, b.S)
    la = [json.loads(x) for x in open(log_a)]
    lb = [json.loads(x) for x in open(log_b)]
    assert [m["energy_per_site"] for m in la] == [m["energy_per_site"] for m in lb]
    assert [m["step"] for m in lb] == [3, 4, 5]
    a.close()
    b.close()


def test_vmc_with_direct_sampling(V):
    # the paper's sampler inside the loop: independent draws from truncated double-layer
    # environments (chi_d = 2), importance weights |psi|^2 / p in the energy and in MinSR
    import scipy.sparse.linalg as sla
    from oracle import exact
    P, vmc = V
    lat = I.Lattice(4, 4, 2, 2)
    H = I.heisenberg(lat)
    e0 = float(sla.eigsh(exact.hamiltonian_sparse(H, lat), k=1, which="SA")[0][0]) / lat.nsites
    th0 = I.peps_random(lat, 21, scale=0.5, bias=1.0)
    run = vmc.VMC(4, 4, 2, 2, 4, H, th0, I.configs_neel(lat, 512), seed=5, lam=1e-3, tau=0.1,
                  sampler="direct", chi_double=2)
    hist = run.run(40)
    th1 = run.theta.cpu().numpy()
    ea, eb = _exact(th0, lat, H), _exact(th1, lat, H)
    print(f"direct sampling: exact E/N start {ea:.5f}, after 40 steps {eb:.5f}, ground state {e0:.5f}; "
          f"weighted {hist[-1]['energy_per_site']:.5f} +- {hist[-1]['stderr_per_site']:.5f}, "
          f"ESS {hist[-1]['ess_fraction']:.2f}")
    assert eb < ea - 0.25 * (ea - e0)
    assert eb >= e0 - 1e-9
    assert min(m["ess_fraction"] for m in hist) > 0.2
    run.close()

"""Learned proposal on the GPU (through the C ABI) against the FP64 oracle: logits, the training
gradient and Adam step, and whole network moves of Metropolis chains (same Philox streams)."""
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


def _bf16(w):
    return torch.as_tensor(w).to(torch.bfloat16).to(torch.float64).numpy()


@pytest.mark.parametrize("wprec", [0, 1])
def test_logits_vs_oracle(P, wprec):
    from oracle import proposal as Q
    Lx, Ly, C = 5, 6, 8
    lat = I.Lattice(Lx, Ly, 2, 1)
    w = I.proposal_init(11, C=C, scale=1.5)
    S = I.configs_uniform(lat, 40, 3)
    prop = P.Proposal(Lx, Ly, w, C=C, wprec=wprec)
    got = prop.logits(torch.as_tensor(S).cuda()).cpu().numpy()
    wref = w if wprec == 0 else _bf16(w)
    ref = np.array([Q.forward(wref, s, Lx, Ly, C).ravel() for s in S])
    tol = 1e-12 if wprec == 0 else 1e-5
    assert np.max(np.abs(got - ref)) <= tol * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("wprec", [0, 1])
def test_train_step_gradient_and_adam_vs_oracle(P, wprec):
    from oracle import proposal as Q
    Lx, Ly, C = 4, 5, 6
    lat = I.Lattice(Lx, Ly, 2, 1)
    w = I.proposal_init(12, C=C, scale=1.5)
    S_in = I.configs_uniform(lat, 33, 1)
    S_tg = I.configs_uniform(lat, 33, 2)
    prop = P.Proposal(Lx, Ly, w, C=C, wprec=wprec)
    loss = prop.train_step(torch.as_tensor(S_in).cuda(), torch.as_tensor(S_tg).cuda(), lr=1e-2)
    torch.cuda.synchronize()
    wref = w if wprec == 0 else _bf16(w)
    l_ref, g_ref = Q.loss_and_grad(wref, S_in, S_tg, Lx, Ly, C)
    g = prop.g.cpu().numpy()
    tol = 1e-10 if wprec == 0 else 1e-4
    assert abs(loss.item() - l_ref) <= tol * max(1.0, abs(l_ref))
    assert np.max(np.abs(g - g_ref)) <= tol * max(1e-3, np.abs(g_ref).max())
    w1, _, _ = Q.adam(w, g, np.zeros_like(w), np.zeros_like(w), 1, lr=1e-2)
    assert np.max(np.abs(prop.w.cpu().numpy() - w1)) < 1e-12


def test_learned_moves_match_oracle_chains(P):
    from oracle import proposal as Q, tn
    lat = I.Lattice(4, 4, 2, 2)
    chi, C = 3, 4
    th = I.peps_random(lat, 61, scale=0.3, bias=1.0)
    w = I.proposal_init(13, C=C, scale=0.5)
    nc = 12
    S0 = I.configs_uniform(lat, nc, 9)
    h = P.PEPS(lat.Lx, lat.Ly, 2, lat.D, chi, max_samples=nc)
    h.set_params(torch.as_tensor(th).cuda())
    prop = P.Proposal(lat.Lx, lat.Ly, w, C=C, wprec=0)
    Sd = torch.as_tensor(S0).cuda()
    lpsi, _, _ = h.amplitudes(Sd)
    acc = torch.zeros(nc, dtype=torch.int64, device="cuda")
    S_ref = S0.copy()
    l_ref = np.array([tn.log_amplitude(th, s, lat, chi)[0] for s in S0])
    logamp = lambda t, s: tn.log_amplitude(t, s, lat, chi)[0]  # noqa: E731
    nacc = 0
    for step in range(4):
        h.sample_learned(prop, Sd, lpsi, seed=777, step=step, accepted=acc)
        for c in range(nc):
            S_ref[c], l_ref[c], a = Q.learned_step(th, w, S_ref[c], l_ref[c], lat, chi, 777, step, c, logamp, C=C)
            nacc += a
    torch.cuda.synchronize()
    assert np.array_equal(Sd.cpu().numpy(), S_ref)
    assert np.max(np.abs(lpsi.cpu().numpy() - l_ref)) < 1e-10
    assert acc.sum().item() == nacc and nacc > 0

"""A whole optimisation step (Metropolis sweeps -> psi, E_loc, O -> MinSR -> parameter update)
captured in one CUDA graph and replayed, against the same calls made eagerly: every call of the
step is asynchronous on the caller's stream (no host round trip inside), so the replayed graph
must reproduce the eager trajectory bit for bit.  Also the asynchronous reporting of a MinSR
breakdown through the handle's status word, and the caller-allocator handle."""
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


def _setup(P, prec, gram, solve, rcond, lam, allocator="torch"):
    lat = I.Lattice(4, 5, 2, 2)
    ns = 64
    th = I.peps_random(lat, 17, scale=0.5, bias=1.0)
    H = I.heisenberg(lat)
    h = P.PEPS(lat.Lx, lat.Ly, 2, lat.D, 3, prec=prec, max_samples=ns, gram=gram, solve=solve, allocator=allocator)
    theta = torch.as_tensor(th).cuda()
    h.set_params(theta)
    S = torch.as_tensor(I.configs_neel(lat, ns)).cuda()
    acc = torch.zeros(ns, dtype=torch.int64, device="cuda")
    O = torch.empty(ns, h.Np, dtype=h.odtype, device="cuda")
    out = {}

    def step():
        h.sample(S, P.MOVE_EXCHANGE, 2, seed=9, sweep0=4, accepted=acc)
        r = h.evaluate(H, S, O_out=O)
        w = h.status_weights(r["status"])
        dth, info = h.minsr_step(r["O"], r["eloc"], w=w, lam=lam, rcond=rcond, tau=0.05)
        h.apply_update(theta, dth)
        out.update(eloc=r["eloc"], logabs=r["logabs"], dth=dth, info=info, w=w)

    return h, theta, S, acc, step, out


@pytest.mark.parametrize("prec,gram,solve,rcond,lam", [
    (0, 0, 0, 0.0, 1e-3),     # FP64 contractions, FP64 Gram, FP64 Cholesky
    (1, 2, 1, 0.0, 1e-3),     # FP32 contractions, float-float Gram, FP32 Cholesky + FP64 refinement
    (1, 0, 0, 1e-8, 1e-4),    # eigendecomposition route (one cooperative Jacobi launch)
])
def test_whole_step_in_a_cuda_graph_matches_eager(P, prec, gram, solve, rcond, lam):
    steps = 3
    # eager: one warm-up step (workspaces, Hamiltonian upload) then `steps` more
    h1, th1, S1, acc1, step1, out1 = _setup(P, prec, gram, solve, rcond, lam)
    for _ in range(1 + steps):
        step1()
    torch.cuda.synchronize()
    # graph: the same warm-up step eagerly, then the step captured once and replayed `steps` times
    h2, th2, S2, acc2, step2, out2 = _setup(P, prec, gram, solve, rcond, lam)
    step2()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        step2()
    for _ in range(steps):
        g.replay()
    torch.cuda.synchronize()
    assert torch.equal(S1, S2)
    assert torch.equal(acc1, acc2)
    assert torch.equal(th1, th2)
    for k in ("eloc", "logabs", "dth", "info", "w"):
        assert torch.equal(torch.nan_to_num(out1[k], nan=-7.0), torch.nan_to_num(out2[k], nan=-7.0)), k
    assert int(acc1.sum()) > 0
    assert float(out1["dth"].abs().max()) > 0.0
    h1.last_status()
    h2.last_status()


def test_minsr_breakdown_is_reported_through_the_status_word(P):
    # lambda far below the rounding of T (split-BF16 Gram of badly scaled O): dtheta is zeroed on
    # the device and the breakdown flag waits in the status word until the caller reads it
    rng = np.random.default_rng(12)
    O = 3e3 * rng.standard_normal((512, 1200)) * (rng.random(1200) < 0.05)
    e = rng.standard_normal(512)
    h = P.PEPS(2, 26, 2, 3, 3, max_samples=2, gram=1)
    Op = np.zeros((512, h.Np))
    Op[:, :1200] = O
    dth, info = h.minsr_step(torch.as_tensor(Op).cuda(), torch.as_tensor(np.stack([e, np.zeros(512)], 1)).cuda(),
                             lam=1e-4, rcond=0.0, tau=0.1)
    word = h.last_status()
    assert word & P.SW_MINSR_BREAKDOWN and h.last_warning is not None
    assert float(info[0]) == -1.0 and bool(torch.all(dth == 0))
    assert h.last_status() == 0  # read and cleared


def test_caller_allocator_and_library_allocator_agree(P):
    # the handle's device memory from PyTorch's caching allocator (peps_create_ex) or from the
    # library's own cudaMalloc (peps_create): the same results
    res = []
    for alloc in ("torch", None):
        h, th, S, acc, step, out = _setup(P, 1, 2, 0, 0.0, 1e-3, allocator=alloc)
        step()
        torch.cuda.synchronize()
        res.append((S.clone(), th.clone(), out["eloc"].clone()))
        h.close()
    assert all(torch.equal(a, b) for a, b in zip(res[0], res[1]))

"""The sample-sharded MinSR pieces of the C library (minsr_partial_sums, minsr_center_rows,
minsr_gram, minsr_solve, minsr_project) on the GPU: the exchange of
paper_2503_12557_gb300.dist carried out in one process over G row blocks (the collectives
replaced by their definitions: sums, concatenations), against the oracle's MinSR on all rows;
and dist.sharded_minsr itself in a one-process NCCL group against minsr_step."""
import os
import socket

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    from paper_2503_12557_gb300 import build, peps
    build.build()
    return peps


def _handle(P, npar, gram=0):
    from paper_2503_12557_gb300 import inputs as I
    for Ly in range(2, 33):
        for D in range(1, 9):
            lat = I.Lattice(2, Ly, 2, D)
            if I.num_params(lat) >= npar:
                return P.PEPS(2, Ly, 2, D, D, max_samples=2, gram=gram)
    raise AssertionError


def _emulated(ops, blocks, lam, rcond, tau):
    from paper_2503_12557_gb300.dist import param_slices
    G = len(blocks)
    Np = blocks[0][0].shape[1]
    sums = sum(ops.partial_sums(O, e, w) for O, e, w in blocks)            # all-reduce
    rows = [ops.center_rows(O, e, w, sums) for O, e, w in blocks]
    c = param_slices(Np, G)
    A = [torch.cat([Ob[:, c[g]:c[g + 1]] for Ob, _ in rows], 0) for g in range(G)]  # all-to-all
    T = sum(ops.gram(A[g]) for g in range(G))                              # all-reduce
    eb = torch.cat([eb for _, eb in rows])                                  # all-gather
    x, info = ops.solve(T, eb, lam, rcond)
    return torch.cat([ops.project(A[g], x, tau) for g in range(G)]), info  # all-gather


@pytest.mark.parametrize("splits,npar,lam,rcond,weighted,gram", [
    ((0, 300, 700), 300, 1e-3, 0.0, True, 0),
    ((0, 100, 250, 333), 500, 1e-4, 1e-9, False, 0),
    ((0, 515, 1030), 1200, 1e-4, 0.0, True, 2),
])
def test_sharded_pieces_vs_oracle(P, splits, npar, lam, rcond, weighted, gram):
    from oracle import minsr
    from paper_2503_12557_gb300.dist import CudaMinSROps
    ns = splits[-1]
    rng = np.random.default_rng(ns + 11)
    O = rng.standard_normal((ns, npar)) + 0.1 * rng.standard_normal(npar)
    e = rng.standard_normal(ns) - 3.0
    w = rng.uniform(0.5, 2.0, ns) if weighted else None
    d_ref, inf_ref = minsr.minsr(O, e, w=w, lam=lam, rcond=rcond, tau=0.1)
    h = _handle(P, npar, gram)
    Op = np.zeros((ns, h.Np))
    Op[:, :npar] = O
    Od = torch.as_tensor(Op).cuda()
    ed = torch.as_tensor(np.stack([e, np.zeros(ns)], 1)).cuda()
    wd = torch.as_tensor(w).cuda() if weighted else None
    blocks = [(Od[a:b].contiguous(), ed[a:b].contiguous(), wd[a:b].contiguous() if weighted else None)
              for a, b in zip(splits[:-1], splits[1:])]
    d, info = _emulated(CudaMinSROps(h), blocks, lam, rcond, 0.1)
    h.last_status()
    d = d.cpu().numpy()[:npar]
    tol = 1e-9 if gram == 0 else 1e-7
    assert np.linalg.norm(d - d_ref) <= tol * np.linalg.norm(d_ref)
    assert int(info[0]) == inf_ref["rank"]
    # the single-process step on all rows gives the same update
    dth, _ = h.minsr_step(Od, ed, w=wd, lam=lam, rcond=rcond, tau=0.1)
    assert np.linalg.norm(dth.cpu().numpy()[:npar] - d) <= tol * np.linalg.norm(d_ref)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_sharded_minsr_in_a_one_process_nccl_group(P):
    import torch.distributed as dist
    from paper_2503_12557_gb300.dist import CudaMinSROps, sharded_minsr
    rng = np.random.default_rng(3)
    h = _handle(P, 800)
    O = torch.as_tensor(rng.standard_normal((400, h.Np))).cuda()
    e = torch.as_tensor(np.stack([rng.standard_normal(400), np.zeros(400)], 1)).cuda()
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(_free_port())
    dist.init_process_group("nccl", rank=0, world_size=1, device_id=torch.device("cuda", torch.cuda.current_device()))
    try:
        d, info = sharded_minsr(CudaMinSROps(h), O, e, None, lam=1e-3, rcond=0.0, tau=0.05)
    finally:
        dist.destroy_process_group()
    ref, _ = h.minsr_step(O, e, lam=1e-3, rcond=0.0, tau=0.05)
    assert torch.allclose(d, ref, rtol=0, atol=1e-12 * float(ref.abs().max()))

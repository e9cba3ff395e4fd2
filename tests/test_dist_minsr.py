"""Sample-sharded MinSR (paper_2503_12557_gb300.dist) on two CPU processes with the gloo backend:
the exchange (global means, all-to-all of Obar's column slices, summed partial Gram, gathered
ebar, replicated solve, gathered dtheta) against the single-process oracle MinSR on all rows.
The processes' local arithmetic here is a plain numpy restatement (the GPU's is the C library's,
tested in test_gpu_dist.py); this test covers the exchange: ragged row counts, ragged parameter
slices, weights, and both solve routes."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


class NumpyOps:
    """The local pieces of the sharded step, written out plainly (Eq. (tdvp_fast) read as in the
    oracle: Obar = sqrt(w / W) (O - m), T = Obar Obar^T, x = (T + lambda)^+ ebar with the
    eigenvalue cutoff rcond * max, dtheta = -tau Obar^T x)."""

    def partial_sums(self, O, eloc, w):
        O = O.numpy()
        wv = np.ones(O.shape[0]) if w is None else w.numpy()
        return torch.as_tensor(np.concatenate([wv @ O, [wv.sum(), wv @ eloc.numpy()[:, 0]]]))

    def center_rows(self, O, eloc, w, g):
        O = O.numpy()
        g = g.numpy()
        Np = O.shape[1]
        W = g[Np]
        wv = np.ones(O.shape[0]) if w is None else w.numpy()
        sw = np.sqrt(wv / W)
        return (torch.as_tensor(sw[:, None] * (O - g[:Np] / W)),
                torch.as_tensor(sw * (eloc.numpy()[:, 0] - g[Np + 1] / W)))

    def gram(self, A):
        A = A.numpy()
        return torch.as_tensor(A @ A.T)

    def solve(self, T, ebar, lam, rcond):
        lmb, V = np.linalg.eigh(T.numpy())
        keep = lmb > rcond * lmb.max() if rcond > 0 else np.ones_like(lmb, dtype=bool)
        f = np.where(keep, 1.0 / (lmb + lam), 0.0)
        x = V @ (f * (V.T @ ebar.numpy()))
        return torch.as_tensor(x), torch.tensor([float(keep.sum()), lmb.min(), lmb.max(), 0.0])

    def project(self, A, x, tau):
        return torch.as_tensor(-tau * (A.numpy().T @ x.numpy()))


def _case(seed):
    rng = np.random.default_rng(seed)
    O = rng.standard_normal((64, 101)) + 0.3 * rng.standard_normal(101)
    e = np.stack([rng.standard_normal(64) - 2.0, np.zeros(64)], 1)
    w = rng.uniform(0.5, 2.0, 64)
    return O, e, w


def _worker(rank, world, port, split, weighted, lam, rcond, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2503_12557_gb300.dist import sharded_minsr
    O, e, w = _case(7)
    lo, hi = split[rank], split[rank + 1]
    d, info = sharded_minsr(NumpyOps(), torch.as_tensor(O[lo:hi]), torch.as_tensor(e[lo:hi]),
                            torch.as_tensor(w[lo:hi]) if weighted else None, lam=lam, rcond=rcond, tau=0.07)
    q.put((rank, d.numpy(), info.numpy()))
    dist.barrier()
    dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("split,weighted,lam,rcond", [
    ((0, 37, 64), True, 1e-3, 0.0),      # ragged rows, weights, all eigenvalues kept
    ((0, 32, 64), False, 0.0, 1e-8),     # the pseudo-inverse cutoff (centring null vector cut)
])
def test_two_process_sharded_minsr_matches_single_process_oracle(split, weighted, lam, rcond):
    from oracle import minsr
    O, e, w = _case(7)
    d_ref, inf_ref = minsr.minsr(O, e[:, 0], w=w if weighted else None, lam=lam, rcond=rcond, tau=0.07)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, split, weighted, lam, rcond, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = dict((r, (d, i)) for r, d, i in (q.get(timeout=120) for _ in procs))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in (0, 1):
        d, info = out[r]
        assert np.linalg.norm(d - d_ref) <= 1e-10 * np.linalg.norm(d_ref), r
        assert int(info[0]) == inf_ref["rank"]
    assert np.array_equal(out[0][0], out[1][0])  # the same dtheta on every process


def test_param_slices_cover_every_parameter_once():
    from paper_2503_12557_gb300.dist import param_slices
    for Np in (1, 7, 101, 21632):
        for G in (1, 2, 3, 8):
            c = param_slices(Np, G)
            assert c[0] == 0 and c[-1] == Np and all(c[i] <= c[i + 1] for i in range(G))
            assert max(c[i + 1] - c[i] for i in range(G)) - min(c[i + 1] - c[i] for i in range(G)) <= 1

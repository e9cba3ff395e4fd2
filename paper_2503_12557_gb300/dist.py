"""Sample-sharded MinSR over several processes (torch.distributed), one GPU per process.

The paper parallelises the sampling over independent samples (Sec. "Finite PEPS and Sampling"):
every process owns its chains, evaluates psi, E_loc and O of its own samples and keeps a copy of
theta.  Only the MinSR step of Eq. (tdvp_fast) couples the samples.  Its exchange, with G
processes, process g holding N_g rows of O and the parameter slice [c_g, c_{g+1}):

  1. the weighted column sums of O, the weight sum and the weighted E_loc sum (all-reduce);
  2. the local rows of Obar and ebar centred with those global means;
  3. Obar from sample-sharded to parameter-sharded (all-to-all): process g gets the
     N_s x K_g block of its slice;
  4. the partial Gram of that block (all-reduce of N_s x N_s);
  5. ebar gathered to every process (all-gather); the same (T + lambda)^+ ebar solved on every
     process;
  6. dtheta on the slice, gathered to every process (all-gather); each applies it to its theta.

The local arithmetic is the C library's (minsr_partial_sums, minsr_center_rows, minsr_gram,
minsr_solve, minsr_project through `CudaMinSROps`); this module only moves buffers between
processes.  The exchange takes an `ops` object so that its bookkeeping (slices, ragged row counts,
padding of the gathers) can be checked on CPU processes with the gloo backend.
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def param_slices(Np: int, G: int):
    """[c_0 = 0, c_1, ..., c_G = Np]: near-equal contiguous parameter slices."""
    return [(Np * g) // G for g in range(G + 1)]


def _all_to_all(recv, send, group=None):
    """recv[h] <- the block process h sends to this one: NCCL's all-to-all, or point-to-point
    pairs on a backend without one (gloo)."""
    if dist.get_backend(group) == "nccl":
        dist.all_to_all(recv, send, group=group)
        return
    G = dist.get_world_size(group)
    me = dist.get_rank(group)
    ops = []
    for h in range(G):
        if h == me:
            recv[h].copy_(send[h])
            continue
        ops.append(dist.P2POp(dist.isend, send[h], h, group))
        ops.append(dist.P2POp(dist.irecv, recv[h], h, group))
    if ops:
        for r in dist.batch_isend_irecv(ops):
            r.wait()


def _all_gather_ragged(x, counts, group=None):
    """Concatenation over the processes of a 1-D tensor whose length differs per process."""
    m = max(counts)
    buf = torch.zeros(m, dtype=x.dtype, device=x.device)
    buf[:x.numel()] = x
    parts = [torch.empty_like(buf) for _ in counts]
    dist.all_gather(parts, buf, group=group)
    return torch.cat([p[:c] for p, c in zip(parts, counts)])


def sharded_minsr(ops, O, eloc, w=None, lam=1e-4, rcond=0.0, tau=0.05, group=None):
    """One MinSR step over the samples of every process; O (N_g x Np), eloc (N_g x 2) and w (N_g or
    None) are this process's rows.  Returns (dtheta (Np), info (4)), the same on every process."""
    G = dist.get_world_size(group)
    me = dist.get_rank(group)
    Np = O.shape[1]
    ng = torch.tensor([O.shape[0]], dtype=torch.int64, device=O.device)
    allc = [torch.zeros_like(ng) for _ in range(G)]
    dist.all_gather(allc, ng, group=group)
    counts = [int(c.item()) for c in allc]
    Ns = sum(counts)
    # 1-2: global means, centred local rows
    sums = ops.partial_sums(O, eloc, w)
    dist.all_reduce(sums, group=group)
    Obar, ebar = ops.center_rows(O, eloc, w, sums)
    # 3: sample-sharded -> parameter-sharded
    c = param_slices(Np, G)
    send = [Obar[:, c[h]:c[h + 1]].contiguous() for h in range(G)]
    recv = [torch.empty(counts[h], c[me + 1] - c[me], dtype=Obar.dtype, device=Obar.device) for h in range(G)]
    _all_to_all(recv, send, group)
    A = torch.cat(recv, 0)
    # 4: partial Gram of this slice, summed
    T = ops.gram(A)
    dist.all_reduce(T, group=group)
    # 5: the replicated solve
    eb = _all_gather_ragged(ebar, counts, group)
    x, info = ops.solve(T, eb, lam, rcond)
    # 6: dtheta on the slice, gathered
    d = ops.project(A, x, tau)
    dtheta = _all_gather_ragged(d, [c[h + 1] - c[h] for h in range(G)], group)
    return dtheta, info


class CudaMinSROps:
    """The local arithmetic of sharded_minsr on the GPU (the C library's MinSR pieces)."""

    def __init__(self, handle):
        self.h = handle

    def partial_sums(self, O, eloc, w):
        return self.h.minsr_partial_sums(O, eloc, w)

    def center_rows(self, O, eloc, w, gsums):
        return self.h.minsr_center_rows(O, eloc, w, gsums)

    def gram(self, A):
        return self.h.minsr_gram(A)

    def solve(self, T, ebar, lam, rcond):
        return self.h.minsr_solve(T, ebar, lam, rcond)

    def project(self, A, x, tau):
        return self.h.minsr_project(A, x, tau)

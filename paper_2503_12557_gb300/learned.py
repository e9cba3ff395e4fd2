"""Host-side schedule of the learned-proposal experiment (driver code; every move, amplitude and
training step runs in the library's kernels).

Chains alternate local single-flip sweeps (peps_sample) with network moves
(peps_sample_learned).  Both kernels are reversible with respect to |psi|^2 on their own, so the
alternation keeps |psi|^2 stationary.  The network is trained on (S_t, S_{t+lag}) pairs taken
from chains that use local moves only, with the binary cross-entropy loss of the proposal.
The gain is measured by the integrated autocorrelation time of a per-chain observable.
"""
from __future__ import annotations

import numpy as np
import torch

from . import peps as P


def tau_int(x, c=5.0):
    """Integrated autocorrelation time of x (T steps x chains), averaged over chains, with
    Sokal's automatic window (smallest W with W >= c tau(W))."""
    x = np.asarray(x, dtype=np.float64)
    x = x - x.mean(axis=0, keepdims=True)
    T = x.shape[0]
    var = np.mean(x * x)
    if var == 0.0:
        return 1.0
    rho = np.array([np.mean(x[: T - t] * x[t:]) / var for t in range(T // 2)])
    tau = 1.0
    for W in range(1, len(rho)):
        tau = 1.0 + 2.0 * np.sum(rho[1:W + 1])
        if W >= c * tau:
            break
    return max(tau, 1.0)


def run_local(h, S, nsteps, seed, sweep0, move=P.MOVE_FLIP, observe=None):
    """nsteps local sweeps; returns (S, list of observations per step, accepted counts)."""
    acc = torch.zeros(S.shape[0], dtype=torch.int64, device=S.device)
    obs = []
    for t in range(nsteps):
        h.sample(S, move, 1, seed=seed, sweep0=sweep0 + t, accepted=acc)
        if observe is not None:
            obs.append(observe(S))
    return S, obs, acc


def collect_pairs(h, S, npairs_steps, lag, seed, sweep0, move=P.MOVE_FLIP):
    """Training pairs (S_t, S_{t+lag}) from local-move chains."""
    ins, outs = [], []
    for k in range(npairs_steps):
        a = S.clone()
        h.sample(S, move, lag, seed=seed, sweep0=sweep0 + k * lag)
        ins.append(a)
        outs.append(S.clone())
    return torch.cat(ins), torch.cat(outs), S


def train(prop, S_in, S_out, steps, lr=3e-3, batch=4096, seed=0):
    g = torch.Generator(device="cpu").manual_seed(seed)
    n = S_in.shape[0]
    losses = []
    for t in range(steps):
        idx = torch.randint(0, n, (min(batch, n),), generator=g).to(S_in.device)
        losses.append(float(prop.train_step(S_in[idx].contiguous(), S_out[idx].contiguous(), lr=lr).item()))
    return losses


def run_mixed(h, prop, S, nsteps, seed, sweep0, move=P.MOVE_FLIP, observe=None):
    """nsteps of (one local sweep + one network move); returns (S, observations, local and
    network acceptance counts)."""
    acc_l = torch.zeros(S.shape[0], dtype=torch.int64, device=S.device)
    acc_n = torch.zeros(S.shape[0], dtype=torch.int64, device=S.device)
    lpsi, _, _ = h.amplitudes(S)
    obs = []
    for t in range(nsteps):
        h.sample(S, move, 1, seed=seed, sweep0=sweep0 + t, accepted=acc_l)
        lpsi, _, _ = h.amplitudes(S)
        h.sample_learned(prop, S, lpsi, seed=seed + 1, step=sweep0 + t, accepted=acc_n)
        if observe is not None:
            obs.append(observe(S))
    return S, obs, acc_l, acc_n

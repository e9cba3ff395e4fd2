"""Learned convolutional proposal for the Metropolis chains (oracle, FP64).

Not in the paper (which samples directly, Sec. "On Direct Sampling"); the component is required
by the hot-path specification, so there is no printed value to pin it to.  It is pinned by
mathematics instead (tests/test_oracle_proposal.py): the convolution against a brute-force loop,
the loss gradient against finite differences, Adam's first step against its closed form, the
network kernel against detailed balance and stationarity of |psi|^2, and the chain step itself
(learned_step: propose, log q both ways, mh_accept) against that exact kernel's rows by a
chi^2 test over many independent moves, with a swapped MH ratio and an inverted draw both
failing it.

Network: x = 1 - 2 s (a +-1 map, 1 channel) -> conv3x3(1 -> C) -> SiLU -> conv3x3(C -> C) -> SiLU
-> conv3x3(C -> 1) -> logits l (Lx x Ly); zero padding at the open boundary; every conv has a bias.
Proposal: q(S'|S) = prod_i Bernoulli(s'_i; sigmoid(l_i(S))), log q = sum_i s'_i l_i - softplus(l_i).
MH: accept with min(1, |psi(S')|^2 q(S|S') / (|psi(S)|^2 q(S'|S))), ratios in FP64 logs.
Training loss: mean over samples and sites of softplus(l_i(S)) - t_i l_i(S) (binary cross-entropy
of the target configuration T given S), minimised with Adam.

Random numbers (Philox4x32-10, key = seed): the proposal's site i of chain c at step k uses
counter (i, k, c, 1); the acceptance uniform uses counter (N, k, c, 1).
"""
from __future__ import annotations

import math

import numpy as np

from paper_2503_12557_gb300.inputs import proposal_shapes
from .philox import uniform53, key_of_seed


def unpack(w, C=16):
    out, o = [], 0
    for shp in proposal_shapes(C):
        n = int(np.prod(shp))
        out.append(w[o:o + n].reshape(shp))
        o += n
    return out


def conv3x3(x, W, b):
    """y[o, i, j] = b[o] + sum_{c, di, dj} W[o, c, di, dj] x[c, i + di - 1, j + dj - 1] (zero padded)."""
    Cin, Lx, Ly = x.shape
    xp = np.zeros((Cin, Lx + 2, Ly + 2), dtype=x.dtype)
    xp[:, 1:-1, 1:-1] = x
    y = np.zeros((W.shape[0], Lx, Ly), dtype=np.result_type(x, W))
    for di in range(3):
        for dj in range(3):
            y += np.einsum("oc,cij->oij", W[:, :, di, dj], xp[:, di:di + Lx, dj:dj + Ly])
    return y + b[:, None, None]


def sigmoid(z):
    return 1.0 / (1.0 + np.exp(-z))


def silu(z):
    return z * sigmoid(z)


def softplus(z):
    return np.logaddexp(0.0, z)


def forward(w, S, Lx, Ly, C=16, keep=False):
    """logits (Lx, Ly) of configuration S (0/1, length Lx*Ly)."""
    W1, b1, W2, b2, W3, b3 = unpack(w, C)
    x = (1.0 - 2.0 * np.asarray(S, dtype=np.float64)).reshape(1, Lx, Ly)
    z1 = conv3x3(x, W1, b1)
    h1 = silu(z1)
    z2 = conv3x3(h1, W2, b2)
    h2 = silu(z2)
    l = conv3x3(h2, W3, b3)[0]
    if keep:
        return l, (x, z1, h1, z2, h2)
    return l


def log_q(l, Sp):
    s = np.asarray(Sp, dtype=np.float64).reshape(l.shape)
    return float(np.sum(s * l - softplus(l)))


def conv3x3_backward(x, W, gy):
    """Gradients of y = conv3x3(x, W, b) given dL/dy: (dL/dx, dL/dW, dL/db)."""
    Cin, Lx, Ly = x.shape
    xp = np.zeros((Cin, Lx + 2, Ly + 2))
    xp[:, 1:-1, 1:-1] = x
    gW = np.zeros_like(W)
    gxp = np.zeros_like(xp)
    for di in range(3):
        for dj in range(3):
            gW[:, :, di, dj] = np.einsum("oij,cij->oc", gy, xp[:, di:di + Lx, dj:dj + Ly])
            gxp[:, di:di + Lx, dj:dj + Ly] += np.einsum("oc,oij->cij", W[:, :, di, dj], gy)
    return gxp[:, 1:-1, 1:-1], gW, gy.sum(axis=(1, 2))


def loss_and_grad(w, S_in, S_tgt, Lx, Ly, C=16):
    """Mean BCE of the targets given the inputs, and its gradient w.r.t. the packed weights."""
    W1, b1, W2, b2, W3, b3 = unpack(w, C)
    grads = [np.zeros_like(p) for p in (W1, b1, W2, b2, W3, b3)]
    n = len(S_in)
    N = Lx * Ly
    loss = 0.0
    for S, Tt in zip(S_in, S_tgt):
        l, (x, z1, h1, z2, h2) = forward(w, S, Lx, Ly, C, keep=True)
        t = np.asarray(Tt, dtype=np.float64).reshape(Lx, Ly)
        loss += float(np.sum(softplus(l) - t * l)) / (n * N)
        gl = (sigmoid(l) - t)[None] / (n * N)
        gh2, gW3, gb3 = conv3x3_backward(h2, W3, gl)
        sz2 = sigmoid(z2)
        gz2 = gh2 * (sz2 * (1.0 + z2 * (1.0 - sz2)))
        gh1, gW2, gb2 = conv3x3_backward(h1, W2, gz2)
        sz1 = sigmoid(z1)
        gz1 = gh1 * (sz1 * (1.0 + z1 * (1.0 - sz1)))
        _, gW1, gb1 = conv3x3_backward(x, W1, gz1)
        for g, d in zip(grads, (gW1, gb1, gW2, gb2, gW3, gb3)):
            g += d
    return loss, np.concatenate([g.ravel() for g in grads])


def adam(w, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (Kingma & Ba); t counts from 1.  Returns new (w, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return w - lr * mh / (np.sqrt(vh) + eps), m, v


def propose(w, S, Lx, Ly, seed, step, chain, C=16):
    """Draw S' ~ q(.|S); returns (S', log q(S'|S))."""
    l = forward(w, S, Lx, Ly, C).ravel()
    key = key_of_seed(seed)
    p = sigmoid(l)
    Sp = np.array([1 if uniform53((i, step, chain, 1), key) < p[i] else 0 for i in range(Lx * Ly)], dtype=np.uint8)
    return Sp, log_q(l.reshape(Lx, Ly), Sp)


def mh_accept(logpsi_new, logpsi_old, lq_fwd, lq_bwd, u):
    """u < |psi'|^2 q(S|S') / (|psi|^2 q(S'|S)), evaluated in logs."""
    if not np.isfinite(logpsi_new):
        return False
    return u < math.exp(min(0.0, 2.0 * (logpsi_new - logpsi_old) + lq_bwd - lq_fwd))


def learned_step(theta, w, S, logpsi, lat, chi, seed, step, chain, logamp, C=16):
    """One network move of one chain.  logamp(theta, S) -> ln|psi(S)|.  Returns (S, logpsi, accepted)."""
    Lx, Ly = lat.Lx, lat.Ly
    Sp, lq_f = propose(w, S, Lx, Ly, seed, step, chain, C)
    lq_b = log_q(forward(w, Sp, Lx, Ly, C), S)
    lnew = logamp(theta, Sp)
    u = uniform53((Lx * Ly, step, chain, 1), key_of_seed(seed))
    if mh_accept(lnew, logpsi, lq_f, lq_b, u):
        return Sp, lnew, True
    return S, logpsi, False


def network_kernel_exact(w, psi, lat, C=16):
    """Full transition matrix of one network move on a tiny lattice with exact amplitudes."""
    from .exact import index_configs
    N = lat.nsites
    Sall = index_configs(N, 2)
    dim = 2 ** N
    p = np.abs(psi) ** 2
    L = np.array([forward(w, s, lat.Lx, lat.Ly, C).ravel() for s in Sall])
    lq = np.array([[np.sum(Sall[b] * L[a] - softplus(L[a])) for b in range(dim)] for a in range(dim)])  # log q(b|a)
    K = np.zeros((dim, dim))
    for a in range(dim):
        for b in range(dim):
            if b == a or p[a] == 0:
                continue
            r = min(1.0, p[b] / p[a] * math.exp(lq[b, a] - lq[a, b]))
            K[a, b] = math.exp(lq[a, b]) * r
        K[a, a] = 1.0 - K[a].sum()
    return K

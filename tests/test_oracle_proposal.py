"""Pins of the learned-proposal oracle (no counterpart in the paper, so parity against the paper
is unpinned): the convolution against a brute-force loop, the loss gradient against central
finite differences, Adam's first step against its closed form, and the network move's exact
transition matrix against detailed balance."""
import math

import numpy as np

from paper_2503_12557_gb300.inputs import Lattice, peps_random, proposal_init, configs_uniform
from oracle import proposal as Q, exact


def test_conv3x3_bruteforce():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((3, 4, 5))
    W = rng.standard_normal((2, 3, 3, 3))
    b = rng.standard_normal(2)
    y = Q.conv3x3(x, W, b)
    ref = np.zeros((2, 4, 5))
    for o in range(2):
        for i in range(4):
            for j in range(5):
                s = b[o]
                for c in range(3):
                    for di in range(3):
                        for dj in range(3):
                            ii, jj = i + di - 1, j + dj - 1
                            if 0 <= ii < 4 and 0 <= jj < 5:
                                s += W[o, c, di, dj] * x[c, ii, jj]
                ref[o, i, j] = s
    assert np.allclose(y, ref, atol=1e-13)


def test_loss_gradient_finite_difference():
    Lx, Ly, C = 3, 4, 4
    w = proposal_init(3, C=C, scale=1.5)
    lat = Lattice(Lx, Ly, 2, 1)
    S_in = configs_uniform(lat, 3, 1)
    S_tg = configs_uniform(lat, 3, 2)
    loss, g = Q.loss_and_grad(w, S_in, S_tg, Lx, Ly, C)
    rng = np.random.default_rng(5)
    h = 1e-6
    for k in rng.choice(len(w), 25, replace=False):
        wp, wm = w.copy(), w.copy()
        wp[k] += h
        wm[k] -= h
        fd = (Q.loss_and_grad(wp, S_in, S_tg, Lx, Ly, C)[0] - Q.loss_and_grad(wm, S_in, S_tg, Lx, Ly, C)[0]) / (2 * h)
        assert abs(fd - g[k]) <= 1e-7 * max(1.0, abs(g[k])) + 1e-9


def test_adam_first_step_closed_form():
    w = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -4.0, 1e-3])
    w1, m, v = Q.adam(w, g, np.zeros(3), np.zeros(3), 1, lr=0.01)
    # bias-corrected first step: m_hat = g, v_hat = g^2 -> w - lr g / (|g| + eps)
    assert np.allclose(w1, w - 0.01 * g / (np.abs(g) + 1e-8), atol=1e-15)


def test_training_lowers_the_loss():
    Lx, Ly, C = 4, 4, 4
    lat = Lattice(Lx, Ly, 2, 1)
    w = proposal_init(4, C=C)
    S = configs_uniform(lat, 8, 1)
    T = S.copy()  # learning the identity map is achievable
    l0 = Q.loss_and_grad(w, S, T, Lx, Ly, C)[0]
    m = np.zeros_like(w)
    v = np.zeros_like(w)
    for t in range(1, 31):
        _, g = Q.loss_and_grad(w, S, T, Lx, Ly, C)
        w, m, v = Q.adam(w, g, m, v, t, lr=0.05)
    assert Q.loss_and_grad(w, S, T, Lx, Ly, C)[0] < 0.7 * l0


def test_network_move_detailed_balance():
    lat = Lattice(3, 3, 2, 2)
    th = peps_random(lat, 5, scale=0.5, bias=1.0)
    psi = exact.state_vector(th, lat)
    p = np.abs(psi) ** 2
    p /= p.sum()
    w = proposal_init(7, C=4, scale=2.0)
    K = Q.network_kernel_exact(w, psi, lat, C=4)
    assert np.allclose(K.sum(1), 1.0, atol=1e-12)
    assert np.min(K) >= -1e-15
    F = p[:, None] * K
    assert np.max(np.abs(F - F.T)) < 1e-14
    assert np.max(np.abs(p @ K - p)) < 1e-13


def test_log_q_is_a_normalised_distribution():
    rng = np.random.default_rng(2)
    l = rng.standard_normal((2, 2))
    tot = 0.0
    for b in range(16):
        s = [(b >> (3 - i)) & 1 for i in range(4)]
        tot += math.exp(Q.log_q(l, s))
    assert abs(tot - 1.0) < 1e-13

"""Pins of the learned-proposal oracle (no counterpart in the paper, so there is no printed
value to pin it to; the pins are mathematical): the convolution against a brute-force loop, the
loss gradient against central finite differences, Adam's first step against its closed form,
the network move's exact transition matrix against detailed balance, and the chain step
(learned_step) against that matrix's rows, with two planted mistakes that must fail."""
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


# ---- the chain step itself (learned_step = propose + log q both ways + mh_accept), not only the
# separately written transition matrix: many independent one-step moves from one state must
# reproduce that state's row of the exact kernel, and two planted mistakes must not

def _tiny_setup():
    lat = Lattice(2, 2, 2, 2)
    th = peps_random(lat, 9, scale=0.8, bias=0.3)
    psi = exact.state_vector(th, lat)
    w = proposal_init(11, C=4, scale=2.0)
    return lat, th, psi, w


def _empirical_row(lat, th, psi, w, a, nchain, step_fn):
    Sall = exact.index_configs(lat.nsites, 2)
    S = Sall[a]
    lpsi = math.log(abs(psi[a]))
    logamp = lambda t, s: math.log(abs(psi[exact.config_index(s, 2)]))  # noqa: E731
    counts = np.zeros(len(Sall))
    for c in range(nchain):
        Sn, _, _ = step_fn(th, w, S.copy(), lpsi, lat, 2, 101, 3, c, logamp, C=4)
        counts[exact.config_index(Sn, 2)] += 1
    return counts


def _chi2(counts, p):
    # Pearson chi^2 over the bins whose expected count is at least 5 (the rest pooled)
    n = counts.sum()
    e = n * p
    big = e >= 5
    obs = np.append(counts[big], counts[~big].sum())
    exp = np.append(e[big], e[~big].sum())
    keep = exp > 0
    obs, exp = obs[keep], exp[keep]
    df = len(obs) - 1
    return float(np.sum((obs - exp) ** 2 / exp)), df


def _chi2_ok(counts, p):
    x2, df = _chi2(counts, p)
    return x2 <= df + 5.0 * math.sqrt(2.0 * df), x2, df


def test_learned_step_reproduces_exact_kernel_rows():
    lat, th, psi, w = _tiny_setup()
    K = Q.network_kernel_exact(w, psi, lat, C=4)
    for a in (3, 6, 12):
        counts = _empirical_row(lat, th, psi, w, a, 3000, Q.learned_step)
        ok, x2, df = _chi2_ok(counts, K[a])
        assert ok, (a, x2, df)


def test_learned_step_planted_mistakes_fail():
    # (i) the forward and backward proposal log-probabilities swapped in the MH ratio;
    # (ii) the proposal's Bernoulli draw inverted (s' = 1 with probability 1 - sigmoid(l)).
    # Each gives a valid-looking chain with the wrong transition probabilities.
    lat, th, psi, w = _tiny_setup()
    K = Q.network_kernel_exact(w, psi, lat, C=4)
    a = 6

    def swapped(theta, w_, S, logpsi, lat_, chi, seed, step, chain, logamp, C=16):
        Sp, lq_f = Q.propose(w_, S, lat_.Lx, lat_.Ly, seed, step, chain, C)
        lq_b = Q.log_q(Q.forward(w_, Sp, lat_.Lx, lat_.Ly, C), S)
        lnew = logamp(theta, Sp)
        u = Q.uniform53((lat_.nsites, step, chain, 1), Q.key_of_seed(seed))
        if Q.mh_accept(lnew, logpsi, lq_b, lq_f, u):  # planted: lq_fwd <-> lq_bwd
            return Sp, lnew, True
        return S, logpsi, False

    def inverted(theta, w_, S, logpsi, lat_, chi, seed, step, chain, logamp, C=16):
        l = Q.forward(w_, S, lat_.Lx, lat_.Ly, C).ravel()
        key = Q.key_of_seed(seed)
        p = Q.sigmoid(l)
        Sp = np.array([1 if Q.uniform53((i, step, chain, 1), key) >= p[i] else 0 for i in range(lat_.nsites)],
                      dtype=np.uint8)  # planted: Bernoulli(1 - p)
        lq_f = Q.log_q(l.reshape(lat_.Lx, lat_.Ly), Sp)
        lq_b = Q.log_q(Q.forward(w_, Sp, lat_.Lx, lat_.Ly, C), S)
        lnew = logamp(theta, Sp)
        u = Q.uniform53((lat_.nsites, step, chain, 1), key)
        if Q.mh_accept(lnew, logpsi, lq_f, lq_b, u):
            return Sp, lnew, True
        return S, logpsi, False

    for fn in (swapped, inverted):
        counts = _empirical_row(lat, th, psi, w, a, 3000, fn)
        ok, x2, df = _chi2_ok(counts, K[a])
        assert not ok, (fn.__name__, x2, df)


def test_mh_accept_boundaries():
    # accept iff u < min(1, exp(2 (ln|psi'| - ln|psi|) + log q(S|S') - log q(S'|S)))
    r = 2 * (0.1 - 0.4) + (-1.0) - (-1.5)  # ln of the ratio: -0.1
    assert Q.mh_accept(0.1, 0.4, -1.5, -1.0, math.exp(r) - 1e-12)
    assert not Q.mh_accept(0.1, 0.4, -1.5, -1.0, math.exp(r) + 1e-12)
    assert not Q.mh_accept(0.1, 0.4, -1.0, -1.5, math.exp(r) - 1e-12)  # the swapped order rejects
    assert Q.mh_accept(5.0, 0.0, 0.0, 0.0, 0.999999)  # ratio above 1: always accepted
    assert not Q.mh_accept(float("-inf"), 0.0, 0.0, 0.0, 0.0)  # psi' = 0
    assert not Q.mh_accept(float("nan"), 0.0, 0.0, 0.0, 0.0)

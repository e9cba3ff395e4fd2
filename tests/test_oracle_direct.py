"""Pins of the oracle's direct sampler (oracle/direct.py).

* With exact contractions (chi and chi_d at the exact rank) the sequential conditionals
  multiply to the Born probability |psi(S)|^2 / <psi|psi> of every configuration of a 3 x 3
  lattice, for real and complex PEPS (psi from the exact state vector): a wrong index, a
  dropped conjugate or a mis-traced leg breaks it.
* With truncated environments p(S) is still a probability distribution over all
  configurations (the conditionals are normalised) and differs from the Born one.
* A drawn configuration's log p equals the evaluated log p of the same configuration, and
  the draw frequencies on a 2 x 2 lattice follow p within statistical error.
"""
import math

import numpy as np
import pytest

from paper_2503_12557_gb300 import inputs as I
from oracle import direct, exact, tn


def _all_logp(th, lat, chi, chi_d):
    T = I.theta_to_tensors(lat, th)
    Dl = direct.lower_double_envs(T, lat, chi_d)
    allS = exact.index_configs(lat.nsites, lat.d)
    lp = np.array([direct.walk(th, lat, chi, chi_d, S=S, Dl=Dl)[1] for S in allS])
    return allS, lp


@pytest.mark.parametrize("cplx", [False, True])
def test_exact_contraction_gives_born_probabilities(cplx):
    lat = I.Lattice(3, 3, 2, 2)
    th = I.peps_random(lat, 31, scale=0.6, bias=0.5, complex_=cplx)
    _, lp = _all_logp(th, lat, 4, 4)
    psi = exact.state_vector(th, lat)
    born = np.abs(psi) ** 2 / np.sum(np.abs(psi) ** 2)
    p = np.exp(lp)
    assert abs(np.sum(p) - 1.0) < 1e-12
    assert np.max(np.abs(p - born)) <= 1e-11 * np.max(born)


def test_truncated_sampler_is_normalised_and_approximate():
    lat = I.Lattice(3, 3, 2, 3)                      # chi = chi_d = 2 truncate (ranks up to 3 and 9)
    th = I.peps_random(lat, 33, scale=0.6, bias=1.0)
    _, lp = _all_logp(th, lat, 2, 2)
    p = np.exp(lp)
    assert abs(np.sum(p) - 1.0) < 1e-12
    psi = exact.state_vector(th, lat)
    born = np.abs(psi) ** 2 / np.sum(np.abs(psi) ** 2)
    assert np.max(np.abs(p - born)) > 1e-6 * np.max(born)      # the truncation matters here
    assert np.sum(np.abs(p - born)) < 0.5                      # and p stays close to Born


def test_drawn_logp_equals_evaluated_logp():
    lat = I.Lattice(4, 3, 2, 2)
    th = I.peps_random(lat, 35, scale=0.5, bias=1.0)
    S, lp, st = direct.sample(th, lat, 3, 3, 12, seed=9, draw=4)
    T = I.theta_to_tensors(lat, th)
    Dl = direct.lower_double_envs(T, lat, 3)
    for s, l in zip(S, lp):
        _, l2, _ = direct.walk(th, lat, 3, 3, S=s, Dl=Dl)
        assert abs(l - l2) < 1e-12
    assert len({tuple(s) for s in S}) > 3                      # different chains draw differently
    S2, lp2, _ = direct.sample(th, lat, 3, 3, 12, seed=9, draw=4)
    assert np.array_equal(S, S2) and np.array_equal(lp, lp2)   # counter-based: reproducible


def test_draw_frequencies_follow_p():
    lat = I.Lattice(2, 2, 2, 2)
    th = I.peps_random(lat, 37, scale=0.8, bias=0.5)
    allS, lp = _all_logp(th, lat, 4, 4)
    p = np.exp(lp)
    n = 3000
    S, _, _ = direct.sample(th, lat, 4, 4, n, seed=11)
    idx = np.array([exact.config_index(s, 2) for s in S])
    freq = np.bincount(idx, minlength=16) / n
    sig = np.sqrt(p * (1 - p) / n)
    assert np.all(np.abs(freq - p) <= 5 * sig + 1e-12)

"""Direct sampling through the C ABI (peps_direct_prepare, peps_direct_sample) against the FP64
oracle: the drawn configurations are identical and log p(S) agrees (real and complex PEPS,
truncated single- and double-layer environments, the 8 x 8 D = 4 chi = 16 shape), log p is
the Born probability at exact contraction, and importance-weighted samples reproduce the exact
energy when the double-layer environments are truncated."""
import numpy as np
import pytest
import torch

from paper_2503_12557_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2503_12557_gb300 import build, peps
    build.build()
    return peps


def _draw(P, lat, chi, chid, th, ns, seed, draw, prec=0, cplx=False):
    h = P.PEPS(lat.Lx, lat.Ly, lat.d, lat.D, chi, prec=prec, max_samples=ns, cplx=cplx)
    h.set_params(torch.as_tensor(th).cuda())
    h.direct_prepare(chid)
    S, lp, st = h.direct_sample(ns, seed=seed, draw=draw)
    torch.cuda.synchronize()
    return h, S.cpu().numpy(), lp.cpu().numpy(), st.cpu().numpy()


@pytest.mark.parametrize("Lx,Ly,D,chi,chid,cplx,seed", [
    (4, 4, 2, 3, 2, False, 1),     # both environments truncated
    (3, 5, 3, 4, 3, False, 2),     # D = 3, ragged Ly
    (4, 3, 2, 3, 2, True, 3),      # complex PEPS
])
def test_direct_samples_match_oracle(P, Lx, Ly, D, chi, chid, cplx, seed):
    from oracle import direct
    lat = I.Lattice(Lx, Ly, 2, D)
    th = I.peps_random(lat, 80 + seed, scale=0.6, bias=1.0, complex_=cplx)
    _, S, lp, st = _draw(P, lat, chi, chid, th, 24, seed=seed, draw=5, cplx=cplx)
    Sr, lpr, str_ = direct.sample(th, lat, chi, chid, 24, seed=seed, draw=5)
    assert np.array_equal(S, Sr)
    assert np.max(np.abs(lp - lpr)) <= 1e-10
    assert np.array_equal(st & 2, str_ & 2)
    assert len({tuple(s) for s in S}) > 4


def test_direct_logp_is_born_at_exact_contraction(P):
    from oracle import exact
    lat = I.Lattice(3, 3, 2, 2)
    th = I.peps_random(lat, 91, scale=0.6, bias=0.5)
    _, S, lp, _ = _draw(P, lat, 4, 4, th, 64, seed=7, draw=0)
    psi = exact.state_vector(th, lat)
    born = np.abs(psi) ** 2 / np.sum(np.abs(psi) ** 2)
    idx = [exact.config_index(s, 2) for s in S]
    assert np.max(np.abs(lp - np.log(born[idx]))) <= 1e-10


def test_direct_compiled_shape_8x8(P):
    from oracle import direct
    lat = I.Lattice(8, 8, 2, 4)
    th = I.peps_random(lat, 93, scale=0.5, bias=1.0)
    _, S, lp, _ = _draw(P, lat, 16, 4, th, 2, seed=11, draw=1)
    Sr, lpr, _ = direct.sample(th, lat, 16, 4, 2, seed=11, draw=1)
    assert np.array_equal(S, Sr)
    assert np.max(np.abs(lp - lpr)) <= 1e-9 * max(1.0, np.max(np.abs(lpr)))


def test_direct_fp32_close(P):
    from oracle import direct
    lat = I.Lattice(4, 4, 2, 2)
    th = I.peps_random(lat, 95, scale=0.6, bias=1.0)
    _, S, lp, _ = _draw(P, lat, 3, 2, th, 32, seed=13, draw=2, prec=1)
    Sr, lpr, _ = direct.sample(th, lat, 3, 2, 32, seed=13, draw=2)
    same = np.all(S == Sr, axis=1)
    print(f"fp32 direct sampling: {same.sum()} of {len(S)} configurations identical, "
          f"|d log p| max {np.max(np.abs(lp - lpr)[same]):.2e}")
    assert same.sum() >= 0.9 * len(S)
    assert np.max(np.abs(lp - lpr)[same]) < 1e-4


def test_importance_weights_recover_the_exact_energy(P):
    # samples from truncated double-layer environments (p differs from Born), weights
    # |psi|^2 / p with psi and E_loc at exact chi: the weighted mean is the exact energy
    from oracle import exact
    lat = I.Lattice(4, 4, 2, 2)
    th = I.peps_random(lat, 97, scale=0.6, bias=1.0)
    H = I.heisenberg(lat)
    ns = 4096
    h, S, lp, st = _draw(P, lat, 4, 1, th, ns, seed=17, draw=0)
    r = h.evaluate(H, torch.as_tensor(S).cuda(), want_O=False)
    torch.cuda.synchronize()
    la = r["logabs"].cpu().numpy()
    e = r["eloc"].cpu().numpy()[:, 0]
    lw = 2 * la - lp
    w = np.exp(lw - lw.max())
    w /= w.sum()
    est = float(np.sum(w * e))
    ess = 1.0 / np.sum(w ** 2)
    err = float(np.sqrt(np.sum(w ** 2 * (e - est) ** 2)))
    psi = exact.state_vector(th, lat)
    e_ex = exact.exact_energy(psi, exact.hamiltonian_sparse(H, lat)).real
    born = np.abs(psi) ** 2 / np.sum(np.abs(psi) ** 2)
    idx = [exact.config_index(s, 2) for s in S]
    print(f"importance-weighted E {est:.5f} +- {err:.5f} (ESS {ess:.0f} of {ns}), exact {e_ex:.5f}; "
          f"max |log p - log Born| {np.max(np.abs(lp - np.log(born[idx]))):.3f}")
    assert np.max(np.abs(lp - np.log(born[idx]))) > 1e-3         # chi_d = 1 is a real approximation
    assert abs(est - e_ex) <= 5 * err
    assert ess > 0.1 * ns


def test_direct_errors(P):
    lat = I.Lattice(4, 4, 2, 2)
    h = P.PEPS(4, 4, 2, 2, 3, max_samples=4)
    h.set_params(torch.as_tensor(I.peps_random(lat, 1)).cuda())
    with pytest.raises(RuntimeError):
        h.direct_sample(2)            # no double-layer environments yet
    with pytest.raises(RuntimeError):
        h.direct_prepare(0)


def test_direct_with_truncated_weight_cutoff(P):
    # the upper environments of the drawn rows under the truncated-weight rule (dynamic chi)
    from oracle import direct
    lat = I.Lattice(4, 5, 2, 2)
    th = I.peps_random(lat, 99, scale=0.6, bias=1.0)
    h = P.PEPS(4, 5, 2, 2, 4, max_samples=16, trunc_weight=2e-3)
    h.set_params(torch.as_tensor(th).cuda())
    h.direct_prepare(3)
    S, lp, _ = h.direct_sample(16, seed=21, draw=3)
    torch.cuda.synchronize()
    Sr, lpr, _ = direct.sample(th, lat, (4, 2e-3), 3, 16, seed=21, draw=3)
    assert np.array_equal(S.cpu().numpy(), Sr)
    assert np.max(np.abs(lp.cpu().numpy() - lpr)) <= 1e-10


def test_direct_complex64(P):
    from oracle import direct
    lat = I.Lattice(4, 3, 2, 2)
    th = I.peps_random(lat, 101, scale=0.6, bias=1.0, complex_=True)
    _, S, lp, _ = _draw(P, lat, 3, 2, th, 24, seed=5, draw=1, prec=1, cplx=True)
    Sr, lpr, _ = direct.sample(th, lat, 3, 2, 24, seed=5, draw=1)
    same = np.all(S == Sr, axis=1)
    assert same.sum() >= 0.9 * len(S)
    assert np.max(np.abs(lp - lpr)[same]) < 1e-4


def test_direct_empty_batch(P):
    lat = I.Lattice(4, 4, 2, 2)
    h = P.PEPS(4, 4, 2, 2, 3, max_samples=4)
    h.set_params(torch.as_tensor(I.peps_random(lat, 1)).cuda())
    h.direct_prepare(2)
    S, lp, st = h.direct_sample(0)
    torch.cuda.synchronize()
    assert S.shape == (0, 16) and lp.numel() == 0

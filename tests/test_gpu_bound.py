"""The variational-bound estimator through the C ABI (peps_local_energy_bound) against the FP64
oracle: E_loc^bound with every amplitude taken at one cut, ln|psi_i| and its phase, for real
and complex PEPS, one- and two-row terms, every cut, the compiled (chi, D) = (16, 4) shape and
FP32; at exact chi it equals the fast estimator."""
import numpy as np
import pytest
import torch

from paper_2503_12557_gb300 import inputs as I

pytestmark = pytest.mark.gpu
TOL = 1e-10


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2503_12557_gb300 import build, peps
    build.build()
    return peps


def _run(P, lat, chi, th, S, H, cut, prec=0, cplx=False):
    h = P.PEPS(lat.Lx, lat.Ly, lat.d, lat.D, chi, prec=prec, max_samples=len(S), cplx=cplx)
    h.set_params(torch.as_tensor(th).cuda())
    r = h.local_energy_bound(H, torch.as_tensor(S).cuda(), cut)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in r.items()}


def _compare(res, ref, tol=TOL):
    ok = ((res["status"] & 1) == 0) & ((ref["status"] & 1) == 0)
    assert ok.sum() >= max(1, int(0.75 * len(ok)))
    assert np.max(np.abs(res["logabs"] - ref["logabs"])[ok]) <= tol
    dph = np.angle(np.exp(1j * (res["phase"] - ref["phase"])))
    assert np.max(np.abs(dph)[ok]) <= 10 * tol
    e = res["eloc"][:, 0] + 1j * res["eloc"][:, 1]
    de = np.abs(e - ref["eloc"]) / np.maximum(1.0, np.abs(ref["eloc"]))
    assert np.max(de[ok]) <= tol, np.max(de)


@pytest.mark.parametrize("cut", [1, 2, 3])
def test_bound_heisenberg_every_cut(P, cut):
    from oracle import bound
    lat = I.Lattice(4, 4, 2, 2)
    th = I.peps_random(lat, 51, scale=0.5, bias=1.0)
    S = I.configs_uniform_sz0(lat, 10, 52)
    H = I.heisenberg(lat)
    res = _run(P, lat, 3, th, S, H, cut)
    _compare(res, bound.evaluate_bound(th, S, lat, 3, H, cut))


def test_bound_two_row_terms_and_ragged_shape(P):
    # J1-J2: diagonal bonds over two rows, some of them across the cut; 5 x 4, D = 3, chi = 5
    from oracle import bound
    lat = I.Lattice(5, 4, 2, 3)
    th = I.peps_random(lat, 53, scale=0.5, bias=1.0)
    S = I.configs_uniform_sz0(lat, 8, 54)
    H = I.j1j2_chiral(lat, J1=1.0, J2=0.5, Jchi=0.0)
    H["terms"] = [t for t in H["terms"] if len(t[0]) == 2]
    res = _run(P, lat, 5, th, S, H, 2)
    _compare(res, bound.evaluate_bound(th, S, lat, 5, H, 2))


def test_bound_complex_chiral(P):
    from oracle import bound
    lat = I.Lattice(4, 4, 2, 2)
    th = I.peps_random(lat, 55, scale=0.6, bias=1.0, complex_=True)
    S = I.configs_uniform_sz0(lat, 8, 56)
    H = I.j1j2_chiral(lat)
    res = _run(P, lat, 3, th, S, H, 2, cplx=True)
    ref = bound.evaluate_bound(th, S, lat, 3, H, 2)
    assert np.max(np.abs(ref["eloc"].imag)) > 1e-3
    _compare(res, ref)


def test_bound_rydberg_flips(P):
    # one-site sigma^x terms (flips) and long-range diagonal pairs
    from oracle import bound
    lat = I.Lattice(4, 5, 2, 2)
    th = I.peps_random(lat, 57, scale=0.5, bias=1.0)
    S = I.configs_uniform(lat, 8, 58)
    H = I.rydberg(lat, delta=1.5)
    res = _run(P, lat, 4, th, S, H, 2)
    _compare(res, bound.evaluate_bound(th, S, lat, 4, H, 2))


def test_bound_compiled_shape_8x8_chi16(P):
    # the (chi, D) = (16, 4) specialisation of the bench workload, two samples
    from oracle import bound
    lat = I.Lattice(8, 8, 2, 4)
    th = I.peps_random(lat, 59, scale=0.5, bias=1.0)
    S = I.configs_uniform_sz0(lat, 2, 60)
    H = I.heisenberg(lat)
    res = _run(P, lat, 16, th, S, H, 4)
    _compare(res, bound.evaluate_bound(th, S, lat, 16, H, 4), tol=1e-9)


def test_bound_fp32_close(P):
    from oracle import bound
    lat = I.Lattice(5, 5, 2, 3)
    th = I.peps_random(lat, 61, scale=0.5, bias=1.0)
    S = I.configs_uniform_sz0(lat, 8, 62)
    H = I.heisenberg(lat)
    res = _run(P, lat, 9, th, S, H, 2, prec=1)
    ref = bound.evaluate_bound(th, S, lat, 9, H, 2)
    dl = np.abs(res["logabs"] - ref["logabs"])
    print(f"fp32 bound |d ln psi_i| max {dl.max():.2e}")
    assert dl.max() <= 1e-5
    e = res["eloc"][:, 0]
    assert abs(np.mean(e) - np.mean(ref["eloc"].real)) / lat.nsites < 1e-4


def test_bound_equals_fast_estimator_at_exact_chi(P):
    # chi = D^(Ly/2) is exact for every cut: both estimators give the exact local energy
    lat = I.Lattice(4, 4, 2, 2)
    th = I.peps_random(lat, 63, scale=0.5, bias=1.0)
    S = torch.as_tensor(I.configs_uniform_sz0(lat, 12, 64)).cuda()
    H = I.heisenberg(lat)
    h = P.PEPS(4, 4, 2, 2, 4, max_samples=12)
    h.set_params(torch.as_tensor(th).cuda())
    fast = h.evaluate(H, S, want_O=False)
    for cut in (1, 2, 3):
        b = h.local_energy_bound(H, S, cut)
        torch.cuda.synchronize()
        e0, e1 = fast["eloc"].cpu().numpy()[:, 0], b["eloc"].cpu().numpy()[:, 0]
        assert np.max(np.abs(e0 - e1) / np.maximum(1.0, np.abs(e0))) < 1e-10
        assert np.max(np.abs(fast["logabs"].cpu().numpy() - b["logabs"].cpu().numpy())) < 1e-10


def test_bound_rejects_bad_cut(P):
    lat = I.Lattice(4, 4, 2, 2)
    h = P.PEPS(4, 4, 2, 2, 3, max_samples=2)
    S = torch.as_tensor(I.configs_uniform_sz0(lat, 2, 1)).cuda()
    for cut in (0, 4):
        with pytest.raises(RuntimeError):
            h.local_energy_bound(I.heisenberg(lat), S, cut)


def test_contraction_error_vs_oracle(P):
    # Delta psi(D_c, D_c^max) = 1 - psi(D_c) / psi(D_c^max), the paper's relative contraction error
    from oracle import tn
    from paper_2503_12557_gb300 import estimators
    lat = I.Lattice(5, 6, 2, 3)
    th = I.peps_random(lat, 65, scale=0.5, bias=1.0)
    S = I.configs_uniform_sz0(lat, 10, 66)
    hs, hl = P.PEPS(5, 6, 2, 3, 3, max_samples=10), P.PEPS(5, 6, 2, 3, 12, max_samples=10)
    for h in (hs, hl):
        h.set_params(torch.as_tensor(th).cuda())
    dpsi, st = estimators.contraction_error(hs, hl, torch.as_tensor(S).cuda())
    torch.cuda.synchronize()
    ref = []
    for s in S:
        a = tn.log_amplitude(th, s, lat, 3)
        b = tn.log_amplitude(th, s, lat, 12)
        ref.append(1.0 - np.exp(a[0] - b[0]) * np.exp(1j * (a[1] - b[1])))
    ref = np.array(ref)
    ok = (st.cpu().numpy() & 1) == 0
    assert np.max(np.abs(dpsi.cpu().numpy() - ref)[ok]) <= 1e-9
    assert np.max(np.abs(ref)) > 1e-6      # chi = 3 is a real truncation here


def test_bound_with_truncated_weight_cutoff(P):
    from oracle import bound
    lat = I.Lattice(5, 4, 2, 3)
    th = I.peps_random(lat, 67, scale=0.5, bias=1.0)
    S = I.configs_uniform_sz0(lat, 8, 68)
    H = I.heisenberg(lat)
    h = P.PEPS(5, 4, 2, 3, 7, max_samples=8, trunc_weight=2e-3)
    h.set_params(torch.as_tensor(th).cuda())
    r = h.local_energy_bound(H, torch.as_tensor(S).cuda(), 2)
    torch.cuda.synchronize()
    res = {k: v.cpu().numpy() for k, v in r.items()}
    _compare(res, bound.evaluate_bound(th, S, lat, (7, 2e-3), H, 2))


def test_bound_complex64(P):
    from oracle import bound
    lat = I.Lattice(4, 4, 2, 2)
    th = I.peps_random(lat, 69, scale=0.6, bias=1.0, complex_=True)
    S = I.configs_uniform_sz0(lat, 8, 70)
    H = I.j1j2_chiral(lat)
    res = _run(P, lat, 3, th, S, H, 2, prec=1, cplx=True)
    ref = bound.evaluate_bound(th, S, lat, 3, H, 2)
    print(f"complex64 bound |d ln psi_i| max {np.max(np.abs(res['logabs'] - ref['logabs'])):.2e}")
    assert np.max(np.abs(res["logabs"] - ref["logabs"])) <= 1e-5
    e = res["eloc"][:, 0] + 1j * res["eloc"][:, 1]
    assert np.max(np.abs(e - ref["eloc"]) / np.maximum(1.0, np.abs(ref["eloc"]))) < 1e-3


def test_bound_empty_batch(P):
    lat = I.Lattice(4, 4, 2, 2)
    h = P.PEPS(4, 4, 2, 2, 3, max_samples=4)
    h.set_params(torch.as_tensor(I.peps_random(lat, 1)).cuda())
    r = h.local_energy_bound(I.heisenberg(lat), torch.zeros(0, 16, dtype=torch.uint8).cuda(), 2)
    torch.cuda.synchronize()
    assert r["eloc"].shape == (0, 2)

"""Complex PEPS through the C ABI (peps_config.cplx = 1) against the FP64 oracle: ln|psi|, the
phase of psi, E_loc of the J1-J2-chiral model (complex three-spin terms), the holomorphic
log-derivatives O, the MinSR step with T = Obar Obar^H (Cholesky and cutoff routes), and
Metropolis chains; complex64 against the reduced-precision gate."""
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


def _handle(P, lat, chi, ns, prec=0):
    return P.PEPS(lat.Lx, lat.Ly, lat.d, lat.D, chi, prec=prec, max_samples=max(ns, 1), cplx=True)


def _theta(lat, seed):
    return I.peps_random(lat, seed, scale=0.6, bias=1.0, complex_=True)


@pytest.mark.parametrize("Lx,Ly,D,chi,ns,seed", [
    (3, 3, 2, 4, 20, 1),     # exact chi
    (4, 4, 2, 3, 16, 2),     # truncating
    (4, 5, 3, 5, 10, 3),     # truncating, D = 3
])
def test_complex_evaluate_vs_oracle(P, Lx, Ly, D, chi, ns, seed):
    from oracle import energy
    lat = I.Lattice(Lx, Ly, 2, D)
    th = _theta(lat, seed)
    S = I.configs_uniform_sz0(lat, ns, seed + 10)
    H = I.j1j2_chiral(lat)
    h = _handle(P, lat, chi, ns)
    h.set_params(torch.as_tensor(th).cuda())
    res = h.evaluate(H, torch.as_tensor(S).cuda())
    torch.cuda.synchronize()
    ref = energy.evaluate(th, S, lat, chi, H=H, want_O=True)
    st = res["status"].cpu().numpy()
    ok = (st & 1) == 0
    assert ok.sum() >= max(1, int(0.8 * ns))
    la, ph = res["logabs"].cpu().numpy(), res["phase"].cpu().numpy()
    assert np.max(np.abs(la - ref["logabs"])[ok]) <= TOL
    dph = np.angle(np.exp(1j * (ph - ref["phase"])))
    assert np.max(np.abs(dph)[ok]) <= 1e-9
    el = res["eloc"].cpu().numpy()
    de = np.abs(el[:, 0] + 1j * el[:, 1] - ref["eloc"]) / np.maximum(1.0, np.abs(ref["eloc"]))
    assert np.max(de[ok]) <= TOL, np.max(de)
    assert np.max(np.abs(ref["eloc"].imag)) > 1e-3  # the chiral term makes E_loc complex
    O = res["O"].cpu().numpy()
    assert O.dtype == np.complex128
    scale = np.maximum(1.0, np.max(np.abs(ref["O"]), axis=1))
    dO = np.max(np.abs(O - ref["O"]), axis=1) / scale
    assert np.max(dO[ok]) <= TOL, np.max(dO)


@pytest.mark.parametrize("Lx,Ly,D,chi,ns,seed", [(3, 3, 2, 4, 16, 31), (4, 4, 2, 3, 12, 32)])
def test_csl_model_vs_oracle(P, Lx, Ly, D, chi, ns, seed):
    # the chiral-spin-liquid model of Eq. (CSL_Model): four-site plaquette ring terms
    # i lam (P - P^-1) over two rows and two columns, next to J1 and J2 bonds
    from oracle import energy
    lat = I.Lattice(Lx, Ly, 2, D)
    th = _theta(lat, seed)
    S = I.configs_uniform_sz0(lat, ns, seed + 10)
    H = I.csl(lat)
    h = _handle(P, lat, chi, ns)
    h.set_params(torch.as_tensor(th).cuda())
    res = h.evaluate(H, torch.as_tensor(S).cuda(), want_O=False)
    torch.cuda.synchronize()
    ref = energy.evaluate(th, S, lat, chi, H=H, want_O=False)
    ok = (res["status"].cpu().numpy() & 1) == 0
    el = res["eloc"].cpu().numpy()
    de = np.abs(el[:, 0] + 1j * el[:, 1] - ref["eloc"]) / np.maximum(1.0, np.abs(ref["eloc"]))
    assert ok.sum() >= max(1, int(0.8 * ns))
    assert np.max(de[ok]) <= TOL, np.max(de)


def test_complex64_reduced_precision(P):
    from oracle import energy
    lat = I.Lattice(5, 5, 2, 3)
    th = _theta(lat, 7)
    S = I.configs_uniform_sz0(lat, 24, 8)
    H = I.j1j2_chiral(lat)
    h = _handle(P, lat, 9, 24, prec=1)
    h.set_params(torch.as_tensor(th).cuda())
    res = h.evaluate(H, torch.as_tensor(S).cuda())
    torch.cuda.synchronize()
    ref = energy.evaluate(th, S, lat, 9, H=H, want_O=False)
    dl = np.abs(res["logabs"].cpu().numpy() - ref["logabs"])
    print(f"complex64 |d ln psi| max {dl.max():.2e} median {np.median(dl):.2e}")
    assert dl.max() <= 1e-5
    el = res["eloc"].cpu().numpy()
    e = el[:, 0] + 1j * el[:, 1]
    assert abs(np.mean(e) - np.mean(ref["eloc"])) / lat.nsites < 1e-4
    assert res["O"].dtype == torch.complex64


@pytest.mark.parametrize("lam,rc", [(1e-3, 0.0), (0.0, 1e-8), (1e-3, 1e-10)])
def test_complex_minsr_vs_oracle(P, lam, rc):
    from oracle import energy, minsr
    lat = I.Lattice(3, 3, 2, 2)
    th = _theta(lat, 4)
    S = I.configs_uniform_sz0(lat, 48, 5)
    H = I.j1j2_chiral(lat)
    ref = energy.evaluate(th, S, lat, 4, H=H, want_O=True)
    h = _handle(P, lat, 4, len(S))
    Od = torch.as_tensor(ref["O"]).cuda()
    ed = torch.as_tensor(np.stack([ref["eloc"].real, ref["eloc"].imag], 1)).cuda()
    dth, info = h.minsr_step(Od, ed, lam=lam, rcond=rc, tau=0.07)
    torch.cuda.synchronize()
    d_ref, inf_ref = minsr.minsr(ref["O"], ref["eloc"], lam=lam, rcond=rc, tau=0.07)
    d = dth.cpu().numpy()
    assert d.dtype == np.complex128
    assert np.linalg.norm(d - d_ref) <= 1e-9 * np.linalg.norm(d_ref)
    assert int(info[0].item()) == inf_ref["rank"]
    # the update path: theta += dtheta on the device
    thd = torch.as_tensor(th).cuda()
    h.apply_update(thd, dth)
    torch.cuda.synchronize()
    assert np.allclose(thd.cpu().numpy(), th + d, rtol=0, atol=1e-15)


def test_complex_sampler_chains_match_oracle(P):
    from oracle import sampler
    lat = I.Lattice(4, 4, 2, 2)
    th = _theta(lat, 9)
    S0 = I.configs_neel(lat, 6)
    h = _handle(P, lat, 3, 6)
    h.set_params(torch.as_tensor(th).cuda())
    Sd, acc, st = h.sample(torch.as_tensor(S0).cuda(), move=P.MOVE_EXCHANGE, nsweeps=3, seed=77, sweep0=2)
    torch.cuda.synchronize()
    Sref, acc_ref, _ = sampler.run_chains(th, S0, lat, 3, "exchange", 77, 3, sweep0=2)
    assert np.array_equal(Sd.cpu().numpy(), Sref)
    assert np.array_equal(acc.cpu().numpy(), acc_ref)
    assert acc_ref.sum() > 0


def test_complex_unsupported_options(P):
    with pytest.raises(RuntimeError):
        P.PEPS(3, 3, 2, 2, 4, gram=1, cplx=True)

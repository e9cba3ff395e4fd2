"""peps_amplitudes_noalloc, the entry point for callers that cannot allocate device memory
(it keeps every intermediate in a fixed 32 MiB device array), checked through the C ABI
against the handle-based peps_amplitudes on two calls in a row.  This file is collected last
so that a stop-at-first-failure run has already run every other test."""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_2503_12557_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _noalloc_fn():
    from paper_2503_12557_gb300 import build, peps
    build.build()
    lib = peps.load()
    f = lib.peps_amplitudes_noalloc
    vp = C.c_void_p
    f.argtypes = [C.POINTER(peps._Config), vp, vp, C.c_int, vp, vp, vp, vp]
    f.restype = C.c_int
    return peps, f


def _call(peps, f, lat, chi, prec, theta, S):
    ns = S.shape[0]
    la = torch.empty(ns, dtype=torch.float64, device="cuda")
    ph = torch.empty(ns, dtype=torch.float64, device="cuda")
    st = torch.empty(ns, dtype=torch.int32, device="cuda")
    cfg = peps._Config(lat.Lx, lat.Ly, lat.d, lat.D, chi, prec, 0)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = f(C.byref(cfg), C.c_void_p(theta.data_ptr()), C.c_void_p(S.data_ptr()), ns, C.c_void_p(la.data_ptr()),
           C.c_void_p(ph.data_ptr()), C.c_void_p(st.data_ptr()), stream)
    return rc, la, ph, st


@pytest.mark.parametrize("prec,tol", [(0, 1e-10), (1, 1e-5)])
def test_noalloc_matches_handle_entry_point_twice(prec, tol):
    peps, f = _noalloc_fn()
    lat = I.Lattice(4, 4, 2, 2)
    chi = 3
    theta = torch.as_tensor(I.peps_random(lat, 1001, scale=0.5, bias=1.0)).cuda()
    h = peps.PEPS(lat.Lx, lat.Ly, lat.d, lat.D, chi, prec=prec, max_samples=64)
    h.set_params(theta)
    for call, seed in enumerate((2001, 2002)):
        S = torch.as_tensor(I.configs_uniform_sz0(lat, 64, seed)).cuda()
        rc, la, ph, st = _call(peps, f, lat, chi, prec, theta, S)
        assert rc == 0, f"call {call}: status {rc}"
        la_ref, ph_ref, st_ref = h.amplitudes(S)
        torch.cuda.synchronize()
        assert np.max(np.abs(la.cpu().numpy() - la_ref.cpu().numpy())) <= tol
        assert np.array_equal(ph.cpu().numpy(), ph_ref.cpu().numpy())
        assert np.array_equal(st.cpu().numpy(), st_ref.cpu().numpy())
    h.close()


@pytest.mark.parametrize("prec,tol", [(0, 1e-10), (1, 1e-5)])
def test_noalloc_many_samples_per_cta(prec, tol):
    # more samples than two CTAs per SM: every CTA reuses its slice of the array for several
    # samples in turn, the case where work buffers left over from an earlier sample would show
    peps, f = _noalloc_fn()
    lat = I.Lattice(4, 4, 2, 2)
    chi = 3
    theta = torch.as_tensor(I.peps_random(lat, 1003, scale=0.5, bias=1.0)).cuda()
    h = peps.PEPS(lat.Lx, lat.Ly, lat.d, lat.D, chi, prec=prec, max_samples=1000)
    h.set_params(theta)
    for seed in (2003, 2004):
        S = torch.as_tensor(I.configs_uniform_sz0(lat, 1000, seed)).cuda()
        rc, la, ph, st = _call(peps, f, lat, chi, prec, theta, S)
        assert rc == 0, f"status {rc}"
        la_ref, ph_ref, st_ref = h.amplitudes(S)
        torch.cuda.synchronize()
        assert np.max(np.abs(la.cpu().numpy() - la_ref.cpu().numpy())) <= tol
        assert np.array_equal(ph.cpu().numpy(), ph_ref.cpu().numpy())
        assert np.array_equal(st.cpu().numpy(), st_ref.cpu().numpy())
    h.close()


def test_noalloc_rejects_problems_beyond_its_scratch():
    peps, f = _noalloc_fn()
    lat = I.Lattice(8, 8, 2, 4)
    theta = torch.zeros(I.num_params(lat), dtype=torch.float64, device="cuda")
    S = torch.zeros(4096, 64, dtype=torch.uint8, device="cuda")
    rc, _, _, _ = _call(peps, f, lat, 16, 0, theta, S)
    assert rc == -6  # PEPS_E_CAPACITY

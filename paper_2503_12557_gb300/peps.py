"""Thin ctypes binding over the C ABI in include/peps_gb300.h (argument marshalling only).

Device buffers are torch CUDA tensors; every call is enqueued on torch's current CUDA stream.
The shared library is loaded on first use from the package's _lib folder (built by
``paper_2503_12557_gb300.build``); a missing library raises instead of falling back to anything.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np
import torch

_LIB = None
_LIBPATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib", "libpeps_gb300.so")

PREC_FP64, PREC_FP32, PREC_MIXED = 0, 1, 2
MOVE_EXCHANGE, MOVE_FLIP = 0, 1
ST_NEAR_DEGENERATE, ST_ZERO_NORM, ST_NONFINITE, ST_NOCONV = 1, 2, 4, 8
SW_MINSR_BREAKDOWN, SW_GRAM_TIMEOUT = 1 << 8, 1 << 9

_ERRORS = {-1: "PEPS_E_ARG", -2: "PEPS_E_SHAPE", -3: "PEPS_E_WORKSPACE", -4: "PEPS_E_CUDA", -5: "PEPS_E_UNSUPPORTED",
           -6: "PEPS_E_CAPACITY", 1: "PEPS_W_NUMERIC"}


class _Config(C.Structure):
    _fields_ = [("Lx", C.c_int), ("Ly", C.c_int), ("d", C.c_int), ("D", C.c_int), ("chi", C.c_int),
                ("prec", C.c_int), ("max_samples", C.c_int), ("gram", C.c_int), ("solve", C.c_int),
                ("cplx", C.c_int), ("trunc_weight", C.c_double)]


class _Term(C.Structure):
    _fields_ = [("nsites", C.c_int), ("sites", C.c_int * 4), ("h_host", C.POINTER(C.c_double))]


class _Ham(C.Structure):
    _fields_ = [("nterms", C.c_int), ("terms", C.POINTER(_Term)), ("npairs", C.c_int),
                ("pair_ij_host", C.POINTER(C.c_int)), ("pair_v_host", C.POINTER(C.c_double)),
                ("onsite_host", C.POINTER(C.c_double))]


_ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_void_p, C.c_size_t)
_FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class _Allocator(C.Structure):
    _fields_ = [("alloc", _ALLOC_FN), ("free", _FREE_FN), ("ctx", C.c_void_p)]


def _torch_alloc(ctx, nbytes):
    try:
        return torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(),
                                                  torch.cuda.current_stream())
    except Exception:
        return None


def _torch_free(ctx, ptr):
    if ptr:
        torch.cuda.caching_allocator_delete(ptr)


# the handle's device memory comes from PyTorch's caching allocator (kept alive for the process)
_TORCH_ALLOCATOR = _Allocator(_ALLOC_FN(_torch_alloc), _FREE_FN(_torch_free), None)


class _BatchItem(C.Structure):
    _fields_ = [("h", C.c_void_p), ("H", C.POINTER(_Ham)), ("S_dev", C.c_void_p), ("Ns", C.c_int),
                ("logabs_dev", C.c_void_p), ("phase_dev", C.c_void_p), ("eloc_dev", C.c_void_p), ("O_dev", C.c_void_p),
                ("status_dev", C.c_void_p)]


def lib_path() -> str:
    return _LIBPATH


def load():
    """Load the CUDA library (raises RuntimeError when it has not been built)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(_LIBPATH):
        raise RuntimeError(f"CUDA library not built: {_LIBPATH} (run python -m paper_2503_12557_gb300.build)")
    L = C.CDLL(_LIBPATH)
    vp, i32, i64, dbl = C.c_void_p, C.c_int, C.c_longlong, C.c_double
    sig = {
        "peps_create": ([C.POINTER(vp), C.POINTER(_Config)], i32),
        "peps_create_ex": ([C.POINTER(vp), C.POINTER(_Config), C.POINTER(_Allocator)], i32),
        "peps_last_status": ([vp, C.POINTER(C.c_int32), vp], i32),
        "peps_status_weights": ([vp, i32, i32, vp, vp], i32),
        "minsr_partial_sums": ([vp, vp, vp, vp, i32, vp, vp], i32),
        "minsr_center_rows": ([vp, vp, vp, vp, i32, vp, vp, vp, vp], i32),
        "minsr_gram": ([vp, vp, i32, i64, vp, vp], i32),
        "minsr_solve": ([vp, vp, vp, i32, dbl, dbl, vp, vp, vp], i32),
        "minsr_project": ([vp, vp, i32, i64, dbl, vp, vp], i32),
        "peps_destroy": ([vp], i32),
        "peps_num_params": ([vp], i64),
        "peps_set_params": ([vp, vp, vp], i32),
        "peps_amplitudes": ([vp, vp, i32, vp, vp, vp, vp], i32),
        "peps_local_energy": ([vp, C.POINTER(_Ham), vp, i32, vp, vp, vp], i32),
        "peps_logderiv": ([vp, vp, i32, vp, vp, vp], i32),
        "peps_evaluate": ([vp, C.POINTER(_Ham), vp, i32, vp, vp, vp, vp, vp, vp], i32),
        "peps_local_energy_bound": ([vp, C.POINTER(_Ham), vp, i32, i32, vp, vp, vp, vp, vp], i32),
        "peps_rotate_params": ([vp, vp, vp, i32, vp, vp], i32),
        "peps_direct_prepare": ([vp, i32, vp], i32),
        "peps_set_env_reuse": ([vp, i32], i32),
        "peps_direct_sample": ([vp, vp, i32, C.c_uint64, C.c_uint64, vp, vp, vp], i32),
        "minsr_step": ([vp, vp, vp, vp, i32, dbl, dbl, dbl, vp, vp, vp], i32),
        "peps_sample": ([vp, i32, vp, i32, i32, C.c_uint64, C.c_uint64, vp, vp, vp], i32),
        "peps_last_error": ([vp], C.c_char_p),
        "peps_apply_update": ([vp, vp, vp, vp], i32),
        "peps_proposal_logits": ([i32, i32, i32, i32, vp, vp, i32, vp, vp], i32),
        "peps_proposal_train_step": ([i32, i32, i32, i32, vp, vp, vp, vp, i32, dbl, vp, vp, i32, vp, vp, vp], i32),
        "peps_sample_learned": ([vp, i32, i32, vp, vp, vp, i32, C.c_uint64, C.c_uint64, vp, vp, vp], i32),
        "peps_timing_enable": ([vp, i32], i32),
        "peps_timing_read": ([vp, vp, vp, i32, vp], i32),
        "peps_probe_fma": ([i32, C.POINTER(dbl), vp], i32),
        "peps_autotune": ([vp, C.POINTER(_Ham), vp, i32, i32, vp, vp], i32),
        "peps_batch_create": ([C.POINTER(vp), C.POINTER(_BatchItem), i32, i32, vp], i32),
        "peps_batch_create_ex": ([C.POINTER(vp), C.POINTER(_BatchItem), i32, i32, vp], i32),
        "peps_batch_autotune": ([C.POINTER(_BatchItem), i32, C.POINTER(i32), vp], i32),
        "peps_batch_launch": ([vp, vp], i32),
        "peps_batch_destroy": ([vp], i32),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _LIB = L
    return L


def exported_symbols():
    return ["peps_create", "peps_destroy", "peps_num_params", "peps_set_params", "peps_amplitudes",
            "peps_local_energy", "peps_logderiv", "peps_evaluate", "minsr_step", "peps_sample", "peps_last_error",
            "peps_timing_enable", "peps_timing_read", "peps_apply_update", "peps_proposal_logits",
            "peps_proposal_train_step", "peps_sample_learned", "peps_amplitudes_noalloc", "peps_probe_fma",
            "peps_autotune", "peps_batch_create", "peps_batch_launch", "peps_batch_destroy",
            "peps_local_energy_bound", "peps_rotate_params", "peps_direct_prepare", "peps_direct_sample",
            "peps_set_env_reuse", "peps_create_ex", "peps_last_status", "peps_status_weights",
            "minsr_partial_sums", "minsr_center_rows", "minsr_gram", "minsr_solve", "minsr_project",
            "peps_batch_create_ex", "peps_batch_autotune"]


def probe_fma(fp64=False):
    """Measured FP32 (or FP64) FMA throughput of the current GPU, TFLOP/s."""
    L = load()
    out = C.c_double(0.0)
    st = L.peps_probe_fma(1 if fp64 else 0, C.byref(out), _stream())
    if st != 0:
        raise RuntimeError(f"peps_probe_fma failed: {_ERRORS.get(st, st)}")
    return out.value


class Proposal:
    """Weights and Adam state of the learned proposal network (device tensors)."""

    def __init__(self, Lx, Ly, w0, C=16, wprec=1):
        self.L = load()
        self.Lx, self.Ly, self.C, self.wprec = Lx, Ly, C, wprec
        self.w = torch.as_tensor(np.asarray(w0, dtype=np.float64)).cuda().contiguous()
        self.m = torch.zeros_like(self.w)
        self.v = torch.zeros_like(self.w)
        self.g = torch.zeros_like(self.w)
        self.loss = torch.zeros(1, dtype=torch.float64, device="cuda")
        self.wlow = self.w.to(torch.bfloat16).contiguous() if wprec == 1 else None
        self.t = 0

    @property
    def wdev(self):
        return self.w if self.wprec == 0 else self.wlow

    def logits(self, S):
        ns = S.shape[0]
        out = torch.empty(ns, self.Lx * self.Ly, dtype=torch.float64, device=S.device)
        st = self.L.peps_proposal_logits(self.Lx, self.Ly, self.C, self.wprec, _ptr(self.wdev), _ptr(S.contiguous()),
                                         ns, _ptr(out), _stream())
        if st != 0:
            raise RuntimeError(f"peps_proposal_logits failed: {_ERRORS.get(st, st)}")
        return out

    def train_step(self, S_in, S_tgt, lr=1e-3):
        self.t += 1
        st = self.L.peps_proposal_train_step(self.Lx, self.Ly, self.C, self.wprec, _ptr(self.w), _ptr(self.m),
                                             _ptr(self.v), _ptr(self.wlow), self.t, float(lr), _ptr(S_in.contiguous()),
                                             _ptr(S_tgt.contiguous()), S_in.shape[0], _ptr(self.g), _ptr(self.loss),
                                             _stream())
        if st != 0:
            raise RuntimeError(f"peps_proposal_train_step failed: {_ERRORS.get(st, st)}")
        return self.loss


TIMING_CLASSES = ["env", "row", "pair", "combine", "sample", "minsr_gram", "minsr_eig", "minsr_other", "pad", "bound", "direct"]


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


class Hamiltonian:
    """ctypes view of a Hamiltonian dict from ``paper_2503_12557_gb300.inputs`` (host memory)."""

    def __init__(self, H, nsites: int, d: int):
        terms = H["terms"]
        self._h = [np.ascontiguousarray(np.stack([np.asarray(h).real, np.asarray(h).imag], -1).ravel(),
                                        dtype=np.float64) for _, h in terms]
        self._terms = (_Term * max(1, len(terms)))()
        for i, (sites, _) in enumerate(terms):
            self._terms[i].nsites = len(sites)
            for j in range(4):
                self._terms[i].sites[j] = int(sites[j]) if j < len(sites) else -1
            self._terms[i].h_host = self._h[i].ctypes.data_as(C.POINTER(C.c_double))
        pairs = H.get("pairs", [])
        self._pij = np.ascontiguousarray(np.array([[i, j] for i, j, _ in pairs], dtype=np.int32).reshape(-1))
        self._pv = np.ascontiguousarray(np.array([v for _, _, v in pairs], dtype=np.float64))
        on = H.get("onsite")
        self._on = None if on is None else np.ascontiguousarray(np.asarray(on, dtype=np.float64).reshape(nsites, d))
        self.c = _Ham()
        self.c.nterms = len(terms)
        self.c.terms = self._terms
        self.c.npairs = len(pairs)
        self.c.pair_ij_host = self._pij.ctypes.data_as(C.POINTER(C.c_int)) if len(pairs) else None
        self.c.pair_v_host = self._pv.ctypes.data_as(C.POINTER(C.c_double)) if len(pairs) else None
        self.c.onsite_host = self._on.ctypes.data_as(C.POINTER(C.c_double)) if self._on is not None else None


class PEPS:
    """One handle of the C library: a lattice, chi and a precision."""

    def __init__(self, Lx, Ly, d, D, chi, prec=PREC_FP64, max_samples=4096, gram=0, solve=0, cplx=False, trunc_weight=0.0,
                 allocator="torch"):
        """allocator: "torch" (the handle's device memory from PyTorch's caching allocator, through
        peps_create_ex) or None (the library's own cudaMalloc, peps_create)."""
        self.L = load()
        self.Lx, self.Ly, self.d, self.D, self.chi, self.prec = Lx, Ly, d, D, chi, prec
        self.max_samples = max_samples
        self.gram = gram
        self.last_warning = None
        self.solve = solve
        self.cplx = bool(cplx)
        self.trunc_weight = float(trunc_weight)
        cfg = _Config(Lx, Ly, d, D, chi, prec, max_samples, gram, solve, int(self.cplx), self.trunc_weight)
        h = C.c_void_p()
        if allocator == "torch":
            st = self.L.peps_create_ex(C.byref(h), C.byref(cfg), C.byref(_TORCH_ALLOCATOR))
        else:
            st = self.L.peps_create(C.byref(h), C.byref(cfg))
        if st != 0:
            raise RuntimeError(f"peps_create failed: {_ERRORS.get(st, st)}")
        self.h = h
        self.Np = int(self.L.peps_num_params(h))
        self._ham_cache = {}

    def close(self):
        if getattr(self, "h", None):
            self.L.peps_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st, what):
        self.last_warning = None
        if st > 0:  # PEPS_W_NUMERIC: the call completed with a numerical warning
            msg = self.L.peps_last_error(self.h)
            self.last_warning = f"{what}: {msg.decode() if msg else 'numerical warning'}"
            return
        if st != 0:
            msg = self.L.peps_last_error(self.h)
            raise RuntimeError(f"{what} failed: {_ERRORS.get(st, st)}: {msg.decode() if msg else ''}")

    @property
    def odtype(self):
        if self.cplx:
            return torch.complex128 if self.prec == PREC_FP64 else torch.complex64
        return torch.float64 if self.prec == PREC_FP64 else torch.float32

    @property
    def tdtype(self):
        """dtype of theta and dtheta."""
        return torch.complex128 if self.cplx else torch.float64

    def set_params(self, theta: torch.Tensor):
        assert theta.is_cuda and theta.dtype == self.tdtype and theta.numel() == self.Np
        theta = theta.contiguous()
        self._check(self.L.peps_set_params(self.h, _ptr(theta), _stream()), "peps_set_params")
        self._theta_ref = theta

    def hamiltonian(self, H):
        key = id(H)
        if key not in self._ham_cache:
            self._ham_cache[key] = (H, Hamiltonian(H, self.Lx * self.Ly, self.d))
        return self._ham_cache[key][1]

    def _S(self, S):
        assert S.is_cuda and S.dtype == torch.uint8 and S.dim() == 2 and S.shape[1] == self.Lx * self.Ly
        return S.contiguous()

    def autotune(self, S, H=None, move=None):
        """Pick the shared-memory budget of each kernel class by timing the candidates on S
        (peps_autotune); returns the chosen budgets in KB (env, row, pair, sampler)."""
        S = self._S(S)
        mv = MOVE_EXCHANGE if move is None else move
        kb = (C.c_int * 4)()
        hc = self.hamiltonian(H) if H is not None else None
        self._check(self.L.peps_autotune(self.h, C.byref(hc.c) if hc is not None else None, _ptr(S), S.shape[0], mv,
                                         kb, _stream()), "peps_autotune")
        return list(kb)

    def amplitudes(self, S):
        S = self._S(S)
        ns = S.shape[0]
        la = torch.empty(ns, dtype=torch.float64, device=S.device)
        ph = torch.empty_like(la)
        st = torch.empty(ns, dtype=torch.int32, device=S.device)
        self._check(self.L.peps_amplitudes(self.h, _ptr(S), ns, _ptr(la), _ptr(ph), _ptr(st), _stream()),
                    "peps_amplitudes")
        return la, ph, st

    def local_energy(self, H, S):
        S = self._S(S)
        ns = S.shape[0]
        e = torch.empty(ns, 2, dtype=torch.float64, device=S.device)
        st = torch.empty(ns, dtype=torch.int32, device=S.device)
        hc = self.hamiltonian(H)
        self._check(self.L.peps_local_energy(self.h, C.byref(hc.c), _ptr(S), ns, _ptr(e), _ptr(st), _stream()),
                    "peps_local_energy")
        return e, st

    def logderiv(self, S, out=None):
        S = self._S(S)
        ns = S.shape[0]
        O = out if out is not None else torch.empty(ns, self.Np, dtype=self.odtype, device=S.device)
        st = torch.empty(ns, dtype=torch.int32, device=S.device)
        self._check(self.L.peps_logderiv(self.h, _ptr(S), ns, _ptr(O), _ptr(st), _stream()), "peps_logderiv")
        return O, st

    def evaluate(self, H, S, want_logpsi=True, want_eloc=True, want_O=True, O_out=None):
        S = self._S(S)
        ns = S.shape[0]
        dev = S.device
        la = torch.empty(ns, dtype=torch.float64, device=dev) if want_logpsi else None
        ph = torch.empty(ns, dtype=torch.float64, device=dev) if want_logpsi else None
        e = torch.empty(ns, 2, dtype=torch.float64, device=dev) if want_eloc else None
        O = (O_out if O_out is not None else torch.empty(ns, self.Np, dtype=self.odtype, device=dev)) if want_O else None
        st = torch.empty(ns, dtype=torch.int32, device=dev)
        hc = self.hamiltonian(H) if H is not None else None
        self._check(self.L.peps_evaluate(self.h, C.byref(hc.c) if hc else None, _ptr(S), ns, _ptr(la), _ptr(ph),
                                         _ptr(e), _ptr(O), _ptr(st), _stream()), "peps_evaluate")
        return dict(logabs=la, phase=ph, eloc=e, O=O, status=st)

    def local_energy_bound(self, H, S, cut):
        """Variational-bound E_loc with every amplitude taken at one cut (1 <= cut <= Lx-1):
        dict of eloc (Ns x 2), logabs and phase of psi_cut(S), status."""
        S = self._S(S)
        ns = S.shape[0]
        dev = S.device
        la = torch.empty(ns, dtype=torch.float64, device=dev)
        ph = torch.empty(ns, dtype=torch.float64, device=dev)
        e = torch.empty(ns, 2, dtype=torch.float64, device=dev)
        st = torch.empty(ns, dtype=torch.int32, device=dev)
        hc = self.hamiltonian(H)
        self._check(self.L.peps_local_energy_bound(self.h, C.byref(hc.c), _ptr(S), ns, int(cut), _ptr(e), _ptr(la),
                                                   _ptr(ph), _ptr(st), _stream()), "peps_local_energy_bound")
        return dict(eloc=e, logabs=la, phase=ph, status=st)

    def set_env_reuse(self, enable=True):
        """Let an evaluation of the unmodified output of the last sample() reuse the sampler's
        upper environments (see peps_set_env_reuse)."""
        self._check(self.L.peps_set_env_reuse(self.h, 1 if enable else 0), "peps_set_env_reuse")

    def direct_prepare(self, chi_double):
        """Double-layer lower environments of the current parameters for direct sampling."""
        self._check(self.L.peps_direct_prepare(self.h, int(chi_double), _stream()), "peps_direct_prepare")

    def direct_sample(self, ns, seed=0, draw=0, S_out=None):
        """ns independent configurations drawn row by row; returns (S, log p(S), status)."""
        dev = torch.device("cuda")
        S = S_out if S_out is not None else torch.empty(ns, self.Lx * self.Ly, dtype=torch.uint8, device=dev)
        lp = torch.empty(ns, dtype=torch.float64, device=dev)
        st = torch.empty(ns, dtype=torch.int32, device=dev)
        self._check(self.L.peps_direct_sample(self.h, _ptr(S), ns, int(seed) & (2 ** 64 - 1), int(draw), _ptr(lp),
                                              _ptr(st), _stream()), "peps_direct_sample")
        return S, lp, st

    def rotate_params(self, M, theta):
        """theta' (complex128, N_p) with the physical index of every site tensor multiplied by the
        d x d matrix M; theta: a device tensor, real or complex."""
        M = np.ascontiguousarray(np.asarray(M, dtype=np.complex128))
        assert M.shape == (self.d, self.d)
        Mh = np.ascontiguousarray(M.view(np.float64).reshape(-1))
        cplx_in = 1 if theta.is_complex() else 0
        theta = theta.to(torch.complex128 if cplx_in else torch.float64).contiguous()
        out = torch.empty(self.Np, dtype=torch.complex128, device=theta.device)
        self._check(self.L.peps_rotate_params(self.h, Mh.ctypes.data, _ptr(theta), cplx_in, _ptr(out), _stream()),
                    "peps_rotate_params")
        return out

    def last_status(self):
        """Synchronise the current stream and read (and clear) the handle's status word (the OR of
        per-sample status bits and MinSR flags since the last read); sets last_warning when a
        MinSR step broke down.  Returns the word."""
        w = C.c_int32(0)
        st = self.L.peps_last_status(self.h, C.byref(w), _stream())
        self.last_warning = None
        if st == -4:
            msg = self.L.peps_last_error(self.h)
            raise RuntimeError(f"peps_last_status: {msg.decode() if msg else ''}")
        if w.value & SW_MINSR_BREAKDOWN:
            msg = self.L.peps_last_error(self.h)
            self.last_warning = f"minsr_step: {msg.decode() if msg else 'numerical warning'}"
        return w.value

    def status_weights(self, status, mask=ST_ZERO_NORM | ST_NONFINITE | ST_NOCONV):
        """MinSR weights 0 for the samples whose status has a bit of mask, else 1 (device)."""
        assert status.is_cuda and status.dtype == torch.int32
        w = torch.empty(status.shape[0], dtype=torch.float64, device=status.device)
        st = self.L.peps_status_weights(_ptr(status.contiguous()), status.shape[0], int(mask), _ptr(w), _stream())
        if st != 0:
            raise RuntimeError(f"peps_status_weights failed: {_ERRORS.get(st, st)}")
        return w

    def minsr_step(self, O, eloc, w=None, lam=1e-4, rcond=0.0, tau=0.05):
        """dtheta and info of one MinSR step, asynchronous on the current stream; a breakdown
        (info[0] = -1, dtheta zero) is reported by last_status()."""
        ns = O.shape[0]
        assert O.dtype == self.odtype and O.shape[1] == self.Np and eloc.shape == (ns, 2)
        dth = torch.empty(self.Np, dtype=self.tdtype, device=O.device)
        info = torch.zeros(4, dtype=torch.float64, device=O.device)
        self._check(self.L.minsr_step(self.h, _ptr(O.contiguous()), _ptr(eloc.contiguous()),
                                      _ptr(w.contiguous()) if w is not None else None, ns, float(lam), float(rcond),
                                      float(tau), _ptr(dth), _ptr(info), _stream()), "minsr_step")
        return dth, info

    # ---- sample-sharded MinSR pieces (paper_2503_12557_gb300.dist): real PEPS only
    def minsr_partial_sums(self, O, eloc, w=None):
        ns = O.shape[0]
        assert O.dtype == self.odtype and O.shape[1] == self.Np and eloc.shape == (ns, 2)
        sums = torch.empty(self.Np + 2, dtype=torch.float64, device=O.device)
        self._check(self.L.minsr_partial_sums(self.h, _ptr(O.contiguous()), _ptr(eloc.contiguous()),
                                              _ptr(w.contiguous()) if w is not None else None, ns, _ptr(sums),
                                              _stream()), "minsr_partial_sums")
        return sums

    def minsr_center_rows(self, O, eloc, w, gsums):
        ns = O.shape[0]
        Ob = torch.empty(ns, self.Np, dtype=torch.float64, device=O.device)
        eb = torch.empty(ns, dtype=torch.float64, device=O.device)
        self._check(self.L.minsr_center_rows(self.h, _ptr(O.contiguous()), _ptr(eloc.contiguous()),
                                             _ptr(w.contiguous()) if w is not None else None, ns,
                                             _ptr(gsums.contiguous()), _ptr(Ob), _ptr(eb), _stream()),
                    "minsr_center_rows")
        return Ob, eb

    def minsr_gram(self, A):
        A = A.contiguous()
        ns, k = A.shape
        T = torch.empty(ns, ns, dtype=torch.float64, device=A.device)
        self._check(self.L.minsr_gram(self.h, _ptr(A), ns, k, _ptr(T), _stream()), "minsr_gram")
        return T

    def minsr_solve(self, T, ebar, lam=1e-4, rcond=0.0):
        ns = T.shape[0]
        x = torch.empty(ns, dtype=torch.float64, device=T.device)
        info = torch.zeros(4, dtype=torch.float64, device=T.device)
        self._check(self.L.minsr_solve(self.h, _ptr(T.contiguous()), _ptr(ebar.contiguous()), ns, float(lam),
                                       float(rcond), _ptr(x), _ptr(info), _stream()), "minsr_solve")
        return x, info

    def minsr_project(self, A, x, tau=0.05):
        A = A.contiguous()
        ns, k = A.shape
        d = torch.empty(k, dtype=torch.float64, device=A.device)
        st = self.L.minsr_project(_ptr(A), _ptr(x.contiguous()), ns, k, float(tau), _ptr(d), _stream())
        if st != 0:
            raise RuntimeError(f"minsr_project failed: {_ERRORS.get(st, st)}")
        return d

    def apply_update(self, theta: torch.Tensor, dtheta: torch.Tensor):
        """theta += dtheta on the device (in place) and refresh the handle's kernel copy."""
        assert theta.is_cuda and theta.dtype == self.tdtype and theta.is_contiguous()
        assert dtheta.dtype == self.tdtype
        self._check(self.L.peps_apply_update(self.h, _ptr(theta), _ptr(dtheta.contiguous()), _stream()),
                    "peps_apply_update")
        self._theta_ref = theta

    def sample_learned(self, prop, S, logpsi, seed=0, step=0, accepted=None):
        """One network move of every chain (S and logpsi updated in place)."""
        S = self._S(S)
        ns = S.shape[0]
        st = torch.empty(ns, dtype=torch.int32, device=S.device)
        self._check(self.L.peps_sample_learned(self.h, prop.C, prop.wprec, _ptr(prop.wdev), _ptr(S), _ptr(logpsi), ns,
                                               int(seed) & (2 ** 64 - 1), int(step), _ptr(accepted), _ptr(st),
                                               _stream()), "peps_sample_learned")
        return S, logpsi, st

    def timing(self, enable=True):
        self._check(self.L.peps_timing_enable(self.h, 1 if enable else 0), "peps_timing_enable")

    def timing_read(self):
        n = len(TIMING_CLASSES)
        ms = (C.c_double * n)()
        la = (C.c_longlong * n)()
        ctr = (C.c_longlong * 4)()
        self._check(self.L.peps_timing_read(self.h, ms, la, n, ctr), "peps_timing_read")
        return ({k: ms[i] for i, k in enumerate(TIMING_CLASSES)}, {k: la[i] for i, k in enumerate(TIMING_CLASSES)},
                dict(jacobi_sweeps=ctr[0], jacobi_rotations=ctr[1], svds=ctr[2]))

    def sample(self, S, move=MOVE_EXCHANGE, nsweeps=1, seed=0, sweep0=0, accepted=None):
        S = self._S(S)
        ns = S.shape[0]
        acc = accepted if accepted is not None else torch.zeros(ns, dtype=torch.int64, device=S.device)
        st = torch.empty(ns, dtype=torch.int32, device=S.device)
        self._check(self.L.peps_sample(self.h, int(move), _ptr(S), ns, int(nsweeps), int(seed) & (2 ** 64 - 1),
                                       int(sweep0), _ptr(acc), _ptr(st), _stream()), "peps_sample")
        return S, acc, st


class Batch:
    """Independent handles (ragged lattices, D, chi, sample counts) evaluated by one persistent
    kernel launch per precision over a work queue of (instance, sample) items, recorded in a
    CUDA graph (peps_batch_*).  items: a list of (PEPS handle, H or None, S (device uint8),
    want_O); the output tensors are allocated here and refreshed in place at every launch().
    budget_kb: shared memory per CTA of the batch kernel (0: default; autotune=True times the
    candidates with peps_batch_autotune and keeps the fastest)."""

    def __init__(self, items, nbranch=4, stream=None, budget_kb=0, autotune=False):
        self.L = load()
        self.stream = stream if stream is not None else torch.cuda.Stream()
        self.keep, arr = [], (_BatchItem * len(items))()
        self.out = []
        for k, (h, H, S, want_O) in enumerate(items):
            S = h._S(S)
            ns = S.shape[0]
            o = dict(S=S, logabs=torch.empty(ns, dtype=torch.float64, device=S.device),
                     phase=torch.empty(ns, dtype=torch.float64, device=S.device),
                     status=torch.zeros(ns, dtype=torch.int32, device=S.device))
            o["eloc"] = torch.empty(ns, 2, dtype=torch.float64, device=S.device) if H is not None else None
            o["O"] = torch.empty(ns, h.Np, dtype=h.odtype, device=S.device) if want_O else None
            hc = h.hamiltonian(H) if H is not None else None
            arr[k].h = h.h
            arr[k].H = C.pointer(hc.c) if hc is not None else None
            arr[k].S_dev = _ptr(S)
            arr[k].Ns = ns
            arr[k].logabs_dev, arr[k].phase_dev = _ptr(o["logabs"]), _ptr(o["phase"])
            arr[k].eloc_dev = _ptr(o["eloc"]) if o["eloc"] is not None else None
            arr[k].O_dev = _ptr(o["O"]) if o["O"] is not None else None
            arr[k].status_dev = _ptr(o["status"])
            self.keep.append((h, hc))
            self.out.append(o)
        self.b = C.c_void_p()
        torch.cuda.current_stream().synchronize()
        sp = C.c_void_p(self.stream.cuda_stream)
        if autotune:
            kb = C.c_int(0)
            st = self.L.peps_batch_autotune(arr, len(items), C.byref(kb), sp)
            if st != 0:
                raise RuntimeError(f"peps_batch_autotune failed: {_ERRORS.get(st, st)}")
            budget_kb = kb.value
        self.budget_kb = budget_kb
        st = self.L.peps_batch_create_ex(C.byref(self.b), arr, len(items), int(budget_kb), sp)
        if st != 0:
            raise RuntimeError(f"peps_batch_create failed: {_ERRORS.get(st, st)}")
        self.stream.synchronize()

    def launch(self):
        st = self.L.peps_batch_launch(self.b, C.c_void_p(self.stream.cuda_stream))
        if st != 0:
            raise RuntimeError(f"peps_batch_launch failed: {_ERRORS.get(st, st)}")

    def close(self):
        if getattr(self, "b", None) and self.b.value:
            self.L.peps_batch_destroy(self.b)
            self.b = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

"""Energy estimators around the C library beyond the fast local estimator of peps_evaluate.

rotated_basis_energy: the unbiased estimator of Sec. "On reusing environments" (and the
appendix on variational upper bounds): a Heisenberg-type H = sum_b J_b S_i . S_j is split into
its x, y and z parts, each diagonal in its own basis; the PEPS is rotated into each basis on
the device (peps_rotate_params), sampled there by its own Metropolis flip chains, and the
diagonal part is averaged over those samples.  No amplitude ratio enters the energy, so no
mixture of boundary-MPS approximations can bias it.

bound_energy: the mean of the variational-bound local energy (peps_local_energy_bound) over a
configuration batch, with its standard error.

contraction_error: the relative contraction error of Sec. "Contraction complexity indicators",
Delta psi(D_c, D_c^max) = (psi(D_c^max) - psi(D_c)) / psi(D_c^max), from the amplitudes of two
handles that differ only in the boundary bond dimension (or truncated-weight cutoff).
"""
from __future__ import annotations

import numpy as np
import torch

from . import inputs as I
from . import peps as P


def rotated_basis_energy(Lx, Ly, D, chi, theta, bonds, S0, burn_in=20, seed=1, prec=P.PREC_FP64, handle=None):
    """(energy, stderr, per-basis list of (mean, stderr, acceptance)) of <H> for the PEPS theta
    (a device tensor, real or complex) and H = sum_{(i, j, J) in bonds} J S_i . S_j, from
    N_s = len(S0) flip chains per basis after burn_in sweeps.  handle: a complex handle of the
    same shape to reuse (its parameters are overwritten)."""
    lat = I.Lattice(Lx, Ly, 2, D)
    ns = len(S0)
    h = handle or P.PEPS(Lx, Ly, 2, D, chi, prec=prec, max_samples=ns, cplx=True)
    out = []
    for a, (V, Hd) in enumerate(I.axis_parts(lat, bonds)):
        h.set_params(h.rotate_params(V.conj().T, theta))
        S = torch.as_tensor(np.asarray(S0, dtype=np.uint8)).cuda().contiguous()
        acc = torch.zeros(ns, dtype=torch.int64, device=S.device)
        h.sample(S, P.MOVE_FLIP, burn_in, seed=seed + 7919 * a, accepted=acc)
        r = h.evaluate(Hd, S, want_logpsi=False, want_eloc=True, want_O=False)
        e = r["eloc"][:, 0].double()
        out.append((float(e.mean()), float(e.std() / np.sqrt(ns)), float(acc.sum()) / (ns * burn_in * Lx * Ly)))
    return sum(m for m, _, _ in out), float(np.sqrt(sum(s * s for _, s, _ in out))), out


def bound_energy(h, H, S, cut):
    """(mean, stderr) of E_loc^bound over the batch S at the given cut, and the raw result."""
    r = h.local_energy_bound(H, S, cut)
    e = r["eloc"][:, 0].double()
    return float(e.mean()), float(e.std() / np.sqrt(e.numel())), r


def contraction_error(h_c, h_max, S):
    """Delta psi(D_c, D_c^max) per configuration (complex), from peps_amplitudes of the handle
    h_c (bond D_c) and h_max (bond D_c^max, the same parameters set on both):
    1 - psi_c / psi_max = 1 - exp(ln|psi_c| - ln|psi_max|) e^{i (phase_c - phase_max)}."""
    la, pa, sa = h_c.amplitudes(S)
    lb, pb, sb = h_max.amplitudes(S)
    z = torch.exp(la - lb) * torch.exp(1j * (pa - pb))
    return 1.0 - z, sa | sb

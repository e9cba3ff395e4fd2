"""MinSR update (oracle, FP64).

Paper: Eq. (tdvp_fast): theta_dot = O^dag (O O^dag)^-1 E_loc with T_SS' = sum_i O_Si O*_S'i
(N_s x N_s), solved by an eigendecomposition / pseudo-inverse; Eq. (tdvp_slow): the SR form
(O^dag O)^-1 O^dag E_loc it replaces.

Readings (the paper is silent on centring, weights, sign, step size and regularisation):
  w_S = 1/N_s (or the caller's weights, normalised to sum 1);
  Obar_{S,k} = sqrt(w_S) (O_{S,k} - sum_S' w_S' O_{S',k});  ebar_S = sqrt(w_S)(E_loc(S) - sum w E_loc);
  T = Obar Obar^dag = V diag(Lambda) V^dag;
  (T + lam)^+ = V diag(1/(Lambda_i + lam) if kept else 0) V^dag, kept = Lambda_i > rcond * max(Lambda)
  when rcond > 0, every eigenvalue when rcond == 0 (then lam must be > 0);
  dtheta = -tau Obar^dag (T + lam)^+ ebar  (imaginary-time step, Eq. (Schrodinger) with a minus sign).
"""
from __future__ import annotations

import numpy as np


def centred(O, eloc, w=None):
    Ns = O.shape[0]
    w = np.full(Ns, 1.0 / Ns) if w is None else np.asarray(w, dtype=np.float64) / np.sum(w)
    sw = np.sqrt(w)
    Obar = sw[:, None] * (O - w @ O)
    ebar = sw * (eloc - w @ eloc)
    return Obar, ebar


def minsr(O, eloc, w=None, lam=1e-4, rcond=0.0, tau=0.05):
    if not (lam > 0 or rcond > 0):
        raise ValueError("need lam > 0 or rcond > 0")
    Obar, ebar = centred(O, eloc, w)
    T = Obar @ np.conj(Obar.T)
    lv, V = np.linalg.eigh(T)
    lmax = float(np.max(lv))
    keep = lv > rcond * lmax if rcond > 0 else np.ones_like(lv, dtype=bool)
    inv = np.where(keep, 1.0 / (lv + lam), 0.0)
    x = V @ (inv * (np.conj(V.T) @ ebar))
    dtheta = -tau * (np.conj(Obar.T) @ x)
    info = dict(rank=int(np.sum(keep)), lmin=float(np.min(lv)), lmax=lmax, T=T, x=x)
    return dtheta, info


def sr_pushthrough(O, eloc, w=None, lam=1e-4, tau=0.05):
    """-tau (Obar^dag Obar + lam)^-1 Obar^dag ebar: the N_p x N_p SR form (equal to minsr for lam > 0)."""
    Obar, ebar = centred(O, eloc, w)
    G = np.conj(Obar.T) @ Obar
    return -tau * np.linalg.solve(G + lam * np.eye(G.shape[0]), np.conj(Obar.T) @ ebar)


def sr_pinv(O, eloc, w=None, tau=0.05, rcond=1e-10):
    """-tau pinv(Obar) ebar via an SVD of Obar (the minimum-norm least-squares SR solution)."""
    Obar, ebar = centred(O, eloc, w)
    U, s, Vh = np.linalg.svd(Obar, full_matrices=False)
    keep = s > rcond * s[0]
    return -tau * (np.conj(Vh[keep].T) @ ((np.conj(U[:, keep].T) @ ebar) / s[keep]))

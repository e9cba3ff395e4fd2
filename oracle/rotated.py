"""Rotated-basis energy estimator (oracle, FP64; test infrastructure only).

Paper: Sec. "On reusing environments and the convenient treatment of long-range
interactions" (terms diagonal in a rotated basis, a global spin rotation of the PEPS and an
independent sample per rotated PEPS) and the appendix on variational upper bounds (this
estimator needs no amplitude ratios, so no mix of boundary-MPS approximations enters it).

For H = sum_alpha H_alpha with H_alpha diagonal in the basis |s>_alpha = V_alpha[:, s]:
    psi_alpha(S) = <S_alpha|psi> = sum_T prod_i conj(V_alpha[t_i, s_i]) psi(T),
i.e. the PEPS with every site tensor rotated on its physical index by M = V_alpha^dagger, and
    <H> = sum_alpha sum_S |psi_alpha(S)|^2 H_alpha(S) / <psi|psi>.
"""
from __future__ import annotations

import numpy as np

from paper_2503_12557_gb300.inputs import Lattice, theta_to_tensors, site_offsets
from . import exact


def rotate_theta(theta, lat: Lattice, M):
    """theta' with T'[x][y][s] = sum_t M[s, t] T[x][y][t] for every site (complex)."""
    T = theta_to_tensors(lat, np.asarray(theta, dtype=np.complex128))
    offs = site_offsets(lat)
    out = np.zeros(offs[-1], dtype=np.complex128)
    k = 0
    for x in range(lat.Lx):
        for y in range(lat.Ly):
            R = np.einsum("st,t...->s...", M, T[x][y])
            out[offs[k]:offs[k + 1]] = R.reshape(-1)
            k += 1
    return out


def diagonal_value(Hd, S):
    """H_alpha(S) of a diagonal Hamiltonian (pairs and on-site terms only)."""
    S = np.asarray(S)
    e = 0.0
    for (i, j, v) in Hd["pairs"]:
        e += v * int(S[i]) * int(S[j])
    for i in range(len(S)):
        e += Hd["onsite"][i][int(S[i])]
    return e


def energy_exact(theta, lat: Lattice, parts):
    """sum_alpha <psi_alpha|H_alpha|psi_alpha> / <psi|psi> from the full rotated state vectors,
    and the per-basis terms."""
    per = []
    for V, Hd in parts:
        psi = exact.state_vector(rotate_theta(theta, lat, V.conj().T), lat)
        Hm = exact.hamiltonian_sparse(Hd, lat)
        per.append(float(np.real(np.vdot(psi, Hm @ psi) / np.vdot(psi, psi))))
    return sum(per), per

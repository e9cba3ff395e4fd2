"""Seeded synthetic inputs shared by the CUDA path, the oracle, the tests and the benchmark.

This module holds no arithmetic of the method (no contraction, truncation, estimator or
solver).  It only draws PEPS tensors and spin configurations from seeded numpy generators and
writes down the model Hamiltonians as lists of local terms.

Conventions (shared by every consumer):

* Lattice sites (x, y), x = 0..Lx-1 top to bottom, y = 0..Ly-1 left to right, linear index
  x*Ly + y (row major).
* Site tensor T[x,y][s, l, u, r, d] (physical index first, then the left, up, right and down
  virtual legs).  Open boundary: a leg that points out of the lattice has dimension 1
  (paper Sec. "On the boundary MPS method": tensors T[x,y] with physical dimension d and
  virtual dimension D).
* theta: all site tensors flattened in C order and concatenated in site order.  Its length is
  the parameter count N_p.
* Local states s in {0..d-1}.  For spin-1/2, s = 0 is up (S^z = +1/2).  For the Rydberg array,
  s = 1 is the Rydberg state |r> (n = 1).
* A Hamiltonian is a dict with
    - "terms":  list of (sites, h) with sites a tuple of linear site indices and h a complex
      d^k x d^k matrix, h[a, b] = <S_loc = a| h |S'_loc = b>; the local index of a tuple of
      states is a = sum_i s_i d^(k-1-i) (first site most significant);
    - "pairs":  list of (i, j, v): diagonal interaction v * s_i * s_j;
    - "onsite": (N, d) array, diagonal single-site energy onsite[i, s_i].
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

__all__ = [
    "Lattice", "leg_dims", "num_params", "site_offsets",
    "peps_random", "theta_to_tensors", "tensors_to_theta",
    "configs_uniform_sz0", "configs_neel", "configs_uniform", "configs_constant",
    "heisenberg", "j1j2_chiral", "rydberg", "pauli", "spin_bonds", "axis_bases", "axis_parts",
    "WORKLOADS",
]


@dataclass(frozen=True)
class Lattice:
    Lx: int
    Ly: int
    d: int
    D: int

    @property
    def nsites(self) -> int:
        return self.Lx * self.Ly


def leg_dims(lat: Lattice, x: int, y: int):
    """(d, Dl, Du, Dr, Dd) of site (x, y) with open-boundary legs of dimension 1."""
    D = lat.D
    return (lat.d,
            1 if y == 0 else D,
            1 if x == 0 else D,
            1 if y == lat.Ly - 1 else D,
            1 if x == lat.Lx - 1 else D)


def site_offsets(lat: Lattice):
    """Start offset of every site tensor inside theta, plus the total N_p at the end."""
    offs = [0]
    for x in range(lat.Lx):
        for y in range(lat.Ly):
            offs.append(offs[-1] + int(np.prod(leg_dims(lat, x, y))))
    return offs


def num_params(lat: Lattice) -> int:
    return site_offsets(lat)[-1]


def theta_to_tensors(lat: Lattice, theta: np.ndarray):
    """Split a flat theta into T[x][y] arrays of shape (d, Dl, Du, Dr, Dd) (views)."""
    offs = site_offsets(lat)
    T = []
    for x in range(lat.Lx):
        row = []
        for y in range(lat.Ly):
            i = x * lat.Ly + y
            row.append(theta[offs[i]:offs[i + 1]].reshape(leg_dims(lat, x, y)))
        T.append(row)
    return T


def tensors_to_theta(lat: Lattice, T) -> np.ndarray:
    return np.concatenate([np.asarray(T[x][y]).ravel() for x in range(lat.Lx) for y in range(lat.Ly)])


def peps_random(lat: Lattice, seed: int, kind: str = "normal", scale: float = 1.0,
                bias: float = 0.0, alpha: float = 0.0, complex_: bool = False) -> np.ndarray:
    """Random PEPS parameters theta (float64 or complex128).

    kind="normal":  entries i.i.d. scale * N(0, 1) (complex: real and imaginary parts each
                    N(0, scale^2 / 2), so E|z|^2 = scale^2).
    bias:           added to the entry with all virtual indices 0, for every physical s
                    ("identity-like bias on the all-zero virtual index").
    alpha > 0:      every virtual leg multiplied by diag(1 / i^alpha), i = 1..D (the algebraically
                    decaying initialisation of Eq. (A_alpha)).
    """
    rng = np.random.default_rng(seed)
    T = []
    for x in range(lat.Lx):
        row = []
        for y in range(lat.Ly):
            shp = leg_dims(lat, x, y)
            if complex_:
                t = (rng.standard_normal(shp) + 1j * rng.standard_normal(shp)) * (scale / math.sqrt(2.0))
            else:
                t = rng.standard_normal(shp) * scale
            if bias != 0.0:
                t[:, 0, 0, 0, 0] += bias
            if alpha > 0.0:
                for leg in range(1, 5):
                    n = shp[leg]
                    w = 1.0 / np.arange(1, n + 1, dtype=np.float64) ** alpha
                    sh = [1] * 5
                    sh[leg] = n
                    t = t * w.reshape(sh)
            row.append(t)
        T.append(row)
    return tensors_to_theta(lat, T)


def peps_near_product(lat: Lattice, seed: int, amp: float = 0.3, noise: float = 0.05) -> np.ndarray:
    """A PEPS close to a product state with a polarised local distribution: every tensor is
    1.0 on the all-zero virtual index plus noise * N(0, 1), and the s = 1 slice is scaled by
    `amp` (so P(s = 1) is about amp^2 / (1 + amp^2) per site, weakly correlated)."""
    theta = peps_random(lat, seed, scale=noise, bias=1.0)
    T = theta_to_tensors(lat, theta)
    for x in range(lat.Lx):
        for y in range(lat.Ly):
            T[x][y][1:] *= amp
    return theta


# ----------------------------------------------------------------------------- configurations

def configs_uniform_sz0(lat: Lattice, ns: int, seed: int) -> np.ndarray:
    """ns configurations drawn i.i.d. uniformly (with replacement) from the S^z = 0 sector."""
    rng = np.random.default_rng(seed)
    n = lat.nsites
    out = np.zeros((ns, n), dtype=np.uint8)
    for i in range(ns):
        up = rng.choice(n, size=n // 2, replace=False)
        out[i, :] = 1
        out[i, up] = 0
    return out


def configs_uniform(lat: Lattice, ns: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.integers(0, lat.d, size=(ns, lat.nsites), dtype=np.uint8)


def configs_neel(lat: Lattice, ns: int) -> np.ndarray:
    x, y = np.meshgrid(np.arange(lat.Lx), np.arange(lat.Ly), indexing="ij")
    s = ((x + y) % 2).astype(np.uint8).ravel()
    return np.tile(s, (ns, 1))


def configs_constant(lat: Lattice, ns: int, value: int = 0) -> np.ndarray:
    return np.full((ns, lat.nsites), value, dtype=np.uint8)


# ----------------------------------------------------------------------------- Hamiltonians

def pauli():
    sx = np.array([[0, 1], [1, 0]], dtype=np.complex128)
    sy = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
    sz = np.array([[1, 0], [0, -1]], dtype=np.complex128)
    return sx, sy, sz


def _kron(*ms):
    out = np.array([[1.0 + 0j]])
    for m in ms:
        out = np.kron(out, m)
    return out


def _spin_ops():
    sx, sy, sz = pauli()
    return 0.5 * sx, 0.5 * sy, 0.5 * sz


def _sdots():
    """S_i . S_j on two spin-1/2 sites, built from Kronecker products of Pauli matrices."""
    S = _spin_ops()
    return sum(_kron(a, a) for a in S)


def _chirality():
    """S_i . (S_j x S_k) on three spin-1/2 sites (Kronecker products of Pauli matrices)."""
    Sx, Sy, Sz = _spin_ops()
    S = (Sx, Sy, Sz)
    eps = {(0, 1, 2): 1, (1, 2, 0): 1, (2, 0, 1): 1, (0, 2, 1): -1, (2, 1, 0): -1, (1, 0, 2): -1}
    out = np.zeros((8, 8), dtype=np.complex128)
    for (a, b, c), e in eps.items():
        out += e * _kron(S[a], S[b], S[c])
    return out


def _nn_bonds(Lx, Ly):
    bonds = []
    for x in range(Lx):
        for y in range(Ly - 1):
            bonds.append((x * Ly + y, x * Ly + y + 1))
    for x in range(Lx - 1):
        for y in range(Ly):
            bonds.append((x * Ly + y, (x + 1) * Ly + y))
    return bonds


def heisenberg(lat: Lattice, J: float = 1.0):
    """H = J sum_<ij> S_i . S_j over the open-boundary nearest-neighbour bonds."""
    h = J * _sdots()
    terms = [((i, j), h.copy()) for (i, j) in _nn_bonds(lat.Lx, lat.Ly)]
    return {"terms": terms, "pairs": [], "onsite": np.zeros((lat.nsites, lat.d))}


def j1j2_chiral(lat: Lattice, J1: float = 1.0, J2: float = 0.5, Jchi: float = 0.3):
    """J1 on nearest-neighbour bonds, J2 on both diagonals of every plaquette, and a three-spin
    chiral term Jchi * S_i . (S_j x S_k) on the four elementary triangles of every plaquette
    (two nearest-neighbour edges plus one diagonal).  Each triangle is listed counter-clockwise
    in the drawing plane (y to the right, x downwards)."""
    Ly = lat.Ly
    terms = [((i, j), J1 * _sdots()) for (i, j) in _nn_bonds(lat.Lx, lat.Ly)]
    chi = Jchi * _chirality()
    for x in range(lat.Lx - 1):
        for y in range(Ly - 1):
            tl, tr = x * Ly + y, x * Ly + y + 1
            bl, br = (x + 1) * Ly + y, (x + 1) * Ly + y + 1
            terms.append(((tl, br), J2 * _sdots()))
            terms.append(((tr, bl), J2 * _sdots()))
            # counter-clockwise with the drawing's up = -x: tl -> bl -> br is counter-clockwise
            for tri in ((tl, bl, br), (tl, bl, tr), (tl, br, tr), (bl, br, tr)):
                terms.append((tri, chi.copy()))
    return {"terms": terms, "pairs": [], "onsite": np.zeros((lat.nsites, lat.d))}


def _cyclic_permutation4(d: int = 2):
    """P on four sites in their listed order: P |s1 s2 s3 s4> = |s4 s1 s2 s3> (the local state of
    site k moves to site k + 1, that of site 4 to site 1).  Matrix element order <out|P|in>."""
    P = np.zeros((d ** 4, d ** 4))
    for a in range(d ** 4):
        s1, s2, s3, s4 = (a // d ** 3) % d, (a // d ** 2) % d, (a // d) % d, a % d
        b = ((s4 * d + s1) * d + s2) * d + s3
        P[b, a] = 1.0
    return P


CSL_J1 = 2.0 * math.cos(0.06 * math.pi) * math.cos(0.14 * math.pi)
CSL_J2 = 2.0 * math.cos(0.06 * math.pi) * math.sin(0.14 * math.pi)
CSL_LAMBDA = 2.0 * math.sin(0.06 * math.pi)


def csl(lat: Lattice, J1: float = CSL_J1, J2: float = CSL_J2, lam: float = CSL_LAMBDA):
    """The chiral-spin-liquid model of Eq. (CSL_Model): J1 on nearest-neighbour bonds, J2 on both
    diagonals of every plaquette, and i lam (P_ijkl - P_ijkl^-1) on every plaquette, P the cyclic
    permutation of the four local states, the corners listed counter-clockwise in the drawing
    plane (y to the right, x downwards: top-left, bottom-left, bottom-right, top-right).  The
    default couplings are the values at which the paper's ground state is a chiral spin liquid."""
    Ly = lat.Ly
    P = _cyclic_permutation4(lat.d)
    ring = 1j * lam * (P - P.T)
    terms = [((i, j), J1 * _sdots()) for (i, j) in _nn_bonds(lat.Lx, lat.Ly)]
    for x in range(lat.Lx - 1):
        for y in range(Ly - 1):
            tl, tr = x * Ly + y, x * Ly + y + 1
            bl, br = (x + 1) * Ly + y, (x + 1) * Ly + y + 1
            terms.append(((tl, br), J2 * _sdots()))
            terms.append(((tr, bl), J2 * _sdots()))
            terms.append(((tl, bl, br, tr), ring.copy()))
    return {"terms": terms, "pairs": [], "onsite": np.zeros((lat.nsites, lat.d))}


def spin_bonds(lat: Lattice, J1: float = 1.0, J2: float = 0.0):
    """(i, j, J) for the J1 nearest-neighbour bonds and, when J2 != 0, both diagonals of every
    plaquette with J2: the bonds of the Heisenberg-type H = sum_b J_b S_i . S_j."""
    out = [(i, j, J1) for (i, j) in _nn_bonds(lat.Lx, lat.Ly)]
    if J2 != 0.0:
        Ly = lat.Ly
        for x in range(lat.Lx - 1):
            for y in range(Ly - 1):
                out.append((x * Ly + y, (x + 1) * Ly + y + 1, J2))
                out.append((x * Ly + y + 1, (x + 1) * Ly + y, J2))
    return out


def axis_bases():
    """For alpha = x, y, z the unitary V_alpha whose column s is the eigenvector of sigma^alpha
    with eigenvalue +1 (s = 0) or -1 (s = 1), so that S^alpha acts as m_s = 1/2 - s on the
    rotated basis state |s>_alpha = V_alpha[:, s]."""
    r = 1.0 / np.sqrt(2.0)
    return [np.array([[r, r], [r, -r]], dtype=np.complex128),
            np.array([[r, r], [1j * r, -1j * r]], dtype=np.complex128),
            np.eye(2, dtype=np.complex128)]


def axis_parts(lat: Lattice, bonds):
    """H = sum_b J_b S_i . S_j split as H_x + H_y + H_z, H_alpha = sum_b J_b S^alpha_i S^alpha_j,
    each written as a diagonal Hamiltonian of its own rotated basis (Sec. "On reusing
    environments": terms diagonal in a rotated basis need no amplitude ratios).  With
    m_s = 1/2 - s:  J m_s m_s' = J (s s' - s/2 - s'/2 + 1/4), i.e. a pair J, on-site -J/2 on
    state 1 of both sites and +J/4 on both states of site i.  Returns [(V_alpha, H_alpha)]
    for alpha = x, y, z, the H_alpha in this module's Hamiltonian format (no terms)."""
    pairs = [(i, j, float(J)) for (i, j, J) in bonds]
    onsite = np.zeros((lat.nsites, lat.d))
    for (i, j, J) in bonds:
        onsite[i, 1] -= 0.5 * J
        onsite[j, 1] -= 0.5 * J
        onsite[i, :] += 0.25 * J
    return [(V, {"terms": [], "pairs": list(pairs), "onsite": onsite.copy()}) for V in axis_bases()]


def rydberg(lat: Lattice, omega: float = 1.0, delta: float = 3.0, Rb: float = 1.7, rmax: float = 4.0):
    """H = (Omega/2) sum_i sigma^x_i - delta sum_i n_i + sum_{i<j, r_ij <= rmax} V0 / r_ij^6 n_i n_j,
    V0 = Omega * Rb^6, lattice spacing 1, each unordered pair once."""
    sx, _, _ = pauli()
    N = lat.nsites
    terms = [((i,), 0.5 * omega * sx) for i in range(N)]
    onsite = np.zeros((N, lat.d))
    onsite[:, 1] = -delta
    V0 = omega * Rb ** 6
    pairs = []
    for i in range(N):
        xi, yi = divmod(i, lat.Ly)
        for j in range(i + 1, N):
            xj, yj = divmod(j, lat.Ly)
            r = math.hypot(xi - xj, yi - yj)
            if r <= rmax + 1e-12:
                pairs.append((i, j, V0 / r ** 6))
    return {"terms": terms, "pairs": pairs, "onsite": onsite}


# ----------------------------------------------------------------------------- named workloads

WORKLOADS = {
    # 4x4 open Heisenberg, D=2, chi=4 (exact), uniform Sz=0 configurations, one MinSR step
    "heis4x4_D2_chi4": dict(Lx=4, Ly=4, d=2, D=2, chi=4, ns=256, init=dict(kind="normal", scale=1.0),
                             seed_theta=1001, seed_S=2001, lam=1e-4, rcond=0.0, tau=0.05),
    # 8x8 open Heisenberg, D=4, chi=16, biased Gaussian tensors with the algebraically decaying
    # virtual legs of Eq. (A_alpha) (alpha = 1.5, the paper's initialisation for optimisation
    # runs), Metropolis exchange chains
    "heis8x8_D4_chi16": dict(Lx=8, Ly=8, d=2, D=4, chi=16, ns=4096,
                              init=dict(kind="normal", scale=0.5, bias=1.0, alpha=1.5),
                              seed_theta=1002, seed_S=2002, seed_chain=3002, lam=1e-4, rcond=0.0, tau=0.05),
    # 12x12 Rydberg array, D=4, chi=24, tensors drawn as for the 8x8 Heisenberg workload
    "rydberg12x12_D4_chi24": dict(Lx=12, Ly=12, d=2, D=4, chi=24, ns=16384,
                                   init=dict(kind="normal", scale=0.5, bias=1.0, alpha=1.5),
                                   seed_theta=1004, seed_S=2004, seed_chain=3004, lam=1e-4, rcond=0.0, tau=0.05),
}


# ----------------------------------------------------------------------------- learned proposal

PROPOSAL_CHANNELS = 16


def proposal_init(seed: int, C: int = PROPOSAL_CHANNELS, scale: float = 1.0):
    """Seeded initial weights of the 3-layer 3x3 convolutional proposal network, packed in one
    float64 vector: W1 (C,1,3,3), b1 (C), W2 (C,C,3,3), b2 (C), W3 (1,C,3,3), b3 (1).
    Entries N(0, scale^2 / fan_in), biases zero."""
    rng = np.random.default_rng(seed)
    parts = [rng.standard_normal((C, 1, 3, 3)) * scale / 3.0, np.zeros(C),
             rng.standard_normal((C, C, 3, 3)) * scale / math.sqrt(9.0 * C), np.zeros(C),
             rng.standard_normal((1, C, 3, 3)) * scale / math.sqrt(9.0 * C), np.zeros(1)]
    return np.concatenate([p.ravel() for p in parts])


def proposal_shapes(C: int = PROPOSAL_CHANNELS):
    return [(C, 1, 3, 3), (C,), (C, C, 3, 3), (C,), (1, C, 3, 3), (1,)]

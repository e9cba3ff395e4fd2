"""Counted arithmetic of the kernels as written (flops = 2 per multiply-add), used for the
roofline figures.  Each formula follows the loop nests of the kernel it names; the one-sided
Jacobi part uses the sweep / rotation counts the library records (peps_timing_read counters).

Notation: chi = boundary bond D_c, D = PEPS bond, n = chi*D (exact product bond),
Lr = D*chi (row length of the truncation matrix X), mX = n rounded up to even.
"""
from __future__ import annotations


def _dims(chi, D):
    n = chi * D
    return n, D * chi, n + (n & 1)


def row_step_flops(chi, D, Ly):
    """One truncating boundary-MPS row step without the Jacobi sweeps (env_row_step)."""
    n, Lr, mX = _dims(chi, D)
    left = (Ly - 1) * (2 * n * D * D * chi * chi            # W = R . E
                       + 2 * n * n * D ** 3                  # Z = W . A
                       + 2 * (n * D) * n * n - 2 * n ** 3 / 3)  # Householder R of Z (n*D x n)
    right_site = (2 * chi ** 3 * D * D                      # P = E . C
                  + 2 * n * Lr * D * D                       # Y = P . A
                  + n * (n + 1) * Lr                         # X = R . Y (R upper triangular)
                  + 2 * mX * Lr                              # row norms
                  + 2 * n * chi * Lr)                        # C = Y . V
    right = (Ly - 1) * right_site + 2 * chi ** 3 * D * D     # + first site
    return left + right


def jacobi_flops(chi, D, sweeps, rotations):
    """One-sided Jacobi work from the recorded counters: every sweep recomputes the mX row
    norms (2 Lr flops each), every pair check is one dot product of length Lr (2 Lr flops; the
    norms are carried by Rutishauser's update), every rotation updates two rows (6 Lr flops)."""
    n, Lr, mX = _dims(chi, D)
    checks = sweeps * (mX // 2) * (mX - 1)
    return 2 * Lr * checks + 6 * Lr * rotations + 2 * mX * Lr * sweeps


def env_flops(Lx, Ly, chi, D, ns, sides, sweeps, rotations):
    """k_env: (Lx-2) truncating row steps per side per sample, plus the Jacobi work."""
    return ns * sides * (Lx - 2) * row_step_flops(chi, D, Ly) + jacobi_flops(chi, D, sweeps, rotations)


def absorb1_flops(chi, D):
    return 4 * chi ** 3 * D * D + 2 * chi * chi * D ** 4


def absorb2_flops(chi, D):
    return 4 * D ** 3 * chi ** 3 + 4 * D ** 5 * chi * chi


def row_kernel_flops(Lx, Ly, chi, D, ns, want_O, windows1=0):
    """k_row over all Lx rows: right and left partials, site environments for O, and
    `windows1` one-column window absorptions (E_loc terms) in total."""
    per_row = 2 * Ly * absorb1_flops(chi, D)
    if want_O:
        per_row += Ly * (4 * chi ** 3 * D * D + 2 * chi * chi * D ** 4)
    return ns * Lx * per_row + windows1 * absorb1_flops(chi, D)


def pair_kernel_flops(Lx, Ly, chi, D, ns, windows2=0):
    return ns * (Lx - 1) * 2 * Ly * absorb2_flops(chi, D) + windows2 * absorb2_flops(chi, D)


def heisenberg_windows(Lx, Ly, ns, frac_antiparallel=0.5):
    """Expected window absorptions of the Heisenberg E_loc: horizontal bonds with unequal
    spins take two one-row columns, vertical bonds one two-row column."""
    h = Lx * (Ly - 1) * frac_antiparallel * 2 * ns
    v = (Lx - 1) * Ly * frac_antiparallel * ns
    return h, v


def sample_flops(Lx, Ly, chi, D, nchains, nsweeps, sweeps, rotations, move="exchange", acc_frac=0.5, passes=None):
    """The sampler per chain: every sweep rebuilds one environment side row by row (Lx-2
    steps); `passes` full passes of the other side (Lx-2 steps each) open the downward sweeps
    and an upward sweep that starts a call (default: one per sweep); per row the right partials,
    the running left partial and the proposal windows; the Jacobi work comes from the counters."""
    passes = nsweeps if passes is None else passes
    steps = (nsweeps + passes) * (Lx - 2) * row_step_flops(chi, D, Ly)
    rows = Lx * (2 * Ly) * absorb1_flops(chi, D)
    props = Lx * (Ly - 1) * acc_frac * 2 * absorb1_flops(chi, D)
    if move == "exchange":
        rows += (Lx - 1) * 2 * Ly * absorb2_flops(chi, D)
        props += (Lx - 1) * Ly * acc_frac * absorb2_flops(chi, D)
    return nchains * (steps + nsweeps * (rows + props)) + jacobi_flops(chi, D, sweeps, rotations)


def gram_flops(ns, npar):
    """k_gram computes the lower-triangle 64x64 tiles in full: about (Ns^2/2 + 32 Ns) Np MACs."""
    nt = (ns + 63) // 64
    return 2.0 * (nt * (nt + 1) // 2) * 64 * 64 * npar


# pipe operations per algorithmic multiply-add of each Gram kernel, counted as flops (2 per
# issued FMA-pipe operation, so that the figure compares with the FMA peaks): FP64 one FMA;
# split-BF16 three tensor products; float-float 13 FP32 operations (product and its FMA error,
# the two cross terms, Knuth's two-sum, three adds into the low word)
GRAM_PIPE_OPS = {0: 1, 1: 3, 2: 13}


def gram_pipe_flops(ns, npar, gram):
    return gram_flops(ns, npar) * GRAM_PIPE_OPS[gram]

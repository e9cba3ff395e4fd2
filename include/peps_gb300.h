/*
 * peps_gb300.h -- C ABI of the GB300 (sm_103a) hot path of the sampling-based finite-PEPS
 * optimiser of arXiv:2503.12557.
 *
 * What the library computes, per configuration S of an Lx x Ly open-boundary PEPS with physical
 * dimension d and virtual dimension D (paper Sec. "Finite PEPS and Sampling", Eq. (PsiS)):
 *   - the boundary-MPS environments E^u[x], E^l[x] of the single-layer network projected on S,
 *     truncated back to bond dimension chi after every MPS-MPO product (Sec. "On the boundary
 *     MPS method"), every tensor divided by its largest modulus with the logarithms kept
 *     (Sec. "On Numerical Stability");
 *   - ln psi(S) (Eq. (boundary_MPS_approx));
 *   - the local energy E_loc(S) = sum_S' <S|H|S'> psi(S')/psi(S) with environment reuse
 *     (Eq. (local_obs), Sec. "On reusing environments"); diagonal terms cost no contraction;
 *   - the log-derivatives O_{S,k} = d ln psi(S) / d theta_k (Sec. "Reformulation of the
 *     imaginary-time Schroedinger equation", Eq. (tdvp));
 *   - the MinSR update dtheta = -tau Obar^dag (Obar Obar^dag + lambda)^+ ebar (Eq. (tdvp_fast));
 *   - Metropolis chains over S whose acceptance uses the same environment-reusing ratios.
 *
 * Conventions
 *   Sites (x, y), x = 0..Lx-1 top to bottom, y = 0..Ly-1, linear index x*Ly + y.
 *   Site tensor T[x,y][s, l, u, r, d]; legs pointing out of the lattice have dimension 1.
 *   theta: all site tensors in C order, concatenated in site order (length N_p, see
 *   peps_num_params).  O rows use the same order.
 *   Configurations: uint8, Ns x (Lx*Ly), row major, values 0..d-1 (a value outside that range
 *   is invalid input; the kernels read it as 0 rather than index out of bounds).
 *   Every pointer argument named *_dev is DEVICE memory owned by the caller; the library never
 *   frees or keeps it beyond the call.  Host pointers are named *_host.
 *   Every call is asynchronous on the caller's CUDA stream (passed as void*, a cudaStream_t;
 *   NULL = legacy default stream).  Argument errors are reported before any launch.
 *   Per-sample numerical problems are status bits written to status_dev (0 = clean):
 *     PEPS_ST_NEAR_DEGENERATE  a truncation cut where the kept and the first discarded singular
 *                              value differ by less than 1e-8 sigma_1 (and the latter is above
 *                              1e-12 sigma_1): the truncated state is not unique there;
 *     PEPS_ST_ZERO_NORM        an environment tensor or partial contraction was exactly zero;
 *     PEPS_ST_NONFINITE        a NaN or Inf appeared (ln psi, E_loc or O of that sample invalid);
 *     PEPS_ST_NOCONV           a one-sided Jacobi SVD hit its sweep limit.
 *   Nothing traps on the device; non-finite parameters or inputs give NaN results and
 *   PEPS_ST_NONFINITE, never an out-of-bounds access.
 */
#ifndef PEPS_GB300_H
#define PEPS_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PEPS_OK = 0,
    PEPS_W_NUMERIC = 1,     /* peps_last_status: a numerical warning since the last read
                               (per-sample status bits, or a MinSR breakdown: dtheta
                               was set to zero, info[0] = -1)                          */
    PEPS_E_ARG = -1,        /* NULL pointer, negative size, bad enum value            */
    PEPS_E_SHAPE = -2,      /* lattice / chi / Ns outside what the handle supports     */
    PEPS_E_WORKSPACE = -3,  /* device allocation failed                                */
    PEPS_E_CUDA = -4,       /* a CUDA runtime call failed (peps_last_error has detail) */
    PEPS_E_UNSUPPORTED = -5, /* option combination not implemented                     */
    PEPS_E_CAPACITY = -6    /* peps_amplitudes_noalloc: the problem needs more than its
                               fixed 32 MiB device scratch array                       */
} peps_status;

enum {
    PEPS_ST_NEAR_DEGENERATE = 1,
    PEPS_ST_ZERO_NORM = 2,
    PEPS_ST_NONFINITE = 4,
    PEPS_ST_NOCONV = 8
};

/* Bits of a handle's status word beyond the per-sample PEPS_ST_* bits (peps_last_status). */
enum {
    PEPS_SW_MINSR_BREAKDOWN = 1 << 8,  /* a minsr_step found T + lambda not positive definite in
                                          floating point; its dtheta was set to zero            */
    PEPS_SW_GRAM_TIMEOUT = 1 << 9      /* a tensor-core Gram gave up on a pipeline wait; its
                                          dtheta was set to zero                                */
};

/* Arithmetic of the contraction kernels.  FP64: every step in double.  FP32: the environment,
 * truncation and sandwich arithmetic in float, logarithms and E_loc accumulated in double.
 * MIXED: the reduced-precision preset of the whole step: the FP32 contraction kernels (CUDA
 * cores; logarithms, E_loc and O's scale in double), the MinSR Gram as float-float pairs on the
 * FP32 pipes (cfg.gram == 0 becomes 2; 1 keeps the split-BF16 tensor-core Gram) and the solve as
 * a float-float Cholesky with FP64 refinement and an FP64 fallback (cfg.solve becomes 2); the
 * handle then reports FP32 (its O is float). */
typedef enum { PEPS_PREC_FP64 = 0, PEPS_PREC_FP32 = 1, PEPS_PREC_MIXED = 2 } peps_prec;

typedef enum { PEPS_MOVE_EXCHANGE = 0, PEPS_MOVE_FLIP = 1 } peps_move;

typedef struct {
    int Lx, Ly;   /* lattice, Lx >= 2, Ly >= 2                                              */
    int d;        /* physical dimension, 2 <= d <= 4                                         */
    int D;        /* virtual bond dimension, 1 <= D <= 8                                     */
    int chi;      /* boundary-MPS bond dimension D_c (paper's notation), D <= chi <= 64      */
    int prec;     /* peps_prec                                                               */
    int max_samples; /* largest Ns any later call may pass (sizes the environment store)     */
    int gram;     /* MinSR Gram matrix: 0 = FP64 on CUDA cores; 1 = split BF16 on the tcgen05
                     tensor cores (Obar = hi + lo, T ~ hi hi^T + hi lo^T + lo hi^T, FP32
                     accumulation; about 1e-5 relative error per entry); 2 = float-float on
                     the FP32 pipes (Obar = hi + lo in floats, exact hi products by FMA plus the
                     cross terms, sums kept as float pairs; about 48 significant bits, for
                     GPUs whose FP64 rate is a small fraction of their FP32 rate)          */
    int solve;    /* MinSR solve when rcond == 0: 0 = FP64 Cholesky; 1 = FP32 Cholesky of
                     T + lambda followed by 4 steps of iterative refinement with FP64 residuals
                     (info[1] reports the final relative residual); 2 = float-float Cholesky
                     (T + lambda as float pairs of about 48 bits, the trailing updates on the
                     FP32 pipes, diagonal blocks and panels in FP64) followed by 2 steps of
                     refinement with FP64 residuals: the FP64 factor's work at a fraction of
                     its time on GPUs whose FP64 rate is a small fraction of their FP32 rate;
                     3 = FP64 Cholesky when rcond == 0, and the tridiagonal eigen route (see
                     minsr_step) instead of the cyclic Jacobi when rcond > 0 */
    int cplx;     /* 0 = real PEPS; 1 = complex PEPS: theta is N_p (re, im) pairs of doubles,
                     O is N_s x N_p complex numbers in the handle's precision ((re, im) pairs
                     of doubles or floats), phases and E_loc are complex.  Not with gram = 1,
                     the learned proposal or peps_amplitudes_noalloc (PEPS_E_UNSUPPORTED). */
    double trunc_weight; /* 0: every truncation keeps min(chi, rank) singular values.  > 0: the
                     truncated-weight rule of Sec. "On the boundary MPS method" (the paper uses
                     1e-4): each cut keeps the fewest singular values, at most chi, whose
                     discarded share of sum sigma^2 is at most trunc_weight (the bond stays
                     padded to chi with zeros).  A cut whose boundary share lies within 1e-9
                     (relative) of trunc_weight is flagged PEPS_ST_NEAR_DEGENERATE.  In [0, 1). */
} peps_config;

/* One local Hamiltonian term: h is a d^k x d^k complex matrix, row major, interleaved
 * (re, im) doubles, h[a][b] = <S_loc = a| h |S'_loc = b>, local index a = sum_i s_{sites[i]}
 * d^(k-1-i).  The sites must lie in one row, or in two adjacent rows, and span at most two
 * adjacent columns (nearest-neighbour bonds, plaquette diagonals, plaquette triangles,
 * single sites). */
typedef struct {
    int nsites;          /* k, 1..4 */
    int sites[4];
    const double* h_host;
} peps_term;

/* H = sum_terms h + sum_pairs v s_i s_j + sum_i onsite[i][s_i].  All host memory, read during
 * the call that receives it. */
typedef struct {
    int nterms;
    const peps_term* terms;
    int npairs;
    const int* pair_ij_host;     /* npairs x 2 site indices                  */
    const double* pair_v_host;   /* npairs coefficients                      */
    const double* onsite_host;   /* (Lx*Ly) x d, may be NULL                 */
} peps_hamiltonian;

typedef struct peps_handle peps_handle;

/* Create a handle for one lattice / chi / precision.  Allocates the parameter copy and the
 * environment store for cfg->max_samples configurations on the current CUDA device.
 * Returns PEPS_E_SHAPE when the sizes are outside the limits stated in peps_config. */
peps_status peps_create(peps_handle** out, const peps_config* cfg);

/* Device-memory callbacks of a handle (peps_create_ex): alloc(ctx, bytes) returns device memory
 * of the current device, aligned to 256 bytes, or NULL on failure; free(ctx, ptr) returns it.
 * The handle calls them at creation (parameter copy, environment store, scratch) and when a
 * later call first needs a workspace (MinSR, direct sampling, the bound estimator, the
 * learned proposal, Hamiltonian tables), never during a stream capture of a call whose
 * workspace already exists, and frees everything through free() in peps_destroy.  Memory that
 * free() releases may be reused by the allocator in the order of the stream the handle's calls
 * ran on. */
typedef struct {
    void* (*alloc)(void* ctx, size_t bytes);
    void (*free)(void* ctx, void* ptr);
    void* ctx;
} peps_allocator;

/* As peps_create, with every device allocation of the handle made through *alloc (copied; NULL
 * = cudaMalloc / cudaFree).  PEPS_E_ARG when a callback is NULL; PEPS_E_WORKSPACE when alloc
 * returns NULL. */
peps_status peps_create_ex(peps_handle** out, const peps_config* cfg, const peps_allocator* alloc);
peps_status peps_destroy(peps_handle* h);

/* The handle's status word: the OR of the per-sample status bits (PEPS_ST_*) of every sample of
 * every evaluation, sampling or estimator call, and of the PEPS_SW_* flags of every minsr_step,
 * since the last peps_last_status (or creation).  Synchronises `stream` (the stream those calls
 * ran on), writes the word to *word_host (may be NULL) and clears it.  Returns PEPS_E_CUDA when
 * PEPS_SW_GRAM_TIMEOUT is set, PEPS_W_NUMERIC when any other bit is set, else PEPS_OK: the
 * numerical warnings of the asynchronous calls, read when the caller chooses to synchronise. */
peps_status peps_last_status(peps_handle* h, int32_t* word_host, void* stream);

/* w_dev[i] = 0 where status_dev[i] & mask, else 1 (Ns doubles, device): weights for minsr_step
 * that leave out the samples a status bit marks (no counterpart in the paper). */
peps_status peps_status_weights(const int32_t* status_dev, int Ns, int mask, double* w_dev, void* stream);

/* N_p = sum over sites of d * Dl * Du * Dr * Dd (boundary legs of dimension 1). */
long long peps_num_params(const peps_handle* h);

/* Copy theta (N_p doubles, or N_p (re, im) pairs of doubles for a complex PEPS; device) into the
 * handle's padded kernel layout (converted to the
 * handle's precision).  Later calls use this copy until the next peps_set_params. */
peps_status peps_set_params(peps_handle* h, const double* theta_dev, void* stream);

/* ln|psi_top(S)| and its phase (0 or pi for a real PEPS), psi_top = E^u[Lx-2] . T_proj[Lx-1]
 * (Eq. (boundary_MPS_approx) with i = Lx-1).  logabs_dev, phase_dev: Ns doubles;
 * status_dev: Ns int32. */
peps_status peps_amplitudes(peps_handle* h, const uint8_t* S_dev, int Ns,
                            double* logabs_dev, double* phase_dev, int32_t* status_dev, void* stream);

/* E_loc(S) (Eq. (local_obs)) for every configuration; eloc_dev: Ns x 2 doubles (re, im).
 * A term inside row x uses psi_x = E^u[x-1] . T_proj[x] . E^l[x+1] for S and S'; a term over
 * rows x, x+1 uses psi_{x,x+1} = E^u[x-1] . T_proj[x] . T_proj[x+1] . E^l[x+2]. */
peps_status peps_local_energy(peps_handle* h, const peps_hamiltonian* H, const uint8_t* S_dev, int Ns,
                              double* eloc_dev, int32_t* status_dev, void* stream);

/* O_{S,k} (Ns x N_p, row major) in the handle's precision: double for FP64, float for FP32.
 * O_{S,k} = delta_{s, s_xy} Env_xy[l,u,r,d] / psi_x(S) for k = (x, y, s, l, u, r, d). */
peps_status peps_logderiv(peps_handle* h, const uint8_t* S_dev, int Ns, void* O_dev,
                          int32_t* status_dev, void* stream);

/* All of the above from one environment pass: any of logabs/phase/eloc/O may be NULL
 * (H must be non-NULL when eloc_dev is).  With a diagonal H (pairs and on-site terms only)
 * and logabs, phase and O all NULL, E_loc needs no amplitude and no contraction runs (the
 * status bits are then all 0). */
peps_status peps_evaluate(peps_handle* h, const peps_hamiltonian* H, const uint8_t* S_dev, int Ns,
                          double* logabs_dev, double* phase_dev, double* eloc_dev, void* O_dev,
                          int32_t* status_dev, void* stream);

/* Reuse of cached environments between sampling and evaluation (Sec. "On reusing environments";
 * opt-in, off by default).  Sweeps alternate direction (even sweep ids down the rows, odd ones
 * up); after a sweep of the FP32 real-PEPS sampler the environments it rebuilt row by row
 * (E^u[0..Lx-2] going down, E^l[1..Lx] going up) are those of the final configurations (every
 * row is final once its own moves are done).  With enable = 1, a peps_evaluate /
 * peps_local_energy / peps_amplitudes / peps_logderiv call whose S_dev and Ns are those of the
 * last peps_sample on this handle, with no parameter change (peps_set_params /
 * peps_apply_update) and no other call that rewrites the environments in between, takes that
 * side from the store and contracts only the other one (peps_amplitudes after a downward
 * sweep: nothing); the status bits of the reused row steps come from the sampler's last sweep.  The caller promises that S_dev was not modified in
 * between.  Results equal those of a full evaluation.  Other precisions and complex handles
 * always recompute.  PEPS_E_ARG for enable outside {0, 1}. */
peps_status peps_set_env_reuse(peps_handle* h, int enable);

/* Direct sampling (Sec. "On Direct Sampling" and the appendix "Direct sampling of PEPS",
 * Alg. `sampling`): independent configurations drawn row by row from the conditional reduced
 * density matrix rho_{S<i}[i] = T^u . D^l[i+1] . T^u*, with T^u = E^u[i-1](S) . T[i] (kept
 * exact) and D^l the double-layer lower boundary MPS.
 * peps_direct_prepare builds D^l[2..Lx] for the parameters last set (one CTA; once per
 * parameter set, reused by every later peps_direct_sample), compressed to chi_double
 * (1 <= chi_double, chi_double D^2 <= 1024; the paper's D_c^double ~ D).  Environments from
 * earlier parameters are allowed: p(S) stays a normalised distribution and the importance
 * weights |psi(S)|^2 / p(S) correct for them. */
peps_status peps_direct_prepare(peps_handle* h, int chi_double, void* stream);
/* peps_direct_sample: Ns configurations (S_dev: Ns x Lx Ly, written) and log p(S) (logp_dev:
 * Ns doubles, the sum of the logs of the drawn conditionals), chain c of draw round `draw`
 * taking its uniforms from Philox4x32-10 at counters (x Ly + y, draw, c, 2) with key seed.
 * A conditional weight below zero (truncated D^l) counts as zero; a site whose weights all
 * vanish is drawn uniformly and sets PEPS_ST_ZERO_NORM.  Ns <= cfg.max_samples.  The
 * importance weight of S for the estimators is |psi(S)|^2 / p(S) (psi from peps_amplitudes). */
peps_status peps_direct_sample(peps_handle* h, uint8_t* S_dev, int Ns, uint64_t seed, uint64_t draw,
                               double* logp_dev, int32_t* status_dev, void* stream);

/* Global rotation of the physical index (Sec. "On reusing environments": a Hamiltonian term
 * diagonal in a rotated basis is evaluated on the PEPS rotated into that basis, sampled on
 * its own).  theta_out[site][s][l,u,r,d] = sum_t M[s][t] theta_in[site][t][l,u,r,d] over the
 * compact N_p layout of h's lattice.  M_host: d x d complex, row major, (re, im) pairs (for the
 * amplitudes <S_alpha|psi> in the basis |s>_alpha = V[:, s], M = V^dagger).  theta_in_dev: N_p
 * doubles (in_cplx = 0) or N_p (re, im) pairs (in_cplx = 1); theta_out_dev: N_p (re, im) pairs
 * (written; must not alias the input).  Feed it to a complex handle (cfg.cplx = 1). */
peps_status peps_rotate_params(const peps_handle* h, const double* M_host, const double* theta_in_dev,
                               int in_cplx, double* theta_out_dev, void* stream);

/* Variational-bound local energy (Sec. "On Variational Upper Bound to the Ground State Energy"
 * and the appendix on variational upper bounds).  One cut i (1 <= cut <= Lx-1, the paper's
 * row index: the upper boundary MPS holds rows 1..i) fixes every amplitude to
 *   psi_i(S) = E^u[i](S) . E^l[i+1](S)
 * (the plain overlap of the two boundary MPS, no conjugation), and
 *   E_loc^bound(S) = sum_S' <S|H|S'> psi_i(S') / psi_i(S),
 * whose |psi_i|^2-weighted mean is the energy <psi_i|H|psi_i> / <psi_i|psi_i> of one state,
 * an upper bound of the ground-state energy.  For every off-diagonal S' the environments
 * are rebuilt (truncated as in peps_amplitudes) on the rows between the first row S' changes
 * and the cut, from S's environments; this costs up to Lx/2 row steps per off-diagonal term.
 * eloc_dev: Ns x 2 doubles (re, im); logabs_dev, phase_dev: ln|psi_i(S)| and its phase (each
 * may be NULL); status_dev: as peps_evaluate, also collecting the bits of every S' row step.
 * Same term restrictions as peps_local_energy; PEPS_E_ARG for a cut outside 1 .. Lx-1. */
peps_status peps_local_energy_bound(peps_handle* h, const peps_hamiltonian* H, const uint8_t* S_dev, int Ns,
                                    int cut, double* eloc_dev, double* logabs_dev, double* phase_dev,
                                    int32_t* status_dev, void* stream);

/* MinSR step (Eq. (tdvp_fast)):
 *   w_S = w_dev[S] / sum w (uniform 1/Ns when w_dev is NULL);
 *   Obar = sqrt(w) (O - w^T O), ebar = sqrt(w) (Re E_loc - w^T Re E_loc);
 *   T = Obar Obar^T = V diag(Lambda) V^T;  kept = Lambda_i > rcond * max Lambda (all when rcond == 0);
 *   dtheta = -tau Obar^T V diag(kept / (Lambda + lambda)) V^T ebar.
 * O_dev: Ns x N_p in the handle's precision (as written by peps_logderiv); eloc_dev: Ns x 2
 * doubles (the real parts are used by a real PEPS, both by a complex one); dtheta_dev: N_p
 * doubles, or N_p (re, im) pairs for a complex PEPS (written).  A complex PEPS runs the same
 * steps on the real embedding W = [[Re Obar, -Im Obar], [Im Obar, Re Obar]] (W W^T is the real
 * form of the Hermitian T = Obar Obar^H), with the rank in info[0] counted once per eigenvalue;
 * info_dev: 4 doubles.  rcond > 0: the eigendecomposition with the cutoff, info = (rank kept,
 * min Lambda, max Lambda, iterations): with cfg.solve 0, 1 or 2 by cyclic Jacobi (iterations =
 * sweeps, -1 at the sweep limit); with cfg.solve == 3 without forming V: Householder reduction of
 * T to tridiagonal form, implicit QR steps with a Wilkinson shift on the tridiagonal form
 * applied to the transformed ebar (the rotations recorded, one double each, in the handle's
 * workspace, then replayed in reverse), and the reflectors applied back (iterations = QR steps;
 * info[0] = -1 and a breakdown as below when an eigenvalue needs more than 60 steps or the
 * record outgrows its 2 max(n^2, 4096) doubles, n = Ns rounded up to even).  The two routes keep
 * the same eigenvalues; their results differ by rounding, the tridiagonal route's error growing
 * as eps max(Lambda) / (smallest kept Lambda + lambda) (both are backward stable; Jacobi has the
 * higher relative accuracy on small eigenvalues).  The tridiagonal route needs about 2 Ns^3
 * FP64 flops in parallel launches against tens of Ns^3 for the Jacobi sweeps, but its QR chain
 * is one thread of sequential FP64 arithmetic, about 0.9 Ns^2 rotations: on a GPU whose FP64
 * rate is a small fraction of its FP32 rate that chain dominates (GB300: 3.2 s at 1024 rows,
 * 47 s at 4096, 184 s at 8192, against 0.37 s and 20 s for the Jacobi).  rcond == 0 (nothing cut, lambda > 0): the same
 * operator (T + lambda)^-1 applied through a Cholesky factorisation, info = (Ns, NaN, NaN, -1)
 * with cfg.solve == 0, info = (Ns, |ebar - (T + lambda) x| / |ebar|, refinement steps, -1)
 * with cfg.solve == 1, where refinement steps = 0 means that the FP32 factor failed or the
 * refined residual stayed above 1e-10 and the FP64 factorisation was used instead; the same
 * with cfg.solve == 2, where the FP64 factorisation replaces the float-float one only when the
 * latter breaks down (a pivot that is not positive).  When T +
 * lambda is not positive definite in floating point even in FP64 (lambda far below the
 * rounding error of T, e.g. a split-BF16 Gram of badly scaled O), info[0] = -1, dtheta_dev is
 * set to zero and the status word gets PEPS_SW_MINSR_BREAKDOWN (peps_last_status then returns
 * PEPS_W_NUMERIC).  Needs lambda > 0 or rcond > 0.  The Gram matrix is FP64 (cfg.gram == 0), split
 * BF16 on the tensor cores (cfg.gram == 1) or float-float on the FP32 pipes (cfg.gram == 2);
 * the factorisation is FP64, FP32 or float-float (cfg.solve), the eigendecomposition FP64, the
 * residuals of the refinement FP64.  The call is
 * asynchronous like every other (no host round trip: the mixed solve's FP64 fallback and the
 * zeroing of dtheta on a breakdown are decided on the device; rcond > 0 runs the whole cyclic
 * Jacobi in one cooperative launch, or the tridiagonal route's launches, about 6 Ns of them); a
 * breakdown is reported by peps_last_status. */
peps_status minsr_step(peps_handle* h, const void* O_dev, const double* eloc_dev, const double* w_dev,
                       int Ns, double lambda, double rcond, double tau, double* dtheta_dev,
                       double* info_dev, void* stream);

/* ---- Sample-sharded MinSR: the step of minsr_step split at its exchange points, for samples
 * spread over several processes (one GPU each).  The paper parallelises over samples (Sec.
 * "Finite PEPS and Sampling"); MinSR then needs the exchange below.  With G processes, process g
 * holding N_g of the N_s = sum N_g samples and the parameter slice [c_g, c_{g+1}) of N_p:
 *   1. minsr_partial_sums on the local rows, summed over the processes (all-reduce, N_p + 2);
 *   2. minsr_center_rows: the local rows of Obar and ebar with those global sums (the same
 *      centring as minsr_step);
 *   3. exchange Obar's column slices (all-to-all): process g gets the N_s x K_g block A_g of
 *      its slice, rows in process order;
 *   4. minsr_gram on A_g, summed over the processes (all-reduce, N_s x N_s): T = Obar Obar^T;
 *   5. ebar gathered to all (N_s); minsr_solve on every process (same x everywhere);
 *   6. minsr_project: dtheta on the slice, gathered to all (all-gather).
 * The result equals minsr_step's on all N_s rows (up to the summation order of the reductions).
 * Real PEPS only (PEPS_E_UNSUPPORTED for a complex handle).  Asynchronous on `stream`.
 * minsr_partial_sums: O_dev (Ns x N_p, handle precision), eloc_dev (Ns x 2), w_dev (Ns or NULL =
 *   every weight 1; the weights need not be normalised); sums_dev (N_p + 2 doubles): column sums
 *   of w O, then sum w, then sum w Re E_loc.
 * minsr_center_rows: gsums_dev the sums added over every process; Obar_dev (Ns x N_p doubles) =
 *   sqrt(w_S / W) (O_S - m), ebar_dev (Ns) = sqrt(w_S / W) (Re E_loc(S) - e) with W the global
 *   sum of weights, m and e the global weighted means.
 * minsr_gram: T_dev (Ns x Ns doubles, written in full) = A A^T for A_dev (Ns x K doubles) in the
 *   handle's Gram mode (cfg.gram); K = 0 gives T = 0.
 * minsr_solve: x_dev (Ns) = (T + lambda)^+ ebar as minsr_step (Cholesky when rcond == 0, else the
 *   eigendecomposition with the cutoff), info_dev (4) as minsr_step; on a breakdown x is zero and
 *   the status word gets PEPS_SW_MINSR_BREAKDOWN.
 * minsr_project: dtheta_dev (K) = -tau A^T x (no handle needed). */
peps_status minsr_partial_sums(peps_handle* h, const void* O_dev, const double* eloc_dev, const double* w_dev, int Ns,
                               double* sums_dev, void* stream);
peps_status minsr_center_rows(peps_handle* h, const void* O_dev, const double* eloc_dev, const double* w_dev, int Ns,
                              const double* gsums_dev, double* Obar_dev, double* ebar_dev, void* stream);
peps_status minsr_gram(peps_handle* h, const double* A_dev, int Ns, long long K, double* T_dev, void* stream);
peps_status minsr_solve(peps_handle* h, const double* T_dev, const double* ebar_dev, int Ns, double lambda,
                        double rcond, double* x_dev, double* info_dev, void* stream);
peps_status minsr_project(const double* A_dev, const double* x_dev, int Ns, long long K, double tau,
                          double* dtheta_dev, void* stream);

/* theta_dev (N_p doubles, device, updated in place) += dtheta_dev, then the handle's kernel
 * copy is refreshed as by peps_set_params (the parameter update that closes an optimisation
 * step, paper Sec. "Reformulation of the imaginary-time Schroedinger equation"). */
peps_status peps_apply_update(peps_handle* h, double* theta_dev, const double* dtheta_dev, void* stream);

/* nsweeps Metropolis sweeps of Ns independent chains (configurations updated in place).
 * Sweep t has id sweep0 + t; an even id runs down the rows, an odd one up.  Downward sweep:
 * bottom environments of the current S; then for x = 0..Lx-1 the moves inside row x in column
 * order (exchange: bonds (x,y)-(x,y+1); flip: sites (x,y)) with psi_x ratios, then (exchange
 * only, x < Lx-1) the vertical bonds (x,y)-(x+1,y) with psi_{x,x+1} ratios, then E^u[x] from
 * the updated row.  Upward sweep: the upper environments of the current S (those the previous
 * sweep of the call left, else computed); then for x = Lx-1..0 the moves inside row x, then
 * (exchange only, x > 0) the vertical bonds (x-1,y)-(x,y) with psi_{x-1,x} ratios, then E^l[x]
 * from the updated row.  Slots are counted from 0 in this visiting order.  Move slot k of sweep t of chain c draws
 * u = Philox4x32-10(counter = (k, sweep0 + t, c, 0), key = seed) as a 53-bit double and
 * accepts iff u < |psi'/psi|^2.  accepted_dev: Ns int64, incremented by the accepted moves.
 * status_dev: Ns int32 (OR of the sweeps' status bits). */
peps_status peps_sample(peps_handle* h, int move, uint8_t* S_dev, int Ns, int nsweeps,
                        uint64_t seed, uint64_t sweep0, long long* accepted_dev,
                        int32_t* status_dev, void* stream);

/* Device timing of the library's own kernels, for profiling.  peps_timing_enable(h, 1) starts
 * recording a CUDA event pair around every launch the handle makes (on the call's stream) and
 * clears the record and the work counters; 0 stops recording.  peps_timing_read synchronises
 * with the recorded events and writes, for each kernel class i < n, the summed milliseconds
 * (ms_host[i]) and the kernel launches (launches_host[i]).  Classes: 0 environment pass,
 * 1 one-row sandwiches, 2 two-row sandwiches, 3 per-sample combine, 4 Metropolis sweeps,
 * 5 MinSR Gram matrix, 6 MinSR eigendecomposition, 7 MinSR centring / apply, 8 parameter copy.
 * counters_host (4 values, may be NULL): one-sided Jacobi sweeps, Jacobi rotations, truncation
 * SVDs performed since the last enable (the counted work behind the flop rates). */
peps_status peps_timing_enable(peps_handle* h, int enable);
peps_status peps_timing_read(peps_handle* h, double* ms_host, long long* launches_host, int n,
                             long long* counters_host);

/* ---- Learned proposal (required by the hot-path specification; not in the paper) ----------
 * Network: x = 1 - 2 s (one +-1 channel) -> conv3x3(1->C) -> SiLU -> conv3x3(C->C) -> SiLU ->
 * conv3x3(C->1) -> per-site logits l(S); zero padding at the open boundary; every conv has a
 * bias.  Weights packed W1 (C,1,3,3), b1 (C), W2 (C,C,3,3), b2 (C), W3 (1,C,3,3), b3 (1):
 * 9 C^2 + 20 C + 1 values.  wprec 0: double weights and activations; wprec 1: bf16
 * weights (__nv_bfloat16) with float activations.  Lx*Ly <= 256, 1 <= C <= 32. */

/* logits_dev (Ns x Lx*Ly doubles) = l(S) for every configuration. */
peps_status peps_proposal_logits(int Lx, int Ly, int C, int wprec, const void* w_dev, const uint8_t* S_dev, int Ns,
                                 double* logits_dev, void* stream);

/* One Adam step (beta 0.9 / 0.999, eps 1e-8, step count t >= 1) on the FP64 master weights
 * w_dev with moments m_dev, v_dev, for the loss mean_{S,i} softplus(l_i(S_in)) - t_i l_i(S_in)
 * over the Ns (S_in, S_tgt) pairs (the binary cross-entropy of the target given the input).
 * The gradient is taken at the weights the forward pass uses (w_dev for wprec 0, the bf16 copy
 * wlow_dev for wprec 1); wlow_dev, when not NULL, is refreshed from the updated master weights.
 * grad_dev: workspace of the weight count (holds the gradient afterwards); loss_dev: 1 double. */
peps_status peps_proposal_train_step(int Lx, int Ly, int C, int wprec, double* w_dev, double* m_dev, double* v_dev,
                                     void* wlow_dev, int t, double lr, const uint8_t* S_in_dev,
                                     const uint8_t* S_tgt_dev, int Ns, double* grad_dev, double* loss_dev,
                                     void* stream);

/* One network move of every chain: S' ~ prod_i Bernoulli(sigmoid(l_i(S))) with site i of chain c
 * drawn from u = Philox4x32-10(counter (i, step, c, 1), key seed); ln|psi_top(S')| from the
 * handle (as peps_amplitudes); accept iff u' < exp(min(0, 2 (ln|psi'| - ln|psi|) + log q(S|S')
 * - log q(S'|S))) with u' from counter (Lx*Ly, step, c, 1).  S_dev and logpsi_dev (the current
 * ln|psi_top(S)|) are updated in place; accepted_dev (Ns int64, may be NULL) is incremented. */
peps_status peps_sample_learned(peps_handle* h, int C, int wprec, const void* w_dev, uint8_t* S_dev,
                                double* logpsi_dev, int Ns, uint64_t seed, uint64_t step,
                                long long* accepted_dev, int32_t* status_dev, void* stream);

/* ln|psi_top(S)| and phase, as peps_amplitudes, for callers that cannot allocate device memory
 * (code running under another framework's allocator, which owns all device memory, or with a
 * device-memory budget fixed before this library is used).  This entry point has no
 * counterpart in the paper; it exists for those callers only.
 *   It needs no handle and calls no allocation routine: every intermediate lives in one
 *   32 MiB device array that the library reserves on every GPU it is loaded on until the
 *   process exits.  cfg gives the lattice, chi and precision (max_samples is ignored);
 *   theta_dev: N_p doubles; S_dev: Ns x (Lx*Ly) uint8; logabs_dev, phase_dev: Ns doubles;
 *   status_dev: Ns int32 or NULL.  All device memory owned by the caller.
 *   Returns PEPS_E_CAPACITY, before any launch, when the parameters, environments and one CTA's
 *   work buffers of this lattice and Ns do not fit in the 32 MiB (about 8 KiB per sample at
 *   4x4, D=2, chi=4 in FP64; larger problems need a handle).  Where two CTAs per SM do not fit,
 *   fewer CTAs share the samples: the same results, less concurrency.
 *   Every call made outside a stream capture looks up the array's device address with the
 *   current device (a cudaDeviceReset moves it); a call made during a capture uses the address
 *   of the last lookup, so make a first call on each device before any stream capture.  All
 *   calls share the array and leave their contents in it: calls that may overlap on the GPU
 *   race and must be serialised. */
peps_status peps_amplitudes_noalloc(const peps_config* cfg, const double* theta_dev, const uint8_t* S_dev, int Ns,
                                    double* logabs_dev, double* phase_dev, int32_t* status_dev, void* stream);

/* Autotuner (no counterpart in the paper).  For each kernel class (environments, one-row
 * sandwiches, two-row sandwiches, sampler) the shared-memory budget per CTA decides which work
 * buffers stay on chip and how many CTAs share an SM.  The call plans every candidate budget
 * (FP32: 72, 110, 220 KB; FP64: 100, 210 KB), runs peps_evaluate (with H when non-NULL) and
 * one sampler sweep of kind `move` on a copy of S_dev, times each class with CUDA events and
 * keeps the fastest budget per class for all later calls.  Results do not depend on the budget
 * (same arithmetic in the same order).  budget_kb_host: 4 ints written (may be NULL).  Allocates
 * temporary device memory (Ns x N_p outputs); synchronises the stream. */
peps_status peps_autotune(peps_handle* h, const peps_hamiltonian* H, const uint8_t* S_dev, int Ns, int move,
                          int* budget_kb_host, void* stream);

/* Multi-instance batch (no counterpart in the paper; the paper evaluates independent samples,
 * Sec. "Finite PEPS and Sampling", and a batch of independent PEPS is the same work with ragged
 * shapes): independent handles (different lattices, D, chi, sample counts) evaluated as one
 * peps_evaluate each, by one persistent kernel launch per scalar type over a work queue of
 * (instance, sample) items, costliest instances first (Lx Ly chi^3 D^3 per sample), each CTA
 * taking the next item with one atomic and running that sample's whole evaluation (both
 * environment sides, every one-row and two-row sandwich, the combine) with the device functions
 * of the per-handle kernels: the results equal the items' peps_evaluate calls bit for bit.  The
 * launches are recorded in one CUDA graph; the items' pointers are read again at every launch
 * (update the contents, not the pointers).  Each launch also ORs the items' status bits into
 * their handles' status words. */
typedef struct {
    peps_handle* h;              /* each handle at most once per batch; timing disabled      */
    const peps_hamiltonian* H;   /* NULL when eloc_dev is NULL                               */
    const uint8_t* S_dev;
    int Ns;                      /* 1 .. h's max_samples                                     */
    double* logabs_dev;
    double* phase_dev;
    double* eloc_dev;            /* may be NULL                                              */
    void* O_dev;                 /* may be NULL                                              */
    int32_t* status_dev;         /* may be NULL                                              */
} peps_batch_item;

typedef struct peps_batch peps_batch;

/* Runs every item once eagerly on `stream` (one-time uploads), then plans every instance's work
 * buffers at one shared-memory budget per CTA (budget_kb; 0 = 72 KB for FP32-only batches, three
 * CTAs per SM, 210 KB otherwise; the buffers that do not fit go to the batch's own global arena, one slice per
 * CTA) and records the graph.  `stream` must not be the legacy default stream (it cannot be
 * captured).  PEPS_E_ARG for a repeated handle or a handle with timing on; PEPS_E_SHAPE when the
 * batch kernel does not fit on an SM at that budget.  Allocates the arena and the queue with
 * cudaMalloc (freed by peps_batch_destroy). */
peps_status peps_batch_create_ex(peps_batch** out, const peps_batch_item* items, int n, int budget_kb, void* stream);
/* peps_batch_create_ex at the default budget (nbranch is ignored: one launch per scalar type). */
peps_status peps_batch_create(peps_batch** out, const peps_batch_item* items, int n, int nbranch, void* stream);
/* Batch autotuner: records the batch at each candidate budget (FP32: 56, 72, 110, 220 KB; with any
 * FP64 item: 100, 210 KB), launches and times it twice with CUDA events (the items' outputs are
 * written), and returns the fastest budget in *budget_kb_host.  The budget decides which work
 * buffers stay on chip and how many CTAs share an SM.  Synchronises the stream. */
peps_status peps_batch_autotune(const peps_batch_item* items, int n, int* budget_kb_host, void* stream);
/* Launch the recorded graph on `stream` (asynchronous). */
peps_status peps_batch_launch(peps_batch* b, void* stream);
peps_status peps_batch_destroy(peps_batch* b);

/* Text of the last error seen by this handle (never NULL). */
const char* peps_last_error(const peps_handle* h);

/* Measured CUDA-core FMA throughput of the current device in TFLOP/s (2 flops per FMA), FP32
 * (fp64 == 0) or FP64 (fp64 != 0): 8 independent FMA chains per thread, every SM filled, timed
 * with CUDA events on `stream` (the call synchronises it).  It is the peak against which the
 * contraction kernels' ALU roofline is quoted.  No counterpart in the paper. */
peps_status peps_probe_fma(int fp64, double* tflops_host, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* PEPS_GB300_H */

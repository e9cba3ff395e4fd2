// Declarations shared by the kernel translation units and the C-ABI layer.
#pragma once
#include "peps_tn.cuh"

namespace peps {

constexpr int NTHREADS = 256;
// resident blocks per SM the sampler, bound and direct-sampling kernels are compiled for: two in
// FP32 (about 100 KB of shared memory each), one in FP64 (about 200 KB)
template <typename T> struct MinBlocks { static constexpr int value = sizeof(T) == 4 ? 2 : 1; };
// the environment kernel in FP32: three blocks per SM (80 registers; measured 10 % faster than
// two at 8x8, D = 4, chi = 16, where the sampler, which also runs the sandwiches, is 9 % slower)
template <typename T> struct EnvBlocks { static constexpr int value = sizeof(T) == 4 ? 3 : 1; };

// term record (ints): number of sites, the sites, window (first row, first column, width,
// two-row flag) and the entry range
enum : int {
  TI_K = 0, TI_S0 = 1, TI_X0 = 5, TI_Y0 = 6, TI_W = 7, TI_TWO = 8, TI_EOFF = 9, TI_ECNT = 10, TI_N = 11
};

struct TermTab {
  int nterm;
  const int* tinfo;     // nterm x TI_N, sorted: one-row terms by row, then two-row terms by row
  const int* ent_ab;    // entries (a, b), h[a][b] != 0
  const double* ent_h;  // entries (re, im)
  const int* row_off;   // Lx+1: one-row terms of row x are [row_off[x], row_off[x+1])
  const int* pair_off;  // Lx: two-row terms of rows x, x+1 are [pair_off[x], pair_off[x+1])
};

struct DiagTab {
  int npairs;
  const int* pair_ij;
  const double* pair_v;
  const double* onsite;  // N x d or null
};

// One instance of a ragged multi-instance batch (k_batch): its geometry, its buffer plans (their
// global-arena slices in the batch's own arena), its handle's buffers and the caller's outputs.
template <typename T>
struct BatchInst {
  Geo g;
  Plan pe, pr, pq;          // environment, one-row and two-row plans
  const T* Tpad;
  const uint8_t* S;
  T* envs;
  double* logs;
  float* wdisc;
  T* O;                     // may be null
  const long long* site_off;
  long long Np;
  TermTab tt;               // in-row and two-row terms (nterm 0 without E_loc)
  DiagTab dg;
  double* rowout;
  double* pairout;
  int* status;
  double* logabs;
  double* phase;
  double* eloc;             // may be null
  int want_e, pairs, sides; // sides: 1 upper only (amplitudes), 3 both
  int Ns;
  long long item0;          // first work-queue index of this instance
};
// k_batch: every CTA takes the next (instance, sample) item of the queue (*next counts them; zero
// it before the launch) and runs that sample's whole evaluation
template <typename T>
cudaError_t launch_batch(const BatchInst<T>* inst, int ninst, long long nitems, unsigned long long* next, int grid,
                         size_t smem, cudaStream_t s);
template <typename T>
cudaError_t kattr_batch(size_t set_bytes, int* occ, size_t occ_smem);

template <typename T>
cudaError_t launch_env(const Geo& g, const Plan& p, int grid, size_t smem, const T* Tpad, const uint8_t* S, int Ns,
                       int sides, T* envs, double* logs, int* status, float* wdisc, cudaStream_t s);
template <typename T>
cudaError_t launch_row(const Geo& g, const Plan& p, int grid, size_t smem, const T* Tpad, const uint8_t* S, int Ns,
                       int x_lo, int x_hi, const T* envs, const double* logs, T* O, const long long* site_off,
                       long long Np, const TermTab& tt, double* rowout, int* status, cudaStream_t s);
template <typename T>
cudaError_t launch_pair(const Geo& g, const Plan& p, int grid, size_t smem, const T* Tpad, const uint8_t* S, int Ns,
                        const T* envs, const double* logs, const TermTab& tt, double* pairout, int* status,
                        cudaStream_t s);
template <typename T>
cudaError_t launch_sample(const Geo& g, const Plan& p, int grid, size_t smem, const Plan& pe, int grid_e,
                          size_t smem_e, const T* Tpad, uint8_t* S, int Ns, int move, int nsweeps,
                          unsigned long long seed, unsigned long long sweep0, T* envs, double* logs,
                          long long* accepted, int* status, int* ustat, cudaStream_t s);
template <typename T>
cudaError_t launch_bound(const Geo& g, const Plan& p, int grid, size_t smem, const T* Tpad, const uint8_t* S, int Ns,
                         int cut, const T* envs, const double* logs, const TermTab& tt, double* bout, double* logabs,
                         double* phase, int* status, cudaStream_t s);
// d x d complex matrix (d <= 4), row major (re, im) pairs, passed by value
struct RotM { double m[32]; };
cudaError_t launch_rotate(int N, int d, const long long* site_off, const RotM& M, const double* in, int in_cplx,
                          double* out, cudaStream_t s);
cudaError_t launch_bound_combine(const Geo& g, int Ns, int nt, const uint8_t* S, const double* bout, const DiagTab& dg,
                                 double* eloc, cudaStream_t s);
template <typename T>
cudaError_t launch_pad(const Geo& g, const double* theta, const long long* site_off, T* Tpad, cudaStream_t s);
cudaError_t launch_combine(const Geo& g, int Ns, const uint8_t* S, const double* rowout, const double* pairout,
                           int use_rows_all, int use_pairs, const DiagTab& dg, double* logabs, double* phase,
                           double* eloc, cudaStream_t s);
// per-kernel attributes: set the dynamic shared-memory limit (set_bytes > 0) and/or report the
// resident blocks per SM at occ_smem bytes (occ != null)
template <typename T>
cudaError_t kattr_env(const Geo& g, size_t set_bytes, int* occ, size_t occ_smem);
template <typename T>
cudaError_t kattr_row(const Geo& g, size_t set_bytes, int* occ, size_t occ_smem);
template <typename T>
cudaError_t kattr_pair(const Geo& g, size_t set_bytes, int* occ, size_t occ_smem);
template <typename T>
cudaError_t kattr_sample(const Geo& g, size_t set_bytes, int* occ, size_t occ_smem);
template <typename T>
cudaError_t kattr_bound(const Geo& g, size_t set_bytes, int* occ, size_t occ_smem);
template <typename T>
inline cudaError_t set_kernel_smem(const Geo& g, size_t bytes) {
  cudaError_t e;
  if ((e = kattr_env<T>(g, bytes, nullptr, 0)) != cudaSuccess) return e;
  if ((e = kattr_row<T>(g, bytes, nullptr, 0)) != cudaSuccess) return e;
  if ((e = kattr_pair<T>(g, bytes, nullptr, 0)) != cudaSuccess) return e;
  if ((e = kattr_bound<T>(g, bytes, nullptr, 0)) != cudaSuccess) return e;
  return kattr_sample<T>(g, bytes, nullptr, 0);
}
// which: 0 k_env, 1 k_row, 2 k_pair, 3 k_sample, 4 k_bound
template <typename T>
inline int occupancy(const Geo& g, int which, size_t smem) {
  int nb = 0;
  switch (which) {
    case 0: kattr_env<T>(g, 0, &nb, smem); break;
    case 1: kattr_row<T>(g, 0, &nb, smem); break;
    case 2: kattr_pair<T>(g, 0, &nb, smem); break;
    case 4: kattr_bound<T>(g, 0, &nb, smem); break;
    default: kattr_sample<T>(g, 0, &nb, smem); break;
  }
  return nb;
}

// ---- direct sampling (peps_direct.cuh)
// Index sizes of the double-layer compression: product bond nb = chi_d D^2, physical P = D^2,
// Jacobi rows mX (even), row length Lr = P chi_d with strides LY (Y, Vt) and LX (X).
struct DlDims {
  int nb, P, chid, Lr, LY, LX, mX;
};
__host__ __device__ inline DlDims dl_dims(int D, int chid) {
  DlDims d;
  d.P = D * D;
  d.chid = chid;
  d.nb = chid * d.P;
  d.Lr = d.P * chid;
  d.LY = d.Lr + 1;
  d.LX = d.Lr + ((8 - d.Lr) % 32 + 32) % 32;
  d.mX = d.nb + (d.nb & 1);
  return d;
}
// element counts of the global work buffers of k_dl_env, in the order B, Rh, Z, Y, X, Vt, C, Cn
__host__ __device__ inline void dl_work_elems(int Ly, int D, int chid, size_t* n8) {
  const DlDims d = dl_dims(D, chid);
  n8[0] = (size_t)Ly * d.nb * d.P * d.nb;
  n8[1] = (size_t)(Ly > 1 ? Ly - 1 : 1) * d.nb * d.nb;
  n8[2] = (size_t)d.nb * d.P * d.nb;
  n8[3] = (size_t)d.nb * d.LY;
  n8[4] = (size_t)d.mX * d.LX;
  n8[5] = (size_t)chid * d.LY;
  n8[6] = (size_t)d.nb * chid;
  n8[7] = (size_t)d.nb * chid;
}
// dynamic shared memory of k_dl_env: reduction scratch, singular values, ranks, Householder taus
__host__ __device__ inline size_t dl_smem_bytes(int D, int chid, size_t esz, size_t rsz) {
  const DlDims d = dl_dims(D, chid);
  size_t b = 40 * 8;
  b += (size_t)(d.mX + 4) * rsz;
  b = (b + 15) / 16 * 16;
  b += (size_t)2 * d.mX * 4;
  b = (b + 15) / 16 * 16;
  b += (size_t)d.nb * esz;
  return b;
}

template <typename T>
struct DlWork {
  T *B, *Rh, *Z, *Y, *X, *Vt, *C, *Cn;
};

template <typename T>
cudaError_t launch_dl_env(const Geo& g, int chid, const T* Tpad, T* DL, const DlWork<T>& w, int* status,
                          cudaStream_t s);
template <typename T>
cudaError_t launch_direct(const Geo& g, const Plan& p, int grid, size_t smem, int chid, const T* Tpad, const T* DL,
                          uint8_t* S, int Ns, unsigned long long seed, unsigned long long draw, double* logp,
                          int* status, cudaStream_t s);
template <typename T>
cudaError_t kattr_direct(const Geo& g, size_t set_bytes, int* occ, size_t occ_smem);

// ---- status bookkeeping (peps_status.cu)
// *word |= OR of st[0..Ns)
cudaError_t launch_status_or(const int* st, int Ns, int* word, cudaStream_t s);
// *word |= bit when *flag != 0
cudaError_t launch_flag_or(const int* flag, int bit, int* word, cudaStream_t s);
// w[i] = (st[i] & mask) ? 0 : 1
cudaError_t launch_status_weights(const int* st, int Ns, int mask, double* w, cudaStream_t s);
// end of a MinSR step: zero dtheta (n doubles) when info[0] < 0 or *gram_err; halve info[0] for a
// complex handle; info[3] = -1 on the factorisation route; flags into *word
cudaError_t launch_minsr_finish(double* info, const int* gram_err, double* dtheta, long long n, int cplx, int chol,
                                int* word, cudaStream_t s);

// ---- MinSR (FP64)
// column means m_k = sum_S w_S O_{S,k} (w normalised), and Obar = sqrt(w)(O - m) written as
// double (Ns x Np)
// (wsum_dev: one device double of scratch for the weight sum, used when w is not NULL)
template <typename TO>
cudaError_t launch_center(const TO* O, const double* w, int Ns, long long Np, double* mean, double* Obar,
                          double* wsum_dev, cudaStream_t s);
cudaError_t launch_center_e(const double* eloc, const double* w, int Ns, double* ebar, cudaStream_t s);
// complex O (Ns x Np (re, im) pairs of TO): the real embedding W (2Ns x 2Np), [Re ebar; Im ebar]
// (2Ns), and dtheta back from [Re; Im] (2Np) to Np (re, im) pairs
template <typename TO>
cudaError_t launch_center_cplx(const TO* O, const double* w, int Ns, long long Np, double* W, double* wsum_dev,
                               cudaStream_t s);
cudaError_t launch_center_e_cplx(const double* eloc, const double* w, int Ns, double* ebar2, cudaStream_t s);
cudaError_t launch_unembed(const double* d2, long long Np, double* dtheta, cudaStream_t s);
// sample-sharded MinSR: local sums (Np column sums of w O, then sum w and sum w Re E_loc), and the
// centring of local rows with the sums reduced over every process
template <typename TO>
cudaError_t launch_partial_sums(const TO* O, const double* w, const double* eloc, int Ns, long long Np, double* sums,
                                cudaStream_t s);
template <typename TO>
cudaError_t launch_center_global(const TO* O, const double* w, const double* eloc, int Ns, long long Np,
                                 const double* g, double* Obar, double* ebar, cudaStream_t s);
cudaError_t launch_gram(const double* Obar, int Ns, long long Np, double* Tm, int ld, cudaStream_t s);
// float-float Gram on the FP32 pipes (hi, lo: Ns x Np floats of scratch)
cudaError_t launch_gram_ff(const double* Obar, int Ns, long long Np, float* hi, float* lo, double* Tm, int ld,
                           cudaStream_t s);
// cyclic Jacobi eigendecomposition of the symmetric n x n matrix A (overwritten by its
// diagonal form), V accumulates the rotations, *info_sweeps (device) = sweeps used or -1 at the
// limit; one cooperative launch (hbuf: n x n scratch, cs: n doubles of scratch, cnt: 2 device
// counters), no host sync
cudaError_t jacobi_eig(double* A, double* V, int n, unsigned long long* cnt, double* hbuf, double* cs,
                       double* info_sweeps, int max_sweeps, cudaStream_t s);
cudaError_t launch_minsr_apply(const double* A, const double* V, const double* ebar, int n, int nreal, double lambda,
                               double rcond, double* y, double* x, double* info, cudaStream_t s);
// x = V diag(kept / (Lambda + lambda)) V^T ebar for the symmetric N x N matrix A (full storage,
// leading dimension ld >= N, overwritten by the Householder reflectors) through its tridiagonal
// form, without forming V (peps_eig.cu); x: ld doubles (zero beyond N); r0 / r1: the rotation
// record's two segments (cap0 / cap1 doubles); ws: td_workspace_doubles(ld) doubles; info as
// launch_minsr_apply plus info[3] = QR steps (-1 and info[0] = -1 when the QR iteration fails).
// *launches = kernels launched.
size_t td_workspace_doubles(int n);
cudaError_t td_pinv_apply(double* A, int ld, int N, const double* ebar, double lambda, double rcond, double* x,
                          double* r0, size_t cap0, double* r1, size_t cap1, double* ws, double* info,
                          cudaStream_t s, long long* launches);
cudaError_t launch_obar_t_x(const double* Obar, const double* x, int Ns, long long Np, double tau, double* dtheta,
                            cudaStream_t s);
// x = (A + lambda I)^-1 ebar by blocked Cholesky (A overwritten by its factor); returns launches
// gate (device flag, may be NULL): every launch does nothing while *gate == 0 (the FP64
// fallback of the mixed solve, decided on the device); a gated run sets info[2] = 0;
// scratch: n doubles (the triangular solves' intermediate vector)
long long chol_solve(double* A, int n, int nreal, double lambda, const double* ebar, double* x, int* bad,
                     double* info, const int* gate, double* scratch, cudaStream_t s, cudaError_t* err);
// the same solve with an FP32 factor (A32: n x n floats, A kept and mirrored to full) and
// `iters` refinement steps with FP64 residuals (r: n doubles, rn: 2 doubles, part: 2 (n + 7) / 8
// doubles of scratch, scratch: n doubles);
// info = (Ns or -1, relative residual, iters, -); *need64 (device) = 1 when the FP64
// factorisation must replace it (factor breakdown or relative residual above 1e-10)
long long chol_solve_mixed(double* A, float* A32, int n, int nreal, double lambda, const double* ebar, double* x,
                           double* r, double* rn, double* part, int iters, int* bad, double* info, int* need64,
                           double* scratch, cudaStream_t s, cudaError_t* err);
// the same with the float-float factor (Fh, Fl: n x n floats each); *need64 = 1 only when the
// pair factorisation broke down; info = (Ns or -1, relative residual after refinement, iters, -)
long long chol_solve_ff(double* A, float* Fh, float* Fl, int n, int nreal, double lambda, const double* ebar, double* x,
                        double* r, double* rn, double* part, int iters, int* bad, double* info, int* need64,
                        double* scratch, cudaStream_t s, cudaError_t* err);
// ---- learned proposal (peps_proposal.cu)
size_t prop_smem_bytes(int Lx, int Ly, int C, int act_bytes, bool train);
cudaError_t launch_prop_logits(int Lx, int Ly, int C, int wprec, const void* w, const uint8_t* S, int Ns, double* logits,
                               int grid, cudaStream_t s);
cudaError_t launch_prop_grad(int Lx, int Ly, int C, int wprec, const void* w, const uint8_t* Sin, const uint8_t* Stg,
                             int Ns, double* grad, double* loss, int grid, cudaStream_t s);
cudaError_t launch_prop_adam(int nw, double* w, double* m, double* v, const double* g, int t, double lr, void* wlow,
                             cudaStream_t s);
cudaError_t launch_prop_draw(int N, int Ns, const double* logits, uint64_t seed, uint64_t step, uint8_t* Sp, double* lq,
                             cudaStream_t s);
cudaError_t launch_prop_logq(int N, int Ns, const double* logits, const uint8_t* S, double* lq, cudaStream_t s);
cudaError_t launch_prop_accept(int N, int Ns, uint64_t seed, uint64_t step, const uint8_t* Sp, const double* lpsi_new,
                               const double* lq_fwd, const double* lq_bwd, uint8_t* S, double* lpsi, long long* accepted,
                               cudaStream_t s);
// ---- tensor-core Gram (peps_gram_tc.cu)
int gram_tc_pad_rows(int Ns);
long long gram_tc_pad_k(long long Np);
cudaError_t launch_gram_tc(const double* Obar, int Ns, long long Np, void* hi, void* lo, double* Tm, int ld, bool mirror,
                           int* err, cudaStream_t s);
// y += x (n doubles)
cudaError_t launch_axpy(double* y, const double* x, long long n, cudaStream_t s);

}  // namespace peps

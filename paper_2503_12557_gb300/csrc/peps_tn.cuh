// Device building blocks of the single-layer boundary-MPS contraction (sm_103a).
//
// Paper: Sec. "On the boundary MPS method" -- E^u[i] approximates the i uppermost rows of the
// network projected on a configuration as an MPS of bond D_c (chi here); each MPS-MPO product
// (bond chi*D) is truncated back to chi.  Sec. "On Numerical Stability" -- every environment
// tensor is divided by its largest modulus and the logarithms are accumulated.
//
// Every dimension is padded: boundary legs of dimension 1 are stored as D (or chi) with zeros,
// so every environment site tensor is chi x D x chi and every projected PEPS tensor is D^4.
// Zero padding changes no contraction value.
//
// Layouts (row major):
//   projected PEPS tensor  A[l][u][r][d]     (for the lower side the u and d legs are swapped on
//                                              load, so both sides run the same code)
//   environment site       e[a][p][b]         a, b in chi (bonds), p in D (open leg)
//   one-row partial        L[a][l][b]         a: E^u bond, l: PEPS bond, b: E^l bond
//   two-row partial        L2[a][i][j][b]
//
// Truncation (the "density matrix algorithm" the paper names, in a QR-based form that never
// squares singular values): left pass Z_k = R_{k-1} M_k, Householder QR of Z_k keeps only R_k
// (R_k^T R_k is the exact left Gram environment of bond k); right pass Y_k = M_k C_k,
// X_k = R_{k-1} Y_k, one-sided Jacobi on the rows of X_k gives its right singular vectors; the
// top chi become the new site tensor and C_{k-1} = Y_k V.  The state it produces is the
// sequential right-to-left SVD compression of the exact product.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <math.h>

namespace peps {

// ------------------------------------------------------------------------------------------
// Scalars.  Every kernel is instantiated for float, double (real PEPS) and cplx<float>,
// cplx<double> (complex PEPS).  The contractions need only +, * and multiply-add; the
// truncation needs conjugates and moduli, provided by the overloads below (identities for
// real types).
template <typename R>
struct cplx {
  R re, im;
  cplx() = default;
  __host__ __device__ constexpr cplx(R r, R i) : re(r), im(i) {}
  __host__ __device__ constexpr cplx(R r) : re(r), im(R(0)) {}
  __host__ __device__ constexpr cplx(int r) : re(R(r)), im(R(0)) {}
  __host__ __device__ cplx& operator+=(const cplx& o) { re += o.re; im += o.im; return *this; }
  __host__ __device__ cplx& operator-=(const cplx& o) { re -= o.re; im -= o.im; return *this; }
  __host__ __device__ cplx& operator*=(R f) { re *= f; im *= f; return *this; }
  __host__ __device__ cplx& operator*=(const cplx& o) {
    const R r = re * o.re - im * o.im;
    im = re * o.im + im * o.re;
    re = r;
    return *this;
  }
};
template <typename R> __host__ __device__ inline cplx<R> operator+(cplx<R> a, const cplx<R>& b) { return a += b; }
template <typename R> __host__ __device__ inline cplx<R> operator-(cplx<R> a, const cplx<R>& b) { return a -= b; }
template <typename R> __host__ __device__ inline cplx<R> operator-(const cplx<R>& a) { return cplx<R>(-a.re, -a.im); }
template <typename R> __host__ __device__ inline cplx<R> operator*(cplx<R> a, const cplx<R>& b) { return a *= b; }
template <typename R> __host__ __device__ inline cplx<R> operator*(cplx<R> a, R f) { return a *= f; }
template <typename R> __host__ __device__ inline cplx<R> operator*(R f, cplx<R> a) { return a *= f; }
template <typename R> __host__ __device__ inline cplx<R> operator/(const cplx<R>& a, R f) { return cplx<R>(a.re / f, a.im / f); }
template <typename R> __host__ __device__ inline bool operator==(const cplx<R>& a, const cplx<R>& b) { return a.re == b.re && a.im == b.im; }
template <typename R> __host__ __device__ inline bool operator!=(const cplx<R>& a, const cplx<R>& b) { return !(a == b); }

template <typename T> struct Scal { using R = T; static constexpr bool complex = false; };
template <typename Q> struct Scal<cplx<Q>> { using R = Q; static constexpr bool complex = true; };

__device__ __forceinline__ float conj_(float x) { return x; }
__device__ __forceinline__ double conj_(double x) { return x; }
template <typename R> __device__ __forceinline__ cplx<R> conj_(const cplx<R>& z) { return cplx<R>(z.re, -z.im); }
__device__ __forceinline__ float abs2_(float x) { return x * x; }
__device__ __forceinline__ double abs2_(double x) { return x * x; }
template <typename R> __device__ __forceinline__ R abs2_(const cplx<R>& z) { return z.re * z.re + z.im * z.im; }
__device__ __forceinline__ float abs_(float x) { return fabsf(x); }
__device__ __forceinline__ double abs_(double x) { return fabs(x); }
template <typename R> __device__ __forceinline__ R abs_(const cplx<R>& z) { return hypot(z.re, z.im); }
// acc + a b
__device__ __forceinline__ float mad(float acc, float a, float b) { return fmaf(a, b, acc); }
__device__ __forceinline__ double mad(double acc, double a, double b) { return fma(a, b, acc); }
template <typename R>
__device__ __forceinline__ cplx<R> mad(const cplx<R>& acc, const cplx<R>& a, const cplx<R>& b) {
  return cplx<R>(fma(a.re, b.re, fma(-a.im, b.im, acc.re)), fma(a.re, b.im, fma(a.im, b.re, acc.im)));
}
// value as (re, im) in double
struct dz { double re, im; };
__device__ __forceinline__ dz to_dz(float x) { return dz{(double)x, 0.0}; }
__device__ __forceinline__ dz to_dz(double x) { return dz{x, 0.0}; }
template <typename R> __device__ __forceinline__ dz to_dz(const cplx<R>& z) { return dz{(double)z.re, (double)z.im}; }
__device__ __forceinline__ double dz_abs(dz a) { return hypot(a.re, a.im); }
__device__ __forceinline__ dz dz_mul(dz a, dz b) { return dz{a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
// a / b (b != 0)
__device__ __forceinline__ dz dz_div(dz a, dz b) {
  const double n = b.re * b.re + b.im * b.im;
  return dz{(a.re * b.re + a.im * b.im) / n, (a.im * b.re - a.re * b.im) / n};
}
// a scalar of type T from a double pair (the imaginary part dropped for real T)
template <typename T> __device__ __forceinline__ T from_dz(dz a) { return (T)a.re; }
template <> __device__ __forceinline__ cplx<float> from_dz<cplx<float>>(dz a) { return cplx<float>((float)a.re, (float)a.im); }
template <> __device__ __forceinline__ cplx<double> from_dz<cplx<double>>(dz a) { return cplx<double>(a.re, a.im); }
__device__ __forceinline__ float re_(float x) { return x; }
__device__ __forceinline__ double re_(double x) { return x; }
template <typename R> __device__ __forceinline__ R re_(const cplx<R>& z) { return z.re; }
// 1 / z
__device__ __forceinline__ float inv_(float x) { return 1.f / x; }
__device__ __forceinline__ double inv_(double x) { return 1.0 / x; }
template <typename R> __device__ __forceinline__ cplx<R> inv_(const cplx<R>& z) {
  const R n = z.re * z.re + z.im * z.im;
  return cplx<R>(z.re / n, -z.im / n);
}
// warp shuffles of any scalar
template <typename T> __device__ __forceinline__ T shfl_xor_(unsigned mask, T v, int m) { return __shfl_xor_sync(mask, v, m); }
template <typename R> __device__ __forceinline__ cplx<R> shfl_xor_(unsigned mask, cplx<R> v, int m) {
  return cplx<R>(__shfl_xor_sync(mask, v.re, m), __shfl_xor_sync(mask, v.im, m));
}

enum : int {
  ST_NEAR_DEGENERATE = 1,
  ST_ZERO_NORM = 2,
  ST_NONFINITE = 4,
  ST_NOCONV = 8
};

constexpr int MAX_LY = 32;  // the longest row (columns) the kernels take

struct Geo {
  int Lx, Ly, d, D, chi;
  int n;   // chi*D, exact product bond
  int se;  // chi*D*chi, one environment site
  int sT;  // D^4, one projected PEPS tensor
  int s2;  // chi*D*D*chi, one two-row partial
  double cut = 0.0;  // truncated-weight cutoff (0: fixed chi)
};

// The same geometry with (chi, D) fixed at compile time: every device routine below is a
// template over the geometry type, so with GeoS the index arithmetic and loop bounds fold to
// constants.  Used for the configurations the library is tuned for; Geo covers the rest.
template <int CHI, int DD>
struct GeoS {
  int Lx, Ly, d;
  double cut;  // truncated-weight cutoff (0: fixed chi)
  static constexpr int D = DD, chi = CHI, n = CHI * DD, se = CHI * DD * CHI, sT = DD * DD * DD * DD,
                       s2 = CHI * DD * DD * CHI;
};

// Row length D chi of the truncation's Jacobi step when it is a compile-time constant, else 0.
template <typename G> struct GeoLr { static constexpr int value = 0; };
template <int CHI, int DD> struct GeoLr<GeoS<CHI, DD>> { static constexpr int value = CHI * DD; };
// Row count chi D^2 of the left pass's QR when it is a compile-time constant, else 0.
template <typename G> struct GeoMz { static constexpr int value = 0; };
template <int CHI, int DD> struct GeoMz<GeoS<CHI, DD>> { static constexpr int value = CHI * DD * DD; };

// ------------------------------------------------------------------------------------------
// buffer plan: every kernel carves its buffers out of dynamic shared memory or out of a
// per-CTA slice of a global scratch arena, as the host planner decided.
enum Buf : int {
  B_R = 0, B_E, B_A, B_A2, B_Z, B_W, B_C, B_SIG, B_SEL, B_RED,
  B_RHIST, B_LP, B_RP, B_T1, B_T2, B_EU, B_EL, B_LW, B_LW2, B_S, B_NBUF
};

struct Plan {
  unsigned long long off[B_NBUF];  // byte offset inside its arena
  unsigned gmask;                  // bit b set: buffer b lives in the global arena
  unsigned long long gstride;      // bytes of global arena per CTA
  int ci;                          // row chunk of the left-pass W buffer
  int cx;                          // chunk of the two-row contractions
  char* gbase;                     // global arena (gstride bytes per CTA)
  unsigned long long* ctr;         // work counters: [0] Jacobi sweeps, [1] rotations, [2] SVDs
};

__device__ __forceinline__ char* buf_ptr(const Plan& p, int b, char* smem, char* gbase) {
  if (p.gmask & (1u << b)) return gbase + (size_t)blockIdx.x * p.gstride + p.off[b];  // gbase = p.gbase
  return smem + p.off[b];
}

// ------------------------------------------------------------------------------------------
// block reductions (blockDim.x a multiple of 32, at most 1024)
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
template <typename R>
__device__ __forceinline__ cplx<R> warp_sum(cplx<R> v) {
  return cplx<R>(warp_sum(v.re), warp_sum(v.im));
}
template <typename T>
__device__ __forceinline__ T warp_max(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// red: at least 33 doubles of shared (or global) scratch.  All threads get the result.
template <typename T>
__device__ T block_sum(T v, double* red) {
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
  __syncthreads();
  if (l == 0) red[w] = (double)v;
  __syncthreads();
  if (w == 0) {
    T t = (l < nw) ? (T)red[l] : T(0);
    t = warp_sum(t);
    if (l == 0) red[32] = (double)t;
  }
  __syncthreads();
  return (T)red[32];
}
template <typename T>
__device__ T block_max(T v, double* red) {
  v = warp_max(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
  __syncthreads();
  if (l == 0) red[w] = (double)v;
  __syncthreads();
  if (w == 0) {
    T t = (l < nw) ? (T)red[l] : T(0);
    t = warp_max(t);
    if (l == 0) red[32] = (double)t;
  }
  __syncthreads();
  return (T)red[32];
}

template <typename R>
__device__ cplx<R> block_sum(cplx<R> v, double* red) {
  const R re = block_sum(v.re, red);
  const R im = block_sum(v.im, red);
  return cplx<R>(re, im);
}

template <typename T>
__device__ void blk_copy(T* dst, const T* src, int n) {
  for (int o = threadIdx.x; o < n; o += blockDim.x) dst[o] = src[o];
}
template <typename T>
__device__ void blk_fill(T* dst, T v, int n) {
  for (int o = threadIdx.x; o < n; o += blockDim.x) dst[o] = v;
}
// unit tensor: 1 at flat index 0, zeros elsewhere (trivial environments and partials)
template <typename T>
__device__ void blk_unit(T* dst, int n) {
  for (int o = threadIdx.x; o < n; o += blockDim.x) dst[o] = (o == 0) ? T(1) : T(0);
}

// Divide v[0..n) by its largest modulus; returns ln(max) (or -inf with ZERO_NORM / NONFINITE
// set in *st when the maximum is 0 or not finite).  Ends with a barrier.
template <typename T>
__device__ double blk_normalize(T* v, int n, double* red, int* st) {
  using R = typename Scal<T>::R;
  R m = 0;
  for (int o = threadIdx.x; o < n; o += blockDim.x) m = fmax(m, abs_(v[o]));
  m = block_max(m, red);
  if (!(m < INFINITY)) {  // NaN or Inf
    if (threadIdx.x == 0) *st |= ST_NONFINITE;
    __syncthreads();
    return -INFINITY;
  }
  if (m == R(0)) {
    if (threadIdx.x == 0) *st |= ST_ZERO_NORM;
    __syncthreads();
    return -INFINITY;
  }
  const R inv = R(1) / m;
  for (int o = threadIdx.x; o < n; o += blockDim.x) v[o] *= inv;
  __syncthreads();
  return log((double)m);
}

// Projected PEPS tensor of site `site` with local state s, as A[l][u][r][d] (swap_ud: as
// A[l][d][r][u], the lower-environment orientation).
template <typename T, typename G>
__device__ void load_A(T* As, const T* Tpad, const G& g, int site, int s, bool swap_ud) {
  if ((unsigned)s >= (unsigned)g.d) s = 0;  // a local state outside [0, d) is not valid input: read as 0
  const T* src = Tpad + ((size_t)site * g.d + s) * g.sT;
  const int D = g.D;
  for (int o = threadIdx.x; o < g.sT; o += blockDim.x) {
    if (!swap_ud) {
      As[o] = src[o];
    } else {
      const int dd = o % D, r = (o / D) % D, u = (o / (D * D)) % D, l = o / (D * D * D);
      As[o] = src[((l * D + dd) * D + r) * D + u];
    }
  }
}

// ------------------------------------------------------------------------------------------
// Householder QR of Z (m x nc, stored column major: element (i, c) at Z[c * m + i], so that the
// column walks of the factorisation are contiguous in shared memory), keeping only R (nc x nc,
// row major, upper triangular, zero below the diagonal).  Reflector convention of LAPACK's
// xLARFG (H = I - tau v v^T, v_0 = 1).
template <typename T>
__device__ __forceinline__ void qr_apply_reflector(const T* zj, int j, T tau, T* zc, int m, int lane) {
  // zc <- (I - conj(tau) v v^H) zc with v = (1, zj[j+1..m))  (H^H of H = I - tau v v^H; real:
  // I - tau v v^T)
  T s = 0;
  for (int i = j + 1 + lane; i < m; i += 32) s = mad(s, conj_(zj[i]), zc[i]);
  s = warp_sum(s);
  const T w = (s + zc[j]) * conj_(tau);
  __syncwarp();
  if (lane == 0) zc[j] -= w;
  for (int i = j + 1 + lane; i < m; i += 32) zc[i] -= zj[i] * w;
  __syncwarp();
}

// Blocked by panels of QB columns: warp 0 computes the panel's reflectors (applying each to
// the rest of the panel), then every warp applies the panel's reflectors, in order, to the
// trailing columns it owns.  Two block barriers per panel.  taus: at least nc entries.
template <typename T>
__device__ void qr_keep_r_smem(T* Z, int m, int nc, T* R, T* taus, int ldr) {
  constexpr int QB = 8;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  const int steps = (m < nc) ? m : nc;
  for (int j0 = 0; j0 < steps; j0 += QB) {
    const int pb = (steps - j0 < QB) ? steps - j0 : QB;
    if (warp == 0) {
      for (int jj = 0; jj < pb; ++jj) {
        const int j = j0 + jj;
        T* zj = Z + (size_t)j * m;
        typename Scal<T>::R part = 0;
        for (int i = j + 1 + lane; i < m; i += 32) part += abs2_(zj[i]);
        const typename Scal<T>::R sigma = warp_sum(part);
        const T alpha = zj[j];
        T tau = 0, beta = alpha;
        if (sigma != 0) {
          // LAPACK's xLARFG: beta = -sign(Re alpha) sqrt(|alpha|^2 + sigma) (real),
          // tau = (beta - alpha) / beta, v = x / (alpha - beta)
          const typename Scal<T>::R nrm = sqrt(abs2_(alpha) + sigma);
          const typename Scal<T>::R bt = (re_(alpha) >= 0) ? -nrm : nrm;
          beta = T(bt);
          tau = (beta - alpha) * (typename Scal<T>::R(1) / bt);
          const T sc = inv_(alpha - beta);
          for (int i = j + 1 + lane; i < m; i += 32) zj[i] *= sc;
        }
        __syncwarp();
        if (tau != T(0))
          for (int c = j + 1; c < j0 + pb; ++c) qr_apply_reflector(zj, j, tau, Z + (size_t)c * m, m, lane);
        if (lane == 0) {
          taus[j] = tau;
          zj[j] = beta;
        }
        __syncwarp();
      }
    }
    __syncthreads();
    for (int c = j0 + pb + warp; c < nc; c += nw) {
      T* zc = Z + (size_t)c * m;
      for (int jj = 0; jj < pb; ++jj) {
        const T tau = taus[j0 + jj];
        if (tau != T(0)) qr_apply_reflector(Z + (size_t)(j0 + jj) * m, j0 + jj, tau, zc, m, lane);
      }
    }
    __syncthreads();
  }
  for (int o = tid; o < ldr * ldr; o += blockDim.x) {
    const int i = o / ldr, c = o % ldr;
    R[o] = (c < nc && i <= c && i < m) ? Z[(size_t)c * m + i] : T(0);
  }
  __syncthreads();
}

// Panel of QB columns (j0 .. j0+pb-1) factored by one warp with the columns in registers
// (element i = lane + 32 r, m <= 32 RPL): per column one warp reduction for the norm and one
// independent reduction per remaining panel column, no shared-memory round trips.
template <typename T, int RPL, int QB>
__device__ __forceinline__ void qr_panel_reg(T* Z, int m, int j0, int pb, T* taus, int lane) {
  T zp[QB][RPL];
#pragma unroll
  for (int q = 0; q < QB; ++q)
#pragma unroll
    for (int r = 0; r < RPL; ++r) {
      const int i = lane + 32 * r;
      zp[q][r] = (q < pb && i < m) ? Z[(size_t)(j0 + q) * m + i] : T(0);
    }
#pragma unroll
  for (int jj = 0; jj < QB; ++jj) {
    if (jj < pb) {
      const int j = j0 + jj;
      T part = 0, aj = 0;
#pragma unroll
      for (int r = 0; r < RPL; ++r) {
        const int i = lane + 32 * r;
        if (i > j) part += zp[jj][r] * zp[jj][r];
        if (r == (j >> 5)) aj = zp[jj][r];
      }
      const T sigma = warp_sum(part);
      const T alpha = __shfl_sync(0xffffffffu, aj, j & 31);
      T tau = 0, beta = alpha;
      if (sigma != T(0)) {
        const T nrm = sqrt(alpha * alpha + sigma);
        beta = (alpha >= T(0)) ? -nrm : nrm;
        tau = (beta - alpha) / beta;
        const T sc = T(1) / (alpha - beta);
#pragma unroll
        for (int r = 0; r < RPL; ++r)
          if (lane + 32 * r > j) zp[jj][r] *= sc;
      }
      if (tau != T(0)) {
        // v = (1 at row j, the scaled column below it); column q <- column q - tau v (v . column q)
        T v[RPL];
#pragma unroll
        for (int r = 0; r < RPL; ++r) {
          const int i = lane + 32 * r;
          v[r] = (i > j) ? zp[jj][r] : (i == j ? T(1) : T(0));
        }
        T d[QB];
#pragma unroll
        for (int q = jj + 1; q < QB; ++q) {
          T s = 0;
#pragma unroll
          for (int r = 0; r < RPL; ++r) s += v[r] * zp[q][r];
          d[q] = s;
        }
#pragma unroll
        for (int q = jj + 1; q < QB; ++q) d[q] = tau * warp_sum(d[q]);
#pragma unroll
        for (int q = jj + 1; q < QB; ++q)
          if (q < pb)
#pragma unroll
            for (int r = 0; r < RPL; ++r) zp[q][r] -= v[r] * d[q];
      }
#pragma unroll
      for (int r = 0; r < RPL; ++r)
        if (lane + 32 * r == j) zp[jj][r] = beta;
      if (lane == 0) taus[j] = tau;
    }
  }
#pragma unroll
  for (int q = 0; q < QB; ++q)
#pragma unroll
    for (int r = 0; r < RPL; ++r) {
      const int i = lane + 32 * r;
      if (q < pb && i < m) Z[(size_t)(j0 + q) * m + i] = zp[q][r];
    }
}

// Register form of the same blocked factorisation (m <= 32 RPL).
//   Panel (warp 0): after column j's reflector is formed, its products with every remaining
//   panel column are taken in one pass over the rows and summed over the warp together, so a
//   panel column costs two warp reductions instead of one per remaining column.
//   Trailing update (all warps): a warp loads CW trailing columns into registers (element
//   i = lane + 32 r), applies the panel's reflectors to each in order and stores them once.
template <typename T, int RPL>
__device__ __noinline__ void qr_keep_r_reg(T* Z, int m, int nc, T* R, T* taus, int ldr) {
  // FP32 with 256 rows: panels of four columns, whose register panel (4 x 8 values a lane)
  // fits the environment kernels' 80 registers; eight columns spilled there
  constexpr int QB = (RPL == 8 && sizeof(T) == 4) ? 4 : 8;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  const int steps = (m < nc) ? m : nc;
  for (int j0 = 0; j0 < steps; j0 += QB) {
    const int pb = (steps - j0 < QB) ? steps - j0 : QB;
    if (warp == 0) {
      if constexpr (RPL * QB * sizeof(T) <= (sizeof(T) == 8 ? 640 : 256)) {
        qr_panel_reg<T, RPL, QB>(Z, m, j0, pb, taus, lane);
      } else {
        for (int jj = 0; jj < pb; ++jj) {
          const int j = j0 + jj;
          T* zj = Z + (size_t)j * m;
          T part = 0;
          for (int i = j + 1 + lane; i < m; i += 32) part += zj[i] * zj[i];
          const T sigma = warp_sum(part);
          const T alpha = zj[j];
          T tau = 0, beta = alpha;
          if (sigma != T(0)) {
            const T nrm = sqrt(alpha * alpha + sigma);
            beta = (alpha >= T(0)) ? -nrm : nrm;
            tau = (beta - alpha) / beta;
            const T sc = T(1) / (alpha - beta);
            for (int i = j + 1 + lane; i < m; i += 32) zj[i] *= sc;
          }
          __syncwarp();
          const int nrem = j0 + pb - 1 - j;  // panel columns right of j
          if (tau != T(0) && nrem > 0) {
            T* zc0 = Z + (size_t)(j + 1) * m;
            T d[QB - 1];
#pragma unroll
            for (int q = 0; q < QB - 1; ++q) d[q] = 0;
            for (int i = j + 1 + lane; i < m; i += 32) {
              const T v = zj[i];
#pragma unroll
              for (int q = 0; q < QB - 1; ++q)
                if (q < nrem) d[q] += v * zc0[(size_t)q * m + i];
            }
#pragma unroll
            for (int q = 0; q < QB - 1; ++q)
              if (q < nrem) d[q] = tau * (warp_sum(d[q]) + zc0[(size_t)q * m + j]);
            __syncwarp();
            for (int i = j + 1 + lane; i < m; i += 32) {
              const T v = zj[i];
#pragma unroll
              for (int q = 0; q < QB - 1; ++q)
                if (q < nrem) zc0[(size_t)q * m + i] -= v * d[q];
            }
            if (lane == 0) {
#pragma unroll
              for (int q = 0; q < QB - 1; ++q)
                if (q < nrem) zc0[(size_t)q * m + j] -= d[q];
            }
          }
          if (lane == 0) {
            taus[j] = tau;
            zj[j] = beta;
          }
          __syncwarp();
        }
      }
    }
    __syncthreads();
    // CW trailing columns per warp at a time (c, c + nw, ...; the later ones may be absent), so
    // that their reductions overlap; one where the columns would not fit in registers
    constexpr int CW = (RPL <= 12) ? 2 : 1;
    for (int c = j0 + pb + warp; c < nc; c += CW * nw) {
      T z[CW][RPL];
#pragma unroll
      for (int w = 0; w < CW; ++w) {
        const int cw = c + w * nw;
#pragma unroll
        for (int r = 0; r < RPL; ++r) {
          const int i = lane + 32 * r;
          z[w][r] = (cw < nc && i < m) ? Z[(size_t)cw * m + i] : T(0);
        }
      }
      for (int jj = 0; jj < pb; ++jj) {
        const int j = j0 + jj;
        const T tau = taus[j];
        if (tau == T(0)) continue;
        const T* v = Z + (size_t)j * m;  // reflector: 1 at row j, v[i] below, 0 above
        T vr[RPL];
        T sdot[CW];
#pragma unroll
        for (int w = 0; w < CW; ++w) sdot[w] = 0;
#pragma unroll
        for (int r = 0; r < RPL; ++r) {
          const int i = lane + 32 * r;
          vr[r] = (i > j && i < m) ? v[i] : (i == j ? T(1) : T(0));
#pragma unroll
          for (int w = 0; w < CW; ++w) sdot[w] += vr[r] * z[w][r];
        }
#pragma unroll
        for (int w = 0; w < CW; ++w) {
          const T wj = tau * warp_sum(sdot[w]);
#pragma unroll
          for (int r = 0; r < RPL; ++r) z[w][r] -= vr[r] * wj;
        }
      }
#pragma unroll
      for (int w = 0; w < CW; ++w) {
        const int cw = c + w * nw;
#pragma unroll
        for (int r = 0; r < RPL; ++r) {
          const int i = lane + 32 * r;
          if (cw < nc && i < m) Z[(size_t)cw * m + i] = z[w][r];
        }
      }
    }
    __syncthreads();
  }
  for (int o = tid; o < ldr * ldr; o += blockDim.x) {
    const int i = o / ldr, c = o % ldr;
    R[o] = (c < nc && i <= c && i < m) ? Z[(size_t)c * m + i] : T(0);
  }
  __syncthreads();
}

// Dispatch on the row count; MC > 0: a compile-time bound on m (m <= MC).  R is written as an
// ldr x ldr row-major upper-triangular matrix (ldr >= nc; the columns from nc on are zero).
template <typename T, int MC = 0>
__device__ void qr_keep_r(T* Z, int m, int nc, T* R, T* taus, int ldr) {
  if constexpr (Scal<T>::complex) {
    qr_keep_r_smem(Z, m, nc, R, taus, ldr);
  } else if constexpr (MC > 0) {
    // the register form is compiled for up to MC rows and runs on the m <= MC rows given
    constexpr int RPL = (MC + 31) / 32;
    if constexpr (RPL <= 24) qr_keep_r_reg<T, RPL>(Z, m, nc, R, taus, ldr);
    else qr_keep_r_smem(Z, m, nc, R, taus, ldr);
  } else {
    if (m <= 256) qr_keep_r_reg<T, 8>(Z, m, nc, R, taus, ldr);
    else if (m <= 768) qr_keep_r_reg<T, 24>(Z, m, nc, R, taus, ldr);
    else qr_keep_r_smem(Z, m, nc, R, taus, ldr);
  }
}

// Round-robin ("chess tournament") ordering of m (even) players: player at position j in
// round r.  Every round pairs position j with position m-1-j; the pairs of one round are
// disjoint and every pair meets once per m-1 rounds.
__device__ __forceinline__ int rr_player(int j, int r, int m) {
  return (j == 0) ? 0 : ((j - 1 + r) % (m - 1)) + 1;
}

template <typename T> struct JacobiTol;
template <> struct JacobiTol<double> { static constexpr double eps = 1.1102230246251565e-16; static constexpr int sweeps = 30; };
template <> struct JacobiTol<float> { static constexpr float eps = 5.9604645e-8f; static constexpr int sweeps = 30; };

// Relative dot product above which a pair of rows of length L is rotated.  FP64: L eps.  FP32:
// 2 sqrt(L) eps, a few times the typical rounding of a converged pair's dot product (sqrt(L)
// eps): L eps (3.8e-6 at L = 64) leaves the kept rows non-orthogonal at a level that shows in
// ln|psi| (on the 8x8, D = 4, chi = 16 workload after ten MinSR steps, against FP64: median
// 3.5e-6 and 12 % of the samples above 1e-5, against 1.9e-6 and 3 % at 2 sqrt(L) eps, for 2 %
// more rotations).
__device__ __forceinline__ double jacobi_tol(int L) { return double(L) * JacobiTol<double>::eps; }
__device__ __forceinline__ float jacobi_tol_f(int L) { return 2.f * sqrtf(float(L)) * JacobiTol<float>::eps; }
template <typename R> __device__ __forceinline__ R jacobi_tol_r(int L);
template <> __device__ __forceinline__ double jacobi_tol_r<double>(int L) { return jacobi_tol(L); }
template <> __device__ __forceinline__ float jacobi_tol_r<float>(int L) { return jacobi_tol_f(L); }

// Rows whose squared norm is at most `tiny` are numerically zero singular values: the Jacobi
// sweeps never rotate them against the others, so they are not orthogonal to the kept
// directions and must not enter the kept basis.  Set them to exactly zero.  Ends with a barrier.
template <typename T>
__device__ void zero_tiny_rows(T* X, int m, int L, int ldx, typename Scal<T>::R tiny) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int p = warp; p < m; p += nw) {
    typename Scal<T>::R s = 0;
    for (int i = lane; i < L; i += 32) s += abs2_(X[(size_t)p * ldx + i]);
    s = warp_sum(s);
    if (s <= tiny)
      for (int i = lane; i < L; i += 32) X[(size_t)p * ldx + i] = T(0);
  }
  __syncthreads();
}

// One-sided (Hestenes) Jacobi on the rows of X (m rows, m even, row length L, leading dim
// ldx): rotate pairs of rows whose relative dot product exceeds the tolerance tol (jacobi_tol_r)
// (well above the sqrt(L) eps rounding noise of a converged pair's dot product), skipping pairs
// where one row is numerically zero (squared norm below (L eps)^2 of the largest), and stop after
// the first sweep in which no pair had a relative dot product of sqrt(tol) or more: by the
// quadratic convergence of cyclic Jacobi, that sweep's rotations leave dot products of order tol,
// so the next sweep would rotate nothing.  On return the rows are sigma_i v_i^T with v_i the
// right singular vectors of the input.
//   Each warp treats four pairs at once (eight lanes per pair).  The squared row norms live in
//   nrm[] (m entries): exact at the start of every sweep, and within a sweep updated after a
//   rotation by Rutishauser's formulas a' = a - t g, b' = b + t g (g the pair's dot product), so
//   that a pair check costs one dot product.
// Returns the number of sweeps, or -1 when the sweep limit was hit.
template <typename T>
__device__ int hestenes_rows_smem(T* X, int m, int L, int ldx, int* flag, unsigned long long* ctr, double* red,
                                  typename Scal<T>::R* nrm) {
  using R = typename Scal<T>::R;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int grp = lane >> 3, sub = lane & 7, ngroups = nw * 4;
  const unsigned gmask = 0xffu << (grp * 8);
  const R eps = JacobiTol<R>::eps;
  const R tol = jacobi_tol_r<R>(L);
  const R stop = sqrt(tol);
  R tiny = 0;
  unsigned long long nrot = 0;
  for (int sweep = 0; sweep < JacobiTol<R>::sweeps; ++sweep) {
    for (int p = warp; p < m; p += nw) {
      R s = 0;
      for (int i = lane; i < L; i += 32) s += abs2_(X[(size_t)p * ldx + i]);
      s = warp_sum(s);
      if (lane == 0) nrm[p] = s;
    }
    if (threadIdx.x == 0) *flag = 0;
    __syncthreads();
    if (sweep == 0) {
      R nmax = 0;
      for (int p = threadIdx.x; p < m; p += blockDim.x) nmax = fmax(nmax, nrm[p]);
      nmax = block_max(nmax, red);
      tiny = nmax * (R(L) * eps) * (R(L) * eps);
    }
    int rotated = 0, big = 0;
    for (int r = 0; r < m - 1; ++r) {
      for (int pi = warp * 4 + grp; pi < m / 2; pi += ngroups) {
        const int p = rr_player(pi, r, m), q = rr_player(m - 1 - pi, r, m);
        T* xp = X + (size_t)p * ldx;
        T* xq = X + (size_t)q * ldx;
        const R a = nrm[p], b = nrm[q];
        T c = 0;
        for (int i = sub; i < L; i += 8) c = mad(c, xp[i], conj_(xq[i]));
        c += shfl_xor_(gmask, c, 4);
        c += shfl_xor_(gmask, c, 2);
        c += shfl_xor_(gmask, c, 1);
        const R ac = abs_(c);
        if (ac != R(0) && a > tiny && b > tiny && ac > tol * sqrt(a * b)) {
          if (ac >= stop * sqrt(a * b)) big = 1;
          // with c = |c| e^{i phi}: rotate (x_p, e^{i phi} x_q), whose product is |c|;
          // zeta = (b - a) / (2|c|); t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)) is the smaller
          // root of t^2 + 2 zeta t - 1 = 0, which makes the rotated rows orthogonal
          const R zeta = (b - a) / (R(2) * ac);
          R t;
          if (fabs(zeta) > R(1e15)) t = R(0.5) / zeta;
          else t = copysign(R(1), zeta) / (fabs(zeta) + sqrt(R(1) + zeta * zeta));
          const R cs = R(1) / sqrt(R(1) + t * t), sn = cs * t;
          const T ph = c * (R(1) / ac);
          for (int i = sub; i < L; i += 8) {
            const T u = xp[i], v = ph * xq[i];
            xp[i] = cs * u - sn * v;
            xq[i] = sn * u + cs * v;
          }
          __syncwarp(gmask);
          if (sub == 0) {
            nrm[p] = fmax(R(0), a - t * ac);
            nrm[q] = b + t * ac;
            ++nrot;
          }
          rotated = 1;
        }
      }
      __syncthreads();
    }
    // bit 0: some pair rotated; bit 1: some pair had a relative dot product of at least `stop`
    const unsigned bits = __ballot_sync(0xffffffffu, rotated) ? (__ballot_sync(0xffffffffu, big) ? 3u : 1u) : 0u;
    if (lane == 0 && bits) atomicOr(flag, (int)bits);
    __syncthreads();
    const int any = *flag;
    __syncthreads();
    if (!(any & 2)) {
      zero_tiny_rows(X, m, L, ldx, tiny);
      if (ctr && nrot) atomicAdd(ctr + 1, nrot);
      if (ctr && threadIdx.x == 0) { atomicAdd(ctr + 0, (unsigned long long)(sweep + 1)); atomicAdd(ctr + 2, 1ull); }
      return sweep + 1;
    }
  }
  zero_tiny_rows(X, m, L, ldx, tiny);
  if (ctr && nrot) atomicAdd(ctr + 1, nrot);
  if (ctr && threadIdx.x == 0) { atomicAdd(ctr + 0, (unsigned long long)JacobiTol<R>::sweeps); atomicAdd(ctr + 2, 1ull); }
  return -1;
}

// Rotation of a pair with squared norms a, b and dot product c, when it is not yet orthogonal
// to the relative tolerance and neither row is numerically zero: zeta = (b - a) / (2c),
// t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)) (the smaller root of t^2 + 2 zeta t - 1 = 0,
// which makes the rotated rows orthogonal), cos = 1 / sqrt(1 + t^2), sin = cos t, and t c for
// the norm updates.  FP32 takes the reciprocal square roots from the SFU (about 2 ulp).  `big`
// is set when the pair's relative dot product |c| / sqrt(a b) is at least `stop`.
__device__ __forceinline__ void jac_params(double a, double b, double c, double tol, double tiny, double stop,
                                           double& cs, double& sn, double& tc, int& big) {
  if (c != 0.0 && a > tiny && b > tiny && fabs(c) > tol * sqrt(a * b)) {
    if (fabs(c) >= stop * sqrt(a * b)) big = 1;
    const double zeta = (b - a) / (2.0 * c);
    const double t = (fabs(zeta) > 1e15) ? 0.5 / zeta : copysign(1.0, zeta) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
    cs = 1.0 / sqrt(1.0 + t * t);
    sn = cs * t;
    tc = t * c;
  }
}
__device__ __forceinline__ void jac_params(float a, float b, float c, float tol, float tiny, float stop, float& cs,
                                           float& sn, float& tc, int& big) {
  const float d = fabsf(c) * rsqrtf(a) * rsqrtf(b);
  if (c != 0.f && a > tiny && b > tiny && d > tol) {
    if (d >= stop) big = 1;
    const float zeta = (b - a) / (2.f * c);
    const float az = fabsf(zeta);
    const float t = (az > 1e15f) ? 0.5f / zeta : copysignf(1.f, zeta) / (az + sqrtf(fmaf(zeta, zeta, 1.f)));
    cs = rsqrtf(fmaf(t, t, 1.f));
    sn = cs * t;
    tc = t * c;
  }
}

// ------------------------------------------------------------------------------------------
// Register form of the same one-sided Jacobi, one 8-lane group per pair (rows of length
// L <= 8 E8, element i = u + 8 e of a row in lane u of a group).
//   The rows are grouped in blocks of four (rows at or beyond m are absent and act as zero
//   rows) and the blocks meet in a round-robin tournament.  In each super-round a warp holds
//   one pair of blocks (P, Q): group g keeps row P_g and, in round t = 0..3, row Q_(g+t)%4,
//   so the four groups rotate four disjoint cross pairs per round; between rounds every group
//   passes its Q row to the group below (one shuffle per element).  In the first super-round
//   of a sweep the 12 pairs inside the two blocks are rotated too: the two groups holding such
//   a pair both compute its rotation from the same values (identical results) and each
//   updates its own row.  Every pair of rows meets once per sweep, as in the row-level
//   ordering, with one block barrier per super-round and the rows read and written once per
//   super-round.  A group sums its dot product over its 8 lanes by an xor butterfly, which
//   leaves the same bits in all 8 lanes.
//   Stopping: the sweeps end after the first sweep in which no pair had a relative dot product
//   |c| / sqrt(a b) of sqrt(tol) or more.  Cyclic Jacobi converges quadratically, so the
//   rotations of such a sweep leave dot products of order (sqrt(tol))^2 = tol: the sweep that
//   would follow finds no pair above tol and would only confirm convergence.
template <typename T>
__device__ __forceinline__ T grp_sum8(T v) {
  v += __shfl_xor_sync(0xffffffffu, v, 4);
  v += __shfl_xor_sync(0xffffffffu, v, 2);
  v += __shfl_xor_sync(0xffffffffu, v, 1);
  return v;
}

template <typename T, int E8>
__device__ __noinline__ int hestenes_rows_grp(T* X, int m, int L, int ldx, int* flag, unsigned long long* ctr,
                                              double* red, T* nrm) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int g = lane >> 3, u = lane & 7;
  const T eps = JacobiTol<T>::eps;
  const T tol = jacobi_tol_r<T>(L);
  const int NB = ((m + 7) / 8) * 2;  // blocks of four rows, an even number of them
  // tiny = (L eps)^2 times the largest squared row norm
  T nmax = 0;
  for (int p = warp; p < m; p += nw) {
    T s = 0;
    for (int i = lane; i < L; i += 32) s += X[(size_t)p * ldx + i] * X[(size_t)p * ldx + i];
    nmax = fmax(nmax, warp_sum(s));
  }
  nmax = block_max(nmax, red);
  const T tiny = nmax * (T(L) * eps) * (T(L) * eps);
  const T stop = sqrt(tol);
  unsigned long long nrot = 0;
  for (int sweep = 0; sweep < JacobiTol<T>::sweeps; ++sweep) {
    if (threadIdx.x == 0) *flag = 0;
    __syncthreads();
    int rotated = 0, big = 0;
    for (int s = 0; s < NB - 1; ++s) {
      for (int bp = warp; bp < NB / 2; bp += nw) {
        const int bP = rr_player(bp, s, NB), bQ = rr_player(NB - 1 - bp, s, NB);
        const int rp = 4 * bP + g;
        int rq = 4 * bQ + g;
        T xp[E8], xq[E8];
#pragma unroll
        for (int e = 0; e < E8; ++e) {
          const int i = u + 8 * e;
          xp[e] = (rp < m && i < L) ? X[(size_t)rp * ldx + i] : T(0);
          xq[e] = (rq < m && i < L) ? X[(size_t)rq * ldx + i] : T(0);
        }
        T np, nq;
        if (s == 0) {
          // exact squared norms at the start of every sweep, then the pairs inside each block
          T ap = 0, aq = 0;
#pragma unroll
          for (int e = 0; e < E8; ++e) { ap += xp[e] * xp[e]; aq += xq[e] * xq[e]; }
          np = grp_sum8(ap);
          nq = grp_sum8(aq);
#pragma unroll
          for (int k = 1; k < 4; ++k) {
            const bool lo = g < (g ^ k);
            T yp[E8], yq[E8];
            T cp = 0, cq = 0;
#pragma unroll
            for (int e = 0; e < E8; ++e) {
              yp[e] = __shfl_xor_sync(0xffffffffu, xp[e], 8 * k);
              yq[e] = __shfl_xor_sync(0xffffffffu, xq[e], 8 * k);
              cp += xp[e] * yp[e];
              cq += xq[e] * yq[e];
            }
            const T mp = __shfl_xor_sync(0xffffffffu, np, 8 * k), mq = __shfl_xor_sync(0xffffffffu, nq, 8 * k);
            cp = grp_sum8(cp);
            cq = grp_sum8(cq);
            T csp = 1, snp = 0, tcp = 0, csq = 1, snq = 0, tcq = 0;
            jac_params(lo ? np : mp, lo ? mp : np, cp, tol, tiny, stop, csp, snp, tcp, big);
            jac_params(lo ? nq : mq, lo ? mq : nq, cq, tol, tiny, stop, csq, snq, tcq, big);
#pragma unroll
            for (int e = 0; e < E8; ++e) {
              xp[e] = lo ? (csp * xp[e] - snp * yp[e]) : (snp * yp[e] + csp * xp[e]);
              xq[e] = lo ? (csq * xq[e] - snq * yq[e]) : (snq * yq[e] + csq * xq[e]);
            }
            np = lo ? fmax(T(0), np - tcp) : np + tcp;
            nq = lo ? fmax(T(0), nq - tcq) : nq + tcq;
            if (snp != T(0) || snq != T(0)) rotated = 1;
            if (lo && u == 0) nrot += (snp != T(0)) + (snq != T(0));
          }
        } else {
          np = (rp < m) ? nrm[rp] : T(0);
          nq = (rq < m) ? nrm[rq] : T(0);
        }
        // the 16 cross pairs: in round t group g pairs P_g with Q_(g+t)%4
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          T c = 0;
#pragma unroll
          for (int e = 0; e < E8; ++e) c += xp[e] * xq[e];
          c = grp_sum8(c);
          T cs = 1, sn = 0, tc = 0;
          jac_params(np, nq, c, tol, tiny, stop, cs, sn, tc, big);
          // late sweeps rotate few pairs: skip the update when no group of the warp rotates
          if (__any_sync(0xffffffffu, sn != T(0))) {
#pragma unroll
            for (int e = 0; e < E8; ++e) {
              const T a = xp[e], b = xq[e];
              xp[e] = cs * a - sn * b;
              xq[e] = sn * a + cs * b;
            }
          }
          np = fmax(T(0), np - tc);
          nq = nq + tc;
          if (sn != T(0)) {
            rotated = 1;
            if (u == 0) ++nrot;
          }
          if (t < 3) {
            const int src = (lane + 8) & 31;
#pragma unroll
            for (int e = 0; e < E8; ++e) xq[e] = __shfl_sync(0xffffffffu, xq[e], src);
            nq = __shfl_sync(0xffffffffu, nq, src);
            rq = 4 * bQ + ((g + t + 1) & 3);
          }
        }
#pragma unroll
        for (int e = 0; e < E8; ++e) {
          const int i = u + 8 * e;
          if (i < L) {
            if (rp < m) X[(size_t)rp * ldx + i] = xp[e];
            if (rq < m) X[(size_t)rq * ldx + i] = xq[e];
          }
        }
        if (u == 0) {
          if (rp < m) nrm[rp] = np;
          if (rq < m) nrm[rq] = nq;
        }
      }
      __syncthreads();
    }
    // bit 0: some pair rotated; bit 1: some pair had a relative dot product of at least `stop`
    const unsigned bits = __ballot_sync(0xffffffffu, rotated) ? (__ballot_sync(0xffffffffu, big) ? 3u : 1u) : 0u;
    if (lane == 0 && bits) atomicOr(flag, (int)bits);
    __syncthreads();
    const int any = *flag;
    __syncthreads();
    if (!(any & 2)) {
      zero_tiny_rows(X, m, L, ldx, tiny);
      if (ctr && nrot) atomicAdd(ctr + 1, nrot);
      if (ctr && threadIdx.x == 0) { atomicAdd(ctr + 0, (unsigned long long)(sweep + 1)); atomicAdd(ctr + 2, 1ull); }
      return sweep + 1;
    }
  }
  zero_tiny_rows(X, m, L, ldx, tiny);
  if (ctr && nrot) atomicAdd(ctr + 1, nrot);
  if (ctr && threadIdx.x == 0) { atomicAdd(ctr + 0, (unsigned long long)JacobiTol<T>::sweeps); atomicAdd(ctr + 2, 1ull); }
  return -1;
}

// Dispatch: the 8-lane-group register form for rows of at most 128 elements (best with a row
// stride ldx = 8 mod 32, so that the four groups' rows fall in different banks), else the
// shared-memory form.  Same contract as hestenes_rows_smem.  LC > 0: the row length is the compile-time LC.
template <typename T, int LC = 0>
__device__ int hestenes_rows(T* X, int m, int L, int ldx, int* flag, unsigned long long* ctr, double* red,
                             typename Scal<T>::R* nrm) {
  if constexpr (Scal<T>::complex) {
    return hestenes_rows_smem(X, m, L, ldx, flag, ctr, red, nrm);
  } else if constexpr (LC > 0) {
    constexpr int E8 = (LC + 7) / 8;
    if constexpr (E8 <= 16) return hestenes_rows_grp<T, E8>(X, m, LC, ldx, flag, ctr, red, nrm);
    else return hestenes_rows_smem(X, m, LC, ldx, flag, ctr, red, nrm);
  } else {
    if (L <= 64) return hestenes_rows_grp<T, 8>(X, m, L, ldx, flag, ctr, red, nrm);
    if (L <= 128) return hestenes_rows_grp<T, 16>(X, m, L, ldx, flag, ctr, red, nrm);
    return hestenes_rows_smem(X, m, L, ldx, flag, ctr, red, nrm);
  }
}

// ------------------------------------------------------------------------------------------
// Sizes (in elements) of the row step's work buffers, shared by every planner:
// Z holds the left pass's column-major Z (n D x n) and, later, the right pass's P, Y, X, Vt, C
// and new-site buffers (Y, X, Vt rows padded to D chi + 1); W holds ci rows of stride
// D^2 chi + 1.
__host__ __device__ inline size_t env_z_elems(int chi, int D) {
  const size_t n = (size_t)chi * D, Lr = (size_t)D * chi, LY = Lr + 1, mX = n + (n & 1);
  const size_t LX = Lr + (size_t)(((8 - (int)Lr) % 32 + 32) % 32);  // X row stride, 8 mod 32
  const size_t zleft = n * D * n;
  const size_t zright = (size_t)chi * D * D * chi + n * LY + mX * LX + (size_t)chi * LY + n * chi + (size_t)chi * D * chi;
  return zleft > zright ? zleft : zright;
}
__host__ __device__ inline size_t env_w_elems(int chi, int D, int ci) { return (size_t)ci * ((size_t)D * D * chi + 1); }
// Size of the one-row sandwich temporaries (the first holds rows padded to chi + 1).
__host__ __device__ inline size_t sandwich1_t_elems(int chi, int D) { return (size_t)D * D * chi * (chi + 1); }

// ------------------------------------------------------------------------------------------
// Per-CTA working set of one boundary-MPS row step.
template <typename T>
struct RowWork {
  T *R, *Rhist, *E, *A, *Z, *W, *C, *sig;
  int* sel;
  double* red;
  int ci;
  unsigned long long* ctr;
};

// Strided contraction over the whole CTA, the form every sandwich step takes:
//   C[cm(m) + cn(n)] = sum_{k1 < K1, k2 < K2} A[am(m) + k1 sa1 + k2 sa2] B[k1 sb1 + k2 sb2 + bn(n)]
// for m < M, n < N, where fm(m) returns (am, cm) and fn(n) returns (bn, cn).  Each thread
// accumulates an RM x RN register tile whose rows m = ti + i tm are interleaved across threads
// (consecutive threads read consecutive rows of A) and whose columns n = tj + j tn are shared by
// the threads of a warp when tm >= 32 (B is read as a broadcast).  Ends with a barrier.
struct Off2 {
  int a, c;
};
template <int RM, int RN, typename T, class FM, class FN>
__device__ __forceinline__ void blk_gemm(const T* __restrict__ A, const T* __restrict__ B, T* __restrict__ C, int M,
                                         int N, int K1, int K2, int sa1, int sa2, int sb1, int sb2, FM fm, FN fn) {
  const int tm = (M + RM - 1) / RM, tn = (N + RN - 1) / RN;
  for (int t = threadIdx.x; t < tm * tn; t += blockDim.x) {
    const int ti = t % tm, tj = t / tm;
    int ao[RM], co[RM], bo[RN], cn[RN];
    bool mv[RM], nv[RN];
#pragma unroll
    for (int i = 0; i < RM; ++i) {
      const int m = ti + i * tm;
      mv[i] = m < M;
      const Off2 o = fm(mv[i] ? m : 0);
      ao[i] = o.a;
      co[i] = o.c;
    }
#pragma unroll
    for (int j = 0; j < RN; ++j) {
      const int n = tj + j * tn;
      nv[j] = n < N;
      const Off2 o = fn(nv[j] ? n : 0);
      bo[j] = o.a;
      cn[j] = o.c;
    }
    T acc[RM][RN];
#pragma unroll
    for (int i = 0; i < RM; ++i)
#pragma unroll
      for (int j = 0; j < RN; ++j) acc[i][j] = T(0);
    for (int k1 = 0; k1 < K1; ++k1) {
      for (int k2 = 0; k2 < K2; ++k2) {
        const int ka = k1 * sa1 + k2 * sa2, kb = k1 * sb1 + k2 * sb2;
        T a[RM], b[RN];
#pragma unroll
        for (int i = 0; i < RM; ++i) a[i] = A[ao[i] + ka];
#pragma unroll
        for (int j = 0; j < RN; ++j) b[j] = B[kb + bo[j]];
#pragma unroll
        for (int i = 0; i < RM; ++i)
#pragma unroll
          for (int j = 0; j < RN; ++j) acc[i][j] = mad(acc[i][j], a[i], b[j]);
      }
    }
#pragma unroll
    for (int i = 0; i < RM; ++i)
#pragma unroll
      for (int j = 0; j < RN; ++j)
        if (mv[i] && nv[j]) C[co[i] + cn[j]] = acc[i][j];
  }
  __syncthreads();
}

// ------------------------------------------------------------------------------------------
// One row step of the boundary MPS: Eout = normalise(truncate_chi(Eprev o T_proj[row])).
//   Eprev, Eout: Ly environment sites (chi x D x chi each), may be global memory.
//   Srow: the Ly local states of the applied row; lower: lower-environment orientation.
// Returns the sum of the Ly log factors; *st collects status bits; *wdisc the largest
// discarded weight (sum of discarded sigma^2 over sum of sigma^2) of any cut.
template <typename T, typename G>
__device__ double env_row_step(const G& g, const T* Eprev, T* Eout, const T* Tpad, int row,
                               const uint8_t* Srow, bool lower, const RowWork<T>& w, int* st,
                               float* wdisc, int* flag) {
  const int chi = g.chi, D = g.D, n = g.n, Ly = g.Ly;
  const int tid = threadIdx.x, NT = blockDim.x;
  const int Lr = D * chi;           // row length of X, Y (open leg x truncated bond)
  const int mX = n + (n & 1);       // Jacobi needs an even row count
  // ---- left pass: R_{-1} = e00, R_k from QR(R_{k-1} M_k), k = 0..Ly-2.  Near the open edge
  // the exact product's bond is small: only the first rk rows of R_{k-1} are nonzero (rk = 1 for
  // R_{-1}, then at most D times the previous count, capped at n), so Z has only rk D nonzero
  // rows, all of them first in its (i, d) row order.  The products and the QR run on those rows
  // alone (Z stored compactly with ld rk D); the dropped rows are exact zeros that would leave
  // every reflector, and so R, unchanged.
  blk_unit(w.R, n * n);
  __shared__ int rks_s[MAX_LY];  // rks_s[k]: nonzero rows of R_{k-1}
  __syncthreads();
  int rk = 1;
  for (int k = 0; k + 1 < Ly; ++k) {
    blk_copy(w.E, Eprev + (size_t)k * g.se, g.se);
    load_A(w.A, Tpad, g, row * Ly + k, Srow[k], lower);
    __syncthreads();
    const int mZ = rk * D;             // nonzero rows of Z; Z is stored column major (ld mZ)
    const int WS = D * D * chi + 1;    // padded row stride of W (no bank conflicts across ii)
    for (int i0 = 0; i0 < rk; i0 += w.ci) {
      const int ci = (rk - i0 < w.ci) ? (rk - i0) : w.ci;
      // W[ii][l][u][b] = sum_a R[i0+ii][(a,l)] E[a][u][b]   (m = (u, b), n = (ii, l), k = a)
      blk_gemm<2, 8>(w.E, w.R + (size_t)i0 * n, w.W, D * chi, ci * D, chi, 1, D * chi, 0, D, 0,
                     [=](int m) { return Off2{m, m}; },
                     [=](int nn) { return Off2{(nn / D) * n + nn % D, (nn / D) * WS + (nn % D) * D * chi}; });
      // Z[(i0+ii, d)][(b, r)] = sum_{l,u} W[ii][l][u][b] A[l][u][r][d]   (m = (ii, b) with ii
      // fastest, n = (r, d), k = (l, u)); Z is column major with column (b, r)
      blk_gemm<4, 4>(w.W, w.A, w.Z, ci * chi, D * D, D * D, 1, chi, 0, D * D, 0,
                     [=](int m) {
                       const int ii = m % ci, b = m / ci;
                       return Off2{ii * WS + b, b * D * mZ + (i0 + ii) * D};
                     },
                     [=](int nn) { return Off2{nn, (nn / D) * mZ + nn % D}; });
    }
    // the columns (b, r) of Z with b at or beyond the bond of E's site k are exact zeros (E's
    // bonds are padded to chi with zeros; the first row has bond D, a truncation keeps at most
    // chi): find the nonzero prefix and factor only it (a zero column leaves every reflector
    // unchanged and is a zero column of R); R's rank, hence the next rk, is at most that width
    __shared__ int ncz_s;
    if (tid == 0) ncz_s = 0;
    __syncthreads();
    {
      int last = 0;
      for (int o = tid; o < mZ * n; o += NT)
        if (w.Z[o] != T(0)) last = max(last, o / mZ + 1);  // NaN compares unequal: kept
      last = __reduce_max_sync(0xffffffffu, (unsigned)last);
      if ((tid & 31) == 0 && last) atomicMax(&ncz_s, last);
    }
    __syncthreads();
    const int ncz = ncz_s;
    qr_keep_r<T, GeoMz<G>::value>(w.Z, mZ, ncz, w.R, w.sig, n);
    blk_copy(w.Rhist + (size_t)k * n * n, w.R, n * n);
    if (tid == 0) rks_s[k] = rk;
    __syncthreads();
    rk = (mZ < ncz) ? mZ : ncz;
    if (rk > n) rk = n;
    if (rk < 1) rk = 1;
  }
  if (tid == 0) rks_s[Ly - 1] = rk;  // the rows of R_{Ly-2}, the right pass's first cut
  __syncthreads();
  // ---- right pass
  // Y and Vt rows are padded to LY = Lr + 1 so that rows read side by side hit different
  // shared-memory banks; X rows to LX = 8 mod 32, the stride at which the Jacobi's four lane
  // groups (eight consecutive elements of four rows each) hit different banks
  const int LY = Lr + 1;
  const int LX = Lr + ((8 - Lr) % 32 + 32) % 32;
  T* P = w.Z;                              // chi*D*D*chi
  T* Y = P + (size_t)chi * D * D * chi;    // n x Lr   (ld LY)
  T* X = Y + (size_t)n * LY;               // mX x Lr  (ld LX)
  T* Vt = X + (size_t)mX * LX;             // chi x Lr (ld LY)
  T* Cn = Vt + (size_t)chi * LY;           // n x chi
  T* Bs = Cn + (size_t)n * chi;            // chi x D x chi (site being written)
  // C_{Ly-1}[(b,r)][c] = delta_{(b,r),0} delta_{c,0}
  blk_unit(w.C, n * chi);
  __syncthreads();
  double logsum = 0.0;
  for (int k = Ly - 1; k >= 0; --k) {
    blk_copy(w.E, Eprev + (size_t)k * g.se, g.se);
    load_A(w.A, Tpad, g, row * Ly + k, Srow[k], lower);
    __syncthreads();
    // P[a][u][r][c] = sum_b E[a][u][b] C[(b,r)][c]   (m = (r, c), n = (a, u), k = b)
    blk_gemm<2, 8>(w.C, w.E, P, D * chi, chi * D, chi, 1, D * chi, 0, 1, 0,
                   [=](int m) { return Off2{m, m}; },
                   [=](int nn) { return Off2{nn * chi, nn * D * chi}; });
    if (k == 0) {
      // first site: its left bond is trivial, keep only row (a,l) = (0,0) of Y = M_0 C_0
      for (int o = tid; o < g.se; o += NT) {
        const int c = o % chi, dd = (o / chi) % D, a = o / (chi * D);
        T s = 0;
        if (a == 0) {
          for (int u = 0; u < D; ++u)
            for (int r = 0; r < D; ++r) s += P[((0 * D + u) * D + r) * chi + c] * w.A[((0 * D + u) * D + r) * D + dd];
        }
        Bs[o] = s;
      }
      __syncthreads();
      logsum += blk_normalize(Bs, g.se, w.red, st);
      blk_copy(Eout, Bs, g.se);
      __syncthreads();
      break;
    }
    // Y[(a,l)][(d,c)] = sum_{u,r} P[a][u][r][c] A[l][u][r][d]   (m = (a, c), n = (l, d), k = (u, r))
    blk_gemm<4, 4>(P, w.A, Y, chi * chi, D * D, D * D, 1, chi, 0, D, 0,
                   [=](int m) { return Off2{(m / chi) * D * D * chi + m % chi, (m / chi) * D * LY + m % chi}; },
                   [=](int nn) { return Off2{(nn / D) * D * D * D + nn % D, (nn / D) * LY + (nn % D) * chi}; });
    // R_{k-1} from the left pass: only its first rks_s[k] rows are nonzero
    const int rkx = rks_s[k] < n ? rks_s[k] : n;
    blk_copy(w.R, w.Rhist + (size_t)(k - 1) * n * n, rkx * n);
    __syncthreads();
    // X = R_{k-1} Y (m = q, n = i, k = j), padded to mX rows, on the nonzero rows of R_{k-1}:
    // a thread takes two columns q and a block of 8 rows i in [8b, 8b + 8), and since R is upper
    // triangular (explicit zeros below the diagonal) its sums start at j = 8b: the terms skipped
    // are exact zeros and the others are added in the same order as the full product.  Rows from
    // rkx on are zero.
    {
      const int nbk = (rkx + 7) / 8, tmq = (Lr + 1) / 2;
      for (int t = tid; t < tmq * nbk; t += NT) {
        const int ti = t % tmq, b = t / tmq;
        const int q0 = ti, q1 = ti + tmq;
        const bool v1 = q1 < Lr;
        T acc0[8], acc1[8];
#pragma unroll
        for (int ii = 0; ii < 8; ++ii) { acc0[ii] = T(0); acc1[ii] = T(0); }
        for (int j = 8 * b; j < n; ++j) {
          const T a0 = Y[(size_t)j * LY + q0], a1 = v1 ? Y[(size_t)j * LY + q1] : T(0);
#pragma unroll
          for (int ii = 0; ii < 8; ++ii) {
            const int i = 8 * b + ii;
            const T r = (i < rkx) ? w.R[(size_t)i * n + j] : T(0);
            acc0[ii] = mad(acc0[ii], a0, r);
            acc1[ii] = mad(acc1[ii], a1, r);
          }
        }
#pragma unroll
        for (int ii = 0; ii < 8; ++ii) {
          const int i = 8 * b + ii;
          if (i < rkx) {
            X[(size_t)i * LX + q0] = acc0[ii];
            if (v1) X[(size_t)i * LX + q1] = acc1[ii];
          }
        }
      }
      for (int o = tid; o < (mX - rkx) * Lr; o += NT) X[(size_t)(rkx + o / Lr) * LX + o % Lr] = T(0);
      __syncthreads();
    }
    // norms, singular values and the selection in the real type (the QR's taus, in the same
    // buffer, are no longer needed)
    using RT = typename Scal<T>::R;
    RT* sig = reinterpret_cast<RT*>(w.sig);
    // only the first rks_s[k] rows of R_{k-1}, hence of X, are nonzero (found by the left
    // pass): the Jacobi runs on those rows (an even count; the rest are exact zeros that no
    // rotation would touch)
    int mJ = rks_s[k] < n ? rks_s[k] : n;  // nonzero rows of R_{k-1} (k >= 1 here)
    mJ += (mJ & 1);
    const int sweeps = hestenes_rows<T, GeoLr<G>::value>(X, mJ < mX ? mJ : mX, Lr, LX, flag, w.ctr, w.red, sig);
    if (sweeps < 0 && tid == 0) *st |= ST_NOCONV;
    // singular values = row norms
    {
      const int lane = tid & 31, warp = tid >> 5, nw = NT >> 5;
      for (int p = warp; p < mX; p += nw) {
        RT s = 0;
        for (int i = lane; i < Lr; i += 32) s += abs2_(X[(size_t)p * LX + i]);
        s = warp_sum(s);
        if (lane == 0) sig[p] = sqrt(s);
      }
    }
    __syncthreads();
    // stable descending rank; the first chi ranks are kept.  A NaN singular value (non-finite
    // input) ranks below every number, so that the ranks stay a permutation and every kept
    // index is valid; the sample is flagged.
    for (int p = tid; p < mX; p += NT) {
      const RT sp = sig[p];
      const RT kp = (sp == sp) ? sp : RT(-1);
      if (!(sp == sp) || isinf(sp)) atomicOr(st, (int)ST_NONFINITE);
      int rk = 0;
      for (int q = 0; q < mX; ++q) {
        const RT sq = sig[q];
        const RT kq = (sq == sq) ? sq : RT(-1);
        rk += (kq > kp) || (kq == kp && q < p);
      }
      w.sel[mX + p] = rk;          // rank of row p
      if (rk < chi) w.sel[rk] = p; // row holding rank rk
      if (rk == chi - 1) sig[mX + 0] = sp;  // sigma_(chi-1)
      if (rk == chi) sig[mX + 1] = sp;      // sigma_(chi)
      if (rk == 0) sig[mX + 2] = sp;        // sigma_(0)
    }
    if (tid == 0 && mX <= chi) { sig[mX + 1] = 0; }
    __syncthreads();
    int nkeep = (mX < chi) ? mX : chi;
    if (g.cut > 0.0) {
      // truncated-weight rule: keep the fewest singular values (at most chi) whose discarded
      // share of sum sigma^2 is at most cut; tail(r) = sum over ranks >= r of sigma^2
      __shared__ int kc_s;
      if (tid == 0) kc_s = mX;
      double part = 0.0;
      for (int p = tid; p < mX; p += NT) part += (double)sig[p] * (double)sig[p];
      const double tot_s = block_sum(part, w.red);  // ends with a barrier
      const double thr = g.cut * tot_s;
      for (int r = tid + 1; r < mX; r += NT) {
        double tail = 0.0;
        for (int p = 0; p < mX; ++p)
          if (w.sel[mX + p] >= r) tail += (double)sig[p] * (double)sig[p];
        if (tail <= thr) atomicMin(&kc_s, r);
      }
      __syncthreads();
      const int kc = kc_s;
      if (tot_s > 0.0 && kc < nkeep) {
        if (tid == 0) {
          // a boundary weight within 1e-9 of the cutoff: the choice is not stable under rounding
          for (int k = kc - 1; k <= kc; ++k) {
            if (k < 1) continue;
            double tail = 0.0;
            for (int p = 0; p < mX; ++p)
              if (w.sel[mX + p] >= k) tail += (double)sig[p] * (double)sig[p];
            if (fabs(tail - thr) <= 1e-9 * thr) *st |= ST_NEAR_DEGENERATE;
          }
        }
        nkeep = kc;
      }
      // discarded weight and near-degenerate cut at the chosen boundary (the oracle's rule)
      RT tot = 0, dis = 0;
      for (int p = tid; p < mX; p += NT) {
        const RT s2 = sig[p] * sig[p];
        tot += s2;
        if (w.sel[mX + p] >= nkeep) dis += s2;
      }
      tot = block_sum(tot, w.red);
      dis = block_sum(dis, w.red);
      if (tid == 0 && nkeep < mX) {
        const RT s0 = sig[mX + 2], sk = sig[w.sel[nkeep - 1]];
        const RT sd = (nkeep < chi) ? sig[w.sel[nkeep]] : sig[mX + 1];
        if (s0 > RT(0) && (sk - sd) < RT(1e-8) * s0 && sd > RT(1e-12) * s0) *st |= ST_NEAR_DEGENERATE;
        if (tot > RT(0)) {
          const float wd = (float)(dis / tot);
          if (wd > *wdisc) *wdisc = wd;
        }
      }
      __syncthreads();
    } else if (mX > chi) {
      // discarded weight and near-degenerate cut (same rule as the oracle)
      RT tot = 0, dis = 0;
      for (int p = tid; p < mX; p += NT) {
        const RT s2 = sig[p] * sig[p];
        tot += s2;
        if (w.sel[mX + p] >= chi) dis += s2;
      }
      tot = block_sum(tot, w.red);
      dis = block_sum(dis, w.red);
      if (tid == 0) {
        const RT s0 = sig[mX + 2], sk = sig[mX + 0], sd = sig[mX + 1];
        if (s0 > RT(0) && (sk - sd) < RT(1e-8) * s0 && sd > RT(1e-12) * s0) *st |= ST_NEAR_DEGENERATE;
        if (tot > RT(0)) {
          const float wd = (float)(dis / tot);
          if (wd > *wdisc) *wdisc = wd;
        }
      }
    }
    // Vt[c'][q] = X[sel(c')][q] / sigma  (the rows of V^H); rows from nkeep on are zero
    for (int o = tid; o < chi * Lr; o += NT) {
      const int q = o % Lr, cp = o / Lr;
      T v = 0;
      if (cp < nkeep) {
        const int p = w.sel[cp];
        const RT s = sig[p];
        if (s > RT(0)) v = X[(size_t)p * LX + q] * (RT(1) / s);
      }
      Vt[(size_t)cp * LY + q] = v;
    }
    __syncthreads();
    // C_{k-1} = Y V: C[j][c'] = sum_q Y[j][q] conj(Vt[c'][q]);  new site B[c'][d][c] = Vt[c'][(d,c)]
    for (int o = tid; o < n * chi; o += NT) {
      const int cp = o % chi, j = o / chi;
      const T* Yr = Y + (size_t)j * LY;
      const T* Vr = Vt + (size_t)cp * LY;
      T s = 0;
      for (int q = 0; q < Lr; ++q) s = mad(s, Yr[q], conj_(Vr[q]));
      Cn[o] = s;
    }
    for (int o = tid; o < g.se; o += NT) Bs[o] = Vt[(size_t)(o / Lr) * LY + o % Lr];  // [c'][d][c]
    __syncthreads();
    logsum += blk_normalize(Bs, g.se, w.red, st);
    blk_copy(Eout + (size_t)k * g.se, Bs, g.se);
    blk_copy(w.C, Cn, n * chi);
    __syncthreads();
  }
  return logsum;
}

// First environment row: row 0 read as an MPS (upper side, e[a=l][p=d][b=r] = A[l][0][r][d])
// or row Lx-1 (lower side, e[l][u][r] = A[l][u][r][0]); every site normalised.
template <typename T, typename G>
__device__ double env_first_row(const G& g, T* Eout, const T* Tpad, int row, const uint8_t* Srow,
                                bool lower, T* Abuf, T* Bs, double* red, int* st) {
  const int chi = g.chi, D = g.D;
  double logsum = 0.0;
  for (int k = 0; k < g.Ly; ++k) {
    load_A(Abuf, Tpad, g, row * g.Ly + k, Srow[k], lower);
    __syncthreads();
    for (int o = threadIdx.x; o < g.se; o += blockDim.x) {
      const int b = o % chi, p = (o / chi) % D, a = o / (chi * D);
      // with the lower orientation Abuf[l][d][r][u]: its "u" slot (index 1) holds the down leg
      Bs[o] = (a < D && b < D) ? Abuf[((a * D + 0) * D + b) * D + p] : T(0);
    }
    __syncthreads();
    logsum += blk_normalize(Bs, g.se, red, st);
    blk_copy(Eout + (size_t)k * g.se, Bs, g.se);
    __syncthreads();
  }
  return logsum;
}

// ------------------------------------------------------------------------------------------
// Quotient m / k for 0 <= m < 2^22 and k >= 1 from a float reciprocal: (m + 1/2) / k lies at
// least 1 / (2k) from every integer, and the two roundings (of 1 / k and of the product) move it
// by at most (m + 1/2) 2^-23 / k < 1 / (2k), so truncation gives the exact quotient.  Cheaper
// than an integer division when k is only known at run time.
struct FDiv {
  int k;
  float r;
};
__device__ __forceinline__ FDiv fdiv_of(int k) { return FDiv{k, __frcp_rn((float)k)}; }
__device__ __forceinline__ int fdiv_q(int m, FDiv d) { return __float2int_rz(((float)m + 0.5f) * d.r); }

// Nonzero prefixes of the bond legs of an upper environment site eu[a][u][x] and a lower one
// el[b][d][z] (chi x D x chi each): a = 1 + the largest left-bond index with a nonzero entry of
// eu, x the same for its right bond, b and z for el (each at least 1).  Near the open edges
// and in the first rows the boundary MPS's bonds are smaller than chi and the row step stores
// them zero-padded (its kept singular values come in descending order, the zero ones last), so
// a contraction over such a bond can stop at the prefix: the skipped terms are exact zeros and
// the kept ones are summed in the same order, which leaves every result unchanged.  NaN and Inf
// entries count as nonzero.  Ends with a barrier; every thread gets the same extents.
struct BondExt {
  int a, x, b, z;
};
template <typename T, typename G>
__device__ BondExt bond_ext(const G& g, const T* eu, const T* el) {
  __shared__ int ext_w[32][4];
  const int chi = g.chi, Dc = g.D * g.chi;
  int ea = 0, ex = 0, eb = 0, ez = 0;
  for (int o = threadIdx.x; o < g.se; o += blockDim.x) {
    const int a = o / Dc + 1, x = o % chi + 1;
    if (eu[o] != T(0)) { ea = max(ea, a); ex = max(ex, x); }
    if (el[o] != T(0)) { eb = max(eb, a); ez = max(ez, x); }
  }
  const unsigned full = 0xffffffffu;
  ea = (int)__reduce_max_sync(full, (unsigned)ea);
  ex = (int)__reduce_max_sync(full, (unsigned)ex);
  eb = (int)__reduce_max_sync(full, (unsigned)eb);
  ez = (int)__reduce_max_sync(full, (unsigned)ez);
  if ((threadIdx.x & 31) == 0) {
    int* w = ext_w[threadIdx.x >> 5];
    w[0] = ea; w[1] = ex; w[2] = eb; w[3] = ez;
  }
  __syncthreads();
  BondExt e{1, 1, 1, 1};
  for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
    e.a = max(e.a, ext_w[i][0]);
    e.x = max(e.x, ext_w[i][1]);
    e.b = max(e.b, ext_w[i][2]);
    e.z = max(e.z, ext_w[i][3]);
  }
  return e;
}

// Zero v[p][q][r] (P x Q x R, row major) outside p < kp, r < kr.  Ends with a barrier.
template <typename T>
__device__ void zero_outside(T* v, int P, int Q, int R, int kp, int kr) {
  if (kp >= P && kr >= R) return;
  const int QR = Q * R;
  for (int o = threadIdx.x; o < P * QR; o += blockDim.x)
    if (o / QR >= kp || o % R >= kr) v[o] = T(0);
  __syncthreads();
}

// ------------------------------------------------------------------------------------------
// One-row sandwich partials.  L[a][l][b] -> L'[x][r][z] over one column with eu[a][u][x],
// A[l][u][r][d], el[b][d][z].  t1: chi*chi*D*D, t2: D*D*chi*(chi+1) elements.  The
// intermediates are laid out so that the index that varies across threads is contiguous in the
// operand it is read from; t2's (x, r) rows are padded to D (chi + 1), so that the two column
// groups a warp reads in the last product (16 rows per group at chi = 16) fall in different
// shared-memory banks.  The bond indices run over the nonzero prefixes of bond_ext (a < ka,
// b < kb, x < kx, z < kz): the intermediates keep their full layouts, entries outside the
// prefixes are neither computed nor read, and L' is zero outside x < kx, z < kz.
template <typename T, typename G>
__device__ void absorb1(const G& g, const T* L, const T* eu, const T* A, const T* el, T* t1, T* t2, T* out) {
  const int chi = g.chi, D = g.D;
  const int PS = D * chi + D;  // padded (x, r) row stride of t2
  const BondExt e = bond_ext(g, eu, el);
  const int kb = e.b, kx = e.x;
  const FDiv fb = fdiv_of(kb), fx = fdiv_of(kx);
  // t1[u][l][x][b] = sum_a L[a][l][b] eu[a][u][x]        (m = (l, b), n = (u, x), k = a)
  blk_gemm<2, 8>(L, eu, t1, D * kb, D * kx, e.a, 1, D * chi, 0, D * chi, 0,
                 [=](int m) {
                   const int l = fdiv_q(m, fb), b = m - l * kb;
                   return Off2{l * chi + b, l * chi * chi + b};
                 },
                 [=](int n) {
                   const int u = fdiv_q(n, fx), x = n - u * kx;
                   return Off2{u * chi + x, u * D * chi * chi + x * chi};
                 });
  // t2[x][r][d][b] = sum_{l,u} t1[u][l][x][b] A[l][u][r][d]   (m = (x, b), n = (r, d), k = (l, u))
  blk_gemm<4, 4>(t1, A, t2, kx * kb, D * D, D, D, chi * chi, D * chi * chi, D * D * D, D * D,
                 [=](int m) {
                   const int x = fdiv_q(m, fb), b = m - x * kb;
                   return Off2{x * chi + b, x * D * PS + b};
                 },
                 [=](int n) { return Off2{n, (n / D) * PS + (n % D) * chi}; });
  // out[x][r][z] = sum_{b,d} el[b][d][z] t2[x][r][d][b]      (m = z, n = (x, r), k = (b, d))
  blk_gemm<1, 4>(el, t2, out, e.z, kx * D, kb, D, D * chi, chi, 1, chi,
                 [=](int m) { return Off2{m, m}; },
                 [=](int n) { return Off2{n * PS, n * chi}; });
  zero_outside(out, chi, D, chi, kx, e.z);
}

// R[x][r][z] -> R'[a][l][b] = sum eu[a][u][x] A[l][u][r][d] el[b][d][z] R[x][r][z].
// t1: D^2 chi (chi+1) elements (its rows padded to chi+1), t2: chi^2 D^2.  Bond indices over
// the nonzero prefixes of bond_ext, as in absorb1; R' is zero outside a < ka, b < kb.
template <typename T, typename G>
__device__ void absorb1_right(const G& g, const T* R, const T* eu, const T* A, const T* el, T* t1, T* t2, T* out) {
  const int chi = g.chi, D = g.D, P = chi + 1;
  const BondExt e = bond_ext(g, eu, el);
  const int ka = e.a, kz = e.z;
  const FDiv fz = fdiv_of(kz), fa = fdiv_of(ka);
  // t1[u][r][z][a] (rows of a padded to P) = sum_x R[x][r][z] eu[a][u][x]   (m = (r, z), n = (a, u))
  blk_gemm<2, 8>(R, eu, t1, D * kz, ka * D, e.x, 1, D * chi, 0, 1, 0,
                 [=](int m) {
                   const int r = fdiv_q(m, fz), z = m - r * kz;
                   return Off2{r * chi + z, (r * chi + z) * P};
                 },
                 [=](int n) { return Off2{n * chi, (n % D) * D * chi * P + n / D}; });
  // t2[z][d][a][l] = sum_{u,r} t1[u][r][z][a] A[l][u][r][d]   (m = (z, a), n = (l, d), k = (u, r))
  blk_gemm<4, 4>(t1, A, t2, kz * ka, D * D, D, D, D * chi * P, chi * P, D * D, D,
                 [=](int m) {
                   const int z = fdiv_q(m, fa), a = m - z * ka;
                   return Off2{z * P + a, z * D * chi * D + a * D};
                 },
                 [=](int n) { return Off2{(n / D) * D * D * D + n % D, (n % D) * chi * D + n / D}; });
  // out[a][l][b] = sum_{z,d} t2[z][d][a][l] el[b][d][z]   (m = (a, l), n = b, k = (z, d))
  blk_gemm<2, 2>(t2, el, out, ka * D, e.b, kz, D, D * chi * D, chi * D, 1, chi,
                 [=](int m) { return Off2{m, m * chi}; },
                 [=](int n) { return Off2{n * D * chi, n}; });
  zero_outside(out, chi, D, chi, ka, e.b);
}

// Site environment of the one-row sandwich: env[l][u][r][d] = sum L[a][l][b] eu[a][u][x]
// el[b][d][z] R[x][r][z]  (= d psi_x / d A[l][u][r][d]).  elT[z][b][d] = el[b][d][z] (the lower
// environment site read transposed, so that the contraction over z has a contiguous operand).
// t1: D^2 chi (chi+1), its (u, l) rows padded to chi (chi + 1); t2: chi^2 D^2.
template <typename T, typename G>
__device__ void site_env1(const G& g, const T* L, const T* eu, const T* elT, const T* R, T* t1, T* t2, T* env) {
  const int chi = g.chi, D = g.D;
  const int S1 = chi * chi + chi;  // padded (u, l) row stride of t1
  // t1[u][l][x][b] = sum_a L[a][l][b] eu[a][u][x]   (as in absorb1, rows padded)
  blk_gemm<2, 8>(L, eu, t1, D * chi, D * chi, chi, 1, D * chi, 0, D * chi, 0,
                 [=](int m) { return Off2{m, (m / chi) * S1 + m % chi}; },
                 [=](int n) { return Off2{n, (n / chi) * D * S1 + (n % chi) * chi}; });
  // t4[b][x][r][d] = sum_z elT[z][b][d] R[x][r][z]   (m = (b, d), n = (x, r), k = z)
  blk_gemm<2, 8>(elT, R, t2, chi * D, chi * D, chi, 1, chi * D, 0, 1, 0,
                 [=](int m) { return Off2{m, (m / D) * chi * D * D + m % D}; },
                 [=](int n) { return Off2{n * chi, n * D}; });
  // env[l][u][r][d] = sum_{b,x} t4[b][x][r][d] t1[u][l][x][b]   (m = (r, d), n = (u, l) with l
  // fastest, so that the two column groups of a warp read t1 rows one padded stride apart)
  blk_gemm<1, 1>(t2, t1, env, D * D, D * D, chi, chi, chi * D * D, D * D, 1, chi,
                 [=](int m) { return Off2{m, m}; },
                 [=](int n) { return Off2{(n / D) * D * S1 + (n % D) * S1, ((n % D) * D + n / D) * D * D}; });
}

template <typename T>
__device__ T blk_dot(const T* a, const T* b, int n, double* red) {
  T s = 0;
  for (int o = threadIdx.x; o < n; o += blockDim.x) s += a[o] * b[o];
  return block_sum(s, red);
}

// ------------------------------------------------------------------------------------------
// Overlap of an upper and a lower boundary MPS across the cut between two rows (the amplitude
// psi_i = E^u[i] . E^l[i+1] of the variational-bound estimator): the plain contraction (no
// conjugation) over the shared physical legs, column by column from the left,
//   L'[x][z] = sum_{a, b, p} L[a][b] eu[a][p][x] el[b][p][z],
// each partial divided by its largest modulus, the log factors added to *lg (the same value
// in every thread).  Lb, Lb2: chi^2 elements; tb: chi D chi.  Returns the last partial.
template <typename T, typename G>
__device__ T mps_overlap(const G& g, const T* EU, const T* EL, T* Lb, T* Lb2, T* tb, double* red, int* st,
                         double* lg) {
  const int chi = g.chi, cd = g.chi * g.D, cc = g.chi * g.chi;
  blk_unit(Lb, cc);
  __syncthreads();
  for (int y = 0; y < g.Ly; ++y) {
    const T* eu = EU + (size_t)y * g.se;
    const T* el = EL + (size_t)y * g.se;
    // tb[b][p][x] = sum_a L[a][b] eu[a][p][x]
    for (int o = threadIdx.x; o < chi * cd; o += blockDim.x) {
      const int b = o / cd, px = o % cd;
      T acc = T(0);
      for (int a = 0; a < chi; ++a) acc += Lb[a * chi + b] * eu[(size_t)a * cd + px];
      tb[o] = acc;
    }
    __syncthreads();
    // L'[x][z] = sum_{b, p} tb[b][p][x] el[b][p][z]
    for (int o = threadIdx.x; o < cc; o += blockDim.x) {
      const int x = o / chi, z = o % chi;
      T acc = T(0);
      for (int bp = 0; bp < cd; ++bp) acc += tb[(size_t)bp * chi + x] * el[(size_t)bp * chi + z];
      Lb2[o] = acc;
    }
    __syncthreads();
    *lg += blk_normalize(Lb2, cc, red, st);
    blk_copy(Lb, Lb2, cc);
    __syncthreads();
  }
  return Lb[0];
}

// ------------------------------------------------------------------------------------------
// Two-row sandwich partials, chunked over the new upper bond (absorb2) / the old upper bond
// (absorb2_right) so that the temporaries hold D^3 chi c elements (c <= cx; absorb2_right's
// first temporary holds chi more).  Intermediates are laid out so that the index that varies
// across threads is contiguous in the operand it is read from.
// L2[a][i][j][b] -> out[x][r1][r2][z] with eu[a][u][x], A1[i][u][r1][v], A2[j][v][r2][d], el[b][d][z].
// Bond indices over the nonzero prefixes of bond_ext, as in absorb1 (the chunks cover x < kx);
// out is zero outside x < kx, z < kz.
template <typename T, typename G>
__device__ void absorb2(const G& g, const T* L2, const T* eu, const T* A1, const T* A2, const T* el,
                        T* t1, T* t2, T* out, int cx) {
  const int chi = g.chi, D = g.D;
  const BondExt e = bond_ext(g, eu, el);
  const int kb = e.b, kx = e.x;
  const FDiv fb = fdiv_of(kb);
  for (int x0 = 0; x0 < kx; x0 += cx) {
    const int c = (kx - x0 < cx) ? kx - x0 : cx;
    const int cc = chi * c;
    const FDiv fbc = fdiv_of(kb * c);
    // t1[i][u][j][b][xx] = sum_a L2[a][i][j][b] eu[a][u][x0+xx]      (m = (i, j, b), n = (u, xx))
    blk_gemm<4, 4>(L2, eu + x0, t1, D * D * kb, D * c, e.a, 1, D * D * chi, 0, D * chi, 0,
                   [=](int m) {
                     const int ij = fdiv_q(m, fb), b = m - ij * kb;
                     return Off2{ij * chi + b, (ij / D) * D * D * cc + ((ij % D) * chi + b) * c};
                   },
                   [=](int n) { return Off2{(n / c) * chi + n % c, (n / c) * D * cc + n % c}; });
    // t2[j][v][b][xx][r1] = sum_{i,u} t1[i][u][j][b][xx] A1[i][u][r1][v]   (m = (j, b, xx), n = (r1, v))
    blk_gemm<4, 4>(t1, A1, t2, D * kb * c, D * D, D, D, D * D * cc, D * cc, D * D * D, D * D,
                   [=](int m) {
                     const int j = fdiv_q(m, fbc), rem = m - j * kb * c;
                     return Off2{j * cc + rem, j * D * D * cc + rem * D};
                   },
                   [=](int n) { return Off2{n, (n % D) * cc * D + n / D}; });
    // t3[r2][d][b][xx][r1] = sum_{j,v} t2[j][v][b][xx][r1] A2[j][v][r2][d]   (into t1; m = (b, xx, r1), n = (r2, d))
    blk_gemm<4, 4>(t2, A2, t1, kb * c * D, D * D, D, D, D * cc * D, cc * D, D * D * D, D * D,
                   [=](int m) { return Off2{m, m}; },
                   [=](int n) { return Off2{n, n * cc * D}; });
    // out[x0+xx][r1][r2][z] = sum_{b,d} el[b][d][z] t3[r2][d][b][xx][r1]   (m = z, n = (xx, r2, r1)
    // with r1 fastest: the two column groups of a warp then read adjacent words of t3)
    blk_gemm<1, 4>(el, t1, out, e.z, c * D * D, kb, D, D * chi, chi, c * D, cc * D,
                   [=](int m) { return Off2{m, m}; },
                   [=](int n) {
                     const int xx = n / (D * D), r2 = (n / D) % D, r1 = n % D;
                     return Off2{r2 * D * cc * D + xx * D + r1, (((x0 + xx) * D + r1) * D + r2) * chi};
                   });
  }
  zero_outside(out, chi, D * D, chi, kx, e.z);
}

// R2[x][r1][r2][z] -> out[a][i][j][b] = sum eu[a][u][x] A1[i][u][r1][v] A2[j][v][r2][d] el[b][d][z] R2[x][r1][r2][z].
// Bond indices over the nonzero prefixes of bond_ext (the chunks cover a < ka); out is zero
// outside a < ka, b < kb.
template <typename T, typename G>
__device__ void absorb2_right(const G& g, const T* R2, const T* eu, const T* A1, const T* A2, const T* el,
                              T* t1, T* t2, T* out, int ca) {
  const int chi = g.chi, D = g.D;
  const BondExt e = bond_ext(g, eu, el);
  const int ka = e.a, kz = e.z;
  const FDiv fz = fdiv_of(kz);
  for (int a0 = 0; a0 < ka; a0 += ca) {
    const int c = (ka - a0 < ca) ? ka - a0 : ca;
    const int cdx = c * D * chi;             // one (u, r1) block of t1, one (v, r2) block of t2
    const int Sz = D * c * D * D + 1;        // z stride of t3 (odd: consecutive z in different banks)
    // t1[u][r1][aa][r2][z] = sum_x R2[x][r1][r2][z] eu[a0+aa][u][x]   (m = (r1, r2, z), n = (aa, u))
    blk_gemm<4, 4>(R2, eu + (size_t)a0 * D * chi, t1, D * D * kz, c * D, e.x, 1, D * D * chi, 0, 1, 0,
                   [=](int m) {
                     const int q = fdiv_q(m, fz), z = m - q * kz;  // q = (r1, r2)
                     return Off2{q * chi + z, (q / D) * cdx + (q % D) * chi + z};
                   },
                   [=](int n) { return Off2{n * chi, (n % D) * D * cdx + (n / D) * D * chi}; });
    // t2[v][r2][aa][i][z] = sum_{u,r1} t1[u][r1][aa][r2][z] A1[i][u][r1][v]   (m = (aa, r2, z), n = (i, v))
    blk_gemm<4, 4>(t1, A1, t2, c * D * kz, D * D, D, D, D * cdx, cdx, D * D, D,
                   [=](int m) {
                     const int q = fdiv_q(m, fz), z = m - q * kz;  // q = (aa, r2)
                     return Off2{q * chi + z, (q % D) * cdx + (q / D) * D * chi + z};
                   },
                   [=](int n) { return Off2{(n / D) * D * D * D + n % D, (n % D) * D * cdx + (n / D) * chi}; });
    // t3[z][d][aa][i][j] (z stride Sz) = sum_{v,r2} t2[v][r2][aa][i][z] A2[j][v][r2][d]   (into t1)
    blk_gemm<4, 4>(t2, A2, t1, c * D * kz, D * D, D, D, D * cdx, cdx, D * D, D,
                   [=](int m) {
                     const int q = fdiv_q(m, fz), z = m - q * kz;  // q = (aa, i)
                     return Off2{q * chi + z, z * Sz + q * D};
                   },
                   [=](int n) { return Off2{(n / D) * D * D * D + n % D, (n % D) * c * D * D + n / D}; });
    // out[a0+aa][i][j][b] = sum_{z,d} t3[z][d][aa][i][j] el[b][d][z]   (m = (aa, i, j), n = b)
    blk_gemm<2, 4>(t1, el, out, c * D * D, e.b, kz, D, Sz, c * D * D, 1, chi,
                   [=](int m) { return Off2{m, (a0 * D * D + m) * chi}; },
                   [=](int n) { return Off2{n * D * chi, n}; });
  }
  zero_outside(out, chi, D * D, chi, ka, e.b);
}

// ------------------------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11), device side, from the published definition.
struct Philox4 { uint32_t v[4]; };

__device__ __forceinline__ Philox4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                                 uint32_t k0, uint32_t k1) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) { k0 += W0; k1 += W1; }
    const uint32_t hi0 = __umulhi(M0, c0), lo0 = M0 * c0;
    const uint32_t hi1 = __umulhi(M1, c2), lo1 = M1 * c2;
    const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
  }
  Philox4 o;
  o.v[0] = c0; o.v[1] = c1; o.v[2] = c2; o.v[3] = c3;
  return o;
}

// 53-bit uniform double in [0, 1) from the first two output words.
__device__ __forceinline__ double uniform53(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint64_t seed) {
  const Philox4 o = philox4x32_10(c0, c1, c2, c3, (uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32));
  return ((double)(o.v[0] >> 5) * 67108864.0 + (double)(o.v[1] >> 6)) * (1.0 / 9007199254740992.0);
}

}  // namespace peps

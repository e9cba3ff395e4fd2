// MinSR pseudo-inverse with a cutoff through the tridiagonal form (paper Eq. (tdvp_fast)): for
// the symmetric T = V diag(Lambda) V^T (N x N, full storage, leading dimension ld),
//   x = V diag(kept_i / (Lambda_i + lambda)) V^T ebar,  kept_i = Lambda_i > rcond max(Lambda)
// without forming V:
//   1. Householder reduction T = Q tridiag(d, e) Q^T, Q = H_0 H_1 ... H_{N-3}, H_k = I - tau_k
//      v_k v_k^T acting on the indices k+1 .. N-1; v_k is stored in row k of T (columns k+1 ..),
//      and y = Q^T ebar is formed alongside;
//   2. implicit QR on the tridiagonal form applied to y (peps_tdql.cuh): eigenvalues, Z^T y and
//      the recorded rotations;
//   3. u = f(Lambda) Z^T y, then u <- Z u (the rotations replayed), then x = Q u.
// Work: 2 N^3 FP64 flops in step 1 (a matrix-vector product and a rank-2 update of the trailing
// block per column), O(N^2) sequential rotations in step 2, O(N^2) in step 3; memory: T in
// place plus the rotation record (about N^2 doubles).  Every step is a launch on the caller's
// stream: no host synchronisation.  Step 2 is one thread of dependent FP64 arithmetic; on a GPU
// whose FP64 rate is a small fraction of its FP32 rate it dominates the route (about 3 us per
// rotation on GB300), which is why the route is opt-in (cfg.solve = 3).
#include "peps_kernels.cuh"
#include "peps_tdql.cuh"

namespace peps {

namespace {
constexpr int TD_TI = 32;   // rank-2 update tile: rows
constexpr int TD_TJ = 128;  // rank-2 update tile: columns (also the tiling of the norm partials)
constexpr int TD_GW = 8;    // matrix-vector product: warps per block (one row per warp at a time)
constexpr int TD_MAXB = 1024;  // largest grid of the product and of the back-transformation

__host__ __device__ inline int cdiv(long long a, long long b) { return (int)((a + b - 1) / b); }
}  // namespace

// partial sums of squares of row 0, columns 2 .. N-1, in tiles of TD_TJ columns (the partials
// the first Householder step reads; later steps get them from the rank-2 update)
__global__ void __launch_bounds__(TD_TJ) k_td_init(const double* __restrict__ A, int N, double* __restrict__ part) {
  __shared__ double red[33];
  const int j = blockIdx.x * TD_TJ + threadIdx.x;
  double v = 0.0;
  if (j >= 2 && j < N) {
    const double a = A[j];
    v = a * a;
  }
  v = block_sum(v, red);
  if (threadIdx.x == 0) part[blockIdx.x] = v;
}

// Householder vector of step k from x = T[k][k+1 .. N-1] (the column below the diagonal, by
// symmetry): H x = beta e_1 with beta = -sign(x_0) |x|, tau = (beta - x_0) / beta, v = x / (x_0 -
// beta) (v_0 = 1).  sigma = sum_{j >= 1} x_j^2 comes as np partials.  sigma = 0: no reflection
// (tau = 0, e_k = x_0).  sc[0] = tau, sc[1] = 1 / (x_0 - beta).
__global__ void k_td_house(const double* __restrict__ A, int ld, int k, const double* __restrict__ part, int np,
                           double* __restrict__ d, double* __restrict__ e, double* __restrict__ tau,
                           double* __restrict__ sc) {
  __shared__ double red[33];
  double s = 0.0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) s += part[i];
  s = block_sum(s, red);
  if (threadIdx.x == 0) {
    const double* row = A + (size_t)k * ld;
    const double x0 = row[k + 1];
    double t = 0.0, v0inv = 0.0, beta = x0;
    if (s > 0.0) {
      const double mu = sqrt(x0 * x0 + s);
      beta = (x0 >= 0.0) ? -mu : mu;
      t = (beta - x0) / beta;
      v0inv = 1.0 / (x0 - beta);
    }
    d[k] = row[k];
    e[k] = beta;
    tau[k] = t;
    sc[0] = t;
    sc[1] = v0inv;
  }
}

// p = tau B v for the trailing block B = T[k+1 .., k+1 ..] (m = N - k - 1), v_j = x_j / (x_0 -
// beta) for j >= 1 and v_0 = 1; one warp per row.  Per block: the partial sum of p_i v_i over
// its rows (part_pv), v over its chunk of columns (vbuf) and the partial dot of v with
// y[k+1 ..] over that chunk (part_y).
__global__ void __launch_bounds__(TD_GW * 32) k_td_gemv(const double* __restrict__ A, int ld, int N, int k,
                                                       const double* __restrict__ sc, const double* __restrict__ y,
                                                       double* __restrict__ p, double* __restrict__ vbuf,
                                                       double* __restrict__ part_pv, double* __restrict__ part_y) {
  __shared__ double red[33];
  const int m = N - k - 1;
  const double t = sc[0], v0inv = sc[1];
  const double* xr = A + (size_t)k * ld + (k + 1);
  const double* B = A + (size_t)(k + 1) * ld + (k + 1);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double pv = 0.0;
  for (int i = blockIdx.x * TD_GW + warp; i < m; i += gridDim.x * TD_GW) {
    double acc = 0.0;
    const double* Bi = B + (size_t)i * ld;
    if (t != 0.0) {
      for (int j = 1 + lane; j < m; j += 32) acc = fma(Bi[j], xr[j], acc);
      acc = warp_sum(acc);
    }
    const double pi = (t != 0.0) ? t * (Bi[0] + v0inv * acc) : 0.0;
    if (lane == 0) {
      p[i] = pi;
      pv = fma(pi, (i == 0) ? 1.0 : xr[i] * v0inv, pv);
    }
  }
  pv = block_sum(pv, red);  // lane 0 of each warp carries its rows' sum, the other lanes 0
  const int ch = cdiv(m, gridDim.x);
  const int j0 = blockIdx.x * ch, j1 = min(m, j0 + ch);
  double yd = 0.0;
  for (int j = j0 + threadIdx.x; j < j1; j += blockDim.x) {
    const double vj = (j == 0) ? 1.0 : xr[j] * v0inv;
    vbuf[j] = vj;
    yd = fma(vj, y[k + 1 + j], yd);
  }
  yd = block_sum(yd, red);
  if (threadIdx.x == 0) {
    part_pv[blockIdx.x] = pv;
    part_y[blockIdx.x] = yd;
  }
}

// sc[2] = alpha = tau (p . v) / 2, sc[3] = tau (v . y[k+1 ..])
__global__ void k_td_scal(const double* __restrict__ part_pv, const double* __restrict__ part_y, int np,
                          double* __restrict__ sc) {
  __shared__ double red[33];
  double a = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) {
    a += part_pv[i];
    b += part_y[i];
  }
  a = block_sum(a, red);
  b = block_sum(b, red);
  if (threadIdx.x == 0) {
    sc[2] = 0.5 * sc[0] * a;
    sc[3] = sc[0] * b;
  }
}

// B <- H B H = B - v w^T - w v^T with w = p - alpha v, over tiles of TD_TI rows x TD_TJ columns
// (256 threads: two row groups of TD_TJ columns).  The blocks of the first tile row also store v
// in row k (the reflector kept for the back-transformation), apply H to y (y[k+1 ..] -= tau (v .
// y) v) and leave in part[blockIdx.x] the sum of squares of the updated B row 0 over their
// columns j >= 2: the next step's sigma.
__global__ void __launch_bounds__(2 * TD_TJ) k_td_rank2(double* __restrict__ A, int ld, int N, int k,
                                                       const double* __restrict__ sc, const double* __restrict__ p,
                                                       const double* __restrict__ vbuf, double* __restrict__ y,
                                                       double* __restrict__ part) {
  __shared__ double vi_s[TD_TI], wi_s[TD_TI];
  __shared__ double red[33];
  const int m = N - k - 1;
  const double alpha = sc[2];
  const int i0 = blockIdx.y * TD_TI;
  const int j = blockIdx.x * TD_TJ + (threadIdx.x % TD_TJ);
  const int rg = threadIdx.x / TD_TJ;
  if (threadIdx.x < TD_TI) {
    const int i = i0 + threadIdx.x;
    const double vi = (i < m) ? vbuf[i] : 0.0;
    vi_s[threadIdx.x] = vi;
    wi_s[threadIdx.x] = (i < m) ? p[i] - alpha * vi : 0.0;
  }
  __syncthreads();
  double sq = 0.0;
  if (j < m) {
    const double vj = vbuf[j], wj = p[j] - alpha * vj;
    double* B = A + (size_t)(k + 1) * ld + (k + 1);
    const int iend = min(TD_TI, m - i0);
    for (int r = rg; r < iend; r += 2) {
      double* bij = B + (size_t)(i0 + r) * ld + j;
      const double nb = *bij - (vi_s[r] * wj + wi_s[r] * vj);
      *bij = nb;
      if (i0 + r == 0 && j >= 2) sq = nb * nb;
    }
    if (blockIdx.y == 0 && rg == 0) {
      A[(size_t)k * ld + (k + 1) + j] = vj;
      y[k + 1 + j] -= sc[3] * vj;
    }
  }
  if (blockIdx.y == 0) {  // the same for every thread of the block
    sq = block_sum(sq, red);
    if (threadIdx.x == 0) part[blockIdx.x] = sq;
  }
}

// the trailing 2 x 2 block needs no reflection
__global__ void k_td_final(const double* __restrict__ A, int ld, int N, double* __restrict__ d,
                           double* __restrict__ e, double* __restrict__ tau) {
  d[N - 2] = A[(size_t)(N - 2) * ld + (N - 2)];
  d[N - 1] = A[(size_t)(N - 1) * ld + (N - 1)];
  e[N - 2] = A[(size_t)(N - 2) * ld + (N - 1)];
  e[N - 1] = 0.0;
  tau[N - 2] = 0.0;
  tau[N - 1] = 0.0;
}

// implicit QR on tridiag(d, e) applied to y, one thread; st[0] = status (0 ok, 1 iteration
// limit, 2 record full), st[1] = doubles recorded, st[2] = QR steps
__global__ void k_td_ql(double* d, double* e, double* y, int N, double* r0, size_t cap0, double* r1, size_t cap1,
                        int maxit, double* st) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  long long steps = 0;
  size_t len = 0;
  const int status = td_ql(d, e, y, N, r0, cap0, r1, cap1, maxit, &steps, &len);
  st[0] = (double)status;
  st[1] = (double)len;
  st[2] = (double)steps;
}

// u_i = kept_i y_i / (Lambda_i + lambda) in place (all zero after a failed QR iteration);
// info = [kept count (-1 after a failure), min Lambda, max Lambda, QR steps (-1 after a failure)]
__global__ void k_td_apply(const double* __restrict__ d, double* __restrict__ y, int N, double lambda, double rcond,
                           const double* __restrict__ st, double* __restrict__ info) {
  __shared__ double red[33];
  double mx = -INFINITY, mn = INFINITY;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    mx = fmax(mx, d[i]);
    mn = fmin(mn, d[i]);
  }
  mx = block_max(mx, red);
  mn = -block_max(-mn, red);
  const bool ok = st[0] == 0.0;
  double cnt = 0.0;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    const bool keep = ok && (rcond > 0.0 ? d[i] > rcond * mx : true);
    y[i] = keep ? y[i] / (d[i] + lambda) : 0.0;
    cnt += keep ? 1.0 : 0.0;
  }
  cnt = block_sum(cnt, red);
  if (threadIdx.x == 0) {
    info[0] = ok ? cnt : -1.0;
    info[1] = mn;
    info[2] = mx;
    info[3] = ok ? st[2] : -1.0;
  }
}

__global__ void k_td_replay(double* u, const double* r0, size_t cap0, const double* r1, const double* st) {
  if (threadIdx.x != 0 || blockIdx.x != 0 || st[0] != 0.0) return;
  td_replay(u, r0, cap0, r1, (size_t)st[1]);
}

// back-transformation x <- H_k x: per-block partials of v_k . x[k+1 ..], then x[k+1 ..] -= tau_k
// (sum of the partials) v_k
__global__ void k_td_bdot(const double* __restrict__ A, int ld, int N, int k, const double* __restrict__ x,
                          double* __restrict__ part) {
  __shared__ double red[33];
  const int m = N - k - 1;
  const double* v = A + (size_t)k * ld + (k + 1);
  double s = 0.0;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x) s = fma(v[j], x[k + 1 + j], s);
  s = block_sum(s, red);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}
__global__ void k_td_baxpy(const double* __restrict__ A, int ld, int N, int k, const double* __restrict__ tau,
                           double* __restrict__ x, const double* __restrict__ part, int np) {
  __shared__ double red[33];
  double s = 0.0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) s += part[i];
  s = block_sum(s, red) * tau[k];
  const int m = N - k - 1;
  const double* v = A + (size_t)k * ld + (k + 1);
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x) x[k + 1 + j] -= s * v[j];
}

size_t td_workspace_doubles(int n) { return 6 * (size_t)n + 3 * TD_MAXB + 64; }

cudaError_t td_pinv_apply(double* A, int ld, int N, const double* ebar, double lambda, double rcond, double* x,
                          double* r0, size_t cap0, double* r1, size_t cap1, double* ws, double* info,
                          cudaStream_t s, long long* launches) {
  if (N < 2) return cudaErrorInvalidValue;
  const int n = ld;
  double* d = ws;
  double* e = d + n;
  double* tau = e + n;
  double* p = tau + n;
  double* vbuf = p + n;
  double* part_n = vbuf + n;  // at most ceil(N / TD_TJ) <= n entries
  double* part_pv = part_n + n;
  double* part_y = part_pv + TD_MAXB;
  double* part_b = part_y + TD_MAXB;
  double* sc = part_b + TD_MAXB;  // 16: Householder scalars, 16 .. 18: QR status
  double* st = sc + 16;
  long long nl = 0;
  cudaError_t err;
  if ((err = cudaMemsetAsync(x, 0, sizeof(double) * n, s)) != cudaSuccess) return err;
  if ((err = cudaMemcpyAsync(x, ebar, sizeof(double) * N, cudaMemcpyDeviceToDevice, s)) != cudaSuccess) return err;
  k_td_init<<<cdiv(N, TD_TJ), TD_TJ, 0, s>>>(A, N, part_n);
  ++nl;
  for (int k = 0; k + 2 < N; ++k) {
    const int m = N - k - 1;
    k_td_house<<<1, 256, 0, s>>>(A, ld, k, part_n, cdiv(N - k, TD_TJ), d, e, tau, sc);
    const int g2 = min(cdiv(m, TD_GW), TD_MAXB);
    k_td_gemv<<<g2, TD_GW * 32, 0, s>>>(A, ld, N, k, sc, x, p, vbuf, part_pv, part_y);
    k_td_scal<<<1, 256, 0, s>>>(part_pv, part_y, g2, sc);
    k_td_rank2<<<dim3(cdiv(m, TD_TJ), cdiv(m, TD_TI)), 2 * TD_TJ, 0, s>>>(A, ld, N, k, sc, p, vbuf, x, part_n);
    nl += 4;
  }
  k_td_final<<<1, 1, 0, s>>>(A, ld, N, d, e, tau);
  k_td_ql<<<1, 32, 0, s>>>(d, e, x, N, r0, cap0, r1, cap1, 60, st);
  k_td_apply<<<1, 1024, 0, s>>>(d, x, N, lambda, rcond, st, info);
  k_td_replay<<<1, 32, 0, s>>>(x, r0, cap0, r1, st);
  nl += 4;
  for (int k = N - 3; k >= 0; --k) {
    const int m = N - k - 1;
    const int gb = min(cdiv(m, 256), 64);
    k_td_bdot<<<gb, 256, 0, s>>>(A, ld, N, k, x, part_b);
    k_td_baxpy<<<gb, 256, 0, s>>>(A, ld, N, k, tau, x, part_b, gb);
    nl += 2;
  }
  if (launches) *launches = nl;
  return cudaGetLastError();
}

}  // namespace peps

// MinSR update in FP64 (paper Eq. (tdvp_fast)): T = Obar Obar^T (N_s x N_s), eigendecomposition
// T = V diag(Lambda) V^T by cyclic Jacobi, pseudo-inverse with cutoff, dtheta = -tau Obar^T x.
#include <cooperative_groups.h>

#include "peps_kernels.cuh"

namespace cg = cooperative_groups;

namespace peps {

// ---- centring: mean_k = sum_S w_S O_{S,k}; Obar_{S,k} = sqrt(w_S) (O_{S,k} - mean_k)
// The weight sum is read from the device (written by k_wsum), so that no host round trip
// separates the two launches.
template <typename TO>
__global__ void k_center(const TO* __restrict__ O, const double* __restrict__ w, int Ns, long long Np,
                         const double* __restrict__ wsum_dev, double* mean, double* Obar) {
  const double wsum = w ? *wsum_dev : 1.0;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < Np; k += (long long)gridDim.x * blockDim.x) {
    double m = 0.0;
    for (int s = 0; s < Ns; ++s) m += (w ? w[s] / wsum : 1.0 / Ns) * (double)O[(size_t)s * Np + k];
    mean[k] = m;
    for (int s = 0; s < Ns; ++s) {
      const double sw = sqrt(w ? w[s] / wsum : 1.0 / Ns);
      Obar[(size_t)s * Np + k] = sw * ((double)O[(size_t)s * Np + k] - m);
    }
  }
}

// ---- complex PEPS: the MinSR of complex O runs as the real MinSR of its embedding.
// With Obar complex (Ns x Np), W = [[Re Obar, -Im Obar], [Im Obar, Re Obar]] (2Ns x 2Np) has
// W W^T = [[Re T, -Im T], [Im T, Re T]], the real form of T = Obar Obar^H, and
// W^T [Re x; Im x] = [Re(Obar^H x); Im(Obar^H x)]: the real pipeline on (W, [Re ebar; Im ebar])
// returns [Re dtheta; Im dtheta].  O: Ns x Np (re, im) pairs of TO.
template <typename TO>
__global__ void k_center_cplx(const TO* __restrict__ O, const double* __restrict__ w, int Ns, long long Np,
                              const double* __restrict__ wsum_dev, double* W) {
  const double wsum = w ? *wsum_dev : 1.0;
  const long long Np2 = 2 * Np;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < Np; k += (long long)gridDim.x * blockDim.x) {
    double mr = 0.0, mi = 0.0;
    for (int s = 0; s < Ns; ++s) {
      const double ws = w ? w[s] / wsum : 1.0 / Ns;
      mr += ws * (double)O[2 * ((size_t)s * Np + k)];
      mi += ws * (double)O[2 * ((size_t)s * Np + k) + 1];
    }
    for (int s = 0; s < Ns; ++s) {
      const double sw = sqrt(w ? w[s] / wsum : 1.0 / Ns);
      const double re = sw * ((double)O[2 * ((size_t)s * Np + k)] - mr);
      const double im = sw * ((double)O[2 * ((size_t)s * Np + k) + 1] - mi);
      W[(size_t)s * Np2 + k] = re;
      W[(size_t)s * Np2 + Np + k] = -im;
      W[(size_t)(Ns + s) * Np2 + k] = im;
      W[(size_t)(Ns + s) * Np2 + Np + k] = re;
    }
  }
}

// [Re ebar; Im ebar] with ebar = sqrt(w) (E_loc - w^T E_loc) (complex E_loc)
__global__ void k_center_e_cplx(const double* eloc, const double* w, int Ns, double* ebar2) {
  __shared__ double red[33];
  double ws = 0.0, mr = 0.0, mi = 0.0;
  for (int i = threadIdx.x; i < Ns; i += blockDim.x) {
    const double wi = w ? w[i] : 1.0;
    ws += wi;
    mr += wi * eloc[2 * i];
    mi += wi * eloc[2 * i + 1];
  }
  ws = block_sum(ws, red);
  mr = block_sum(mr, red) / ws;
  mi = block_sum(mi, red) / ws;
  for (int i = threadIdx.x; i < Ns; i += blockDim.x) {
    const double sw = sqrt((w ? w[i] : 1.0) / ws);
    ebar2[i] = sw * (eloc[2 * i] - mr);
    ebar2[Ns + i] = sw * (eloc[2 * i + 1] - mi);
  }
}

// dtheta (Np (re, im) pairs) from the embedding's [Re; Im] (2Np)
__global__ void k_unembed(const double* d2, long long Np, double* dtheta) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < Np; k += (long long)gridDim.x * blockDim.x) {
    dtheta[2 * k] = d2[k];
    dtheta[2 * k + 1] = d2[Np + k];
  }
}

__global__ void k_wsum(const double* w, int Ns, double* out) {
  __shared__ double red[33];
  double s = 0.0;
  for (int i = threadIdx.x; i < Ns; i += blockDim.x) s += w[i];
  s = block_sum(s, red);
  if (threadIdx.x == 0) *out = s;
}

// ebar_S = sqrt(w_S) (Re E_loc(S) - sum_S' w_S' Re E_loc(S')); eloc is (re, im) interleaved
__global__ void k_center_e(const double* eloc, const double* w, int Ns, double* ebar) {
  __shared__ double red[33];
  double ws = 0.0, m = 0.0;
  for (int i = threadIdx.x; i < Ns; i += blockDim.x) {
    const double wi = w ? w[i] : 1.0;
    ws += wi;
    m += wi * eloc[2 * i];
  }
  ws = block_sum(ws, red);
  m = block_sum(m, red) / ws;
  for (int i = threadIdx.x; i < Ns; i += blockDim.x) {
    const double wi = (w ? w[i] : 1.0) / ws;
    ebar[i] = sqrt(wi) * (eloc[2 * i] - m);
  }
}

// ---- sample-sharded MinSR: the centring split into local sums (reduced across processes by the
// caller) and the centring of the local rows with the global sums.
// sums[k] = sum_S w_S O_{S,k} (k < Np), sums[Np] = sum_S w_S, sums[Np + 1] = sum_S w_S Re E_loc(S)
// (w NULL: every w_S = 1)
template <typename TO>
__global__ void k_colsum(const TO* __restrict__ O, const double* __restrict__ w, int Ns, long long Np,
                         double* __restrict__ sums) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < Np; k += (long long)gridDim.x * blockDim.x) {
    double m = 0.0;
    for (int s = 0; s < Ns; ++s) m += (w ? w[s] : 1.0) * (double)O[(size_t)s * Np + k];
    sums[k] = m;
  }
}

__global__ void k_wsums(const double* __restrict__ w, const double* __restrict__ eloc, int Ns, double* out) {
  __shared__ double red[33];
  double ws = 0.0, we = 0.0;
  for (int i = threadIdx.x; i < Ns; i += blockDim.x) {
    const double wi = w ? w[i] : 1.0;
    ws += wi;
    we += wi * eloc[2 * i];
  }
  ws = block_sum(ws, red);
  we = block_sum(we, red);
  if (threadIdx.x == 0) { out[0] = ws; out[1] = we; }
}

// Obar_{S,k} = sqrt(w_S / W) (O_{S,k} - g_k / W), ebar_S = sqrt(w_S / W) (Re E_loc(S) - g_E / W) with
// the global sums g (layout of k_colsum / k_wsums: Np column sums, W, g_E)
template <typename TO>
__global__ void k_center_global(const TO* __restrict__ O, const double* __restrict__ w, int Ns, long long Np,
                                const double* __restrict__ g, double* __restrict__ Obar) {
  const double W = g[Np];
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < Np; k += (long long)gridDim.x * blockDim.x) {
    const double m = g[k] / W;
    for (int s = 0; s < Ns; ++s) {
      const double sw = sqrt((w ? w[s] : 1.0) / W);
      Obar[(size_t)s * Np + k] = sw * ((double)O[(size_t)s * Np + k] - m);
    }
  }
}

__global__ void k_center_e_global(const double* __restrict__ eloc, const double* __restrict__ w, int Ns, long long Np,
                                  const double* __restrict__ g, double* __restrict__ ebar) {
  const double W = g[Np], m = g[Np + 1] / W;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < Ns; i += gridDim.x * blockDim.x)
    ebar[i] = sqrt((w ? w[i] : 1.0) / W) * (eloc[2 * i] - m);
}

template <typename TO>
cudaError_t launch_partial_sums(const TO* O, const double* w, const double* eloc, int Ns, long long Np, double* sums,
                                cudaStream_t s) {
  const long long blocks = (Np + 255) / 256;
  k_colsum<TO><<<(int)(blocks < 4096 ? (blocks > 0 ? blocks : 1) : 4096), 256, 0, s>>>(O, w, Ns, Np, sums);
  k_wsums<<<1, 1024, 0, s>>>(w, eloc, Ns, sums + Np);
  return cudaGetLastError();
}
template cudaError_t launch_partial_sums<double>(const double*, const double*, const double*, int, long long, double*,
                                                 cudaStream_t);
template cudaError_t launch_partial_sums<float>(const float*, const double*, const double*, int, long long, double*,
                                                cudaStream_t);

template <typename TO>
cudaError_t launch_center_global(const TO* O, const double* w, const double* eloc, int Ns, long long Np,
                                 const double* g, double* Obar, double* ebar, cudaStream_t s) {
  const long long blocks = (Np + 255) / 256;
  k_center_global<TO><<<(int)(blocks < 4096 ? (blocks > 0 ? blocks : 1) : 4096), 256, 0, s>>>(O, w, Ns, Np, g, Obar);
  k_center_e_global<<<(Ns + 255) / 256 > 0 ? (Ns + 255) / 256 : 1, 256, 0, s>>>(eloc, w, Ns, Np, g, ebar);
  return cudaGetLastError();
}
template cudaError_t launch_center_global<double>(const double*, const double*, const double*, int, long long,
                                                  const double*, double*, double*, cudaStream_t);
template cudaError_t launch_center_global<float>(const float*, const double*, const double*, int, long long,
                                                 const double*, double*, double*, cudaStream_t);

// ---- Gram T = Obar Obar^T, 64 x 64 output tiles, K staged through shared memory in chunks
// of 16; only tiles with ti >= tj are computed, the upper triangle is mirrored.
constexpr int GT = 64, GK = 16;
__global__ void __launch_bounds__(256) k_gram(const double* __restrict__ Ob, int Ns, long long Np, double* Tm, int ld) {
  __shared__ double As[GK][GT + 1], Bs[GK][GT + 1];
  const int nt = (Ns + GT - 1) / GT;
  // linear index over lower-triangle tiles
  int t = blockIdx.x, ti = 0;
  while (t >= ti + 1) { t -= ti + 1; ++ti; }
  const int tj = t;
  if (ti >= nt) return;
  const int r0 = ti * GT, c0 = tj * GT;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;  // each thread: 4 x 4 outputs
  double acc[4][4] = {};
  for (long long k0 = 0; k0 < Np; k0 += GK) {
    for (int o = threadIdx.x; o < GK * GT; o += blockDim.x) {
      const int kk = o % GK, rr = o / GK;
      const long long k = k0 + kk;
      As[kk][rr] = (r0 + rr < Ns && k < Np) ? Ob[(size_t)(r0 + rr) * Np + k] : 0.0;
      Bs[kk][rr] = (c0 + rr < Ns && k < Np) ? Ob[(size_t)(c0 + rr) * Np + k] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GK; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) { a[i] = As[kk][ty * 4 + i]; b[i] = Bs[kk][tx * 4 + i]; }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int r = r0 + ty * 4 + i, c = c0 + tx * 4 + j;
      if (r < Ns && c < Ns) {
        Tm[(size_t)r * ld + c] = acc[i][j];
        Tm[(size_t)c * ld + r] = acc[i][j];
      }
    }
}

// ---- cyclic Jacobi, parallel round-robin ordering.  One launch per round: every thread owns
// one 2x2 block (pair I, pair J) of the old matrix and writes the rotated block into the new
// one; rotation parameters are recomputed from the old diagonal blocks (classical two-sided
// Jacobi, Golub & Van Loan sym.schur2: tau = (a_qq - a_pp) / (2 a_pq), t = sign(tau) /
// (|tau| + sqrt(1 + tau^2)), c = 1/sqrt(1+t^2), s = t c; B = J^T A J with J = [[c, s], [-s, c]]).
__device__ __forceinline__ void jac_params(const double* A, int n, int p, int q, double* c, double* s) {
  const double apq = A[(size_t)p * n + q];
  const double app = A[(size_t)p * n + p], aqq = A[(size_t)q * n + q];
  if (apq == 0.0 || fabs(apq) <= 1e-15 * sqrt(fabs(app * aqq))) { *c = 1.0; *s = 0.0; return; }
  const double tau = (aqq - app) / (2.0 * apq);
  double t;
  if (fabs(tau) > 1e150) t = 0.5 / tau;
  else t = copysign(1.0, tau) / (fabs(tau) + sqrt(1.0 + tau * tau));
  *c = 1.0 / sqrt(1.0 + t * t);
  *s = t * (*c);
}

// One round of the parallel ordering, in two phases separated by a grid barrier: (1) the
// rotation of every pair of the round from the old matrix A (cs: c, s of pair J at 2J, 2J + 1;
// nrot counts the rotations), (2) every thread owns 2 x 2 blocks (pair I, pair J) of A and writes
// the rotated block into An, and V's columns of every pair are rotated.  The parameters are
// computed once per pair, not once per block.
__device__ __forceinline__ void jacobi_round_params(const double* __restrict__ A, double* cs, int n, int r,
                                                    unsigned long long* nrot, long long t0, long long tstride) {
  const int h = n / 2;
  for (long long J = t0; J < h; J += tstride) {
    const int p = rr_player((int)J, r, n), q = rr_player(n - 1 - (int)J, r, n);
    double c, s;
    jac_params(A, n, p, q, &c, &s);
    cs[2 * J] = c;
    cs[2 * J + 1] = s;
    if (s != 0.0) atomicAdd(nrot, 1ull);
  }
}

__device__ __forceinline__ void jacobi_round_apply(const double* __restrict__ A, double* __restrict__ An, double* V,
                                                   const double* __restrict__ cs, int n, int r, long long t0,
                                                   long long tstride) {
  const int h = n / 2;
  const long long nblk = (long long)h * h;
  const long long nv = (long long)n * h;
  for (long long o = t0; o < nblk + nv; o += tstride) {
    if (o < nblk) {
      const int I = (int)(o / h), J = (int)(o % h);
      const int pI = rr_player(I, r, n), qI = rr_player(n - 1 - I, r, n);
      const int pJ = rr_player(J, r, n), qJ = rr_player(n - 1 - J, r, n);
      const double cI = cs[2 * I], sI = cs[2 * I + 1], cJ = cs[2 * J], sJ = cs[2 * J + 1];
      const double a00 = A[(size_t)pI * n + pJ], a01 = A[(size_t)pI * n + qJ];
      const double a10 = A[(size_t)qI * n + pJ], a11 = A[(size_t)qI * n + qJ];
      // columns: (x, y) -> (c x - s y, s x + c y)
      const double b00 = cJ * a00 - sJ * a01, b01 = sJ * a00 + cJ * a01;
      const double b10 = cJ * a10 - sJ * a11, b11 = sJ * a10 + cJ * a11;
      // rows
      double d00 = cI * b00 - sI * b10, d01 = cI * b01 - sI * b11;
      double d10 = sI * b00 + cI * b10, d11 = sI * b01 + cI * b11;
      if (I == J && sI != 0.0) { d01 = 0.0; d10 = 0.0; }  // the annihilated pair
      An[(size_t)pI * n + pJ] = d00;
      An[(size_t)pI * n + qJ] = d01;
      An[(size_t)qI * n + pJ] = d10;
      An[(size_t)qI * n + qJ] = d11;
    } else {
      const long long v = o - nblk;
      const int i = (int)(v / h), J = (int)(v % h);
      const double c = cs[2 * J], s = cs[2 * J + 1];
      if (s != 0.0) {
        const int pJ = rr_player(J, r, n), qJ = rr_player(n - 1 - J, r, n);
        const double x = V[(size_t)i * n + pJ], y = V[(size_t)i * n + qJ];
        V[(size_t)i * n + pJ] = c * x - s * y;
        V[(size_t)i * n + qJ] = s * x + c * y;
      }
    }
  }
}

// The whole cyclic Jacobi in one cooperative launch (every CTA resident, so that the grid-wide
// barriers between the phases cannot wait on a CTA that never runs): V = I, then up to
// max_sweeps sweeps of n - 1 rounds, ping-ponging between A and B; a sweep that applied no
// rotation ends the iteration (every thread reads the sweep's counter after the same barrier,
// so all take the same branch).  The diagonal form ends in A.  cnt: 2 device counters (the
// current and the next sweep's); cs: n doubles of scratch; sweeps_out[0] = sweeps used, or -1
// when the limit was reached.
__global__ void __launch_bounds__(256) k_jacobi_coop(double* A, double* B, double* V, double* cs, int n,
                                                     int max_sweeps, unsigned long long* cnt, double* sweeps_out) {
  cg::grid_group grid = cg::this_grid();
  const long long t0 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long ts = (long long)gridDim.x * blockDim.x;
  for (long long o = t0; o < (long long)n * n; o += ts) V[o] = ((o / n) == (o % n)) ? 1.0 : 0.0;
  if (t0 == 0) { cnt[0] = 0ull; cnt[1] = 0ull; }
  grid.sync();
  double* cur = A;
  double* nxt = B;
  int sweeps = -1;
  for (int sw = 0; sw < max_sweeps; ++sw) {
    unsigned long long* c = cnt + (sw & 1);
    if (t0 == 0) cnt[(sw + 1) & 1] = 0ull;  // the next sweep's counter (read by all before the last barrier)
    for (int r = 0; r < n - 1; ++r) {
      jacobi_round_params(cur, cs, n, r, c, t0, ts);
      grid.sync();
      jacobi_round_apply(cur, nxt, V, cs, n, r, t0, ts);
      grid.sync();
      double* t = cur; cur = nxt; nxt = t;
    }
    const unsigned long long rot = *(volatile unsigned long long*)c;
    grid.sync();
    if (rot == 0ull) { sweeps = sw + 1; break; }
  }
  if (cur != A)
    for (long long o = t0; o < (long long)n * n; o += ts) A[o] = cur[o];
  if (t0 == 0) *sweeps_out = (double)sweeps;
}

// A (n x n, n even) -> diagonal form in place (hbuf: a second n x n buffer), V = accumulated
// rotations, info_sweeps = sweeps used (-1 at the sweep limit), all on the device: one
// cooperative launch, no host synchronisation.  cnt: 2 unsigned long long, cs: n doubles of
// device scratch.
cudaError_t jacobi_eig(double* A, double* V, int n, unsigned long long* cnt, double* hbuf, double* cs,
                       double* info_sweeps, int max_sweeps, cudaStream_t s) {
  int dev = 0, nsm = 0, per_sm = 0;
  cudaError_t e;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_jacobi_coop, 256, 0)) != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorLaunchOutOfResources;
  const long long work = (long long)(n / 2) * (n / 2) + (long long)n * (n / 2);
  long long blocks = (work + 255) / 256;
  const long long cap = (long long)nsm * per_sm;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  void* args[] = {&A, &hbuf, &V, &cs, &n, &max_sweeps, &cnt, &info_sweeps};
  return cudaLaunchCooperativeKernel((const void*)k_jacobi_coop, dim3((unsigned)blocks), dim3(256), args, 0, s);
}

// info: [rank kept, min Lambda, max Lambda]; y = f(Lambda) .* (V^T ebar); x = V y
__global__ void k_minsr_scalars(const double* A, int n, int nreal, double rcond, double* info) {
  __shared__ double red[33];
  double mx = -INFINITY, mn = INFINITY;
  // a padding index (n = nreal + 1) has a zero row and column and is never rotated: it stays last
  for (int i = threadIdx.x; i < nreal; i += blockDim.x) {
    const double l = A[(size_t)i * n + i];
    mx = fmax(mx, l);
    mn = fmin(mn, l);
  }
  mx = block_max(mx, red);
  mn = -block_max(-mn, red);
  int cnt = 0;
  for (int i = threadIdx.x; i < nreal; i += blockDim.x) cnt += (rcond > 0.0) ? (A[(size_t)i * n + i] > rcond * mx) : 1;
  const double c = block_sum((double)cnt, red);
  if (threadIdx.x == 0) { info[0] = c; info[1] = mn; info[2] = mx; }
}

__global__ void k_vt_e(const double* A, const double* V, const double* ebar, int n, double lambda, double rcond,
                       const double* info, double* y) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int j = 0; j < n; ++j) s += V[(size_t)j * n + i] * ebar[j];
    const double l = A[(size_t)i * n + i];
    const bool keep = (rcond > 0.0) ? (l > rcond * info[2]) : true;
    y[i] = keep ? s / (l + lambda) : 0.0;
  }
}

__global__ void k_v_y(const double* V, const double* y, int n, double* x) {
  const int lane = threadIdx.x & 31;
  for (int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; j < n; j += (gridDim.x * blockDim.x) >> 5) {
    double s = 0.0;
    for (int i = lane; i < n; i += 32) s += V[(size_t)j * n + i] * y[i];
    s = warp_sum(s);
    if (lane == 0) x[j] = s;
  }
}

__global__ void k_obar_t_x(const double* __restrict__ Ob, const double* __restrict__ x, int Ns, long long Np,
                           double tau, double* dtheta) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < Np; k += (long long)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int i = 0; i < Ns; ++i) s += Ob[(size_t)i * Np + k] * x[i];
    dtheta[k] = -tau * s;
  }
}

// ---- host wrappers
// wsum_dev: one device double for the weight sum (used only when w is not NULL)
template <typename TO>
cudaError_t launch_center(const TO* O, const double* w, int Ns, long long Np, double* mean, double* Obar,
                          double* wsum_dev, cudaStream_t s) {
  if (w) k_wsum<<<1, 256, 0, s>>>(w, Ns, wsum_dev);
  const long long blocks = (Np + 255) / 256;
  k_center<TO><<<(int)(blocks < 4096 ? blocks : 4096), 256, 0, s>>>(O, w, Ns, Np, wsum_dev, mean, Obar);
  return cudaGetLastError();
}
template cudaError_t launch_center<double>(const double*, const double*, int, long long, double*, double*, double*,
                                           cudaStream_t);
template cudaError_t launch_center<float>(const float*, const double*, int, long long, double*, double*, double*,
                                          cudaStream_t);

template <typename TO>
cudaError_t launch_center_cplx(const TO* O, const double* w, int Ns, long long Np, double* W, double* wsum_dev,
                               cudaStream_t s) {
  if (w) k_wsum<<<1, 256, 0, s>>>(w, Ns, wsum_dev);
  const long long blocks = (Np + 255) / 256;
  k_center_cplx<TO><<<(int)(blocks < 4096 ? blocks : 4096), 256, 0, s>>>(O, w, Ns, Np, wsum_dev, W);
  return cudaGetLastError();
}
template cudaError_t launch_center_cplx<double>(const double*, const double*, int, long long, double*, double*,
                                                cudaStream_t);
template cudaError_t launch_center_cplx<float>(const float*, const double*, int, long long, double*, double*,
                                               cudaStream_t);

cudaError_t launch_center_e_cplx(const double* eloc, const double* w, int Ns, double* ebar2, cudaStream_t s) {
  k_center_e_cplx<<<1, 1024, 0, s>>>(eloc, w, Ns, ebar2);
  return cudaGetLastError();
}

cudaError_t launch_unembed(const double* d2, long long Np, double* dtheta, cudaStream_t s) {
  const long long b = (Np + 255) / 256;
  k_unembed<<<(int)(b < 4096 ? (b > 0 ? b : 1) : 4096), 256, 0, s>>>(d2, Np, dtheta);
  return cudaGetLastError();
}

cudaError_t launch_center_e(const double* eloc, const double* w, int Ns, double* ebar, cudaStream_t s) {
  k_center_e<<<1, 1024, 0, s>>>(eloc, w, Ns, ebar);
  return cudaGetLastError();
}

// ---- float-float ("double-single") Gram on the FP32 pipes
// Obar split once into hi = float(x), lo = float(x - hi) (x = hi + lo to about 48 bits).
__global__ void k_split_ff(const double* __restrict__ x, size_t n, float* __restrict__ hi, float* __restrict__ lo) {
  for (size_t o = blockIdx.x * (size_t)blockDim.x + threadIdx.x; o < n; o += (size_t)gridDim.x * blockDim.x) {
    const double v = x[o];
    const float h = __double2float_rn(v);
    hi[o] = h;
    lo[o] = __double2float_rn(v - (double)h);
  }
}

// T = Obar Obar^T from the float pairs: each product a b with a = ah + al, b = bh + bl is taken
// as p + e + c, p = ah bh rounded, e = fma(ah, bh, -p) its exact error, c = ah bl + al bh (al bl,
// about 2^-48 of the product, dropped); the running sum is a float pair (sh, sl): sh + p by
// Knuth's two-sum, its error and e + c into sl, renormalised after every GK k-steps; the result
// is sh + sl in double.  The error-free steps use the _rn intrinsics so that no multiply and add
// are fused.  Same lower-triangle 64 x 64 tiling as k_gram.
__global__ void __launch_bounds__(256) k_gram_ff(const float* __restrict__ Oh, const float* __restrict__ Ol, int Ns,
                                                 long long Np, double* Tm, int ld) {
  __shared__ float Ah[GK][GT + 1], Al[GK][GT + 1], Bh[GK][GT + 1], Bl[GK][GT + 1];
  const int nt = (Ns + GT - 1) / GT;
  int t = blockIdx.x, ti = 0;
  while (t >= ti + 1) { t -= ti + 1; ++ti; }
  const int tj = t;
  if (ti >= nt) return;
  const int r0 = ti * GT, c0 = tj * GT;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  float sh[4][4], sl[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) { sh[i][j] = 0.f; sl[i][j] = 0.f; }
  for (long long k0 = 0; k0 < Np; k0 += GK) {
    for (int o = threadIdx.x; o < GK * GT; o += blockDim.x) {
      const int kk = o % GK, rr = o / GK;
      const long long k = k0 + kk;
      const bool ra = (r0 + rr < Ns && k < Np), rb = (c0 + rr < Ns && k < Np);
      Ah[kk][rr] = ra ? Oh[(size_t)(r0 + rr) * Np + k] : 0.f;
      Al[kk][rr] = ra ? Ol[(size_t)(r0 + rr) * Np + k] : 0.f;
      Bh[kk][rr] = rb ? Oh[(size_t)(c0 + rr) * Np + k] : 0.f;
      Bl[kk][rr] = rb ? Ol[(size_t)(c0 + rr) * Np + k] : 0.f;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < GK; ++kk) {
      float ah[4], al[4], bh[4], bl[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        ah[i] = Ah[kk][ty * 4 + i]; al[i] = Al[kk][ty * 4 + i];
        bh[i] = Bh[kk][tx * 4 + i]; bl[i] = Bl[kk][tx * 4 + i];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const float p = __fmul_rn(ah[i], bh[j]);
          const float e = __fmaf_rn(ah[i], bh[j], -p);
          const float c = __fmaf_rn(ah[i], bl[j], __fmul_rn(al[i], bh[j]));
          const float s0 = __fadd_rn(sh[i][j], p);
          const float bb = __fsub_rn(s0, sh[i][j]);
          const float er = __fadd_rn(__fsub_rn(sh[i][j], __fsub_rn(s0, bb)), __fsub_rn(p, bb));
          sh[i][j] = s0;
          sl[i][j] = __fadd_rn(sl[i][j], __fadd_rn(er, __fadd_rn(e, c)));
        }
    }
    // renormalise the pairs (fast two-sum: |sh| >= |sl|)
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float s0 = __fadd_rn(sh[i][j], sl[i][j]);
        sl[i][j] = __fsub_rn(sl[i][j], __fsub_rn(s0, sh[i][j]));
        sh[i][j] = s0;
      }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int r = r0 + ty * 4 + i, c = c0 + tx * 4 + j;
      // the cross terms make the pair (r, c) and (c, r) round differently: only the lower
      // entry's thread writes both (a diagonal tile would otherwise race on them)
      if (r < Ns && c < Ns && c <= r) {
        const double v = (double)sh[i][j] + (double)sl[i][j];
        Tm[(size_t)r * ld + c] = v;
        Tm[(size_t)c * ld + r] = v;
      }
    }
}

cudaError_t launch_gram_ff(const double* Obar, int Ns, long long Np, float* hi, float* lo, double* Tm, int ld,
                           cudaStream_t s) {
  const size_t n = (size_t)Ns * (size_t)Np;
  k_split_ff<<<1216, 256, 0, s>>>(Obar, n, hi, lo);
  const int nt = (Ns + GT - 1) / GT;
  k_gram_ff<<<nt * (nt + 1) / 2, 256, 0, s>>>(hi, lo, Ns, Np, Tm, ld);
  return cudaGetLastError();
}

cudaError_t launch_gram(const double* Obar, int Ns, long long Np, double* Tm, int ld, cudaStream_t s) {
  const int nt = (Ns + GT - 1) / GT;
  const int ntiles = nt * (nt + 1) / 2;
  k_gram<<<ntiles, 256, 0, s>>>(Obar, Ns, Np, Tm, ld);
  return cudaGetLastError();
}

cudaError_t launch_minsr_apply(const double* A, const double* V, const double* ebar, int n, int nreal, double lambda,
                               double rcond, double* y, double* x, double* info, cudaStream_t s) {
  k_minsr_scalars<<<1, 1024, 0, s>>>(A, n, nreal, rcond, info);
  k_vt_e<<<(n + 255) / 256, 256, 0, s>>>(A, V, ebar, n, lambda, rcond, info, y);
  k_v_y<<<(n * 32 + 255) / 256, 256, 0, s>>>(V, y, n, x);
  return cudaGetLastError();
}

cudaError_t launch_obar_t_x(const double* Obar, const double* x, int Ns, long long Np, double tau, double* dtheta,
                            cudaStream_t s) {
  const long long blocks = (Np + 255) / 256;
  k_obar_t_x<<<(int)(blocks < 4096 ? blocks : 4096), 256, 0, s>>>(Obar, x, Ns, Np, tau, dtheta);
  return cudaGetLastError();
}

}  // namespace peps

namespace peps {
__global__ void k_axpy(double* y, const double* x, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] += x[i];
}
cudaError_t launch_axpy(double* y, const double* x, long long n, cudaStream_t s) {
  const long long b = (n + 255) / 256;
  k_axpy<<<(int)(b < 1024 ? (b > 0 ? b : 1) : 1024), 256, 0, s>>>(y, x, n);
  return cudaGetLastError();
}
}  // namespace peps

// ------------------------------------------------------------------------------------------
// (T + lambda I)^-1 ebar by a blocked right-looking Cholesky factorisation (FP64), the MinSR
// solve when no eigenvalue is cut (rcond == 0): the same operator as the eigendecomposition
// route, V diag(1/(Lambda + lambda)) V^T, at n^3/3 instead of Jacobi's O(n^3) per sweep.
namespace peps {
constexpr int CB = 64;

// Storage of the factor: a plain matrix (double or float), or a float pair hi + lo (about 48
// bits, the float-float factor), read and written through double.
template <typename T>
struct FacPlain {
  T* a;
  __device__ __forceinline__ double get(size_t o) const { return (double)a[o]; }
  __device__ __forceinline__ void set(size_t o, double v) const { a[o] = (T)v; }
};
struct FacFF {
  float *h, *l;
  __device__ __forceinline__ double get(size_t o) const { return (double)h[o] + (double)l[o]; }
  __device__ __forceinline__ void set(size_t o, double v) const {
    const float hi = __double2float_rn(v);
    h[o] = hi;
    l[o] = __double2float_rn(v - (double)hi);
  }
};

// sqrt(d) and 1 / sqrt(d) of a pivot d > 0.  Double: the single-precision reciprocal square root
// refined by two Newton steps y <- y (3 - d y^2) / 2 (each doubles the correct bits: 23 -> 46 ->
// beyond double), a short chain of FP64 operations where sqrt and a division would each take a
// long one on a GPU with few FP64 units; outside the float range the plain sqrt and division.
__device__ __forceinline__ void pivot_sqrt(double d, double& s, double& r) {
  if (d > 1e-30 && d < 1e30) {
    double y = (double)rsqrtf((float)d);
    y = y * fma(-0.5 * d, y * y, 1.5);
    y = y * fma(-0.5 * d, y * y, 1.5);
    r = y;
    s = d * y;
  } else {
    s = sqrt(d);
    r = 1.0 / s;
  }
}
__device__ __forceinline__ void pivot_sqrt(float d, float& s, float& r) {
  s = sqrtf(d);
  r = 1.f / s;
}

// factor the CB x CB diagonal block at (k0, k0) in place (lower triangle), one CTA.  Per column
// j: thread 0 takes the pivot's square root and its reciprocal; then every thread updates its
// share of the trailing triangle with column j still unscaled (a_il -= a_ij a_lj / a_jj; four
// threads per row, the columns of a row interleaved) and scales column j - 1 by its reciprocal
// (no column is read and written in the same phase): two barriers per column.
// gate (may be NULL): a device flag; the launch does nothing while it is 0 (a factorisation
// enqueued before the decision whether it is needed has been taken on the device)
template <typename T, typename F>
__global__ void __launch_bounds__(256) k_chol_diag(F A, int n, int k0, int* bad, const int* gate) {
  if (gate && !*gate) return;
  __shared__ T L[CB][CB + 1];
  __shared__ T rd[CB];
  const int nb = min(CB, n - k0);
  const int tid = threadIdx.x, row = tid >> 2, part = tid & 3;
  for (int o = tid; o < nb * nb; o += blockDim.x) {
    const int i = o / nb, j = o % nb;
    L[i][j] = (T)A.get((size_t)(k0 + i) * n + k0 + j);
  }
  __syncthreads();
  for (int j = 0; j < nb; ++j) {
    if (tid == 0) {
      const T d = L[j][j];
      const bool ok = d > T(0);  // false for NaN too
      T dj, rj;
      pivot_sqrt(ok ? d : T(1), dj, rj);
      if (!ok) *bad = 1;
      L[j][j] = dj;
      rd[j] = rj;
    }
    __syncthreads();
    const T r2 = rd[j] * rd[j];
    const int i = j + 1 + row;
    if (i < nb) {
      const T lij = L[i][j] * r2;
      for (int l = j + 1 + part; l <= i; l += 4) L[i][l] -= lij * L[l][j];
    }
    if (j > 0 && tid > j - 1 && tid < nb) L[tid][j - 1] *= rd[j - 1];
    __syncthreads();
  }
  if (nb > 0 && tid > nb - 1 && tid < nb) L[tid][nb - 1] *= rd[nb - 1];  // (no row below the last pivot)
  __syncthreads();
  for (int o = tid; o < nb * nb; o += blockDim.x) {
    const int i = o / nb, j = o % nb;
    A.set((size_t)(k0 + i) * n + k0 + j, (j <= i) ? (double)L[i][j] : 0.0);
  }
}

// panel below the diagonal block: A_ik <- A_ik L_kk^-T (the block is full, CB columns: the panel
// exists only when CB rows follow the diagonal block).  TRSM_RB rows per CTA, one thread per
// row, the row in registers and solved column by column: each solved entry (times the diagonal
// reciprocal) updates the later entries, independent multiply-adds.
constexpr int TRSM_RB = 32;
template <typename T, typename F>
__global__ void __launch_bounds__(TRSM_RB) k_chol_trsm(F A, int n, int k0, const int* gate) {
  if (gate && !*gate) return;
  __shared__ T L[CB][CB + 1];
  __shared__ T rd[CB];
  for (int o = threadIdx.x; o < CB * CB; o += blockDim.x) L[o / CB][o % CB] = (T)A.get((size_t)(k0 + o / CB) * n + k0 + o % CB);
  __syncthreads();
  for (int j = threadIdx.x; j < CB; j += blockDim.x) rd[j] = T(1) / L[j][j];
  __syncthreads();
  const int r = k0 + CB + blockIdx.x * TRSM_RB + threadIdx.x;
  if (r >= n) return;
  const size_t ar = (size_t)r * n + k0;
  T x[CB];
#pragma unroll
  for (int j = 0; j < CB; ++j) x[j] = (T)A.get(ar + j);
#pragma unroll
  for (int j = 0; j < CB; ++j) {
    x[j] *= rd[j];
#pragma unroll
    for (int jj = j + 1; jj < CB; ++jj) x[jj] -= x[j] * L[jj][j];
  }
#pragma unroll
  for (int j = 0; j < CB; ++j) A.set(ar + j, (double)x[j]);
}

// trailing update A_ij -= A_ik A_jk^T for the lower-triangle tiles right of/below the panel
template <typename T>
__global__ void __launch_bounds__(256) k_chol_update(T* A, int n, int k0, const int* gate) {
  if (gate && !*gate) return;
  __shared__ T As[CB][CB + 1], Bs[CB][CB + 1];
  const int nt = (n - k0 - CB + CB - 1) / CB;
  int t = blockIdx.x, ti = 0;
  while (t >= ti + 1) { t -= ti + 1; ++ti; }
  const int tj = t;
  if (ti >= nt) return;
  const int r0 = k0 + CB + ti * CB, c0 = k0 + CB + tj * CB;
  for (int o = threadIdx.x; o < CB * CB; o += blockDim.x) {
    const int rr = o / CB, kk = o % CB;
    As[kk][rr] = (r0 + rr < n) ? A[(size_t)(r0 + rr) * n + k0 + kk] : T(0);
    Bs[kk][rr] = (c0 + rr < n) ? A[(size_t)(c0 + rr) * n + k0 + kk] : T(0);
  }
  __syncthreads();
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  T acc[4][4] = {};
  for (int kk = 0; kk < CB; ++kk) {
    T a[4], b[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) { a[i] = As[kk][ty * 4 + i]; b[i] = Bs[kk][tx * 4 + i]; }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int r = r0 + ty * 4 + i, c = c0 + tx * 4 + j;
      if (r < n && c < n && c <= r) A[(size_t)r * n + c] -= acc[i][j];
    }
}

// The same trailing update on the float-float factor: the panel's columns as float pairs, each
// product a b = (ah + al)(bh + bl) taken as p + e + c (p = ah bh rounded, e its exact error by
// fma, c = ah bl + al bh; al bl, about 2^-48 of the product, dropped) and summed into a float
// pair by Knuth's two-sum, as the float-float Gram does; the pair is then subtracted from A_ij
// with one more two-sum and stored renormalised.
constexpr int UK = 32;  // panel columns staged per pass (four UK x CB float tiles: 33 KB)
__global__ void __launch_bounds__(256) k_chol_update_ff(float* Ah, float* Al, int n, int k0, const int* gate) {
  if (gate && !*gate) return;
  __shared__ float Ph[UK][CB + 1], Pl[UK][CB + 1], Qh[UK][CB + 1], Ql[UK][CB + 1];
  const int nt = (n - k0 - CB + CB - 1) / CB;
  int t = blockIdx.x, ti = 0;
  while (t >= ti + 1) { t -= ti + 1; ++ti; }
  const int tj = t;
  if (ti >= nt) return;
  const int r0 = k0 + CB + ti * CB, c0 = k0 + CB + tj * CB;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  float sh[4][4], sl[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) { sh[i][j] = 0.f; sl[i][j] = 0.f; }
  for (int kc = 0; kc < CB; kc += UK) {
  __syncthreads();
  for (int o = threadIdx.x; o < UK * CB; o += blockDim.x) {
    const int rr = o / UK, kk = o % UK;
    const bool ra = r0 + rr < n, rb = c0 + rr < n;
    const size_t oa = (size_t)(r0 + rr) * n + k0 + kc + kk, ob = (size_t)(c0 + rr) * n + k0 + kc + kk;
    Ph[kk][rr] = ra ? Ah[oa] : 0.f;
    Pl[kk][rr] = ra ? Al[oa] : 0.f;
    Qh[kk][rr] = rb ? Ah[ob] : 0.f;
    Ql[kk][rr] = rb ? Al[ob] : 0.f;
  }
  __syncthreads();
#pragma unroll 4
  for (int kk = 0; kk < UK; ++kk) {
    float ah[4], al[4], bh[4], bl[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      ah[i] = Ph[kk][ty * 4 + i]; al[i] = Pl[kk][ty * 4 + i];
      bh[i] = Qh[kk][tx * 4 + i]; bl[i] = Ql[kk][tx * 4 + i];
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float p = __fmul_rn(ah[i], bh[j]);
        const float e = __fmaf_rn(ah[i], bh[j], -p);
        const float c = __fmaf_rn(ah[i], bl[j], __fmul_rn(al[i], bh[j]));
        const float s0 = __fadd_rn(sh[i][j], p);
        const float bb = __fsub_rn(s0, sh[i][j]);
        const float er = __fadd_rn(__fsub_rn(sh[i][j], __fsub_rn(s0, bb)), __fsub_rn(p, bb));
        sh[i][j] = s0;
        sl[i][j] = __fadd_rn(sl[i][j], __fadd_rn(er, __fadd_rn(e, c)));
      }
  }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int r = r0 + ty * 4 + i, c = c0 + tx * 4 + j;
      if (r < n && c < n && c <= r) {
        const size_t o = (size_t)r * n + c;
        // (xh + xl) - (sh + sl): two-sum of the high parts, the rest into the low part
        const float xh = Ah[o], xl = Al[o];
        const float d0 = __fsub_rn(xh, sh[i][j]);
        const float bb = __fsub_rn(d0, xh);
        const float er = __fadd_rn(__fsub_rn(xh, __fsub_rn(d0, bb)), __fsub_rn(-sh[i][j], bb));
        const float lo = __fadd_rn(er, __fsub_rn(xl, sl[i][j]));
        const float hi = __fadd_rn(d0, lo);
        Ah[o] = hi;
        Al[o] = __fsub_rn(lo, __fsub_rn(hi, d0));
      }
    }
}

__global__ void k_add_diag(double* A, int n, int nreal, double lambda, const int* gate) {
  if (gate && !*gate) return;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    A[(size_t)i * n + i] += (i < nreal) ? lambda : 1.0;  // a padding index gets 1 (its rhs is 0)
}

// L y = v then L^T z = y by blocks of CB rows, one launch per block and direction, spread over
// the whole GPU (the single-CTA form held every row update on one SM).  In a forward launch
// every CTA stages the diagonal block in shared memory and solves its CB rows from v (read only
// in that launch) with one warp, column by column in registers (lane l holds rows l and l + 32:
// each solved entry is broadcast by a shuffle and subtracted from the rows below it), CTA 0
// stores them in y, and the warps of all CTAs subtract the block's contribution from the rows
// below it (one warp per row, disjoint rows); the backward launch mirrors it on L^T with four
// threads per row above the block.  The right-hand sides are carried in FP64 whatever the
// factor's storage.
template <typename F>
__global__ void __launch_bounds__(256) k_trsv_fwd(F L, int n, int k0, double* v, double* y, const int* gate) {
  if (gate && !*gate) return;
  __shared__ double Ld[CB][CB + 1];
  __shared__ double ys[CB];
  __shared__ double rdg[CB];
  const int nb = min(CB, n - k0);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int o = threadIdx.x; o < nb * nb; o += blockDim.x) {
    const int i = o / nb, j = o - i * nb;
    if (j <= i) Ld[i][j] = L.get((size_t)(k0 + i) * n + k0 + j);
  }
  __syncthreads();
  if (threadIdx.x < nb) rdg[threadIdx.x] = 1.0 / Ld[threadIdx.x][threadIdx.x];
  __syncthreads();
  if (warp == 0) {
    double v0 = (lane < nb) ? v[k0 + lane] : 0.0, v1 = (lane + 32 < nb) ? v[k0 + lane + 32] : 0.0;
    for (int j = 0; j < nb; ++j) {
      const double vj = (j < 32) ? __shfl_sync(0xffffffffu, v0, j) : __shfl_sync(0xffffffffu, v1, j - 32);
      const double yj = vj * rdg[j];
      if (lane == 0) ys[j] = yj;
      if (lane > j && lane < nb) v0 -= Ld[lane][j] * yj;
      if (lane + 32 > j && lane + 32 < nb) v1 -= Ld[lane + 32][j] * yj;
    }
  }
  __syncthreads();
  if (blockIdx.x == 0)
    for (int j = threadIdx.x; j < nb; j += blockDim.x) y[k0 + j] = ys[j];
  const int nw = blockDim.x >> 5;
  for (int i = k0 + nb + blockIdx.x * nw + warp; i < n; i += gridDim.x * nw) {
    const size_t li = (size_t)i * n + k0;
    double s = 0.0;
    for (int l = lane; l < nb; l += 32) s += L.get(li + l) * ys[l];
    s = warp_sum(s);
    if (lane == 0) v[i] -= s;
  }
}

template <typename F>
__global__ void __launch_bounds__(256) k_trsv_bwd(F L, int n, int k0, double* y, double* z, const int* gate) {
  if (gate && !*gate) return;
  __shared__ double Ld[CB][CB + 1];
  __shared__ double zs[CB];
  __shared__ double rdg[CB];
  const int nb = min(CB, n - k0);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int o = threadIdx.x; o < nb * nb; o += blockDim.x) {
    const int i = o / nb, j = o - i * nb;
    if (j <= i) Ld[i][j] = L.get((size_t)(k0 + i) * n + k0 + j);
  }
  __syncthreads();
  if (threadIdx.x < nb) rdg[threadIdx.x] = 1.0 / Ld[threadIdx.x][threadIdx.x];
  __syncthreads();
  if (warp == 0) {
    double y0 = (lane < nb) ? y[k0 + lane] : 0.0, y1 = (lane + 32 < nb) ? y[k0 + lane + 32] : 0.0;
    for (int j = nb - 1; j >= 0; --j) {
      const double yj = (j < 32) ? __shfl_sync(0xffffffffu, y0, j) : __shfl_sync(0xffffffffu, y1, j - 32);
      const double zj = yj * rdg[j];
      if (lane == 0) zs[j] = zj;
      if (lane < j) y0 -= Ld[j][lane] * zj;
      if (lane + 32 < j) y1 -= Ld[j][lane + 32] * zj;
    }
  }
  __syncthreads();
  if (blockIdx.x == 0)
    for (int j = threadIdx.x; j < nb; j += blockDim.x) z[k0 + j] = zs[j];
  // rows above the block: four threads per row, each summing a quarter of the block's columns,
  // combined by two shuffles (warp-uniform trips)
  const int tot = 4 * k0;
  for (int t0 = blockIdx.x * blockDim.x; t0 < tot; t0 += gridDim.x * blockDim.x) {
    const int t = t0 + threadIdx.x, i = t >> 2, part = t & 3;
    double s = 0.0;
    if (t < tot)
      for (int l = part; l < nb; l += 4) s += L.get((size_t)(k0 + l) * n + i) * zs[l];
    s += __shfl_xor_sync(0xffffffffu, s, 1);
    s += __shfl_xor_sync(0xffffffffu, s, 2);
    if (t < tot && part == 0) y[i] -= s;
  }
}

__global__ void k_vcopy(const double* src, double* dst, int n, const int* gate) {
  if (gate && !*gate) return;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) dst[i] = src[i];
}
__global__ void k_vadd(const double* src, double* dst, int n, const int* gate) {
  if (gate && !*gate) return;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) dst[i] += src[i];
}

// (L L^T)^-1 b into x (x += it when accumulate).  accumulate == 0: b is read only (copied to x
// first).  accumulate != 0: b is overwritten (it carries the solve).  scratch: n doubles.
// Returns the launches issued.
template <typename F>
static long long chol_apply(F L, int n, double* b, double* x, int accumulate, double* scratch, const int* gate,
                            cudaStream_t s) {
  long long launches = 0;
  double* v = accumulate ? b : x;
  if (!accumulate) {
    k_vcopy<<<(n + 255) / 256, 256, 0, s>>>(b, x, n, gate);
    ++launches;
  }
  for (int k0 = 0; k0 < n; k0 += CB) {
    const int rows = n - k0 - CB;  // rows below the block
    const int grid = rows > 0 ? min(2 * 152, (rows + 7) / 8) : 1;
    k_trsv_fwd<F><<<grid, 256, 0, s>>>(L, n, k0, v, scratch, gate);
    ++launches;
  }
  // the forward pass is done with v: the backward one writes the solution there
  for (int k0 = ((n - 1) / CB) * CB; k0 >= 0; k0 -= CB) {
    const int grid = k0 > 0 ? min(4 * 152, (4 * k0 + 255) / 256) : 1;
    k_trsv_bwd<F><<<grid, 256, 0, s>>>(L, n, k0, scratch, v, gate);
    ++launches;
  }
  if (accumulate) {
    k_vadd<<<(n + 255) / 256, 256, 0, s>>>(v, x, n, gate);
    ++launches;
  }
  return launches;
}

// blocked factorisation of the lower triangle of A (n x n) in place; returns launches
template <typename T>
static long long chol_factor(T* A, int n, int* bad, const int* gate, cudaStream_t s) {
  long long launches = 0;
  for (int k0 = 0; k0 < n; k0 += CB) {
    k_chol_diag<T, FacPlain<T>><<<1, 256, 0, s>>>(FacPlain<T>{A}, n, k0, bad, gate);
    ++launches;
    const int rest = n - k0 - CB;
    if (rest > 0) {
      const int nrb = (rest + CB - 1) / CB;
      k_chol_trsm<T, FacPlain<T>><<<(rest + TRSM_RB - 1) / TRSM_RB, TRSM_RB, 0, s>>>(FacPlain<T>{A}, n, k0, gate);
      k_chol_update<T><<<nrb * (nrb + 1) / 2, 256, 0, s>>>(A, n, k0, gate);
      launches += 2;
    }
  }
  return launches;
}

// gate (may be NULL): the fallback flag of the mixed solve; a factorisation it gates marks the
// fallback in info[2] = 0
__global__ void k_chol_info(const int* bad, int nreal, double* info, const int* gate) {
  if (gate && !*gate) return;
  info[0] = *bad ? -1.0 : (double)nreal;
  info[1] = NAN;
  info[2] = gate ? 0.0 : NAN;
}

__global__ void k_zero_int(int* p, const int* gate) {
  if (gate && !*gate) return;
  *p = 0;
}

// Returns launches issued; *err for a CUDA error.  info[0] = Ns (-1 if T + lambda was not
// positive definite in floating point), info[1..2] = NaN (no eigenvalues computed).  With a gate,
// every launch does nothing unless *gate != 0 when it runs.
long long chol_solve(double* A, int n, int nreal, double lambda, const double* ebar, double* x, int* bad,
                     double* info, const int* gate, double* scratch, cudaStream_t s, cudaError_t* err) {
  long long launches = 0;
  k_zero_int<<<1, 1, 0, s>>>(bad, gate);
  k_add_diag<<<(n + 255) / 256, 256, 0, s>>>(A, n, nreal, lambda, gate);
  launches += 2;
  launches += chol_factor<double>(A, n, bad, gate, s);
  launches += chol_apply(FacPlain<double>{A}, n, const_cast<double*>(ebar), x, 0, scratch, gate, s);
  k_chol_info<<<1, 1, 0, s>>>(bad, nreal, info, gate);
  launches += 1;
  *err = cudaGetLastError();
  return launches;
}

// ---- mixed-precision solve: FP32 factor of T + lambda, FP64 residuals
// A32 (lower) = float(A + d) with d_i = lambda (i < nreal) or 1 (padding); the FP64 A is kept
__global__ void k_lower_to_f32(const double* A, float* A32, int n, int nreal, double lambda) {
  const size_t nn = (size_t)n * n;
  for (size_t o = blockIdx.x * (size_t)blockDim.x + threadIdx.x; o < nn; o += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(o / n), j = (int)(o % n);
    double v = (j <= i) ? A[o] : 0.0;
    if (i == j) v += (i < nreal) ? lambda : 1.0;
    A32[o] = (float)v;
  }
}

// A[j][i] = A[i][j] for j > i (the Gram kernels may leave the upper triangle unset)
__global__ void k_mirror(double* A, int n) {
  const size_t nn = (size_t)n * n;
  for (size_t o = blockIdx.x * (size_t)blockDim.x + threadIdx.x; o < nn; o += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(o / n), j = (int)(o % n);
    if (j > i) A[o] = A[(size_t)j * n + i];
  }
}

// r = b - (A + d) x, one warp per row; every block writes its partial |r|^2 and |b|^2 to
// part[2 blockIdx.x ..] (summed in a fixed order by k_rnorm, so that the norms, and the fallback
// decision taken on them, do not depend on the order in which blocks finish)
__global__ void k_residual(const double* __restrict__ A, int n, int nreal, double lambda, const double* b,
                           const double* x, double* r, double* part) {
  __shared__ double red_r[8], red_b[8];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nwarps = (gridDim.x * blockDim.x) >> 5;
  double acc_r = 0.0, acc_b = 0.0;
  for (int i = warp; i < n; i += nwarps) {
    double sacc = 0.0;
    for (int j = lane; j < n; j += 32) sacc += A[(size_t)i * n + j] * x[j];
    sacc = warp_sum(sacc);
    const double ri = b[i] - sacc - ((i < nreal) ? lambda : 1.0) * x[i];
    if (lane == 0) {
      r[i] = ri;
      acc_r += ri * ri;
      acc_b += b[i] * b[i];
    }
  }
  if (lane == 0) { red_r[wib] = acc_r; red_b[wib] = acc_b; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double sr = 0.0, sb = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { sr += red_r[w]; sb += red_b[w]; }
    part[2 * blockIdx.x] = sr;
    part[2 * blockIdx.x + 1] = sb;
  }
}

// rn[0..1] = the blocks' partial norms summed in block order (one thread)
__global__ void k_rnorm(const double* part, int nblocks, double* rn) {
  double sr = 0.0, sb = 0.0;
  for (int k = 0; k < nblocks; ++k) { sr += part[2 * k]; sb += part[2 * k + 1]; }
  rn[0] = sr;
  rn[1] = sb;
}

// info of the FP32 solve; need64 = 1 when its factor broke down or the refined relative residual
// stayed above 1e-10 (the FP64 factorisation then replaces it, gated on this flag)
__global__ void k_mixed_info(const int* bad, int nreal, const double* rn, int iters, double* info, int* need64) {
  info[0] = *bad ? -1.0 : (double)nreal;
  info[1] = (rn[1] > 0.0) ? sqrt(rn[0] / rn[1]) : 0.0;
  info[2] = (double)iters;
  *need64 = (*bad || !(rn[0] <= 1e-20 * rn[1])) ? 1 : 0;
}

long long chol_solve_mixed(double* A, float* A32, int n, int nreal, double lambda, const double* ebar, double* x,
                           double* r, double* rn, double* part, int iters, int* bad, double* info, int* need64,
                           double* scratch, cudaStream_t s, cudaError_t* err) {
  long long launches = 0;
  cudaMemsetAsync(bad, 0, sizeof(int), s);
  k_mirror<<<1024, 256, 0, s>>>(A, n);
  k_lower_to_f32<<<1024, 256, 0, s>>>(A, A32, n, nreal, lambda);
  launches += 2;
  launches += chol_factor<float>(A32, n, bad, nullptr, s);
  launches += chol_apply(FacPlain<float>{A32}, n, const_cast<double*>(ebar), x, 0, scratch, nullptr, s);
  const int rgrid = (n + 7) / 8;
  for (int it = 0; it < iters; ++it) {
    k_residual<<<rgrid, 256, 0, s>>>(A, n, nreal, lambda, ebar, x, r, part);
    launches += 1 + chol_apply(FacPlain<float>{A32}, n, r, x, 1, scratch, nullptr, s);
  }
  k_residual<<<rgrid, 256, 0, s>>>(A, n, nreal, lambda, ebar, x, r, part);
  k_rnorm<<<1, 1, 0, s>>>(part, rgrid, rn);
  k_mixed_info<<<1, 1, 0, s>>>(bad, nreal, rn, iters, info, need64);
  launches += 3;
  *err = cudaGetLastError();
  return launches;
}

// ---- float-float factor (solve = 2): T + lambda split into float pairs (about 48 bits, the
// precision of the float-float Gram that usually produced T), the trailing updates on the FP32
// pipes (k_chol_update_ff), the diagonal blocks and panels in FP64 through the pair accessor,
// then `iters` steps of refinement with FP64 residuals as in the FP32 mixed solve.  On this part
// FP64 runs at 1/64 of the FP32 rate, so the factor's n^3/6 multiply-adds cost several times
// less as float pairs (about 13 FP32 operations each) than in FP64.  The FP64 factorisation
// replaces it only when the pair factorisation breaks down (need64 = 1); info[1] is the relative
// residual after refinement.
__global__ void k_lower_to_ff(const double* A, float* Fh, float* Fl, int n, int nreal, double lambda) {
  const size_t nn = (size_t)n * n;
  for (size_t o = blockIdx.x * (size_t)blockDim.x + threadIdx.x; o < nn; o += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(o / n), j = (int)(o % n);
    double v = (j <= i) ? A[o] : 0.0;
    if (i == j) v += (i < nreal) ? lambda : 1.0;
    const float h = __double2float_rn(v);
    Fh[o] = h;
    Fl[o] = __double2float_rn(v - (double)h);
  }
}

__global__ void k_ff_info(const int* bad, int nreal, const double* rn, int iters, double* info, int* need64) {
  info[0] = *bad ? -1.0 : (double)nreal;
  info[1] = (rn[1] > 0.0) ? sqrt(rn[0] / rn[1]) : 0.0;
  info[2] = (double)iters;
  *need64 = *bad ? 1 : 0;
}

long long chol_solve_ff(double* A, float* Fh, float* Fl, int n, int nreal, double lambda, const double* ebar, double* x,
                        double* r, double* rn, double* part, int iters, int* bad, double* info, int* need64,
                        double* scratch, cudaStream_t s, cudaError_t* err) {
  long long launches = 0;
  cudaMemsetAsync(bad, 0, sizeof(int), s);
  k_mirror<<<1024, 256, 0, s>>>(A, n);
  k_lower_to_ff<<<1024, 256, 0, s>>>(A, Fh, Fl, n, nreal, lambda);
  launches += 2;
  const FacFF F{Fh, Fl};
  for (int k0 = 0; k0 < n; k0 += CB) {
    k_chol_diag<double, FacFF><<<1, 256, 0, s>>>(F, n, k0, bad, nullptr);
    ++launches;
    const int rest = n - k0 - CB;
    if (rest > 0) {
      const int nrb = (rest + CB - 1) / CB;
      k_chol_trsm<double, FacFF><<<(rest + TRSM_RB - 1) / TRSM_RB, TRSM_RB, 0, s>>>(F, n, k0, nullptr);
      k_chol_update_ff<<<nrb * (nrb + 1) / 2, 256, 0, s>>>(Fh, Fl, n, k0, nullptr);
      launches += 2;
    }
  }
  launches += chol_apply(F, n, const_cast<double*>(ebar), x, 0, scratch, nullptr, s);
  const int rgrid = (n + 7) / 8;
  for (int it = 0; it < iters; ++it) {
    k_residual<<<rgrid, 256, 0, s>>>(A, n, nreal, lambda, ebar, x, r, part);
    launches += 1 + chol_apply(F, n, r, x, 1, scratch, nullptr, s);
  }
  k_residual<<<rgrid, 256, 0, s>>>(A, n, nreal, lambda, ebar, x, r, part);
  k_rnorm<<<1, 1, 0, s>>>(part, rgrid, rn);
  k_ff_info<<<1, 1, 0, s>>>(bad, nreal, rn, iters, info, need64);
  launches += 3;
  *err = cudaGetLastError();
  return launches;
}
}  // namespace peps

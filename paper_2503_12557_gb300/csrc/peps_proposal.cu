// Learned proposal for the Metropolis chains (not in the paper; required by the hot-path
// specification): a 3-layer 3x3 convolutional network on the +-1 configuration map gives
// per-site logits l(S); a move draws every site of S' from Bernoulli(sigmoid(l_i(S))) and is
// accepted with min(1, |psi(S')|^2 q(S|S') / (|psi(S)|^2 q(S'|S))), so the chain stays exact.
// Training minimises the mean binary cross-entropy of a later configuration of the chain given
// the current one, with Adam.
//
// Weights are packed W1 (C,1,3,3), b1 (C), W2 (C,C,3,3), b2 (C), W3 (1,C,3,3), b3 (1).
// Precision variants: TW = double with TA = double (the variant checked against the FP64
// oracle), TW = bf16 with TA = float (the fast variant).  Gradients, Adam state and the master
// weights are FP64.
#include <cuda_bf16.h>

#include "peps_kernels.cuh"

namespace peps {

__host__ __device__ inline int prop_nweights(int C) { return 9 * C + C + 9 * C * C + C + 9 * C + 1; }

template <typename TA>
__device__ __forceinline__ TA sigm(TA z) { return TA(1) / (TA(1) + exp(-z)); }
template <typename TA>
__device__ __forceinline__ TA softplus_(TA z) { return fmax(z, TA(0)) + log1p(exp(-fabs(z))); }

template <typename TW>
__device__ __forceinline__ double wload(const TW* w, int i) { return (double)w[i]; }
template <>
__device__ __forceinline__ double wload<__nv_bfloat16>(const __nv_bfloat16* w, int i) { return (double)__bfloat162float(w[i]); }

struct PropGeo {
  int Lx, Ly, C, N;
};

// y[o][p] = b[o] + sum_{c,di,dj} W[o][c][di][dj] x[c][p + (di-1, dj-1)]   (zero padded)
template <typename TA>
__device__ void conv_fwd(const PropGeo& g, const TA* x, int Cin, const TA* W, const TA* b, int Cout, TA* y) {
  for (int o = threadIdx.x; o < Cout * g.N; o += blockDim.x) {
    const int oc = o / g.N, p = o % g.N, i = p / g.Ly, j = p % g.Ly;
    TA s = b[oc];
    for (int c = 0; c < Cin; ++c) {
      const TA* Wc = W + ((size_t)oc * Cin + c) * 9;
      const TA* xc = x + (size_t)c * g.N;
      for (int di = 0; di < 3; ++di) {
        const int ii = i + di - 1;
        if (ii < 0 || ii >= g.Lx) continue;
        for (int dj = 0; dj < 3; ++dj) {
          const int jj = j + dj - 1;
          if (jj < 0 || jj >= g.Ly) continue;
          s += Wc[di * 3 + dj] * xc[ii * g.Ly + jj];
        }
      }
    }
    y[o] = s;
  }
  __syncthreads();
}

// shared-memory layout of one CTA: weights (TA), x, z1, h1, z2, h2, l, and two gradient maps
template <typename TA>
struct PropSmem {
  TA *w, *x, *z1, *h1, *z2, *h2, *l, *g1, *g2;
  double* gacc;  // per-CTA gradient accumulator (training only)
};

template <typename TA>
__device__ PropSmem<TA> prop_carve(const PropGeo& g, char* smem, bool train) {
  PropSmem<TA> s;
  const int nw = prop_nweights(g.C);
  TA* p = (TA*)smem;
  s.w = p; p += nw;
  s.x = p; p += g.N;
  s.z1 = p; p += g.C * g.N;
  s.h1 = p; p += g.C * g.N;
  s.z2 = p; p += g.C * g.N;
  s.h2 = p; p += g.C * g.N;
  s.l = p; p += g.N;
  s.g1 = p; p += g.C * g.N;
  s.g2 = p; p += g.C * g.N;
  size_t off = (size_t)((char*)p - smem);
  off = (off + 15) / 16 * 16;
  s.gacc = train ? (double*)(smem + off) : nullptr;
  return s;
}

template <typename TA>
__device__ void prop_forward_one(const PropGeo& g, const PropSmem<TA>& s, const uint8_t* S) {
  const int C = g.C;
  const TA* W1 = s.w;
  const TA* b1 = W1 + 9 * C;
  const TA* W2 = b1 + C;
  const TA* b2 = W2 + 9 * C * C;
  const TA* W3 = b2 + C;
  const TA* b3 = W3 + 9 * C;
  for (int p = threadIdx.x; p < g.N; p += blockDim.x) s.x[p] = TA(1) - TA(2) * (TA)S[p];
  __syncthreads();
  conv_fwd(g, s.x, 1, W1, b1, C, s.z1);
  for (int o = threadIdx.x; o < C * g.N; o += blockDim.x) s.h1[o] = s.z1[o] * sigm(s.z1[o]);
  __syncthreads();
  conv_fwd(g, s.h1, C, W2, b2, C, s.z2);
  for (int o = threadIdx.x; o < C * g.N; o += blockDim.x) s.h2[o] = s.z2[o] * sigm(s.z2[o]);
  __syncthreads();
  conv_fwd(g, s.h2, C, W3, b3, 1, s.l);
}

template <typename TA, typename TW>
__device__ void prop_load_weights(const PropGeo& g, const TW* w, TA* ws) {
  for (int i = threadIdx.x; i < prop_nweights(g.C); i += blockDim.x) ws[i] = (TA)wload(w, i);
  __syncthreads();
}

template <typename TA, typename TW>
__global__ void __launch_bounds__(256) k_prop_logits(PropGeo g, const TW* __restrict__ w, const uint8_t* __restrict__ S,
                                                     int Ns, double* logits) {
  extern __shared__ __align__(16) char smem[];
  PropSmem<TA> s = prop_carve<TA>(g, smem, false);
  prop_load_weights<TA, TW>(g, w, s.w);
  for (int c = blockIdx.x; c < Ns; c += gridDim.x) {
    prop_forward_one<TA>(g, s, S + (size_t)c * g.N);
    for (int p = threadIdx.x; p < g.N; p += blockDim.x) logits[(size_t)c * g.N + p] = (double)s.l[p];
    __syncthreads();
  }
}

// gradient of y = conv(x, W, b) given gy: gW, gb accumulated into gacc (double, per CTA),
// gx (optional) written
template <typename TA>
__device__ void conv_bwd(const PropGeo& g, const TA* x, int Cin, const TA* W, int Cout, const TA* gy, double* gW,
                         double* gb, TA* gx) {
  // weights: gW[o][c][di][dj] += sum_p gy[o][p] x[c][p + off]
  for (int t = threadIdx.x; t < Cout * Cin * 9; t += blockDim.x) {
    const int k = t % 9, c = (t / 9) % Cin, o = t / (9 * Cin), di = k / 3, dj = k % 3;
    TA s = 0;
    for (int i = 0; i < g.Lx; ++i) {
      const int ii = i + di - 1;
      if (ii < 0 || ii >= g.Lx) continue;
      for (int j = 0; j < g.Ly; ++j) {
        const int jj = j + dj - 1;
        if (jj < 0 || jj >= g.Ly) continue;
        s += gy[(size_t)o * g.N + i * g.Ly + j] * x[(size_t)c * g.N + ii * g.Ly + jj];
      }
    }
    gW[t] += (double)s;
  }
  for (int o = threadIdx.x; o < Cout; o += blockDim.x) {
    TA s = 0;
    for (int p = 0; p < g.N; ++p) s += gy[(size_t)o * g.N + p];
    gb[o] += (double)s;
  }
  if (gx) {
    // gx[c][q] = sum_{o,di,dj} W[o][c][di][dj] gy[o][q - off]
    for (int t = threadIdx.x; t < Cin * g.N; t += blockDim.x) {
      const int c = t / g.N, q = t % g.N, i = q / g.Ly, j = q % g.Ly;
      TA s = 0;
      for (int o = 0; o < Cout; ++o)
        for (int di = 0; di < 3; ++di) {
          const int pi = i - di + 1;
          if (pi < 0 || pi >= g.Lx) continue;
          for (int dj = 0; dj < 3; ++dj) {
            const int pj = j - dj + 1;
            if (pj < 0 || pj >= g.Ly) continue;
            s += W[((size_t)o * Cin + c) * 9 + di * 3 + dj] * gy[(size_t)o * g.N + pi * g.Ly + pj];
          }
        }
      gx[t] = s;
    }
  }
  __syncthreads();
}

// forward + backward of the mean BCE over Ns (input, target) pairs; grad (double, zeroed by
// the caller) and loss (double) accumulated atomically once per CTA
template <typename TA, typename TW>
__global__ void __launch_bounds__(256) k_prop_grad(PropGeo g, const TW* __restrict__ w, const uint8_t* __restrict__ Sin,
                                                   const uint8_t* __restrict__ Stg, int Ns, double* grad, double* loss) {
  extern __shared__ __align__(16) char smem[];
  PropSmem<TA> s = prop_carve<TA>(g, smem, true);
  const int C = g.C, nw = prop_nweights(C);
  prop_load_weights<TA, TW>(g, w, s.w);
  for (int i = threadIdx.x; i < nw; i += blockDim.x) s.gacc[i] = 0.0;
  __shared__ double lacc;
  if (threadIdx.x == 0) lacc = 0.0;
  __syncthreads();
  const TA inv = TA(1) / ((TA)Ns * (TA)g.N);
  double* gW1 = s.gacc;
  double* gb1 = gW1 + 9 * C;
  double* gW2 = gb1 + C;
  double* gb2 = gW2 + 9 * C * C;
  double* gW3 = gb2 + C;
  double* gb3 = gW3 + 9 * C;
  const TA* W2 = s.w + 9 * C + C;
  const TA* W3 = W2 + 9 * C * C + C;
  for (int c = blockIdx.x; c < Ns; c += gridDim.x) {
    prop_forward_one<TA>(g, s, Sin + (size_t)c * g.N);
    const uint8_t* t = Stg + (size_t)c * g.N;
    // loss and dL/dl
    TA lpart = 0;
    for (int p = threadIdx.x; p < g.N; p += blockDim.x) {
      const TA l = s.l[p], tv = (TA)t[p];
      lpart += softplus_(l) - tv * l;
      s.g2[p] = (sigm(l) - tv) * inv;
    }
    lpart = warp_sum(lpart);
    if ((threadIdx.x & 31) == 0) atomicAdd(&lacc, (double)lpart * (double)inv);
    __syncthreads();
    // layer 3: gh2 -> g1
    conv_bwd(g, s.h2, C, W3, 1, s.g2, gW3, gb3, s.g1);
    for (int o = threadIdx.x; o < C * g.N; o += blockDim.x) {
      const TA z = s.z2[o], sg = sigm(z);
      s.g1[o] *= sg * (TA(1) + z * (TA(1) - sg));
    }
    __syncthreads();
    // layer 2: gz2 (g1) -> gh1 (g2)
    conv_bwd(g, s.h1, C, W2, C, s.g1, gW2, gb2, s.g2);
    for (int o = threadIdx.x; o < C * g.N; o += blockDim.x) {
      const TA z = s.z1[o], sg = sigm(z);
      s.g2[o] *= sg * (TA(1) + z * (TA(1) - sg));
    }
    __syncthreads();
    conv_bwd(g, s.x, 1, s.w, C, s.g2, gW1, gb1, (TA*)nullptr);
  }
  for (int i = threadIdx.x; i < nw; i += blockDim.x) atomicAdd(grad + i, s.gacc[i]);
  if (threadIdx.x == 0) atomicAdd(loss, lacc);
}

// Adam on the FP64 master weights (Kingma & Ba), also refreshing the low-precision copy
__global__ void k_prop_adam(int nw, double* w, double* m, double* v, const double* g, int t, double lr,
                            __nv_bfloat16* wlow) {
  const double b1 = 0.9, b2 = 0.999, eps = 1e-8;
  const double c1 = 1.0 - pow(b1, (double)t), c2 = 1.0 - pow(b2, (double)t);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nw; i += gridDim.x * blockDim.x) {
    const double gi = g[i];
    const double mi = b1 * m[i] + (1.0 - b1) * gi;
    const double vi = b2 * v[i] + (1.0 - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const double wi = w[i] - lr * (mi / c1) / (sqrt(vi / c2) + eps);
    w[i] = wi;
    if (wlow) wlow[i] = __float2bfloat16((float)wi);
  }
}

// S' ~ prod_i Bernoulli(sigmoid(l_i)) with u_i = Philox(counter (i, step, chain, 1)), and
// lq = log q(S'|S) = sum_i s'_i l_i - softplus(l_i); one warp per chain
__global__ void k_prop_draw(int N, int Ns, const double* logits, uint64_t seed, uint64_t step, uint8_t* Sp, double* lq) {
  const int lane = threadIdx.x & 31;
  for (int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < Ns; c += (gridDim.x * blockDim.x) >> 5) {
    double acc = 0.0;
    for (int i = lane; i < N; i += 32) {
      const double l = logits[(size_t)c * N + i];
      const double p = 1.0 / (1.0 + exp(-l));
      const double u = uniform53((uint32_t)i, (uint32_t)step, (uint32_t)c, 1u, seed);
      const int s = (u < p) ? 1 : 0;
      Sp[(size_t)c * N + i] = (uint8_t)s;
      acc += s * l - (fmax(l, 0.0) + log1p(exp(-fabs(l))));
    }
    acc = warp_sum(acc);
    if (lane == 0) lq[c] = acc;
  }
}

// log q(S|S') from the logits of S': one warp per chain
__global__ void k_prop_logq(int N, int Ns, const double* logits, const uint8_t* S, double* lq) {
  const int lane = threadIdx.x & 31;
  for (int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < Ns; c += (gridDim.x * blockDim.x) >> 5) {
    double acc = 0.0;
    for (int i = lane; i < N; i += 32) {
      const double l = logits[(size_t)c * N + i];
      acc += (double)S[(size_t)c * N + i] * l - (fmax(l, 0.0) + log1p(exp(-fabs(l))));
    }
    acc = warp_sum(acc);
    if (lane == 0) lq[c] = acc;
  }
}

// accept iff u < exp(min(0, 2 (ln|psi'| - ln|psi|) + log q(S|S') - log q(S'|S))),
// u = Philox(counter (N, step, chain, 1)); one warp per chain
__global__ void k_prop_accept(int N, int Ns, uint64_t seed, uint64_t step, const uint8_t* Sp, const double* lpsi_new,
                              const double* lq_fwd, const double* lq_bwd, uint8_t* S, double* lpsi,
                              long long* accepted) {
  const int lane = threadIdx.x & 31;
  for (int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < Ns; c += (gridDim.x * blockDim.x) >> 5) {
    const double u = uniform53((uint32_t)N, (uint32_t)step, (uint32_t)c, 1u, seed);
    const double ln = lpsi_new[c];
    const double a = 2.0 * (ln - lpsi[c]) + lq_bwd[c] - lq_fwd[c];
    const bool acc = isfinite(ln) && (u < exp(fmin(0.0, a)));
    if (acc) {
      for (int i = lane; i < N; i += 32) S[(size_t)c * N + i] = Sp[(size_t)c * N + i];
      if (lane == 0) {
        lpsi[c] = ln;
        if (accepted) accepted[c] += 1;
      }
    }
  }
}

size_t prop_smem_bytes(int Lx, int Ly, int C, int act_bytes, bool train) {
  const int N = Lx * Ly;
  size_t b = (size_t)act_bytes * (prop_nweights(C) + 2 * N + 6 * (size_t)C * N);
  b = (b + 15) / 16 * 16;
  if (train) b += sizeof(double) * prop_nweights(C);
  return b;
}

cudaError_t launch_prop_logits(int Lx, int Ly, int C, int wprec, const void* w, const uint8_t* S, int Ns, double* logits,
                               int grid, cudaStream_t s) {
  PropGeo g{Lx, Ly, C, Lx * Ly};
  if (wprec == 0) {
    const size_t sm = prop_smem_bytes(Lx, Ly, C, 8, false);
    cudaFuncSetAttribute(k_prop_logits<double, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_prop_logits<double, double><<<grid, 256, sm, s>>>(g, (const double*)w, S, Ns, logits);
  } else {
    const size_t sm = prop_smem_bytes(Lx, Ly, C, 4, false);
    cudaFuncSetAttribute(k_prop_logits<float, __nv_bfloat16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_prop_logits<float, __nv_bfloat16><<<grid, 256, sm, s>>>(g, (const __nv_bfloat16*)w, S, Ns, logits);
  }
  return cudaGetLastError();
}

cudaError_t launch_prop_grad(int Lx, int Ly, int C, int wprec, const void* w, const uint8_t* Sin, const uint8_t* Stg,
                             int Ns, double* grad, double* loss, int grid, cudaStream_t s) {
  PropGeo g{Lx, Ly, C, Lx * Ly};
  if (wprec == 0) {
    const size_t sm = prop_smem_bytes(Lx, Ly, C, 8, true);
    cudaFuncSetAttribute(k_prop_grad<double, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_prop_grad<double, double><<<grid, 256, sm, s>>>(g, (const double*)w, Sin, Stg, Ns, grad, loss);
  } else {
    const size_t sm = prop_smem_bytes(Lx, Ly, C, 4, true);
    cudaFuncSetAttribute(k_prop_grad<float, __nv_bfloat16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_prop_grad<float, __nv_bfloat16><<<grid, 256, sm, s>>>(g, (const __nv_bfloat16*)w, Sin, Stg, Ns, grad, loss);
  }
  return cudaGetLastError();
}

cudaError_t launch_prop_adam(int nw, double* w, double* m, double* v, const double* g, int t, double lr, void* wlow,
                             cudaStream_t s) {
  k_prop_adam<<<(nw + 255) / 256, 256, 0, s>>>(nw, w, m, v, g, t, lr, (__nv_bfloat16*)wlow);
  return cudaGetLastError();
}

cudaError_t launch_prop_draw(int N, int Ns, const double* logits, uint64_t seed, uint64_t step, uint8_t* Sp, double* lq,
                             cudaStream_t s) {
  k_prop_draw<<<(Ns * 32 + 255) / 256, 256, 0, s>>>(N, Ns, logits, seed, step, Sp, lq);
  return cudaGetLastError();
}

cudaError_t launch_prop_logq(int N, int Ns, const double* logits, const uint8_t* S, double* lq, cudaStream_t s) {
  k_prop_logq<<<(Ns * 32 + 255) / 256, 256, 0, s>>>(N, Ns, logits, S, lq);
  return cudaGetLastError();
}

cudaError_t launch_prop_accept(int N, int Ns, uint64_t seed, uint64_t step, const uint8_t* Sp, const double* lpsi_new,
                               const double* lq_fwd, const double* lq_bwd, uint8_t* S, double* lpsi, long long* accepted,
                               cudaStream_t s) {
  k_prop_accept<<<(Ns * 32 + 255) / 256, 256, 0, s>>>(N, Ns, seed, step, Sp, lpsi_new, lq_fwd, lq_bwd, S, lpsi, accepted);
  return cudaGetLastError();
}

}  // namespace peps

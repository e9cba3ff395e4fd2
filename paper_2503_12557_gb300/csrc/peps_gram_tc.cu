// MinSR Gram matrix T = Obar Obar^T on the 5th-generation tensor cores (tcgen05, sm_103a) in
// split BF16: every entry of Obar is written as hi + lo with hi = bf16(x), lo = bf16(x - hi),
// and T ~ hi hi^T + hi lo^T + lo hi^T (the lo lo^T term, of relative size 2^-16, is dropped),
// accumulated in FP32 in tensor memory.  Only tiles on or below the diagonal are computed; a
// separate kernel mirrors them when the full matrix is needed.
//
// One CTA computes a 128 x 128 tile with one tcgen05.mma.cta_group::1.kind::f16 stream
// (M = 128, N = 128, K = 16 per instruction): warp 0 issues the TMA loads (128B-swizzled K-major
// tiles of 128 rows x 64 columns for hi/lo of the row block and of the column block), warp 1
// issues the MMAs, all four warps drain the FP32 accumulator from tensor memory.  A STAGES-deep
// ring of shared-memory buffers is handed between the two roles with mbarriers.  Every wait is
// bounded: on a timeout the kernel records an error, lets its own copies drain (bounded), frees
// its tensor memory and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "peps_kernels.cuh"

namespace peps {
namespace {

constexpr int TM = 128, TN = 128, TK = 64;   // tile sizes (TK bf16 = 128 bytes = one swizzle row)
constexpr int STAGES = 3;
constexpr int TILE_BYTES = TM * TK * 2;      // 16 KB per operand tile
constexpr int STAGE_BYTES = 4 * TILE_BYTES;  // hi_i, lo_i, hi_j, lo_j
constexpr unsigned long long WAIT_LIMIT = 1ull << 26;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait; returns false on timeout
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  for (unsigned long long i = 0; i < WAIT_LIMIT; ++i)
    if (mbar_try(bar, parity)) return true;
  return false;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst)),
      "l"((uint64_t)map), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, 8-row groups 1024 bytes
// apart.  Bits: [0,14) start >> 4, [16,30) leading byte offset >> 4 (unused for this layout,
// set to 1), [32,46) stride byte offset >> 4, [46,48) descriptor version 1, [61,64) layout
// 2 = 128-byte swizzle.
__device__ __forceinline__ uint64_t smem_desc(const void* p) {
  const uint64_t a = (uint64_t)(smem_u32(p) >> 4) & 0x3FFFull;
  return a | (1ull << 16) | ((uint64_t)(1024 >> 4) << 32) | (1ull << 46) | (2ull << 61);
}

// Instruction descriptor of kind::f16: FP32 accumulator (bits [4,6) = 1), BF16 A and B
// ([7,10) = 1, [10,13) = 1), both K-major, N >> 3 at [17,23), M >> 4 at [24,29).
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TN >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(a), "l"(b), "r"(IDESC), "r"(acc));
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__global__ void __launch_bounds__(128, 1) k_gram_tc(const __grid_constant__ CUtensorMap map_hi,
                                                    const __grid_constant__ CUtensorMap map_lo, int ntile, int nk,
                                                    int Ns, double* Tm, int ld, int* err) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  // 1024-byte aligned ring of stages
  uint8_t* ring = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t full_bar[STAGES], empty_bar[STAGES], done_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ int failed;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // tile (ti, tj) with ti >= tj from the linear block index
  int t = blockIdx.x, ti = 0;
  while (t >= ti + 1) { t -= ti + 1; ++ti; }
  const int tj = t;
  if (ti >= ntile) return;
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    mbar_init(&done_bar, 1);
    failed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 2) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)), "r"(TN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_slot;
  const int r0 = ti * TM, c0 = tj * TN;
  if (warp == 0 && lane == 0) {
    // TMA producer
    for (int kt = 0; kt < nk; ++kt) {
      const int s = kt % STAGES;
      if (kt >= STAGES && !mbar_wait(&empty_bar[s], ((kt / STAGES) - 1) & 1)) { atomicExch(&failed, 1); break; }
      if (failed) break;
      uint8_t* st = ring + (size_t)s * STAGE_BYTES;
      mbar_expect_tx(&full_bar[s], STAGE_BYTES);
      tma_load_2d(st + 0 * TILE_BYTES, &map_hi, kt * TK, r0, &full_bar[s]);
      tma_load_2d(st + 1 * TILE_BYTES, &map_lo, kt * TK, r0, &full_bar[s]);
      tma_load_2d(st + 2 * TILE_BYTES, &map_hi, kt * TK, c0, &full_bar[s]);
      tma_load_2d(st + 3 * TILE_BYTES, &map_lo, kt * TK, c0, &full_bar[s]);
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer
    for (int kt = 0; kt < nk; ++kt) {
      const int s = kt % STAGES;
      if (!mbar_wait(&full_bar[s], (kt / STAGES) & 1)) { atomicExch(&failed, 1); break; }
      if (failed) break;
      asm volatile("tcgen05.fence::after_thread_sync;");
      uint8_t* st = ring + (size_t)s * STAGE_BYTES;
      const uint64_t ahi = smem_desc(st), alo = smem_desc(st + TILE_BYTES);
      const uint64_t bhi = smem_desc(st + 2 * TILE_BYTES), blo = smem_desc(st + 3 * TILE_BYTES);
#pragma unroll
      for (int kk = 0; kk < TK / 16; ++kk) {
        const uint64_t off = (uint64_t)((kk * 32) >> 4);  // 16 bf16 = 32 bytes along K
        mma_bf16(tmem, ahi + off, bhi + off, (kt > 0 || kk > 0) ? 1u : 0u);
        mma_bf16(tmem, ahi + off, blo + off, 1u);
        mma_bf16(tmem, alo + off, bhi + off, 1u);
      }
      mma_commit(&empty_bar[s]);
    }
    mma_commit(&done_bar);
  }
  __syncwarp();
  // epilogue: every warp drains its 32 accumulator lanes
  const bool ok = mbar_wait(&done_bar, 0);
  if (!ok) atomicExch(&failed, 1);
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (ok && !failed) {
    // every MMA has completed (done_bar), so the operand ring is free: each warp stages its
    // 32 x 32 block there (row = lane on the way in, padded to 33 against bank conflicts) and
    // writes it out row by row, a warp's 32 lanes storing 32 consecutive columns
    float* stage = reinterpret_cast<float*>(ring) + (size_t)warp * 32 * 33;
#pragma unroll 1
    for (int cc = 0; cc < TN; cc += 32) {
      uint32_t v[32];
      const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)cc;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,"
          "%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
            "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]),
            "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
            "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int j = 0; j < 32; ++j) stage[lane * 33 + j] = __uint_as_float(v[j]);
      __syncwarp();
      const int col = c0 + cc + lane;
      for (int r = 0; r < 32; ++r) {
        const int row = r0 + warp * 32 + r;
        if (row < Ns && col < Ns && col <= row) Tm[(size_t)row * ld + col] = (double)stage[r * 33 + lane];
      }
      __syncwarp();
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (failed && threadIdx.x == 0) atomicExch(err, 1);
  if (warp == 2) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TN));
  }
}

// hi/lo bf16 split of Obar (Ns x Np, double) into zero-padded (Npad x Kpad) row-major arrays
__global__ void k_split_bf16(const double* __restrict__ Ob, int Ns, long long Np, int Npad, long long Kpad,
                             __nv_bfloat16* hi, __nv_bfloat16* lo) {
  const long long total = (long long)Npad * Kpad;
  for (long long o = blockIdx.x * (long long)blockDim.x + threadIdx.x; o < total; o += (long long)gridDim.x * blockDim.x) {
    const long long r = o / Kpad, k = o % Kpad;
    const double x = (r < Ns && k < Np) ? Ob[r * Np + k] : 0.0;
    const __nv_bfloat16 h = __float2bfloat16((float)x);
    hi[o] = h;
    lo[o] = __float2bfloat16((float)(x - (double)__bfloat162float(h)));
  }
}

// fill the upper triangle from the lower one (32 x 32 tiles through shared memory)
__global__ void k_mirror_lower(double* T, int n) {
  __shared__ double tile[32][33];
  const int bi = blockIdx.y, bj = blockIdx.x;
  if (bj > bi) return;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  for (int k = ty; k < 32; k += 8) {
    const int r = bi * 32 + k, c = bj * 32 + tx;
    tile[k][tx] = (r < n && c < n) ? T[(size_t)r * n + c] : 0.0;
  }
  __syncthreads();
  for (int k = ty; k < 32; k += 8) {
    const int r = bj * 32 + k, c = bi * 32 + tx;  // transposed position (upper triangle)
    if (r < n && c < n && c > r) T[(size_t)r * n + c] = tile[tx][k];
  }
}

typedef CUresult (*EncodeTiled)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled get_encode() {
  static EncodeTiled fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiled)p;
  }
  return fn;
}

}  // namespace

int gram_tc_pad_rows(int Ns) { return (Ns + TM - 1) / TM * TM; }
long long gram_tc_pad_k(long long Np) { return (Np + TK - 1) / TK * TK; }

// T (lower triangle, or full when mirror) = split-BF16 tensor-core Gram of Obar.  hi, lo:
// workspaces of gram_tc_pad_rows(Ns) x gram_tc_pad_k(Np) bf16 each.  err: device int, set to 1
// when a pipeline wait timed out.  Returns a CUDA error, or cudaErrorNotSupported when the
// tensor-map encoder is unavailable.
cudaError_t launch_gram_tc(const double* Obar, int Ns, long long Np, void* hi, void* lo, double* Tm, int ld, bool mirror,
                           int* err, cudaStream_t s) {
  const int Npad = gram_tc_pad_rows(Ns);
  const long long Kpad = gram_tc_pad_k(Np);
  k_split_bf16<<<4096, 256, 0, s>>>(Obar, Ns, Np, Npad, Kpad, (__nv_bfloat16*)hi, (__nv_bfloat16*)lo);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  EncodeTiled enc = get_encode();
  if (!enc) return cudaErrorNotSupported;
  CUtensorMap mh, ml;
  const cuuint64_t dims[2] = {(cuuint64_t)Kpad, (cuuint64_t)Npad};
  const cuuint64_t strides[1] = {(cuuint64_t)Kpad * 2};
  const cuuint32_t box[2] = {TK, TM};
  const cuuint32_t estr[2] = {1, 1};
  if (enc(&mh, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, hi, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
          CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS ||
      enc(&ml, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, lo, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
          CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return cudaErrorInvalidValue;
  const int ntile = Npad / TM;
  const int nk = (int)(Kpad / TK);
  const size_t smem = (size_t)STAGES * STAGE_BYTES + 1024;
  e = cudaFuncSetAttribute(k_gram_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_gram_tc<<<ntile * (ntile + 1) / 2, 128, smem, s>>>(mh, ml, ntile, nk, Ns, Tm, ld, err);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (mirror) {
    dim3 grid((ld + 31) / 32, (ld + 31) / 32), block(32, 8);
    k_mirror_lower<<<grid, block, 0, s>>>(Tm, ld);
    e = cudaGetLastError();
  }
  return e;
}

}  // namespace peps

// peps_amplitudes_noalloc: ln psi_top(S) for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at all: code that runs inside another framework's
// allocator (which owns every byte of device memory and forbids side allocations), code that
// must not touch the allocator because it runs while a memory pool is being resized or torn
// down, or code in a process whose device memory budget is fixed up front.  For them this
// entry point keeps every intermediate (padded parameter copy, boundary-MPS environments,
// per-CTA work buffers, per-sample bookkeeping) in one file-scope device array of
// kNoAllocBytes (32 MiB) that the library reserves on every GPU it is loaded on, for the life
// of the process.  The caller passes only its inputs and outputs.
//
// Every call made outside a stream capture looks up that device's address of the array (with
// the device current) and keeps it; a call made while the stream is being captured uses the
// address of the last such lookup, so make a first call before any stream capture.  When the
// problem does not fit with two CTAs per SM, fewer CTAs share the work (same results, less
// concurrency).  Every call shares the one array and leaves its last contents there: calls
// that may overlap on the GPU (two streams, two host threads) race on it and must be
// serialised by the caller.
#include <mutex>
#include <utility>

#include "peps_kernels.cuh"
#include "peps_gb300.h"

namespace {

constexpr size_t kNoAllocBytes = 32ull << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
void* g_scratch_addr[kMaxDevices];
cudaError_t g_scratch_err[kMaxDevices];
std::mutex g_scratch_mu;

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

// start offset of every site tensor in theta (boundary legs of dimension 1), written on the
// device so that no host buffer has to be copied in
__global__ void k_noalloc_site_offsets(int Lx, int Ly, int d, int D, long long* off) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  long long acc = 0;
  for (int x = 0; x < Lx; ++x)
    for (int y = 0; y < Ly; ++y) {
      off[x * Ly + y] = acc;
      acc += (long long)d * (y == 0 ? 1 : D) * (x == 0 ? 1 : D) * (y == Ly - 1 ? 1 : D) * (x == Lx - 1 ? 1 : D);
    }
  off[Lx * Ly] = acc;
}

// every buffer of the environment and one-row kernels lives in the scratch arena (no dynamic
// shared memory is requested)
void global_plan(peps::Plan& p, const std::pair<int, size_t>* bufs, int nb) {
  p.gmask = 0;
  size_t off = 0;
  for (int b = 0; b < peps::B_NBUF; ++b) p.off[b] = 0;
  for (int i = 0; i < nb; ++i) {
    p.gmask |= 1u << bufs[i].first;
    p.off[bufs[i].first] = off;
    off += align256(bufs[i].second);
  }
  p.gstride = off;
}

template <typename T>
peps_status run(const peps_config& c, const double* theta, const uint8_t* S, int Ns, double* logabs, double* phase,
                int32_t* status, cudaStream_t s, char* base) {
  using namespace peps;
  Geo g;
  g.Lx = c.Lx; g.Ly = c.Ly; g.d = c.d; g.D = c.D; g.chi = c.chi;
  g.n = c.chi * c.D;
  g.se = c.chi * c.D * c.chi;
  g.sT = c.D * c.D * c.D * c.D;
  g.s2 = c.chi * c.D * c.D * c.chi;
  g.cut = c.trunc_weight;
  const int N = c.Lx * c.Ly, n = g.n, chi = g.chi, D = g.D, Ly = g.Ly;
  const int mX = n + (n & 1), Lr = D * chi, ci = n < 8 ? n : 8;
  const size_t E = sizeof(T);
  const size_t zsz = env_z_elems(chi, D);
  const size_t t1 = sandwich1_t_elems(chi, D);
  const std::pair<int, size_t> benv[] = {
      {B_RED, 40 * 8}, {B_SIG, (mX + 4) * E}, {B_SEL, 2 * (size_t)mX * 4}, {B_A, (size_t)g.sT * E},
      {B_E, (size_t)g.se * E}, {B_C, (size_t)n * chi * E}, {B_W, env_w_elems(chi, D, ci) * E},
      {B_R, (size_t)n * n * E}, {B_Z, zsz * E}, {B_RHIST, (size_t)(Ly > 1 ? Ly - 1 : 1) * n * n * E}};
  const std::pair<int, size_t> brow[] = {
      {B_RED, 40 * 8}, {B_A, (size_t)g.sT * E}, {B_EU, (size_t)g.se * E}, {B_EL, (size_t)g.se * E},
      {B_T1, t1 * E}, {B_T2, t1 * E}, {B_LW, (size_t)g.se * E}, {B_LW2, (size_t)g.se * E},
      {B_LP, (size_t)(Ly + 1) * g.se * E}, {B_RP, (size_t)(Ly + 1) * g.se * E}};
  Plan pe{}, pr{};
  global_plan(pe, benv, (int)(sizeof(benv) / sizeof(benv[0])));
  global_plan(pr, brow, (int)(sizeof(brow) / sizeof(brow[0])));
  pe.ci = pr.ci = ci;
  pe.cx = pr.cx = chi;
  pe.ctr = pr.ctr = nullptr;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return PEPS_E_CUDA;
  // carve the scratch array: the fixed buffers first, then one work-buffer slice per CTA
  size_t off = 0;
  auto take = [&](size_t bytes) { char* p = base + off; off += align256(bytes); return p; };
  long long* site_off = (long long*)take(sizeof(long long) * (N + 1));
  T* Tpad = (T*)take((size_t)N * g.d * g.sT * E);
  T* envs = (T*)take((size_t)Ns * 2 * g.Lx * Ly * g.se * E);
  double* logs = (double*)take(sizeof(double) * (size_t)Ns * 2 * g.Lx);
  double* rowout = (double*)take(sizeof(double) * 4 * (size_t)Ns * g.Lx);
  float* wdisc = (float*)take(sizeof(float) * (size_t)Ns);
  int* st_own = (int*)take(sizeof(int) * (size_t)Ns);
  if (off > kNoAllocBytes) return PEPS_E_CAPACITY;
  // the kernels loop over samples with a grid stride, so fewer CTAs give the same results;
  // take two per SM where the slices fit, else as many as fit, and give up below one
  const size_t stride = pe.gstride > pr.gstride ? pe.gstride : pr.gstride;
  const size_t fit = (kNoAllocBytes - off) / (stride > 0 ? stride : 1);
  int grid = (2 * nsm < Ns) ? 2 * nsm : Ns;
  if ((size_t)grid > fit) grid = (int)fit;
  if (grid < 1) return PEPS_E_CAPACITY;
  char* arena_base = take((size_t)grid * stride);
  if (off > kNoAllocBytes) return PEPS_E_CAPACITY;
  pe.gbase = pr.gbase = arena_base;
  int* st = status ? (int*)status : st_own;
  // what the kernels accumulate into must start at zero
  if (cudaMemsetAsync(st, 0, sizeof(int) * (size_t)Ns, s) != cudaSuccess) return PEPS_E_CUDA;
  if (cudaMemsetAsync(wdisc, 0, sizeof(float) * (size_t)Ns, s) != cudaSuccess) return PEPS_E_CUDA;
  k_noalloc_site_offsets<<<1, 32, 0, s>>>(g.Lx, g.Ly, g.d, g.D, site_off);
  if (launch_pad<T>(g, theta, site_off, Tpad, s) != cudaSuccess) return PEPS_E_CUDA;
  if (launch_env<T>(g, pe, grid, 0, Tpad, S, Ns, 1, envs, logs, st, wdisc, s) != cudaSuccess) return PEPS_E_CUDA;
  TermTab none{};
  if (launch_row<T>(g, pr, grid, 0, Tpad, S, Ns, g.Lx - 1, g.Lx, envs, logs, (T*)nullptr, site_off, 0, none, rowout,
                    st, s) != cudaSuccess)
    return PEPS_E_CUDA;
  DiagTab dg{};
  if (launch_combine(g, Ns, S, rowout, rowout, 0, 0, dg, logabs, phase, nullptr, s) != cudaSuccess) return PEPS_E_CUDA;
  return PEPS_OK;
}

}  // namespace

extern "C" peps_status peps_amplitudes_noalloc(const peps_config* cfg, const double* theta_dev, const uint8_t* S_dev,
                                               int Ns, double* logabs_dev, double* phase_dev, int32_t* status_dev,
                                               void* stream) {
  if (!cfg || !theta_dev || Ns < 0 || (Ns > 0 && (!S_dev || !logabs_dev || !phase_dev))) return PEPS_E_ARG;
  const peps_config c = *cfg;
  if (c.Lx < 2 || c.Ly < 2 || c.Ly > peps::MAX_LY || c.d < 2 || c.d > 4 || c.D < 1 || c.D > 8 || c.chi < c.D ||
      c.chi > 64)
    return PEPS_E_SHAPE;
  if (c.prec != PEPS_PREC_FP64 && c.prec != PEPS_PREC_FP32) return PEPS_E_ARG;
  if (c.cplx) return PEPS_E_UNSUPPORTED;  // real PEPS only
  if (!(c.trunc_weight >= 0.0 && c.trunc_weight < 1.0)) return PEPS_E_ARG;
  if (Ns == 0) return PEPS_OK;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return PEPS_E_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  // the array's device address: looked up with this device current on every call made outside
  // a stream capture (a cudaDeviceReset reloads the module and moves the array), and taken from
  // the last lookup while the stream is being captured (no runtime query may run then)
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) return PEPS_E_CUDA;
  void* addr = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (cap == cudaStreamCaptureStatusNone) {
      g_scratch_err[dev] = cudaGetSymbolAddress(&g_scratch_addr[dev], g_noalloc_scratch);
    }
    if (g_scratch_err[dev] != cudaSuccess) g_scratch_addr[dev] = nullptr;
    addr = g_scratch_addr[dev];
  }
  if (!addr) return PEPS_E_CUDA;
  char* base = (char*)addr;
  return (c.prec == PEPS_PREC_FP64) ? run<double>(c, theta_dev, S_dev, Ns, logabs_dev, phase_dev, status_dev, s, base)
                                    : run<float>(c, theta_dev, S_dev, Ns, logabs_dev, phase_dev, status_dev, s, base);
}

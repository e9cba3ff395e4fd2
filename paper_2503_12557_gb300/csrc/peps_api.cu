// C ABI of the finite-PEPS hot path (declared in include/peps_gb300.h): handle, buffer planner,
// Hamiltonian packing and the entry points.  Host code only; every step of the path runs in
// the kernels of peps_kernels.cu and peps_minsr.cu.
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>
#include <algorithm>

#include "peps_kernels.cuh"
#include "peps_gb300.h"
#include <map>
#include <mutex>

using namespace peps;

struct KPlan {
  Plan p;
  size_t smem = 0;
  int grid = 0;
};

struct peps_handle {
  peps_config cfg{};
  int elem = 0;  // scalar of the kernels: 0 double, 1 float, 2 cplx<double>, 3 cplx<float>
  size_t budget[4] = {0, 0, 0, 0};  // shared-memory budget per kernel class (env, row, pair, sample)
  Geo g{};
  long long Np = 0;
  int nsm = 0;
  size_t esz = 8;  // bytes per real
  void* Tpad = nullptr;
  long long* site_off = nullptr;  // device, N+1
  std::vector<long long> site_off_h;
  void* envs = nullptr;
  double* logs = nullptr;
  float* wdisc = nullptr;
  double* rowout = nullptr;
  double* pairout = nullptr;
  int* status_tmp = nullptr;
  char* gscratch = nullptr;
  size_t gscratch_bytes = 0;
  KPlan kp[4];  // env, row, pair, sample
  KPlan kb;     // variational-bound estimator (row-step buffers of the env budget)
  double* bout = nullptr;  // k_bound's per-(sample, term) sums
  size_t bout_cap = 0;
  // direct sampling: double-layer environments, their work buffers, the sampler's plan and arena
  int dl_chid = 0;
  void* DL = nullptr;
  size_t DL_bytes = 0;
  void* dl_work = nullptr;
  size_t dl_work_bytes = 0;
  int* dl_status = nullptr;
  KPlan kd;
  char* dscratch = nullptr;
  size_t dscratch_bytes = 0;
  // reuse of the sampler's upper environments by the next evaluation (opt-in): the last
  // sampled batch (pointer, size, parameter generation) and the upper row steps' status bits
  int env_reuse = 0;
  const uint8_t* rs_S = nullptr;
  int rs_Ns = 0;
  long long param_gen = 0, rs_gen = -1;
  int rs_up = 0;  // the last sweep ran up the rows: the stored lower environments are current
  int* ustat = nullptr;
  // Hamiltonian cache
  std::vector<char> ham_key;
  std::vector<int> h_tinfo, h_ab, h_rowoff, h_pairoff, h_pij;
  std::vector<double> h_eh, h_pv, h_onsite;
  int* d_tinfo = nullptr;
  int* d_ab = nullptr;
  double* d_eh = nullptr;
  int* d_rowoff = nullptr;
  int* d_pairoff = nullptr;
  int* d_pij = nullptr;
  double* d_pv = nullptr;
  double* d_onsite = nullptr;
  int n_pair_terms = 0;
  TermTab tt{};
  DiagTab dg{};
  // MinSR workspace
  int ms_cap = 0;
  long long ms_np = 0;
  double *Obar = nullptr, *Tm = nullptr, *Vm = nullptr, *Hm = nullptr, *mean = nullptr, *ebar = nullptr,
         *yv = nullptr, *xv = nullptr, *cnt = nullptr;
  double* td = nullptr;  // tridiagonal eigen route: vectors and partial sums (td_workspace_doubles)
  // timing: event pairs per kernel class, recorded on the call's stream when enabled
  bool timing = false;
  std::vector<cudaEvent_t> evpool;
  std::vector<int> evclass;
  std::vector<long long> evlaunches;
  size_t evn = 0;
  unsigned long long* ctr = nullptr;  // device work counters (8)
  // learned-proposal workspace (allocated on first use)
  uint8_t* lp_Sp = nullptr;
  double *lp_l0 = nullptr, *lp_l1 = nullptr, *lp_aux = nullptr;
  // split-BF16 operands of the tensor-core Gram
  void *g_hi = nullptr, *g_lo = nullptr;
  // status word (device): OR of the per-sample status bits and the MinSR flags since the last
  // peps_last_status
  int* sword = nullptr;
  // device memory: the caller's allocator when one was given to peps_create_ex, else cudaMalloc
  peps_allocator alloc{};
  bool has_alloc = false;
  std::string err;
};

static cudaError_t h_malloc(peps_handle* h, void** p, size_t bytes) {
  *p = nullptr;
  if (!h->has_alloc) return cudaMalloc(p, bytes);
  void* q = h->alloc.alloc(h->alloc.ctx, bytes ? bytes : 1);
  if (!q) return cudaErrorMemoryAllocation;
  *p = q;
  return cudaSuccess;
}

static void h_free(peps_handle* h, void* p) {
  if (!p) return;
  if (h->has_alloc) h->alloc.free(h->alloc.ctx, p);
  else cudaFree(p);
}

// Run f(T{}) with T the handle's kernel scalar.
template <typename F>
static auto dispatch_elem(const peps_handle* h, F&& f) {
  switch (h->elem) {
    case 0: return f(double{});
    case 1: return f(float{});
    case 2: return f(cplx<double>{});
    default: return f(cplx<float>{});
  }
}

enum { TC_ENV = 0, TC_ROW, TC_PAIR, TC_COMBINE, TC_SAMPLE, TC_GRAM, TC_EIG, TC_MINSR, TC_PAD, TC_BOUND, TC_DIRECT, TC_N };

// Record a start event for kernel class c (returns the slot, or -1 when timing is off).
static int tstart(peps_handle* h, int c, cudaStream_t s) {
  if (!h->timing) return -1;
  if (h->evn + 2 > h->evpool.size()) {
    for (int i = 0; i < 64; ++i) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      h->evpool.push_back(e);
    }
    h->evclass.resize(h->evpool.size() / 2);
    h->evlaunches.resize(h->evpool.size() / 2);
  }
  const int slot = (int)(h->evn / 2);
  cudaEventRecord(h->evpool[h->evn], s);
  h->evclass[slot] = c;
  h->evlaunches[slot] = 1;
  h->evn += 2;
  return slot;
}
static void tstop(peps_handle* h, int slot, cudaStream_t s, long long launches = 1) {
  if (slot < 0) return;
  cudaEventRecord(h->evpool[2 * slot + 1], s);
  h->evlaunches[slot] = launches;
}

static peps_status fail(peps_handle* h, peps_status st, const std::string& msg) {
  if (h) h->err = msg;
  return st;
}
static peps_status cuda_fail(peps_handle* h, cudaError_t e, const char* where) {
  if (h) h->err = std::string(where) + ": " + cudaGetErrorString(e);
  return PEPS_E_CUDA;
}
#define CK(call, where)                                      \
  do {                                                       \
    cudaError_t _e = (call);                                 \
    if (_e != cudaSuccess) return cuda_fail(h, _e, where);   \
  } while (0)

static size_t al(size_t x, size_t a = 256) { return (x + a - 1) / a * a; }

// Place buffers (byte sizes, in priority order) into shared memory up to `budget`, the rest
// into the per-CTA global arena.
static void place(Plan& p, size_t& smem, size_t budget, const std::vector<std::pair<int, size_t>>& bufs) {
  p.gmask = 0;
  for (int b = 0; b < B_NBUF; ++b) p.off[b] = 0;
  size_t s = 0, gl = 0;
  for (auto& b : bufs) {
    const size_t sz = al(b.second, 16);
    if (s + sz <= budget) {
      p.off[b.first] = s;
      s += sz;
    } else {
      p.gmask |= 1u << b.first;
      p.off[b.first] = gl;
      gl += al(sz, 256);
    }
  }
  smem = s;
  p.gstride = gl;
}

// As place(), for the sampler: the `common` buffers first, then two groups that are never live
// at the same time (the boundary-MPS row step and the sandwich partials) overlaid on the same
// shared-memory region.
static void place_overlay(Plan& p, size_t& smem, size_t budget, const std::vector<std::pair<int, size_t>>& common,
                          const std::vector<std::pair<int, size_t>>& ga, const std::vector<std::pair<int, size_t>>& gb) {
  p.gmask = 0;
  for (int b = 0; b < B_NBUF; ++b) p.off[b] = 0;
  size_t s = 0, gl = 0;
  auto put1 = [&](const std::pair<int, size_t>& b, size_t& cur) {
    const size_t sz = al(b.second, 16);
    if (cur + sz <= budget) {
      p.off[b.first] = cur;
      cur += sz;
    } else {
      p.gmask |= 1u << b.first;
      p.off[b.first] = gl;
      gl += al(sz, 256);
    }
  };
  for (auto& b : common) put1(b, s);
  size_t sa = s, sb = s;
  for (auto& b : ga) put1(b, sa);
  for (auto& b : gb) put1(b, sb);
  smem = std::max(sa, sb);
  p.gstride = gl;
}

// Default shared-memory budget per CTA: FP64 one CTA per SM (the FP64 pipe is the limit), FP32
// two CTAs per SM.
// Default shared-memory budget per CTA and kernel class (0 env, 1 row, 2 pair, 3 sampler): FP64
// one CTA per SM (the FP64 pipe is the limit); FP32 three CTAs per SM (72 KB each, the larger
// buffers in the L2-resident arena) for the environment, one-row and sampler kernels (the
// sampler's moves and row steps run as separate launches in FP32), two for the two-row kernel.
static size_t default_budget(const peps_handle* h, int cls) {
  if (h->esz >= 8) return 210 * 1024;
  return (cls == 2) ? 110 * 1024 : 72 * 1024;
}
// budget of the bound and direct-sampling plans (compiled for two CTAs per SM in FP32)
static size_t wide_budget(const peps_handle* h) { return (h->esz >= 8) ? 210 * 1024 : 110 * 1024; }

static void plan_all(peps_handle* h) {
  const Geo& g = h->g;
  const size_t E = h->esz;
  const int n = g.n, chi = g.chi, D = g.D, Ly = g.Ly;
  const int mX = n + (n & 1);
  const int Lr = D * chi;
  for (int i = 0; i < 4; ++i)
    if (h->budget[i] == 0) h->budget[i] = default_budget(h, i);
  size_t budget = h->budget[0];
  int ci = std::min(n, 8);
  const size_t zsz = env_z_elems(chi, D);
  // one-row / two-row temporaries
  const size_t t1row = sandwich1_t_elems(chi, D);
  int cx = chi;
  while (cx > 1 && (size_t)D * D * D * chi * cx > 8192) cx = (cx + 1) / 2;
  const size_t t2row = (size_t)D * D * D * chi * cx + chi;  // absorb2_right's first temporary: + chi
  // env plan
  {
    KPlan& k = h->kp[0];
    k.p.ci = ci;
    k.p.cx = cx;
    std::vector<std::pair<int, size_t>> b = {
        {B_RED, 40 * 8}, {B_SIG, (mX + 4) * E}, {B_SEL, 2 * mX * 4}, {B_A, (size_t)g.sT * E}, {B_E, (size_t)g.se * E},
        {B_C, (size_t)n * chi * E}, {B_W, env_w_elems(chi, D, ci) * E}, {B_R, (size_t)n * n * E}, {B_Z, zsz * E},
        {B_RHIST, (size_t)std::max(1, Ly - 1) * n * n * E}};
    place(k.p, k.smem, budget, b);
  }
  // bound plan: the env plan's row-step buffers, then S', the overlap partials and the
  // rebuilt environment rows (two per side, used alternately)
  {
    KPlan& k = h->kb;
    k.p.ci = ci;
    k.p.cx = cx;
    std::vector<std::pair<int, size_t>> b = {
        {B_RED, 40 * 8}, {B_SIG, (mX + 4) * E}, {B_SEL, 2 * mX * 4}, {B_A, (size_t)g.sT * E}, {B_E, (size_t)g.se * E},
        {B_C, (size_t)n * chi * E}, {B_W, env_w_elems(chi, D, ci) * E}, {B_R, (size_t)n * n * E}, {B_Z, zsz * E},
        {B_RHIST, (size_t)std::max(1, Ly - 1) * n * n * E}, {B_S, (size_t)g.Lx * g.Ly},
        {B_LW, (size_t)2 * chi * chi * E}, {B_LW2, (size_t)g.se * E}, {B_LP, (size_t)2 * Ly * g.se * E},
        {B_RP, (size_t)2 * Ly * g.se * E}};
    place(k.p, k.smem, wide_budget(h), b);
  }
  // row plan
  budget = h->budget[1];
  {
    KPlan& k = h->kp[1];
    k.p.ci = ci;
    k.p.cx = cx;
    std::vector<std::pair<int, size_t>> b = {
        {B_RED, 40 * 8}, {B_A, (size_t)g.sT * E}, {B_EU, (size_t)g.se * E}, {B_EL, (size_t)g.se * E},
        {B_T1, t1row * E}, {B_T2, t1row * E}, {B_LW, (size_t)g.se * E}, {B_LW2, (size_t)g.se * E},
        {B_LP, (size_t)(Ly + 1) * g.se * E}, {B_RP, (size_t)(Ly + 1) * g.se * E}};
    place(k.p, k.smem, budget, b);
  }
  // pair plan
  budget = h->budget[2];
  {
    KPlan& k = h->kp[2];
    k.p.ci = ci;
    k.p.cx = cx;
    std::vector<std::pair<int, size_t>> b = {
        {B_RED, 40 * 8}, {B_A, (size_t)g.sT * E}, {B_A2, (size_t)g.sT * E}, {B_EU, (size_t)g.se * E},
        {B_EL, (size_t)g.se * E}, {B_T1, t2row * E}, {B_T2, t2row * E}, {B_LW, (size_t)g.s2 * E},
        {B_LW2, (size_t)g.s2 * E}, {B_LP, (size_t)(Ly + 1) * g.s2 * E}, {B_RP, (size_t)(Ly + 1) * g.s2 * E}};
    place(k.p, k.smem, budget, b);
  }
  // sampler plan: union of the above
  budget = h->budget[3];
  {
    KPlan& k = h->kp[3];
    k.p.ci = ci;
    k.p.cx = cx;
    int cxs = cx;
    while (cxs > 1 && (size_t)D * D * D * chi * cxs > 4096) cxs = (cxs + 1) / 2;
    k.p.cx = cxs;
    const size_t tt = std::max(t1row, (size_t)D * D * D * chi * cxs + chi);
    const size_t lw = std::max((size_t)g.s2, (size_t)g.se);
    // the row step (E^u / E^l updates) and the move sandwiches never overlap in time
    std::vector<std::pair<int, size_t>> common = {
        {B_RED, 40 * 8}, {B_SIG, (mX + 4) * E}, {B_SEL, 2 * mX * 4}, {B_S, (size_t)g.Lx * g.Ly}, {B_A, (size_t)g.sT * E}};
    std::vector<std::pair<int, size_t>> rowstep = {
        {B_E, (size_t)g.se * E}, {B_C, (size_t)n * chi * E}, {B_W, env_w_elems(chi, D, ci) * E},
        {B_R, (size_t)n * n * E}, {B_Z, zsz * E}, {B_RHIST, (size_t)std::max(1, Ly - 1) * n * n * E}};
    std::vector<std::pair<int, size_t>> sandwich = {
        {B_A2, (size_t)g.sT * E}, {B_EU, (size_t)g.se * E}, {B_EL, (size_t)g.se * E}, {B_T1, tt * E},
        {B_T2, tt * E}, {B_LW, lw * E}, {B_LW2, lw * E}, {B_LP, lw * E}, {B_RP, (size_t)(Ly + 1) * lw * E}};
    place_overlay(k.p, k.smem, budget, common, rowstep, sandwich);
  }
}

// The dynamic shared-memory limit is a property of a kernel instantiation, shared by every handle
// that launches it: only ever raise it (per precision and compiled shape), so that handles with
// different budgets can coexist.  Keyed by the scalar type (float and complex<float> kernels are
// different instantiations of the same size).
static std::mutex g_attr_mu;
static std::map<std::pair<int, int>, size_t> g_attr_max;

static peps_status finish_plans(peps_handle* h) {
  size_t maxsmem = h->kb.smem;
  for (auto& k : h->kp) maxsmem = std::max(maxsmem, k.smem);
  cudaError_t e = cudaSuccess;
  {
    std::lock_guard<std::mutex> lk(g_attr_mu);
    const int variant = (h->g.chi == 16 && h->g.D == 4) ? 1 : (h->g.chi == 24 && h->g.D == 4) ? 2 : 0;
    int dev = 0;
    cudaGetDevice(&dev);
    size_t& cur = g_attr_max[{h->elem * 64 + dev, variant}];  // per kernel scalar type
    if (maxsmem > cur) {
      e = dispatch_elem(h, [&](auto z) { return set_kernel_smem<decltype(z)>(h->g, maxsmem); });
      if (e == cudaSuccess) cur = maxsmem;
    }
  }
  if (e != cudaSuccess) return cuda_fail(h, e, "cudaFuncSetAttribute");
  size_t gmax = 0;
  for (int i = 0; i < 4; ++i) {
    KPlan& k = h->kp[i];
    int occ = dispatch_elem(h, [&](auto z) { return occupancy<decltype(z)>(h->g, i, k.smem); });
    if (occ < 1) return fail(h, PEPS_E_SHAPE, "kernel does not fit on an SM");
    k.grid = h->nsm * occ;
    gmax = std::max(gmax, (size_t)k.grid * (size_t)k.p.gstride);
  }
  {
    KPlan& k = h->kb;
    int occ = dispatch_elem(h, [&](auto z) { return occupancy<decltype(z)>(h->g, 4, k.smem); });
    if (occ < 1) return fail(h, PEPS_E_SHAPE, "bound kernel does not fit on an SM");
    k.grid = h->nsm * occ;
    gmax = std::max(gmax, (size_t)k.grid * (size_t)k.p.gstride);
  }
  if (gmax > h->gscratch_bytes) {
    if (h->gscratch) h_free(h, h->gscratch);
    h->gscratch = nullptr;
    h->gscratch_bytes = 0;
    e = h_malloc(h, (void**)&h->gscratch, gmax);
    if (e != cudaSuccess) return fail(h, PEPS_E_WORKSPACE, "scratch allocation failed");
    h->gscratch_bytes = gmax;
  }
  if (!h->ctr) {
    if (h_malloc(h, (void**)&h->ctr, 8 * sizeof(unsigned long long)) != cudaSuccess)
      return fail(h, PEPS_E_WORKSPACE, "counter allocation failed");
    cudaMemset(h->ctr, 0, 8 * sizeof(unsigned long long));
  }
  for (auto& k : h->kp) {
    k.p.gbase = h->gscratch;
    k.p.ctr = h->ctr;
  }
  h->kb.p.gbase = h->gscratch;
  h->kb.p.ctr = h->ctr;
  return PEPS_OK;
}

extern "C" peps_status peps_create(peps_handle** out, const peps_config* cfg) {
  return peps_create_ex(out, cfg, nullptr);
}

extern "C" peps_status peps_create_ex(peps_handle** out, const peps_config* cfg, const peps_allocator* alloc) {
  if (!out || !cfg) return PEPS_E_ARG;
  *out = nullptr;
  if (alloc && (!alloc->alloc || !alloc->free)) return PEPS_E_ARG;
  peps_config c = *cfg;
  if (c.Lx < 2 || c.Ly < 2 || c.Ly > MAX_LY || c.d < 2 || c.d > 4 || c.D < 1 || c.D > 8 || c.chi < c.D ||
      c.chi > 64 || c.max_samples < 1)
    return PEPS_E_SHAPE;
  if (c.prec != PEPS_PREC_FP64 && c.prec != PEPS_PREC_FP32 && c.prec != PEPS_PREC_MIXED) return PEPS_E_ARG;
  if (c.prec == PEPS_PREC_MIXED) {
    // the mixed-precision preset: the FP32 contraction kernels, a float-float Gram unless the
    // caller asked for the tensor-core one, and the float-float Cholesky with FP64 refinement
    c.prec = PEPS_PREC_FP32;
    if (c.gram == 0) c.gram = 2;
    c.solve = 2;
  }
  if (c.gram != 0 && c.gram != 1 && c.gram != 2) return PEPS_E_ARG;
  if (c.solve < 0 || c.solve > 3) return PEPS_E_ARG;
  if (c.cplx != 0 && c.cplx != 1) return PEPS_E_ARG;
  if (!(c.trunc_weight >= 0.0 && c.trunc_weight < 1.0)) return PEPS_E_ARG;
  if (c.cplx && c.gram == 1) return PEPS_E_UNSUPPORTED;  // the split-BF16 Gram is real only
  peps_handle* h = new peps_handle();
  h->cfg = c;
  if (alloc) {
    h->alloc = *alloc;
    h->has_alloc = true;
  }
  h->elem = (c.cplx ? 2 : 0) + (c.prec == PEPS_PREC_FP64 ? 0 : 1);
  h->esz = (size_t)((c.prec == PEPS_PREC_FP64) ? 8 : 4) * (c.cplx ? 2 : 1);
  Geo& g = h->g;
  g.Lx = c.Lx; g.Ly = c.Ly; g.d = c.d; g.D = c.D; g.chi = c.chi;
  g.n = c.chi * c.D;
  g.se = c.chi * c.D * c.chi;
  g.sT = c.D * c.D * c.D * c.D;
  g.s2 = c.chi * c.D * c.D * c.chi;
  g.cut = c.trunc_weight;
  const int N = c.Lx * c.Ly;
  h->site_off_h.assign(N + 1, 0);
  for (int x = 0; x < c.Lx; ++x)
    for (int y = 0; y < c.Ly; ++y) {
      const long long b = (long long)c.d * (y == 0 ? 1 : c.D) * (x == 0 ? 1 : c.D) * (y == c.Ly - 1 ? 1 : c.D) *
                          (x == c.Lx - 1 ? 1 : c.D);
      h->site_off_h[x * c.Ly + y + 1] = h->site_off_h[x * c.Ly + y] + b;
    }
  h->Np = h->site_off_h[N];
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&h->nsm, cudaDevAttrMultiProcessorCount, dev);
  auto bad = [&](peps_status st, const char* m) {
    h->err = m;
    peps_destroy(h);
    return st;
  };
  if (h_malloc(h, (void**)&h->Tpad, (size_t)N * c.d * g.sT * h->esz) != cudaSuccess) return bad(PEPS_E_WORKSPACE, "Tpad");
  if (h_malloc(h, (void**)&h->site_off, sizeof(long long) * (N + 1)) != cudaSuccess) return bad(PEPS_E_WORKSPACE, "site_off");
  cudaMemcpy(h->site_off, h->site_off_h.data(), sizeof(long long) * (N + 1), cudaMemcpyHostToDevice);
  const size_t envb = (size_t)c.max_samples * 2 * c.Lx * c.Ly * g.se * h->esz;
  if (h_malloc(h, (void**)&h->envs, envb) != cudaSuccess) return bad(PEPS_E_WORKSPACE, "environment store");
  if (h_malloc(h, (void**)&h->logs, sizeof(double) * (size_t)c.max_samples * 2 * c.Lx) != cudaSuccess) return bad(PEPS_E_WORKSPACE, "logs");
  if (h_malloc(h, (void**)&h->wdisc, sizeof(float) * (size_t)c.max_samples) != cudaSuccess) return bad(PEPS_E_WORKSPACE, "wdisc");
  if (h_malloc(h, (void**)&h->rowout, sizeof(double) * 4 * (size_t)c.max_samples * c.Lx) != cudaSuccess) return bad(PEPS_E_WORKSPACE, "rowout");
  if (h_malloc(h, (void**)&h->pairout, sizeof(double) * 4 * (size_t)c.max_samples * c.Lx) != cudaSuccess) return bad(PEPS_E_WORKSPACE, "pairout");
  if (h_malloc(h, (void**)&h->status_tmp, sizeof(int) * (size_t)c.max_samples) != cudaSuccess) return bad(PEPS_E_WORKSPACE, "status");
  if (h_malloc(h, (void**)&h->ustat, sizeof(int) * (size_t)c.max_samples) != cudaSuccess) return bad(PEPS_E_WORKSPACE, "status");
  if (h_malloc(h, (void**)&h->sword, sizeof(int)) != cudaSuccess) return bad(PEPS_E_WORKSPACE, "status word");
  cudaMemset(h->sword, 0, sizeof(int));
  cudaMemset(h->Tpad, 0, (size_t)N * c.d * g.sT * h->esz);
  plan_all(h);
  peps_status st = finish_plans(h);
  if (st != PEPS_OK) {
    std::string m = h->err;
    peps_destroy(h);
    return st;
  }
  *out = h;
  return PEPS_OK;
}

extern "C" peps_status peps_destroy(peps_handle* h) {
  if (!h) return PEPS_E_ARG;
  void* ptrs[] = {h->Tpad, h->site_off, h->envs, h->logs, h->wdisc, h->rowout, h->pairout, h->status_tmp,
                  h->gscratch, h->d_tinfo, h->d_ab, h->d_eh, h->d_rowoff, h->d_pairoff, h->d_pij, h->d_pv,
                  h->d_onsite, h->Obar, h->Tm, h->Vm, h->Hm, h->mean, h->ebar, h->yv, h->xv, h->cnt, h->td, h->ctr,
                  h->lp_Sp, h->lp_l0, h->lp_l1, h->lp_aux, h->g_hi, h->g_lo, h->bout, h->DL, h->dl_work,
                  h->dl_status, h->dscratch, h->ustat, h->sword};
  for (void* p : ptrs)
    if (p) h_free(h, p);
  for (cudaEvent_t e : h->evpool) cudaEventDestroy(e);
  delete h;
  return PEPS_OK;
}

extern "C" long long peps_num_params(const peps_handle* h) { return h ? h->Np : -1; }

extern "C" const char* peps_last_error(const peps_handle* h) { return (h && !h->err.empty()) ? h->err.c_str() : ""; }

extern "C" peps_status peps_set_params(peps_handle* h, const double* theta_dev, void* stream) {
  if (!h || !theta_dev) return fail(h, PEPS_E_ARG, "null argument");
  ++h->param_gen;  // stored environments no longer belong to the parameters
  cudaStream_t s = (cudaStream_t)stream;
  const int ts = tstart(h, TC_PAD, s);
  cudaError_t e = dispatch_elem(h, [&](auto z) {
    using T = decltype(z);
    return launch_pad<T>(h->g, theta_dev, h->site_off, (T*)h->Tpad, s);
  });
  if (e != cudaSuccess) return cuda_fail(h, e, "pad theta");
  tstop(h, ts, s);
  return PEPS_OK;
}

// ---- Hamiltonian packing -----------------------------------------------------------------
template <typename V>
static void put(std::vector<char>& k, const V* p, size_t n) {
  const char* c = (const char*)p;
  k.insert(k.end(), c, c + n * sizeof(V));
}

template <typename V>
static cudaError_t upload(peps_handle* hd, V** d, const std::vector<V>& h, cudaStream_t s) {
  if (*d) { h_free(hd, *d); *d = nullptr; }
  if (h.empty()) return cudaSuccess;
  cudaError_t e = h_malloc(hd, (void**)d, sizeof(V) * h.size());
  if (e != cudaSuccess) return e;
  return cudaMemcpyAsync(*d, h.data(), sizeof(V) * h.size(), cudaMemcpyHostToDevice, s);
}

static peps_status set_hamiltonian(peps_handle* h, const peps_hamiltonian* H, cudaStream_t s) {
  const Geo& g = h->g;
  const int N = g.Lx * g.Ly, d = g.d;
  if (H->nterms < 0 || H->npairs < 0) return fail(h, PEPS_E_ARG, "negative term count");
  if ((H->nterms > 0 && !H->terms) || (H->npairs > 0 && (!H->pair_ij_host || !H->pair_v_host)))
    return fail(h, PEPS_E_ARG, "null term arrays");
  // content key
  std::vector<char> key;
  put(key, &H->nterms, 1);
  for (int t = 0; t < H->nterms; ++t) {
    const peps_term& tm = H->terms[t];
    if (tm.nsites < 1 || tm.nsites > 4 || !tm.h_host) return fail(h, PEPS_E_ARG, "bad term");
    int dk = 1;
    for (int i = 0; i < tm.nsites; ++i) dk *= d;
    put(key, &tm.nsites, 1);
    put(key, tm.sites, 4);
    put(key, tm.h_host, (size_t)dk * dk * 2);
  }
  put(key, &H->npairs, 1);
  if (H->npairs) {
    put(key, H->pair_ij_host, (size_t)2 * H->npairs);
    put(key, H->pair_v_host, (size_t)H->npairs);
  }
  const int has_on = H->onsite_host ? 1 : 0;
  put(key, &has_on, 1);
  if (has_on) put(key, H->onsite_host, (size_t)N * d);
  if (key == h->ham_key && !key.empty()) return PEPS_OK;
  // pack terms
  struct Rec { int two, x0; std::vector<int> ti; std::vector<int> ab; std::vector<double> hv; };
  std::vector<Rec> recs;
  for (int t = 0; t < H->nterms; ++t) {
    const peps_term& tm = H->terms[t];
    int xmin = 1 << 30, xmax = -1, ymin = 1 << 30, ymax = -1;
    for (int i = 0; i < tm.nsites; ++i) {
      const int sidx = tm.sites[i];
      if (sidx < 0 || sidx >= N) return fail(h, PEPS_E_ARG, "term site out of range");
      for (int j = 0; j < i; ++j)
        if (tm.sites[j] == sidx) return fail(h, PEPS_E_ARG, "repeated site in a term");
      xmin = std::min(xmin, sidx / g.Ly); xmax = std::max(xmax, sidx / g.Ly);
      ymin = std::min(ymin, sidx % g.Ly); ymax = std::max(ymax, sidx % g.Ly);
    }
    if (xmax - xmin > 1) return fail(h, PEPS_E_UNSUPPORTED, "term spans more than two rows");
    if (ymax - ymin > 1) return fail(h, PEPS_E_UNSUPPORTED, "term spans more than two columns");
    Rec r;
    r.two = (xmax > xmin);
    r.x0 = xmin;
    r.ti.assign(TI_N, 0);
    r.ti[TI_K] = tm.nsites;
    for (int i = 0; i < 4; ++i) r.ti[TI_S0 + i] = (i < tm.nsites) ? tm.sites[i] : -1;
    r.ti[TI_X0] = xmin;
    r.ti[TI_Y0] = ymin;
    r.ti[TI_W] = ymax - ymin + 1;
    r.ti[TI_TWO] = r.two;
    int dk = 1;
    for (int i = 0; i < tm.nsites; ++i) dk *= d;
    for (int a = 0; a < dk; ++a)
      for (int b = 0; b < dk; ++b) {
        const double re = tm.h_host[2 * ((size_t)a * dk + b)], im = tm.h_host[2 * ((size_t)a * dk + b) + 1];
        if (re != 0.0 || im != 0.0) {
          r.ab.push_back(a);
          r.ab.push_back(b);
          r.hv.push_back(re);
          r.hv.push_back(im);
        }
      }
    recs.push_back(std::move(r));
  }
  std::stable_sort(recs.begin(), recs.end(), [](const Rec& a, const Rec& b) {
    return a.two != b.two ? a.two < b.two : a.x0 < b.x0;
  });
  h->h_tinfo.clear(); h->h_ab.clear(); h->h_eh.clear();
  h->h_rowoff.assign(g.Lx + 1, 0);
  h->h_pairoff.assign(g.Lx, 0);
  int t = 0;
  const int nt = (int)recs.size();
  std::vector<int> cnt1(g.Lx, 0), cnt2(g.Lx, 0);
  for (auto& r : recs) (r.two ? cnt2 : cnt1)[r.x0]++;
  for (int x = 0; x < g.Lx; ++x) h->h_rowoff[x + 1] = h->h_rowoff[x] + cnt1[x];
  h->h_pairoff[0] = h->h_rowoff[g.Lx];
  for (int x = 0; x + 1 < g.Lx; ++x) h->h_pairoff[x + 1] = h->h_pairoff[x] + cnt2[x];
  for (auto& r : recs) {
    r.ti[TI_EOFF] = (int)h->h_ab.size() / 2;
    r.ti[TI_ECNT] = (int)r.ab.size() / 2;
    h->h_tinfo.insert(h->h_tinfo.end(), r.ti.begin(), r.ti.end());
    h->h_ab.insert(h->h_ab.end(), r.ab.begin(), r.ab.end());
    h->h_eh.insert(h->h_eh.end(), r.hv.begin(), r.hv.end());
    ++t;
  }
  (void)t;
  h->n_pair_terms = 0;
  for (int x = 0; x < g.Lx; ++x) h->n_pair_terms += cnt2[x];
  h->h_pij.assign(H->pair_ij_host, H->pair_ij_host + 2 * (size_t)H->npairs);
  h->h_pv.assign(H->pair_v_host, H->pair_v_host + (size_t)H->npairs);
  for (int p = 0; p < H->npairs; ++p)
    if (h->h_pij[2 * p] < 0 || h->h_pij[2 * p] >= N || h->h_pij[2 * p + 1] < 0 || h->h_pij[2 * p + 1] >= N)
      return fail(h, PEPS_E_ARG, "pair site out of range");
  if (has_on) h->h_onsite.assign(H->onsite_host, H->onsite_host + (size_t)N * d);
  else h->h_onsite.clear();
  CK(upload(h, &h->d_tinfo, h->h_tinfo, s), "upload terms");
  CK(upload(h, &h->d_ab, h->h_ab, s), "upload terms");
  CK(upload(h, &h->d_eh, h->h_eh, s), "upload terms");
  CK(upload(h, &h->d_rowoff, h->h_rowoff, s), "upload terms");
  CK(upload(h, &h->d_pairoff, h->h_pairoff, s), "upload terms");
  CK(upload(h, &h->d_pij, h->h_pij, s), "upload pairs");
  CK(upload(h, &h->d_pv, h->h_pv, s), "upload pairs");
  CK(upload(h, &h->d_onsite, h->h_onsite, s), "upload onsite");
  CK(cudaStreamSynchronize(s), "hamiltonian upload");
  h->tt.nterm = nt;
  h->tt.tinfo = h->d_tinfo;
  h->tt.ent_ab = h->d_ab;
  h->tt.ent_h = h->d_eh;
  h->tt.row_off = h->d_rowoff;
  h->tt.pair_off = h->d_pairoff;
  h->dg.npairs = H->npairs;
  h->dg.pair_ij = h->d_pij;
  h->dg.pair_v = h->d_pv;
  h->dg.onsite = has_on ? h->d_onsite : nullptr;
  h->ham_key.swap(key);
  return PEPS_OK;
}

// ---- evaluation pipeline -----------------------------------------------------------------
template <typename T>
static peps_status run_eval(peps_handle* h, const peps_hamiltonian* H, const uint8_t* S, int Ns, double* logabs,
                            double* phase, double* eloc, void* O, int32_t* status, cudaStream_t s, int sides) {
  const Geo& g = h->g;
  int* st = status ? (int*)status : h->status_tmp;
  // the sampler's upper environments belong to S when S is the unmodified output of the last
  // peps_sample on this handle (caller's promise, enabled by peps_set_env_reuse) and the
  // parameters have not changed since
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(s, &cap);
  // (after an upward sweep the lower side is the stored one, which an amplitude-only call,
  // needing just the upper side, cannot use)
  const bool reuse = h->env_reuse && cap == cudaStreamCaptureStatusNone && Ns > 0 && S == h->rs_S && Ns == h->rs_Ns &&
                     h->rs_gen == h->param_gen && !(h->rs_up && sides == 1);
  if (reuse) CK(cudaMemcpyAsync(st, h->ustat, sizeof(int) * Ns, cudaMemcpyDeviceToDevice, s), "copy status");
  else CK(cudaMemsetAsync(st, 0, sizeof(int) * Ns, s), "memset status");
  CK(cudaMemsetAsync(h->wdisc, 0, sizeof(float) * Ns, s), "memset wdisc");
  if (Ns == 0) return PEPS_OK;
  if (reuse) sides = (sides == 3) ? (h->rs_up ? 1 : 2) : 0;
  else h->rs_gen = -1;  // the store's upper rows now belong to this batch
  TermTab none{};
  const bool want_e = (eloc != nullptr);
  if (want_e) {
    peps_status ps = set_hamiltonian(h, H, s);
    if (ps != PEPS_OK) return ps;
  }
  if (want_e && h->tt.nterm == 0 && !O && !logabs && !phase) {
    // a diagonal Hamiltonian and no amplitude requested: E_loc(S) needs no contraction
    const int ts = tstart(h, TC_COMBINE, s);
    CK(launch_combine(g, Ns, S, h->rowout, h->pairout, 0, 0, h->dg, nullptr, nullptr, eloc, s), "combine kernel");
    tstop(h, ts, s);
    return PEPS_OK;
  }
  const KPlan& ke = h->kp[0];
  int ts = -1;
  if (sides != 0) {
    ts = tstart(h, TC_ENV, s);
    CK(launch_env<T>(g, ke.p, std::min(ke.grid, Ns * (sides == 3 ? 2 : 1)), ke.smem, (const T*)h->Tpad, S, Ns, sides,
                     (T*)h->envs, h->logs, st, h->wdisc, s), "env kernel");
    tstop(h, ts, s);
  }
  const KPlan& kr = h->kp[1];
  const bool all_rows = want_e || (O != nullptr);
  const int x_lo = all_rows ? 0 : g.Lx - 1;
  ts = tstart(h, TC_ROW, s);
  CK(launch_row<T>(g, kr.p, std::min(kr.grid, Ns * (g.Lx - x_lo)), kr.smem, (const T*)h->Tpad, S, Ns, x_lo, g.Lx,
                   (const T*)h->envs, h->logs, (T*)O, h->site_off, h->Np, want_e ? h->tt : none, h->rowout, st, s),
     "row kernel");
  tstop(h, ts, s);
  const bool pairs = want_e && h->n_pair_terms > 0;
  if (pairs) {
    const KPlan& kq = h->kp[2];
    ts = tstart(h, TC_PAIR, s);
    CK(launch_pair<T>(g, kq.p, std::min(kq.grid, Ns * (g.Lx - 1)), kq.smem, (const T*)h->Tpad, S, Ns,
                      (const T*)h->envs, h->logs, h->tt, h->pairout, st, s), "pair kernel");
    tstop(h, ts, s);
  }
  DiagTab dg = want_e ? h->dg : DiagTab{};
  ts = tstart(h, TC_COMBINE, s);
  CK(launch_combine(g, Ns, S, h->rowout, h->pairout, want_e ? 1 : 0, pairs ? 1 : 0, dg, logabs, phase, eloc, s),
     "combine kernel");
  CK(launch_status_or(st, Ns, h->sword, s), "status word");
  tstop(h, ts, s, 2);
  return PEPS_OK;
}

static peps_status check_eval(peps_handle* h, const uint8_t* S, int Ns) {
  if (!h) return PEPS_E_ARG;
  if (Ns < 0 || (Ns > 0 && !S)) return fail(h, PEPS_E_ARG, "bad configuration batch");
  if (Ns > h->cfg.max_samples) return fail(h, PEPS_E_SHAPE, "Ns exceeds max_samples");
  return PEPS_OK;
}

extern "C" peps_status peps_evaluate(peps_handle* h, const peps_hamiltonian* H, const uint8_t* S_dev, int Ns,
                                     double* logabs_dev, double* phase_dev, double* eloc_dev, void* O_dev,
                                     int32_t* status_dev, void* stream) {
  peps_status c = check_eval(h, S_dev, Ns);
  if (c != PEPS_OK) return c;
  if (eloc_dev && !H) return fail(h, PEPS_E_ARG, "eloc requested without a Hamiltonian");
  const int sides = (eloc_dev || O_dev) ? 3 : 1;
  return dispatch_elem(h, [&](auto z) {
    return run_eval<decltype(z)>(h, H, S_dev, Ns, logabs_dev, phase_dev, eloc_dev, O_dev, status_dev,
                                 (cudaStream_t)stream, sides);
  });
}

extern "C" peps_status peps_amplitudes(peps_handle* h, const uint8_t* S_dev, int Ns, double* logabs_dev,
                                       double* phase_dev, int32_t* status_dev, void* stream) {
  if (h && (!logabs_dev || !phase_dev) && Ns > 0) return fail(h, PEPS_E_ARG, "null output");
  return peps_evaluate(h, nullptr, S_dev, Ns, logabs_dev, phase_dev, nullptr, nullptr, status_dev, stream);
}

extern "C" peps_status peps_local_energy(peps_handle* h, const peps_hamiltonian* H, const uint8_t* S_dev, int Ns,
                                         double* eloc_dev, int32_t* status_dev, void* stream) {
  if (h && (!H || (!eloc_dev && Ns > 0))) return fail(h, PEPS_E_ARG, "null argument");
  return peps_evaluate(h, H, S_dev, Ns, nullptr, nullptr, eloc_dev, nullptr, status_dev, stream);
}

extern "C" peps_status peps_logderiv(peps_handle* h, const uint8_t* S_dev, int Ns, void* O_dev, int32_t* status_dev,
                                     void* stream) {
  if (h && !O_dev && Ns > 0) return fail(h, PEPS_E_ARG, "null output");
  return peps_evaluate(h, nullptr, S_dev, Ns, nullptr, nullptr, nullptr, O_dev, status_dev, stream);
}

// ---- direct sampling ---------------------------------------------------------------------
static std::mutex g_direct_mu;
static std::map<std::pair<int, int>, size_t> g_direct_attr;

extern "C" peps_status peps_direct_prepare(peps_handle* h, int chi_double, void* stream) {
  if (!h) return PEPS_E_ARG;
  const Geo& g = h->g;
  const int D = g.D, Ly = g.Ly, Lx = g.Lx;
  if (chi_double < 1 || chi_double * D * D > 1024) return fail(h, PEPS_E_ARG, "chi_double outside 1 .. 1024 / D^2");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t E = h->esz;
  const DlDims dd = dl_dims(D, chi_double);
  const size_t sd = (size_t)chi_double * dd.P * chi_double;
  // double-layer rows and the compression's work buffers
  const size_t dlb = (size_t)(Lx + 1) * Ly * sd * E;
  size_t n8[8];
  dl_work_elems(Ly, D, chi_double, n8);
  size_t wb = 0;
  for (int i = 0; i < 8; ++i) wb += al(n8[i] * E);
  if (dlb > h->DL_bytes) {
    if (h->DL) h_free(h, h->DL);
    h->DL = nullptr;
    h->DL_bytes = 0;
    if (h_malloc(h, (void**)&h->DL, dlb) != cudaSuccess) return fail(h, PEPS_E_WORKSPACE, "double-layer environments");
    h->DL_bytes = dlb;
  }
  if (wb > h->dl_work_bytes) {
    if (h->dl_work) h_free(h, h->dl_work);
    h->dl_work = nullptr;
    h->dl_work_bytes = 0;
    if (h_malloc(h, (void**)&h->dl_work, wb) != cudaSuccess) return fail(h, PEPS_E_WORKSPACE, "double-layer work buffers");
    h->dl_work_bytes = wb;
  }
  if (!h->dl_status && h_malloc(h, (void**)&h->dl_status, sizeof(int)) != cudaSuccess)
    return fail(h, PEPS_E_WORKSPACE, "status");
  // the sampler's buffer plan: the row step's buffers, then the configuration, two E^u rows,
  // the candidates, the right partials, the contraction temporaries and one ket site (and its
  // conjugate)
  const int n = g.n, chi = g.chi, mX = n + (n & 1), ci = std::min(n, 8);
  const size_t AB = (size_t)chi * D, rsz = AB * chi_double * AB, ksz = (size_t)g.d * D * AB * AB;
  const size_t tsz = (size_t)g.d * D * chi_double * AB * AB;
  KPlan& k = h->kd;
  k.p.ci = ci;
  k.p.cx = h->kp[0].p.cx;
  std::vector<std::pair<int, size_t>> b = {
      {B_RED, 40 * 8}, {B_SIG, (mX + 4) * E}, {B_SEL, 2 * mX * 4}, {B_A, (size_t)g.sT * E}, {B_E, (size_t)g.se * E},
      {B_C, (size_t)n * chi * E}, {B_W, env_w_elems(chi, D, ci) * E}, {B_R, (size_t)n * n * E},
      {B_Z, env_z_elems(chi, D) * E}, {B_RHIST, (size_t)std::max(1, Ly - 1) * n * n * E}, {B_S, (size_t)Lx * Ly},
      {B_EU, (size_t)2 * Ly * g.se * E}, {B_LW2, (size_t)(g.d + 1) * rsz * E}, {B_RP, (size_t)(Ly + 1) * rsz * E},
      {B_LP, tsz * E}, {B_LW, tsz * E}, {B_T1, ksz * E}, {B_T2, ksz * E}};
  place(k.p, k.smem, wide_budget(h), b);
  cudaError_t e = cudaSuccess;
  {
    std::lock_guard<std::mutex> lk(g_direct_mu);
    int dev = 0;
    cudaGetDevice(&dev);
    size_t& cur = g_direct_attr[{h->elem, dev}];
    if (k.smem > cur) {
      e = dispatch_elem(h, [&](auto z) { return kattr_direct<decltype(z)>(g, k.smem, nullptr, 0); });
      if (e == cudaSuccess) cur = k.smem;
    }
  }
  if (e != cudaSuccess) return cuda_fail(h, e, "cudaFuncSetAttribute (direct)");
  int occ = 0;
  e = dispatch_elem(h, [&](auto z) { return kattr_direct<decltype(z)>(g, 0, &occ, k.smem); });
  if (e != cudaSuccess || occ < 1) return fail(h, PEPS_E_SHAPE, "direct-sampling kernel does not fit on an SM");
  k.grid = h->nsm * occ;
  const size_t ab = (size_t)k.grid * k.p.gstride;
  if (ab > h->dscratch_bytes) {
    if (h->dscratch) h_free(h, h->dscratch);
    h->dscratch = nullptr;
    h->dscratch_bytes = 0;
    if (h_malloc(h, (void**)&h->dscratch, ab) != cudaSuccess) return fail(h, PEPS_E_WORKSPACE, "direct-sampling arena");
    h->dscratch_bytes = ab;
  }
  k.p.gbase = h->dscratch;
  k.p.ctr = h->ctr;
  h->dl_chid = chi_double;
  const int ts = tstart(h, TC_DIRECT, s);
  e = dispatch_elem(h, [&](auto z) {
    using T = decltype(z);
    DlWork<T> w;
    T** ptrs[8] = {&w.B, &w.Rh, &w.Z, &w.Y, &w.X, &w.Vt, &w.C, &w.Cn};
    char* base = (char*)h->dl_work;
    for (int i = 0; i < 8; ++i) {
      *ptrs[i] = (T*)base;
      base += al(n8[i] * E);
    }
    return launch_dl_env<T>(g, chi_double, (const T*)h->Tpad, (T*)h->DL, w, h->dl_status, s);
  });
  if (e != cudaSuccess) return cuda_fail(h, e, "double-layer kernel");
  tstop(h, ts, s);
  return PEPS_OK;
}

extern "C" peps_status peps_direct_sample(peps_handle* h, uint8_t* S_dev, int Ns, uint64_t seed, uint64_t draw,
                                          double* logp_dev, int32_t* status_dev, void* stream) {
  peps_status c = check_eval(h, S_dev, Ns);
  if (c != PEPS_OK) return c;
  if (!h->DL || h->dl_chid < 1) return fail(h, PEPS_E_ARG, "peps_direct_prepare has not been called");
  if (!logp_dev && Ns > 0) return fail(h, PEPS_E_ARG, "null log p output");
  h->rs_gen = -1;  // S_dev is overwritten
  cudaStream_t s = (cudaStream_t)stream;
  int* st = status_dev ? (int*)status_dev : h->status_tmp;
  if (Ns == 0) return PEPS_OK;
  const KPlan& k = h->kd;
  const int ts = tstart(h, TC_DIRECT, s);
  cudaError_t e = dispatch_elem(h, [&](auto z) {
    using T = decltype(z);
    return launch_direct<T>(h->g, k.p, std::min(k.grid, Ns), k.smem, h->dl_chid, (const T*)h->Tpad, (const T*)h->DL,
                            S_dev, Ns, seed, draw, logp_dev, st, s);
  });
  if (e != cudaSuccess) return cuda_fail(h, e, "direct-sampling kernel");
  CK(launch_status_or(st, Ns, h->sword, s), "status word");
  tstop(h, ts, s, 2);
  return PEPS_OK;
}

// ---- global rotation of the physical index ------------------------------------------------
extern "C" peps_status peps_rotate_params(const peps_handle* h, const double* M_host, const double* theta_in_dev,
                                          int in_cplx, double* theta_out_dev, void* stream) {
  peps_handle* hh = const_cast<peps_handle*>(h);
  if (!h || !M_host || !theta_in_dev || !theta_out_dev) return fail(hh, PEPS_E_ARG, "null argument");
  if (in_cplx != 0 && in_cplx != 1) return fail(hh, PEPS_E_ARG, "in_cplx must be 0 or 1");
  if ((const void*)theta_in_dev == (const void*)theta_out_dev) return fail(hh, PEPS_E_ARG, "in and out must differ");
  RotM M{};
  const int d = h->g.d;
  for (int i = 0; i < 2 * d * d; ++i) M.m[i] = M_host[i];
  cudaError_t e = launch_rotate(h->g.Lx * h->g.Ly, d, h->site_off, M, theta_in_dev, in_cplx, theta_out_dev,
                                (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(hh, e, "rotate kernel");
  return PEPS_OK;
}

extern "C" peps_status peps_set_env_reuse(peps_handle* h, int enable) {
  if (!h || (enable != 0 && enable != 1)) return fail(h, PEPS_E_ARG, "enable must be 0 or 1");
  h->env_reuse = enable;
  h->rs_gen = -1;
  return PEPS_OK;
}

// ---- variational-bound estimator ---------------------------------------------------------
extern "C" peps_status peps_local_energy_bound(peps_handle* h, const peps_hamiltonian* H, const uint8_t* S_dev,
                                               int Ns, int cut, double* eloc_dev, double* logabs_dev,
                                               double* phase_dev, int32_t* status_dev, void* stream) {
  peps_status c = check_eval(h, S_dev, Ns);
  if (c != PEPS_OK) return c;
  if (!H || (!eloc_dev && Ns > 0)) return fail(h, PEPS_E_ARG, "null argument");
  if (cut < 1 || cut > h->g.Lx - 1) return fail(h, PEPS_E_ARG, "cut outside 1 .. Lx-1");
  cudaStream_t s = (cudaStream_t)stream;
  int* st = status_dev ? (int*)status_dev : h->status_tmp;
  CK(cudaMemsetAsync(st, 0, sizeof(int) * Ns, s), "memset status");
  CK(cudaMemsetAsync(h->wdisc, 0, sizeof(float) * Ns, s), "memset wdisc");
  if (Ns == 0) return PEPS_OK;
  peps_status ps = set_hamiltonian(h, H, s);
  if (ps != PEPS_OK) return ps;
  h->rs_gen = -1;  // the environment store is rewritten for this batch
  const int nt = std::max(h->tt.nterm, 1);
  const size_t need = (size_t)h->cfg.max_samples * nt * 2;
  if (need > h->bout_cap) {
    if (h->bout) h_free(h, h->bout);
    h->bout = nullptr;
    h->bout_cap = 0;
    if (h_malloc(h, (void**)&h->bout, need * sizeof(double)) != cudaSuccess) return fail(h, PEPS_E_WORKSPACE, "bound buffer");
    h->bout_cap = need;
  }
  const KPlan& ke = h->kp[0];
  const KPlan& kb = h->kb;
  int ts = tstart(h, TC_ENV, s);
  cudaError_t e = dispatch_elem(h, [&](auto z) {
    using T = decltype(z);
    return launch_env<T>(h->g, ke.p, std::min(ke.grid, Ns * 2), ke.smem, (const T*)h->Tpad, S_dev, Ns, 3, (T*)h->envs,
                         h->logs, st, h->wdisc, s);
  });
  if (e != cudaSuccess) return cuda_fail(h, e, "env kernel");
  tstop(h, ts, s);
  ts = tstart(h, TC_BOUND, s);
  e = dispatch_elem(h, [&](auto z) {
    using T = decltype(z);
    const long long items = (long long)Ns * nt;
    return launch_bound<T>(h->g, kb.p, (int)std::min<long long>(kb.grid, items), kb.smem, (const T*)h->Tpad, S_dev, Ns,
                           cut, (const T*)h->envs, h->logs, h->tt, h->bout, logabs_dev, phase_dev, st, s);
  });
  if (e != cudaSuccess) return cuda_fail(h, e, "bound kernel");
  tstop(h, ts, s);
  ts = tstart(h, TC_COMBINE, s);
  CK(launch_bound_combine(h->g, Ns, nt, S_dev, h->bout, h->dg, eloc_dev, s), "bound combine kernel");
  CK(launch_status_or(st, Ns, h->sword, s), "status word");
  tstop(h, ts, s, 2);
  return PEPS_OK;
}

// ---- sampler -----------------------------------------------------------------------------
extern "C" peps_status peps_sample(peps_handle* h, int move, uint8_t* S_dev, int Ns, int nsweeps, uint64_t seed,
                                   uint64_t sweep0, long long* accepted_dev, int32_t* status_dev, void* stream) {
  peps_status c = check_eval(h, S_dev, Ns);
  if (c != PEPS_OK) return c;
  if (move != PEPS_MOVE_EXCHANGE && move != PEPS_MOVE_FLIP) return fail(h, PEPS_E_ARG, "bad move kind");
  if (nsweeps < 0) return fail(h, PEPS_E_ARG, "negative sweep count");
  cudaStream_t s = (cudaStream_t)stream;
  int* st = status_dev ? (int*)status_dev : h->status_tmp;
  CK(cudaMemsetAsync(st, 0, sizeof(int) * Ns, s), "memset status");
  h->rs_gen = -1;
  if (Ns == 0 || nsweeps == 0) return PEPS_OK;
  CK(cudaMemsetAsync(h->ustat, 0, sizeof(int) * Ns, s), "memset status");
  const KPlan& k = h->kp[3];
  const int grid = std::min(k.grid, Ns);
  const int ts = tstart(h, TC_SAMPLE, s);
  cudaError_t e = dispatch_elem(h, [&](auto z) {
    using T = decltype(z);
    const KPlan& ke = h->kp[0];
    return launch_sample<T>(h->g, k.p, grid, k.smem, ke.p, std::min(ke.grid, Ns), ke.smem, (const T*)h->Tpad, S_dev, Ns,
                            move, nsweeps, seed, sweep0, (T*)h->envs, h->logs, accepted_dev, st, h->ustat, s);
  });
  if (e != cudaSuccess) return cuda_fail(h, e, "sampler kernel");
  // the split FP32 sweep leaves the environments of the final configurations on the side it
  // rebuilt last (E^u after a downward sweep, E^l after an upward one), with their row steps'
  // status bits in ustat; the single-launch sampler does not record the bits
  if (h->elem == 1) {
    h->rs_S = S_dev;
    h->rs_Ns = Ns;
    h->rs_gen = h->param_gen;
    h->rs_up = (int)((sweep0 + (uint64_t)nsweeps - 1) & 1ull);
  } else {
    h->rs_gen = -1;
  }
  CK(launch_status_or(st, Ns, h->sword, s), "status word");
  // kernel launches of the call: the FP32 split sweep launches a one-side k_env pass (every
  // downward sweep, and an upward sweep that opens the call), then per row k_sweep_moves and,
  // except after the last row, k_env_row; the other precisions one k_sample; then the status OR
  long long nl = 1;
  if (h->elem == 1) {
    for (int t = 0; t < nsweeps; ++t) {
      const bool up = ((sweep0 + (uint64_t)t) & 1ull) != 0;
      nl += (up && t > 0 ? 0 : 1) + 2 * (long long)h->cfg.Lx - 1;
    }
  } else {
    nl += 1;
  }
  tstop(h, ts, s, nl);
  return PEPS_OK;
}

// ---- MinSR -------------------------------------------------------------------------------
// doubles in each of the MinSR V and H buffers: n x n, and at least 4096 so that the rotation
// record of the tridiagonal eigen route (about n^2 doubles, relatively more for tiny n) fits
static size_t rec_doubles(int n) { return std::max((size_t)n * n, (size_t)4096); }

// MinSR workspace for Ns rows of Np real columns (a complex handle passes its real embedding:
// 2 Ns x 2 Np)
static peps_status ensure_minsr(peps_handle* h, int Ns, long long Np) {
  const int n = Ns + (Ns & 1);
  if (h->ms_cap >= n && h->ms_np >= Np) return PEPS_OK;
  double** bufs[] = {&h->Obar, &h->Tm, &h->Vm, &h->Hm, &h->mean, &h->ebar, &h->yv, &h->xv, &h->cnt, &h->td};
  for (double** b : bufs)
    if (*b) { h_free(h, *b); *b = nullptr; }
  const size_t nn = (size_t)n * n;
  const size_t nr = rec_doubles(n);  // V and H: also the tridiagonal route's rotation record
  // Obar holds n rows (the capacity): a later call with an even Ns up to n reuses it
  if (h_malloc(h, (void**)&h->Obar, sizeof(double) * (size_t)n * Np) != cudaSuccess ||
      h_malloc(h, (void**)&h->Tm, sizeof(double) * nn) != cudaSuccess || h_malloc(h, (void**)&h->Vm, sizeof(double) * nr) != cudaSuccess ||
      h_malloc(h, (void**)&h->Hm, sizeof(double) * nr) != cudaSuccess ||
      h_malloc(h, (void**)&h->td, sizeof(double) * td_workspace_doubles(n)) != cudaSuccess ||
      h_malloc(h, (void**)&h->mean, sizeof(double) * (size_t)Np) != cudaSuccess ||
      h_malloc(h, (void**)&h->ebar, sizeof(double) * n) != cudaSuccess || h_malloc(h, (void**)&h->yv, sizeof(double) * n) != cudaSuccess ||
      h_malloc(h, (void**)&h->xv, sizeof(double) * n) != cudaSuccess || h_malloc(h, (void**)&h->cnt, sizeof(double) * 16) != cudaSuccess)
    return fail(h, PEPS_E_WORKSPACE, "MinSR workspace allocation failed");
  if (h->cfg.gram == 1 || h->cfg.gram == 2) {
    if (h->g_hi) { h_free(h, h->g_hi); h->g_hi = nullptr; }
    if (h->g_lo) { h_free(h, h->g_lo); h->g_lo = nullptr; }
    const size_t e = (h->cfg.gram == 1) ? (size_t)gram_tc_pad_rows(Ns) * (size_t)gram_tc_pad_k(h->Np) * 2
                                        : (size_t)n * (size_t)Np * sizeof(float);  // the capacity, n rows
    if (h_malloc(h, (void**)&h->g_hi, e) != cudaSuccess || h_malloc(h, (void**)&h->g_lo, e) != cudaSuccess)
      return fail(h, PEPS_E_WORKSPACE, "Gram workspace allocation failed");
  }
  h->ms_cap = n;
  h->ms_np = Np;
  return PEPS_OK;
}

// MinSR scratch slots (h->cnt, 16 doubles): 0 factor breakdown (int), 2 weight sum, 3 FP64
// fallback flag of the mixed solve (int), 4 tensor-core Gram wait timeout (int), 6-7 residual
// norms, 8-9 Jacobi rotation counters (unsigned long long)

// T = A A^T (Ns x Ns, written to T with leading dimension ld) in the handle's Gram mode
static peps_status minsr_gram_into(peps_handle* h, const double* A, int Ns, long long K, double* T, int ld,
                                   bool mirror, cudaStream_t s) {
  int* gerr = (int*)(h->cnt + 4);
  const int ts = tstart(h, TC_GRAM, s);
  if (h->cfg.gram == 1) {
    CK(launch_gram_tc(A, Ns, K, h->g_hi, h->g_lo, T, ld, mirror, gerr, s), "tensor-core Gram");
    tstop(h, ts, s, mirror ? 3 : 2);
  } else if (h->cfg.gram == 2) {
    CK(launch_gram_ff(A, Ns, K, (float*)h->g_hi, (float*)h->g_lo, T, ld, s), "float-float Gram");
    tstop(h, ts, s, 2);
  } else {
    CK(launch_gram(A, Ns, K, T, ld, s), "Gram");
    tstop(h, ts, s);
  }
  return PEPS_OK;
}

// x = (T + lambda)^+ ebar on the handle's workspace: h->Tm (n x n, n = Ns rounded up to even, the
// Gram written, padding zero), h->ebar (n, padding zero) -> h->xv; info_dev as minsr_step
static peps_status minsr_solve_core(peps_handle* h, int Ns, double lambda, double rcond, double* info_dev,
                                    cudaStream_t s) {
  const int n = Ns + (Ns & 1);
  int* need64 = (int*)(h->cnt + 3);
  cudaError_t e = cudaSuccess;
  if (rcond > 0.0 && h->cfg.solve == 3) {
    // eigendecomposition with the pseudo-inverse cutoff through the tridiagonal form, applied to
    // ebar without forming V (opt-in: its QR chain is one thread of FP64 arithmetic, slower on
    // this GPU than the parallel Jacobi up to 8192 rows); the QR step count written to info[3]
    const int ts = tstart(h, TC_EIG, s);
    long long nl = 0;
    const size_t nr = rec_doubles(n);
    CK(td_pinv_apply(h->Tm, n, Ns, h->ebar, lambda, rcond, h->xv, h->Vm, nr, h->Hm, nr, h->td, info_dev, s, &nl),
       "tridiagonal eigen route");
    tstop(h, ts, s, nl);
  } else if (rcond > 0.0) {
    // eigendecomposition with the pseudo-inverse cutoff: one cooperative launch, the sweep count
    // written to info[3] on the device
    int ts = tstart(h, TC_EIG, s);
    CK(jacobi_eig(h->Tm, h->Vm, n, (unsigned long long*)(h->cnt + 8), h->Hm, h->yv, info_dev + 3, 40, s), "Jacobi");
    tstop(h, ts, s, 1);
    ts = tstart(h, TC_MINSR, s);
    CK(launch_minsr_apply(h->Tm, h->Vm, h->ebar, n, Ns, lambda, rcond, h->yv, h->xv, info_dev, s), "MinSR apply");
    tstop(h, ts, s, 3);
  } else {
    // nothing is cut: (T + lambda)^+ = (T + lambda)^-1, solved by Cholesky.  The mixed solve's
    // FP64 fallback is enqueued behind a device flag, so no host decision is needed.
    const int ts = tstart(h, TC_EIG, s);
    long long nl = 0;
    if (h->cfg.solve == 1 || h->cfg.solve == 2) {
      // h->Hm: the residual norms' block partials at its start, the solves' vector from n on;
      // h->Vm (n x n doubles) holds the FP32 factor, or the float-float factor's two n x n halves
      if (h->cfg.solve == 1)
        nl = chol_solve_mixed(h->Tm, (float*)h->Vm, n, Ns, lambda, h->ebar, h->xv, h->yv, h->cnt + 6, h->Hm, 4,
                              (int*)h->cnt, info_dev, need64, h->Hm + n, s, &e);
      else
        nl = chol_solve_ff(h->Tm, (float*)h->Vm, (float*)h->Vm + (size_t)n * n, n, Ns, lambda, h->ebar, h->xv, h->yv,
                           h->cnt + 6, h->Hm, 2, (int*)h->cnt, info_dev, need64, h->Hm + n, s, &e);
      if (e != cudaSuccess) return cuda_fail(h, e, "Cholesky");
      nl += chol_solve(h->Tm, n, Ns, lambda, h->ebar, h->xv, (int*)h->cnt, info_dev, need64, h->yv, s, &e);
    } else {
      nl = chol_solve(h->Tm, n, Ns, lambda, h->ebar, h->xv, (int*)h->cnt, info_dev, nullptr, h->yv, s, &e);
    }
    if (e != cudaSuccess) return cuda_fail(h, e, "Cholesky");
    tstop(h, ts, s, nl);
  }
  return PEPS_OK;
}

static peps_status check_minsr_args(peps_handle* h, int Ns, double lambda, double rcond) {
  if (Ns < 2) return fail(h, PEPS_E_ARG, "MinSR needs at least two samples");
  if (!(lambda > 0.0 || rcond > 0.0) || lambda < 0.0 || rcond < 0.0)
    return fail(h, PEPS_E_ARG, "MinSR needs lambda > 0 or rcond > 0");
  return PEPS_OK;
}

extern "C" peps_status minsr_step(peps_handle* h, const void* O_dev, const double* eloc_dev, const double* w_dev,
                                  int Ns, double lambda, double rcond, double tau, double* dtheta_dev,
                                  double* info_dev, void* stream) {
  if (!h) return PEPS_E_ARG;
  if (!O_dev || !eloc_dev || !dtheta_dev || !info_dev) return fail(h, PEPS_E_ARG, "bad MinSR argument");
  peps_status ps = check_minsr_args(h, Ns, lambda, rcond);
  if (ps != PEPS_OK) return ps;
  // a complex handle solves the real embedding (2 Ns rows, 2 N_p columns), see launch_center_cplx
  const bool cx = h->cfg.cplx != 0;
  const int Ns_c = Ns;
  const long long Np_c = h->Np;
  if (cx) Ns = 2 * Ns;
  const long long Np = cx ? 2 * h->Np : h->Np;
  ps = ensure_minsr(h, Ns, Np);
  if (ps != PEPS_OK) return ps;
  cudaStream_t s = (cudaStream_t)stream;
  const int n = Ns + (Ns & 1);
  double* wsum = h->cnt + 2;
  int* gerr = (int*)(h->cnt + 4);
  int ts = tstart(h, TC_MINSR, s);
  CK(cudaMemsetAsync(h->ebar, 0, sizeof(double) * n, s), "memset");
  CK(cudaMemsetAsync(gerr, 0, sizeof(int), s), "memset");
  cudaError_t e = dispatch_elem(h, [&](auto z) {
    using T = decltype(z);
    using R = typename Scal<T>::R;
    if constexpr (Scal<T>::complex) {
      const cudaError_t e1 = launch_center_cplx<R>((const R*)O_dev, w_dev, Ns_c, Np_c, h->Obar, wsum, s);
      return e1 != cudaSuccess ? e1 : launch_center_e_cplx(eloc_dev, w_dev, Ns_c, h->ebar, s);
    } else {
      const cudaError_t e1 = launch_center<T>((const T*)O_dev, w_dev, Ns, Np, h->mean, h->Obar, wsum, s);
      return e1 != cudaSuccess ? e1 : launch_center_e(eloc_dev, w_dev, Ns, h->ebar, s);
    }
  });
  if (e != cudaSuccess) return cuda_fail(h, e, "centre O and E_loc");
  CK(cudaMemsetAsync(h->Tm, 0, sizeof(double) * (size_t)n * n, s), "memset");
  tstop(h, ts, s, (w_dev ? 3 : 2) + 2);
  if ((ps = minsr_gram_into(h, h->Obar, Ns, Np, h->Tm, n, rcond > 0.0, s)) != PEPS_OK) return ps;
  if ((ps = minsr_solve_core(h, Ns, lambda, rcond, info_dev, s)) != PEPS_OK) return ps;
  ts = tstart(h, TC_MINSR, s);
  CK(launch_obar_t_x(h->Obar, h->xv, Ns, Np, tau, cx ? h->mean : dtheta_dev, s), "Obar^T x");
  if (cx) CK(launch_unembed(h->mean, Np_c, dtheta_dev, s), "dtheta");
  // a breakdown or a Gram timeout zeroes dtheta on the device and is reported through the
  // status word (peps_last_status)
  CK(launch_minsr_finish(info_dev, h->cfg.gram == 1 ? gerr : nullptr, dtheta_dev, cx ? 2 * Np_c : Np, cx ? 1 : 0,
                         rcond > 0.0 ? 0 : 1, h->sword, s),
     "MinSR finish");
  tstop(h, ts, s, cx ? 4 : 3);
  return PEPS_OK;
}

// ---- sample-sharded MinSR pieces ---------------------------------------------------------
static peps_status check_sharded(peps_handle* h) {
  if (!h) return PEPS_E_ARG;
  if (h->cfg.cplx) return fail(h, PEPS_E_UNSUPPORTED, "sample-sharded MinSR: real PEPS only");
  return PEPS_OK;
}

extern "C" peps_status minsr_partial_sums(peps_handle* h, const void* O_dev, const double* eloc_dev,
                                          const double* w_dev, int Ns, double* sums_dev, void* stream) {
  peps_status ps = check_sharded(h);
  if (ps != PEPS_OK) return ps;
  if (Ns < 0 || !sums_dev || (Ns > 0 && (!O_dev || !eloc_dev))) return fail(h, PEPS_E_ARG, "bad argument");
  cudaStream_t s = (cudaStream_t)stream;
  const int ts = tstart(h, TC_MINSR, s);
  cudaError_t e = (h->esz == 8) ? launch_partial_sums<double>((const double*)O_dev, w_dev, eloc_dev, Ns, h->Np, sums_dev, s)
                                : launch_partial_sums<float>((const float*)O_dev, w_dev, eloc_dev, Ns, h->Np, sums_dev, s);
  if (e != cudaSuccess) return cuda_fail(h, e, "partial sums");
  tstop(h, ts, s, 2);
  return PEPS_OK;
}

extern "C" peps_status minsr_center_rows(peps_handle* h, const void* O_dev, const double* eloc_dev,
                                         const double* w_dev, int Ns, const double* gsums_dev, double* Obar_dev,
                                         double* ebar_dev, void* stream) {
  peps_status ps = check_sharded(h);
  if (ps != PEPS_OK) return ps;
  if (Ns < 0 || !gsums_dev || (Ns > 0 && (!O_dev || !eloc_dev || !Obar_dev || !ebar_dev)))
    return fail(h, PEPS_E_ARG, "bad argument");
  if (Ns == 0) return PEPS_OK;
  cudaStream_t s = (cudaStream_t)stream;
  const int ts = tstart(h, TC_MINSR, s);
  cudaError_t e = (h->esz == 8)
                      ? launch_center_global<double>((const double*)O_dev, w_dev, eloc_dev, Ns, h->Np, gsums_dev,
                                                     Obar_dev, ebar_dev, s)
                      : launch_center_global<float>((const float*)O_dev, w_dev, eloc_dev, Ns, h->Np, gsums_dev,
                                                    Obar_dev, ebar_dev, s);
  if (e != cudaSuccess) return cuda_fail(h, e, "centre rows");
  tstop(h, ts, s, 2);
  return PEPS_OK;
}

extern "C" peps_status minsr_gram(peps_handle* h, const double* A_dev, int Ns, long long K, double* T_dev,
                                  void* stream) {
  peps_status ps = check_sharded(h);
  if (ps != PEPS_OK) return ps;
  if (Ns < 1 || K < 0 || !A_dev || !T_dev) return fail(h, PEPS_E_ARG, "bad argument");
  if ((ps = ensure_minsr(h, Ns, K > 0 ? K : 1)) != PEPS_OK) return ps;
  cudaStream_t s = (cudaStream_t)stream;
  int* gerr = (int*)(h->cnt + 4);
  CK(cudaMemsetAsync(gerr, 0, sizeof(int), s), "memset");
  CK(cudaMemsetAsync(T_dev, 0, sizeof(double) * (size_t)Ns * Ns, s), "memset");
  if (K == 0) return PEPS_OK;
  if ((ps = minsr_gram_into(h, A_dev, Ns, K, T_dev, Ns, true, s)) != PEPS_OK) return ps;
  if (h->cfg.gram == 1) CK(launch_flag_or(gerr, PEPS_SW_GRAM_TIMEOUT, h->sword, s), "status word");
  return PEPS_OK;
}

extern "C" peps_status minsr_solve(peps_handle* h, const double* T_dev, const double* ebar_dev, int Ns, double lambda,
                                   double rcond, double* x_dev, double* info_dev, void* stream) {
  peps_status ps = check_sharded(h);
  if (ps != PEPS_OK) return ps;
  if (!T_dev || !ebar_dev || !x_dev || !info_dev) return fail(h, PEPS_E_ARG, "bad argument");
  if ((ps = check_minsr_args(h, Ns, lambda, rcond)) != PEPS_OK) return ps;
  if ((ps = ensure_minsr(h, Ns, h->ms_np > 0 ? h->ms_np : 1)) != PEPS_OK) return ps;
  cudaStream_t s = (cudaStream_t)stream;
  const int n = Ns + (Ns & 1);
  int ts = tstart(h, TC_MINSR, s);
  CK(cudaMemsetAsync(h->Tm, 0, sizeof(double) * (size_t)n * n, s), "memset");
  CK(cudaMemcpy2DAsync(h->Tm, sizeof(double) * n, T_dev, sizeof(double) * Ns, sizeof(double) * Ns, Ns,
                       cudaMemcpyDeviceToDevice, s), "copy T");
  CK(cudaMemsetAsync(h->ebar, 0, sizeof(double) * n, s), "memset");
  CK(cudaMemcpyAsync(h->ebar, ebar_dev, sizeof(double) * Ns, cudaMemcpyDeviceToDevice, s), "copy ebar");
  tstop(h, ts, s, 4);
  if ((ps = minsr_solve_core(h, Ns, lambda, rcond, info_dev, s)) != PEPS_OK) return ps;
  ts = tstart(h, TC_MINSR, s);
  CK(cudaMemcpyAsync(x_dev, h->xv, sizeof(double) * Ns, cudaMemcpyDeviceToDevice, s), "copy x");
  CK(launch_minsr_finish(info_dev, nullptr, x_dev, Ns, 0, rcond > 0.0 ? 0 : 1, h->sword, s), "MinSR finish");
  tstop(h, ts, s, 3);
  return PEPS_OK;
}

extern "C" peps_status minsr_project(const double* A_dev, const double* x_dev, int Ns, long long K, double tau,
                                     double* dtheta_dev, void* stream) {
  if (Ns < 0 || K < 0 || (K > 0 && (!A_dev || !x_dev || !dtheta_dev))) return PEPS_E_ARG;
  if (K == 0) return PEPS_OK;
  if (launch_obar_t_x(A_dev, x_dev, Ns, K, tau, dtheta_dev, (cudaStream_t)stream) != cudaSuccess) return PEPS_E_CUDA;
  return PEPS_OK;
}

extern "C" peps_status peps_last_status(peps_handle* h, int32_t* word_host, void* stream) {
  if (!h) return PEPS_E_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  int w = 0;
  CK(cudaMemcpyAsync(&w, h->sword, sizeof(int), cudaMemcpyDeviceToHost, s), "read status word");
  CK(cudaMemsetAsync(h->sword, 0, sizeof(int), s), "clear status word");
  CK(cudaStreamSynchronize(s), "status word sync");
  if (word_host) *word_host = w;
  if (w & PEPS_SW_GRAM_TIMEOUT) return fail(h, PEPS_E_CUDA, "tensor-core Gram: a pipeline wait timed out; dtheta set to zero");
  if (w & PEPS_SW_MINSR_BREAKDOWN) {
    h->err = "T + lambda is not positive definite in floating point; dtheta set to zero";
    return PEPS_W_NUMERIC;
  }
  if (w) {
    h->err = "per-sample status bits set";
    return PEPS_W_NUMERIC;
  }
  return PEPS_OK;
}

extern "C" peps_status peps_status_weights(const int32_t* status_dev, int Ns, int mask, double* w_dev, void* stream) {
  if (Ns < 0 || (Ns > 0 && (!status_dev || !w_dev))) return PEPS_E_ARG;
  if (launch_status_weights((const int*)status_dev, Ns, mask, w_dev, (cudaStream_t)stream) != cudaSuccess)
    return PEPS_E_CUDA;
  return PEPS_OK;
}

// ---- autotuner ---------------------------------------------------------------------------
// Per kernel class, the shared-memory budget decides which work buffers stay on chip and how many
// CTAs share an SM; the best choice depends on (chi, D), the lattice and the precision.  Every
// candidate is planned, run once on the caller's configurations and timed with the handle's
// events; each class keeps its fastest budget.
static float class_ms(peps_handle* h, int cls) {
  float tot = 0.f;
  for (size_t k = 0; k < h->evn / 2; ++k) {
    if (h->evclass[k] != cls) continue;
    float ms = 0.f;
    if (cudaEventSynchronize(h->evpool[2 * k + 1]) == cudaSuccess &&
        cudaEventElapsedTime(&ms, h->evpool[2 * k], h->evpool[2 * k + 1]) == cudaSuccess)
      tot += ms;
  }
  return tot;
}

extern "C" peps_status peps_autotune(peps_handle* h, const peps_hamiltonian* H, const uint8_t* S_dev, int Ns,
                                     int move, int* budget_kb_host, void* stream) {
  peps_status c = check_eval(h, S_dev, Ns);
  if (c != PEPS_OK) return c;
  if (Ns < 1) return fail(h, PEPS_E_ARG, "autotune needs at least one configuration");
  if (move != PEPS_MOVE_EXCHANGE && move != PEPS_MOVE_FLIP) return fail(h, PEPS_E_ARG, "bad move kind");
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  std::vector<size_t> cand = (h->esz >= 8) ? std::vector<size_t>{100 * 1024, 210 * 1024}
                                           : std::vector<size_t>{72 * 1024, 110 * 1024, 220 * 1024};
  for (auto& b : cand) b = std::min(b, (size_t)optin - 2048);
  // scratch outputs and a copy of the configurations for the sampler trial
  const size_t N = (size_t)h->g.Lx * h->g.Ly;
  double *la = nullptr, *ph = nullptr, *el = nullptr;
  void* O = nullptr;
  uint8_t* S2 = nullptr;
  long long* acc = nullptr;
  auto cleanup = [&]() {
    void* ps[] = {la, ph, el, O, S2, acc};
    for (void* q : ps)
      if (q) h_free(h, q);
  };
  if (h_malloc(h, (void**)&la, sizeof(double) * Ns) != cudaSuccess ||
      h_malloc(h, (void**)&ph, sizeof(double) * Ns) != cudaSuccess ||
      h_malloc(h, (void**)&el, sizeof(double) * 2 * Ns) != cudaSuccess ||
      h_malloc(h, &O, (size_t)Ns * h->Np * h->esz) != cudaSuccess ||
      h_malloc(h, (void**)&S2, (size_t)Ns * N) != cudaSuccess ||
      h_malloc(h, (void**)&acc, sizeof(long long) * Ns) != cudaSuccess) {
    cleanup();
    return fail(h, PEPS_E_WORKSPACE, "autotune scratch allocation failed");
  }
  const bool was_timing = h->timing;
  const int cls[4] = {TC_ENV, TC_ROW, TC_PAIR, TC_SAMPLE};
  std::vector<std::vector<float>> ms(4, std::vector<float>(cand.size(), 1e30f));
  peps_status st = PEPS_OK;
  for (size_t ci = 0; ci < cand.size() && st == PEPS_OK; ++ci) {
    for (int i = 0; i < 4; ++i) h->budget[i] = cand[ci];
    plan_all(h);
    st = finish_plans(h);
    if (st != PEPS_OK) break;
    for (int rep = 0; rep < 2 && st == PEPS_OK; ++rep) {  // the first repetition warms up
      h->timing = true;
      h->evn = 0;
      st = peps_evaluate(h, H, S_dev, Ns, la, ph, H ? el : nullptr, O, nullptr, stream);
      if (st == PEPS_OK) {
        CK(cudaMemcpyAsync(S2, S_dev, (size_t)Ns * N, cudaMemcpyDeviceToDevice, s), "copy configurations");
        st = peps_sample(h, move, S2, Ns, 1, 0x5eedull, 0, acc, nullptr, stream);
      }
      if (st == PEPS_OK && rep == 1)
        for (int i = 0; i < 4; ++i) ms[i][ci] = class_ms(h, cls[i]);
      h->timing = false;
    }
  }
  h->timing = was_timing;
  h->evn = 0;
  h->rs_gen = -1;
  cleanup();
  if (st != PEPS_OK) {
    for (int i = 0; i < 4; ++i) h->budget[i] = default_budget(h, i);
    plan_all(h);
    finish_plans(h);
    return st;
  }
  for (int i = 0; i < 4; ++i) {
    size_t best = 0;
    for (size_t ci = 1; ci < cand.size(); ++ci)
      if (ms[i][ci] < ms[i][best]) best = ci;
    if (i == 2 && !(H && h->n_pair_terms > 0)) best = 0;  // the pair kernel did not run: keep the smallest
    h->budget[i] = cand[best];
    if (budget_kb_host) budget_kb_host[i] = (int)(cand[best] / 1024);
  }
  plan_all(h);
  return finish_plans(h);
}

// ---- multi-instance batch in one CUDA graph ------------------------------------------------
struct peps_batch {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  void* inst_dev[4] = {nullptr, nullptr, nullptr, nullptr};  // BatchInst<T> arrays, one per scalar type
  char* arena[4] = {nullptr, nullptr, nullptr, nullptr};
  unsigned long long* next = nullptr;                        // 4 queue counters
  size_t budget = 0;
  std::string err;
};
static void batch_free(peps_batch* b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (int k = 0; k < 4; ++k) {
    if (b->inst_dev[k]) cudaFree(b->inst_dev[k]);
    if (b->arena[k]) cudaFree(b->arena[k]);
  }
  if (b->next) cudaFree(b->next);
  delete b;
}

// The environment, one-row and two-row plans of handle h at a shared-memory budget per CTA
// (the handle's own plans are left as they were).
static void plans_at(peps_handle* h, size_t budget, Plan* pe, Plan* pr, Plan* pq, size_t smem[3]) {
  KPlan kp[4] = {h->kp[0], h->kp[1], h->kp[2], h->kp[3]};
  KPlan kb = h->kb;
  size_t bud[4] = {h->budget[0], h->budget[1], h->budget[2], h->budget[3]};
  h->budget[0] = h->budget[1] = h->budget[2] = budget;
  plan_all(h);
  *pe = h->kp[0].p;
  *pr = h->kp[1].p;
  *pq = h->kp[2].p;
  for (int c = 0; c < 3; ++c) smem[c] = h->kp[c].smem;
  for (int c = 0; c < 4; ++c) { h->kp[c] = kp[c]; h->budget[c] = bud[c]; }
  h->kb = kb;
}

// What the graph records for one scalar type's group: the queue launch and the buffers it zeroes
// and reports into.
struct BatchGroup {
  int elem = -1;
  size_t smem = 0;
  int grid = 0;
  int ninst = 0;
  long long nitems = 0;
  std::vector<int*> status;
  std::vector<float*> wdisc;
  std::vector<int> ns;
  std::vector<int*> sword;
};

// Plans, allocations and the descriptor upload of one group (before the capture: nothing here
// may run while a stream is being captured).
template <typename T>
static peps_status batch_prepare(peps_batch* b, const peps_batch_item* items, const std::vector<int>& idx, int elem,
                                 size_t budget, int nsm, BatchGroup* grp) {
  std::vector<BatchInst<T>> inst(idx.size());
  size_t smem = 0, stride = 0;
  long long item0 = 0;
  grp->elem = elem;
  for (size_t k = 0; k < idx.size(); ++k) {
    const peps_batch_item& it = items[idx[k]];
    peps_handle* h = it.h;
    BatchInst<T>& q = inst[k];
    size_t sm[3];
    plans_at(h, budget, &q.pe, &q.pr, &q.pq, sm);
    smem = std::max(smem, std::max(sm[0], std::max(sm[1], sm[2])));
    stride = std::max(stride, (size_t)std::max(q.pe.gstride, std::max(q.pr.gstride, q.pq.gstride)));
    const bool want_e = it.eloc_dev != nullptr;
    q.g = h->g;
    q.Tpad = (const T*)h->Tpad;
    q.S = it.S_dev;
    q.envs = (T*)h->envs;
    q.logs = h->logs;
    q.wdisc = h->wdisc;
    q.O = (T*)it.O_dev;
    q.site_off = h->site_off;
    q.Np = h->Np;
    q.tt = want_e ? h->tt : TermTab{};
    q.dg = want_e ? h->dg : DiagTab{};
    q.rowout = h->rowout;
    q.pairout = h->pairout;
    q.status = it.status_dev ? (int*)it.status_dev : h->status_tmp;
    q.logabs = it.logabs_dev;
    q.phase = it.phase_dev;
    q.eloc = it.eloc_dev;
    q.want_e = want_e ? 1 : 0;
    q.pairs = (want_e && h->n_pair_terms > 0) ? 1 : 0;
    q.sides = (want_e || it.O_dev) ? 3 : 1;
    q.Ns = it.Ns;
    q.item0 = item0;
    item0 += it.Ns;
    grp->status.push_back(q.status);
    grp->wdisc.push_back(q.wdisc);
    grp->ns.push_back(it.Ns);
    grp->sword.push_back(h->sword);
  }
  // one CTA per (SM x resident blocks) at the batch's shared memory; every CTA its arena slice.
  // The kernel's dynamic shared-memory limit is only ever raised (other batches may be recorded
  // with larger budgets); a budget above what an SM offers is a shape error, and its CUDA error
  // is cleared so that later calls do not report it.
  {
    std::lock_guard<std::mutex> lk(g_attr_mu);
    size_t& cur = g_attr_max[{1000 + elem, 0}];
    if (smem > cur) {
      if (kattr_batch<T>(smem, nullptr, 0) != cudaSuccess) {
        cudaGetLastError();
        b->err = "batch kernel: shared memory above the SM's limit";
        return PEPS_E_SHAPE;
      }
      cur = smem;
    }
  }
  int occ = 0;
  if (kattr_batch<T>(0, &occ, smem) != cudaSuccess || occ < 1) {
    cudaGetLastError();
    b->err = "batch kernel does not fit on an SM";
    return PEPS_E_SHAPE;
  }
  const int grid = nsm * occ;
  stride = std::max<size_t>(stride, 256);
  if (cudaMalloc(&b->arena[elem], (size_t)grid * stride) != cudaSuccess) {
    cudaGetLastError();
    return PEPS_E_WORKSPACE;
  }
  for (auto& q : inst) {
    for (Plan* pl : {&q.pe, &q.pr, &q.pq}) {
      pl->gbase = b->arena[elem];
      pl->gstride = stride;
    }
  }
  if (cudaMalloc(&b->inst_dev[elem], sizeof(BatchInst<T>) * inst.size()) != cudaSuccess) {
    cudaGetLastError();
    return PEPS_E_WORKSPACE;
  }
  if (cudaMemcpy(b->inst_dev[elem], inst.data(), sizeof(BatchInst<T>) * inst.size(), cudaMemcpyHostToDevice) !=
      cudaSuccess)
    return PEPS_E_CUDA;
  grp->smem = smem;
  grp->grid = grid;
  grp->ninst = (int)inst.size();
  grp->nitems = item0;
  return PEPS_OK;
}

// Recorded into the graph: zero the queue counter and what the kernels accumulate into, run the
// queue, then fold the status bits into every handle's status word.
template <typename T>
static peps_status batch_record(peps_batch* b, const BatchGroup& grp, cudaStream_t s) {
  if (cudaMemsetAsync(b->next + grp.elem, 0, sizeof(unsigned long long), s) != cudaSuccess) return PEPS_E_CUDA;
  for (int k = 0; k < grp.ninst; ++k)
    if (cudaMemsetAsync(grp.status[k], 0, sizeof(int) * grp.ns[k], s) != cudaSuccess ||
        cudaMemsetAsync(grp.wdisc[k], 0, sizeof(float) * grp.ns[k], s) != cudaSuccess)
      return PEPS_E_CUDA;
  if (launch_batch<T>((const BatchInst<T>*)b->inst_dev[grp.elem], grp.ninst, grp.nitems, b->next + grp.elem, grp.grid,
                      grp.smem, s) != cudaSuccess)
    return PEPS_E_CUDA;
  for (int k = 0; k < grp.ninst; ++k)
    if (launch_status_or(grp.status[k], grp.ns[k], grp.sword[k], s) != cudaSuccess) return PEPS_E_CUDA;
  return PEPS_OK;
}

// FP32: three CTAs per SM, the environment kernels' occupancy; FP64: one
static size_t default_batch_budget(const peps_batch_item* items, int n) {
  for (int i = 0; i < n; ++i)
    if (items[i].h->esz >= 8) return 210 * 1024;
  return 72 * 1024;
}

extern "C" peps_status peps_batch_create_ex(peps_batch** out, const peps_batch_item* items, int n, int budget_kb,
                                            void* stream) {
  if (!out || !items || n < 1 || budget_kb < 0) return PEPS_E_ARG;
  *out = nullptr;
  cudaStream_t s = (cudaStream_t)stream;
  if (!s) return PEPS_E_ARG;  // the legacy default stream cannot be captured
  for (int i = 0; i < n; ++i) {
    const peps_batch_item& it = items[i];
    if (!it.h || it.Ns < 1 || !it.S_dev || !it.logabs_dev || !it.phase_dev) return PEPS_E_ARG;
    if (it.eloc_dev && !it.H) return PEPS_E_ARG;
    if (it.Ns > it.h->cfg.max_samples) return PEPS_E_SHAPE;
    if (it.h->timing) return fail(it.h, PEPS_E_ARG, "disable timing before recording a batch");
    for (int j = 0; j < i; ++j)
      if (items[j].h == it.h) return fail(it.h, PEPS_E_ARG, "a handle appears twice in one batch");
  }
  // one eager pass: uploads the Hamiltonians and every other one-time state
  for (int i = 0; i < n; ++i) {
    const peps_batch_item& it = items[i];
    peps_status st = peps_evaluate(it.h, it.H, it.S_dev, it.Ns, it.logabs_dev, it.phase_dev, it.eloc_dev, it.O_dev,
                                   it.status_dev, stream);
    if (st != PEPS_OK) return st;
  }
  if (cudaStreamSynchronize(s) != cudaSuccess) return PEPS_E_CUDA;
  const size_t budget = budget_kb ? (size_t)budget_kb * 1024 : default_batch_budget(items, n);
  // the queue of each scalar type: the costliest instances first (per-sample work grows as
  // Lx Ly chi^3 D^3), so that the last items are the cheap ones
  std::vector<std::vector<int>> grp(4);
  std::vector<double> cost(n);
  for (int i = 0; i < n; ++i) {
    const Geo& g = items[i].h->g;
    cost[i] = (double)g.Lx * g.Ly * (double)g.chi * g.chi * g.chi * g.D * g.D * g.D;
    grp[items[i].h->elem].push_back(i);
  }
  for (auto& v : grp) std::stable_sort(v.begin(), v.end(), [&](int a, int c) { return cost[a] > cost[c]; });
  peps_batch* b = new peps_batch();
  b->budget = budget;
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (cudaMalloc(&b->next, 4 * sizeof(unsigned long long)) != cudaSuccess) {
    batch_free(b);
    return PEPS_E_WORKSPACE;
  }
  std::vector<BatchGroup> groups;
  peps_status st = PEPS_OK;
  for (int e = 0; e < 4 && st == PEPS_OK; ++e) {
    if (grp[e].empty()) continue;
    groups.emplace_back();
    switch (e) {
      case 0: st = batch_prepare<double>(b, items, grp[e], e, budget, nsm, &groups.back()); break;
      case 1: st = batch_prepare<float>(b, items, grp[e], e, budget, nsm, &groups.back()); break;
      case 2: st = batch_prepare<cplx<double>>(b, items, grp[e], e, budget, nsm, &groups.back()); break;
      default: st = batch_prepare<cplx<float>>(b, items, grp[e], e, budget, nsm, &groups.back()); break;
    }
  }
  if (st != PEPS_OK) {
    if (!b->err.empty()) items[0].h->err = b->err;
    batch_free(b);
    return st;
  }
  if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    batch_free(b);
    return PEPS_E_CUDA;
  }
  for (const BatchGroup& gr : groups) {
    if (st != PEPS_OK) break;
    switch (gr.elem) {
      case 0: st = batch_record<double>(b, gr, s); break;
      case 1: st = batch_record<float>(b, gr, s); break;
      case 2: st = batch_record<cplx<double>>(b, gr, s); break;
      default: st = batch_record<cplx<float>>(b, gr, s); break;
    }
  }
  cudaGraph_t graph = nullptr;
  const cudaError_t ec = cudaStreamEndCapture(s, &graph);
  b->graph = graph;
  if (st != PEPS_OK || ec != cudaSuccess || !graph || cudaGraphInstantiate(&b->exec, graph, 0) != cudaSuccess) {
    if (st != PEPS_OK && !b->err.empty()) items[0].h->err = b->err;
    batch_free(b);
    return st != PEPS_OK ? st : PEPS_E_CUDA;
  }
  *out = b;
  return PEPS_OK;
}

extern "C" peps_status peps_batch_create(peps_batch** out, const peps_batch_item* items, int n, int nbranch,
                                         void* stream) {
  (void)nbranch;
  return peps_batch_create_ex(out, items, n, 0, stream);
}

extern "C" peps_status peps_batch_launch(peps_batch* b, void* stream) {
  if (!b || !b->exec) return PEPS_E_ARG;
  return cudaGraphLaunch(b->exec, (cudaStream_t)stream) == cudaSuccess ? PEPS_OK : PEPS_E_CUDA;
}

// Batch autotuner: the shared-memory budget per CTA decides which work buffers of every
// instance stay on chip and how many CTAs share an SM (the batch kernel's tile of work per SM);
// each candidate batch is recorded, launched and timed, the fastest budget kept.
extern "C" peps_status peps_batch_autotune(const peps_batch_item* items, int n, int* budget_kb_host, void* stream) {
  if (!items || n < 1 || !budget_kb_host) return PEPS_E_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  bool fp64 = false;
  for (int i = 0; i < n; ++i) fp64 = fp64 || items[i].h->esz >= 8;
  const std::vector<int> cand = fp64 ? std::vector<int>{100, 210} : std::vector<int>{56, 72, 110, 220};
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  int best_kb = 0;
  peps_status st = PEPS_OK;
  for (int kb : cand) {
    peps_batch* b = nullptr;
    st = peps_batch_create_ex(&b, items, n, kb, stream);
    if (st == PEPS_E_SHAPE) { st = PEPS_OK; continue; }  // this budget does not fit
    if (st != PEPS_OK) break;
    float ms = 0.f;
    if (cudaGraphLaunch(b->exec, s) != cudaSuccess || cudaEventRecord(e0, s) != cudaSuccess ||
        cudaGraphLaunch(b->exec, s) != cudaSuccess || cudaEventRecord(e1, s) != cudaSuccess ||
        cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
      batch_free(b);
      st = PEPS_E_CUDA;
      break;
    }
    batch_free(b);
    if (ms < best) { best = ms; best_kb = kb; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st == PEPS_OK && best_kb == 0) st = PEPS_E_SHAPE;
  *budget_kb_host = best_kb;
  return st;
}

extern "C" peps_status peps_batch_destroy(peps_batch* b) {
  if (!b) return PEPS_E_ARG;
  batch_free(b);
  return PEPS_OK;
}

// ---- timing and work counters ----------------------------------------------------------
extern "C" peps_status peps_timing_enable(peps_handle* h, int enable) {
  if (!h) return PEPS_E_ARG;
  h->timing = (enable != 0);
  h->evn = 0;
  if (h->ctr) CK(cudaMemset(h->ctr, 0, 8 * sizeof(unsigned long long)), "reset counters");
  return PEPS_OK;
}

extern "C" peps_status peps_timing_read(peps_handle* h, double* ms_host, long long* launches_host, int n,
                                        long long* counters_host) {
  if (!h || n < 0 || (n > 0 && (!ms_host || !launches_host))) return PEPS_E_ARG;
  for (int i = 0; i < n; ++i) { ms_host[i] = 0.0; launches_host[i] = 0; }
  for (size_t k = 0; k < h->evn / 2; ++k) {
    CK(cudaEventSynchronize(h->evpool[2 * k + 1]), "event sync");
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, h->evpool[2 * k], h->evpool[2 * k + 1]), "event time");
    const int c = h->evclass[k];
    if (c < n) { ms_host[c] += ms; launches_host[c] += h->evlaunches[k]; }
  }
  if (counters_host) {
    unsigned long long c[8];
    CK(cudaMemcpy(c, h->ctr, sizeof(c), cudaMemcpyDeviceToHost), "read counters");
    for (int i = 0; i < 4; ++i) counters_host[i] = (long long)c[i];
  }
  return PEPS_OK;
}

// ---- parameter update --------------------------------------------------------------------
extern "C" peps_status peps_apply_update(peps_handle* h, double* theta_dev, const double* dtheta_dev, void* stream) {
  if (!h || !theta_dev || !dtheta_dev) return fail(h, PEPS_E_ARG, "null argument");
  cudaStream_t s = (cudaStream_t)stream;
  const int ts = tstart(h, TC_PAD, s);
  CK(launch_axpy(theta_dev, dtheta_dev, h->Np * (h->cfg.cplx ? 2 : 1), s), "theta update");
  tstop(h, ts, s);
  return peps_set_params(h, theta_dev, stream);
}

// ---- learned proposal --------------------------------------------------------------------
static bool prop_shape_ok(int Lx, int Ly, int C, int wprec) {
  if (Lx < 1 || Ly < 1 || Lx * Ly > 256 || C < 1 || C > 32 || (wprec != 0 && wprec != 1)) return false;
  return prop_smem_bytes(Lx, Ly, C, wprec == 0 ? 8 : 4, true) <= 220 * 1024;
}

static int prop_grid(int Ns) {
  int dev = 0, nsm = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  return Ns < nsm ? (Ns > 0 ? Ns : 1) : nsm;
}

extern "C" peps_status peps_proposal_logits(int Lx, int Ly, int C, int wprec, const void* w_dev, const uint8_t* S_dev,
                                            int Ns, double* logits_dev, void* stream) {
  if (!prop_shape_ok(Lx, Ly, C, wprec)) return PEPS_E_SHAPE;
  if (Ns < 0 || (Ns > 0 && (!w_dev || !S_dev || !logits_dev))) return PEPS_E_ARG;
  if (Ns == 0) return PEPS_OK;
  cudaError_t e = launch_prop_logits(Lx, Ly, C, wprec, w_dev, S_dev, Ns, logits_dev, prop_grid(Ns), (cudaStream_t)stream);
  return e == cudaSuccess ? PEPS_OK : PEPS_E_CUDA;
}

extern "C" peps_status peps_proposal_train_step(int Lx, int Ly, int C, int wprec, double* w_dev, double* m_dev,
                                                double* v_dev, void* wlow_dev, int t, double lr,
                                                const uint8_t* S_in_dev, const uint8_t* S_tgt_dev, int Ns,
                                                double* grad_dev, double* loss_dev, void* stream) {
  if (!prop_shape_ok(Lx, Ly, C, wprec)) return PEPS_E_SHAPE;
  if (!w_dev || !m_dev || !v_dev || !grad_dev || !loss_dev || t < 1 || Ns < 1 || !S_in_dev || !S_tgt_dev ||
      (wprec == 1 && !wlow_dev))
    return PEPS_E_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const int nw = 9 * C * C + 20 * C + 1;
  if (cudaMemsetAsync(grad_dev, 0, sizeof(double) * nw, s) != cudaSuccess) return PEPS_E_CUDA;
  if (cudaMemsetAsync(loss_dev, 0, sizeof(double), s) != cudaSuccess) return PEPS_E_CUDA;
  const void* wf = (wprec == 0) ? (const void*)w_dev : (const void*)wlow_dev;
  if (launch_prop_grad(Lx, Ly, C, wprec, wf, S_in_dev, S_tgt_dev, Ns, grad_dev, loss_dev, prop_grid(Ns), s) != cudaSuccess)
    return PEPS_E_CUDA;
  if (launch_prop_adam(nw, w_dev, m_dev, v_dev, grad_dev, t, lr, wlow_dev, s) != cudaSuccess) return PEPS_E_CUDA;
  return PEPS_OK;
}

static peps_status ensure_learned(peps_handle* h) {
  if (h->lp_Sp) return PEPS_OK;
  const size_t ns = (size_t)h->cfg.max_samples, N = (size_t)h->g.Lx * h->g.Ly;
  if (h_malloc(h, (void**)&h->lp_Sp, ns * N) != cudaSuccess || h_malloc(h, (void**)&h->lp_l0, sizeof(double) * ns * N) != cudaSuccess ||
      h_malloc(h, (void**)&h->lp_l1, sizeof(double) * ns * N) != cudaSuccess ||
      h_malloc(h, (void**)&h->lp_aux, sizeof(double) * ns * 4) != cudaSuccess)
    return fail(h, PEPS_E_WORKSPACE, "learned-proposal workspace allocation failed");
  return PEPS_OK;
}

extern "C" peps_status peps_sample_learned(peps_handle* h, int C, int wprec, const void* w_dev, uint8_t* S_dev,
                                           double* logpsi_dev, int Ns, uint64_t seed, uint64_t step,
                                           long long* accepted_dev, int32_t* status_dev, void* stream) {
  if (h) h->rs_gen = -1;  // S_dev is overwritten
  peps_status c = check_eval(h, S_dev, Ns);
  if (c != PEPS_OK) return c;
  if (!prop_shape_ok(h->g.Lx, h->g.Ly, C, wprec)) return fail(h, PEPS_E_SHAPE, "proposal network shape");
  if (Ns > 0 && (!w_dev || !logpsi_dev)) return fail(h, PEPS_E_ARG, "null argument");
  if (h->cfg.cplx) return fail(h, PEPS_E_UNSUPPORTED, "learned proposal: real PEPS only");
  if (Ns == 0) return PEPS_OK;
  peps_status ps = ensure_learned(h);
  if (ps != PEPS_OK) return ps;
  cudaStream_t s = (cudaStream_t)stream;
  const int N = h->g.Lx * h->g.Ly;
  double* lq_f = h->lp_aux;
  double* lq_b = h->lp_aux + Ns;
  double* lpsi_new = h->lp_aux + 2 * (size_t)Ns;
  double* ph_new = h->lp_aux + 3 * (size_t)Ns;
  const int ts = tstart(h, TC_SAMPLE, s);
  CK(launch_prop_logits(h->g.Lx, h->g.Ly, C, wprec, w_dev, S_dev, Ns, h->lp_l0, prop_grid(Ns), s), "proposal logits");
  CK(launch_prop_draw(N, Ns, h->lp_l0, seed, step, h->lp_Sp, lq_f, s), "proposal draw");
  CK(launch_prop_logits(h->g.Lx, h->g.Ly, C, wprec, w_dev, h->lp_Sp, Ns, h->lp_l1, prop_grid(Ns), s), "proposal logits");
  CK(launch_prop_logq(N, Ns, h->lp_l1, S_dev, lq_b, s), "proposal log q");
  tstop(h, ts, s, 4);
  ps = (h->esz == 8) ? run_eval<double>(h, nullptr, h->lp_Sp, Ns, lpsi_new, ph_new, nullptr, nullptr, status_dev, s, 1)
                     : run_eval<float>(h, nullptr, h->lp_Sp, Ns, lpsi_new, ph_new, nullptr, nullptr, status_dev, s, 1);
  if (ps != PEPS_OK) return ps;
  const int ts2 = tstart(h, TC_SAMPLE, s);
  CK(launch_prop_accept(N, Ns, seed, step, h->lp_Sp, lpsi_new, lq_f, lq_b, S_dev, logpsi_dev, accepted_dev, s),
     "proposal accept");
  tstop(h, ts2, s);
  return PEPS_OK;
}

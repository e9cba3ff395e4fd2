// Contraction kernels of the finite-PEPS hot path (sm_103a): environment pass, one- and two-row
// sandwiches (amplitudes, local-energy ratios, log-derivatives), per-sample combine, and the
// Metropolis sweep.  All kernels are persistent: each CTA loops over work items
// (blockIdx.x, blockIdx.x + gridDim.x, ...) and owns one slice of the global scratch arena.
// Included by peps_kernels_f64.cu and peps_kernels_f32.cu, which instantiate it for one real
// type each (two translation units compile in parallel).
#pragma once
#include "peps_kernels.cuh"

namespace peps {

// ------------------------------------------------------------------------------------------
// environment store: per sample 2*Lx rows of Ly sites; slot x+1 holds E^u[x] (x = -1..Lx-2),
// slot Lx+x-1 holds E^l[x] (x = 1..Lx).  logs: cumulative log factor of every slot.
template <typename G>
__host__ __device__ inline size_t env_sample_elems(const G& g) { return (size_t)2 * g.Lx * g.Ly * g.se; }
template <typename G>
__device__ inline int slot_up(const G& g, int x) { return x + 1; }
template <typename G>
__device__ inline int slot_lo(const G& g, int x) { return g.Lx + x - 1; }

template <typename T>
__device__ RowWork<T> carve_row(const Plan& p, char* smem, char* gbase) {
  RowWork<T> w;
  w.R = (T*)buf_ptr(p, B_R, smem, gbase);
  w.Rhist = (T*)buf_ptr(p, B_RHIST, smem, gbase);
  w.E = (T*)buf_ptr(p, B_E, smem, gbase);
  w.A = (T*)buf_ptr(p, B_A, smem, gbase);
  w.Z = (T*)buf_ptr(p, B_Z, smem, gbase);
  w.W = (T*)buf_ptr(p, B_W, smem, gbase);
  w.C = (T*)buf_ptr(p, B_C, smem, gbase);
  w.sig = (T*)buf_ptr(p, B_SIG, smem, gbase);
  w.sel = (int*)buf_ptr(p, B_SEL, smem, gbase);
  w.red = (double*)buf_ptr(p, B_RED, smem, gbase);
  w.ci = p.ci;
  w.ctr = p.ctr;
  return w;
}

// Upper environments E^u[-1..Lx-2] of configuration Ss into env (one sample's store).
template <typename T, typename G>
__device__ void build_upper(const G& g, const T* Tpad, const uint8_t* Ss, T* env, double* logs,
                            const RowWork<T>& w, int* st, float* wd, int* flag) {
  const size_t row = (size_t)g.Ly * g.se;
  // trivial E^u[-1], and the trivial E^l[Lx] that closes psi_top = E^u[Lx-2] . T_proj[Lx-1]
  T* trivial = env + (size_t)slot_up(g, -1) * row;
  T* trivial_lo = env + (size_t)slot_lo(g, g.Lx) * row;
  for (int k = 0; k < g.Ly; ++k) {
    blk_unit(trivial + (size_t)k * g.se, g.se);
    blk_unit(trivial_lo + (size_t)k * g.se, g.se);
  }
  if (threadIdx.x == 0) { logs[slot_up(g, -1)] = 0.0; logs[slot_lo(g, g.Lx)] = 0.0; }
  __syncthreads();
  double lg = env_first_row(g, env + (size_t)slot_up(g, 0) * row, Tpad, 0, Ss, false, w.A, w.Z, w.red, st);
  if (threadIdx.x == 0) logs[slot_up(g, 0)] = lg;
  for (int x = 1; x <= g.Lx - 2; ++x) {
    lg += env_row_step(g, env + (size_t)slot_up(g, x - 1) * row, env + (size_t)slot_up(g, x) * row, Tpad, x,
                       Ss + (size_t)x * g.Ly, false, w, st, wd, flag);
    if (threadIdx.x == 0) logs[slot_up(g, x)] = lg;
  }
  __syncthreads();
}

// Lower environments E^l[2..Lx] (and E^l[1] when full) of configuration Ss.
template <typename T, typename G>
__device__ void build_lower(const G& g, const T* Tpad, const uint8_t* Ss, T* env, double* logs,
                            const RowWork<T>& w, int* st, float* wd, int* flag, int xmin) {
  const size_t row = (size_t)g.Ly * g.se;
  T* trivial = env + (size_t)slot_lo(g, g.Lx) * row;
  for (int k = 0; k < g.Ly; ++k) blk_unit(trivial + (size_t)k * g.se, g.se);
  if (threadIdx.x == 0) logs[slot_lo(g, g.Lx)] = 0.0;
  __syncthreads();
  double lg = env_first_row(g, env + (size_t)slot_lo(g, g.Lx - 1) * row, Tpad, g.Lx - 1,
                            Ss + (size_t)(g.Lx - 1) * g.Ly, true, w.A, w.Z, w.red, st);
  if (threadIdx.x == 0) logs[slot_lo(g, g.Lx - 1)] = lg;
  for (int x = g.Lx - 2; x >= xmin; --x) {
    lg += env_row_step(g, env + (size_t)slot_lo(g, x + 1) * row, env + (size_t)slot_lo(g, x) * row, Tpad, x,
                       Ss + (size_t)x * g.Ly, true, w, st, wd, flag);
    if (threadIdx.x == 0) logs[slot_lo(g, x)] = lg;
  }
  __syncthreads();
}

// One side (0 upper, 1 lower) of sample smp's environments, with the whole CTA.
template <typename T, typename G>
__device__ __forceinline__ void env_item(const G g, const RowWork<T>& w, const T* __restrict__ Tpad,
                                         const uint8_t* __restrict__ S,
                         int smp, int side, T* envs, double* logs, int* status, float* wdisc) {
  __shared__ int st, flag;
  __shared__ float wd;
  const int N = g.Lx * g.Ly;
  if (threadIdx.x == 0) { st = 0; wd = 0.f; }
  __syncthreads();
  T* env = envs + (size_t)smp * env_sample_elems(g);
  double* lg = logs + (size_t)smp * 2 * g.Lx;
  const uint8_t* Ss = S + (size_t)smp * N;
  if (side == 0) build_upper(g, Tpad, Ss, env, lg, w, &st, &wd, &flag);
  else build_lower(g, Tpad, Ss, env, lg, w, &st, &wd, &flag, 1);
  if (threadIdx.x == 0) {
    if (st) atomicOr(status + smp, st);
    if (wdisc) atomicMax((int*)(wdisc + smp), __float_as_int(wd));  // wd >= 0: int order = float order
  }
  __syncthreads();
}

template <typename T, typename G>
__global__ void __launch_bounds__(NTHREADS, EnvBlocks<T>::value) k_env(G g, Plan plan, const T* __restrict__ Tpad,
                                                  const uint8_t* __restrict__ S, int Ns, int sides, T* envs,
                                                  double* logs, int* status, float* wdisc) {
  extern __shared__ __align__(16) char smem[];
  RowWork<T> w = carve_row<T>(plan, smem, plan.gbase);
  const int nside = (sides == 3) ? 2 : 1;
  for (int item = blockIdx.x; item < Ns * nside; item += gridDim.x) {
    const int smp = item / nside;
    const int side = (sides == 3) ? (item % nside) : (sides == 1 ? 0 : 1);
    env_item(g, w, Tpad, S, smp, side, envs, logs, status, wdisc);
  }
}

// ------------------------------------------------------------------------------------------
// Sandwich bookkeeping shared by the row and pair kernels.
template <typename G>
__device__ inline void site_dims(const G& g, int x, int y, int* Dl, int* Du, int* Dr, int* Dd) {
  *Dl = (y == 0) ? 1 : g.D;
  *Du = (x == 0) ? 1 : g.D;
  *Dr = (y == g.Ly - 1) ? 1 : g.D;
  *Dd = (x == g.Lx - 1) ? 1 : g.D;
}

// local state of `site` in configuration Ss after replacing the term's sites by the digits of b
__device__ inline int state_after(const int* ti, int site, const uint8_t* Ss, int b, int d) {
  const int k = ti[TI_K];
  int pw = 1;
  for (int t = k - 1; t >= 0; --t) {
    if (ti[TI_S0 + t] == site) return (b / pw) % d;
    pw *= d;
  }
  return Ss[site];
}

__device__ inline int local_index(const int* ti, const uint8_t* Ss, int d) {
  int a = 0;
  for (int t = 0; t < ti[TI_K]; ++t) a = a * d + Ss[ti[TI_S0 + t]];
  return a;
}

// ------------------------------------------------------------------------------------------
// One-row sandwich at row x of sample smp: psi_x, O of row x, E_loc terms inside row x.
// One-row sandwich at row x of sample smp, with the whole CTA.
template <typename T, typename G>
__device__ __forceinline__ void row_item(const G g, const Plan plan, char* smem, const T* __restrict__ Tpad,
                                         const uint8_t* __restrict__ S, int smp, int x, const T* envs,
                                         const double* logs, T* O, const long long* site_off, long long Np,
                                         const TermTab tt, double* rowout, int* status) {
  char* gbase = plan.gbase;
  T* LP = (T*)buf_ptr(plan, B_LP, smem, gbase);   // (Ly+1) x se
  T* RP = (T*)buf_ptr(plan, B_RP, smem, gbase);   // (Ly+1) x se
  T* t1 = (T*)buf_ptr(plan, B_T1, smem, gbase);
  T* t2 = (T*)buf_ptr(plan, B_T2, smem, gbase);
  T* eu = (T*)buf_ptr(plan, B_EU, smem, gbase);
  T* el = (T*)buf_ptr(plan, B_EL, smem, gbase);
  T* A = (T*)buf_ptr(plan, B_A, smem, gbase);
  T* LW = (T*)buf_ptr(plan, B_LW, smem, gbase);
  T* LW2 = (T*)buf_ptr(plan, B_LW2, smem, gbase);
  double* red = (double*)buf_ptr(plan, B_RED, smem, gbase);
  __shared__ double logL[MAX_LY + 1], logR[MAX_LY + 1];
  __shared__ int st;
  const int N = g.Lx * g.Ly, Ly = g.Ly, se = g.se;
  const size_t rowsz = (size_t)Ly * se;
  const uint8_t* Ss = S + (size_t)smp * N;
  const T* env = envs + (size_t)smp * env_sample_elems(g);
  const double* lg = logs + (size_t)smp * 2 * g.Lx;
  const T* EU = env + (size_t)slot_up(g, x - 1) * rowsz;
  const T* EL = env + (size_t)slot_lo(g, x + 1) * rowsz;
  if (threadIdx.x == 0) st = 0;
  // right partials R[Ly] = unit, R[y] = R[y+1] absorbed over column y
  blk_unit(RP + (size_t)Ly * se, se);
  if (threadIdx.x == 0) logR[Ly] = 0.0;
  __syncthreads();
  for (int y = Ly - 1; y >= 0; --y) {
    blk_copy(eu, EU + (size_t)y * se, se);
    blk_copy(el, EL + (size_t)y * se, se);
    load_A(A, Tpad, g, x * Ly + y, Ss[x * Ly + y], false);
    __syncthreads();
    absorb1_right(g, RP + (size_t)(y + 1) * se, eu, A, el, t1, t2, RP + (size_t)y * se);
    const double l = blk_normalize(RP + (size_t)y * se, se, red, &st);
    if (threadIdx.x == 0) logR[y] = logR[y + 1] + l;
  }
  // left partials
  blk_unit(LP, se);
  if (threadIdx.x == 0) logL[0] = 0.0;
  __syncthreads();
  for (int y = 0; y < Ly; ++y) {
    blk_copy(eu, EU + (size_t)y * se, se);
    blk_copy(el, EL + (size_t)y * se, se);
    load_A(A, Tpad, g, x * Ly + y, Ss[x * Ly + y], false);
    __syncthreads();
    absorb1(g, LP + (size_t)y * se, eu, A, el, t1, t2, LP + (size_t)(y + 1) * se);
    const double l = blk_normalize(LP + (size_t)(y + 1) * se, se, red, &st);
    if (threadIdx.x == 0) logL[y + 1] = logL[y] + l;
  }
  __syncthreads();
  const T val = LP[(size_t)Ly * se];
  const double lpsi_norm = logL[Ly];
  const double env_log = lg[slot_up(g, x - 1)] + lg[slot_lo(g, x + 1)];
  // ---- log-derivatives of row x
  if (O != nullptr) {
    for (int y = 0; y < Ly; ++y) {
      const int site = x * Ly + y;
      blk_copy(eu, EU + (size_t)y * se, se);
      {
        // the lower environment site transposed, elT[z][b][d] = el[b][d][z] (into LW2)
        const T* ely = EL + (size_t)y * se;
        const int cd = g.chi * g.D;
        for (int o = threadIdx.x; o < se; o += blockDim.x) LW2[o] = ely[(size_t)(o % cd) * g.chi + o / cd];
      }
      __syncthreads();
      site_env1(g, LP + (size_t)y * se, eu, LW2, RP + (size_t)(y + 1) * se, t1, t2, A);
      const double sc = exp(logL[y] + logR[y + 1] - lpsi_norm);
      int Dl, Du, Dr, Dd;
      site_dims(g, x, y, &Dl, &Du, &Dr, &Dd);
      const int blk = Dl * Du * Dr * Dd;
      const int s_here = Ss[site];
      T* Orow = O + (size_t)smp * Np + site_off[site];
      const int D = g.D;
      for (int o = threadIdx.x; o < g.d * blk; o += blockDim.x) {
        const int s = o / blk, c = o % blk;
        const int dd = c % Dd, r = (c / Dd) % Dr, u = (c / (Dd * Dr)) % Du, l = c / (Dd * Dr * Du);
        T v = T(0);
        if (s == s_here) {
          const dz e = to_dz(A[((l * D + u) * D + r) * D + dd]);
          v = from_dz<T>(dz_div(dz{e.re * sc, e.im * sc}, to_dz(val)));
        }
        Orow[o] = v;
      }
      __syncthreads();
    }
  }
  // ---- local-energy terms inside row x
  double ere = 0.0, eim = 0.0;
  if (tt.nterm > 0) {
    for (int ti_ = tt.row_off[x]; ti_ < tt.row_off[x + 1]; ++ti_) {
      const int* ti = tt.tinfo + (size_t)ti_ * TI_N;
      const int a = local_index(ti, Ss, g.d);
      for (int e = ti[TI_EOFF]; e < ti[TI_EOFF] + ti[TI_ECNT]; ++e) {
        if (tt.ent_ab[2 * e] != a) continue;
        const int b = tt.ent_ab[2 * e + 1];
        const double hr = tt.ent_h[2 * e], hi = tt.ent_h[2 * e + 1];
        if (b == a) { ere += hr; eim += hi; continue; }
        const int y0 = ti[TI_Y0], w = ti[TI_W];
        blk_copy(LW, LP + (size_t)y0 * se, se);
        double lw = logL[y0];
        __syncthreads();
        for (int c = y0; c < y0 + w; ++c) {
          const int site = x * Ly + c;
          blk_copy(eu, EU + (size_t)c * se, se);
          blk_copy(el, EL + (size_t)c * se, se);
          load_A(A, Tpad, g, site, state_after(ti, site, Ss, b, g.d), false);
          __syncthreads();
          absorb1(g, LW, eu, A, el, t1, t2, LW2);
          lw += blk_normalize(LW2, se, red, &st);
          blk_copy(LW, LW2, se);
          __syncthreads();
        }
        const T v = blk_dot(LW, RP + (size_t)(y0 + w) * se, se, red);
        lw += logR[y0 + w];
        const dz q = dz_div(to_dz(v), to_dz(val));
        const double f = exp(lw - lpsi_norm);
        ere += (hr * q.re - hi * q.im) * f;
        eim += (hr * q.im + hi * q.re) * f;
      }
    }
  }
  if (threadIdx.x == 0) {
    double* out = rowout + ((size_t)smp * g.Lx + x) * 4;
    const dz vz = to_dz(val);
    const double av = dz_abs(vz);
    out[0] = (av > 0.0) ? log(av) + lpsi_norm + env_log : -INFINITY;
    out[1] = (vz.im == 0.0) ? ((vz.re < 0.0) ? 3.141592653589793 : 0.0) : atan2(vz.im, vz.re);
    out[2] = ere;
    out[3] = eim;
    int s = st;
    if (!(av > 0.0) || !isfinite(out[0]) || !isfinite(ere) || !isfinite(eim)) s |= ST_NONFINITE;
    if (s) atomicOr(status + smp, s);
  }
  __syncthreads();
}

template <typename T, typename G>
__global__ void __launch_bounds__(NTHREADS, EnvBlocks<T>::value) k_row(G g, Plan plan, const T* __restrict__ Tpad,
                                                  const uint8_t* __restrict__ S, int Ns, int x_lo, int x_hi,
                                                  const T* envs, const double* logs, T* O, const long long* site_off,
                                                  long long Np, TermTab tt, double* rowout, int* status) {
  extern __shared__ __align__(16) char smem[];
  const int nx = x_hi - x_lo;
  for (int item = blockIdx.x; item < Ns * nx; item += gridDim.x)
    row_item(g, plan, smem, Tpad, S, item / nx, x_lo + item % nx, envs, logs, O, site_off, Np, tt, rowout, status);
}

// ------------------------------------------------------------------------------------------
// Two-row sandwich at rows x, x+1: psi_{x,x+1} and the E_loc terms spanning the two rows.
// Two-row sandwich at rows x, x+1 of sample smp, with the whole CTA.
template <typename T, typename G>
__device__ __forceinline__ void pair_item(const G g, const Plan plan, char* smem, const T* __restrict__ Tpad,
                                          const uint8_t* __restrict__ S, int smp, int x, const T* envs,
                                          const double* logs, const TermTab tt, double* pairout, int* status) {
  char* gbase = plan.gbase;
  T* LP = (T*)buf_ptr(plan, B_LP, smem, gbase);   // (Ly+1) x s2
  T* RP = (T*)buf_ptr(plan, B_RP, smem, gbase);   // (Ly+1) x s2
  T* t1 = (T*)buf_ptr(plan, B_T1, smem, gbase);
  T* t2 = (T*)buf_ptr(plan, B_T2, smem, gbase);
  T* eu = (T*)buf_ptr(plan, B_EU, smem, gbase);
  T* el = (T*)buf_ptr(plan, B_EL, smem, gbase);
  T* A1 = (T*)buf_ptr(plan, B_A, smem, gbase);
  T* A2 = (T*)buf_ptr(plan, B_A2, smem, gbase);
  T* LW = (T*)buf_ptr(plan, B_LW, smem, gbase);
  T* LW2 = (T*)buf_ptr(plan, B_LW2, smem, gbase);
  double* red = (double*)buf_ptr(plan, B_RED, smem, gbase);
  __shared__ double logL[MAX_LY + 1], logR[MAX_LY + 1];
  __shared__ int st;
  const int N = g.Lx * g.Ly, Ly = g.Ly, se = g.se, s2 = g.s2;
  const size_t rowsz = (size_t)Ly * se;
  // skip row pairs without terms
  if (tt.nterm == 0 || tt.pair_off[x] == tt.pair_off[x + 1]) {
    if (threadIdx.x == 0) {
      double* out = pairout + ((size_t)smp * g.Lx + x) * 4;
      out[0] = 0.0; out[1] = 0.0; out[2] = 0.0; out[3] = 0.0;
    }
    return;
  }
  const uint8_t* Ss = S + (size_t)smp * N;
  const T* env = envs + (size_t)smp * env_sample_elems(g);
  const T* EU = env + (size_t)slot_up(g, x - 1) * rowsz;
  const T* EL = env + (size_t)slot_lo(g, x + 2) * rowsz;
  if (threadIdx.x == 0) st = 0;
  blk_unit(RP + (size_t)Ly * s2, s2);
  if (threadIdx.x == 0) logR[Ly] = 0.0;
  __syncthreads();
  for (int y = Ly - 1; y >= 0; --y) {
    blk_copy(eu, EU + (size_t)y * se, se);
    blk_copy(el, EL + (size_t)y * se, se);
    load_A(A1, Tpad, g, x * Ly + y, Ss[x * Ly + y], false);
    load_A(A2, Tpad, g, (x + 1) * Ly + y, Ss[(x + 1) * Ly + y], false);
    __syncthreads();
    absorb2_right(g, RP + (size_t)(y + 1) * s2, eu, A1, A2, el, t1, t2, RP + (size_t)y * s2, plan.cx);
    const double l = blk_normalize(RP + (size_t)y * s2, s2, red, &st);
    if (threadIdx.x == 0) logR[y] = logR[y + 1] + l;
  }
  blk_unit(LP, s2);
  if (threadIdx.x == 0) logL[0] = 0.0;
  __syncthreads();
  // the left partials are only needed up to the last window start; build them all
  for (int y = 0; y < Ly; ++y) {
    blk_copy(eu, EU + (size_t)y * se, se);
    blk_copy(el, EL + (size_t)y * se, se);
    load_A(A1, Tpad, g, x * Ly + y, Ss[x * Ly + y], false);
    load_A(A2, Tpad, g, (x + 1) * Ly + y, Ss[(x + 1) * Ly + y], false);
    __syncthreads();
    absorb2(g, LP + (size_t)y * s2, eu, A1, A2, el, t1, t2, LP + (size_t)(y + 1) * s2, plan.cx);
    const double l = blk_normalize(LP + (size_t)(y + 1) * s2, s2, red, &st);
    if (threadIdx.x == 0) logL[y + 1] = logL[y] + l;
  }
  __syncthreads();
  const T val = LP[(size_t)Ly * s2];
  const double lpsi_norm = logL[Ly];
  double ere = 0.0, eim = 0.0;
  for (int ti_ = tt.pair_off[x]; ti_ < tt.pair_off[x + 1]; ++ti_) {
    const int* ti = tt.tinfo + (size_t)ti_ * TI_N;
    const int a = local_index(ti, Ss, g.d);
    for (int e = ti[TI_EOFF]; e < ti[TI_EOFF] + ti[TI_ECNT]; ++e) {
      if (tt.ent_ab[2 * e] != a) continue;
      const int b = tt.ent_ab[2 * e + 1];
      const double hr = tt.ent_h[2 * e], hi = tt.ent_h[2 * e + 1];
      if (b == a) { ere += hr; eim += hi; continue; }
      const int y0 = ti[TI_Y0], w = ti[TI_W];
      blk_copy(LW, LP + (size_t)y0 * s2, s2);
      double lw = logL[y0];
      __syncthreads();
      for (int c = y0; c < y0 + w; ++c) {
        blk_copy(eu, EU + (size_t)c * se, se);
        blk_copy(el, EL + (size_t)c * se, se);
        load_A(A1, Tpad, g, x * Ly + c, state_after(ti, x * Ly + c, Ss, b, g.d), false);
        load_A(A2, Tpad, g, (x + 1) * Ly + c, state_after(ti, (x + 1) * Ly + c, Ss, b, g.d), false);
        __syncthreads();
        absorb2(g, LW, eu, A1, A2, el, t1, t2, LW2, plan.cx);
        lw += blk_normalize(LW2, s2, red, &st);
        blk_copy(LW, LW2, s2);
        __syncthreads();
      }
      const T v = blk_dot(LW, RP + (size_t)(y0 + w) * s2, s2, red);
      lw += logR[y0 + w];
      const dz q = dz_div(to_dz(v), to_dz(val));
      const double f = exp(lw - lpsi_norm);
      ere += (hr * q.re - hi * q.im) * f;
      eim += (hr * q.im + hi * q.re) * f;
    }
  }
  if (threadIdx.x == 0) {
    double* out = pairout + ((size_t)smp * g.Lx + x) * 4;
    out[0] = 0.0;
    out[1] = 0.0;
    out[2] = ere;
    out[3] = eim;
    int s = st;
    if (!(dz_abs(to_dz(val)) != 0.0) || !isfinite(ere) || !isfinite(eim)) s |= ST_NONFINITE;
    if (s) atomicOr(status + smp, s);
  }
  __syncthreads();
}

template <typename T, typename G>
__global__ void __launch_bounds__(NTHREADS) k_pair(G g, Plan plan, const T* __restrict__ Tpad,
                                                   const uint8_t* __restrict__ S, int Ns, const T* envs,
                                                   const double* logs, TermTab tt, double* pairout, int* status) {
  extern __shared__ __align__(16) char smem[];
  const int nx = g.Lx - 1;
  for (int item = blockIdx.x; item < Ns * nx; item += gridDim.x)
    pair_item(g, plan, smem, Tpad, S, item / nx, item % nx, envs, logs, tt, pairout, status);
}

// ------------------------------------------------------------------------------------------
// Per-sample combine: ln psi_top from row Lx-1, E_loc = diagonal + row terms + pair terms.
// One warp (all 32 lanes) per sample.
__device__ __forceinline__ void combine_sample(const Geo g, int smp, const uint8_t* __restrict__ S,
                                               const double* rowout, const double* pairout, int use_rows_all,
                                               int use_pairs, const DiagTab dg, double* logabs, double* phase,
                                               double* eloc) {
  const int lane = threadIdx.x & 31;
  const int N = g.Lx * g.Ly;
  const uint8_t* Ss = S + (size_t)smp * N;
  double re = 0.0, im = 0.0;
  if (eloc) {
    for (int p = lane; p < dg.npairs; p += 32) re += dg.pair_v[p] * (double)Ss[dg.pair_ij[2 * p]] * (double)Ss[dg.pair_ij[2 * p + 1]];
    if (dg.onsite)
      for (int i = lane; i < N; i += 32) re += dg.onsite[(size_t)i * g.d + (Ss[i] < g.d ? Ss[i] : 0)];
    if (use_rows_all)
      for (int x = lane; x < g.Lx; x += 32) {
        re += rowout[((size_t)smp * g.Lx + x) * 4 + 2];
        im += rowout[((size_t)smp * g.Lx + x) * 4 + 3];
      }
    if (use_pairs)
      for (int x = lane; x < g.Lx - 1; x += 32) {
        re += pairout[((size_t)smp * g.Lx + x) * 4 + 2];
        im += pairout[((size_t)smp * g.Lx + x) * 4 + 3];
      }
    re = warp_sum(re);
    im = warp_sum(im);
  }
  if (lane == 0) {
    const double* top = rowout + ((size_t)smp * g.Lx + (g.Lx - 1)) * 4;
    if (logabs) logabs[smp] = top[0];
    if (phase) phase[smp] = top[1];
    if (eloc) { eloc[2 * smp] = re; eloc[2 * smp + 1] = im; }
  }
}

#ifdef PEPS_DEFINE_COMMON
__global__ void k_combine(Geo g, int Ns, const uint8_t* __restrict__ S, const double* rowout, const double* pairout,
                          int use_rows_all, int use_pairs, DiagTab dg, double* logabs, double* phase, double* eloc) {
  const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarp = (gridDim.x * blockDim.x) >> 5;
  for (int smp = wid; smp < Ns; smp += nwarp)
    combine_sample(g, smp, S, rowout, pairout, use_rows_all, use_pairs, dg, logabs, phase, eloc);
}
// Global rotation of the physical index: out[site][s][c] = sum_t M[s][t] in[site][t][c] for the
// compact parameter layout (site blocks [s][l][u][r][d]); in: real or (re, im) pairs, out:
// (re, im) pairs.  One CTA per site (persistent over sites).
__global__ void k_rotate_theta(int N, int d, const long long* __restrict__ site_off, RotM M,
                               const double* __restrict__ in, int in_cplx, double* __restrict__ out) {
  for (int site = blockIdx.x; site < N; site += gridDim.x) {
    const long long off = site_off[site];
    const long long blk = (site_off[site + 1] - off) / d;
    for (long long o = threadIdx.x; o < d * blk; o += blockDim.x) {
      const int s = (int)(o / blk);
      const long long c = o % blk;
      double re = 0.0, im = 0.0;
      for (int t = 0; t < d; ++t) {
        const long long k = off + t * blk + c;
        const double xr = in_cplx ? in[2 * k] : in[k], xi = in_cplx ? in[2 * k + 1] : 0.0;
        const double mr = M.m[2 * (s * d + t)], mi = M.m[2 * (s * d + t) + 1];
        re += mr * xr - mi * xi;
        im += mr * xi + mi * xr;
      }
      out[2 * (off + o)] = re;
      out[2 * (off + o) + 1] = im;
    }
  }
}

// E_loc^bound = diagonal pairs + on-site terms + the per-term sums of k_bound.  One warp per sample.
__global__ void k_bound_combine(Geo g, int Ns, int nt, const uint8_t* __restrict__ S, const double* bout, DiagTab dg,
                                double* eloc) {
  const int lane = threadIdx.x & 31;
  const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarp = (gridDim.x * blockDim.x) >> 5;
  const int N = g.Lx * g.Ly;
  for (int smp = wid; smp < Ns; smp += nwarp) {
    const uint8_t* Ss = S + (size_t)smp * N;
    double re = 0.0, im = 0.0;
    for (int p = lane; p < dg.npairs; p += 32) re += dg.pair_v[p] * (double)Ss[dg.pair_ij[2 * p]] * (double)Ss[dg.pair_ij[2 * p + 1]];
    if (dg.onsite)
      for (int i = lane; i < N; i += 32) re += dg.onsite[(size_t)i * g.d + (Ss[i] < g.d ? Ss[i] : 0)];
    for (int t = lane; t < nt; t += 32) {
      re += bout[((size_t)smp * nt + t) * 2];
      im += bout[((size_t)smp * nt + t) * 2 + 1];
    }
    re = warp_sum(re);
    im = warp_sum(im);
    if (lane == 0) { eloc[2 * smp] = re; eloc[2 * smp + 1] = im; }
  }
}
#endif

// ------------------------------------------------------------------------------------------
// Buffers of the moves of one row, carved from the sampler's plan.
template <typename T>
struct MoveBufs {
  T *RP, *t1, *t2, *eu, *el, *A1, *A2, *LW, *LW2, *LC;
  double* red;
};
template <typename T>
__device__ MoveBufs<T> carve_moves(const Plan& plan, char* smem, char* gbase) {
  MoveBufs<T> b;
  b.RP = (T*)buf_ptr(plan, B_RP, smem, gbase);
  b.t1 = (T*)buf_ptr(plan, B_T1, smem, gbase);
  b.t2 = (T*)buf_ptr(plan, B_T2, smem, gbase);
  b.eu = (T*)buf_ptr(plan, B_EU, smem, gbase);
  b.el = (T*)buf_ptr(plan, B_EL, smem, gbase);
  b.A1 = (T*)buf_ptr(plan, B_A, smem, gbase);
  b.A2 = (T*)buf_ptr(plan, B_A2, smem, gbase);
  b.LW = (T*)buf_ptr(plan, B_LW, smem, gbase);
  b.LW2 = (T*)buf_ptr(plan, B_LW2, smem, gbase);
  b.LC = (T*)buf_ptr(plan, B_LP, smem, gbase);
  b.red = (double*)buf_ptr(plan, B_RED, smem, gbase);
  return b;
}

// Random slots before row x in a sweep: the rows already visited (x of them going down,
// Lx-1-x going up) times the moves of a row (in-row moves plus, for exchanges, Ly vertical ones).
template <typename G>
__device__ inline unsigned sweep_slot0(const G& g, int x, int up, int move) {
  const unsigned per = (unsigned)(((move == 0) ? g.Ly - 1 : g.Ly) + ((move == 0) ? g.Ly : 0));
  return (unsigned)(up ? (g.Lx - 1 - x) : x) * per;
}

// The moves of row x of one chain in a sweep going down (up = 0) or up (up = 1): the in-row
// moves (exchange (x,y)<->(x,y+1), flip (x,y), y in order) judged with
// psi_x = E^u[x-1] . T[x] . E^l[x+1], then the vertical exchanges of the rows (xt, xt+1), with
// xt = x going down (x < Lx-1) and xt = x-1 going up (x > 0), judged with
// psi_{xt,xt+1} = E^u[xt-1] . T[xt] . T[xt+1] . E^l[xt+2].  Slots from slot0 on; Sl (shared) is
// updated in place; *acc counts the accepted moves (the same value in every thread).
template <typename T, typename G>
__device__ void row_moves(const G& g, const Plan& plan, const MoveBufs<T>& b, const T* Tpad, uint8_t* Sl,
                          const T* env, int x, int up, int move, unsigned slot0, unsigned long long sweep_id, int c,
                          unsigned long long seed, long long* acc, int* st) {
  __shared__ double logR[MAX_LY + 1];
  __shared__ double logLc, lcur;
  __shared__ int accept_flag;
  const int Ly = g.Ly, Lx = g.Lx, se = g.se, s2 = g.s2;
  const size_t rowsz = (size_t)Ly * se;
  const int nmv = (move == 0) ? Ly - 1 : Ly;
  unsigned slot = slot0;
  T *RP = b.RP, *t1 = b.t1, *t2 = b.t2, *eu = b.eu, *el = b.el, *A1 = b.A1, *A2 = b.A2, *LW = b.LW, *LW2 = b.LW2,
    *LC = b.LC;
  double* red = b.red;
  // ---- moves inside row x with psi_x (E^u[x-1], E^l[x+1])
  {
    const T* EU = env + (size_t)slot_up(g, x - 1) * rowsz;
    const T* EL = env + (size_t)slot_lo(g, x + 1) * rowsz;
    blk_unit(RP + (size_t)Ly * se, se);
    if (threadIdx.x == 0) logR[Ly] = 0.0;
    __syncthreads();
    for (int y = Ly - 1; y >= 0; --y) {
      blk_copy(eu, EU + (size_t)y * se, se);
      blk_copy(el, EL + (size_t)y * se, se);
      load_A(A1, Tpad, g, x * Ly + y, Sl[x * Ly + y], false);
      __syncthreads();
      absorb1_right(g, RP + (size_t)(y + 1) * se, eu, A1, el, t1, t2, RP + (size_t)y * se);
      const double l = blk_normalize(RP + (size_t)y * se, se, red, st);
      if (threadIdx.x == 0) logR[y] = logR[y + 1] + l;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      const double v = dz_abs(to_dz(RP[0]));
      lcur = (v != 0.0) ? log(v) + logR[0] : -INFINITY;
      logLc = 0.0;
    }
    blk_unit(LC, se);
    __syncthreads();
    for (int y = 0; y < nmv; ++y) {
      const double u = uniform53(slot, (uint32_t)sweep_id, (uint32_t)c, 0u, seed);
      ++slot;
      const int i0 = x * Ly + y, i1 = i0 + 1;
      const bool possible = (move == 0) ? (Sl[i0] != Sl[i1]) : true;
      int taken = 0;
      if (possible) {
        // the window: LC with column y in its proposed state (LW2, kept: it is the next LC if
        // the move is accepted), then for an exchange column y+1 as well (LW)
        const int w_ = (move == 0) ? 2 : 1;
        double lw = logLc, l0 = 0.0;
        for (int cc = 0; cc < w_; ++cc) {
          const int site = i0 + cc;
          int s_new;
          if (move == 0) s_new = (cc == 0) ? Sl[i1] : Sl[i0];
          else s_new = g.d - 1 - Sl[site];
          blk_copy(eu, EU + (size_t)(y + cc) * se, se);
          blk_copy(el, EL + (size_t)(y + cc) * se, se);
          load_A(A1, Tpad, g, site, s_new, false);
          __syncthreads();
          if (cc == 0) {
            absorb1(g, LC, eu, A1, el, t1, t2, LW2);
            l0 = blk_normalize(LW2, se, red, st);
            lw += l0;
          } else {
            absorb1(g, LW2, eu, A1, el, t1, t2, LW);
            lw += blk_normalize(LW, se, red, st);
          }
          __syncthreads();
        }
        const T v = blk_dot(w_ == 2 ? LW : LW2, RP + (size_t)(y + w_) * se, se, red);
        if (threadIdx.x == 0) {
          const double av = dz_abs(to_dz(v));
          const double l1 = (av != 0.0) ? log(av) + lw + logR[y + w_] : -INFINITY;
          accept_flag = (isfinite(l1) && u < exp(2.0 * (l1 - lcur))) ? 1 : 0;
          if (accept_flag) {
            lcur = l1;
            if (move == 0) { const uint8_t tmp = Sl[i0]; Sl[i0] = Sl[i1]; Sl[i1] = tmp; }
            else Sl[i0] = (uint8_t)(g.d - 1 - Sl[i0]);
          }
        }
        __syncthreads();
        *acc += accept_flag;
        taken = accept_flag;
        if (taken) {
          // column y now holds the proposed state: the new LC is the window's first column
          blk_copy(LC, LW2, se);
          if (threadIdx.x == 0) logLc += l0;
          __syncthreads();
        }
      }
      if (!taken) {
        blk_copy(eu, EU + (size_t)y * se, se);
        blk_copy(el, EL + (size_t)y * se, se);
        load_A(A1, Tpad, g, x * Ly + y, Sl[x * Ly + y], false);
        __syncthreads();
        absorb1(g, LC, eu, A1, el, t1, t2, LW2);
        const double l = blk_normalize(LW2, se, red, st);
        blk_copy(LC, LW2, se);
        if (threadIdx.x == 0) logLc += l;
        __syncthreads();
      }
    }
  }
  // ---- vertical moves (xt, y) <-> (xt+1, y) with psi_{xt,xt+1} (E^u[xt-1], E^l[xt+2])
  const int xt = up ? x - 1 : x;
  if (move == 0 && xt >= 0 && xt < Lx - 1) {
    const T* EU = env + (size_t)slot_up(g, xt - 1) * rowsz;
    const T* EL2 = env + (size_t)slot_lo(g, xt + 2) * rowsz;
    blk_unit(RP + (size_t)Ly * s2, s2);
    if (threadIdx.x == 0) logR[Ly] = 0.0;
    __syncthreads();
    for (int y = Ly - 1; y >= 0; --y) {
      blk_copy(eu, EU + (size_t)y * se, se);
      blk_copy(el, EL2 + (size_t)y * se, se);
      load_A(A1, Tpad, g, xt * Ly + y, Sl[xt * Ly + y], false);
      load_A(A2, Tpad, g, (xt + 1) * Ly + y, Sl[(xt + 1) * Ly + y], false);
      __syncthreads();
      absorb2_right(g, RP + (size_t)(y + 1) * s2, eu, A1, A2, el, t1, t2, RP + (size_t)y * s2, plan.cx);
      const double l = blk_normalize(RP + (size_t)y * s2, s2, red, st);
      if (threadIdx.x == 0) logR[y] = logR[y + 1] + l;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      const double v = dz_abs(to_dz(RP[0]));
      lcur = (v != 0.0) ? log(v) + logR[0] : -INFINITY;
      logLc = 0.0;
    }
    blk_unit(LC, s2);
    __syncthreads();
    for (int y = 0; y < Ly; ++y) {
      const double u = uniform53(slot, (uint32_t)sweep_id, (uint32_t)c, 0u, seed);
      ++slot;
      const int i0 = xt * Ly + y, i1 = (xt + 1) * Ly + y;
      blk_copy(eu, EU + (size_t)y * se, se);
      blk_copy(el, EL2 + (size_t)y * se, se);
      int taken = 0;
      if (Sl[i0] != Sl[i1]) {
        load_A(A1, Tpad, g, i0, Sl[i1], false);
        load_A(A2, Tpad, g, i1, Sl[i0], false);
        __syncthreads();
        absorb2(g, LC, eu, A1, A2, el, t1, t2, LW2, plan.cx);
        const double l0 = blk_normalize(LW2, s2, red, st);
        const double lw = logLc + l0;
        const T v = blk_dot(LW2, RP + (size_t)(y + 1) * s2, s2, red);
        if (threadIdx.x == 0) {
          const double av = dz_abs(to_dz(v));
          const double l1 = (av != 0.0) ? log(av) + lw + logR[y + 1] : -INFINITY;
          accept_flag = (isfinite(l1) && u < exp(2.0 * (l1 - lcur))) ? 1 : 0;
          if (accept_flag) {
            lcur = l1;
            const uint8_t tmp = Sl[i0]; Sl[i0] = Sl[i1]; Sl[i1] = tmp;
          }
        }
        __syncthreads();
        *acc += accept_flag;
        taken = accept_flag;
        if (taken) {
          // the proposal's window is the new LC
          blk_copy(LC, LW2, s2);
          if (threadIdx.x == 0) logLc += l0;
          __syncthreads();
        }
      }
      if (!taken) {
        load_A(A1, Tpad, g, i0, Sl[i0], false);
        load_A(A2, Tpad, g, i1, Sl[i1], false);
        __syncthreads();
        absorb2(g, LC, eu, A1, A2, el, t1, t2, LW2, plan.cx);
        const double l = blk_normalize(LW2, s2, red, st);
        blk_copy(LC, LW2, s2);
        if (threadIdx.x == 0) logLc += l;
        __syncthreads();
      }
    }
  }
}

// Trivial boundary rows of a sweep: E^u[-1] (going down) or E^l[Lx] (going up), log 0.
template <typename T, typename G>
__device__ void sweep_trivial_row(const G& g, T* env, double* lg, int up) {
  const size_t rowsz = (size_t)g.Ly * g.se;
  const int slot = up ? slot_lo(g, g.Lx) : slot_up(g, -1);
  for (int k = 0; k < g.Ly; ++k) blk_unit(env + (size_t)slot * rowsz + (size_t)k * g.se, g.se);
  if (threadIdx.x == 0) lg[slot] = 0.0;
}

// ------------------------------------------------------------------------------------------
// The Metropolis sweep split by rows (FP32: the row steps then run at the environment kernel's
// occupancy).  A downward sweep = k_env (lower environments of every chain), then for
// x = 0 .. Lx-1: k_sweep_moves(x) and k_env_row(x) (E^u[x] from the updated row); an upward
// sweep starts from the upper environments (the previous sweep's, or k_env's at the start of a
// call) and runs x = Lx-1 .. 0 with k_env_row building E^l[x].
template <typename T, typename G>
__global__ void __launch_bounds__(NTHREADS, EnvBlocks<T>::value) k_sweep_moves(G g, Plan plan,
                                                        const T* __restrict__ Tpad, uint8_t* S, int Ns, int move,
                                                        int x, int up, unsigned long long seed,
                                                        unsigned long long sweep_id, T* envs, double* logs,
                                                        long long* accepted, int* status) {
  extern __shared__ __align__(16) char smem[];
  char* gbase = plan.gbase;
  const MoveBufs<T> b = carve_moves<T>(plan, smem, gbase);
  uint8_t* Sl = (uint8_t*)buf_ptr(plan, B_S, smem, gbase);
  __shared__ int st;
  const int N = g.Lx * g.Ly;
  const unsigned slot0 = sweep_slot0(g, x, up, move);
  for (int c = blockIdx.x; c < Ns; c += gridDim.x) {
    uint8_t* Sg = S + (size_t)c * N;
    for (int i = threadIdx.x; i < N; i += blockDim.x) Sl[i] = Sg[i];
    if (threadIdx.x == 0) st = 0;
    long long acc = 0;
    T* env = envs + (size_t)c * env_sample_elems(g);
    double* lg = logs + (size_t)c * 2 * g.Lx;
    if ((!up && x == 0) || (up && x == g.Lx - 1)) sweep_trivial_row(g, env, lg, up);
    __syncthreads();
    row_moves(g, plan, b, Tpad, Sl, env, x, up, move, slot0, sweep_id, c, seed, &acc, &st);
    for (int i = threadIdx.x; i < N; i += blockDim.x) Sg[i] = Sl[i];
    if (threadIdx.x == 0) {
      if (accepted) accepted[c] += acc;
      if (st) atomicOr(status + c, st);
    }
    __syncthreads();
  }
}

// One environment row of every chain from its (updated) row x, for the sweep's direction:
// going down E^u[x] (the first row for x = 0, else one row step from E^u[x-1]), going up E^l[x]
// (the last row for x = Lx-1, else one row step from E^l[x+1]); compiled for the environment
// kernel's occupancy.  ustat (may be null): also collects the row steps' status bits (the last
// sweep's, for a later evaluation that reuses these environments).
template <typename T, typename G>
__global__ void __launch_bounds__(NTHREADS, EnvBlocks<T>::value) k_env_row(G g, Plan plan, const T* __restrict__ Tpad,
                                                      const uint8_t* __restrict__ S, int Ns, int x, int lower,
                                                      T* envs, double* logs, int* status, int* ustat) {
  extern __shared__ __align__(16) char smem[];
  char* gbase = plan.gbase;
  RowWork<T> w = carve_row<T>(plan, smem, gbase);
  __shared__ int st, flag;
  __shared__ float wd;
  const int N = g.Lx * g.Ly;
  const size_t rowsz = (size_t)g.Ly * g.se;
  for (int c = blockIdx.x; c < Ns; c += gridDim.x) {
    if (threadIdx.x == 0) { st = 0; wd = 0.f; }
    __syncthreads();
    T* env = envs + (size_t)c * env_sample_elems(g);
    double* lg = logs + (size_t)c * 2 * g.Lx;
    const uint8_t* Ss = S + (size_t)c * N;
    double l;
    int slot;
    if (!lower) {
      slot = slot_up(g, x);
      if (x == 0) l = env_first_row(g, env + (size_t)slot * rowsz, Tpad, 0, Ss, false, w.A, w.Z, w.red, &st);
      else l = lg[slot_up(g, x - 1)] + env_row_step(g, env + (size_t)slot_up(g, x - 1) * rowsz, env + (size_t)slot * rowsz,
                                                    Tpad, x, Ss + (size_t)x * g.Ly, false, w, &st, &wd, &flag);
    } else {
      slot = slot_lo(g, x);
      if (x == g.Lx - 1)
        l = env_first_row(g, env + (size_t)slot * rowsz, Tpad, x, Ss + (size_t)x * g.Ly, true, w.A, w.Z, w.red, &st);
      else l = lg[slot_lo(g, x + 1)] + env_row_step(g, env + (size_t)slot_lo(g, x + 1) * rowsz, env + (size_t)slot * rowsz,
                                                    Tpad, x, Ss + (size_t)x * g.Ly, true, w, &st, &wd, &flag);
    }
    if (threadIdx.x == 0) {
      lg[slot] = l;
      if (st) atomicOr(status + c, st);
      if (st && ustat) atomicOr(ustat + c, st);
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------------------------------
// Metropolis sweeps in one launch: one CTA per chain (persistent over chains); the FP64 and
// complex path.  Sweeps alternate direction with the sweep id (even: down the rows, odd: up),
// each starting from the environments the previous one left: going down, the lower
// environments of the current configuration (built at the sweep's start) and E^u rebuilt row
// by row; going up, the upper ones (the previous sweep's, or built at the start of the launch)
// and E^l rebuilt row by row.  Same moves, slots and decisions as the split FP32 sweep.
template <typename T, typename G>
__global__ void __launch_bounds__(NTHREADS, MinBlocks<T>::value) k_sample(G g, Plan plan, const T* __restrict__ Tpad, uint8_t* S,
                                                     int Ns, int move, int nsweeps, unsigned long long seed,
                                                     unsigned long long sweep0, T* envs, double* logs,
                                                     long long* accepted, int* status) {
  extern __shared__ __align__(16) char smem[];
  char* gbase = plan.gbase;
  RowWork<T> w = carve_row<T>(plan, smem, gbase);
  const MoveBufs<T> b = carve_moves<T>(plan, smem, gbase);
  uint8_t* Sl = (uint8_t*)buf_ptr(plan, B_S, smem, gbase);
  __shared__ int st, flag;
  __shared__ float wd;
  const int N = g.Lx * g.Ly, Ly = g.Ly, Lx = g.Lx;
  const size_t rowsz = (size_t)Ly * g.se;
  for (int c = blockIdx.x; c < Ns; c += gridDim.x) {
    uint8_t* Sg = S + (size_t)c * N;
    for (int i = threadIdx.x; i < N; i += blockDim.x) Sl[i] = Sg[i];
    if (threadIdx.x == 0) { st = 0; wd = 0.f; }
    long long acc = 0;
    T* env = envs + (size_t)c * env_sample_elems(g);
    double* lg = logs + (size_t)c * 2 * Lx;
    __syncthreads();
    for (int t = 0; t < nsweeps; ++t) {
      const unsigned long long sweep_id = sweep0 + (unsigned long long)t;
      const int up = (int)(sweep_id & 1ull);
      if (!up) {
        build_lower(g, Tpad, Sl, env, lg, w, &st, &wd, &flag, 1);
        sweep_trivial_row(g, env, lg, 0);
        __syncthreads();
        for (int x = 0; x < Lx; ++x) {
          row_moves(g, plan, b, Tpad, Sl, env, x, 0, move, sweep_slot0(g, x, 0, move), sweep_id, c, seed, &acc, &st);
          if (x < Lx - 1) {
            const size_t sl = (size_t)slot_up(g, x) * rowsz;
            double l;
            if (x == 0) l = env_first_row(g, env + sl, Tpad, 0, Sl, false, w.A, w.Z, w.red, &st);
            else l = lg[slot_up(g, x - 1)] + env_row_step(g, env + (size_t)slot_up(g, x - 1) * rowsz, env + sl, Tpad, x,
                                                           Sl + (size_t)x * Ly, false, w, &st, &wd, &flag);
            if (threadIdx.x == 0) lg[slot_up(g, x)] = l;
            __syncthreads();
          }
        }
      } else {
        if (t == 0) build_upper(g, Tpad, Sl, env, lg, w, &st, &wd, &flag);
        sweep_trivial_row(g, env, lg, 1);
        __syncthreads();
        for (int x = Lx - 1; x >= 0; --x) {
          row_moves(g, plan, b, Tpad, Sl, env, x, 1, move, sweep_slot0(g, x, 1, move), sweep_id, c, seed, &acc, &st);
          if (x > 0) {
            const size_t sl = (size_t)slot_lo(g, x) * rowsz;
            double l;
            if (x == Lx - 1) l = env_first_row(g, env + sl, Tpad, x, Sl + (size_t)x * Ly, true, w.A, w.Z, w.red, &st);
            else l = lg[slot_lo(g, x + 1)] + env_row_step(g, env + (size_t)slot_lo(g, x + 1) * rowsz, env + sl, Tpad, x,
                                                           Sl + (size_t)x * Ly, true, w, &st, &wd, &flag);
            if (threadIdx.x == 0) lg[slot_lo(g, x)] = l;
            __syncthreads();
          }
        }
      }
    }
    for (int i = threadIdx.x; i < N; i += blockDim.x) Sg[i] = Sl[i];
    if (threadIdx.x == 0) {
      if (accepted) accepted[c] += acc;
      if (st) atomicOr(status + c, st);
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------------------------------
// Variational-bound local energy with one fixed cut: every amplitude is
// psi_i(S) = E^u[i-1](S) . E^l[i](S) (0-based rows; the upper MPS holds rows 0..i-1).  One work
// item per (sample, term): for every off-diagonal entry h[a][b] of the term the environments of
// S' (the term's sites set to the digits of b) are rebuilt only on the rows between the first
// changed row and the cut, starting from S's stored environments (rows farther from the cut
// are identical for S and S'), then overlapped.  bout[(smp nt + t)]: the term's sum
// h[a][b] psi_i(S') / psi_i(S) (diagonal entries included) as (re, im); item t = 0 also writes
// ln|psi_i(S)| and its phase.
template <typename T, typename G>
__global__ void __launch_bounds__(NTHREADS, MinBlocks<T>::value) k_bound(G g, Plan plan, const T* __restrict__ Tpad,
                                                    const uint8_t* __restrict__ S, int Ns, int cut,
                                                    const T* envs, const double* logs, TermTab tt, double* bout,
                                                    double* logabs, double* phase, int* status) {
  extern __shared__ __align__(16) char smem[];
  char* gbase = plan.gbase;
  RowWork<T> w = carve_row<T>(plan, smem, gbase);
  uint8_t* Sl = (uint8_t*)buf_ptr(plan, B_S, smem, gbase);
  T* EUb = (T*)buf_ptr(plan, B_LP, smem, gbase);   // 2 rows: rebuilt upper environments
  T* ELb = (T*)buf_ptr(plan, B_RP, smem, gbase);   // 2 rows: rebuilt lower environments
  T* Lb = (T*)buf_ptr(plan, B_LW, smem, gbase);    // 2 chi^2: overlap partials
  T* tb = (T*)buf_ptr(plan, B_LW2, smem, gbase);   // chi D chi
  T* Lb2 = Lb + (size_t)g.chi * g.chi;
  __shared__ int st, flag;
  __shared__ float wd;
  const int N = g.Lx * g.Ly, Ly = g.Ly, Lx = g.Lx;
  const size_t rowsz = (size_t)Ly * g.se;
  const int nt = tt.nterm > 0 ? tt.nterm : 1;
  const int su = slot_up(g, cut - 1), sl = slot_lo(g, cut);
  for (int item = blockIdx.x; item < Ns * nt; item += gridDim.x) {
    const int smp = item / nt, t = item % nt;
    const uint8_t* Ss = S + (size_t)smp * N;
    const T* env = envs + (size_t)smp * env_sample_elems(g);
    const double* lg = logs + (size_t)smp * 2 * Lx;
    if (threadIdx.x == 0) { st = 0; wd = 0.f; }
    __syncthreads();
    double l0 = lg[su] + lg[sl];
    const dz z0 = to_dz(mps_overlap(g, env + (size_t)su * rowsz, env + (size_t)sl * rowsz, Lb, Lb2, tb, w.red, &st, &l0));
    double ere = 0.0, eim = 0.0;
    if (t < tt.nterm) {
      const int* ti = tt.tinfo + (size_t)t * TI_N;
      const int a = local_index(ti, Ss, g.d);
      for (int e = ti[TI_EOFF]; e < ti[TI_EOFF] + ti[TI_ECNT]; ++e) {
        if (tt.ent_ab[2 * e] != a) continue;
        const int b = tt.ent_ab[2 * e + 1];
        const double hr = tt.ent_h[2 * e], hi = tt.ent_h[2 * e + 1];
        if (b == a) { ere += hr; eim += hi; continue; }
        // S' and the rows it changes on each side of the cut
        for (int i = threadIdx.x; i < N; i += blockDim.x) Sl[i] = (uint8_t)state_after(ti, i, Ss, b, g.d);
        int rlo = Lx, rhi = -1;
        for (int k = 0; k < ti[TI_K]; ++k) {
          const int site = ti[TI_S0 + k], r = site / Ly;
          if (state_after(ti, site, Ss, b, g.d) == Ss[site]) continue;
          if (r < cut) rlo = min(rlo, r);
          else rhi = max(rhi, r);
        }
        __syncthreads();
        const T* EU = env + (size_t)su * rowsz;
        double lu = lg[su];
        if (rlo < cut) {
          const T* prev = env + (size_t)slot_up(g, rlo - 1) * rowsz;
          lu = lg[slot_up(g, rlo - 1)];
          for (int r = rlo; r < cut; ++r) {
            T* out = EUb + (size_t)((r - rlo) & 1) * rowsz;
            if (r == 0) lu = env_first_row(g, out, Tpad, 0, Sl, false, w.A, w.Z, w.red, &st);
            else lu += env_row_step(g, prev, out, Tpad, r, Sl + (size_t)r * Ly, false, w, &st, &wd, &flag);
            prev = out;
          }
          EU = prev;
        }
        const T* EL = env + (size_t)sl * rowsz;
        double ll = lg[sl];
        if (rhi >= cut) {
          const T* prev = env + (size_t)slot_lo(g, rhi + 1) * rowsz;
          ll = lg[slot_lo(g, rhi + 1)];
          for (int r = rhi; r >= cut; --r) {
            T* out = ELb + (size_t)((rhi - r) & 1) * rowsz;
            if (r == Lx - 1) ll = env_first_row(g, out, Tpad, Lx - 1, Sl + (size_t)(Lx - 1) * Ly, true, w.A, w.Z, w.red, &st);
            else ll += env_row_step(g, prev, out, Tpad, r, Sl + (size_t)r * Ly, true, w, &st, &wd, &flag);
            prev = out;
          }
          EL = prev;
        }
        double l1 = lu + ll;
        const dz z1 = to_dz(mps_overlap(g, EU, EL, Lb, Lb2, tb, w.red, &st, &l1));
        if (z1.re != 0.0 || z1.im != 0.0) {
          const dz q = dz_div(z1, z0);
          const double f = exp(l1 - l0);
          ere += (hr * q.re - hi * q.im) * f;
          eim += (hr * q.im + hi * q.re) * f;
        }
      }
    }
    if (threadIdx.x == 0) {
      double* o = bout + ((size_t)smp * nt + t) * 2;
      o[0] = ere;
      o[1] = eim;
      const double av = dz_abs(z0);
      int s = st;
      if (t == 0) {
        const double la = (av > 0.0) ? log(av) + l0 : -INFINITY;
        if (logabs) logabs[smp] = la;
        if (phase) phase[smp] = (z0.im == 0.0) ? ((z0.re < 0.0) ? 3.141592653589793 : 0.0) : atan2(z0.im, z0.re);
      }
      if (!(av > 0.0) || !isfinite(ere) || !isfinite(eim)) s |= ST_NONFINITE;
      if (s) atomicOr(status + smp, s);
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------------------------------
// theta (compact, double) -> padded kernel layout [site][s][l][u][r][d] in T
template <typename T>
__global__ void k_pad_theta(Geo g, const double* __restrict__ theta, const long long* site_off, T* Tpad) {
  const long long total = (long long)g.Lx * g.Ly * g.d * g.sT;
  const int D = g.D;
  for (long long o = blockIdx.x * (long long)blockDim.x + threadIdx.x; o < total; o += (long long)gridDim.x * blockDim.x) {
    const int dd = o % D, r = (o / D) % D, u = (o / (D * D)) % D, l = (o / (D * D * D)) % D;
    const int s = (o / g.sT) % g.d;
    const int site = (int)(o / ((long long)g.sT * g.d));
    const int x = site / g.Ly, y = site % g.Ly;
    int Dl, Du, Dr, Dd;
    site_dims(g, x, y, &Dl, &Du, &Dr, &Dd);
    T v = T(0);
    if (l < Dl && u < Du && r < Dr && dd < Dd) {
      const long long k = site_off[site] + (((long long)s * Dl + l) * Du + u) * Dr * Dd + (long long)r * Dd + dd;
      if constexpr (Scal<T>::complex) v = from_dz<T>(dz{theta[2 * k], theta[2 * k + 1]});  // (re, im) pairs
      else v = (T)theta[k];
    }
    Tpad[o] = v;
  }
}

// ------------------------------------------------------------------------------------------
// host-side launch wrappers (explicit instantiations for double and float).  Every launch goes
// to the kernel instantiated for the handle's (chi, D) when one exists, else to the runtime-
// geometry kernel.
template <typename F>
static cudaError_t with_geo(const Geo& g, F&& f) {
  if (g.chi == 16 && g.D == 4) return f(GeoS<16, 4>{g.Lx, g.Ly, g.d, g.cut});
  if (g.chi == 24 && g.D == 4) return f(GeoS<24, 4>{g.Lx, g.Ly, g.d, g.cut});
  return f(g);
}
// complex PEPS run the runtime-shape kernels only
template <typename T, typename F>
static cudaError_t with_geo_for(const Geo& g, F&& f) {
  if constexpr (Scal<T>::complex) return f(g);
  else return with_geo(g, f);
}

// Each translation unit defines PEPS_PART_ENV, PEPS_PART_ROW (k_row, k_pair, parameter padding)
// or PEPS_PART_SAMPLE and instantiates its kernels with PEPS_INST_<part>(T).
#define PEPS_KATTR(NAME, KERNEL)                                                                                   \
  template <typename T>                                                                                          \
  cudaError_t NAME(const Geo& g, size_t set_bytes, int* occ, size_t occ_smem) {                                  \
    return with_geo_for<T>(g, [&](auto gg) {                                                                            \
      using GG = decltype(gg);                                                                                   \
      cudaError_t e = cudaSuccess;                                                                               \
      if (set_bytes) e = cudaFuncSetAttribute(KERNEL<T, GG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)set_bytes); \
      if (e == cudaSuccess && occ) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, KERNEL<T, GG>, NTHREADS, occ_smem); \
      return e;                                                                                                  \
    });                                                                                                          \
  }

#ifdef PEPS_PART_BATCH
// ------------------------------------------------------------------------------------------
// Ragged multi-instance batch in one persistent launch (runtime-shape kernels: every instance
// has its own lattice, D and chi).  The work queue lists (instance, sample) items, the costliest
// instances first; each CTA takes the next item with one atomic and runs that sample's whole
// evaluation with the same device functions as the per-handle kernels (so the results are bit
// for bit theirs): the environment sides, the one-row sandwiches of every row needed, the two-row
// sandwiches, and the combine.  The caller zeroes *next and every instance's status and wdisc.
// the three phases as separate functions: their register allocations stay separate instead of
// one inlined body holding every phase's live ranges
// (an instance whose (chi, D) has a compiled specialisation runs it, as the per-handle kernels do)
template <typename T, typename G>
__device__ __noinline__ void batch_env(const BatchInst<T>& b, G g, char* smem, int smp) {
  RowWork<T> w = carve_row<T>(b.pe, smem, b.pe.gbase);
  env_item(g, w, b.Tpad, b.S, smp, 0, b.envs, b.logs, b.status, b.wdisc);
  if (b.sides == 3) env_item(g, w, b.Tpad, b.S, smp, 1, b.envs, b.logs, b.status, b.wdisc);
}
template <typename T, typename G>
__device__ __noinline__ void batch_row(const BatchInst<T>& b, G g, char* smem, int smp, int x) {
  row_item(g, b.pr, smem, b.Tpad, b.S, smp, x, b.envs, b.logs, b.O, b.site_off, b.Np, b.tt, b.rowout, b.status);
}
template <typename T, typename G>
__device__ __noinline__ void batch_pair(const BatchInst<T>& b, G g, char* smem, int smp, int x) {
  pair_item(g, b.pq, smem, b.Tpad, b.S, smp, x, b.envs, b.logs, b.tt, b.pairout, b.status);
}
template <typename T, typename G>
__device__ __forceinline__ void batch_sample(const BatchInst<T>& b, G g, char* smem, int smp) {
  batch_env<T, G>(b, g, smem, smp);
  const int x_lo = (b.sides == 3) ? 0 : g.Lx - 1;
  for (int x = x_lo; x < g.Lx; ++x) batch_row<T, G>(b, g, smem, smp, x);
  if (b.pairs)
    for (int x = 0; x + 1 < g.Lx; ++x) batch_pair<T, G>(b, g, smem, smp, x);
}

template <typename T>
__global__ void __launch_bounds__(NTHREADS, EnvBlocks<T>::value) k_batch(const BatchInst<T>* __restrict__ inst, int ninst, long long nitems,
                                                    unsigned long long* next) {
  extern __shared__ __align__(16) char smem[];
  __shared__ long long item_s;
  for (;;) {
    if (threadIdx.x == 0) item_s = (long long)atomicAdd(next, 1ull);
    __syncthreads();
    const long long item = item_s;
    if (item >= nitems) break;
    int i = 0;
    while (i + 1 < ninst && inst[i + 1].item0 <= item) ++i;
    const BatchInst<T>& b = inst[i];
    const int smp = (int)(item - b.item0);
    const Geo g = b.g;
    if constexpr (!Scal<T>::complex) {
      if (g.chi == 16 && g.D == 4) batch_sample<T>(b, GeoS<16, 4>{g.Lx, g.Ly, g.d, g.cut}, smem, smp);
      else if (g.chi == 24 && g.D == 4) batch_sample<T>(b, GeoS<24, 4>{g.Lx, g.Ly, g.d, g.cut}, smem, smp);
      else batch_sample<T>(b, g, smem, smp);
    } else {
      batch_sample<T>(b, g, smem, smp);
    }
    __syncthreads();
    if (threadIdx.x < 32)
      combine_sample(g, smp, b.S, b.rowout, b.pairout, b.want_e, b.pairs, b.dg, b.logabs, b.phase, b.eloc);
    __syncthreads();
  }
}

template <typename T>
cudaError_t launch_batch(const BatchInst<T>* inst, int ninst, long long nitems, unsigned long long* next, int grid,
                         size_t smem, cudaStream_t s) {
  k_batch<T><<<grid, NTHREADS, smem, s>>>(inst, ninst, nitems, next);
  return cudaGetLastError();
}
template <typename T>
cudaError_t kattr_batch(size_t set_bytes, int* occ, size_t occ_smem) {
  cudaError_t e = cudaSuccess;
  if (set_bytes) e = cudaFuncSetAttribute(k_batch<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)set_bytes);
  if (e == cudaSuccess && occ) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, k_batch<T>, NTHREADS, occ_smem);
  return e;
}
#define PEPS_INST_BATCH(T)                                                                                       \
  template cudaError_t launch_batch<T>(const BatchInst<T>*, int, long long, unsigned long long*, int, size_t,     \
                                       cudaStream_t);                                                             \
  template cudaError_t kattr_batch<T>(size_t, int*, size_t);
#endif

#ifdef PEPS_PART_ENV
template <typename T>
cudaError_t launch_env(const Geo& g, const Plan& p, int grid, size_t smem, const T* Tpad, const uint8_t* S, int Ns,
                       int sides, T* envs, double* logs, int* status, float* wdisc, cudaStream_t s) {
  return with_geo_for<T>(g, [&](auto gg) {
    k_env<T, decltype(gg)><<<grid, NTHREADS, smem, s>>>(gg, p, Tpad, S, Ns, sides, envs, logs, status, wdisc);
    return cudaGetLastError();
  });
}
PEPS_KATTR(kattr_env, k_env)
#define PEPS_INST_ENV(T)                                                                                          \
  template cudaError_t launch_env<T>(const Geo&, const Plan&, int, size_t, const T*, const uint8_t*, int, int, T*, \
                                     double*, int*, float*, cudaStream_t);                                        \
  template cudaError_t kattr_env<T>(const Geo&, size_t, int*, size_t);
#endif

#ifdef PEPS_PART_ROW
template <typename T>
cudaError_t launch_row(const Geo& g, const Plan& p, int grid, size_t smem, const T* Tpad, const uint8_t* S, int Ns,
                       int x_lo, int x_hi, const T* envs, const double* logs, T* O, const long long* site_off,
                       long long Np, const TermTab& tt, double* rowout, int* status, cudaStream_t s) {
  return with_geo_for<T>(g, [&](auto gg) {
    k_row<T, decltype(gg)><<<grid, NTHREADS, smem, s>>>(gg, p, Tpad, S, Ns, x_lo, x_hi, envs, logs, O, site_off, Np,
                                                        tt, rowout, status);
    return cudaGetLastError();
  });
}
template <typename T>
cudaError_t launch_pair(const Geo& g, const Plan& p, int grid, size_t smem, const T* Tpad, const uint8_t* S, int Ns,
                        const T* envs, const double* logs, const TermTab& tt, double* pairout, int* status, cudaStream_t s) {
  return with_geo_for<T>(g, [&](auto gg) {
    k_pair<T, decltype(gg)><<<grid, NTHREADS, smem, s>>>(gg, p, Tpad, S, Ns, envs, logs, tt, pairout, status);
    return cudaGetLastError();
  });
}
template <typename T>
cudaError_t launch_pad(const Geo& g, const double* theta, const long long* site_off, T* Tpad, cudaStream_t s) {
  k_pad_theta<T><<<304, 256, 0, s>>>(g, theta, site_off, Tpad);
  return cudaGetLastError();
}
PEPS_KATTR(kattr_row, k_row)
PEPS_KATTR(kattr_pair, k_pair)
#define PEPS_INST_ROW(T)                                                                                          \
  template cudaError_t launch_row<T>(const Geo&, const Plan&, int, size_t, const T*, const uint8_t*, int, int, int, \
                                     const T*, const double*, T*, const long long*, long long, const TermTab&,    \
                                     double*, int*, cudaStream_t);                                                \
  template cudaError_t launch_pair<T>(const Geo&, const Plan&, int, size_t, const T*, const uint8_t*, int, const T*, \
                                      const double*, const TermTab&, double*, int*, cudaStream_t);                \
  template cudaError_t launch_pad<T>(const Geo&, const double*, const long long*, T*, cudaStream_t);              \
  template cudaError_t kattr_row<T>(const Geo&, size_t, int*, size_t);                                           \
  template cudaError_t kattr_pair<T>(const Geo&, size_t, int*, size_t);
#endif

#ifdef PEPS_PART_SAMPLE
// FP32 runs the sweep split by rows (k_env for the lower environments, then k_sweep_moves and
// k_env_row per row; the environment plan pe / grid_e / smem_e for the row steps); the other
// precisions run the single-launch k_sample.
template <typename T>
cudaError_t launch_sample(const Geo& g, const Plan& p, int grid, size_t smem, const Plan& pe, int grid_e,
                          size_t smem_e, const T* Tpad, uint8_t* S, int Ns, int move, int nsweeps,
                          unsigned long long seed, unsigned long long sweep0, T* envs, double* logs,
                          long long* accepted, int* status, int* ustat, cudaStream_t s) {
  return with_geo_for<T>(g, [&](auto gg) {
    using GG = decltype(gg);
    if constexpr (sizeof(T) == 4) {
      for (int t = 0; t < nsweeps; ++t) {
        const unsigned long long sid = sweep0 + t;
        const int up = (int)(sid & 1ull);
        int* us = (t == nsweeps - 1) ? ustat : nullptr;
        if (!up) {
          k_env<T, GG><<<grid_e, NTHREADS, smem_e, s>>>(gg, pe, Tpad, S, Ns, 2, envs, logs, status, nullptr);
          for (int x = 0; x < g.Lx; ++x) {
            k_sweep_moves<T, GG><<<grid, NTHREADS, smem, s>>>(gg, p, Tpad, S, Ns, move, x, 0, seed, sid, envs, logs,
                                                              accepted, status);
            if (x < g.Lx - 1)
              k_env_row<T, GG><<<grid_e, NTHREADS, smem_e, s>>>(gg, pe, Tpad, S, Ns, x, 0, envs, logs, status, us);
          }
        } else {
          // the previous sweep of this call left the upper environments of these configurations
          if (t == 0) k_env<T, GG><<<grid_e, NTHREADS, smem_e, s>>>(gg, pe, Tpad, S, Ns, 1, envs, logs, status, nullptr);
          for (int x = g.Lx - 1; x >= 0; --x) {
            k_sweep_moves<T, GG><<<grid, NTHREADS, smem, s>>>(gg, p, Tpad, S, Ns, move, x, 1, seed, sid, envs, logs,
                                                              accepted, status);
            if (x > 0)
              k_env_row<T, GG><<<grid_e, NTHREADS, smem_e, s>>>(gg, pe, Tpad, S, Ns, x, 1, envs, logs, status, us);
          }
        }
      }
    } else {
      k_sample<T, GG><<<grid, NTHREADS, smem, s>>>(gg, p, Tpad, S, Ns, move, nsweeps, seed, sweep0, envs, logs,
                                                   accepted, status);
    }
    return cudaGetLastError();
  });
}
template <typename T>
cudaError_t kattr_sample(const Geo& g, size_t set_bytes, int* occ, size_t occ_smem) {
  return with_geo_for<T>(g, [&](auto gg) {
    using GG = decltype(gg);
    cudaError_t e = cudaSuccess;
    if (set_bytes) {
      e = cudaFuncSetAttribute(k_sample<T, GG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)set_bytes);
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_sweep_moves<T, GG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)set_bytes);
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_env_row<T, GG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)set_bytes);
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_env<T, GG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)set_bytes);
    }
    if (e == cudaSuccess && occ) {
      if constexpr (sizeof(T) == 4)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, k_sweep_moves<T, GG>, NTHREADS, occ_smem);
      else
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, k_sample<T, GG>, NTHREADS, occ_smem);
    }
    return e;
  });
}
#define PEPS_INST_SAMPLE(T)                                                                                       \
  template cudaError_t launch_sample<T>(const Geo&, const Plan&, int, size_t, const Plan&, int, size_t, const T*, \
                                        uint8_t*, int, int, int, unsigned long long, unsigned long long, T*,      \
                                        double*, long long*, int*, int*, cudaStream_t);                           \
  template cudaError_t kattr_sample<T>(const Geo&, size_t, int*, size_t);
#endif

#ifdef PEPS_PART_BOUND
template <typename T>
cudaError_t launch_bound(const Geo& g, const Plan& p, int grid, size_t smem, const T* Tpad, const uint8_t* S, int Ns,
                         int cut, const T* envs, const double* logs, const TermTab& tt, double* bout, double* logabs,
                         double* phase, int* status, cudaStream_t s) {
  return with_geo_for<T>(g, [&](auto gg) {
    k_bound<T, decltype(gg)><<<grid, NTHREADS, smem, s>>>(gg, p, Tpad, S, Ns, cut, envs, logs, tt, bout, logabs, phase,
                                                          status);
    return cudaGetLastError();
  });
}
PEPS_KATTR(kattr_bound, k_bound)
#define PEPS_INST_BOUND(T)                                                                                        \
  template cudaError_t launch_bound<T>(const Geo&, const Plan&, int, size_t, const T*, const uint8_t*, int, int,  \
                                       const T*, const double*, const TermTab&, double*, double*, double*, int*,  \
                                       cudaStream_t);                                                             \
  template cudaError_t kattr_bound<T>(const Geo&, size_t, int*, size_t);
#endif

#ifdef PEPS_DEFINE_COMMON
cudaError_t launch_rotate(int N, int d, const long long* site_off, const RotM& M, const double* in, int in_cplx,
                          double* out, cudaStream_t s) {
  k_rotate_theta<<<N < 1024 ? N : 1024, 256, 0, s>>>(N, d, site_off, M, in, in_cplx, out);
  return cudaGetLastError();
}
cudaError_t launch_bound_combine(const Geo& g, int Ns, int nt, const uint8_t* S, const double* bout, const DiagTab& dg,
                                 double* eloc, cudaStream_t s) {
  const int blocks = (Ns * 32 + 255) / 256;
  k_bound_combine<<<blocks > 0 ? blocks : 1, 256, 0, s>>>(g, Ns, nt, S, bout, dg, eloc);
  return cudaGetLastError();
}
cudaError_t launch_combine(const Geo& g, int Ns, const uint8_t* S, const double* rowout, const double* pairout,
                           int use_rows_all, int use_pairs, const DiagTab& dg, double* logabs, double* phase,
                           double* eloc, cudaStream_t s) {
  const int blocks = (Ns * 32 + 255) / 256;
  k_combine<<<blocks > 0 ? blocks : 1, 256, 0, s>>>(g, Ns, S, rowout, pairout, use_rows_all, use_pairs, dg, logabs, phase, eloc);
  return cudaGetLastError();
}
#endif

}  // namespace peps

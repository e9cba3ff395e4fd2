// Direct sampling of a finite PEPS (Sec. "On Direct Sampling", appendix "Direct sampling of
// PEPS", Alg. `sampling`): double-layer lower boundary MPS D^l built once per parameter set,
// then every configuration drawn row by row from the conditional reduced density matrix
//   rho_{S<i}[i] = T^u_{S<i}[i] . D^l[i+1] . (T^u_{S<i}[i])^*,
// T^u = E^u[i-1](S) . T[i] with the physical legs open (kept exact), sites left to right.
// Included by peps_direct_{f32,f64,c32,c64}.cu, one scalar type each.
#pragma once
#include "peps_kernels_impl.cuh"

namespace peps {

// ------------------------------------------------------------------------------------------
// Double-layer lower environments D^l[x], x = Lx .. 1 (0-based rows x .. Lx-1 traced), one CTA.
// D^l[x] site y: [c][(u, u')][e] (chi_d x D^2 x chi_d, padded), (u, u') the up legs of row x
// in the ket and the bra; D^l[Lx] is the trivial row.  Row x: the exact product
//   B_y[(c, L)][U][(f, R)] = sum_{p=(d,d')} D^l[x+1]_y[c][p][f] M_y[L][U][R][p],
//   M_y[(l,l')][(u,u')][(r,r')][(d,d')] = sum_s T[s][l][u][r][d] conj(T[s][l'][u'][r'][d']),
// compressed to chi_d by the QR-based density-matrix truncation (left pass: R factors of
// R_{k-1} B_k; right pass: one-sided Jacobi of X = R_{k-1} Y_k, the top chi_d right singular
// vectors kept), every site divided by its largest modulus.  *status: status bits.
template <typename T, typename G>
__global__ void __launch_bounds__(NTHREADS) k_dl_env(G g, int chid, const T* __restrict__ Tpad, T* DL, DlWork<T> w,
                                                     int* status) {
  using RT = typename Scal<T>::R;
  extern __shared__ __align__(16) char smem[];
  const DlDims dd = dl_dims(g.D, chid);
  double* red = (double*)smem;
  RT* sig = (RT*)(smem + 40 * 8);
  size_t off = 40 * 8 + (size_t)(dd.mX + 4) * sizeof(RT);
  off = (off + 15) / 16 * 16;
  int* sel = (int*)(smem + off);
  off += (size_t)2 * dd.mX * 4;
  off = (off + 15) / 16 * 16;
  T* taus = (T*)(smem + off);
  __shared__ int st, flag;
  const int tid = threadIdx.x, NT = blockDim.x;
  const int Ly = g.Ly, D = g.D, d = g.d, P = dd.P, nb = dd.nb, Lr = dd.Lr, LY = dd.LY, LX = dd.LX, mX = dd.mX;
  const size_t sd = (size_t)chid * P * chid, rowsz = (size_t)Ly * sd, bsz = (size_t)nb * P * nb;
  if (tid == 0) st = 0;
  T* last = DL + (size_t)g.Lx * rowsz;
  for (int k = 0; k < Ly; ++k) blk_unit(last + (size_t)k * sd, (int)sd);
  __syncthreads();
  for (int x = g.Lx - 1; x >= 1; --x) {
    const T* Dn = DL + (size_t)(x + 1) * rowsz;
    T* Dx = DL + (size_t)x * rowsz;
    // ---- exact double-layer product
    for (int y = 0; y < Ly; ++y) {
      const T* Ts = Tpad + (size_t)(x * Ly + y) * d * g.sT;
      const T* Dy = Dn + (size_t)y * sd;
      T* By = w.B + (size_t)y * bsz;
      for (size_t o = tid; o < bsz; o += NT) {
        const int b = (int)(o % nb), U = (int)((o / nb) % P), a = (int)(o / ((size_t)nb * P));
        const int c = a / P, L = a % P, f = b / P, R = b % P;
        const int l = L / D, l2 = L % D, u = U / D, u2 = U % D, r = R / D, r2 = R % D;
        T acc = T(0);
        for (int p = 0; p < P; ++p) {
          const T dv = Dy[((size_t)c * P + p) * chid + f];
          if (dv == T(0)) continue;
          const int dn = p / D, dn2 = p % D;
          T m = T(0);
          for (int s = 0; s < d; ++s)
            m += Ts[(size_t)s * g.sT + ((l * D + u) * D + r) * D + dn] *
                 conj_(Ts[(size_t)s * g.sT + ((l2 * D + u2) * D + r2) * D + dn2]);
          acc += dv * m;
        }
        By[o] = acc;
      }
    }
    __syncthreads();
    // ---- left pass: R_k from the QR of Z = R_{k-1} B_k ((i, p) rows, b columns; column major)
    const int mZ = nb * P;
    for (int k = 0; k + 1 < Ly; ++k) {
      const T* Bk = w.B + (size_t)k * bsz;
      const T* Rp = w.Rh + (size_t)(k - 1) * nb * nb;
      for (size_t o = tid; o < (size_t)mZ * nb; o += NT) {
        const int row = (int)(o % mZ), b = (int)(o / mZ);
        const int i = row / P, p = row % P;
        T acc = T(0);
        if (k == 0) {
          if (i == 0) acc = Bk[(size_t)p * nb + b];   // R_{-1} = e_00: the left boundary bond
        } else {
          for (int a = i; a < nb; ++a) acc += Rp[(size_t)i * nb + a] * Bk[((size_t)a * P + p) * nb + b];
        }
        w.Z[o] = acc;
      }
      __syncthreads();
      qr_keep_r_smem(w.Z, mZ, nb, w.Rh + (size_t)k * nb * nb, taus, nb);
    }
    // ---- right pass
    blk_unit(w.C, nb * chid);
    __syncthreads();
    for (int k = Ly - 1; k >= 0; --k) {
      const T* Bk = w.B + (size_t)k * bsz;
      // Y[a][(p, c)] = sum_b B_k[a][p][b] C[b][c]
      for (int o = tid; o < nb * Lr; o += NT) {
        const int c = o % chid, p = (o / chid) % P, a = o / Lr;
        const T* Br = Bk + ((size_t)a * P + p) * nb;
        T acc = T(0);
        for (int b = 0; b < nb; ++b) acc += Br[b] * w.C[(size_t)b * chid + c];
        w.Y[(size_t)a * LY + p * chid + c] = acc;
      }
      __syncthreads();
      T* site = Dx + (size_t)k * sd;
      if (k == 0) {
        // first site: its left bond is trivial, keep row a = 0 of Y
        for (int o = tid; o < (int)sd; o += NT) {
          const int c = o % chid, p = (o / chid) % P, ap = o / (P * chid);
          site[o] = (ap == 0) ? w.Y[p * chid + c] : T(0);
        }
        __syncthreads();
        blk_normalize(site, (int)sd, red, &st);
        break;
      }
      const T* Rp = w.Rh + (size_t)(k - 1) * nb * nb;
      for (int o = tid; o < mX * Lr; o += NT) {
        const int q = o % Lr, i = o / Lr;
        T acc = T(0);
        if (i < nb)
          for (int j = i; j < nb; ++j) acc += Rp[(size_t)i * nb + j] * w.Y[(size_t)j * LY + q];
        w.X[(size_t)i * LX + q] = acc;
      }
      __syncthreads();
      const int sweeps = hestenes_rows<T, 0>(w.X, mX, Lr, LX, &flag, nullptr, red, sig);
      if (sweeps < 0 && tid == 0) st |= ST_NOCONV;
      {
        const int lane = tid & 31, warp = tid >> 5, nw = NT >> 5;
        for (int p = warp; p < mX; p += nw) {
          RT s = 0;
          for (int i = lane; i < Lr; i += 32) s += abs2_(w.X[(size_t)p * LX + i]);
          s = warp_sum(s);
          if (lane == 0) sig[p] = sqrt(s);
        }
      }
      __syncthreads();
      // stable descending ranks (NaN below every number)
      for (int p = tid; p < mX; p += NT) {
        const RT sp = sig[p];
        const RT kp = (sp == sp) ? sp : RT(-1);
        if (!(sp == sp) || isinf(sp)) atomicOr(&st, (int)ST_NONFINITE);
        int rk = 0;
        for (int q = 0; q < mX; ++q) {
          const RT sq = sig[q];
          const RT kq = (sq == sq) ? sq : RT(-1);
          rk += (kq > kp) || (kq == kp && q < p);
        }
        if (rk < chid) sel[rk] = p;
      }
      __syncthreads();
      const int nkeep = (mX < chid) ? mX : chid;
      // Vt[c'][q] = X[sel(c')][q] / sigma: the kept rows of V^H
      for (int o = tid; o < chid * Lr; o += NT) {
        const int q = o % Lr, cp = o / Lr;
        T v = T(0);
        if (cp < nkeep) {
          const int p = sel[cp];
          const RT s = sig[p];
          if (s > RT(0)) v = w.X[(size_t)p * LX + q] * (RT(1) / s);
        }
        w.Vt[(size_t)cp * LY + q] = v;
      }
      __syncthreads();
      for (int o = tid; o < nb * chid; o += NT) {
        const int cp = o % chid, j = o / chid;
        T acc = T(0);
        for (int q = 0; q < Lr; ++q) acc = mad(acc, w.Y[(size_t)j * LY + q], conj_(w.Vt[(size_t)cp * LY + q]));
        w.Cn[o] = acc;
      }
      for (int o = tid; o < (int)sd; o += NT) site[o] = w.Vt[(size_t)(o / Lr) * LY + o % Lr];
      __syncthreads();
      blk_normalize(site, (int)sd, red, &st);
      blk_copy(w.C, w.Cn, nb * chid);
      __syncthreads();
    }
  }
  if (tid == 0) *status = st;
}

// Ket site y of T^u, K[s][dd][B][A] = sum_u E^u_y[a][u][b] T[s][l][u][r][dd] (A = (a, l),
// B = (b, r)), and its complex conjugate in the same layout.  Ends with a barrier.
template <typename T, typename G>
__device__ void ket_site(const G& g, const T* E, const T* Ts, T* K, T* KCj) {
  const int D = g.D, chi = g.chi, AB = chi * D;
  const size_t ksz = (size_t)g.d * D * AB * AB;
  for (size_t o = threadIdx.x; o < ksz; o += blockDim.x) {
    const int A = (int)(o % AB), B = (int)((o / AB) % AB), dd = (int)((o / ((size_t)AB * AB)) % D),
              s = (int)(o / ((size_t)AB * AB * D));
    const int a = A / D, l = A % D, b = B / D, r = B % D;
    T acc = T(0);
    for (int u = 0; u < D; ++u)
      acc += E[((size_t)a * D + u) * chi + b] * Ts[(size_t)s * g.sT + ((l * D + u) * D + r) * D + dd];
    K[o] = acc;
    KCj[o] = conj_(acc);
  }
  __syncthreads();
}

// ------------------------------------------------------------------------------------------
// Direct sampling: one CTA per configuration (persistent).  Row x of chain c in draw round t:
//   K_y[s][dd][B][A] = sum_u E^u[x-1]_y[a][u][b] T[s][l][u][r][dd]   (A = (a, l), B = (b, r)),
//   the ket sites of T^u (and KC_y = conj(K_y), same layout);
//   right partials with the physical legs traced, R_y[A][c][A'] (c the D^l bond), from the
//   right; then left to right, for every candidate s of site y,
//   cand_s[B][e][B'] = sum L[A][c][A'] K[A][s][d][B] D^l[c][(d, d')][e] conj(K[A'][s][d'][B']),
//   w_s = Re <cand_s, R_{y+1}> (negative weights count as zero), s drawn with
//   u = uniform53(Philox(x Ly + y, t, c, 2; seed)), L = cand_s normalised.  After the row,
//   E^u[x] = truncate_chi(E^u[x-1] . T_proj[x]) by the environment kernels' row step.
// Every contraction is a register-tiled blk_gemm; the temporaries' layouts put the index that
// varies across threads at stride 1 in the operand it is read from.
// logp[c] = sum of the logs of the drawn conditionals (FP64).
template <typename T, typename G>
__global__ void __launch_bounds__(NTHREADS, MinBlocks<T>::value) k_direct(G g, Plan plan, int chid, const T* __restrict__ Tpad,
                                                     const T* __restrict__ DL, uint8_t* S, int Ns,
                                                     unsigned long long seed, unsigned long long draw, double* logp,
                                                     int* status) {
  extern __shared__ __align__(16) char smem[];
  char* gbase = plan.gbase;
  RowWork<T> w = carve_row<T>(plan, smem, gbase);
  uint8_t* Sl = (uint8_t*)buf_ptr(plan, B_S, smem, gbase);
  T* EU = (T*)buf_ptr(plan, B_EU, smem, gbase);    // two E^u rows, used alternately
  T* Ky = (T*)buf_ptr(plan, B_T1, smem, gbase);    // K[s][dd][B][A] of the current site
  T* KCy = (T*)buf_ptr(plan, B_T2, smem, gbase);   // conj(K), same layout
  T* RP = (T*)buf_ptr(plan, B_RP, smem, gbase);    // (Ly+1) x R[A][c][A']
  T* V1 = (T*)buf_ptr(plan, B_LP, smem, gbase);
  T* V2 = (T*)buf_ptr(plan, B_LW, smem, gbase);
  T* LC = (T*)buf_ptr(plan, B_LW2, smem, gbase);   // d candidates + the running left partial
  double* red = w.red;
  __shared__ int st, flag;
  __shared__ float wd;
  __shared__ double pw[8];
  __shared__ int pick;
  const int tid = threadIdx.x, NT = blockDim.x;
  const int Ly = g.Ly, Lx = g.Lx, D = g.D, d = g.d, chi = g.chi, N = Lx * Ly;
  const int AB = chi * D, P = D * D, CA = chid * AB;
  const size_t rowsz = (size_t)Ly * g.se, sd = (size_t)chid * P * chid;
  const size_t ksz = (size_t)d * D * AB * AB, rsz = (size_t)AB * chid * AB;
  T* Lp = LC + (size_t)d * rsz;
  // register-tile edge of the large contractions (complex double: smaller, to stay in registers)
  constexpr int TE = sizeof(T) >= 16 ? 4 : 8;
  for (int c = blockIdx.x; c < Ns; c += gridDim.x) {
    if (tid == 0) { st = 0; wd = 0.f; }
    // E^u[-1]: the trivial row
    for (int k = 0; k < Ly; ++k) blk_unit(EU + (size_t)k * g.se, g.se);
    __syncthreads();
    double lp = 0.0;
    int cur = 0;
    for (int x = 0; x < Lx; ++x) {
      const T* Eu = EU + (size_t)cur * rowsz;
      const T* Dn = DL + (size_t)(x + 1) * Ly * sd;
      // right partials, physical legs traced
      blk_unit(RP + (size_t)Ly * rsz, (int)rsz);
      __syncthreads();
      for (int y = Ly - 1; y >= 0; --y) {
        ket_site(g, Eu + (size_t)y * g.se, Tpad + (size_t)(x * Ly + y) * d * g.sT, Ky, KCy);
        const T* Dg = Dn + (size_t)y * sd;
        const T* Rn = RP + (size_t)(y + 1) * rsz;
        T* Ry = RP + (size_t)y * rsz;
        // V1[s][B'][dd][e][A] = sum_B K[A][s][dd][B] R[B][e][B']   (m = (A, s dd), n = (e, B'), k = B)
        blk_gemm<TE, TE>(Ky, Rn, V1, AB * d * D, CA, AB, 1, AB, 0, CA, 0,
                       [=](int m) {
                         const int A = m % AB, q = m / AB, s = q / D, dd = q % D;
                         return Off2{q * AB * AB + A, ((s * AB * D + dd) * chid) * AB + A};
                       },
                       [=](int n) {
                         const int e = n / AB, Bp = n % AB;
                         return Off2{n, (Bp * D * chid + e) * AB};
                       });
        // V2[s][d'][B'][A][c] = sum_{dd, e} V1[s][B'][dd][e][A] D^l[c][(dd, d')][e]
        //   (m = (A, B', s), n = (c, d'), k = (dd, e))
        blk_gemm<2, 16>(V1, Dg, V2, AB * AB * d, chid * D, D, chid, chid * AB, AB, D * chid, 1,
                       [=](int m) {
                         const int A = m % AB, Bp = (m / AB) % AB, s = m / (AB * AB);
                         return Off2{((s * AB + Bp) * D * chid) * AB + A, ((s * D * AB + Bp) * AB + A) * chid};
                       },
                       [=](int n) {
                         const int cc = n / D, dp = n % D;
                         return Off2{(cc * P + dp) * chid, dp * AB * AB * chid + cc};
                       });
        // R_y[A][c][A'] = sum_{(s, d'), B'} conj(K)[A'][s][d'][B'] V2[s][d'][B'][A][c]
        //   (m = A', n = (A, c), k = ((s, d'), B'))
        blk_gemm<TE, TE>(KCy, V2, Ry, AB, CA, d * D, AB, AB * AB, AB, AB * CA, CA,
                       [=](int m) { return Off2{m, m}; },
                       [=](int n) { return Off2{n, n * AB}; });
        blk_normalize(Ry, (int)rsz, red, &st);
      }
      // left to right: draw the row
      blk_unit(Lp, (int)rsz);
      __syncthreads();
      for (int y = 0; y < Ly; ++y) {
        ket_site(g, Eu + (size_t)y * g.se, Tpad + (size_t)(x * Ly + y) * d * g.sT, Ky, KCy);
        const T* Dg = Dn + (size_t)y * sd;
        const T* Rn = RP + (size_t)(y + 1) * rsz;
        // W1[s][B][c][dd][A'] = sum_A L[A][c][A'] K[A][s][dd][B]   (m = (A', c), n = (s dd, B), k = A)
        blk_gemm<TE, TE>(Lp, Ky, V1, CA, d * D * AB, AB, 1, CA, 0, 1, 0,
                       [=](int m) {
                         const int Ap = m % AB, cc = m / AB;
                         return Off2{cc * AB + Ap, cc * D * AB + Ap};
                       },
                       [=](int n) {
                         const int B = n % AB, q = n / AB, s = q / D, dd = q % D;
                         return Off2{n * AB, ((s * AB + B) * chid * D + dd) * AB};
                       });
        // W2[s][d'][A'][e][B] = sum_{c, dd} W1[s][B][c][dd][A'] D^l[c][(dd, d')][e]
        //   (m = (A', B, s), n = (d', e), k = (c, dd))
        blk_gemm<2, 16>(V1, Dg, V2, AB * AB * d, D * chid, chid, D, D * AB, AB, P * chid, D * chid,
                       [=](int m) {
                         const int Ap = m % AB, B = (m / AB) % AB, s = m / (AB * AB);
                         return Off2{((s * AB + B) * chid * D) * AB + Ap, ((s * D * AB + Ap) * chid) * AB + B};
                       },
                       [=](int n) {
                         const int dp = n / chid, e = n % chid;
                         return Off2{dp * chid + e, (dp * AB * chid + e) * AB};
                       });
        // cand_s[B][e][B'] = sum_{d', A'} W2[s][d'][A'][e][B] conj(K)[A'][s][d'][B']
        //   (per s: m = (B, e), n = B', k = (d', A'))
        for (int s = 0; s < d; ++s)
          blk_gemm<TE, TE>(V2 + (size_t)s * D * AB * CA, KCy + (size_t)s * D * AB * AB, LC + (size_t)s * rsz, CA, AB, D,
                         AB, AB * CA, CA, AB * AB, 1,
                         [=](int m) {
                           const int B = m % AB, e = m / AB;
                           return Off2{e * AB + B, (B * chid + e) * AB};
                         },
                         [=](int n) { return Off2{n * AB, n}; });
        // weights, then the draw
        for (int s = 0; s < d; ++s) {
          double part = 0.0;
          for (size_t o = tid; o < rsz; o += NT) part += (double)re_(LC[(size_t)s * rsz + o] * Rn[o]);
          const double ws = block_sum(part, red);
          if (tid == 0) pw[s] = (ws > 0.0) ? ws : 0.0;
        }
        if (tid == 0) {
          double tot = 0.0;
          for (int s = 0; s < d; ++s) tot += pw[s];
          if (!(tot > 0.0) || !isfinite(tot)) {
            st |= ST_ZERO_NORM;
            for (int s = 0; s < d; ++s) pw[s] = 1.0;
            tot = (double)d;
          }
          const double u = uniform53((uint32_t)(x * Ly + y), (uint32_t)draw, (uint32_t)c, 2u, seed);
          double acc = 0.0;
          int s_pick = d - 1;
          for (int s = 0; s < d; ++s) {
            acc += pw[s] / tot;
            if (u < acc) { s_pick = s; break; }
          }
          pick = s_pick;
          const double ps = pw[s_pick] / tot;
          pw[d] = (ps > 0.0) ? log(ps) : -INFINITY;
          Sl[x * Ly + y] = (uint8_t)s_pick;
        }
        __syncthreads();
        lp += pw[d];
        blk_copy(Lp, LC + (size_t)pick * rsz, (int)rsz);
        __syncthreads();
        blk_normalize(Lp, (int)rsz, red, &st);
      }
      // E^u[x] from the drawn row
      if (x < Lx - 1) {
        T* out = EU + (size_t)(cur ^ 1) * rowsz;
        if (x == 0) env_first_row(g, out, Tpad, 0, Sl, false, w.A, w.Z, red, &st);
        else env_row_step(g, Eu, out, Tpad, x, Sl + (size_t)x * Ly, false, w, &st, &wd, &flag);
        cur ^= 1;
        __syncthreads();
      }
    }
    uint8_t* Sg = S + (size_t)c * N;
    for (int i = tid; i < N; i += NT) Sg[i] = Sl[i];
    if (tid == 0) {
      logp[c] = lp;
      status[c] = st;
    }
    __syncthreads();
  }
}

template <typename T>
cudaError_t launch_dl_env(const Geo& g, int chid, const T* Tpad, T* DL, const DlWork<T>& w, int* status,
                          cudaStream_t s) {
  const size_t sm = dl_smem_bytes(g.D, chid, sizeof(T), sizeof(typename Scal<T>::R));
  cudaError_t e = cudaFuncSetAttribute(k_dl_env<T, Geo>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  k_dl_env<T, Geo><<<1, NTHREADS, sm, s>>>(g, chid, Tpad, DL, w, status);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_direct(const Geo& g, const Plan& p, int grid, size_t smem, int chid, const T* Tpad, const T* DL,
                          uint8_t* S, int Ns, unsigned long long seed, unsigned long long draw, double* logp,
                          int* status, cudaStream_t s) {
  k_direct<T, Geo><<<grid, NTHREADS, smem, s>>>(g, p, chid, Tpad, DL, S, Ns, seed, draw, logp, status);
  return cudaGetLastError();
}

template <typename T>
cudaError_t kattr_direct(const Geo& g, size_t set_bytes, int* occ, size_t occ_smem) {
  cudaError_t e = cudaSuccess;
  if (set_bytes) e = cudaFuncSetAttribute(k_direct<T, Geo>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)set_bytes);
  if (e == cudaSuccess && occ) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, k_direct<T, Geo>, NTHREADS, occ_smem);
  return e;
}

#define PEPS_INST_DIRECT(T)                                                                                        \
  template cudaError_t launch_dl_env<T>(const Geo&, int, const T*, T*, const DlWork<T>&, int*, cudaStream_t);      \
  template cudaError_t launch_direct<T>(const Geo&, const Plan&, int, size_t, int, const T*, const T*, uint8_t*,   \
                                        int, unsigned long long, unsigned long long, double*, int*, cudaStream_t); \
  template cudaError_t kattr_direct<T>(const Geo&, size_t, int*, size_t);

}  // namespace peps

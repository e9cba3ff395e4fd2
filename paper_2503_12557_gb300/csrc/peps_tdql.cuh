// Implicit symmetric QR on a tridiagonal matrix, applied to one vector (the eigenvalue part of
// the MinSR pseudo-inverse of Eq. (tdvp_fast) after the Householder reduction to tridiagonal
// form).  Plain scalar code, callable from one device thread or from host code.
//
// T0 = tridiag(d, e) (d: N diagonal entries, e: N - 1 off-diagonal ones).  Each QR step works
// on an unreduced block [l, h] with the shift of the trailing 2 x 2 block that is closer to its
// last diagonal entry (Wilkinson), chasing the bulge from the top down with plane rotations
// G_k on the index pair (k, k + 1):  new_k = c old_k + s old_{k+1},  new_{k+1} = -s old_k + c
// old_{k+1}, applied as T <- G T G^T.  When every off-diagonal entry is negligible, d holds the
// eigenvalues Lambda and T0 = Z diag(Lambda) Z^T with Z = G_1^T G_2^T ... G_M^T.
//   td_ql:     d <- Lambda, y <- Z^T y (each rotation applied to y as it is made), and the
//              rotations recorded in order, one double each (td_enc), every QR step closed by
//              its (l, h) as two doubles;
//   td_replay: u <- Z u (the recorded rotations transposed, in reverse order).
// The record lives in two segments, r0[0, cap0) then r1[0, cap1), so that two separate
// buffers can hold it.
#pragma once
#include <math.h>
#include <float.h>
#include <stddef.h>

namespace peps {

// One double per rotation with c >= 0 (Stewart's economical storage of plane rotations):
// |s| < c stores s / 2 (|rho| < 0.36), otherwise sign(s) 2 / c (|rho| >= 2.8; c = 0 gives an
// infinity).  The decoded pair differs from the stored one by rounding only.
__host__ __device__ __forceinline__ double td_enc(double c, double s) {
  return (fabs(s) < c) ? 0.5 * s : copysign(2.0 / c, s);
}
__host__ __device__ __forceinline__ void td_dec(double rho, double& c, double& s) {
  if (fabs(rho) < 1.0) {
    s = 2.0 * rho;
    c = sqrt(1.0 - s * s);
  } else {
    c = 2.0 / fabs(rho);
    const double q = 1.0 - c * c;
    s = copysign(sqrt(q > 0.0 ? q : 0.0), rho);
  }
}

__host__ __device__ __forceinline__ void td_rec_put(double* r0, size_t cap0, double* r1, size_t i, double v) {
  if (i < cap0) r0[i] = v; else r1[i - cap0] = v;
}
__host__ __device__ __forceinline__ double td_rec_get(const double* r0, size_t cap0, const double* r1, size_t i) {
  return (i < cap0) ? r0[i] : r1[i - cap0];
}

// |e_i| negligible against its diagonal neighbours (or against the whole matrix, below eps^2)
__host__ __device__ __forceinline__ bool td_negligible(const double* d, const double* e, int i, double anorm) {
  const double a = fabs(e[i]);
  return a <= DBL_EPSILON * (fabs(d[i]) + fabs(d[i + 1])) || a <= DBL_EPSILON * DBL_EPSILON * anorm;
}

// Returns 0 on success, 1 when a trailing eigenvalue needed more than maxit QR steps, 2 when
// the record would pass its capacity; *steps = QR steps taken, *len = doubles recorded.
__host__ __device__ inline int td_ql(double* __restrict__ d, double* __restrict__ e, double* __restrict__ y, int N,
                                     double* r0, size_t cap0, double* r1, size_t cap1, int maxit, long long* steps,
                                     size_t* len) {
  double anorm = 0.0;
  for (int i = 0; i < N; ++i) anorm = fmax(anorm, fabs(d[i]));
  double emax = 0.0;
  for (int i = 0; i + 1 < N; ++i) emax = fmax(emax, fabs(e[i]));
  anorm += 2.0 * emax;
  const size_t cap = cap0 + cap1;
  size_t pos = 0;
  long long nstep = 0;
  int status = 0;
  int h = N - 1, it = 0;
  while (h > 0) {
    if (td_negligible(d, e, h - 1, anorm)) {
      e[h - 1] = 0.0;
      --h;
      it = 0;
      continue;
    }
    int l = h - 1;
    while (l > 0 && !td_negligible(d, e, l - 1, anorm)) --l;
    if (l > 0) e[l - 1] = 0.0;
    if (++it > maxit) { status = 1; break; }
    if (pos + (size_t)(h - l) + 2 > cap) { status = 2; break; }
    ++nstep;
    // shift: the eigenvalue of the trailing 2 x 2 block closer to d[h]
    const double dl = 0.5 * (d[h - 1] - d[h]), bt = e[h - 1];
    const double rt = hypot(dl, bt);
    const double den = dl + (dl >= 0.0 ? rt : -rt);
    const double mu = d[h] - (den != 0.0 ? bt * bt / den : 0.0);
    // the chase; a = d[k], f = e[k], yk = y[k] are carried as the rotations update them
    double x = d[l] - mu, z = e[l];
    double a = d[l], f = e[l], yk = y[l];
    for (int k = l; k < h; ++k) {
      const double b = d[k + 1];
      const double g = (k + 1 < h) ? e[k + 1] : 0.0;
      const double yk1 = y[k + 1];
      double r = hypot(x, z), c = 1.0, s = 0.0;
      if (r != 0.0) {
        c = x / r;
        s = z / r;
        if (c < 0.0) { c = -c; s = -s; r = -r; }
      }
      td_rec_put(r0, cap0, r1, pos++, td_enc(c, s));
      if (k > l) e[k - 1] = r;  // the bulge against e[k - 1] annihilated
      const double cc = c * c, ss = s * s, cs = c * s;
      d[k] = cc * a + 2.0 * cs * f + ss * b;
      const double bn = ss * a - 2.0 * cs * f + cc * b;
      const double fn = cs * (b - a) + (cc - ss) * f;
      y[k] = c * yk + s * yk1;
      yk = c * yk1 - s * yk;
      a = bn;
      x = fn;        // e[k] after the rotation: the next rotation annihilates the bulge against it
      z = s * g;     // the new bulge at (k, k + 2)
      f = c * g;     // e[k + 1] after the rotation
      if (k + 1 == h) e[k] = fn;
    }
    d[h] = a;
    y[h] = yk;
    td_rec_put(r0, cap0, r1, pos++, (double)l);
    td_rec_put(r0, cap0, r1, pos++, (double)h);
  }
  *steps = nstep;
  *len = pos;
  return status;
}

// u <- Z u for the rotations td_ql recorded (len doubles)
__host__ __device__ inline void td_replay(double* __restrict__ u, const double* r0, size_t cap0, const double* r1,
                                          size_t len) {
  size_t p = len;
  while (p >= 2) {
    const int h = (int)td_rec_get(r0, cap0, r1, p - 1);
    const int l = (int)td_rec_get(r0, cap0, r1, p - 2);
    p -= 2;
    double uk1 = u[h];
    for (int k = h - 1; k >= l; --k) {
      double c, s;
      td_dec(td_rec_get(r0, cap0, r1, --p), c, s);
      const double uk = u[k];
      u[k + 1] = s * uk + c * uk1;
      uk1 = c * uk - s * uk1;
    }
    u[l] = uk1;
  }
}

}  // namespace peps

// Row f2: the vector-Jacobian product of the Kepler drift of every particle
// (the drift of a particle with no neighbours, Sec. 2.1.2) for the adjoint
// of the soft kick-drift-kick (the soft force's VJP is in direct.cu).
//
// The state-transition matrix comes from the forward map evaluated in dual
// numbers with six directions (one per input coordinate), the universal
// anomaly's derivative from one Newton step taken in dual arithmetic at the
// converged value (implicit-function theorem).
#include <math.h>

#include "p3t_internal.cuh"

namespace {

// ---- dual numbers with six directions ----------------------------------------
struct D6 {
  double v, d[6];
};
__device__ __forceinline__ D6 dc(double v) {
  D6 r;
  r.v = v;
  for (int i = 0; i < 6; ++i) r.d[i] = 0.0;
  return r;
}
__device__ __forceinline__ D6 operator+(const D6 &a, const D6 &b) {
  D6 r; r.v = a.v + b.v;
  for (int i = 0; i < 6; ++i) r.d[i] = a.d[i] + b.d[i];
  return r;
}
__device__ __forceinline__ D6 operator-(const D6 &a, const D6 &b) {
  D6 r; r.v = a.v - b.v;
  for (int i = 0; i < 6; ++i) r.d[i] = a.d[i] - b.d[i];
  return r;
}
__device__ __forceinline__ D6 operator*(const D6 &a, const D6 &b) {
  D6 r; r.v = a.v * b.v;
  for (int i = 0; i < 6; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i];
  return r;
}
__device__ __forceinline__ D6 operator*(double s, const D6 &a) {
  D6 r; r.v = s * a.v;
  for (int i = 0; i < 6; ++i) r.d[i] = s * a.d[i];
  return r;
}
__device__ __forceinline__ D6 operator+(double s, const D6 &a) {
  D6 r = a; r.v = s + a.v;
  return r;
}
__device__ __forceinline__ D6 operator/(const D6 &a, const D6 &b) {
  D6 r; r.v = a.v / b.v;
  const double ib = 1.0 / b.v;
  for (int i = 0; i < 6; ++i) r.d[i] = (a.d[i] - r.v * b.d[i]) * ib;
  return r;
}
__device__ __forceinline__ D6 dsqrt(const D6 &a) {
  D6 r; r.v = sqrt(a.v);
  const double h = 0.5 / r.v;
  for (int i = 0; i < 6; ++i) r.d[i] = a.d[i] * h;
  return r;
}
__device__ __forceinline__ D6 dfun(const D6 &a, double f, double df) {
  D6 r; r.v = f;
  for (int i = 0; i < 6; ++i) r.d[i] = df * a.d[i];
  return r;
}

// Stumpff functions C(z) = (1 - cos sqrt z) / z, S(z) = (sqrt z - sin sqrt z) /
// z^(3/2) (and their hyperbolic forms for z < 0); for |z| < 1 their series
// C = sum (-z)^k / (2k+2)!, S = sum (-z)^k / (2k+3)!, 12 terms (truncation
// below 1e-26)
__device__ void stumpff_d(const D6 &z, D6 &C, D6 &S) {
  if (fabs(z.v) < 1.0) {
    double cc[12], ss[12];
    double f = 2.0;  // (2k + 2)!
    for (int k = 0; k < 12; ++k) {
      if (k > 0) f *= (double)(2 * k + 1) * (double)(2 * k + 2);
      const double sign = (k & 1) ? -1.0 : 1.0;
      cc[k] = sign / f;
      ss[k] = sign / (f * (double)(2 * k + 3));
    }
    D6 c = dc(cc[11]), s = dc(ss[11]);
    for (int k = 10; k >= 0; --k) {
      c = dc(cc[k]) + z * c;
      s = dc(ss[k]) + z * s;
    }
    C = c;
    S = s;
  } else if (z.v > 0.0) {
    const D6 q = dsqrt(z);
    const D6 cq = dfun(q, cos(q.v), -sin(q.v)), sq = dfun(q, sin(q.v), cos(q.v));
    C = (dc(1.0) - cq) / z;
    S = (q - sq) / (z * q);
  } else {
    const D6 mz = dc(0.0) - z;
    const D6 q = dsqrt(mz);
    const D6 chq = dfun(q, cosh(q.v), sinh(q.v)), shq = dfun(q, sinh(q.v), cosh(q.v));
    C = (chq - dc(1.0)) / mz;
    S = (shq - q) / (mz * q);
  }
}

// the universal anomaly (values only), Newton from the series inversion
__device__ double chi_solve(double r0, double sig, double bet, double alpha, double tau,
                            double dt, double mu) {
  const double ir0 = 1.0 / r0, x1 = tau * ir0;
  double chi = x1 * (1.0 - 0.5 * sig * x1 * ir0 +
                     (0.5 * sig * sig * ir0 * ir0 - bet * ir0 / 6.0) * x1 * x1);
  if (alpha > 0.0 && 16.0 * dt * dt * alpha * alpha * alpha * mu > 4.0 * 9.869604401089358)
    chi = tau * alpha;
  for (int it = 0; it < 64; ++it) {
    const D6 zd = dc(alpha * chi * chi);
    D6 C, S;
    stumpff_d(zd, C, S);
    const double z = zd.v, chi2 = chi * chi;
    const double F = sig * chi2 * C.v + bet * chi2 * chi * S.v + r0 * chi - tau;
    const double Fp = sig * chi * (1.0 - z * S.v) + bet * chi2 * C.v + r0;
    double d = F / Fp;
    const double lim = 0.5 * (fabs(chi) + r0);
    d = d > lim ? lim : (d < -lim ? -lim : d);
    chi -= d;
    if (fabs(d) <= 1e-15 * fabs(chi) || d == 0.0) break;
  }
  return chi;
}

// lam_in = Phi^T lam_out for the drift of one particle by dt
__global__ void k_kepler_vjp(int64_t n, const double *x, const double *y, const double *z,
                             const double *vx, const double *vy, const double *vz, double dt,
                             double mu, double *lx, double *ly, double *lz, double *lvx,
                             double *lvy, double *lvz) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    D6 X[3] = {dc(x[i]), dc(y[i]), dc(z[i])}, V[3] = {dc(vx[i]), dc(vy[i]), dc(vz[i])};
    for (int a = 0; a < 3; ++a) { X[a].d[a] = 1.0; V[a].d[3 + a] = 1.0; }
    const double sq = sqrt(mu), isq = 1.0 / sq, imu = 1.0 / mu;
    const D6 r0 = dsqrt(X[0] * X[0] + X[1] * X[1] + X[2] * X[2]);
    const D6 v2 = V[0] * V[0] + V[1] * V[1] + V[2] * V[2];
    const D6 rv = X[0] * V[0] + X[1] * V[1] + X[2] * V[2];
    const D6 alpha = 2.0 * (dc(1.0) / r0) - imu * v2;
    const D6 sig = isq * rv;
    const D6 bet = dc(1.0) - alpha * r0;
    const double tau = sq * dt;
    const double chiv = chi_solve(r0.v, sig.v, bet.v, alpha.v, tau, dt, mu);
    // one Newton step in dual arithmetic at the converged value
    D6 chi = dc(chiv);
    {
      const D6 zz = alpha * chi * chi;
      D6 C, S;
      stumpff_d(zz, C, S);
      const D6 chi2 = chi * chi;
      const D6 F = sig * chi2 * C + bet * chi2 * chi * S + r0 * chi - dc(tau);
      const D6 Fp = sig * chi * (dc(1.0) - zz * S) + bet * chi2 * C + r0;
      chi = chi - F / Fp;
    }
    const D6 zz = alpha * chi * chi;
    D6 C, S;
    stumpff_d(zz, C, S);
    const D6 chi2 = chi * chi;
    const D6 f = dc(1.0) - chi2 * C / r0;
    const D6 g = dc(dt) - isq * (chi2 * chi * S);
    D6 nx[3];
    for (int a = 0; a < 3; ++a) nx[a] = f * X[a] + g * V[a];
    const D6 r = dsqrt(nx[0] * nx[0] + nx[1] * nx[1] + nx[2] * nx[2]);
    const D6 fd = sq * ((zz * S - dc(1.0)) * chi / (r * r0));
    const D6 gd = dc(1.0) - chi2 * C / r;
    D6 nv[3];
    for (int a = 0; a < 3; ++a) nv[a] = fd * X[a] + gd * V[a];
    const double lo[6] = {lx[i], ly[i], lz[i], lvx[i], lvy[i], lvz[i]};
    double li[6];
    for (int b = 0; b < 6; ++b) {
      double s = 0.0;
      for (int a = 0; a < 3; ++a) s += lo[a] * nx[a].d[b] + lo[3 + a] * nv[a].d[b];
      li[b] = s;
    }
    lx[i] = li[0]; ly[i] = li[1]; lz[i] = li[2];
    lvx[i] = li[3]; lvy[i] = li[4]; lvz[i] = li[5];
  }
}

}  // namespace

int p3t_run_kepler_vjp(p3t_ctx *c, const p3t_particles *p, double dt, double *lx, double *ly,
                       double *lz, double *lvx, double *lvy, double *lvz, cudaStream_t s) {
  const int64_t n = p->n;
  if (n == 0) return P3T_OK;
  k_kepler_vjp<<<(unsigned)p3t_grid(n, 128, (int64_t)c->num_sms * P3T_NSM_BLOCKS), 128, 0, s>>>(
      n, p->x, p->y, p->z, p->vx, p->vy, p->vz, dt, c->prm.G * c->prm.m_star, lx, ly, lz, lvx,
      lvy, lvz);
  p3t_note_launches(1);
  return cudaGetLastError() == cudaSuccess ? P3T_OK : P3T_ERR_CUDA;
}

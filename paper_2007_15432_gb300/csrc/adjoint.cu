// Adjoint: the vector-Jacobian product of the Kepler drift of every particle
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

// 1 / n! as a double (exact product of the integers up to 18!, then one
// rounding per factor)
__host__ __device__ constexpr double inv_fact(int n) {
  double f = 1.0;
  for (int i = 2; i <= n; ++i) f *= (double)i;
  return 1.0 / f;
}

// Stumpff functions C(z) = (1 - cos sqrt z) / z, S(z) = (sqrt z - sin sqrt z) /
// z^(3/2) (hyperbolic forms for z < 0) and their derivatives C', S' as plain
// numbers.  |z| < 1: the series C = sum (-z)^k / (2k+2)!, S = sum (-z)^k /
// (2k+3)! and their term-by-term derivatives, NT terms; otherwise the closed
// forms with C' = (1 - z S - 2C) / (2z), S' = (C - 3S) / (2z).
template <int NT>
__device__ __forceinline__ void stumpff_series(double z, double &C, double &S, double &dC,
                                               double &dS) {
  const double mz = -z;
  double c = inv_fact(2 * NT), s_ = inv_fact(2 * NT + 1);
  double dc_ = (double)(NT - 1) * c, ds_ = (double)(NT - 1) * s_;
#pragma unroll
  for (int k = NT - 2; k >= 0; --k) {
    c = fma(mz, c, inv_fact(2 * k + 2));
    s_ = fma(mz, s_, inv_fact(2 * k + 3));
    if (k >= 1) {
      dc_ = fma(mz, dc_, (double)k * inv_fact(2 * k + 2));
      ds_ = fma(mz, ds_, (double)k * inv_fact(2 * k + 3));
    }
  }
  C = c;
  S = s_;
  dC = -dc_;
  dS = -ds_;
}

__device__ void stumpff4(double z, double &C, double &S, double &dC, double &dS) {
  if (fabs(z) < 0.01) {
    stumpff_series<6>(z, C, S, dC, dS);  // truncation below |z|^6 / 14! ~ 1e-23
  } else if (fabs(z) < 1.0) {
    stumpff_series<12>(z, C, S, dC, dS);  // below 1 / 26! ~ 2.5e-27
  } else {
    if (z > 0.0) {
      const double q = sqrt(z);
      C = (1.0 - cos(q)) / z;
      S = (q - sin(q)) / (z * q);
    } else {
      const double q = sqrt(-z);
      C = (cosh(q) - 1.0) / (-z);
      S = (sinh(q) - q) / (-z * q);
    }
    const double i2z = 0.5 / z;
    dC = (1.0 - z * S - 2.0 * C) * i2z;
    dS = (C - 3.0 * S) * i2z;
  }
}

// C and S of a dual argument: values at z.v, derivatives by the chain rule
__device__ __forceinline__ void stumpff_d(const D6 &z, D6 &C, D6 &S) {
  double c, s_, dc_, ds_;
  stumpff4(z.v, c, s_, dc_, ds_);
  C = dfun(z, c, dc_);
  S = dfun(z, s_, ds_);
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
    const double z = alpha * chi * chi, chi2 = chi * chi;
    double C, S, dC, dS;
    stumpff4(z, C, S, dC, dS);
    const double F = sig * chi2 * C + bet * chi2 * chi * S + r0 * chi - tau;
    const double Fp = sig * chi * (1.0 - z * S) + bet * chi2 * C + r0;
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
  pdl_wait();
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
  pdl_launch(k_kepler_vjp, dim3((unsigned)p3t_grid(n, 128, (int64_t)c->num_sms * P3T_NSM_BLOCKS)), dim3(128), 0, s, 
      n, p->x, p->y, p->z, p->vx, p->vy, p->vz, dt, c->prm.G * c->prm.m_star, lx, ly, lz, lvx,
      lvy, lvz);
  p3t_note_launches(1);
  return cudaGetLastError() == cudaSuccess ? P3T_OK : P3T_ERR_CUDA;
}

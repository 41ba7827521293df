// Soft step: kick, Hermite-4 hard step of the neighbour
// clusters, Kepler drift of isolated particles, energy.
//
// Compiled with -fmad=false.  The Hermite force, predictor, corrector and
// step rule are evaluated in one fixed order with IEEE division and square
// root, so that the block-step schedule (decided by comparing FP64 step
// estimates with dt / 2^k) does not depend on the machine.
#include "p3t_internal.cuh"

namespace {

constexpr int kBlock = 256;

// ---- soft kick (procedure steps 3 and 8) ------------------------------------
// Members of a composite formed by the last hard step (Sec. 2.4.1;
// slot[i] >= 0, its entry in ent) are kicked with the composite's mass-
// weighted mean acceleration sum_l m_l a_l / sum_l m_l (ascending l); the
// composite's lowest member records the dissipation sum_l m_l |h (a_l -
// a_c)|^2 / 2 at its entry.
__global__ void k_kick(int64_t n, double *vx, double *vy, double *vz,
                       const double *ax, const double *ay, const double *az,
                       double h, const int32_t *slot, const int4 *ent, const double *m,
                       double *esoft) {
  pdl_wait();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t s = slot ? slot[i] : -1;
    if (s < 0) {
      vx[i] += ax[i] * h;
      vy[i] += ay[i] * h;
      vz[i] += az[i] * h;
      continue;
    }
    const int4 e = ent[s];
    double M = 0.0, A[3] = {0.0, 0.0, 0.0};
    for (int l = e.z; l < e.w; ++l) {
      const int q = ent[l].x;
      M += m[q];
      A[0] += m[q] * ax[q]; A[1] += m[q] * ay[q]; A[2] += m[q] * az[q];
    }
    const double ac[3] = {A[0] / M, A[1] / M, A[2] / M};
    vx[i] += ac[0] * h;
    vy[i] += ac[1] * h;
    vz[i] += ac[2] * h;
    if (e.x == e.y) {
      double Es = 0.0;
      for (int l = e.z; l < e.w; ++l) {
        const int q = ent[l].x;
        const double dx = (ax[q] - ac[0]) * h, dy = (ay[q] - ac[1]) * h, dz = (az[q] - ac[2]) * h;
        Es += 0.5 * m[q] * (dx * dx + dy * dy + dz * dz);
      }
      esoft[s] = Es;
    }
  }
}

// ---- Kepler drift, universal variables --------------------------------------
// Stumpff functions C(z) = sum (-z)^k / (2k+2)!, S(z) = sum (-z)^k / (2k+3)!,
// as nested series for |z| < 1 (4 terms below |z| = 1e-3, 6 below 1e-2, 10
// above; truncation below 1e-19 of the result in each band) and in closed
// form otherwise.
__device__ __forceinline__ void stumpff(double z, double &C, double &S) {
  constexpr double c0 = 1.0 / 2.0, c1 = -1.0 / 24.0, c2 = 1.0 / 720.0,
                   c3 = -1.0 / 40320.0, c4 = 1.0 / 3628800.0,
                   c5 = -1.0 / 479001600.0, c6 = 1.0 / 87178291200.0,
                   c7 = -1.0 / 20922789888000.0, c8 = 1.0 / 6402373705728000.0,
                   c9 = -1.0 / 2432902008176640000.0;
  constexpr double s0 = 1.0 / 6.0, s1 = -1.0 / 120.0, s2 = 1.0 / 5040.0,
                   s3 = -1.0 / 362880.0, s4 = 1.0 / 39916800.0,
                   s5 = -1.0 / 6227020800.0, s6 = 1.0 / 1307674368000.0,
                   s7 = -1.0 / 355687428096000.0, s8 = 1.0 / 121645100408832000.0,
                   s9 = -1.0 / 51090942171709440000.0;
  const double az = fabs(z);
  if (az < 1e-3) {
    double c = __fma_rn(z, c3, c2), s = __fma_rn(z, s3, s2);
    c = __fma_rn(z, c, c1); s = __fma_rn(z, s, s1);
    C = __fma_rn(z, c, c0); S = __fma_rn(z, s, s0);
  } else if (az < 1e-2) {
    double c = __fma_rn(z, c5, c4), s = __fma_rn(z, s5, s4);
    c = __fma_rn(z, c, c3); s = __fma_rn(z, s, s3);
    c = __fma_rn(z, c, c2); s = __fma_rn(z, s, s2);
    c = __fma_rn(z, c, c1); s = __fma_rn(z, s, s1);
    C = __fma_rn(z, c, c0); S = __fma_rn(z, s, s0);
  } else if (az < 1.0) {
    double c = __fma_rn(z, c9, c8), s = __fma_rn(z, s9, s8);
    c = __fma_rn(z, c, c7); s = __fma_rn(z, s, s7);
    c = __fma_rn(z, c, c6); s = __fma_rn(z, s, s6);
    c = __fma_rn(z, c, c5); s = __fma_rn(z, s, s5);
    c = __fma_rn(z, c, c4); s = __fma_rn(z, s, s4);
    c = __fma_rn(z, c, c3); s = __fma_rn(z, s, s3);
    c = __fma_rn(z, c, c2); s = __fma_rn(z, s, s2);
    c = __fma_rn(z, c, c1); s = __fma_rn(z, s, s1);
    C = __fma_rn(z, c, c0); S = __fma_rn(z, s, s0);
  } else if (z > 0.0) {
    const double q = sqrt(z);
    C = (1.0 - cos(q)) / z;
    S = (q - sin(q)) / (z * q);
  } else {
    const double q = sqrt(-z);
    C = (cosh(q) - 1.0) / (-z);
    S = (sinh(q) - q) / (-z * q);
  }
}

// Per-call constants of the drift: mu, sqrt(mu), 1 / sqrt(mu), 1 / mu.
struct KepConst {
  double mu, sq, isq, imu;
};

// Advances (X, V) by dt on the Kepler orbit about mu.  Universal anomaly chi
// solves F(chi) = sig chi^2 C + (1 - alpha r0) chi^3 S + r0 chi - sqrt(mu) dt
// = 0 (z = alpha chi^2, sig = r0 v_r0 / sqrt(mu)) by Newton-Raphson from the
// third-order series inversion of F; F'(chi) = r(chi) and F''(chi) = sig (1 -
// z C) + (1 - alpha r0) chi (1 - z S).  A Newton step d leaves an error of
// about |F'' / (2 F')| d^2, so the iteration stops once 16 times that bound
// is below 2^-53 |chi| (or |d| <= 1e-10 |chi|).  Then Lagrange f, g.
__device__ bool kepler_uv(double X[3], double V[3], double dt, const KepConst &K) {
  const double r02 = __fma_rn(X[0], X[0], __fma_rn(X[1], X[1], X[2] * X[2]));
  const double v2 = __fma_rn(V[0], V[0], __fma_rn(V[1], V[1], V[2] * V[2]));
  const double rv = __fma_rn(X[0], V[0], __fma_rn(X[1], V[1], X[2] * V[2]));
  const double ir0 = rsqrt(r02);
  const double r0 = r02 * ir0;
  const double alpha = __fma_rn(-v2, K.imu, 2.0 * ir0);
  const double sig = rv * K.isq;  // r0 v_r0 / sqrt(mu)
  const double tau = K.sq * dt;
  const double bet = __fma_rn(-alpha, r0, 1.0);
  // inversion of tau = r0 chi + sig chi^2 / 2 + bet chi^3 / 6 + O(chi^4)
  const double x1 = tau * ir0, hs = 0.5 * sig * ir0;
  double chi = x1 * __fma_rn(__fma_rn(hs, hs + hs, -bet * ir0 * (1.0 / 6.0) * ir0), x1 * x1,
                             __fma_rn(-hs, x1, 1.0));
  // beyond a quarter period (16 dt^2 alpha^3 mu > (2 pi)^2) start from the mean motion
  if (alpha > 0.0 && 16.0 * dt * dt * alpha * alpha * alpha * K.mu > 4.0 * 9.869604401089358)
    chi = tau * alpha;
  double C = 0.5, S = 1.0 / 6.0, z = 0.0;
  bool ok = false;
  for (int it = 0; it < 64; ++it) {
    z = alpha * chi * chi;
    stumpff(z, C, S);
    const double chi2 = chi * chi;
    const double F = __fma_rn(sig * chi2, C, __fma_rn(bet * chi2 * chi, S, __fma_rn(r0, chi, -tau)));
    const double Fp = __fma_rn(sig * chi, __fma_rn(-z, S, 1.0), __fma_rn(bet * chi2, C, r0));
    const double Fpp = __fma_rn(sig, __fma_rn(-z, C, 1.0), bet * chi * __fma_rn(-z, S, 1.0));
    const double iFp = 1.0 / Fp;
    double d = F * iFp;
    const double lim = 0.5 * (fabs(chi) + r0);
    if (d > lim) d = lim;
    if (d < -lim) d = -lim;
    chi -= d;
    const double rest = 0.5 * fabs(Fpp * iFp) * d * d;
    if (16.0 * rest <= 1.1102230246251565e-16 * fabs(chi) || fabs(d) <= 1e-10 * fabs(chi) ||
        d == 0.0) {
      ok = true;
      break;
    }
  }
  z = alpha * chi * chi;
  stumpff(z, C, S);
  const double chi2 = chi * chi;
  const double f = __fma_rn(-chi2 * ir0, C, 1.0);
  const double g = __fma_rn(-chi2 * chi, S * K.isq, dt);
  double nx[3];
  for (int a = 0; a < 3; ++a) nx[a] = __fma_rn(f, X[a], g * V[a]);
  const double ir = rsqrt(__fma_rn(nx[0], nx[0], __fma_rn(nx[1], nx[1], nx[2] * nx[2])));
  const double fd = K.sq * ir * ir0 * __fma_rn(z, S, -1.0) * chi;
  const double gd = __fma_rn(-chi2 * ir, C, 1.0);
  for (int a = 0; a < 3; ++a) {
    const double nv = __fma_rn(fd, X[a], gd * V[a]);
    X[a] = nx[a];
    V[a] = nv;
  }
  return ok;
}

__device__ __forceinline__ double ldexp_fast(double x, int k) {
  const long long b = __double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7ff);
  if (e > 0 && e < 0x7ff && e + k > 0 && e + k < 0x7ff)
    return __longlong_as_double(b + ((long long)k << 52));
  return ldexp(x, k);
}
__device__ __forceinline__ int ilogb_fast(double x) {
  const int e = (int)((__double_as_longlong(x) >> 52) & 0x7ff);
  return (e > 0 && e < 0x7ff) ? e - 1023 : ilogb(x);
}

// Conversions by integer operations.  On this part a conversion between FP64
// and FP32 or from an integer to FP64 takes the FP64 pipe like an FP64
// multiply (about 64 cycles of a sub-partition); along the serial block steps
// of a close encounter these sit on the critical path, so where the result is
// a normal number they are done on the bits instead, with the same results.
// (float)(a 2^k), rounded to nearest even, for a 2^k in FP32's normal range
// (the FP64 forms of the rare cases out of line: inlined, the compiler
// predicates them into every call, and predicated-off FP64 instructions still
// take the FP64 pipe)
__device__ __noinline__ float d2f_scaled_fp64(double a, int k) { return (float)ldexp_fast(a, k); }
__device__ __noinline__ double f2d_fp64(float f) { return (double)f; }
__device__ __noinline__ double i2d_fp64(int64_t x) { return (double)x; }
__device__ __forceinline__ float d2f_scaled(double a, int k) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(a);
  const int ed = (int)((b >> 52) & 0x7ff);
  const int ef = ed - 1023 + k + 127;
  if (ed == 0 || ed == 0x7ff || ef <= 0 || ef >= 255) return d2f_scaled_fp64(a, k);
  const unsigned long long m = b & 0xfffffffffffffull;
  unsigned r = ((unsigned)ef << 23) | (unsigned)(m >> 29);
  const unsigned long long rem = m & 0x1fffffffull, half = 0x10000000ull;
  if (rem > half || (rem == half && (r & 1u))) ++r;  // a carry into the exponent is right
  return __uint_as_float(r | ((unsigned)(b >> 32) & 0x80000000u));
}
// (double)f, exact
__device__ __forceinline__ double f2d_exact(float f) {
  const unsigned u = __float_as_uint(f);
  const int ef = (int)((u >> 23) & 0xff);
  if (ef == 0 || ef == 0xff) return f2d_fp64(f);
  return __longlong_as_double((long long)((unsigned long long)(u & 0x80000000u) << 32 |
                                          (unsigned long long)(ef - 127 + 1023) << 52 |
                                          (unsigned long long)(u & 0x7fffffu) << 29));
}
// (double)x for 0 <= x < 2^53, exact
__device__ __forceinline__ double i2d_exact(int64_t x) {
  if (x <= 0) return i2d_fp64(x);
  const int e = 63 - __clzll(x);
  return __longlong_as_double((long long)((unsigned long long)(e + 1023) << 52 |
                                          (((unsigned long long)x << (52 - e)) &
                                           0xfffffffffffffull)));
}

// Mixed path: the same drift in float-float arithmetic (FP32 instructions,
// ~2^-47 relative per operation) for bound orbits whose Stumpff argument
// stays below 1e-2 (a soft step is a small fraction of an orbit): the same
// universal-anomaly equation, the third-order start, Newton steps until the
// step is below 2^-44 of chi, Stumpff series to z^4 (the next term is below
// 1e-19 of the first), Lagrange f, g.  The FP64 pipe then carries only the
// splits of the state into float-float pairs and back.  Anything else (an
// unbound or long arc, no convergence in four steps) returns false and takes
// the FP64 solver, on the untouched state.  The drift's results agree with
// the FP64 solver's to ~1e-14 relative.
struct KepFF {
  FF sq, isq, imu;
};
// x = hi + lo with hi = (float)x and lo = (float)(x - hi) (the difference
// exact); the conversions on the bits, one FP64 subtraction
__device__ __forceinline__ FF ff_split(double x) {
  const float h = d2f_scaled(x, 0);
  return {h, d2f_scaled(x - f2d_exact(h), 0)};
}
__device__ __forceinline__ double ff_to_double(FF a) { return f2d_exact(a.h) + f2d_exact(a.l); }
__device__ __forceinline__ FF ff_sub(FF a, FF b) { return ff_add(a, ff_neg(b)); }
__device__ __forceinline__ FF ff_c(float h, float l) { return {h, l}; }
// the Stumpff series' coefficients as float-float constants
#define P3T_FFC(name, v) constexpr float name##h = (float)(v), name##l = (float)((v) - (double)(float)(v))
P3T_FFC(kC0, 1.0 / 2.0); P3T_FFC(kC1, -1.0 / 24.0); P3T_FFC(kC2, 1.0 / 720.0);
P3T_FFC(kC3, -1.0 / 40320.0); P3T_FFC(kC4, 1.0 / 3628800.0);
P3T_FFC(kS0, 1.0 / 6.0); P3T_FFC(kS1, -1.0 / 120.0); P3T_FFC(kS2, 1.0 / 5040.0);
P3T_FFC(kS3, -1.0 / 362880.0); P3T_FFC(kS4, 1.0 / 39916800.0);
#undef P3T_FFC
__device__ __forceinline__ void stumpff_ff(FF z, FF &C, FF &S) {
  FF c = ff_add(ff_c(kC3h, kC3l), ff_mul(z, ff_c(kC4h, kC4l)));
  FF t = ff_add(ff_c(kS3h, kS3l), ff_mul(z, ff_c(kS4h, kS4l)));
  c = ff_add(ff_c(kC2h, kC2l), ff_mul(z, c)); t = ff_add(ff_c(kS2h, kS2l), ff_mul(z, t));
  c = ff_add(ff_c(kC1h, kC1l), ff_mul(z, c)); t = ff_add(ff_c(kS1h, kS1l), ff_mul(z, t));
  C = ff_add(ff_c(kC0h, kC0l), ff_mul(z, c)); S = ff_add(ff_c(kS0h, kS0l), ff_mul(z, t));
}

__device__ bool kepler_ff(double X[3], double V[3], double dt, const KepFF &K) {
  const FF x[3] = {ff_split(X[0]), ff_split(X[1]), ff_split(X[2])};
  const FF v[3] = {ff_split(V[0]), ff_split(V[1]), ff_split(V[2])};
  const FF r02 = ff_add(ff_add(ff_mul(x[0], x[0]), ff_mul(x[1], x[1])), ff_mul(x[2], x[2]));
  const FF v2 = ff_add(ff_add(ff_mul(v[0], v[0]), ff_mul(v[1], v[1])), ff_mul(v[2], v[2]));
  const FF rv = ff_add(ff_add(ff_mul(x[0], v[0]), ff_mul(x[1], v[1])), ff_mul(x[2], v[2]));
  const FF ir0 = ff_rsqrt(r02);
  const FF r0 = ff_mul(r02, ir0);
  const FF alpha = ff_sub(ff_mulf(ir0, 2.0f), ff_mul(v2, K.imu));
  const FF sig = ff_mul(rv, K.isq);
  const FF dtf = ff_split(dt);
  const FF tau = ff_mul(K.sq, dtf);
  const FF bet = ff_sub(ff_c(1.0f, 0.0f), ff_mul(alpha, r0));
  // inversion of tau = r0 chi + sig chi^2 / 2 + bet chi^3 / 6 + O(chi^4)
  const FF x1 = ff_mul(tau, ir0), hs = ff_mulf(ff_mul(sig, ir0), 0.5f);
  const FF q = ff_sub(ff_mulf(ff_mul(hs, hs), 2.0f),
                      ff_mulf(ff_mul(ff_mul(bet, ir0), ir0), 1.0f / 6.0f));
  FF chi = ff_mul(x1, ff_add(ff_sub(ff_c(1.0f, 0.0f), ff_mul(hs, x1)),
                             ff_mul(q, ff_mul(x1, x1))));
  if (!(alpha.h > 0.0f)) return false;
  FF z = ff_mul(alpha, ff_mul(chi, chi)), C, S;
  bool conv = false;
  for (int it = 0; it < 4; ++it) {
    if (!(fabsf(z.h) < 1e-2f)) return false;
    stumpff_ff(z, C, S);
    const FF chi2 = ff_mul(chi, chi);
    const FF F = ff_sub(ff_add(ff_add(ff_mul(ff_mul(sig, chi2), C),
                                      ff_mul(ff_mul(bet, ff_mul(chi2, chi)), S)),
                               ff_mul(r0, chi)),
                        tau);
    const FF Fp = ff_add(ff_add(ff_mul(ff_mul(sig, chi), ff_sub(ff_c(1.0f, 0.0f), ff_mul(z, S))),
                                ff_mul(ff_mul(bet, chi2), C)),
                         r0);
    const FF d = ff_div(F, Fp);
    chi = ff_sub(chi, d);
    z = ff_mul(alpha, ff_mul(chi, chi));
    if (fabsf(d.h) <= 5.684341886080802e-14f * fabsf(chi.h)) {  // 2^-44
      conv = true;
      break;
    }
  }
  if (!conv || !(fabsf(z.h) < 1e-2f)) return false;
  stumpff_ff(z, C, S);
  const FF chi2 = ff_mul(chi, chi);
  const FF f = ff_sub(ff_c(1.0f, 0.0f), ff_mul(ff_mul(chi2, ir0), C));
  const FF g = ff_sub(dtf, ff_mul(ff_mul(chi2, chi), ff_mul(S, K.isq)));
  FF nx[3];
  for (int a = 0; a < 3; ++a) nx[a] = ff_add(ff_mul(f, x[a]), ff_mul(g, v[a]));
  const FF ir = ff_rsqrt(
      ff_add(ff_add(ff_mul(nx[0], nx[0]), ff_mul(nx[1], nx[1])), ff_mul(nx[2], nx[2])));
  const FF fd = ff_mul(ff_mul(ff_mul(K.sq, ir), ir0),
                       ff_mul(ff_sub(ff_mul(z, S), ff_c(1.0f, 0.0f)), chi));
  const FF gd = ff_sub(ff_c(1.0f, 0.0f), ff_mul(ff_mul(chi2, ir), C));
  for (int a = 0; a < 3; ++a) {
    const FF nv = ff_add(ff_mul(fd, x[a]), ff_mul(gd, v[a]));
    X[a] = ff_to_double(nx[a]);
    V[a] = ff_to_double(nv);
  }
  return true;
}

__device__ __forceinline__ KepFF kep_ff(const KepConst &K) {
  return {ff_split(K.sq), ff_split(K.isq), ff_split(K.imu)};
}

template <bool MIXED>
__global__ void k_kepler(const int64_t *d_nsingle, const int32_t *singles,
                         p3t_particles p, double dt, KepConst K, DevStatus *st) {
  pdl_wait();
  const int64_t ns = *d_nsingle;
  KepFF KF;
  if constexpr (MIXED) KF = kep_ff(K);
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < ns;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int32_t i = singles[k];
    double X[3] = {p.x[i], p.y[i], p.z[i]}, V[3] = {p.vx[i], p.vy[i], p.vz[i]};
    bool done = false;
    if constexpr (MIXED) done = kepler_ff(X, V, dt, KF);
    if (!done && !kepler_uv(X, V, dt, K)) dev_fail(st, P3T_ERR_TIMEOUT, 60, 0);
    p.x[i] = X[0]; p.y[i] = X[1]; p.z[i] = X[2];
    p.vx[i] = V[0]; p.vy[i] = V[1]; p.vz[i] = V[2];
  }
}

// every particle of p (p3t_kepler_drift)
template <bool MIXED>
__global__ void k_kepler_all(p3t_particles p, double dt, KepConst K, DevStatus *st) {
  pdl_wait();
  KepFF KF;
  if constexpr (MIXED) KF = kep_ff(K);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < p.n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double X[3] = {p.x[i], p.y[i], p.z[i]}, V[3] = {p.vx[i], p.vy[i], p.vz[i]};
    bool done = false;
    if constexpr (MIXED) done = kepler_ff(X, V, dt, KF);
    if (!done && !kepler_uv(X, V, dt, K)) dev_fail(st, P3T_ERR_TIMEOUT, 60, 0);
    p.x[i] = X[0]; p.y[i] = X[1]; p.z[i] = X[2];
    p.vx[i] = V[0]; p.vy[i] = V[1]; p.vz[i] = V[2];
  }
}

// ---- Hermite-4 with block steps (+ collisions), one block per cluster ------
// Clusters of up to 32 members (nearly all) run one warp each, so that the
// FP64 instructions of their few work items are not spread over idle lanes
// of several warps; clusters of 33 to 128 members run one 128-thread block
// each, their work items (member components, or (active member, source)
// terms) dealt round-robin over the four warps so that one long cluster keeps
// the FP64 pipes of all four SM sub-partitions busy.  Each active member's
// force is the sum, in the fixed order star term first then sources in
// ascending index, of terms computed in parallel (state in shared memory) or,
// above 128 members, by one thread per member (state in a global workspace).
//
// Perfect accretion (Sec. 2.4.1; on when f_radius > 0 and physical
// radii are given): at every force evaluation each evaluated member records
// the lowest-index member outside its composite that it touches, r < f (R_k
// + R_j).  After the correction the touching members (with the composites
// they belong to) become one composite: centre-of-mass position and velocity
// at the block time, hard force and jerk the mass-weighted mean over the
// composite with its inner pairs left out, a first step eta0 |a| / |j|.  The
// dissipated energy is the change of the affected members' kinetic, star and
// pair energy (changeover functions replaced by unity, the cluster standing
// for the neighbours).  One thread does this bookkeeping in a fixed order;
// collisions are rare.
constexpr int kHMax = 128;  // largest cluster kept in shared memory
// the largest cluster integrated by one warp is a launch-shape choice
// (p3t_set_tuning; 8 by default): larger ones take a block of four warps,
// whose pair terms then run on four sub-partitions' FP64 pipes.  The one-warp
// kernel is compiled for clusters of up to 8, 16 and 32 members (its shared
// memory grows with the bound, so the smallest that fits is launched).
constexpr int32_t kNone = 0x7fffffff;  // no collision partner

template <int KM>
struct HSmall {  // a cluster of <= KM members
  double x[3][KM], v[3][KM], a[3][KM], j[3][KM];
  double p[3][KM], pv[3][KM];
  double a1[3][KM], j1[3][KM], a2e[3][KM], a3[3][KM];
  double m[KM], iro[KM], rp[KM];
  // one batch of pair terms: B = NT / (nc + 1) members x (nc + 1) terms, at
  // most NT (a batch is one pass of the block's threads), and at least the
  // nc + 1 terms of one member
  static constexpr int kT = KM + 1 > 32 ? KM + 1 : 32;
  double T[kT][6];
  int64_t t[KM];
  int32_t lvl[KM], act[KM], set[KM], nset[KM], partner[KM], chg[KM];
};

static_assert(sizeof(HSmall<kHMax>) <= 48 * 1024,
              "HSmall must fit the default dynamic shared memory");

struct HCtl {  // per-block control, shared memory
  int64_t red[2][4];
  int32_t wcount[4];
  int64_t cluster;
  int nact, any, ncomp, stop;
  double edisp;
};

template <int KM>
struct SmallView {
  HSmall<KM> *S;
  static constexpr bool kBig = false;
  __device__ double &x(int q, int k) const { return S->x[q][k]; }
  __device__ double &v(int q, int k) const { return S->v[q][k]; }
  __device__ double &a(int q, int k) const { return S->a[q][k]; }
  __device__ double &j(int q, int k) const { return S->j[q][k]; }
  __device__ double &p(int q, int k) const { return S->p[q][k]; }
  __device__ double &pv(int q, int k) const { return S->pv[q][k]; }
  __device__ double &a1(int q, int k) const { return S->a1[q][k]; }
  __device__ double &j1(int q, int k) const { return S->j1[q][k]; }
  __device__ double &a2e(int q, int k) const { return S->a2e[q][k]; }
  __device__ double &a3(int q, int k) const { return S->a3[q][k]; }
  __device__ double &m(int k) const { return S->m[k]; }
  __device__ double &iro(int k) const { return S->iro[k]; }
  __device__ double &rp(int k) const { return S->rp[k]; }
  __device__ int64_t &t(int k) const { return S->t[k]; }
  __device__ int32_t &lvl(int k) const { return S->lvl[k]; }
  __device__ int32_t &act(int k) const { return S->act[k]; }
  __device__ int32_t &set(int k) const { return S->set[k]; }
  __device__ int32_t &nset(int k) const { return S->nset[k]; }
  __device__ int32_t &partner(int k) const { return S->partner[k]; }
  __device__ int32_t &chg(int k) const { return S->chg[k]; }
};

// global workspace of the large clusters: 33 double, 1 int64 and 6 int32
// arrays of cap entries, a cluster's members at its member offset
struct HBig {
  double *d;
  int64_t *t;
  int32_t *i;
  int64_t cap;
};
struct BigView {
  double *d;
  int64_t *tt;
  int32_t *ii;
  int64_t cap, off;
  static constexpr bool kBig = true;
  __device__ double &D(int arr, int k) const { return d[arr * cap + off + k]; }
  __device__ int32_t &I(int arr, int k) const { return ii[arr * cap + off + k]; }
  __device__ double &x(int q, int k) const { return D(q, k); }
  __device__ double &v(int q, int k) const { return D(3 + q, k); }
  __device__ double &a(int q, int k) const { return D(6 + q, k); }
  __device__ double &j(int q, int k) const { return D(9 + q, k); }
  __device__ double &p(int q, int k) const { return D(12 + q, k); }
  __device__ double &pv(int q, int k) const { return D(15 + q, k); }
  __device__ double &a1(int q, int k) const { return D(18 + q, k); }
  __device__ double &j1(int q, int k) const { return D(21 + q, k); }
  __device__ double &a2e(int q, int k) const { return D(24 + q, k); }
  __device__ double &a3(int q, int k) const { return D(27 + q, k); }
  __device__ double &m(int k) const { return D(30, k); }
  __device__ double &iro(int k) const { return D(31, k); }
  __device__ double &rp(int k) const { return D(32, k); }
  __device__ int64_t &t(int k) const { return tt[off + k]; }
  __device__ int32_t &lvl(int k) const { return I(0, k); }
  __device__ int32_t &act(int k) const { return I(1, k); }
  __device__ int32_t &set(int k) const { return I(2, k); }
  __device__ int32_t &nset(int k) const { return I(3, k); }
  __device__ int32_t &partner(int k) const { return I(4, k); }
  __device__ int32_t &chg(int k) const { return I(5, k); }
};

// composites handed to the kick and the merge (Sec. 2.4.1)
struct CollOut {
  unsigned long long *ctr;  // (records << 32) | entries
  int4 *ent;                // {particle, lowest member of its composite, lo, hi}
  int4 *rec;                // {cluster label, first entry, entries, 0}
  double *rec_e;            // energy dissipated in the cluster
  int32_t *slot;            // particle -> its entry, or -1
  int64_t ent_cap, rec_cap;
};

// x 2^k and ilogb(x) read from and written to the exponent field with integer
// operations when x (and the result) are normal -- the same values as ldexp
// and ilogb, without an FP64 instruction (one costs 64 cycles of a
// sub-partition's FP64 pipe on this part) -- and by ldexp / ilogb otherwise.
// The step estimates only choose a power-of-two step: formed in FP32 from
// components scaled by an exact power of two 2^k (j by s, a2 by s^2, a3 by
// s^3, s = 2^e close to the step) so that nothing overflows FP32.
__device__ __forceinline__ float norm3f(double a, double b, double c, int k) {
  const float x = d2f_scaled(a, k), y = d2f_scaled(b, k), z = d2f_scaled(c, k);
  return sqrtf(x * x + y * y + z * z);
}

// largest dt / 2^lvl not above dt_des, at most twice the previous step, and
// commensurate with the current time t (units of dt / 2^40).  The search
// starts at a lower bound from the binary exponents and t's trailing zeros
// give the commensurability level directly; the result is the same as
// stepping lvl up one at a time.
__device__ __forceinline__ int quantise_level(double dt_des, double dt, int prev,
                                              int64_t t, bool &underflow) {
  int lvl = 0;
  const long long bd = __double_as_longlong(dt), bs = __double_as_longlong(dt_des);
  const int edt = (int)((bd >> 52) & 0x7ff);
  if (bd > 0 && edt > P3T_KMAX && edt < 0x7ff &&
      (bs & 0x7fffffffffffffffLL) <= 0x7ff0000000000000LL) {
    // dt positive and normal down to dt / 2^KMAX, dt_des not NaN: as integers
    // the bit patterns order like the values (negative dt_des, -0 included,
    // below every positive one), and dt / 2^l is dt's pattern less l << 52
    if (bs > 0 && bs < bd) {
      int l0 = ilogb_fast(dt) - ilogb_fast(dt_des) - 1;  // dt / 2^l > dt_des for l <= l0
      lvl = l0 < 0 ? 0 : (l0 > P3T_KMAX ? P3T_KMAX : l0);
    }
    while (lvl < P3T_KMAX && bd - ((long long)lvl << 52) > bs) ++lvl;
    if (bd - ((long long)lvl << 52) > bs) underflow = true;
  } else {
    if (dt_des > 0.0 && dt_des < dt) {
      int l0 = ilogb(dt) - ilogb(dt_des) - 1;
      lvl = l0 < 0 ? 0 : (l0 > P3T_KMAX ? P3T_KMAX : l0);
    }
    while (lvl < P3T_KMAX && ldexp(dt, -lvl) > dt_des) ++lvl;
    if (ldexp(dt, -lvl) > dt_des) underflow = true;
  }
  if (lvl < prev - 1) lvl = prev - 1;
  if (t != 0) {
    const int need = P3T_KMAX - __ffsll((long long)t) + 1;  // 2^(40-lvl) must divide t
    if (lvl < need) lvl = need;
  }
  return lvl > P3T_KMAX ? P3T_KMAX : lvl;
}

// first step eta0 |a| / |j| = (eta0 |a| / |j s|) s, s = 2^e
template <class V>
__device__ __forceinline__ int first_level(const V &S, int k, const p3t_params &prm, double dt,
                                           int64_t t, bool &underflow) {
  const int e = ilogb_fast(dt);
  const float an = norm3f(S.a(0, k), S.a(1, k), S.a(2, k), 0);
  const float jn = norm3f(S.j(0, k), S.j(1, k), S.j(2, k), e);
  const double dtd = jn > 0.0f ? ldexp_fast(f2d_exact((float)prm.eta0 * an / jn), e) : dt;
  return quantise_level(dtd, dt, 0, t, underflow);
}

// term of source j (j == nc: the star) on member k at the block-time state
// (p, pv): the (1 - K) pair force and its jerk (Eq. hardforce), one
// reciprocal square root per pair, 1/max(r_out) taken as min(1/r_out).  The
// star is a source at the origin, at rest, of mass M_*, with 1/r_out = 0 (so
// y = 0: no changeover): the same instructions then give exactly the star
// term -G M_* x / |x|^3 and its jerk, with no divergent path.  Members of k's
// own composite are left out; with `detect`, hit reports contact r < f (R_k +
// R_j) with another member.
template <class V>
__device__ __forceinline__ void hard_term(const V &S, int nc, int k, int j,
                                          const p3t_params &prm, double i1mg, bool detect,
                                          double out[6], bool &hit) {
  for (int q = 0; q < 6; ++q) out[q] = 0.0;
  hit = false;
  const bool star = j == nc;
  if (!star && (j == k || S.set(j) == S.set(k))) return;
  const int js = star ? k : j;  // an index that can be read
  const double xk = S.p(0, k), yk = S.p(1, k), zk = S.p(2, k);
  const double vxk = S.pv(0, k), vyk = S.pv(1, k), vzk = S.pv(2, k);
  const double rx = xk - (star ? 0.0 : S.p(0, js)), ry = yk - (star ? 0.0 : S.p(1, js)),
               rz = zk - (star ? 0.0 : S.p(2, js));
  const double ux = vxk - (star ? 0.0 : S.pv(0, js)), uy = vyk - (star ? 0.0 : S.pv(1, js)),
               uz = vzk - (star ? 0.0 : S.pv(2, js));
  const double r2 = __fma_rn(rx, rx, __fma_rn(ry, ry, rz * rz));
  if (detect && !star) {
    const double sr = prm.f_radius * (S.rp(k) + S.rp(js));
    hit = r2 < sr * sr;
  }
  if (r2 == 0.0) return;
  const double rinv = rsqrt(r2);
  const double r = r2 * rinv;
  const double irot = star ? 0.0 : (S.iro(k) < S.iro(js) ? S.iro(k) : S.iro(js));
  const double yv = r * irot;
  if (yv >= 1.0) return;
  double w = 1.0, dK = 0.0;
  if (yv > prm.gamma) {
    const double xs = (yv - prm.gamma) * i1mg;
    const double x2 = xs * xs, x3 = x2 * xs, x4 = x2 * x2, u = 1.0 - xs;
    w = 1.0 - x4 * (35.0 - 84.0 * xs + 70.0 * x2 - 20.0 * x3);
    dK = 140.0 * x3 * (u * u * u) * i1mg;
  }
  const double rinv2 = rinv * rinv;
  const double g3 = prm.G * (star ? prm.m_star : S.m(js)) * (rinv2 * rinv);
  const double f = g3 * w;
  const double rv = __fma_rn(rx, ux, __fma_rn(ry, uy, rz * uz));
  out[0] = f * rx; out[1] = f * ry; out[2] = f * rz;
  const double c = __fma_rn(dK * rv * rinv, irot, 3.0 * w * rv * rinv2);
  out[3] = g3 * __fma_rn(-c, rx, w * ux);
  out[4] = g3 * __fma_rn(-c, ry, w * uy);
  out[5] = g3 * __fma_rn(-c, rz, w * uz);
}

// the members with pred(k), ascending, into act[0..); returns their number
template <int NT, class V, class Pred>
__device__ int build_list(const V &S, HCtl &C, int nc, Pred pred) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  int base = 0;
  for (int c0 = 0; c0 < nc; c0 += NT) {
    const int k = c0 + tid;
    const bool on = k < nc && pred(k);
    const unsigned bal = __ballot_sync(0xffffffffu, on);
    if (lane == 0) C.wcount[warp] = __popc(bal);
    __syncthreads();
    int off = base, tot = 0;
    for (int q = 0; q < NT / 32; ++q) {
      if (q < warp) off += C.wcount[q];
      tot += C.wcount[q];
    }
    if (on) S.act(off + __popc(bal & ((1u << lane) - 1u))) = k;
    base += tot;
    __syncthreads();
  }
  return base;
}

// forces on the listed members act[0..nact) from (p, pv) into (a1, j1); with
// `detect`, each one's lowest touching partner into partner[]; then the
// composites' mean force
template <int NT, class V>
__device__ void block_forces(const V &S, HCtl &C, double (*Tb)[6], int nc, int nact, int item,
                             const p3t_params &prm, double i1mg, bool detect) {
  if constexpr (!V::kBig) {
    const int per = nc + 1;
    const int B = NT / per > 0 ? NT / per : 1;  // members per batch
    for (int b0 = 0; b0 < nact; b0 += B) {
      const int nb = min(B, nact - b0);
      const int items = nb * per;
      for (int i = item; i < items; i += NT) {
        const int bm = i / per, jj = i - bm * per;
        const int k = S.act(b0 + bm);
        bool hit;
        hard_term(S, nc, k, jj, prm, i1mg, detect, Tb[i], hit);
        if (hit) atomicMin(&S.partner(k), jj);
      }
      __syncthreads();
      for (int i = item; i < nb * 6; i += NT) {
        const int bm = i / 6, q = i - bm * 6;
        const int k = S.act(b0 + bm);
        const int base = bm * per;
        double acc = 0.0;
        acc -= Tb[base + nc][q];
        for (int jj = 0; jj < nc; ++jj) acc -= Tb[base + jj][q];
        if (q < 3) S.a1(q, k) = acc; else S.j1(q - 3, k) = acc;
      }
      __syncthreads();
    }
  } else {
    for (int b = threadIdx.x; b < nact; b += NT) {
      const int k = S.act(b);
      double acc[6], out[6];
      bool hit;
      hard_term(S, nc, k, nc, prm, i1mg, false, out, hit);
      for (int q = 0; q < 6; ++q) acc[q] = 0.0 - out[q];
      for (int jj = 0; jj < nc; ++jj) {
        hard_term(S, nc, k, jj, prm, i1mg, detect, out, hit);
        for (int q = 0; q < 6; ++q) acc[q] -= out[q];
        if (hit && S.partner(k) == kNone) S.partner(k) = jj;
      }
      for (int q = 0; q < 3; ++q) { S.a1(q, k) = acc[q]; S.j1(q, k) = acc[3 + q]; }
    }
    __syncthreads();
  }
  if (C.ncomp) {
    // composite force: sum_l m_l a_l / sum_l m_l, ascending l (sets of >= 2)
    for (int b = item; b < nact; b += NT) {
      const int r = S.act(b);
      if (S.set(r) != r) continue;
      int size = 0;
      double M = 0.0, A[3] = {0, 0, 0}, J[3] = {0, 0, 0};
      for (int l = 0; l < nc; ++l) {
        if (S.set(l) != r) continue;
        ++size;
        M += S.m(l);
        for (int q = 0; q < 3; ++q) { A[q] += S.m(l) * S.a1(q, l); J[q] += S.m(l) * S.j1(q, l); }
      }
      if (size < 2) continue;
      for (int l = 0; l < nc; ++l) {
        if (S.set(l) != r) continue;
        for (int q = 0; q < 3; ++q) { S.a1(q, l) = A[q] / M; S.j1(q, l) = J[q] / M; }
      }
    }
    __syncthreads();
  }
}

// minimum over the warp of a value in [0, 2^63): the minimum of the high
// words, then of the low words among the lanes that hold it (two warp
// reductions instead of five dependent shuffle steps)
__device__ __forceinline__ int64_t warp_min64(int64_t v) {
  const unsigned hi = (unsigned)((unsigned long long)v >> 32), lo = (unsigned)v;
  const unsigned hmin = __reduce_min_sync(0xffffffffu, hi);
  const unsigned lmin = __reduce_min_sync(0xffffffffu, hi == hmin ? lo : 0xffffffffu);
  return (int64_t)(((unsigned long long)hmin << 32) | lmin);
}

// the block minima of two non-negative values (one warp: no shared memory)
template <int NT>
__device__ __forceinline__ void block_min2(int64_t &a, int64_t &b, int64_t (*red)[4]) {
  a = warp_min64(a);
  b = warp_min64(b);
  if constexpr (NT > 32) {
    if ((threadIdx.x & 31) == 0) {
      red[0][threadIdx.x >> 5] = a;
      red[1][threadIdx.x >> 5] = b;
    }
    __syncthreads();
    int64_t ra = red[0][0], rb = red[1][0];
    for (int q = 1; q < NT / 32; ++q) {
      ra = red[0][q] < ra ? red[0][q] : ra;
      rb = red[1][q] < rb ? red[1][q] : rb;
    }
    __syncthreads();
    a = ra;
    b = rb;
  }
}

// energy of the members with chg & 1 as far as replacing them can change it:
// kinetic and star energy, and the pair energy of every pair with one end
// among them (once), pairs in one set left out; state (p, pv)
template <class V>
__device__ double set_energy(const V &S, int nc, bool new_sets, const p3t_params &prm) {
  double E = 0.0;
  for (int k = 0; k < nc; ++k) {
    if (!(S.chg(k) & 1)) continue;
    const double vx = S.pv(0, k), vy = S.pv(1, k), vz = S.pv(2, k);
    const double x = S.p(0, k), y = S.p(1, k), z = S.p(2, k);
    E += 0.5 * S.m(k) * (vx * vx + vy * vy + vz * vz);
    E -= prm.G * prm.m_star * S.m(k) / sqrt(x * x + y * y + z * z);
  }
  for (int k = 0; k < nc; ++k) {
    if (!(S.chg(k) & 1)) continue;
    const int sk = new_sets ? S.set(k) : S.nset(k);
    for (int l = 0; l < nc; ++l) {
      const int sl = new_sets ? S.set(l) : S.nset(l);
      if (l == k || ((S.chg(l) & 1) && l < k) || sl == sk) continue;
      const double dx = S.p(0, k) - S.p(0, l), dy = S.p(1, k) - S.p(1, l),
                   dz = S.p(2, k) - S.p(2, l);
      const double r2 = dx * dx + dy * dy + dz * dz;
      if (r2 == 0.0) continue;
      E -= prm.G * S.m(k) * S.m(l) / sqrt(r2);
    }
  }
  return E;
}

// one thread: joins the touching members into composites at block time tn.
// On entry (p, pv) hold every member's state at tn; nset holds the sets
// before, set receives the sets after.
template <class V>
__device__ void collide_serial(const V &S, HCtl &C, int nc, int64_t tn, const p3t_params &prm) {
  for (int k = 0; k < nc; ++k) S.nset(k) = S.set(k);
  for (int k = 0; k < nc; ++k) {
    if (S.partner(k) == kNone) continue;
    const int ra = S.set(k), rb = S.set(S.partner(k));
    const int lo = ra < rb ? ra : rb, hi = ra < rb ? rb : ra;
    for (int l = 0; l < nc; ++l)
      if (S.set(l) == hi) S.set(l) = lo;
  }
  for (int k = 0; k < nc; ++k) S.chg(k) = 0;
  for (int k = 0; k < nc; ++k)
    if (S.partner(k) != kNone) S.chg(S.set(k)) = 2;
  for (int k = 0; k < nc; ++k)
    if (S.chg(S.set(k)) & 2) S.chg(k) |= 1;
  const double Eb = set_energy(S, nc, false, prm);  // sets before (nset)
  for (int r = 0; r < nc; ++r) {
    if (!(S.chg(r) & 1) || S.set(r) != r) continue;
    double Ms = 0.0, Q[6] = {0, 0, 0, 0, 0, 0};
    for (int l = 0; l < nc; ++l) {
      if (S.set(l) != r) continue;
      Ms += S.m(l);
      for (int q = 0; q < 3; ++q) { Q[q] += S.m(l) * S.p(q, l); Q[3 + q] += S.m(l) * S.pv(q, l); }
    }
    for (int l = 0; l < nc; ++l) {
      if (S.set(l) != r) continue;
      for (int q = 0; q < 3; ++q) { S.p(q, l) = Q[q] / Ms; S.pv(q, l) = Q[3 + q] / Ms; }
    }
  }
  const double Ea = set_energy(S, nc, true, prm);
  C.edisp += Eb - Ea;
  for (int k = 0; k < nc; ++k) {
    if (!(S.chg(k) & 1)) continue;
    for (int q = 0; q < 3; ++q) { S.x(q, k) = S.p(q, k); S.v(q, k) = S.pv(q, k); }
    S.t(k) = tn;
  }
  C.ncomp = 1;
}

// one thread: the cluster's composites (sets of >= 2) to the global list
template <class V>
__device__ void emit_composites(const V &S, const HCtl &C, int nc, int64_t off,
                                const int32_t *cl_mem, const CollOut &co, DevStatus *st) {
  int ne = 0;
  for (int r = 0; r < nc; ++r) {
    if (S.set(r) != r) continue;
    int size = 0;
    for (int l = 0; l < nc; ++l) size += S.set(l) == r;
    if (size >= 2) ne += size;
  }
  if (ne == 0) return;
  const unsigned long long old =
      atomicAdd(co.ctr, (1ull << 32) | (unsigned long long)ne);
  const int64_t rec = (int64_t)(old >> 32), e0 = (int64_t)(old & 0xffffffffull);
  if (rec >= co.rec_cap || e0 + ne > co.ent_cap) {
    dev_fail(st, P3T_ERR_CAPACITY, 63, e0 + ne);
    return;
  }
  co.rec[rec] = make_int4(cl_mem[off], (int)e0, ne, 0);
  co.rec_e[rec] = C.edisp;
  int e = (int)e0;
  for (int r = 0; r < nc; ++r) {
    if (S.set(r) != r) continue;
    int size = 0;
    for (int l = 0; l < nc; ++l) size += S.set(l) == r;
    if (size < 2) continue;
    const int lo = e, hi = e + size;
    for (int l = 0; l < nc; ++l) {
      if (S.set(l) != r) continue;
      const int32_t i = cl_mem[off + l];
      co.ent[e] = make_int4(i, cl_mem[off + r], lo, hi);
      co.slot[i] = e;
      ++e;
    }
  }
}

// block-step integration of one cluster (the whole block takes part)
template <int NT, class V>
__device__ void integrate_cluster(const V &S, HCtl &C, double (*Tb)[6], int64_t off, int nc,
                                  const int32_t *cl_mem, const p3t_particles &p,
                                  const p3t_params &prm, double dt, bool coll,
                                  const CollOut &co, unsigned long long &steps,
                                  bool &underflow, DevStatus *st, int64_t iter_limit,
                                  int32_t *rec) {
  const int tid = threadIdx.x;
  const int item = (tid & 31) * (NT / 32) + (tid >> 5);  // consecutive items -> different warps
  bool uf = false;  // a step of this cluster fell below dt / 2^40
  const int64_t T = ((int64_t)1) << P3T_KMAX;
  const double unit = ldexp(dt, -P3T_KMAX);
  const double idt = 1.0 / dt;
  const double i1mg = 1.0 / (1.0 - prm.gamma);
  // a step of level l is D = unit 2^(40 - l) exactly, so D^n = RN(unit^n)
  // 2^(n (40 - l)) and RN(D^n c) = RN(unit^n c) 2^(n (40 - l)) with unit^n
  // formed by the same successive products: the corrector's powers of D and
  // of 1/D are these constants shifted in the exponent (the same bits as the
  // products, no FP64 instruction)
  const double u2 = unit * unit, u3 = u2 * unit, u4 = u3 * unit, u5 = u4 * unit;
  const double c3u = u3 * (1.0 / 6.0), c4u = u4 * (1.0 / 24.0), c5u = u5 * (1.0 / 120.0);
  const double idt2 = idt * idt, idt3 = idt2 * idt;
  for (int k = item; k < nc; k += NT) {
    const int32_t i = cl_mem[off + k];
    S.x(0, k) = p.x[i]; S.x(1, k) = p.y[i]; S.x(2, k) = p.z[i];
    S.v(0, k) = p.vx[i]; S.v(1, k) = p.vy[i]; S.v(2, k) = p.vz[i];
    for (int q = 0; q < 3; ++q) { S.p(q, k) = S.x(q, k); S.pv(q, k) = S.v(q, k); }
    S.m(k) = p.m[i];
    S.iro(k) = 1.0 / p.r_out[i];
    S.rp(k) = coll ? p.r_phys[i] : 0.0;
    S.set(k) = k;
    S.partner(k) = kNone;
    if (rec) rec[i] = 0;
  }
  if (tid == 0) { C.any = 0; C.ncomp = 0; C.stop = 0; C.edisp = 0.0; }
  __syncthreads();
  // initial forces of every member (the block-time state is the initial
  // state), first steps
  int nact = build_list<NT>(S, C, nc, [](int) { return true; });
  block_forces<NT>(S, C, Tb, nc, nact, item, prm, i1mg, coll);
  for (int k = item; k < nc; k += NT) {
    for (int q = 0; q < 3; ++q) { S.a(q, k) = S.a1(q, k); S.j(q, k) = S.j1(q, k); }
    S.t(k) = 0;
    S.lvl(k) = first_level(S, k, prm, dt, 0, uf);
    if (S.partner(k) != kNone) C.any = 1;
  }
  if (uf) C.stop = 1;
  __syncthreads();
  int64_t tn = 0, iter = 0;
  for (;;) {
    // a step below dt / 2^40 ends the cluster's integration (the error is
    // recorded when the block finishes): every thread reads the flag after
    // the barrier that follows its last write
    if (C.stop) break;
    if (C.any) {
      // collisions found by the last evaluation: every member's state at tn
      for (int k = item; k < nc; k += NT)
        if (S.t(k) == tn)
          for (int q = 0; q < 3; ++q) { S.p(q, k) = S.x(q, k); S.pv(q, k) = S.v(q, k); }
      __syncthreads();
      if (tid == 0) collide_serial(S, C, nc, tn, prm);
      __syncthreads();
      nact = build_list<NT>(S, C, nc, [&](int k) { return (S.chg(k) & 1) != 0; });
      block_forces<NT>(S, C, Tb, nc, nact, item, prm, i1mg, false);
      for (int b = item; b < nact; b += NT) {
        const int k = S.act(b);
        for (int q = 0; q < 3; ++q) { S.a(q, k) = S.a1(q, k); S.j(q, k) = S.j1(q, k); }
        S.lvl(k) = first_level(S, k, prm, dt, tn, uf);
      }
      for (int k = item; k < nc; k += NT) S.partner(k) = kNone;
      if (uf) C.stop = 1;
      __syncthreads();
      if (tid == 0) C.any = 0;
      __syncthreads();
      if (C.stop) break;
    }
    int64_t e_min = T, t_min = T;
    for (int k = tid; k < nc; k += NT) {
      const int64_t e = S.t(k) + (T >> S.lvl(k));
      e_min = e < e_min ? e : e_min;
      t_min = S.t(k) < t_min ? S.t(k) : t_min;
    }
    block_min2<NT>(e_min, t_min, C.red);
    tn = e_min;
    const int64_t tmin = t_min;
    if (tmin >= T) break;
    if (++iter > iter_limit) {
      if (tid == 0) dev_fail(st, P3T_ERR_TIMEOUT, 61, 0);
      break;
    }
    // predict every member (component items)
    for (int i = item; i < nc * 3; i += NT) {
      const int k = i / 3, q = i - 3 * k;
      const double D = i2d_exact(tn - S.t(k)) * unit;
      const double jq = S.j(q, k), aq = S.a(q, k), vq = S.v(q, k);
      // Horner form, fused: x + D (v + D (a/2 + D j/6)), v + D (a + D j/2)
      // (the halvings exact, as exponent shifts)
      S.p(q, k) = __fma_rn(__fma_rn(__fma_rn(jq * (1.0 / 6.0), D, ldexp_fast(aq, -1)), D, vq),
                           D, S.x(q, k));
      S.pv(q, k) = __fma_rn(__fma_rn(ldexp_fast(jq, -1), D, aq), D, vq);
    }
    __syncthreads();
    nact = build_list<NT>(S, C, nc, [&](int k) { return S.t(k) + (T >> S.lvl(k)) == tn; });
    block_forces<NT>(S, C, Tb, nc, nact, item, prm, i1mg, coll);
    // correct (component items of the active members)
    for (int i = item; i < nact * 3; i += NT) {
      const int b = i / 3, q = i - 3 * b;
      const int k = S.act(b);
      const int lv = S.lvl(k), sh = P3T_KMAX - lv;
      const double D = ldexp_fast(unit, sh);
      // 1 / D = 2^lvl (1 / dt) exactly (D = dt 2^-lvl): a product, not a division
      const double iD2 = ldexp_fast(idt2, 2 * lv), iD3 = ldexp_fast(idt3, 3 * lv);
      const double da = S.a(q, k) - S.a1(q, k);
      const double j0 = S.j(q, k), j1 = S.j1(q, k);
      const double A2 = __fma_rn(-D, __fma_rn(2.0, j1, 4.0 * j0), -6.0 * da) * iD2;
      const double A3 = __fma_rn(6.0 * D, j0 + j1, 12.0 * da) * iD3;
      S.a2e(q, k) = __fma_rn(D, A3, A2);
      S.a3(q, k) = A3;
      const double c3 = ldexp_fast(c3u, 3 * sh), c4 = ldexp_fast(c4u, 4 * sh),
                   c5 = ldexp_fast(c5u, 5 * sh);
      S.x(q, k) = __fma_rn(A3, c5, __fma_rn(A2, c4, S.p(q, k)));
      S.v(q, k) = __fma_rn(A3, c4, __fma_rn(A2, c3, S.pv(q, k)));
      S.a(q, k) = S.a1(q, k);
      S.j(q, k) = j1;
    }
    __syncthreads();
    // new steps of the active members
    for (int b = item; b < nact; b += NT) {
      const int k = S.act(b);
      const double D = ldexp_fast(unit, P3T_KMAX - S.lvl(k));
      const int e = ilogb_fast(D);  // dt = sqrt(eta num_s / den_s) s
      const float an = norm3f(S.a(0, k), S.a(1, k), S.a(2, k), 0);
      const float jn = norm3f(S.j(0, k), S.j(1, k), S.j(2, k), e);
      const float a2n = norm3f(S.a2e(0, k), S.a2e(1, k), S.a2e(2, k), 2 * e);
      const float a3n = norm3f(S.a3(0, k), S.a3(1, k), S.a3(2, k), 3 * e);
      const float num = an * a2n + jn * jn, den = jn * a3n + a2n * a2n;
      const double dtd =
          den > 0.0f ? ldexp_fast(f2d_exact(sqrtf((float)prm.eta * num / den)), e) : dt;
      S.t(k) = tn;
      S.lvl(k) = quantise_level(dtd, dt, S.lvl(k), tn, uf);
      if (S.partner(k) != kNone) C.any = 1;
      if (rec) rec[cl_mem[off + k]] += 1;
    }
    if (uf) C.stop = 1;
    if (tid == 0) steps += (unsigned long long)nact;
    __syncthreads();
  }
  for (int k = item; k < nc; k += NT) {
    const int32_t i = cl_mem[off + k];
    p.x[i] = S.x(0, k); p.y[i] = S.x(1, k); p.z[i] = S.x(2, k);
    p.vx[i] = S.v(0, k); p.vy[i] = S.v(1, k); p.vz[i] = S.v(2, k);
  }
  if (tid == 0 && C.ncomp) emit_composites(S, C, nc, off, cl_mem, co, st);
  if (uf) underflow = true;
  __syncthreads();
}

// clusters of nc_lo..nc_hi members; NT threads per block; state in shared
// memory for up to KM members or (BIG) in the global workspace.  One block
// per cluster, clusters handed out dynamically (a long encounter keeps its
// block while the others move on).
template <int NT, int KM, bool BIG>
__global__ void __launch_bounds__(NT) k_hermite_block(
    const int64_t *d_ncl, const int64_t *cl_off, const int32_t *cl_mem, p3t_particles p,
    p3t_params prm, double dt, int nc_lo, int nc_hi, unsigned long long *steps_out,
    int64_t *cursor, const int32_t *list, const int64_t *d_nlist, HBig big, CollOut co,
    DevStatus *st, int64_t iter_limit, int32_t *rec) {
  pdl_wait();
  __shared__ HCtl C;
  extern __shared__ __align__(16) unsigned char hsm[];
  static_assert(BIG || HSmall<KM>::kT >= NT, "a batch of pair terms must fit HSmall::T");
  HSmall<KM> *Sm = reinterpret_cast<HSmall<KM> *>(hsm);
  const int tid = threadIdx.x;
  // every cluster, or (list) the clusters of this kernel's sizes
  const int64_t ncl = list ? *d_nlist : *d_ncl;
  const bool coll = prm.f_radius > 0.0 && p.r_phys != nullptr;
  unsigned long long steps = 0;
  bool underflow = false;
  for (int64_t k = blockIdx.x;; k += gridDim.x) {
    // clusters of up to 128 members are handed out by a cursor (a long
    // encounter keeps its block while the others move on); the rare larger
    // ones are dealt statically
    int64_t c = k;
    if constexpr (!BIG) {
      if (tid == 0) C.cluster = atomicAdd(reinterpret_cast<unsigned long long *>(cursor), 1ull);
      __syncthreads();
      c = C.cluster;
      __syncthreads();
    }
    if (c >= ncl) break;
    if (list) c = list[c];
    const int64_t off = cl_off[c];
    const int nc = (int)(cl_off[c + 1] - off);
    if (nc < nc_lo || nc > nc_hi) continue;
    if constexpr (BIG) {
      const BigView S{big.d, big.t, big.i, big.cap, off};
      integrate_cluster<NT>(S, C, nullptr, off, nc, cl_mem, p, prm, dt, coll, co, steps,
                            underflow, st, iter_limit, rec);
    } else {
      const SmallView<KM> S{Sm};
      integrate_cluster<NT>(S, C, Sm->T, off, nc, cl_mem, p, prm, dt, coll, co, steps,
                            underflow, st, iter_limit, rec);
    }
  }
  if (underflow) dev_fail(st, P3T_ERR_DT_UNDERFLOW, 62, 0);
  if (tid == 0 && steps_out && steps) atomicAdd(steps_out, steps);
}

__global__ void k_zero_i64_five(int64_t *p) {
  pdl_wait(); p[0] = 0; p[1] = 0; p[2] = 0; p[3] = 0; p[4] = 0; }

// the clusters of more than hw members: up to kHMax into list[0..), larger
// ones into list[cap..); their numbers into n[0], n[1] (zeroed before).  The
// order within a list is arrival order: each cluster is integrated on its own,
// so the results do not depend on it.
__global__ void k_cluster_classes(const int64_t *d_ncl, const int64_t *cl_off, int hw,
                                  int64_t cap, int32_t *list, int64_t *n) {
  pdl_wait();
  const int64_t ncl = *d_ncl;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < ncl;
       c += (int64_t)gridDim.x * blockDim.x) {
    const int64_t nc = cl_off[c + 1] - cl_off[c];
    if (nc <= hw) continue;
    const int big = nc > kHMax ? 1 : 0;
    const int64_t slot = (int64_t)atomicAdd(reinterpret_cast<unsigned long long *>(&n[big]), 1ull);
    if (slot < cap) list[big * cap + slot] = (int32_t)c;
  }
}

__global__ void k_zero_u64(unsigned long long *p) {
  pdl_wait(); *p = 0ull; }

// ---- energy ----------------------------------------------------------------
__device__ __forceinline__ void two_sum_f(float &hi, float &lo, float b) {
  const float s = hi + b;
  const float bb = s - hi;
  lo += (hi - (s - bb)) + (b - bb);
  hi = s;
}

constexpr int kETile = 256;

// E = sum m v^2/2 - sum G M m / r - 1/2 sum_i sum_{j != i} G m_i m_j / r_ij
template <bool MIXED>
__global__ void __launch_bounds__(kETile) k_energy(p3t_particles p, p3t_params prm,
                                                   double *part) {
  pdl_wait();
  __shared__ double s_x[kETile], s_y[kETile], s_z[kETile], s_m[kETile];
  __shared__ float4 s_h[kETile], s_l[kETile];
  __shared__ double s_red[3][kETile / 32];
  const int64_t n = p.n;
  const int64_t i = blockIdx.x * (int64_t)kETile + threadIdx.x;
  const bool valid = i < n;
  double ek = 0.0, es = 0.0, ep = 0.0;
  double xi = 0, yi = 0, zi = 0, mi = 0;
  float xh = 0, yh = 0, zh = 0, xl = 0, yl = 0, zl = 0;
  if (valid) {
    xi = p.x[i]; yi = p.y[i]; zi = p.z[i]; mi = p.m[i];
    ek = 0.5 * mi * (p.vx[i] * p.vx[i] + p.vy[i] * p.vy[i] + p.vz[i] * p.vz[i]);
    es = -prm.G * prm.m_star * mi / sqrt(xi * xi + yi * yi + zi * zi);
    xh = (float)xi; yh = (float)yi; zh = (float)zi;
    xl = (float)(xi - (double)xh); yl = (float)(yi - (double)yh); zl = (float)(zi - (double)zh);
  }
  float sh = 0.f, sl = 0.f;
  double sd = 0.0;
  for (int64_t base = 0; base < n; base += kETile) {
    const int64_t j = base + threadIdx.x;
    __syncthreads();
    if (j < n) {
      const double X = p.x[j], Y = p.y[j], Z = p.z[j];
      if (MIXED) {
        const float hx = (float)X, hy = (float)Y, hz = (float)Z;
        s_h[threadIdx.x] = make_float4(hx, hy, hz, (float)p.m[j]);
        s_l[threadIdx.x] = make_float4((float)(X - (double)hx), (float)(Y - (double)hy),
                                       (float)(Z - (double)hz), 0.f);
      } else {
        s_x[threadIdx.x] = X; s_y[threadIdx.x] = Y; s_z[threadIdx.x] = Z;
        s_m[threadIdx.x] = p.m[j];
      }
    } else {
      if (MIXED) { s_h[threadIdx.x] = make_float4(0.f, 0.f, 0.f, 0.f); s_l[threadIdx.x] = s_h[threadIdx.x]; }
      else { s_x[threadIdx.x] = 0.0; s_y[threadIdx.x] = 0.0; s_z[threadIdx.x] = 0.0; s_m[threadIdx.x] = 0.0; }
    }
    __syncthreads();
    const int lim = (int)min((int64_t)kETile, n - base);
    if (MIXED) {
      float b = 0.f;
      for (int q = 0; q < lim; ++q) {
        const float4 H = s_h[q], L = s_l[q];
        const float dx = (xh - H.x) + (xl - L.x);
        const float dy = (yh - H.y) + (yl - L.y);
        const float dz = (zh - H.z) + (zl - L.z);
        const float r2 = dx * dx + dy * dy + dz * dz;
        float ri = r2 > 0.f ? rsqrtf(r2) : 0.f;
        ri = ri * (1.5f - 0.5f * r2 * ri * ri);  // one Newton step
        b += H.w * ri;
      }
      two_sum_f(sh, sl, b);
    } else {
      for (int q = 0; q < lim; ++q) {
        if (base + q == i) continue;
        const double dx = xi - s_x[q], dy = yi - s_y[q], dz = zi - s_z[q];
        sd += s_m[q] * rsqrt(dx * dx + dy * dy + dz * dz);
      }
    }
  }
  if (valid) ep = MIXED ? -0.5 * prm.G * mi * ((double)sh + (double)sl) : -0.5 * prm.G * mi * sd;
  else ep = 0.0;
  double v[3] = {ek, es, ep};
  for (int q = 0; q < 3; ++q)
    for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
  if ((threadIdx.x & 31) == 0)
    for (int q = 0; q < 3; ++q) s_red[q][threadIdx.x >> 5] = v[q];
  __syncthreads();
  if (threadIdx.x < 3) {  // per-block partials, added in block order afterwards
    double s = 0.0;
    for (int w = 0; w < kETile / 32; ++w) s += s_red[threadIdx.x][w];
    part[3 * (int64_t)blockIdx.x + threadIdx.x] = s;
  }
}

// the three sums over the block partials in block order (one warp each, a
// fixed lane-strided order and shuffle tree): the same result on every run
__global__ void k_energy_final(const double *part, int64_t nblocks, double *out) {
  pdl_wait();
  const int q = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __shared__ double sum[3];
  if (q < 3) {
    double s = 0.0;
    for (int64_t b = lane; b < nblocks; b += 32) s += part[3 * b + q];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) sum[q] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    out[1] = sum[0]; out[2] = sum[1]; out[3] = sum[2];
    out[0] = sum[0] + sum[1] + sum[2];
  }
}


// ---- the merge after the second kick (procedure step 9) --------------------
// One block: every composite's lowest member gets the summed mass and the
// radius of the summed volume; the dissipation totals are summed in a fixed
// order (clusters by label, composites by lowest member) so that they do not
// depend on the order the hard step appended them in.
__global__ void k_merge_sets(const int4 *ent, int64_t ne, const int4 *rec, const double *rec_e,
                             int64_t nrec, const double *esoft, double *m, double *rp,
                             double *sorted_h, double *sorted_s, double *out) {
  pdl_wait();
  for (int64_t s = threadIdx.x; s < ne; s += blockDim.x) {
    const int4 e = ent[s];
    if (e.x != e.y) continue;
    double M = 0.0, V = 0.0;
    for (int l = e.z; l < e.w; ++l) {
      const int q = ent[l].x;
      M += m[q];
      if (rp) V += rp[q] * rp[q] * rp[q];
    }
    m[e.x] = M;
    if (rp) rp[e.x] = cbrt(V);
    int64_t rank = 0;
    for (int64_t u = 0; u < ne; ++u) rank += ent[u].x == ent[u].y && ent[u].y < e.y;
    sorted_s[rank] = esoft[s];
  }
  for (int64_t r = threadIdx.x; r < nrec; r += blockDim.x) {
    int64_t rank = 0;
    for (int64_t u = 0; u < nrec; ++u) rank += rec[u].x < rec[r].x;
    sorted_h[rank] = rec_e[r];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t nsets = 0;
    for (int64_t u = 0; u < ne; ++u) nsets += ent[u].x == ent[u].y;
    double eh = 0.0, es = 0.0;
    for (int64_t r = 0; r < nrec; ++r) eh += sorted_h[r];
    for (int64_t q = 0; q < nsets; ++q) es += sorted_s[q];
    out[0] = eh;
    out[1] = es;
  }
}

__global__ void k_merge_keep(int64_t n, const int32_t *slot, const int4 *ent, int32_t *keep) {
  pdl_wait();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t s = slot[i];
    keep[i] = (s < 0 || ent[s].x == ent[s].y) ? 1 : 0;
  }
}

// survivors to their new places in the scratch arrays (10 arrays of n)
__global__ void k_merge_gather(int64_t n, const int32_t *keep, const int64_t *pos,
                               p3t_particles p, double *scr, int32_t *new_index) {
  pdl_wait();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (!keep[i]) {
      new_index[i] = -1;
      continue;
    }
    const int64_t d = pos[i];
    new_index[i] = (int32_t)d;
    scr[d] = p.x[i]; scr[n + d] = p.y[i]; scr[2 * n + d] = p.z[i];
    scr[3 * n + d] = p.vx[i]; scr[4 * n + d] = p.vy[i]; scr[5 * n + d] = p.vz[i];
    scr[6 * n + d] = p.m[i]; scr[7 * n + d] = p.r_out[i]; scr[8 * n + d] = p.r_search[i];
    if (p.r_phys) scr[9 * n + d] = p.r_phys[i];
  }
}

__global__ void k_merge_reset(const int4 *ent, int64_t ne, int32_t *slot,
                              unsigned long long *ctr) {
  pdl_wait();
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < ne;
       s += (int64_t)gridDim.x * blockDim.x)
    slot[ent[s].x] = -1;
  if (blockIdx.x == 0 && threadIdx.x == 0) *ctr = 0ull;
}

__global__ void k_iota(int64_t n, int32_t *a) {
  pdl_wait();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    a[i] = (int32_t)i;
}

CollOut coll_out(p3t_ctx *c) {
  CollOut co;
  co.ctr = c->coll_ctr;
  co.ent = c->coll_ent;
  co.rec = c->coll_rec;
  co.rec_e = c->coll_rec_e;
  co.slot = c->coll_slot;
  co.ent_cap = c->cap;
  co.rec_cap = c->cap / 2 + 1;
  return co;
}

}  // namespace

int p3t_run_kick(p3t_ctx *c, p3t_particles *p, const double *ax,
                 const double *ay, const double *az, double h, cudaStream_t s) {
  if (p->n == 0) return P3T_OK;
  const int64_t g = p3t_grid(p->n, kBlock, (int64_t)c->num_sms * P3T_NSM_BLOCKS);
  const bool coll = c->prm.f_radius > 0.0;
  pdl_launch(k_kick, dim3((unsigned)g), dim3(kBlock), 0, s, p->n, p->vx, p->vy, p->vz, ax, ay, az, h,
                                        coll ? c->coll_slot : nullptr, c->coll_ent, p->m,
                                        c->coll_esoft);
  p3t_note_launches(1);
  return cudaGetLastError() == cudaSuccess ? P3T_OK : P3T_ERR_CUDA;
}

int p3t_run_hard_step(p3t_ctx *c, p3t_particles *p, const p3t_clusters *cl,
                      double dt, uint64_t *n_steps, cudaStream_t s) {
  const int64_t n = p->n;
  const int64_t maxb = (int64_t)c->num_sms * P3T_NSM_BLOCKS;
  const double mu = c->prm.G * c->prm.m_star;
  HBig big{c->hw, c->ht, c->hl, c->cap};
  const CollOut co = coll_out(c);
  unsigned long long *steps = n_steps ? reinterpret_cast<unsigned long long *>(n_steps)
                                      : c->hsteps;
  pdl_launch(k_zero_u64, dim3(1), dim3(1), 0, s, steps);
  pdl_launch(k_zero_i64_five, dim3(1), dim3(1), 0, s, c->hcursor);
  // the clusters of the four-warp and workspace kernels, listed once so that
  // those kernels do not step through every small cluster
  const int hw = c->hwarp_max;
  pdl_launch(k_cluster_classes, dim3((unsigned)p3t_grid(n / 2 + 1, kBlock, maxb)), dim3(kBlock), 0,
             s, &cl->counts[1], cl->cl_off, hw, c->hlist_cap, c->hlist, c->hcursor + 3);
  // Kepler drift, small clusters and large clusters touch disjoint particles:
  // run them on three streams forked from and joined back to the caller's
  P3T_CUDA_TRY(cudaEventRecord(c->ev_fork, s));
  P3T_CUDA_TRY(cudaStreamWaitEvent(c->aux[0], c->ev_fork, 0));
  P3T_CUDA_TRY(cudaStreamWaitEvent(c->aux[1], c->ev_fork, 0));
  const int64_t ncl_max = (n / 2) > 0 ? n / 2 : 1;
  const int64_t nbig = c->num_sms < 32 ? c->num_sms : 32;
  // clusters of 2..hw members: a warp each (stream aux[0]), up to 32 such
  // one-warp blocks an SM (the FP64 latency of their block steps, not the
  // FP64 pipe, limits them: 16 an SM took 40 us more a step); up to 128: a
  // 128-thread block each, then > 128 (stream aux[1])
  const unsigned gw = (unsigned)p3t_grid(ncl_max * 32, 32, (int64_t)c->num_sms * 32);
  if (hw <= 8)
    pdl_launch(k_hermite_block<32, 8, false>, dim3(gw), dim3(32), sizeof(HSmall<8>), c->aux[0], 
        &cl->counts[1], cl->cl_off, cl->cl_mem, *p, c->prm, dt, 2, hw, steps, c->hcursor,
        (const int32_t *)nullptr, (const int64_t *)nullptr, big, co, c->status, c->hermite_limit,
        c->hermite_rec);
  else if (hw <= 16)
    pdl_launch(k_hermite_block<32, 16, false>, dim3(gw), dim3(32), sizeof(HSmall<16>), c->aux[0], 
        &cl->counts[1], cl->cl_off, cl->cl_mem, *p, c->prm, dt, 2, hw, steps, c->hcursor,
        (const int32_t *)nullptr, (const int64_t *)nullptr, big, co, c->status, c->hermite_limit,
        c->hermite_rec);
  else
    pdl_launch(k_hermite_block<32, 32, false>, dim3(gw), dim3(32), sizeof(HSmall<32>), c->aux[0], 
        &cl->counts[1], cl->cl_off, cl->cl_mem, *p, c->prm, dt, 2, hw, steps, c->hcursor,
        (const int32_t *)nullptr, (const int64_t *)nullptr, big, co, c->status, c->hermite_limit,
        c->hermite_rec);
  pdl_launch(k_hermite_block<128, kHMax, false>, dim3((unsigned)p3t_grid(ncl_max * 128, 128, (int64_t)c->num_sms * 2)), dim3(128), sizeof(HSmall<kHMax>), c->aux[1], 
      &cl->counts[1], cl->cl_off, cl->cl_mem, *p, c->prm, dt, hw + 1, kHMax, steps,
      c->hcursor + 1, (const int32_t *)c->hlist, (const int64_t *)(c->hcursor + 3),
      big, co, c->status, c->hermite_limit, c->hermite_rec);
  pdl_launch(k_hermite_block<128, 1, true>, dim3((unsigned)p3t_grid(ncl_max, 1, nbig)), dim3(128), 0, c->aux[1], 
      &cl->counts[1], cl->cl_off, cl->cl_mem, *p, c->prm, dt, kHMax + 1, 0x7fffffff, steps,
      c->hcursor + 2, (const int32_t *)(c->hlist + c->hlist_cap),
      (const int64_t *)(c->hcursor + 4), big, co, c->status, c->hermite_limit, c->hermite_rec);
  KepConst kc;
  kc.mu = mu;
  kc.sq = sqrt(mu);
  kc.isq = 1.0 / kc.sq;
  kc.imu = 1.0 / mu;
  auto kep = c->prm.precision == P3T_MIXED ? k_kepler<true> : k_kepler<false>;
  pdl_launch(kep, dim3((unsigned)p3t_grid(n, 128, maxb)), dim3(128), 0, s, &cl->counts[0], cl->singles, *p, dt, kc,
                                                        c->status);
  P3T_CUDA_TRY(cudaEventRecord(c->ev_join[0], c->aux[0]));
  P3T_CUDA_TRY(cudaEventRecord(c->ev_join[1], c->aux[1]));
  P3T_CUDA_TRY(cudaStreamWaitEvent(s, c->ev_join[0], 0));
  P3T_CUDA_TRY(cudaStreamWaitEvent(s, c->ev_join[1], 0));
  p3t_note_launches(7);
  return cudaGetLastError() == cudaSuccess ? P3T_OK : P3T_ERR_CUDA;
}

int p3t_run_kepler_drift(p3t_ctx *c, p3t_particles *p, double dt, cudaStream_t s) {
  if (p->n == 0) return P3T_OK;
  KepConst kc;
  kc.mu = c->prm.G * c->prm.m_star;
  kc.sq = sqrt(kc.mu);
  kc.isq = 1.0 / kc.sq;
  kc.imu = 1.0 / kc.mu;
  auto kep = c->prm.precision == P3T_MIXED ? k_kepler_all<true> : k_kepler_all<false>;
  pdl_launch(kep, dim3((unsigned)p3t_grid(p->n, 128, (int64_t)c->num_sms * P3T_NSM_BLOCKS)), dim3(128), 0, s, 
      *p, dt, kc, c->status);
  p3t_note_launches(1);
  return cudaGetLastError() == cudaSuccess ? P3T_OK : P3T_ERR_CUDA;
}

// Procedure step 9 for composites (Sec. 2.4.1).  Synchronises the stream: the
// caller needs the new particle count on the host.
int p3t_run_merge(p3t_ctx *c, p3t_particles *p, int32_t *new_index, double *e_disp,
                  int64_t *n_merged, cudaStream_t s) {
  const int64_t n = p->n;
  const int64_t maxb = (int64_t)c->num_sms * P3T_NSM_BLOCKS;
  unsigned long long ctr = 0;
  P3T_CUDA_TRY(cudaMemcpyAsync(&ctr, c->coll_ctr, sizeof(ctr), cudaMemcpyDeviceToHost, s));
  P3T_CUDA_TRY(cudaStreamSynchronize(s));
  int64_t nrec = (int64_t)(ctr >> 32), ne = (int64_t)(ctr & 0xffffffffull);
  const CollOut co = coll_out(c);
  if (nrec > co.rec_cap) nrec = co.rec_cap;  // a capacity error is already recorded
  if (ne > co.ent_cap) ne = co.ent_cap;
  if (nrec == 0 || ne == 0 || n == 0) {
    if (e_disp) e_disp[0] = e_disp[1] = 0.0;
    if (n_merged) *n_merged = 0;
    if (new_index && n > 0) {
      pdl_launch(k_iota, dim3((unsigned)p3t_grid(n, kBlock, maxb)), dim3(kBlock), 0, s, n, new_index);
      p3t_note_launches(1);
    }
    return cudaGetLastError() == cudaSuccess ? P3T_OK : P3T_ERR_CUDA;
  }
  double *scr = c->hw;              // 10 n for the gather
  double *sorted_h = c->hw + 10 * c->cap, *sorted_s = sorted_h + c->cap;
  double *out = c->epart;
  int32_t *keep = c->flag;
  int64_t *pos = c->pos;
  int32_t *ni = new_index ? new_index : c->flag + c->cap;
  int64_t *d_n = c->counters + 16, *d_total = c->counters + 17;
  P3T_CUDA_TRY(cudaMemcpyAsync(d_n, &n, sizeof(n), cudaMemcpyHostToDevice, s));
  pdl_launch(k_merge_sets, dim3(1), dim3(1024), 0, s, co.ent, ne, co.rec, co.rec_e, nrec, c->coll_esoft, p->m,
                                  p->r_phys, sorted_h, sorted_s, out);
  const unsigned g = (unsigned)p3t_grid(n, kBlock, maxb);
  pdl_launch(k_merge_keep, dim3(g), dim3(kBlock), 0, s, n, c->coll_slot, co.ent, keep);
  int rc = p3t_scan_i32_to_i64(keep, pos, d_n, n, d_total, c->scan_state, c->scan_words, c->status, c->poll_limit, s);
  if (rc) return rc;
  pdl_launch(k_merge_gather, dim3(g), dim3(kBlock), 0, s, n, keep, pos, *p, scr, ni);
  double *dst[10] = {p->x, p->y, p->z, p->vx, p->vy, p->vz, p->m, p->r_out, p->r_search,
                     p->r_phys};
  for (int q = 0; q < 10; ++q)
    if (dst[q])
      P3T_CUDA_TRY(cudaMemcpyAsync(dst[q], scr + q * n, sizeof(double) * n,
                                   cudaMemcpyDeviceToDevice, s));
  pdl_launch(k_merge_reset, dim3((unsigned)p3t_grid(ne, kBlock, maxb)), dim3(kBlock), 0, s, co.ent, ne, c->coll_slot,
                                                                        c->coll_ctr);
  p3t_note_launches(5);
  double eo[2];
  int64_t total = 0;
  P3T_CUDA_TRY(cudaMemcpyAsync(eo, out, sizeof(eo), cudaMemcpyDeviceToHost, s));
  P3T_CUDA_TRY(cudaMemcpyAsync(&total, d_total, sizeof(total), cudaMemcpyDeviceToHost, s));
  P3T_CUDA_TRY(cudaStreamSynchronize(s));
  if (e_disp) { e_disp[0] = eo[0]; e_disp[1] = eo[1]; }
  if (n_merged) *n_merged = n - total;
  p->n = total;
  return cudaGetLastError() == cudaSuccess ? P3T_OK : P3T_ERR_CUDA;
}

int p3t_run_energy(p3t_ctx *c, const p3t_particles *p, double *out, cudaStream_t s) {
  const int64_t g = (p->n + kETile - 1) / kETile;
  double *part = c->hw;  // 3 g <= 33 cap doubles
  if (p->n > 0) {
    if (c->prm.precision == P3T_MIXED)
      pdl_launch(k_energy<true>, dim3((unsigned)g), dim3(kETile), 0, s, *p, c->prm, part);
    else
      pdl_launch(k_energy<false>, dim3((unsigned)g), dim3(kETile), 0, s, *p, c->prm, part);
  }
  pdl_launch(k_energy_final, dim3(1), dim3(96), 0, s, part, g, out);
  p3t_note_launches(p->n > 0 ? 2 : 1);
  return cudaGetLastError() == cudaSuccess ? P3T_OK : P3T_ERR_CUDA;
}

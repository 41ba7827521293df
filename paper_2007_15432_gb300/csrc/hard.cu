// Rows a7-a10 of the soft step: kick, Hermite-4 hard step of the neighbour
// clusters, Kepler drift of isolated particles, energy.
//
// Compiled with -fmad=false.  The Hermite force, predictor, corrector and
// step rule are evaluated in one fixed order with IEEE division and square
// root, so that the block-step schedule (decided by comparing FP64 step
// estimates with dt / 2^k) does not depend on the machine.
#include "p3t_internal.cuh"

namespace {

constexpr int kBlock = 256;
constexpr int64_t kHermiteIterLimit = 1 << 24;  // block steps per cluster

// ---- row a7: soft kick (procedure steps 3 and 8) ----------------------------
__global__ void k_kick(int64_t n, double *vx, double *vy, double *vz,
                       const double *ax, const double *ay, const double *az,
                       double h) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    vx[i] += ax[i] * h;
    vy[i] += ay[i] * h;
    vz[i] += az[i] * h;
  }
}

// ---- row a9: Kepler drift, universal variables ------------------------------
// Stumpff functions C(z) = sum (-z)^k / (2k+2)!, S(z) = sum (-z)^k / (2k+3)!,
// as nested series for |z| < 1 and in closed form otherwise.
__device__ __forceinline__ void stumpff(double z, double &C, double &S) {
  if (fabs(z) < 1.0) {
    // Horner in z with coefficients (-1)^k / (2k+2)! and (-1)^k / (2k+3)!
    // (compile-time constants: no division at run time); |z| < 1 keeps the
    // truncation below 1e-20
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
    C = c0 + z * (c1 + z * (c2 + z * (c3 + z * (c4 + z * (c5 + z * (c6 + z * (c7 + z * (c8 + z * c9))))))));
    S = s0 + z * (s1 + z * (s2 + z * (s3 + z * (s4 + z * (s5 + z * (s6 + z * (s7 + z * (s8 + z * s9))))))));
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

// Advances (X, V) by dt on the Kepler orbit about mu.  Universal anomaly chi
// solves sqrt(mu) dt = (r0 v_r0/sqrt(mu)) chi^2 C + (1 - alpha r0) chi^3 S
// + r0 chi (z = alpha chi^2) by Newton-Raphson; then Lagrange f, g.
__device__ bool kepler_uv(double X[3], double V[3], double dt, double mu) {
  const double r0 = sqrt(X[0] * X[0] + X[1] * X[1] + X[2] * X[2]);
  const double v2 = V[0] * V[0] + V[1] * V[1] + V[2] * V[2];
  const double rv = X[0] * V[0] + X[1] * V[1] + X[2] * V[2];
  const double ir0 = 1.0 / r0, imu = 1.0 / mu;
  const double alpha = 2.0 * ir0 - v2 * imu;
  const double sq = sqrt(mu), isq = 1.0 / sq;
  const double sig = rv * isq;  // r0 v_r0 / sqrt(mu)
  const double tau = sq * dt;
  // series of the universal Kepler equation: chi = tau/r0 - sig tau^2/(2 r0^3) + O(tau^3)
  double chi = tau * ir0 - 0.5 * sig * tau * tau * ir0 * ir0 * ir0;
  if (alpha > 0.0) {
    const double P = 2.0 * 3.141592653589793 / (alpha * sqrt(alpha) * sq);
    if (fabs(dt) > 0.25 * P) chi = tau * alpha;
  }
  double C = 0.5, S = 1.0 / 6.0, z = 0.0;
  bool ok = false;
  for (int it = 0; it < 64; ++it) {
    z = alpha * chi * chi;
    stumpff(z, C, S);
    const double chi2 = chi * chi;
    const double F = sig * chi2 * C + (1.0 - alpha * r0) * chi2 * chi * S + r0 * chi - tau;
    const double Fp = sig * chi * (1.0 - z * S) + (1.0 - alpha * r0) * chi2 * C + r0;
    double d = F / Fp;
    const double lim = 0.5 * (fabs(chi) + r0);
    if (d > lim) d = lim;
    if (d < -lim) d = -lim;
    chi -= d;
    // quadratic convergence: after a correction below 1e-10 relative the
    // remaining error (~ its square) is below rounding
    if (fabs(d) <= 1e-10 * fabs(chi) || d == 0.0) { ok = true; break; }
  }
  z = alpha * chi * chi;
  stumpff(z, C, S);
  const double chi2 = chi * chi;
  const double f = 1.0 - chi2 * ir0 * C;
  const double g = dt - chi2 * chi * S * isq;
  double nx[3];
  for (int a = 0; a < 3; ++a) nx[a] = f * X[a] + g * V[a];
  const double r = sqrt(nx[0] * nx[0] + nx[1] * nx[1] + nx[2] * nx[2]);
  const double ir = 1.0 / r;
  const double fd = sq * ir * ir0 * (z * S - 1.0) * chi;
  const double gd = 1.0 - chi2 * ir * C;
  for (int a = 0; a < 3; ++a) {
    const double nv = fd * X[a] + gd * V[a];
    X[a] = nx[a];
    V[a] = nv;
  }
  return ok;
}

__global__ void k_kepler(const int64_t *d_nsingle, const int32_t *singles,
                         p3t_particles p, double dt, double mu, DevStatus *st) {
  const int64_t ns = *d_nsingle;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < ns;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int32_t i = singles[k];
    double X[3] = {p.x[i], p.y[i], p.z[i]}, V[3] = {p.vx[i], p.vy[i], p.vz[i]};
    if (!kepler_uv(X, V, dt, mu)) dev_fail(st, P3T_ERR_TIMEOUT, 60, 0);
    p.x[i] = X[0]; p.y[i] = X[1]; p.z[i] = X[2];
    p.vx[i] = V[0]; p.vy[i] = V[1]; p.vz[i] = V[2];
  }
}

// ---- row a8: Hermite-4 with block steps, one warp per cluster ---------------
struct HWork {
  double *x, *y, *z, *vx, *vy, *vz;        // state at the member's own time
  double *px, *py, *pz, *pvx, *pvy, *pvz;  // predicted to the block time
  double *ax, *ay, *az, *jx, *jy, *jz;     // a, jerk at the member's own time
  double *m, *ro;
  int64_t *t;                              // time, units of dt / 2^40
  int32_t *lvl;                            // step = dt / 2^lvl
};

// hard acceleration and jerk of member k (Eq. hardforce): star term, then the
// (1 - K) pair terms over the other members in ascending order; one
// reciprocal square root per pair, 1/max(r_out) taken as min(1/r_out)
__device__ void hard_acc_jerk(int nc, const double *x, const double *y,
                              const double *z, const double *vx, const double *vy,
                              const double *vz, const double *m, const double *ro,
                              const p3t_params &prm, double i1mg, int k, double acc[3],
                              double jerk[3]) {
  double ax = 0, ay = 0, az = 0, jx = 0, jy = 0, jz = 0;
  {
    const double r2 = x[k] * x[k] + y[k] * y[k] + z[k] * z[k];
    const double rinv = 1.0 / sqrt(r2);
    const double rinv2 = rinv * rinv;
    const double f = prm.G * prm.m_star * (rinv2 * rinv);
    const double rv = x[k] * vx[k] + y[k] * vy[k] + z[k] * vz[k];
    ax -= f * x[k]; ay -= f * y[k]; az -= f * z[k];
    const double c = 3.0 * rv * rinv2;
    jx -= f * (vx[k] - c * x[k]);
    jy -= f * (vy[k] - c * y[k]);
    jz -= f * (vz[k] - c * z[k]);
  }
  const double irok = 1.0 / ro[k];
  for (int j = 0; j < nc; ++j) {
    if (j == k) continue;
    const double rx = x[k] - x[j], ry = y[k] - y[j], rz = z[k] - z[j];
    const double ux = vx[k] - vx[j], uy = vy[k] - vy[j], uz = vz[k] - vz[j];
    const double r2 = rx * rx + ry * ry + rz * rz;
    if (r2 == 0.0) continue;
    const double rinv = 1.0 / sqrt(r2);
    const double r = r2 * rinv;
    const double irj = 1.0 / ro[j];
    const double irot = irok < irj ? irok : irj;
    const double yv = r * irot;
    if (yv >= 1.0) continue;
    double w = 1.0, dK = 0.0;
    if (yv > prm.gamma) {
      const double xs = (yv - prm.gamma) * i1mg;
      const double x2 = xs * xs, x3 = x2 * xs, x4 = x2 * x2, u = 1.0 - xs;
      w = 1.0 - x4 * (35.0 - 84.0 * xs + 70.0 * x2 - 20.0 * x3);
      dK = 140.0 * x3 * (u * u * u) * i1mg;
    }
    const double rinv2 = rinv * rinv;
    const double g3 = prm.G * m[j] * (rinv2 * rinv);
    const double f = g3 * w;
    const double rv = rx * ux + ry * uy + rz * uz;
    ax -= f * rx; ay -= f * ry; az -= f * rz;
    const double c = 3.0 * w * rv * rinv2 + dK * rv * rinv * irot;
    jx -= g3 * (w * ux - c * rx);
    jy -= g3 * (w * uy - c * ry);
    jz -= g3 * (w * uz - c * rz);
  }
  acc[0] = ax; acc[1] = ay; acc[2] = az;
  jerk[0] = jx; jerk[1] = jy; jerk[2] = jz;
}

// The step estimates only choose a power-of-two step: formed in FP32 from
// components scaled by an exact power of two 2^k (j by s, a2 by s^2, a3 by
// s^3, s = 2^e close to the step) so that nothing overflows FP32.
__device__ __forceinline__ float norm3f(double a, double b, double c, int k) {
  const float x = (float)ldexp(a, k), y = (float)ldexp(b, k), z = (float)ldexp(c, k);
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
  if (dt_des > 0.0 && dt_des < dt) {
    int l0 = ilogb(dt) - ilogb(dt_des) - 1;  // dt / 2^l > dt_des for every l <= l0
    lvl = l0 < 0 ? 0 : (l0 > P3T_KMAX ? P3T_KMAX : l0);
  }
  while (lvl < P3T_KMAX && ldexp(dt, -lvl) > dt_des) ++lvl;
  if (ldexp(dt, -lvl) > dt_des) underflow = true;
  if (lvl < prev - 1) lvl = prev - 1;
  if (t != 0) {
    const int need = P3T_KMAX - __ffsll((long long)t) + 1;  // 2^(40-lvl) must divide t
    if (lvl < need) lvl = need;
  }
  return lvl > P3T_KMAX ? P3T_KMAX : lvl;
}

// Block-step integration of one cluster over [0, dt] by a group of NL lanes
// (NL = 32: a warp per cluster; NL = 4: eight small clusters per warp).
// Members are taken k = lane, lane + NL, ...; the arithmetic per member does
// not depend on NL.
template <int NL>
__device__ void integrate_cluster(int64_t off, int nc, const int32_t *cl_mem,
                                  const p3t_particles &p, const HWork &w,
                                  const p3t_params &prm, double dt, int lane,
                                  unsigned mask, unsigned long long &steps,
                                  bool &underflow, DevStatus *st) {
  const int64_t T = ((int64_t)1) << P3T_KMAX;
  const double unit = ldexp(dt, -P3T_KMAX);
  const double i1mg = 1.0 / (1.0 - prm.gamma);
  double *x = w.x + off, *y = w.y + off, *z = w.z + off;
  double *vx = w.vx + off, *vy = w.vy + off, *vz = w.vz + off;
  double *px = w.px + off, *py = w.py + off, *pz = w.pz + off;
  double *pvx = w.pvx + off, *pvy = w.pvy + off, *pvz = w.pvz + off;
  double *ax = w.ax + off, *ay = w.ay + off, *az = w.az + off;
  double *jx = w.jx + off, *jy = w.jy + off, *jz = w.jz + off;
  double *m = w.m + off, *ro = w.ro + off;
  int64_t *t = w.t + off;
  int32_t *lvl = w.lvl + off;
  for (int k = lane; k < nc; k += NL) {
    const int32_t i = cl_mem[off + k];
    x[k] = p.x[i]; y[k] = p.y[i]; z[k] = p.z[i];
    vx[k] = p.vx[i]; vy[k] = p.vy[i]; vz[k] = p.vz[i];
    m[k] = p.m[i]; ro[k] = p.r_out[i];
  }
  __syncwarp(mask);
  for (int k = lane; k < nc; k += NL) {
    double a[3], j[3];
    hard_acc_jerk(nc, x, y, z, vx, vy, vz, m, ro, prm, i1mg, k, a, j);
    ax[k] = a[0]; ay[k] = a[1]; az[k] = a[2];
    jx[k] = j[0]; jy[k] = j[1]; jz[k] = j[2];
    const int e = ilogb(dt);  // eta0 |a| / |j| = (eta0 |a| / |j s|) s
    const float an = norm3f(a[0], a[1], a[2], 0), jn = norm3f(j[0], j[1], j[2], e);
    const double dtd = jn > 0.0f ? ldexp((double)((float)prm.eta0 * an / jn), e) : dt;
    t[k] = 0;
    lvl[k] = quantise_level(dtd, dt, 0, 0, underflow);
  }
  __syncwarp(mask);
  int64_t iter = 0;
  for (;;) {
    int64_t tn = T, tmin = T;
    for (int k = lane; k < nc; k += NL) {
      const int64_t e = t[k] + (T >> lvl[k]);
      tn = e < tn ? e : tn;
      tmin = t[k] < tmin ? t[k] : tmin;
    }
#pragma unroll
    for (int o = NL / 2; o > 0; o >>= 1) {
      const int64_t a = __shfl_xor_sync(mask, tn, o);
      const int64_t b = __shfl_xor_sync(mask, tmin, o);
      tn = a < tn ? a : tn;
      tmin = b < tmin ? b : tmin;
    }
    if (tmin >= T) break;
    if (++iter > kHermiteIterLimit) {
      if (lane == 0) dev_fail(st, P3T_ERR_TIMEOUT, 61, 0);
      break;
    }
    // predict every member to the block time
    for (int k = lane; k < nc; k += NL) {
      const double D = (double)(tn - t[k]) * unit;
      const double D2 = D * D, D3 = D2 * D;
      px[k] = x[k] + vx[k] * D + ax[k] * D2 * 0.5 + jx[k] * D3 * (1.0 / 6.0);
      py[k] = y[k] + vy[k] * D + ay[k] * D2 * 0.5 + jy[k] * D3 * (1.0 / 6.0);
      pz[k] = z[k] + vz[k] * D + az[k] * D2 * 0.5 + jz[k] * D3 * (1.0 / 6.0);
      pvx[k] = vx[k] + ax[k] * D + jx[k] * D2 * 0.5;
      pvy[k] = vy[k] + ay[k] * D + jy[k] * D2 * 0.5;
      pvz[k] = vz[k] + az[k] * D + jz[k] * D2 * 0.5;
    }
    __syncwarp(mask);
    // evaluate and correct the active members
    for (int k = lane; k < nc; k += NL) {
      if (t[k] + (T >> lvl[k]) != tn) continue;
      double a1[3], j1[3];
      hard_acc_jerk(nc, px, py, pz, pvx, pvy, pvz, m, ro, prm, i1mg, k, a1, j1);
      const double D = (double)(T >> lvl[k]) * unit;
      const double D2 = D * D, D3 = D2 * D, D4 = D3 * D, D5 = D4 * D;
      const double iD = 1.0 / D, iD2 = iD * iD, iD3 = iD2 * iD;
      const double a0[3] = {ax[k], ay[k], az[k]}, j0[3] = {jx[k], jy[k], jz[k]};
      double A2[3], A3[3], A2e[3];
      for (int q = 0; q < 3; ++q) {
        const double da = a0[q] - a1[q];
        A2[q] = (-6.0 * da - D * (4.0 * j0[q] + 2.0 * j1[q])) * iD2;
        A3[q] = (12.0 * da + 6.0 * D * (j0[q] + j1[q])) * iD3;
        A2e[q] = A2[q] + D * A3[q];
      }
      x[k] = px[k] + A2[0] * D4 * (1.0 / 24.0) + A3[0] * D5 * (1.0 / 120.0);
      y[k] = py[k] + A2[1] * D4 * (1.0 / 24.0) + A3[1] * D5 * (1.0 / 120.0);
      z[k] = pz[k] + A2[2] * D4 * (1.0 / 24.0) + A3[2] * D5 * (1.0 / 120.0);
      vx[k] = pvx[k] + A2[0] * D3 * (1.0 / 6.0) + A3[0] * D4 * (1.0 / 24.0);
      vy[k] = pvy[k] + A2[1] * D3 * (1.0 / 6.0) + A3[1] * D4 * (1.0 / 24.0);
      vz[k] = pvz[k] + A2[2] * D3 * (1.0 / 6.0) + A3[2] * D4 * (1.0 / 24.0);
      ax[k] = a1[0]; ay[k] = a1[1]; az[k] = a1[2];
      jx[k] = j1[0]; jy[k] = j1[1]; jz[k] = j1[2];
      const int e = ilogb(D);  // dt = sqrt(eta num_s / den_s) s
      const float an = norm3f(a1[0], a1[1], a1[2], 0), jn = norm3f(j1[0], j1[1], j1[2], e);
      const float a2n = norm3f(A2e[0], A2e[1], A2e[2], 2 * e);
      const float a3n = norm3f(A3[0], A3[1], A3[2], 3 * e);
      const float num = an * a2n + jn * jn, den = jn * a3n + a2n * a2n;
      const double dtd = den > 0.0f ? ldexp((double)sqrtf((float)prm.eta * num / den), e) : dt;
      t[k] = tn;
      lvl[k] = quantise_level(dtd, dt, lvl[k], tn, underflow);
      ++steps;
    }
    __syncwarp(mask);
  }
  for (int k = lane; k < nc; k += NL) {
    const int32_t i = cl_mem[off + k];
    p.x[i] = x[k]; p.y[i] = y[k]; p.z[i] = z[k];
    p.vx[i] = vx[k]; p.vy[i] = vy[k]; p.vz[i] = vz[k];
  }
  __syncwarp(mask);
}

// ---- clusters of up to kHMax members: one 128-thread block per cluster ------
// Work items (member components, or (active member, source) terms) are dealt
// round-robin over the block's four warps, so one cluster keeps the FP64
// pipes of all four SM sub-partitions busy: on this part a warp instruction
// of FP64 occupies its sub-partition's pipe for ~64 cycles, and a cluster's
// block steps are a serial chain.  Each active member's force is the sum, in
// the fixed order star term first then sources in ascending index, of terms
// computed in parallel.
constexpr int kHB = 128;
constexpr int kHMax = 128;

struct HShared {
  double x[3][kHMax], v[3][kHMax], a[3][kHMax], j[3][kHMax];
  double p[3][kHMax], pv[3][kHMax];
  double a1[3][kHMax], j1[3][kHMax], a2e[3][kHMax], a3[3][kHMax];
  double m[kHMax], iro[kHMax];
  double T[kHMax + 1][6];  // one batch: B members x (nc + 1) terms, at most kHMax + 1
  int64_t t[kHMax];
  int32_t lvl[kHMax], act[kHMax];
  int64_t red[2][4];
  int32_t wcount[4];
  int64_t cluster;
  int nact;
};

// term of source j (j == nc: the star) on member k, from arrays X, V
__device__ __forceinline__ void hard_term(const HShared &S, const double (*X)[kHMax],
                                          const double (*V)[kHMax], int nc, int k, int j,
                                          const p3t_params &prm, double i1mg, double out[6]) {
  for (int q = 0; q < 6; ++q) out[q] = 0.0;
  const double xk = X[0][k], yk = X[1][k], zk = X[2][k];
  const double vxk = V[0][k], vyk = V[1][k], vzk = V[2][k];
  if (j == nc) {
    const double r2 = xk * xk + yk * yk + zk * zk;
    const double rinv = 1.0 / sqrt(r2);
    const double rinv2 = rinv * rinv;
    const double f = prm.G * prm.m_star * (rinv2 * rinv);
    const double rv = xk * vxk + yk * vyk + zk * vzk;
    out[0] = f * xk; out[1] = f * yk; out[2] = f * zk;
    const double c = 3.0 * rv * rinv2;
    out[3] = f * (vxk - c * xk);
    out[4] = f * (vyk - c * yk);
    out[5] = f * (vzk - c * zk);
    return;
  }
  if (j == k) return;
  const double rx = xk - X[0][j], ry = yk - X[1][j], rz = zk - X[2][j];
  const double ux = vxk - V[0][j], uy = vyk - V[1][j], uz = vzk - V[2][j];
  const double r2 = rx * rx + ry * ry + rz * rz;
  if (r2 == 0.0) return;
  const double rinv = 1.0 / sqrt(r2);
  const double r = r2 * rinv;
  const double irot = S.iro[k] < S.iro[j] ? S.iro[k] : S.iro[j];
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
  const double g3 = prm.G * S.m[j] * (rinv2 * rinv);
  const double f = g3 * w;
  const double rv = rx * ux + ry * uy + rz * uz;
  out[0] = f * rx; out[1] = f * ry; out[2] = f * rz;
  const double c = 3.0 * w * rv * rinv2 + dK * rv * rinv * irot;
  out[3] = g3 * (w * ux - c * rx);
  out[4] = g3 * (w * uy - c * ry);
  out[5] = g3 * (w * uz - c * rz);
}

// forces on the active members S.act[0..nact) from arrays X, V into a1, j1
__device__ void block_forces(HShared &S, const double (*X)[kHMax], const double (*V)[kHMax],
                             int nc, int nact, int item, const p3t_params &prm, double i1mg) {
  const int per = nc + 1;
  const int B = kHB / per > 0 ? kHB / per : 1;  // members per batch
  for (int b0 = 0; b0 < nact; b0 += B) {
    const int nb = min(B, nact - b0);
    const int items = nb * per;
    for (int i = item; i < items; i += kHB) {
      const int bm = i / per, jj = i - bm * per;
      hard_term(S, X, V, nc, S.act[b0 + bm], jj, prm, i1mg, S.T[i]);
    }
    __syncthreads();
    for (int i = item; i < nb * 6; i += kHB) {
      const int bm = i / 6, q = i - bm * 6;
      const int k = S.act[b0 + bm];
      const int base = bm * per;
      double acc = 0.0;
      acc -= S.T[base + nc][q];
      for (int jj = 0; jj < nc; ++jj) acc -= S.T[base + jj][q];
      if (q < 3) S.a1[q][k] = acc; else S.j1[q - 3][k] = acc;
    }
    __syncthreads();
  }
}

__device__ __forceinline__ int64_t block_min(int64_t v, int64_t *red4) {
  for (int o = 16; o > 0; o >>= 1) {
    const int64_t u = __shfl_xor_sync(0xffffffffu, v, o);
    v = u < v ? u : v;
  }
  if ((threadIdx.x & 31) == 0) red4[threadIdx.x >> 5] = v;
  __syncthreads();
  int64_t r = red4[0];
  for (int q = 1; q < kHB / 32; ++q) r = red4[q] < r ? red4[q] : r;
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(kHB) k_hermite_block(
    const int64_t *d_ncl, const int64_t *cl_off, const int32_t *cl_mem, p3t_particles p,
    p3t_params prm, double dt, unsigned long long *steps_out, int64_t *cursor,
    DevStatus *st) {
  __shared__ HShared S;
  const int tid = threadIdx.x;
  const int item = (tid & 31) * (kHB / 32) + (tid >> 5);  // consecutive items -> different warps
  const int64_t ncl = *d_ncl;
  const int64_t T = ((int64_t)1) << P3T_KMAX;
  const double unit = ldexp(dt, -P3T_KMAX);
  const double i1mg = 1.0 / (1.0 - prm.gamma);
  unsigned long long steps = 0;
  bool underflow = false;
  for (;;) {
    if (tid == 0) S.cluster = atomicAdd(reinterpret_cast<unsigned long long *>(cursor), 1ull);
    __syncthreads();
    const int64_t c = S.cluster;
    __syncthreads();
    if (c >= ncl) break;
    const int64_t off = cl_off[c];
    const int nc = (int)(cl_off[c + 1] - off);
    if (nc > kHMax) continue;  // the warp path takes these
    for (int k = item; k < nc; k += kHB) {
      const int32_t i = cl_mem[off + k];
      S.x[0][k] = p.x[i]; S.x[1][k] = p.y[i]; S.x[2][k] = p.z[i];
      S.v[0][k] = p.vx[i]; S.v[1][k] = p.vy[i]; S.v[2][k] = p.vz[i];
      S.m[k] = p.m[i];
      S.iro[k] = 1.0 / p.r_out[i];
      S.act[k] = k;
    }
    __syncthreads();
    // initial forces of every member, first steps
    block_forces(S, S.x, S.v, nc, nc, item, prm, i1mg);
    for (int k = item; k < nc; k += kHB) {
      for (int q = 0; q < 3; ++q) { S.a[q][k] = S.a1[q][k]; S.j[q][k] = S.j1[q][k]; }
      const int e = ilogb(dt);
      const float an = norm3f(S.a[0][k], S.a[1][k], S.a[2][k], 0);
      const float jn = norm3f(S.j[0][k], S.j[1][k], S.j[2][k], e);
      const double dtd = jn > 0.0f ? ldexp((double)((float)prm.eta0 * an / jn), e) : dt;
      S.t[k] = 0;
      S.lvl[k] = quantise_level(dtd, dt, 0, 0, underflow);
    }
    __syncthreads();
    int64_t iter = 0;
    for (;;) {
      int64_t e_min = T, t_min = T;
      for (int k = tid; k < nc; k += kHB) {
        const int64_t e = S.t[k] + (T >> S.lvl[k]);
        e_min = e < e_min ? e : e_min;
        t_min = S.t[k] < t_min ? S.t[k] : t_min;
      }
      const int64_t tn = block_min(e_min, S.red[0]);
      const int64_t tmin = block_min(t_min, S.red[1]);
      if (tmin >= T) break;
      if (++iter > kHermiteIterLimit) {
        if (tid == 0) dev_fail(st, P3T_ERR_TIMEOUT, 61, 0);
        break;
      }
      // predict every member (component items)
      for (int i = item; i < nc * 3; i += kHB) {
        const int k = i / 3, q = i - 3 * k;
        const double D = (double)(tn - S.t[k]) * unit;
        const double D2 = D * D, D3 = D2 * D;
        S.p[q][k] = S.x[q][k] + S.v[q][k] * D + S.a[q][k] * D2 * 0.5 + S.j[q][k] * D3 * (1.0 / 6.0);
        S.pv[q][k] = S.v[q][k] + S.a[q][k] * D + S.j[q][k] * D2 * 0.5;
      }
      // active members in ascending order
      {
        const bool on = tid < nc && S.t[tid] + (T >> S.lvl[tid]) == tn;
        const unsigned bal = __ballot_sync(0xffffffffu, on);
        if ((tid & 31) == 0) S.wcount[tid >> 5] = __popc(bal);
        __syncthreads();
        int base = 0;
        for (int q = 0; q < (tid >> 5); ++q) base += S.wcount[q];
        if (on) S.act[base + __popc(bal & ((1u << (tid & 31)) - 1u))] = tid;
        if (tid == 0) {
          int tot = 0;
          for (int q = 0; q < kHB / 32; ++q) tot += S.wcount[q];
          S.nact = tot;
        }
      }
      // (kHMax == kHB: member k is thread k here)
      __syncthreads();
      const int nact = S.nact;
      block_forces(S, S.p, S.pv, nc, nact, item, prm, i1mg);
      // correct (component items of the active members)
      for (int i = item; i < nact * 3; i += kHB) {
        const int b = i / 3, q = i - 3 * b;
        const int k = S.act[b];
        const double D = (double)(T >> S.lvl[k]) * unit;
        const double D2 = D * D, D3 = D2 * D, D4 = D3 * D, D5 = D4 * D;
        const double iD = 1.0 / D, iD2 = iD * iD, iD3 = iD2 * iD;
        const double da = S.a[q][k] - S.a1[q][k];
        const double j0 = S.j[q][k], j1 = S.j1[q][k];
        const double A2 = (-6.0 * da - D * (4.0 * j0 + 2.0 * j1)) * iD2;
        const double A3 = (12.0 * da + 6.0 * D * (j0 + j1)) * iD3;
        S.a2e[q][k] = A2 + D * A3;
        S.a3[q][k] = A3;
        S.x[q][k] = S.p[q][k] + A2 * D4 * (1.0 / 24.0) + A3 * D5 * (1.0 / 120.0);
        S.v[q][k] = S.pv[q][k] + A2 * D3 * (1.0 / 6.0) + A3 * D4 * (1.0 / 24.0);
        S.a[q][k] = S.a1[q][k];
        S.j[q][k] = j1;
      }
      __syncthreads();
      // new steps of the active members
      for (int b = item; b < nact; b += kHB) {
        const int k = S.act[b];
        const double D = (double)(T >> S.lvl[k]) * unit;
        const int e = ilogb(D);
        const float an = norm3f(S.a[0][k], S.a[1][k], S.a[2][k], 0);
        const float jn = norm3f(S.j[0][k], S.j[1][k], S.j[2][k], e);
        const float a2n = norm3f(S.a2e[0][k], S.a2e[1][k], S.a2e[2][k], 2 * e);
        const float a3n = norm3f(S.a3[0][k], S.a3[1][k], S.a3[2][k], 3 * e);
        const float num = an * a2n + jn * jn, den = jn * a3n + a2n * a2n;
        const double dtd = den > 0.0f ? ldexp((double)sqrtf((float)prm.eta * num / den), e) : dt;
        S.t[k] = tn;
        S.lvl[k] = quantise_level(dtd, dt, S.lvl[k], tn, underflow);
      }
      if (tid == 0) steps += (unsigned long long)nact;
      __syncthreads();
    }
    for (int k = item; k < nc; k += kHB) {
      const int32_t i = cl_mem[off + k];
      p.x[i] = S.x[0][k]; p.y[i] = S.x[1][k]; p.z[i] = S.x[2][k];
      p.vx[i] = S.v[0][k]; p.vy[i] = S.v[1][k]; p.vz[i] = S.v[2][k];
    }
    __syncthreads();
  }
  if (underflow) dev_fail(st, P3T_ERR_DT_UNDERFLOW, 62, 0);
  if (tid == 0 && steps_out && steps) atomicAdd(steps_out, steps);
}

__global__ void k_zero_i64_one(int64_t *p) { *p = 0; }

// clusters of more than kHMax members (a percolating cluster): one warp each,
// members over lanes, state in the global workspace
__global__ void k_hermite(const int64_t *d_ncl, const int64_t *cl_off,
                          const int32_t *cl_mem, p3t_particles p, HWork w,
                          p3t_params prm, double dt,
                          unsigned long long *steps_out, DevStatus *st) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t ncl = *d_ncl;
  unsigned long long steps = 0;
  bool underflow = false;
  for (int64_t c = warp; c < ncl; c += nwarps) {
    const int64_t off = cl_off[c];
    const int nc = (int)(cl_off[c + 1] - off);
    if (nc <= kHMax) continue;
    integrate_cluster<32>(off, nc, cl_mem, p, w, prm, dt, lane, 0xffffffffu, steps,
                          underflow, st);
  }
  if (underflow) dev_fail(st, P3T_ERR_DT_UNDERFLOW, 62, 0);
  for (int o = 16; o > 0; o >>= 1) steps += __shfl_xor_sync(0xffffffffu, steps, o);
  if (lane == 0 && steps_out && steps) atomicAdd(steps_out, steps);
}

__global__ void k_zero_u64(unsigned long long *p) { *p = 0ull; }

// ---- row a10: energy --------------------------------------------------------
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
                                                   double *out) {
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
        sd += s_m[q] / sqrt(dx * dx + dy * dy + dz * dz);
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
  if (threadIdx.x < 3) {
    double s = 0.0;
    for (int w = 0; w < kETile / 32; ++w) s += s_red[threadIdx.x][w];
    atomicAdd(&out[1 + threadIdx.x], s);
  }
}

__global__ void k_energy_init(double *out) {
  if (threadIdx.x < 4) out[threadIdx.x] = 0.0;
}
__global__ void k_energy_final(double *out) { out[0] = out[1] + out[2] + out[3]; }

}  // namespace

int p3t_run_kick(p3t_ctx *c, p3t_particles *p, const double *ax,
                 const double *ay, const double *az, double h, cudaStream_t s) {
  if (p->n == 0) return P3T_OK;
  const int64_t g = p3t_grid(p->n, kBlock, (int64_t)c->num_sms * P3T_NSM_BLOCKS);
  k_kick<<<(unsigned)g, kBlock, 0, s>>>(p->n, p->vx, p->vy, p->vz, ax, ay, az, h);
  p3t_note_launches(1);
  return cudaGetLastError() == cudaSuccess ? P3T_OK : P3T_ERR_CUDA;
}

int p3t_run_hard_step(p3t_ctx *c, p3t_particles *p, const p3t_clusters *cl,
                      double dt, uint64_t *n_steps, cudaStream_t s) {
  const int64_t n = p->n;
  const int64_t maxb = (int64_t)c->num_sms * P3T_NSM_BLOCKS;
  const double mu = c->prm.G * c->prm.m_star;
  HWork w;
  const int64_t cap = c->cap;
  double *b = c->hw;
  double **f[] = {&w.x, &w.y, &w.z, &w.vx, &w.vy, &w.vz, &w.px, &w.py, &w.pz,
                  &w.pvx, &w.pvy, &w.pvz, &w.ax, &w.ay, &w.az, &w.jx, &w.jy, &w.jz,
                  &w.m, &w.ro};
  for (int q = 0; q < 20; ++q) *f[q] = b + q * cap;
  w.t = c->ht;
  w.lvl = c->hl;
  unsigned long long *steps = n_steps ? reinterpret_cast<unsigned long long *>(n_steps)
                                      : c->hsteps;
  k_zero_u64<<<1, 1, 0, s>>>(steps);
  // Kepler drift, small clusters and large clusters touch disjoint particles:
  // run them on three streams forked from and joined back to the caller's
  P3T_CUDA_TRY(cudaEventRecord(c->ev_fork, s));
  P3T_CUDA_TRY(cudaStreamWaitEvent(c->aux[0], c->ev_fork, 0));
  P3T_CUDA_TRY(cudaStreamWaitEvent(c->aux[1], c->ev_fork, 0));
  // clusters of <= kHMax members: a block each, handed out dynamically (a
  // long encounter keeps its block while the others move on); larger ones: a
  // warp each
  const int64_t ncl_max = (n / 2) > 0 ? n / 2 : 1;
  k_zero_i64_one<<<1, 1, 0, c->aux[0]>>>(c->hcursor);
  k_hermite_block<<<(unsigned)p3t_grid(ncl_max * kHB, kHB, (int64_t)c->num_sms * 4), kHB, 0,
                    c->aux[0]>>>(&cl->counts[1], cl->cl_off, cl->cl_mem, *p, c->prm, dt, steps,
                                 c->hcursor, c->status);
  k_hermite<<<(unsigned)p3t_grid(ncl_max * 32, 128, maxb), 128, 0, c->aux[1]>>>(
      &cl->counts[1], cl->cl_off, cl->cl_mem, *p, w, c->prm, dt, steps, c->status);
  k_kepler<<<(unsigned)p3t_grid(n, 128, maxb), 128, 0, s>>>(&cl->counts[0], cl->singles, *p,
                                                             dt, mu, c->status);
  P3T_CUDA_TRY(cudaEventRecord(c->ev_join[0], c->aux[0]));
  P3T_CUDA_TRY(cudaEventRecord(c->ev_join[1], c->aux[1]));
  P3T_CUDA_TRY(cudaStreamWaitEvent(s, c->ev_join[0], 0));
  P3T_CUDA_TRY(cudaStreamWaitEvent(s, c->ev_join[1], 0));
  p3t_note_launches(5);
  return cudaGetLastError() == cudaSuccess ? P3T_OK : P3T_ERR_CUDA;
}

int p3t_run_energy(p3t_ctx *c, const p3t_particles *p, double *out, cudaStream_t s) {
  k_energy_init<<<1, 32, 0, s>>>(out);
  if (p->n > 0) {
    const unsigned g = (unsigned)((p->n + kETile - 1) / kETile);
    if (c->prm.precision == P3T_MIXED)
      k_energy<true><<<g, kETile, 0, s>>>(*p, c->prm, out);
    else
      k_energy<false><<<g, kETile, 0, s>>>(*p, c->prm, out);
  }
  k_energy_final<<<1, 1, 0, s>>>(out);
  p3t_note_launches(p->n > 0 ? 3 : 2);
  return cudaGetLastError() == cudaSuccess ? P3T_OK : P3T_ERR_CUDA;
}

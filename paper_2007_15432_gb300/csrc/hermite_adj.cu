// Adjoint of the hard part of a soft step (procedure step 5) for the members
// of neighbour clusters: the vector-Jacobian product of the cluster's
// Hermite-4 block-step integration over [0, dt] (Sec. 2.1.2; Eq. hardforce)
// with the block schedule held fixed, through forward-mode tangents.
//
// One thread per (cluster member, direction): the direction is one of the
// member's six state components or its mass.  The thread integrates the
// whole cluster in plain FP64 arithmetic (each formula as written: the
// predictor to the jerk, the Makino & Aarseth corrector, the Aarseth step,
// the first step eta0 |a| / |j|, block steps dt / 2^k, k <= 40, at most
// twice the previous one and commensurate with the particle time) carrying
// one tangent along with every value; the step decisions use the values
// only, so the tangent is the derivative of the integration with its
// schedule fixed.  The tangent of the final state, dotted with the adjoint
// of the final state, is one component of Phi^T lam (or dL/dm for a mass
// direction).  Clusters above kTMax members are not integrated here
// (P3T_ERR_CAPACITY).  No collisions (f_radius = 0).
#include <math.h>

#include "p3t_internal.cuh"

namespace {

constexpr int kTMax = 16;  // largest cluster the tangent kernel integrates
constexpr int kLv = 40;    // finest block level, dt / 2^40

struct D1 {
  double v, d;  // value and tangent
};
__device__ __forceinline__ D1 dk(double v) { return {v, 0.0}; }
__device__ __forceinline__ D1 operator+(D1 a, D1 b) { return {a.v + b.v, a.d + b.d}; }
__device__ __forceinline__ D1 operator-(D1 a, D1 b) { return {a.v - b.v, a.d - b.d}; }
__device__ __forceinline__ D1 operator-(D1 a) { return {-a.v, -a.d}; }
__device__ __forceinline__ D1 operator*(D1 a, D1 b) { return {a.v * b.v, a.d * b.v + a.v * b.d}; }
__device__ __forceinline__ D1 operator*(double s, D1 a) { return {s * a.v, s * a.d}; }
__device__ __forceinline__ D1 operator/(D1 a, D1 b) {
  const double q = a.v / b.v;
  return {q, (a.d - q * b.d) / b.v};
}
__device__ __forceinline__ D1 operator/(D1 a, double s) { return {a.v / s, a.d / s}; }
__device__ __forceinline__ D1 dsqrt(D1 a) {
  const double r = sqrt(a.v);
  return {r, a.v > 0.0 ? a.d / (2.0 * r) : 0.0};
}

// level of the step dt_des: the largest dt / 2^l not above it, l <= 40, at
// most twice the previous step, commensurate with the time t (units dt/2^40)
__device__ int level_of(double dt_des, double dt, int prev, int64_t t, bool &uf) {
  int l = 0;
  while (l < kLv && ldexp(dt, -l) > dt_des) ++l;
  if (ldexp(dt, -l) > dt_des) uf = true;
  if (l < prev - 1) l = prev - 1;
  while (l < kLv && (t & ((((int64_t)1) << (kLv - l)) - 1)) != 0) ++l;
  return l;
}

// hard acceleration and jerk of member k (Eq. hardforce): the star and the
// (1 - K) part of every other member's pull, the jerk with dK/dt
__device__ void acc_jerk(int nc, const D1 (*x)[3], const D1 (*v)[3], const D1 *m,
                         const double *ro, int k, const p3t_params &prm, D1 a[3], D1 j[3]) {
  for (int c = 0; c < 3; ++c) { a[c] = dk(0.0); j[c] = dk(0.0); }
  {
    const D1 r2 = x[k][0] * x[k][0] + x[k][1] * x[k][1] + x[k][2] * x[k][2];
    const D1 r = dsqrt(r2);
    const D1 r3 = r2 * r, r5 = r3 * r2;
    const D1 rv = x[k][0] * v[k][0] + x[k][1] * v[k][1] + x[k][2] * v[k][2];
    const double GM = prm.G * prm.m_star;
    for (int c = 0; c < 3; ++c) {
      a[c] = a[c] - (GM * x[k][c]) / r3;
      j[c] = j[c] - GM * (v[k][c] / r3 - ((3.0 * rv) * x[k][c]) / r5);
    }
  }
  const double i1mg = 1.0 / (1.0 - prm.gamma);
  for (int q = 0; q < nc; ++q) {
    if (q == k) continue;
    D1 rr[3], uu[3];
    for (int c = 0; c < 3; ++c) { rr[c] = x[k][c] - x[q][c]; uu[c] = v[k][c] - v[q][c]; }
    const D1 r2 = rr[0] * rr[0] + rr[1] * rr[1] + rr[2] * rr[2];
    if (r2.v == 0.0) continue;
    const D1 r = dsqrt(r2);
    const double roij = ro[k] > ro[q] ? ro[k] : ro[q];
    const D1 y = r / roij;
    if (y.v >= 1.0) continue;
    D1 w = dk(1.0), dK = dk(0.0);
    if (y.v > prm.gamma) {
      const D1 xs = (y - dk(prm.gamma)) * dk(i1mg);
      const D1 x2 = xs * xs, x3 = x2 * xs, us = dk(1.0) - xs;
      w = dk(1.0) - x2 * x2 * (dk(35.0) - 84.0 * xs + 70.0 * x2 - 20.0 * x3);
      dK = (140.0 * xs * xs * xs * us * us * us) / (1.0 - prm.gamma);
    }
    const D1 r3 = r2 * r, r5 = r3 * r2;
    const D1 rv = rr[0] * uu[0] + rr[1] * uu[1] + rr[2] * uu[2];
    const D1 Gm = prm.G * m[q];
    const D1 dw = dK * rv / (r * dk(roij));  // -d(1 - K)/dt
    for (int c = 0; c < 3; ++c) {
      a[c] = a[c] - Gm * w * rr[c] / r3;
      j[c] = j[c] - Gm * (w * (uu[c] / r3 - ((3.0 * rv) * rr[c]) / r5) - dw * rr[c] / r3);
    }
  }
}

__device__ __forceinline__ double norm3v(const D1 *u) {
  return sqrt(u[0].v * u[0].v + u[1].v * u[1].v + u[2].v * u[2].v);
}

// thread t: member slot u = t / 7 of the cluster list, direction t % 7
// (x, y, z, vx, vy, vz, m); writes the state directions' results to
// lin[6 u + dir] and adds the mass direction's to gm
__global__ void k_hermite_tangent(const int64_t *counts, const int64_t *cl_off,
                                  const int32_t *cl_mem, p3t_particles p, p3t_params prm,
                                  double dt, const double *lx, const double *ly, const double *lz,
                                  const double *lvx, const double *lvy, const double *lvz,
                                  double *lin, double *gm, DevStatus *st) {
  pdl_wait();
  const int64_t ncl = counts[1], nmem = counts[2];
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < 7 * nmem;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t u = t / 7;
    const int dir = (int)(t - 7 * u);
    int64_t lo = 0, hi = ncl;  // the cluster c with cl_off[c] <= u < cl_off[c + 1]
    while (hi - lo > 1) {
      const int64_t mid = (lo + hi) / 2;
      if (cl_off[mid] <= u) lo = mid; else hi = mid;
    }
    const int64_t off = cl_off[lo];
    const int nc = (int)(cl_off[lo + 1] - off);
    if (nc > kTMax) {
      dev_fail(st, P3T_ERR_CAPACITY, 80, nc);
      continue;
    }
    const int ks = (int)(u - off);  // the seeded member
    D1 x[kTMax][3], v[kTMax][3], a[kTMax][3], jk[kTMax][3], m[kTMax];
    D1 px[kTMax][3], pv[kTMax][3], a1[kTMax][3], j1[kTMax][3];
    double ro[kTMax];
    int64_t tt[kTMax];
    int lvl[kTMax];
    bool act[kTMax];
    for (int k = 0; k < nc; ++k) {
      const int32_t i = cl_mem[off + k];
      x[k][0] = dk(p.x[i]); x[k][1] = dk(p.y[i]); x[k][2] = dk(p.z[i]);
      v[k][0] = dk(p.vx[i]); v[k][1] = dk(p.vy[i]); v[k][2] = dk(p.vz[i]);
      m[k] = dk(p.m[i]);
      ro[k] = p.r_out[i];
    }
    if (dir < 3) x[ks][dir].d = 1.0;
    else if (dir < 6) v[ks][dir - 3].d = 1.0;
    else m[ks].d = 1.0;
    const int64_t T = ((int64_t)1) << kLv;
    const double unit = ldexp(dt, -kLv);
    bool uf = false;
    for (int k = 0; k < nc; ++k) {
      acc_jerk(nc, x, v, m, ro, k, prm, a[k], jk[k]);
      const double jn = norm3v(jk[k]);
      const double d0 = jn > 0.0 ? prm.eta0 * norm3v(a[k]) / jn : dt;
      tt[k] = 0;
      lvl[k] = level_of(d0, dt, 0, 0, uf);
    }
    for (int64_t blocks = 0; !uf; ++blocks) {
      if (blocks > ((int64_t)1 << 24)) { dev_fail(st, P3T_ERR_TIMEOUT, 81, 0); break; }
      int64_t tn = T, tmin = T;
      for (int k = 0; k < nc; ++k) {
        const int64_t e = tt[k] + (T >> lvl[k]);
        tn = e < tn ? e : tn;
        tmin = tt[k] < tmin ? tt[k] : tmin;
      }
      if (tmin >= T) break;
      for (int k = 0; k < nc; ++k) {
        const double D = (double)(tn - tt[k]) * unit, D2 = D * D, D3 = D2 * D;
        for (int c = 0; c < 3; ++c) {
          px[k][c] = x[k][c] + D * v[k][c] + (D2 * a[k][c]) / 2.0 + (D3 * jk[k][c]) / 6.0;
          pv[k][c] = v[k][c] + D * a[k][c] + (D2 * jk[k][c]) / 2.0;
        }
        act[k] = tt[k] + (T >> lvl[k]) == tn;
      }
      for (int k = 0; k < nc; ++k)
        if (act[k]) acc_jerk(nc, px, pv, m, ro, k, prm, a1[k], j1[k]);
      for (int k = 0; k < nc; ++k) {
        if (!act[k]) continue;
        const double D = (double)(T >> lvl[k]) * unit;
        const double D2 = D * D, D3 = D2 * D, D4 = D3 * D, D5 = D4 * D;
        D1 A2[3], A3[3], A2e[3];
        for (int c = 0; c < 3; ++c) {
          const D1 da = a[k][c] - a1[k][c];
          A2[c] = (-6.0 * da - D * (4.0 * jk[k][c] + 2.0 * j1[k][c])) / D2;
          A3[c] = (12.0 * da + (6.0 * D) * (jk[k][c] + j1[k][c])) / D3;
          A2e[c] = A2[c] + D * A3[c];
        }
        for (int c = 0; c < 3; ++c) {
          x[k][c] = px[k][c] + (D4 * A2[c]) / 24.0 + (D5 * A3[c]) / 120.0;
          v[k][c] = pv[k][c] + (D3 * A2[c]) / 6.0 + (D4 * A3[c]) / 24.0;
          a[k][c] = a1[k][c];
          jk[k][c] = j1[k][c];
        }
        const double an = norm3v(a[k]), jn = norm3v(jk[k]);
        const double a2n = norm3v(A2e), a3n = norm3v(A3);
        const double num = an * a2n + jn * jn, den = jn * a3n + a2n * a2n;
        const double dd = den > 0.0 ? sqrt(prm.eta * num / den) : dt;
        tt[k] = tn;
        lvl[k] = level_of(dd, dt, lvl[k], tn, uf);
      }
    }
    if (uf) dev_fail(st, P3T_ERR_DT_UNDERFLOW, 82, 0);
    double r = 0.0;
    for (int k = 0; k < nc; ++k) {
      const int32_t i = cl_mem[off + k];
      r += lx[i] * x[k][0].d + ly[i] * x[k][1].d + lz[i] * x[k][2].d +
           lvx[i] * v[k][0].d + lvy[i] * v[k][1].d + lvz[i] * v[k][2].d;
    }
    if (dir < 6) lin[6 * u + dir] = r;
    else gm[cl_mem[u]] += r;
  }
}

// the members' adjoints before the hard step, from lin
__global__ void k_member_adjoint(const int64_t *counts, const int32_t *cl_mem, const double *lin,
                                 double *lx, double *ly, double *lz, double *lvx, double *lvy,
                                 double *lvz) {
  pdl_wait();
  const int64_t nmem = counts[2];
  for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < nmem;
       u += (int64_t)gridDim.x * blockDim.x) {
    const int32_t i = cl_mem[u];
    lx[i] = lin[6 * u]; ly[i] = lin[6 * u + 1]; lz[i] = lin[6 * u + 2];
    lvx[i] = lin[6 * u + 3]; lvy[i] = lin[6 * u + 4]; lvz[i] = lin[6 * u + 5];
  }
}

}  // namespace

// Phi^T lam for the hard part of a soft step: cluster members through the
// tangent kernel, isolated particles through the Kepler drift's adjoint
// (applied to every particle first; the members' results then replace it)
int p3t_run_hard_step_vjp(p3t_ctx *c, const p3t_particles *p, const p3t_clusters *cl, double dt,
                          double *lx, double *ly, double *lz, double *lvx, double *lvy,
                          double *lvz, double *gm, cudaStream_t s) {
  const int64_t n = p->n;
  if (n == 0) return P3T_OK;
  const int64_t maxb = (int64_t)c->num_sms * P3T_NSM_BLOCKS;
  pdl_launch(k_hermite_tangent, dim3((unsigned)p3t_grid(7 * n, 128, maxb)), dim3(128), 0, s, 
      cl->counts, cl->cl_off, cl->cl_mem, *p, c->prm, dt, lx, ly, lz, lvx, lvy, lvz, c->hadj, gm,
      c->status);
  int rc = p3t_run_kepler_vjp(c, p, dt, lx, ly, lz, lvx, lvy, lvz, s);
  if (rc) return rc;
  pdl_launch(k_member_adjoint, dim3((unsigned)p3t_grid(n, 128, maxb)), dim3(128), 0, s, cl->counts, cl->cl_mem,
                                                                     c->hadj, lx, ly, lz, lvx,
                                                                     lvy, lvz);
  p3t_note_launches(2);
  return cudaGetLastError() == cudaSuccess ? P3T_OK : P3T_ERR_CUDA;
}

// Soft step: cut-off radii, Morton keys and sort, octree
// with monopole + quadrupole moments.  Compiled with -fmad=false: the keys
// and the integer grid geometry must be bit-identical on every IEEE machine.
#include <math.h>

#include "p3t_internal.cuh"
#include "exact_conv.cuh"

namespace {

constexpr int kBlock = 256;

// order-preserving map of doubles to unsigned 64-bit integers
__device__ __forceinline__ unsigned long long ord_bits(double v) {
  unsigned long long b = (unsigned long long)__double_as_longlong(v);
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ double ord_double(unsigned long long b) {
  b = (b >> 63) ? (b & 0x7fffffffffffffffull) : ~b;
  return __longlong_as_double((long long)b);
}

// =========================================================================
// Cut-off radii (Eq. routi2, Eq. rsearch).  Random velocity
// u = v - sqrt(G M_* / |x|) phi_hat (phi_hat: cylindrical azimuth),
// v_ran = rms |u| over radial bins uniform in ln R_cyl.
// =========================================================================
// per segment d: bits[4d] min R, bits[4d + 1] max R, bits[4d + 2], [4d + 3]
// the largest r_out and r_search (shared scheme)
__global__ void k_cut_init(unsigned long long *bits, int nseg, double *bsum,
                           unsigned long long *bcnt, int nb) {
  pdl_wait();
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  for (int d = t; d < nseg; d += gridDim.x * blockDim.x) {
    bits[4 * d] = ~0ull; bits[4 * d + 1] = 0ull; bits[4 * d + 2] = 0ull; bits[4 * d + 3] = 0ull;
  }
  for (int k = t; k < nb; k += gridDim.x * blockDim.x) { bsum[k] = 0.0; bcnt[k] = 0ull; }
}

// a block's slice of its segment: blocks [d * slices, (d + 1) * slices) take
// segment d in contiguous slices
__device__ __forceinline__ void seg_slice(const SegView &sv, int slices, int &d, int64_t &a,
                                          int64_t &b) {
  d = (int)(blockIdx.x / slices);
  const int sl = (int)(blockIdx.x % slices);
  const int64_t s0 = seg_lo(sv, d), len = seg_hi(sv, d) - s0;
  a = s0 + len * sl / slices;
  b = s0 + len * (sl + 1) / slices;
}

__global__ void k_cut_range(SegView sv, int slices, const double *x, const double *y,
                            unsigned long long *bits) {
  pdl_wait();
  int d;
  int64_t a, b;
  seg_slice(sv, slices, d, a, b);
  unsigned long long lo = ~0ull, hi = 0ull;
  for (int64_t i = a + threadIdx.x; i < b; i += blockDim.x) {
    unsigned long long v = ord_bits(sqrt(x[i] * x[i] + y[i] * y[i]));
    lo = v < lo ? v : lo;
    hi = v > hi ? v : hi;
  }
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long u = __shfl_xor_sync(0xffffffffu, lo, o);
    unsigned long long c = __shfl_xor_sync(0xffffffffu, hi, o);
    lo = u < lo ? u : lo;
    hi = c > hi ? c : hi;
  }
  if ((threadIdx.x & 31) == 0) { atomicMin(&bits[4 * d], lo); atomicMax(&bits[4 * d + 1], hi); }
}

// radial bins of each segment (several segments): their number (as for a
// single system), first global bin and log R range
__global__ void k_cut_segbins(SegView sv, int vran_bins, const unsigned long long *bits,
                              int32_t *seg_nb, int32_t *seg_base, double *seg_l) {
  pdl_wait();
  __shared__ int wsum[32];
  __shared__ int carry;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < sv.nseg; base += blockDim.x) {
    const int d = base + threadIdx.x;
    int nb = 0;
    if (d < sv.nseg) {
      nb = vran_bins;
      if (nb <= 0) {
        const int64_t t = (seg_hi(sv, d) - seg_lo(sv, d)) / 1000;
        nb = (int)(t < 1 ? 1 : (t > 1024 ? 1024 : t));
      }
      seg_nb[d] = nb;
      seg_l[2 * d] = log(ord_double(bits[4 * d]));
      seg_l[2 * d + 1] = log(ord_double(bits[4 * d + 1]));
    }
    int x = nb;
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += t;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
      const int w0 = lane < nw ? wsum[lane] : 0;
      int y = w0;
      for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, y, o);
        if (lane >= o) y += t;
      }
      if (lane < nw) wsum[lane] = y - w0;
    }
    __syncthreads();
    const int ex = carry + wsum[warp] + (x - nb);
    if (d < sv.nseg) seg_base[d] = ex;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry = ex + nb;
    __syncthreads();
  }
}

// bin of ln R among nb bins uniform on [lmin, lmax]: floor(nb (ln R - lmin) /
// (lmax - lmin)) clamped to [0, nb - 1], decided in FP64.  An FP32 estimate
// decides it first when no integer lies within its error bound of the
// estimate (logf and the roundings to FP32 stay within 2e-6 absolute on ln R
// and on each bound); otherwise the FP64 expression is evaluated.
__device__ __forceinline__ int cut_bin(double R, double Rmin, double Rmax,
                                       double lmin, double lmax, int nb) {
  int k = 0;
  if (Rmax > Rmin && R > Rmin) {
    const float lminf = (float)lmin, span = (float)lmax - lminf;
    const float tf = (logf((float)R) - lminf) / span * (float)nb;
    const float margin = 8e-6f * (float)nb / span + 1e-3f;
    double f;
    if (span > 0.0f && margin < 0.25f && floorf(tf - margin) == floorf(tf + margin)) {
      f = (double)floorf(tf);
    } else {
      double t = (log(R) - lmin) / (lmax - lmin);
      f = floor(t * (double)nb);
    }
    k = f < 0.0 ? 0 : (f > (double)(nb - 1) ? nb - 1 : (int)f);
  }
  return k;
}

// |u|^2 and the radial bin of every particle (kept for k_cut_final); bin
// counts (integer atomics, first into the block's shared histogram);
// (bin, index) pairs for a stable sort by bin
constexpr int kMaxBins = 4096;
__global__ void k_cut_u2(SegView sv, const double *x, const double *y, const double *z,
                         const double *vx, const double *vy, const double *vz, double mu,
                         const unsigned long long *bits, int nb, const int32_t *seg_nb,
                         const int32_t *seg_base, const double *seg_l, double *u2,
                         uint64_t *key, int32_t *idx, int32_t *bin, unsigned long long *bcnt) {
  pdl_wait();
  __shared__ uint32_t h[kMaxBins];
  for (int k = threadIdx.x; k < nb; k += blockDim.x) h[k] = 0;
  __syncthreads();
  const int64_t n = sv.n;
  // one segment: its range here; several: per particle below
  const double Rmin0 = ord_double(bits[0]), Rmax0 = ord_double(bits[1]);
  const double lmin0 = log(Rmin0), lmax0 = log(Rmax0);
  const double smu = sqrt(mu);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double R2 = x[i] * x[i] + y[i] * y[i];
    const double R = sqrt(R2);
    const double r = sqrt(R2 + z[i] * z[i]);
    const double vk = smu * rsqrt(r);  // sqrt(mu / r)
    double px = 0.0, py = 0.0;
    if (R > 0.0) {
      const double iR = rsqrt(R2);
      px = -y[i] * iR;
      py = x[i] * iR;
    }
    double ux = vx[i] - vk * px, uy = vy[i] - vk * py, uz = vz[i];
    u2[i] = ux * ux + uy * uy + uz * uz;
    int k;
    if (sv.nseg == 1) {
      k = cut_bin(R, Rmin0, Rmax0, lmin0, lmax0, nb);
    } else {
      const int d = seg_of(sv, i);
      k = seg_base[d] + cut_bin(R, ord_double(bits[4 * d]), ord_double(bits[4 * d + 1]),
                                seg_l[2 * d], seg_l[2 * d + 1], seg_nb[d]);
    }
    key[i] = (uint64_t)k;
    idx[i] = (int32_t)i;
    bin[i] = k;
    atomicAdd(&h[k], 1u);
  }
  __syncthreads();
  for (int k = threadIdx.x; k < nb; k += blockDim.x)
    if (h[k]) atomicAdd(&bcnt[k], (unsigned long long)h[k]);
}

// exclusive offsets of the bins (at most 4096): one block, chunks of its
// size scanned with warp shuffles and carried
__global__ void k_cut_offsets(int nb, const unsigned long long *bcnt, int64_t *boff) {
  pdl_wait();
  __shared__ int64_t wsum[32];
  __shared__ int64_t carry;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < nb; base += blockDim.x) {
    const int k = base + threadIdx.x;
    const int64_t v = k < nb ? (int64_t)bcnt[k] : 0;
    int64_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t t = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += t;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
      const int64_t w0 = lane < nw ? wsum[lane] : 0;
      int64_t y = w0;
      for (int o = 1; o < 32; o <<= 1) {
        const int64_t t = __shfl_up_sync(0xffffffffu, y, o);
        if (lane >= o) y += t;
      }
      if (lane < nw) wsum[lane] = y - w0;
    }
    __syncthreads();
    const int64_t ex = carry + wsum[warp] + (x - v);
    if (k < nb) boff[k] = ex;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry = ex + v;
    __syncthreads();
  }
  if (threadIdx.x == 0) boff[nb] = carry;
}

// v_ran of each bin, sqrt(sum |u|^2 / count), the sum by one warp per bin
// over its members in index order (a fixed lane-strided order and a fixed
// shuffle tree: the same sum on every run)
__global__ void k_cut_binsum(int nb, const int64_t *boff, const int32_t *sorted_idx,
                             const double *u2, double *bvr) {
  pdl_wait();
  const int lane = threadIdx.x & 31;
  const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t k = w0; k < nb; k += nw) {
    double sum = 0.0;
    for (int64_t j = boff[k] + lane; j < boff[k + 1]; j += 32) sum += u2[sorted_idx[j]];
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if (lane == 0) bvr[k] = sqrt(sum / (double)(boff[k + 1] - boff[k]));
  }
}

// x^(1/3) for x >= 0: the inverse cube root z = x^(-1/3) by Newton's method
// on f(z) = z^-3 - x, z <- z (4 - x z^3) / 3 (quadratic convergence), from an
// FP32 seed (relative error ~1e-7) in two steps, then x^(1/3) = x z^2; inputs
// outside the FP32 seed's normal range take cbrt
__device__ __forceinline__ double cbrt_pos(double x) {
  if (!(x > 1e-30 && x < 1e30)) return cbrt(x);
  double z = (double)rcbrtf((float)x);
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    const double z3 = z * z * z;
    z = z * (4.0 - x * z3) * (1.0 / 3.0);
  }
  return x * z * z;
}

__global__ void k_cut_final(SegView sv, const double *x, const double *y,
                            const double *z, const double *vx, const double *vy,
                            const double *vz, const double *m, p3t_params prm,
                            unsigned long long *bits, const int32_t *bin,
                            const double *bvr, double *r_out, double *r_search) {
  pdl_wait();
  const double imu = 1.0 / (prm.G * prm.m_star), i3ms = 1.0 / (3.0 * prm.m_star);
  const int64_t n = sv.n;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double r2 = x[i] * x[i] + y[i] * y[i] + z[i] * z[i];
    const double ir = rsqrt(r2);
    double v2 = vx[i] * vx[i] + vy[i] * vy[i] + vz[i] * vz[i];
    double alpha = 2.0 * ir - v2 * imu;  // 1/a, vis-viva
    double a = alpha > 0.0 ? 1.0 / alpha : r2 * ir;
    double rhill = cbrt_pos(m[i] * i3ms) * a;
    const double vr = bvr[bin[i]];
    // Eq. routi2 (P3T_CUT_HILL_VRAN) or Eq. routi (the other two); Eq. rsearch
    const double ro = prm.cutoff_mode == P3T_CUT_HILL_VRAN
                          ? fmax(prm.rcut0 * rhill, prm.rcut1 * vr * prm.dt_soft)
                          : prm.rcut0 * rhill;
    const double rs = prm.rs0 * ro + prm.rs1 * vr * prm.dt_soft;
    r_out[i] = ro;
    r_search[i] = rs;
    if (prm.cutoff_mode == P3T_CUT_SHARED) {
      // non-negative doubles order like their bit patterns
      const int d = seg_at(sv, i);
      atomicMax(&bits[4 * d + 2], (unsigned long long)__double_as_longlong(ro));
      atomicMax(&bits[4 * d + 3], (unsigned long long)__double_as_longlong(rs));
    }
  }
}

// shared cut-off (Eq. rout1): every particle gets the largest r_out and the
// largest search radius
__global__ void k_cut_shared(SegView sv, const unsigned long long *bits, double *r_out,
                             double *r_search) {
  pdl_wait();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < sv.n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int d = seg_at(sv, i);
    r_out[i] = __longlong_as_double((long long)bits[4 * d + 2]);
    r_search[i] = __longlong_as_double((long long)bits[4 * d + 3]);
  }
}

// =========================================================================
// Keys, sort, octree, moments.
// =========================================================================
__global__ void k_set_i64(int64_t *dst, int64_t v) {
  pdl_wait(); *dst = v; }

__global__ void k_box_init(unsigned long long *bits, int nseg) {
  pdl_wait();
  for (int d = threadIdx.x; d < nseg; d += blockDim.x)
    for (int a = 0; a < 3; ++a) { bits[6 * d + a] = ~0ull; bits[6 * d + 3 + a] = 0ull; }
}

// min / max of the positions of each segment: warp and block reductions over
// a block's slice of its segment, then six atomics per block
__global__ void k_box(SegView sv, int slices, const double *x, const double *y,
                      const double *z, unsigned long long *bits6) {
  pdl_wait();
  __shared__ unsigned long long red[6][kBlock / 32];
  int d;
  int64_t sa, sb;
  seg_slice(sv, slices, d, sa, sb);
  unsigned long long *bits = bits6 + 6 * d;
  unsigned long long lo[3] = {~0ull, ~0ull, ~0ull}, hi[3] = {0ull, 0ull, 0ull};
  // four elements a trip, their loads issued before the first is used
  for (int64_t i0 = sa + threadIdx.x; i0 < sb; i0 += 4 * (int64_t)blockDim.x) {
    double v[4][3];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int64_t i = i0 + k * (int64_t)blockDim.x;
      if (i < sb) { v[k][0] = x[i]; v[k][1] = y[i]; v[k][2] = z[i]; }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (i0 + k * (int64_t)blockDim.x < sb) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          const unsigned long long b = ord_bits(v[k][a]);
          lo[a] = b < lo[a] ? b : lo[a];
          hi[a] = b > hi[a] ? b : hi[a];
        }
      }
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    for (int o = 16; o > 0; o >>= 1) {
      unsigned long long u = __shfl_xor_sync(0xffffffffu, lo[a], o);
      unsigned long long v = __shfl_xor_sync(0xffffffffu, hi[a], o);
      lo[a] = u < lo[a] ? u : lo[a];
      hi[a] = v > hi[a] ? v : hi[a];
    }
    if ((threadIdx.x & 31) == 0) { red[a][threadIdx.x >> 5] = lo[a]; red[3 + a][threadIdx.x >> 5] = hi[a]; }
  }
  __syncthreads();
  if (threadIdx.x < 6) {
    const int a = threadIdx.x;
    unsigned long long r = red[a][0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
      r = a < 3 ? (red[a][w] < r ? red[a][w] : r) : (red[a][w] > r ? red[a][w] : r);
    if (a < 3) atomicMin(&bits[a], r); else atomicMax(&bits[a], r);
  }
}

// root cube of each segment: corner at the per-axis minimum, side = largest
// extent; box[5 d ..]: corner, side L, quantisation scale S
__global__ void k_box_final(const unsigned long long *bits6, double *box5, int nseg) {
  pdl_wait();
  for (int d = threadIdx.x; d < nseg; d += blockDim.x) {
    const unsigned long long *bits = bits6 + 6 * d;
    double *box = box5 + 5 * d;
    double lo[3], hi[3];
    for (int a = 0; a < 3; ++a) { lo[a] = ord_double(bits[a]); hi[a] = ord_double(bits[3 + a]); }
    double L = fmax(hi[0] - lo[0], fmax(hi[1] - lo[1], hi[2] - lo[2]));
    if (!(L > 0.0)) L = 1.0;
    box[0] = lo[0]; box[1] = lo[1]; box[2] = lo[2]; box[3] = L;
    box[4] = (double)P3T_QMAX / L;  // quantisation scale S
  }
}

__device__ __forceinline__ uint64_t spread3(uint64_t v) {
  v &= 0x1fffffull;
  v = (v | (v << 32)) & 0x1f00000000ffffull;
  v = (v | (v << 16)) & 0x1f0000ff0000ffull;
  v = (v | (v << 8)) & 0x100f00f00f00f00full;
  v = (v | (v << 4)) & 0x10c30c30c30c30c3ull;
  v = (v | (v << 2)) & 0x1249249249249249ull;
  return v;
}
__device__ __forceinline__ uint32_t compact3(uint64_t v) {
  v &= 0x1249249249249249ull;
  v = (v ^ (v >> 2)) & 0x10c30c30c30c30c3ull;
  v = (v ^ (v >> 4)) & 0x100f00f00f00f00full;
  v = (v ^ (v >> 8)) & 0x1f0000ff0000ffull;
  v = (v ^ (v >> 16)) & 0x1f00000000ffffull;
  v = (v ^ (v >> 32)) & 0x1fffffull;
  return (uint32_t)v;
}

// Morton key of each particle on its segment's grid.  rekey = 0: slot s holds
// particle s (idx[s] = s), and the particle's record (x, y, z, m, r_out,
// r_search) is packed for the gather (one 48-byte read per particle there in
// place of six scattered 8-byte ones); rekey = 1: slot s holds particle idx[s]
// (the keys of an order already sorted)
__global__ void k_keys(SegView sv, const double *x, const double *y,
                       const double *z, const double *m, const double *ro,
                       const double *rs, const double *box5, uint64_t *keys,
                       int32_t *idx, double *pack, int rekey, int64_t *d_n) {
  pdl_wait();
  const int64_t n = sv.n;
  if (d_n && blockIdx.x == 0 && threadIdx.x == 0) *d_n = n;  // for the count-driven primitives
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n;
       s += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = rekey ? (int64_t)idx[s] : s;
    const double *box = box5 + 5 * seg_at(sv, i);
    const CellScale cs = cell_scale(box[3]);
    const double X = x[i], Y = y[i], Z = z[i];
    const uint64_t qx = quantise(X, box[0], cs), qy = quantise(Y, box[1], cs),
                   qz = quantise(Z, box[2], cs);
    keys[s] = (spread3(qx) << 2) | (spread3(qy) << 1) | spread3(qz);
    if (!rekey) {
      idx[s] = (int32_t)s;
      double2 *o = reinterpret_cast<double2 *>(pack + 6 * s);
      o[0] = make_double2(X, Y);
      o[1] = make_double2(Z, m[s]);
      o[2] = make_double2(ro[s], rs[s]);
    }
  }
}

// the segment of the particle in each slot, as the key of a stable sort
// that brings each segment's particles together in key order
__global__ void k_segkey(SegView sv, const int32_t *idx, uint64_t *keys) {
  pdl_wait();
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < sv.n;
       s += (int64_t)gridDim.x * blockDim.x)
    keys[s] = (uint64_t)seg_of(sv, idx[s]);
}

// gather sorted copies: the FP64 arrays the FP64 path reads, or the
// float-float packing the mixed path reads (each path writes only its own)
template <bool MIXED>
__global__ void k_gather(int64_t n, const int32_t *idx, const uint64_t *keys,
                         const double *pack, double *sx, double *sy, double *sz, double *sm,
                         double *sro, double *srs, int32_t *sq, float4 *spA,
                         float4 *spB, float *srs32, float *sml) {
  pdl_wait();
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n;
       s += (int64_t)gridDim.x * blockDim.x) {
    const int32_t i = idx[s];
    const double2 *rec = reinterpret_cast<const double2 *>(pack + 6 * (int64_t)i);
    const double2 r0 = rec[0], r1 = rec[1], r2 = rec[2];
    const double X = r0.x, Y = r0.y, Z = r1.x, M = r1.y, RO = r2.x, RS = r2.y;
    srs[s] = RS;
    const uint64_t k = keys[s];
    sq[3 * s + 0] = (int32_t)compact3(k >> 2);
    sq[3 * s + 1] = (int32_t)compact3(k >> 1);
    sq[3 * s + 2] = (int32_t)compact3(k);
    if constexpr (!MIXED) {
      sx[s] = X; sy[s] = Y; sz[s] = Z; sm[s] = M; sro[s] = RO;
      continue;
    }
    float xh, xl, yh, yl, zh, zl, mh, ml, roh, rol, r2h, r2l;
    split_f32(X, xh, xl);
    split_f32(Y, yh, yl);
    split_f32(Z, zh, zl);
    split_f32(M, mh, ml);
    split_f32(RO, roh, rol);
    split_f32(RS * RS, r2h, r2l);
    spA[s] = make_float4(xh, yh, zh, mh);
    sml[s] = ml;
    spB[s] = make_float4(xl, yl, zl, 1.0f / roh);  // FP32 path only
    srs32[s] = r2h * 1.00001f;  // walk's candidate test: r^2 vs r_search^2, widened
  }
}

// common prefix of two keys in levels (0..21)
__device__ __forceinline__ int lcp_levels(uint64_t a, uint64_t b) {
  uint64_t d = a ^ b;
  if (d == 0) return P3T_BITS;
  return (__clzll((long long)d) - 1) / 3;
}

// Each particle's common prefix with its predecessor (lp, levels; -1 at a
// segment's first particle), its leaf level and the number of nodes it starts.
// The cell of i at level l holds more than `leaf` particles iff some window
// of leaf + 1 consecutive sorted particles containing i (within its segment)
// shares the level-l prefix; the window prefixes w(a) = lcp(a, a + leaf) of a
// block's tile and the `leaf` positions before it are formed once in shared
// memory.  (Each segment's particles are a contiguous sorted run with a tree
// of its own.)
constexpr int kLevelTile = 256;  // = kBlock
__global__ void __launch_bounds__(kLevelTile)
k_lcp_levels(SegView sv, const uint64_t *keys, int leaf, int8_t *lp, int8_t *lv,
             int32_t *ncount) {
  pdl_wait();
  __shared__ int8_t w[kLevelTile + 32];  // leaf <= 32
  const int64_t n = sv.n;
  for (int64_t t0 = (int64_t)blockIdx.x * kLevelTile; t0 < n;
       t0 += (int64_t)gridDim.x * kLevelTile) {
    __syncthreads();
    for (int j = threadIdx.x; j < kLevelTile + leaf; j += kLevelTile) {
      const int64_t a = t0 - leaf + j;
      w[j] = (a >= 0 && a + leaf < n) ? (int8_t)lcp_levels(keys[a], keys[a + leaf]) : (int8_t)-1;
    }
    __syncthreads();
    const int64_t i = t0 + threadIdx.x;
    if (i < n) {
      const int d = seg_at(sv, i);
      const int64_t s0 = seg_lo(sv, d), s1 = seg_hi(sv, d);
      const uint64_t k = keys[i];
      const int p = i == s0 ? -1 : lcp_levels(keys[i - 1], k);
      lp[i] = (int8_t)p;
      int D = -1;
      const int64_t a0 = i - leaf > s0 ? i - leaf : s0;
      const int64_t a1 = i < s1 - 1 - leaf ? i : s1 - 1 - leaf;
      for (int64_t a = a0; a <= a1; ++a) D = max(D, (int)w[a - (t0 - leaf)]);
      const int L = min(D + 1, P3T_BITS);
      lv[i] = (int8_t)L;
      ncount[i] = max(0, L - p);
    }
  }
}

// The nodes a particle starts (levels lp + 1 .. lv, deepest last in preorder):
// their first particle and level, and the identity order for the level sort;
// the member counts come from k_node_counts
__global__ void k_nodes_pre(SegView sv, const int8_t *lp, const int8_t *lv,
                            const int64_t *nstart, int64_t *cnt, int64_t node_cap,
                            int32_t *pre_first, int32_t *pre_level, uint64_t *lvl_keys,
                            int32_t *bfs2pre, DevStatus *st) {
  pdl_wait();
  // the node count (cnt[1], from the scan) clamped to the capacity in cnt[3]:
  // the later kernels index with the clamped value
  const int64_t nn = cnt[1];
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (nn > node_cap) dev_fail(st, P3T_ERR_CAPACITY, 10, nn);
    cnt[3] = nn < node_cap ? nn : node_cap;
  }
  if (nn > node_cap || st->code != 0) return;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < sv.n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int l0 = (int)lp[i] + 1, L = (int)lv[i];
    for (int l = l0; l <= L; ++l) {
      const int64_t id = nstart[i] + (l - l0);
      pre_first[id] = (int32_t)i;
      pre_level[id] = l;
      lvl_keys[id] = (uint64_t)l;
      bfs2pre[id] = (int32_t)id;
    }
  }
}

// Members of each node: the node's cell (level l, first particle i) ends at
// the first sorted key at or above kend = (prefix of key i at level l, plus
// one) shifted back, or at the segment's end -- a lower bound found with 8
// independent probes a round: galloping from i (probe steps 1..8, then 8x
// larger each round), then narrowing the last interval ninefold a round.  A
// node's search is its own thread's: the longest chain (the root) is about a
// dozen rounds, not one search per level in a row.
__global__ void k_node_counts(SegView sv, const uint64_t *keys, const int64_t *d_nnode,
                              int64_t node_cap, const int32_t *pre_first,
                              const int32_t *pre_level, int32_t *pre_count, DevStatus *st) {
  pdl_wait();
  if (*d_nnode > node_cap || st->code != 0) return;
  const int64_t nn = *d_nnode;
  for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < nn;
       b += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = pre_first[b];
    const int l = pre_level[b];
    const int64_t s1 = seg_hi(sv, seg_at(sv, i));
    int64_t end = s1;
    if (l > 0) {
      const int sh = 3 * (P3T_BITS - l);
      const uint64_t kend = ((keys[i] >> sh) + 1) << sh;
      // invariant: keys[lo] < kend; the answer lies in (lo, hi]
      int64_t lo = i, hi = s1, step = 1;
      for (;;) {  // gallop
        uint64_t kp[8];
#pragma unroll
        for (int m = 0; m < 8; ++m) {
          const int64_t q = lo + (m + 1) * step;
          kp[m] = q < s1 ? __ldg(&keys[q]) : ~0ull;
        }
        int f = 8;
#pragma unroll
        for (int m = 7; m >= 0; --m)
          if (kp[m] >= kend) f = m;
        if (f < 8) {
          hi = lo + (f + 1) * step < s1 ? lo + (f + 1) * step : s1;
          lo += f * step;
          break;
        }
        lo += 8 * step;
        step *= 8;
      }
      while (hi - lo > 1) {  // narrow (lo, hi]
        const int64_t w = (hi - lo + 8) / 9;
        uint64_t kp[8];
#pragma unroll
        for (int m = 0; m < 8; ++m) {
          const int64_t q = lo + (m + 1) * w;
          kp[m] = q < hi ? __ldg(&keys[q]) : ~0ull;
        }
        int f = 8;
#pragma unroll
        for (int m = 7; m >= 0; --m)
          if (kp[m] >= kend) f = m;
        const int64_t nhi = lo + (f + 1) * w;
        if (nhi < hi) hi = nhi;
        lo += f * w;
      }
      end = hi;
    }
    pre_count[b] = (int32_t)(end - i);
  }
}

__global__ void k_pre2bfs(const int64_t *d_nnode, int64_t node_cap,
                          const int32_t *bfs2pre, int32_t *pre2bfs) {
  pdl_wait();
  const int64_t nn = min(*d_nnode, node_cap);
  for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < nn;
       b += (int64_t)gridDim.x * blockDim.x)
    pre2bfs[bfs2pre[b]] = (int32_t)b;
}

__global__ void k_nodes_bfs(const int64_t *d_nnode, int64_t node_cap,
                            const int32_t *bfs2pre, const int32_t *pre2bfs,
                            const int32_t *pre_first, const int32_t *pre_count,
                            const int32_t *pre_level, const int8_t *lp,
                            const int8_t *lv, const int64_t *nstart,
                            const int32_t *sq, TreeNode *node,
                            int gs, int32_t *flags, int32_t *node_done, DevStatus *st) {
  pdl_wait();
  const int64_t nn = min(*d_nnode, node_cap);
  for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < nn;
       b += (int64_t)gridDim.x * blockDim.x) {
    const int32_t pre = bfs2pre[b];
    const int32_t first = pre_first[pre], count = pre_count[pre], l = pre_level[pre];
    TreeNode nd;
    nd.level = l;
    nd.first = first;
    nd.count = count;
    const int sh = P3T_BITS - l;
    for (int a = 0; a < 3; ++a) nd.c2[a] = (2 * (sq[3 * first + a] >> sh) + 1) << sh;
    const bool internal = l < (int)lv[first];
    if (internal && pre + 1 < nn) {
      nd.child0 = pre2bfs[pre + 1];
      const int64_t e = (int64_t)first + count;
      int k = 0;
      int64_t c = pre + 1;
      for (;;) {
        ++k;
        const int64_t cend = (int64_t)pre_first[c] + pre_count[c];
        if (cend >= e) break;
        c = nstart[cend] + (l + 1) - ((int)lp[cend] + 1);
        if (k >= 8 || c <= pre || c >= nn) {  // cannot happen in a consistent tree
          dev_fail(st, P3T_ERR_INVALID, 11, 0);
          break;
        }
      }
      nd.nchild = k;
      node_done[b] = k;
    } else {
      nd.child0 = -1;
      nd.nchild = 0;
      node_done[b] = 0;
    }
    // bit 0: a leaf; bit 1: a target group without a parent (a root; the
    // parents flag the others)
    const bool small = count <= gs || nd.nchild == 0;
    flags[pre] = (internal ? 0 : 1) | (l == 0 && small ? 2 : 0);
    // geometry (qlo, qhi, R) is filled bottom-up by k_moments and the parent
    // links by k_parents
    TreeNode *o = &node[b];
    o->level = nd.level; o->first = nd.first; o->count = nd.count;
    o->c2[0] = nd.c2[0]; o->c2[1] = nd.c2[1]; o->c2[2] = nd.c2[2];
    o->child0 = nd.child0; o->nchild = nd.nchild;
    o->parent = -1;  // set for children by k_parents
  }
}

// parent links, and the target-group flag (bit 1 of the preorder flags) of
// every child: a node holding <= gs particles (or a leaf) whose parent holds
// more
__global__ void k_parents(const int64_t *d_nnode, int64_t node_cap, TreeNode *node,
                          const int32_t *bfs2pre, int gs, int32_t *flags) {
  pdl_wait();
  const int64_t nn = min(*d_nnode, node_cap);
  for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < nn;
       b += (int64_t)gridDim.x * blockDim.x) {
    const int32_t c0 = node[b].child0, nc = node[b].nchild;
    if (nc > 0 && (c0 <= b || (int64_t)c0 + nc > nn)) continue;  // inconsistent: skip
    const bool big = node[b].count > gs;
    for (int k = 0; k < nc; ++k) {
      TreeNode &cn = node[c0 + k];
      cn.parent = (int32_t)b;
      if (big && (cn.count <= gs || cn.nchild == 0)) flags[bfs2pre[c0 + k]] |= 2;
    }
  }
}

// the leaf list and the target-group list in key order from the flag-pair
// scan (leaf positions in bits 0-30, group positions from bit 31), and both
// counts from its total
__global__ void k_lists(const int64_t *d_nnode, int64_t node_cap, const int32_t *flags,
                        const int64_t *pos, const int32_t *pre2bfs, const int64_t *d_total,
                        int32_t *leaf_list, int32_t *group_list, int64_t *d_nleaf,
                        int64_t *d_ngroup) {
  pdl_wait();
  const int64_t nn = min(*d_nnode, node_cap);
  constexpr int64_t kLow = (1ll << 31) - 1;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const int64_t t = *d_total;
    *d_nleaf = t & kLow;
    *d_ngroup = t >> 31;
  }
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < nn;
       p += (int64_t)gridDim.x * blockDim.x) {
    const int32_t f = flags[p];
    if (!f) continue;
    const int64_t q = pos[p];
    const int32_t b = pre2bfs[p];
    if (f & 1) leaf_list[q & kLow] = b;
    if (f & 2) group_list[q >> 31] = b;
  }
}

__device__ __forceinline__ void finish_node(TreeNode *nd, Mom64 *m64, Mom32 *m32,
                                            double rsmax, double u, int64_t b,
                                            const Mom64 &mm) {
  double rq = ceil(rsmax / u) + 1.0;
  nd->R = rq < 8388608.0 ? (int32_t)rq : 8388608;
  m64[b] = mm;
  Mom32 f;
  const float hx = (float)mm.cx, hy = (float)mm.cy, hz = (float)mm.cz;
  const float mh = (float)mm.M;
  f.hi = make_float4(hx, hy, hz, mh);
  f.lo = make_float4((float)(mm.cx - (double)hx), (float)(mm.cy - (double)hy),
                     (float)(mm.cz - (double)hz), (float)(mm.M - (double)mh));
  f.q0 = make_float4((float)mm.qxx, (float)mm.qyy, (float)mm.qzz, (float)mm.qxy);
  f.q1 = make_float4((float)mm.qxz, (float)mm.qyz, 0.f, 0.f);
  m32[b] = f;
}

// Moments, one thread per node, level by level with no atomics: first every
// leaf from its members, then the internal nodes of one level per launch,
// deepest level first, from their (finished) children.  (A warp instruction
// of FP64 occupies a sub-partition's pipe for ~64 cycles however few of its
// lanes are active, so every lane carries a node of its own.)  A leaf's
// members are summed about a reference point r (its first member): M, D =
// sum m d, S_ab = sum m d_a d_b with d = x - r; then com = r + D / M and the
// traceless quadrupole about the com, Q_ab = 3 C_ab - delta_ab tr C with C_ab
// = S_ab - M e_a e_b, e = D / M (the definition sum m (3 d'_a d'_b - d'^2
// delta_ab), d' = x - com, expanded).  An internal node sums its children with
// the parallel-axis shift of Q.
__global__ void k_moments_leaf(
    const int64_t *d_nleaf, const int32_t *leaf_list, TreeNode *node, Mom64 *m64, Mom32 *m32,
    double *nrs, const double *sx, const double *sy, const double *sz, const double *sm,
    const double *srs, const int32_t *sq, const double *box, SegView sv) {
  pdl_wait();
  const int64_t nleaf = *d_nleaf;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nleaf;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = leaf_list[t];
    TreeNode *nd = &node[b];
    const int32_t f = nd->first, c = nd->count;
    const double u = ldexp(box[5 * seg_at(sv, f) + 3], -P3T_BITS);
    const double rx = sx[f], ry = sy[f], rz = sz[f];
    double M = 0.0, D[3] = {0, 0, 0}, S[6] = {0, 0, 0, 0, 0, 0}, rs = 0.0;
    int32_t lo[3] = {P3T_QMAX, P3T_QMAX, P3T_QMAX}, hi[3] = {-1, -1, -1};
    for (int32_t i = f; i < f + c; ++i) {
      const double m = sm[i], dx = sx[i] - rx, dy = sy[i] - ry, dz = sz[i] - rz;
      const double mx = m * dx, my = m * dy, mz = m * dz;
      M += m; D[0] += mx; D[1] += my; D[2] += mz;
      S[0] = __fma_rn(mx, dx, S[0]); S[1] = __fma_rn(my, dy, S[1]); S[2] = __fma_rn(mz, dz, S[2]);
      S[3] = __fma_rn(mx, dy, S[3]); S[4] = __fma_rn(mx, dz, S[4]); S[5] = __fma_rn(my, dz, S[5]);
      rs = fmax(rs, srs[i]);
#pragma unroll
      for (int a = 0; a < 3; ++a) { lo[a] = min(lo[a], sq[3 * i + a]); hi[a] = max(hi[a], sq[3 * i + a]); }
    }
    Mom64 mm = {};
    const double iM = 1.0 / M;
    const double e[3] = {D[0] * iM, D[1] * iM, D[2] * iM};
    mm.M = M; mm.cx = rx + e[0]; mm.cy = ry + e[1]; mm.cz = rz + e[2];
    const double Cxx = S[0] - M * e[0] * e[0], Cyy = S[1] - M * e[1] * e[1],
                 Czz = S[2] - M * e[2] * e[2];
    const double tr = Cxx + Cyy + Czz;
    mm.qxx = 3.0 * Cxx - tr; mm.qyy = 3.0 * Cyy - tr; mm.qzz = 3.0 * Czz - tr;
    mm.qxy = 3.0 * (S[3] - M * e[0] * e[1]);
    mm.qxz = 3.0 * (S[4] - M * e[0] * e[2]);
    mm.qyz = 3.0 * (S[5] - M * e[1] * e[2]);
    for (int a = 0; a < 3; ++a) { nd->qlo[a] = lo[a]; nd->qhi[a] = hi[a]; }
    nrs[b] = rs;
    finish_node(nd, m64, m32, rs, u, b, mm);
  }
}

// Mixed path: the same moments with no FP64 instruction, written straight to
// the Mom32 record the mixed walk reads (the FP64 record is not formed).
// Positions come as float-float pairs (spA hi, spB lo) and masses as spA.w +
// the lo array; d = x - r, M and D are float-float (the centre of mass then
// carries ~2^-44 of the coordinates, the float-float redo's need), S and the
// quadrupole are FP32 (the walk reads Q in FP32).  The search reach is the
// largest r_search as a bit pattern (non-negative doubles order like their
// bits), and R = ceil(rs / u) + 1 comes from integer operations (reach_cells:
// the value of the FP64 expression the FP64 path evaluates).
__device__ __forceinline__ int64_t max_bits(int64_t a, double v) {
  const int64_t b = __double_as_longlong(v);
  return b > a ? b : a;
}

__device__ __forceinline__ int32_t leaf_moments32(
    int64_t b, TreeNode *node, Mom32 *m32, double *nrs, const float4 *spA, const float4 *spB,
    const float *sml, const double *srs, const int32_t *sq, const double *box,
    const SegView &sv) {
  {
    TreeNode *nd = &node[b];
    const int4 r2 = reinterpret_cast<const int4 *>(nd)[2], r3 = reinterpret_cast<const int4 *>(nd)[3];
    const int32_t f = r3.z, c = r3.w;
    const double L = box[5 * seg_at(sv, f) + 3];
    const float4 A0 = spA[f], B0 = spB[f];
    FF M{0.f, 0.f}, D[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
    float S[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    int64_t rsb = 0;
    int32_t lo[3] = {P3T_QMAX, P3T_QMAX, P3T_QMAX}, hi[3] = {-1, -1, -1};
    for (int32_t i = f; i < f + c; ++i) {
      const float4 A = spA[i], B = spB[i];
      const FF dx = ff_add({A.x, B.x}, {-A0.x, -B0.x});
      const FF dy = ff_add({A.y, B.y}, {-A0.y, -B0.y});
      const FF dz = ff_add({A.z, B.z}, {-A0.z, -B0.z});
      const FF m = ff_fast(A.w, sml[i]);
      M = ff_add(M, m);
      D[0] = ff_add(D[0], ff_mul(m, dx));
      D[1] = ff_add(D[1], ff_mul(m, dy));
      D[2] = ff_add(D[2], ff_mul(m, dz));
      const float mx = m.h * dx.h, my = m.h * dy.h, mz = m.h * dz.h;
      S[0] = fmaf(mx, dx.h, S[0]); S[1] = fmaf(my, dy.h, S[1]); S[2] = fmaf(mz, dz.h, S[2]);
      S[3] = fmaf(mx, dy.h, S[3]); S[4] = fmaf(mx, dz.h, S[4]); S[5] = fmaf(my, dz.h, S[5]);
      rsb = max_bits(rsb, srs[i]);
#pragma unroll
      for (int a = 0; a < 3; ++a) { lo[a] = min(lo[a], sq[3 * i + a]); hi[a] = max(hi[a], sq[3 * i + a]); }
    }
    const FF e[3] = {ff_div(D[0], M), ff_div(D[1], M), ff_div(D[2], M)};
    const FF cx = ff_add({A0.x, B0.x}, e[0]), cy = ff_add({A0.y, B0.y}, e[1]),
             cz = ff_add({A0.z, B0.z}, e[2]);
    const float Mh = M.h, ex = e[0].h, ey = e[1].h, ez = e[2].h;
    const float Cxx = S[0] - Mh * ex * ex, Cyy = S[1] - Mh * ey * ey, Czz = S[2] - Mh * ez * ez;
    const float tr = Cxx + Cyy + Czz;
    Mom32 o;
    o.hi = make_float4(cx.h, cy.h, cz.h, M.h);
    o.lo = make_float4(cx.l, cy.l, cz.l, M.l);
    o.q0 = make_float4(3.f * Cxx - tr, 3.f * Cyy - tr, 3.f * Czz - tr, 3.f * (S[3] - Mh * ex * ey));
    o.q1 = make_float4(3.f * (S[4] - Mh * ex * ez), 3.f * (S[5] - Mh * ey * ez), 0.f, 0.f);
    for (int a = 0; a < 3; ++a) { nd->qlo[a] = lo[a]; nd->qhi[a] = hi[a]; }
    const double rs = __longlong_as_double(rsb);
    nrs[b] = rs;
    nd->R = reach_cells(rs, L, cell_scale(L));
    m32[b] = o;
    return r2.w;
  }
}

// One internal node of the mixed path from its children's Mom32 records, by
// one thread, the eight child slots added in the fixed pairwise tree ((s0 +
// s4) + (s2 + s6)) + ((s1 + s5) + (s3 + s7)) (zero past the last child).  The
// children were written by other threads of the same launch: read through L2.
template <int NQ, class T, class F, class A>
__device__ __forceinline__ void tree8_acc(int nch, F slot, A add, T (&r)[NQ]) {
  // the children fill slots 0 .. nch - 1; an empty slot is zero and adding
  // zero to a (normalised) sum returns it, so empty slots and their additions
  // are skipped: the same values as the full tree
  T a[NQ], b[NQ], c[NQ], d[NQ];
  slot(0, a);
  if (nch > 4) {
    slot(4, b);
#pragma unroll
    for (int q = 0; q < NQ; ++q) a[q] = add(a[q], b[q]);
  }
  if (nch > 2) {
    slot(2, b);
    if (nch > 6) {
      slot(6, c);
#pragma unroll
      for (int q = 0; q < NQ; ++q) b[q] = add(b[q], c[q]);
    }
#pragma unroll
    for (int q = 0; q < NQ; ++q) a[q] = add(a[q], b[q]);
  }
  if (nch > 1) {
    slot(1, b);
    if (nch > 5) {
      slot(5, c);
#pragma unroll
      for (int q = 0; q < NQ; ++q) b[q] = add(b[q], c[q]);
    }
    if (nch > 3) {
      slot(3, c);
      if (nch > 7) {
        slot(7, d);
#pragma unroll
        for (int q = 0; q < NQ; ++q) c[q] = add(c[q], d[q]);
      }
#pragma unroll
      for (int q = 0; q < NQ; ++q) b[q] = add(b[q], c[q]);
    }
#pragma unroll
    for (int q = 0; q < NQ; ++q) r[q] = add(a[q], b[q]);
  } else {
#pragma unroll
    for (int q = 0; q < NQ; ++q) r[q] = a[q];
  }
}

__device__ __forceinline__ Mom32 ldcg_mom32(const Mom32 *m) {
  Mom32 o;
  o.hi = __ldcg(&m->hi); o.lo = __ldcg(&m->lo); o.q0 = __ldcg(&m->q0); o.q1 = __ldcg(&m->q1);
  return o;
}

__device__ int32_t node_moments32(int64_t b, TreeNode *node, Mom32 *m32, double *nrs,
                                  const double *box, const SegView &sv) {
  TreeNode *pn = &node[b];
  const int4 r2 = __ldcg(reinterpret_cast<const int4 *>(pn) + 2),
             r3 = __ldcg(reinterpret_cast<const int4 *>(pn) + 3);
  const int32_t c0 = r3.x, nch = r3.y;
  if (nch < 1 || nch > 8) return r2.w;  // only a node with children is completed
  int64_t rsb = 0;
  int32_t plo[3] = {P3T_QMAX, P3T_QMAX, P3T_QMAX}, phi[3] = {-1, -1, -1};
  for (int k = 0; k < nch; ++k) {
    rsb = max_bits(rsb, __ldcg(&nrs[c0 + k]));
    const TreeNode *cn = &node[c0 + k];
    for (int a = 0; a < 3; ++a) {
      plo[a] = min(plo[a], __ldcg(&cn->qlo[a]));
      phi[a] = max(phi[a], __ldcg(&cn->qhi[a]));
    }
  }
  FF P[4];
  tree8_acc<4>(nch, [&](int k, FF (&t)[4]) {
    const float4 hi = __ldcg(&m32[c0 + k].hi), lo = __ldcg(&m32[c0 + k].lo);
    const FF M = ff_fast(hi.w, lo.w);
    t[0] = M;
    t[1] = ff_mul(M, ff_fast(hi.x, lo.x));
    t[2] = ff_mul(M, ff_fast(hi.y, lo.y));
    t[3] = ff_mul(M, ff_fast(hi.z, lo.z));
  }, [](FF x, FF y) { return ff_add(x, y); }, P);
  const FF pc[3] = {ff_div(P[1], P[0]), ff_div(P[2], P[0]), ff_div(P[3], P[0])};
  float Q[6];
  tree8_acc<6>(nch, [&](int k, float (&t)[6]) {
    {
      const Mom32 cm = ldcg_mom32(&m32[c0 + k]);
      const float M = cm.hi.w;
      const float dx = ff_add(ff_fast(cm.hi.x, cm.lo.x), ff_neg(pc[0])).h;
      const float dy = ff_add(ff_fast(cm.hi.y, cm.lo.y), ff_neg(pc[1])).h;
      const float dz = ff_add(ff_fast(cm.hi.z, cm.lo.z), ff_neg(pc[2])).h;
      const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
      const float tx = 3.f * dx, ty = 3.f * dy;
      t[0] = fmaf(M, fmaf(tx, dx, -d2), cm.q0.x);
      t[1] = fmaf(M, fmaf(ty, dy, -d2), cm.q0.y);
      t[2] = fmaf(M, fmaf(3.f * dz, dz, -d2), cm.q0.z);
      t[3] = fmaf(M, tx * dy, cm.q0.w);
      t[4] = fmaf(M, tx * dz, cm.q1.x);
      t[5] = fmaf(M, ty * dz, cm.q1.y);
    }
  }, [](float x, float y) { return x + y; }, Q);
  Mom32 o;
  o.hi = make_float4(pc[0].h, pc[1].h, pc[2].h, P[0].h);
  o.lo = make_float4(pc[0].l, pc[1].l, pc[2].l, P[0].l);
  o.q0 = make_float4(Q[0], Q[1], Q[2], Q[3]);
  o.q1 = make_float4(Q[4], Q[5], 0.f, 0.f);
  for (int a = 0; a < 3; ++a) { pn->qlo[a] = plo[a]; pn->qhi[a] = phi[a]; }
  const double rs = __longlong_as_double(rsb);
  nrs[b] = rs;
  const double L = box[5 * seg_at(sv, r3.z) + 3];
  pn->R = reach_cells(rs, L, cell_scale(L));
  m32[b] = o;
  return r2.w;
}

// All moments of the mixed path in one launch, bottom-up: a thread per leaf
// computes the leaf, then counts itself off at its parent (node_done, preset
// to the number of children by k_nodes_bfs); the child that brings the count
// to zero computes the parent from all its children and climbs on (each
// node's record gives its parent in the same load as its children).  Nothing waits, and a node's result does
// not depend on which child arrives last.  (In FP32 and float-float a node
// costs a few thousand cycles of latency, so the climb's serial tail at the
// top levels is short; the FP64 path keeps its level launches.)
__global__ void k_moments_up32(
    const int64_t *d_nleaf, const int32_t *leaf_list, TreeNode *node, Mom32 *m32, double *nrs,
    const float4 *spA, const float4 *spB, const float *sml, const double *srs,
    const int32_t *sq, const double *box, SegView sv, int32_t *node_done) {
  pdl_wait();
  const int64_t nleaf = *d_nleaf;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nleaf;
       t += (int64_t)gridDim.x * blockDim.x) {
    int32_t p = leaf_moments32(leaf_list[t], node, m32, nrs, spA, spB, sml, srs, sq, box, sv);
    while (p >= 0) {
      __threadfence();  // this node's record before the count
      if (atomicSub(&node_done[p], 1) != 1) break;  // siblings still to come
      __threadfence();  // the siblings' records after their counts
      p = node_moments32(p, node, m32, nrs, box, sv);
    }
  }
}

// first breadth-first id at level >= l (levels ascend in breadth-first order)
__device__ __forceinline__ int64_t level_begin(const TreeNode *node, int64_t nn, int l) {
  int64_t lo = 0, hi = nn;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (node[mid].level < l) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// first breadth-first id of every level 0..21 and the node count (levels
// ascend in breadth-first order): one thread per level
__global__ void k_level_offsets(const int64_t *d_nnode, int64_t node_cap, const TreeNode *node,
                                int64_t *lvl_start) {
  pdl_wait();
  const int64_t nn = min(*d_nnode, node_cap);
  const int l = threadIdx.x;
  if (l <= P3T_BITS + 1) lvl_start[l] = l == P3T_BITS + 1 ? nn : level_begin(node, nn, l);
}

// The internal nodes of one level (levels 0..20), one thread per node, from
// their finished children; launched level by level, deepest first.  (A grid
// barrier between levels in one cooperative launch was measured slower than
// the launches: its waits dominated.)
// Internal nodes of one level from their finished children.  Every level is
// small enough that its time is the latency of one warp's FP64 instruction
// stream (one FP64 warp instruction per 64 cycles of a sub-partition), so a
// node's children are spread over L lanes (L = 8, 4, 2 or 1, the largest that
// keeps the level within about one warp per sub-partition), lane sub holding
// the child slots sub, sub + L, ... of the node's eight.  Each child's terms
// are rounded on their own and the eight slots (zero where there is no child)
// are added in one fixed pairwise tree, slots s and s + 4, then s + 2, then
// s + 1: in registers while the stride is a multiple of L, by shuffles below
// it.  The sums are therefore the same bits for every L, so a node's moments
// do not depend on how many nodes share its level (a tree built alone or
// beside other systems' trees).  The loop runs in warp-uniform chunks so that
// every lane reaches every shuffle; groups past the level's end or at leaves
// contribute nothing.
__device__ __forceinline__ double shfl_down_group(double v, int o) {
  return __shfl_xor_sync(0xffffffffu, v, o);
}

// the fixed pairwise tree over slots: J = 8 / L slots in this lane's
// registers, then the shuffles between the L lanes of the group
template <int L, int NQ>
__device__ __forceinline__ void slot_tree(double (&v)[8 / L][NQ]) {
#pragma unroll
  for (int S = 4; S >= L; S >>= 1)
#pragma unroll
    for (int j = 0; j < S / L; ++j)
#pragma unroll
      for (int q = 0; q < NQ; ++q) v[j][q] += v[j + S / L][q];
#pragma unroll
  for (int o = L >> 1; o > 0; o >>= 1)
#pragma unroll
    for (int q = 0; q < NQ; ++q) v[0][q] += shfl_down_group(v[0][q], o);
}

template <int L>
__device__ void moments_level_L(int64_t b0, int64_t nn, TreeNode *node, Mom64 *m64, Mom32 *m32,
                                double *nrs, const double *box, const SegView &sv) {
  constexpr int J = 8 / L;
  const int lane = threadIdx.x & 31, sub = lane & (L - 1);
  const int per_warp = 32 / L;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t wb = warp * per_warp; wb < nn; wb += nwarps * per_warp) {
    const int64_t gi = wb + lane / L;
    const bool valid = gi < nn;
    const int64_t b = b0 + (valid ? gi : 0);
    TreeNode *pn = &node[b];
    const int32_t c0 = valid ? pn->child0 : 0, nch = valid ? pn->nchild : 0;
    double prs = 0.0;
    int32_t plo[3] = {P3T_QMAX, P3T_QMAX, P3T_QMAX}, phi[3] = {-1, -1, -1};
    double t[J][4];  // M, M cx, M cy, M cz
#pragma unroll
    for (int j = 0; j < J; ++j) {
      const int k = sub + j * L;
      t[j][0] = t[j][1] = t[j][2] = t[j][3] = 0.0;
      if (k < nch) {
        const Mom64 &cm = m64[c0 + k];
        t[j][0] = cm.M;
        t[j][1] = cm.M * cm.cx;
        t[j][2] = cm.M * cm.cy;
        t[j][3] = cm.M * cm.cz;
        prs = fmax(prs, nrs[c0 + k]);
        const TreeNode &cn = node[c0 + k];
        for (int a = 0; a < 3; ++a) { plo[a] = min(plo[a], cn.qlo[a]); phi[a] = max(phi[a], cn.qhi[a]); }
      }
    }
    slot_tree<L, 4>(t);
    for (int o = L >> 1; o > 0; o >>= 1) {
      for (int a = 0; a < 3; ++a) {
        plo[a] = min(plo[a], __shfl_xor_sync(0xffffffffu, plo[a], o));
        phi[a] = max(phi[a], __shfl_xor_sync(0xffffffffu, phi[a], o));
      }
      prs = fmax(prs, shfl_down_group(prs, o));
    }
    Mom64 pm = {};
    if (nch > 0) {
      const double iM = 1.0 / t[0][0];
      pm.M = t[0][0]; pm.cx = t[0][1] * iM; pm.cy = t[0][2] * iM; pm.cz = t[0][3] * iM;
    }
    double Q[J][6];  // xx, yy, zz, xy, xz, yz
#pragma unroll
    for (int j = 0; j < J; ++j) {
      const int k = sub + j * L;
      for (int q = 0; q < 6; ++q) Q[j][q] = 0.0;
      if (k < nch) {
        const Mom64 &cm = m64[c0 + k];
        const double dx = cm.cx - pm.cx, dy = cm.cy - pm.cy, dz = cm.cz - pm.cz;
        const double d2 = __fma_rn(dx, dx, __fma_rn(dy, dy, dz * dz));
        const double tx = 3.0 * dx, ty = 3.0 * dy;
        Q[j][0] = __fma_rn(cm.M, __fma_rn(tx, dx, -d2), cm.qxx);
        Q[j][1] = __fma_rn(cm.M, __fma_rn(ty, dy, -d2), cm.qyy);
        Q[j][2] = __fma_rn(cm.M, __fma_rn(3.0 * dz, dz, -d2), cm.qzz);
        Q[j][3] = __fma_rn(cm.M, tx * dy, cm.qxy);
        Q[j][4] = __fma_rn(cm.M, tx * dz, cm.qxz);
        Q[j][5] = __fma_rn(cm.M, ty * dz, cm.qyz);
      }
    }
    slot_tree<L, 6>(Q);
    if (valid && nch > 0 && sub == 0) {
      pm.qxx = Q[0][0]; pm.qyy = Q[0][1]; pm.qzz = Q[0][2];
      pm.qxy = Q[0][3]; pm.qxz = Q[0][4]; pm.qyz = Q[0][5];
      for (int a = 0; a < 3; ++a) { pn->qlo[a] = plo[a]; pn->qhi[a] = phi[a]; }
      nrs[b] = prs;
      finish_node(pn, m64, m32, prs, ldexp(box[5 * seg_at(sv, pn->first) + 3], -P3T_BITS), b,
                  pm);
    }
  }
}

__device__ void moments_level(int level, const int64_t *lvl_start, TreeNode *node, Mom64 *m64,
                              Mom32 *m32, double *nrs, const double *box, const SegView &sv,
                              int64_t warp_target) {
  const int64_t b0 = lvl_start[level], b1 = lvl_start[level + 1];
  const int64_t nn = b1 - b0;
  if (nn <= 0) return;
  int L = 8;
  while (L > 1 && nn * L > 32 * warp_target) L >>= 1;
  switch (L) {
    case 8: moments_level_L<8>(b0, nn, node, m64, m32, nrs, box, sv); break;
    case 4: moments_level_L<4>(b0, nn, node, m64, m32, nrs, box, sv); break;
    case 2: moments_level_L<2>(b0, nn, node, m64, m32, nrs, box, sv); break;
    default: moments_level_L<1>(b0, nn, node, m64, m32, nrs, box, sv); break;
  }
}

// levels kDeepLevel and deeper share one single-block launch
constexpr int kDeepLevel = 12;


// levels level_hi down to level_lo; several levels only with a single block
// (a block barrier between levels)
__global__ void k_moments_level(int level_hi, int level_lo, const int64_t *lvl_start,
                                TreeNode *node, Mom64 *m64, Mom32 *m32, double *nrs,
                                const double *box, SegView sv, int64_t warp_target) {
  pdl_wait();
  for (int l = level_hi; l >= level_lo; --l) {
    moments_level(l, lvl_start, node, m64, m32, nrs, box, sv, warp_target);
    if (l > level_lo) {
      __threadfence_block();
      __syncthreads();
    }
  }
}

__global__ void k_tree_stats(const int64_t *d_nnode, int64_t node_cap,
                             const TreeNode *node, int64_t *stats) {
  pdl_wait();
  const int64_t nn = min(*d_nnode, node_cap);
  unsigned long long depth = 0, maxleaf = 0, nleaf = 0;
  for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < nn;
       b += (int64_t)gridDim.x * blockDim.x) {
    depth = max(depth, (unsigned long long)node[b].level);
    if (node[b].nchild == 0) { ++nleaf; maxleaf = max(maxleaf, (unsigned long long)node[b].count); }
  }
  for (int o = 16; o > 0; o >>= 1) {
    depth = max(depth, __shfl_xor_sync(0xffffffffu, depth, o));
    maxleaf = max(maxleaf, __shfl_xor_sync(0xffffffffu, maxleaf, o));
    nleaf += __shfl_xor_sync(0xffffffffu, nleaf, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(reinterpret_cast<unsigned long long *>(&stats[2]), depth);
    atomicMax(reinterpret_cast<unsigned long long *>(&stats[3]), maxleaf);
    atomicAdd(reinterpret_cast<unsigned long long *>(&stats[1]), nleaf);
  }
}

}  // namespace

// counters layout (int64): [0] n, [1] nodes, [2] leaves, [3] nodes clamped to
// the capacity, [4..7] tree stats, [8] candidates, [9] candidates clamped,
// [10] neighbour entries, [11] cluster members, [12] walk group cursor
// radial bins of a system of n particles (Sec. 2.1.3 reading C3)
static int cut_bins(int vran_bins, int64_t n) {
  int nb = vran_bins;
  if (nb <= 0) { int64_t t = n / 1000; nb = (int)(t < 1 ? 1 : (t > 1024 ? 1024 : t)); }
  return nb;
}

int p3t_run_cutoffs(p3t_ctx *c, p3t_particles *p, cudaStream_t s) {
  const int64_t n = p->n;
  if (n == 0) return P3T_OK;
  const SegView sv{c->seg_off, (int)c->nseg, n};
  int64_t nbt = 0;  // bins of all segments
  if (c->nseg == 1) {
    nbt = cut_bins(c->prm.vran_bins, n);
  } else {
    for (int64_t d = 0; d < c->nseg; ++d)
      nbt += cut_bins(c->prm.vran_bins, c->seg_off_h[d + 1] - c->seg_off_h[d]);
  }
  if (nbt > kMaxBins) return P3T_ERR_INVALID;
  const int nb = (int)nbt;
  double *bsum = c->epart;  // reuse: >= 4096 doubles
  unsigned long long *bcnt = reinterpret_cast<unsigned long long *>(c->epart + 4096);
  const int64_t g = p3t_grid(n, kBlock, (int64_t)c->num_sms * P3T_NSM_BLOCKS);
  pdl_launch(k_cut_init, dim3(4), dim3(kBlock), 0, s, c->box_bits, (int)c->nseg, bsum, bcnt, nb);
  const int rsl = c->nseg == 1 ? (int)g : (int)((g + c->nseg - 1) / c->nseg);
  pdl_launch(k_cut_range, dim3((unsigned)(rsl * c->nseg)), dim3(kBlock), 0, s, sv, rsl, p->x, p->y, c->box_bits);
  if (c->nseg > 1)
    pdl_launch(k_cut_segbins, dim3(1), dim3(1024), 0, s, sv, c->prm.vran_bins, c->box_bits, c->seg_nb,
                                     c->seg_base, c->seg_l);
  const double mu = c->prm.G * c->prm.m_star;
  // per-bin sums in a fixed order (particles grouped by bin with the stable
  // radix sort, then one warp per bin): the radii do not depend on timing
  double *u2 = c->hw;
  int64_t *boff = c->pos;
  int64_t *d_n = &c->counters[18];
  pdl_launch(k_set_i64, dim3(1), dim3(1), 0, s, d_n, n);
  int32_t *bin = c->flag;  // the bins of k_cut_u2, read by k_cut_final (N int32)
  pdl_launch(k_cut_u2, dim3((unsigned)g), dim3(kBlock), 0, s, sv, p->x, p->y, p->z, p->vx, p->vy, p->vz, mu,
                                          c->box_bits, nb, c->seg_nb, c->seg_base, c->seg_l,
                                          u2, c->keys, c->idx, bin, bcnt);
  int rc = p3t_radix_sort(&c->keys, &c->idx, &c->keys_alt, &c->idx_alt, d_n, c->cap, 0, 16,
                          c->radix_hist, c->radix_hist_cap, s);
  if (rc) return rc;
  pdl_launch(k_cut_offsets, dim3(1), dim3(1024), 0, s, nb, bcnt, boff);
  pdl_launch(k_cut_binsum, dim3((unsigned)p3t_grid((int64_t)nb * 32, kBlock, (int64_t)c->num_sms * 4)), dim3(kBlock), 0, s, nb, boff, c->idx, u2, bsum);
  pdl_launch(k_cut_final, dim3((unsigned)g), dim3(kBlock), 0, s, sv, p->x, p->y, p->z, p->vx, p->vy,
                                             p->vz, p->m, c->prm, c->box_bits, bin, bsum,
                                             p->r_out, p->r_search);
  if (c->prm.cutoff_mode == P3T_CUT_SHARED)
    pdl_launch(k_cut_shared, dim3((unsigned)g), dim3(kBlock), 0, s, sv, c->box_bits, p->r_out, p->r_search);
  // init, range, n, u2, offsets, bin sums, final (+ shared, + segment bins);
  // the sort counts itself
  p3t_note_launches(7 + (c->prm.cutoff_mode == P3T_CUT_SHARED) + (c->nseg > 1));
  return cudaGetLastError() == cudaSuccess ? P3T_OK : P3T_ERR_CUDA;
}

int p3t_run_build_tree(p3t_ctx *c, const p3t_particles *p, cudaStream_t s) {
  const int64_t n = p->n;
  const int leaf = c->prm.leaf_size;
  const int64_t maxb = (int64_t)c->num_sms * P3T_NSM_BLOCKS;
  const int64_t g = p3t_grid(n, kBlock, maxb);
  int64_t *cnt = c->counters;
  int rc;
  const int nseg = (int)c->nseg;
  const SegView sv{c->seg_off, nseg, n};
  // one root cube per segment: a few blocks per SM in all, in slices of the
  // segments
  const int bsl = nseg >= 4 * c->num_sms ? 1 : 4 * c->num_sms / nseg;
  pdl_launch(k_box_init, dim3(1), dim3(256), 0, s, c->box_bits, nseg);
  pdl_launch(k_box, dim3((unsigned)(bsl * nseg)), dim3(kBlock), 0, s, sv, bsl, p->x, p->y, p->z, c->box_bits);
  pdl_launch(k_box_final, dim3(1), dim3(256), 0, s, c->box_bits, c->box, nseg);
  pdl_launch(k_keys, dim3((unsigned)g), dim3(kBlock), 0, s, sv, p->x, p->y, p->z, p->m, p->r_out, p->r_search,
                                        c->box, c->keys, c->idx, c->pack, 0, &cnt[0]);
  rc = p3t_radix_sort(&c->keys, &c->idx, &c->keys_alt, &c->idx_alt, &cnt[0], c->cap,
                      0, 64, c->radix_hist, c->radix_hist_cap, s);
  if (rc) return rc;
  if (nseg > 1) {
    // stable sort by segment (the most significant digit of (segment, key)),
    // then the keys of the new order
    int sbits = 0;
    while ((1 << sbits) < nseg) ++sbits;
    pdl_launch(k_segkey, dim3((unsigned)g), dim3(kBlock), 0, s, sv, c->idx, c->keys);
    rc = p3t_radix_sort(&c->keys, &c->idx, &c->keys_alt, &c->idx_alt, &cnt[0], c->cap,
                        0, sbits, c->radix_hist, c->radix_hist_cap, s);
    if (rc) return rc;
    pdl_launch(k_keys, dim3((unsigned)g), dim3(kBlock), 0, s, sv, p->x, p->y, p->z, p->m, p->r_out, p->r_search,
                                          c->box, c->keys, c->idx, c->pack, 1, nullptr);
    p3t_note_launches(2);
  }
  auto gather = c->prm.precision == P3T_MIXED ? k_gather<true> : k_gather<false>;
  pdl_launch(gather, dim3((unsigned)g), dim3(kBlock), 0, s, n, c->idx, c->keys, c->pack, c->sx, c->sy, c->sz,
                                          c->sm, c->sro, c->srs, c->sq, c->spA, c->spB,
                                          c->srs32, c->sml);
  pdl_launch(k_lcp_levels, dim3((unsigned)p3t_grid(n, kLevelTile, maxb)), dim3(kLevelTile), 0, s, 
      sv, c->keys, leaf, c->lp, c->lv, c->ncount);
  rc = p3t_scan_i32_to_i64(c->ncount, c->nstart, &cnt[0], c->cap, &cnt[1], c->scan_state, c->scan_words, c->status, c->poll_limit, s);
  if (rc) return rc;
  pdl_launch(k_nodes_pre, dim3((unsigned)g), dim3(kBlock), 0, s, sv, c->lp, c->lv, c->nstart, cnt, c->node_cap,
                                             c->pre_first, c->pre_level, c->lvl_keys,
                                             c->bfs2pre, c->status);
  pdl_launch(k_node_counts, dim3((unsigned)p3t_grid(c->node_cap, kBlock, maxb)), dim3(kBlock), 0, s, 
      sv, c->keys, &cnt[1], c->node_cap, c->pre_first, c->pre_level, c->pre_count, c->status);
  rc = p3t_radix_sort(&c->lvl_keys, &c->bfs2pre, &c->lvl_keys_alt, &c->bfs2pre_alt, &cnt[3],
                      c->node_cap, 0, 8, c->radix_hist, c->radix_hist_cap, s);
  if (rc) return rc;
  const int64_t gn = p3t_grid(c->node_cap, kBlock, maxb);
  pdl_launch(k_pre2bfs, dim3((unsigned)gn), dim3(kBlock), 0, s, &cnt[3], c->node_cap, c->bfs2pre, c->pre2bfs);
  pdl_launch(k_nodes_bfs, dim3((unsigned)gn), dim3(kBlock), 0, s, &cnt[3], c->node_cap, c->bfs2pre, c->pre2bfs,
                                              c->pre_first, c->pre_count, c->pre_level,
                                              c->lp, c->lv, c->nstart, c->sq, c->node,
                                              c->prm.group_size, c->node_flag, c->node_done,
                                              c->status);
  pdl_launch(k_parents, dim3((unsigned)gn), dim3(kBlock), 0, s, &cnt[3], c->node_cap, c->node,
             c->bfs2pre, c->prm.group_size, c->node_flag);
  // leaves (bit 0) and target groups (bit 1) counted by one scan
  rc = p3t_scan_flag_pairs(c->node_flag, c->flag_pos, &cnt[3], c->node_cap, &cnt[19],
                           c->scan_state, c->scan_words, c->status, c->poll_limit, s);
  if (rc) return rc;
  pdl_launch(k_lists, dim3((unsigned)gn), dim3(kBlock), 0, s, &cnt[3], c->node_cap, c->node_flag,
             c->flag_pos, c->pre2bfs, &cnt[19], c->leaf_list, c->group_list, &cnt[2], &cnt[15]);
  if (c->prm.precision == P3T_MIXED) {
    pdl_launch(k_moments_up32, dim3((unsigned)p3t_grid(c->node_cap, 128, maxb)), dim3(128), 0, s, 
        &cnt[2], c->leaf_list, c->node, c->mom32, c->nrs, c->spA, c->spB, c->sml, c->srs,
        c->sq, c->box, sv, c->node_done);
    p3t_note_launches(1);
  } else {
    pdl_launch(k_moments_leaf, dim3((unsigned)p3t_grid(c->node_cap, 128, maxb)), dim3(128), 0, s, 
        &cnt[2], c->leaf_list, c->node, c->mom64, c->mom32, c->nrs, c->sx, c->sy, c->sz, c->sm,
        c->srs, c->sq, c->box, sv);
    // internal nodes, level by level, deepest first
    int64_t *lvl_start = c->counters + 32;  // [P3T_BITS + 2]
    pdl_launch(k_level_offsets, dim3(1), dim3(32), 0, s, &cnt[3], c->node_cap, c->node, lvl_start);
    // the deep levels (empty or nearly so in a disk) in one single-block
    // launch, then one launch a level at about one warp per sub-partition
    pdl_launch(k_moments_level, dim3(1), dim3(128), 0, s, P3T_BITS - 1, kDeepLevel, lvl_start, c->node, c->mom64,
                                      c->mom32, c->nrs, c->box, sv, 4);
    const int64_t wt = (int64_t)c->num_sms * 4;
    for (int l = kDeepLevel - 1; l >= 0; --l)
      pdl_launch(k_moments_level, dim3((unsigned)c->num_sms), dim3(128), 0, s, l, l, lvl_start, c->node, c->mom64,
                                                           c->mom32, c->nrs, c->box, sv, wt);
    p3t_note_launches(3 + kDeepLevel);  // leaves, level offsets, deep levels, one a level
  }
  // own kernels here (the scans, sorts and moments count themselves): box 3,
  // keys, gather, lcp_levels, nodes_pre, node_counts, pre2bfs, nodes_bfs,
  // parents, lists
  p3t_note_launches(12);
  return cudaGetLastError() == cudaSuccess ? P3T_OK : P3T_ERR_CUDA;
}

// tree statistics on demand (diagnostics; not part of the step)
int p3t_run_tree_stats(p3t_ctx *c, cudaStream_t s) {
  int64_t *cnt = c->counters;
  P3T_CUDA_TRY(cudaMemsetAsync(&cnt[4], 0, 4 * sizeof(int64_t), s));
  const int64_t gn = p3t_grid(c->node_cap, kBlock, (int64_t)c->num_sms * P3T_NSM_BLOCKS);
  pdl_launch(k_tree_stats, dim3((unsigned)gn), dim3(kBlock), 0, s, &cnt[3], c->node_cap, c->node, &cnt[4]);
  p3t_note_launches(1);
  return cudaGetLastError() == cudaSuccess ? P3T_OK : P3T_ERR_CUDA;
}

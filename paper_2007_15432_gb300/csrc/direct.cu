// All-pairs sums of the soft force of Eq. softforce (the tree at theta = 0)
// and of its vector-Jacobian product (the adjoint), cut-off radii held fixed:
//   a_k = -G sum_j m_j K(r_kj / r_out,kj) r_kj / r_kj^3,
//   g_k += s sum_j J(r_kj) (m_k lam_j - m_j lam_k),  gm_k += s sum_j phi_kj lam_j . r_kj,
// J = phi I + psi r r^T, phi = K / r^3, psi = K'(y) / (r_out r^4) - 3 K / r^5.
//
// Layout: k_direct_pack writes every particle once as packed 4-vectors in
// the pair arithmetic's type; a block is 8 warps over 64 targets (two per
// lane); each warp takes one eighth of the block's source range and stages
// it 32 sources at a time in its own shared-memory slots (one broadcast load
// per 4-vector, shared by the lane's two targets).  A grid column
// (blockIdx.y) is one split of the sources; each block adds its 8 warps in
// order and writes its per-target sums to part[(split * C + c) * n + k];
// the last block of a target tile to finish adds the splits in order: the
// result does not depend on scheduling.
//
// Precision: FP64 throughout, or (MIXED) float-float positions whose
// difference (hi_k - hi_j) + (lo_k - lo_j) carries the relative coordinate
// to about 2^-24 of itself, FP32 pair terms summed in FP32 over a 32-source
// chunk and the chunk sums kept as float-float (TwoSum), so that no FP64
// instruction runs inside the pair loop.
#include <math.h>

#include <type_traits>

#include "p3t_internal.cuh"

namespace {

constexpr int kDW = 8;          // warps per block
constexpr int kDT = 2;          // targets per lane
constexpr int kDTB = 32 * kDT;  // targets per block
#ifndef P3T_DIRECT_MINB_MIXED
#define P3T_DIRECT_MINB_MIXED 3  // resident blocks per SM asked of the FP32 kernels
#endif

template <typename T>
struct alignas(4 * sizeof(T)) Q4 {
  T x, y, z, w;
};

template <bool MIXED>
struct DT {
  using T = double;
};
template <>
struct DT<true> {
  using T = float;
};

__device__ __forceinline__ double rsq(double a) { return rsqrt(a); }

// hi + lo += p without losing the rounding error of the addition (TwoSum)
__device__ __forceinline__ void two_sum_acc(float &hi, float &lo, float p) {
  const float s = hi + p;
  const float b = s - hi;
  lo += (hi - (s - b)) + (p - b);
  hi = s;
}

// one pair term: k the target (its mass, 1/r_out and adjoint), j the source
template <typename T, bool VJP>
__device__ __forceinline__ void pair_term(T rx, T ry, T rz, const Q4<T> &A, T iroj,
                                          const Q4<T> &L, T mk, T irok, T lxk, T lyk, T lzk,
                                          T g, T i1mg, T *acc) {
  // the FP64 path's term (the mixed path uses pair_term2)
  static_assert(std::is_same<T, double>::value, "FP64 pair term");
  const T r2 = rx * rx + ry * ry + rz * rz;
  const T ir = rsq(r2);
  const T irout = irok < iroj ? irok : iroj;  // 1 / max(r_out,k, r_out,j)
  const T yv = r2 * ir * irout;
  // y <= gamma: K = K' = 0.  The target itself (r2 = 0) gives 0 * inf = NaN
  // and leaves here too.
  if (!(yv > g)) return;
  T K = 1, dKr = 0;     // K(y) and K'(y) / r_out
  if (yv < (T)1) {
    const T u = (yv - g) * i1mg, u2 = u * u, u3 = u2 * u;
    K = u2 * u2 * ((T)35 - (T)84 * u + (T)70 * u2 - (T)20 * u3);
    if constexpr (VJP) {
      const T v = (T)1 - u;
      dKr = (T)140 * u3 * (v * v * v) * i1mg * irout;
    }
  }
  const T ir2 = ir * ir;
  const T phi = K * ir2 * ir;
  if constexpr (!VJP) {
    const T w = A.w * phi;  // m_j K / r^3
    acc[0] += w * rx;
    acc[1] += w * ry;
    acc[2] += w * rz;
  } else {
    const T psi = ir2 * ir2 * (dKr - (T)3 * K * ir);
    const T wx = mk * L.x - A.w * lxk, wy = mk * L.y - A.w * lyk, wz = mk * L.z - A.w * lzk;
    const T prw = psi * (rx * wx + ry * wy + rz * wz);
    acc[0] += phi * wx + prw * rx;
    acc[1] += phi * wy + prw * ry;
    acc[2] += phi * wz + prw * rz;
    acc[3] += phi * (L.x * rx + L.y * ry + L.z * rz);
  }
}

// The mixed kernels' pair term for a lane's two targets at once, one per half
// of each packed FP32 pair (f32x2 instructions round each half as the scalar
// one would), the source's values duplicated into both halves.  Branch-free:
// the changeover variable u = clamp((y - gamma) / (1 - gamma), 0, 1) gives K =
// 0 below gamma, 1 beyond r_out and the polynomial between (35 - 84 + 70 - 20
// = 1 exactly), and r^2 is kept above 1e-18 so that the target itself (r = 0,
// y = 0, K = 0) and far-away dummy targets add exact zeros without an inf.
// (Any real pair that close has y <= gamma: K = K' = 0 as well.)
struct PairConst2 {
  f2 g, i1mg, c35, c84, c70, c20, one, three, c140i;
};
template <bool VJP>
__device__ __forceinline__ void pair_term2(f2 rx, f2 ry, f2 rz, const Q4<float> &A, float iroj,
                                           const Q4<float> &L, f2 mk, f2 irok, f2 lxk, f2 lyk,
                                           f2 lzk, const PairConst2 &k, f2 *acc) {
  f2 r2 = fma2(rx, rx, fma2(ry, ry, mul2(rz, rz)));
  r2 = f2_pk(fmaxf(f2_lo(r2), 1e-18f), fmaxf(f2_hi(r2), 1e-18f));
  const f2 ir = f2_pk(rsqrtf(f2_lo(r2)), rsqrtf(f2_hi(r2)));
  const f2 irout = f2_pk(fminf(f2_lo(irok), iroj), fminf(f2_hi(irok), iroj));
  const f2 yv = mul2(mul2(r2, ir), irout);
  const f2 t = mul2(sub2(yv, k.g), k.i1mg);
  const f2 u = f2_pk(__saturatef(f2_lo(t)), __saturatef(f2_hi(t)));
  const f2 u2 = mul2(u, u), u3 = mul2(u2, u);
  const f2 poly = fma2(fma2(fma2(sub2(0ull, k.c20), u, k.c70), u, sub2(0ull, k.c84)), u, k.c35);
  const f2 K = mul2(mul2(u2, u2), poly);
  const f2 ir2 = mul2(ir, ir);
  const f2 phi = mul2(mul2(K, ir2), ir);
  if constexpr (!VJP) {
    const f2 w = mul2(f2_dup(A.w), phi);  // m_j K / r^3
    acc[0] = fma2(w, rx, acc[0]);
    acc[1] = fma2(w, ry, acc[1]);
    acc[2] = fma2(w, rz, acc[2]);
  } else {
    const f2 v = sub2(k.one, u);
    const f2 dKr = mul2(mul2(mul2(k.c140i, u3), mul2(mul2(v, v), v)), irout);
    const f2 psi = mul2(mul2(ir2, ir2), sub2(dKr, mul2(mul2(k.three, K), ir)));
    const f2 mA = f2_dup(A.w);
    const f2 wx = sub2(mul2(mk, f2_dup(L.x)), mul2(mA, lxk));
    const f2 wy = sub2(mul2(mk, f2_dup(L.y)), mul2(mA, lyk));
    const f2 wz = sub2(mul2(mk, f2_dup(L.z)), mul2(mA, lzk));
    const f2 prw = mul2(psi, fma2(rx, wx, fma2(ry, wy, mul2(rz, wz))));
    acc[0] = add2(acc[0], fma2(phi, wx, mul2(prw, rx)));
    acc[1] = add2(acc[1], fma2(phi, wy, mul2(prw, ry)));
    acc[2] = add2(acc[2], fma2(phi, wz, mul2(prw, rz)));
    acc[3] = fma2(phi, fma2(f2_dup(L.x), rx, fma2(f2_dup(L.y), ry, mul2(f2_dup(L.z), rz))),
                  acc[3]);
  }
}

// outputs: with one split, the block writes out_c[k] = (add ? out_c[k] : 0)
// + scale * sum itself; with several, the sums go to part
struct DOut {
  double *o[4];
  double scale;
  int add;
};

// Packs every particle once per call: A = (x_hi, y_hi, z_hi, m), B = (x_lo,
// y_lo, z_lo, 1 / r_out), L = (lam, 0), in the pair arithmetic's type (the
// lo parts are zero in FP64), so that no conversion or FP64 division is
// repeated per block.
template <bool MIXED, bool VJP>
__global__ void k_direct_pack(int64_t n, const double *x, const double *y, const double *z,
                              const double *m, const double *ro, const double *lx,
                              const double *ly, const double *lz,
                              Q4<typename DT<MIXED>::T> *A, Q4<typename DT<MIXED>::T> *B,
                              Q4<typename DT<MIXED>::T> *L) {
  pdl_wait();
  using T = typename DT<MIXED>::T;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
       j += (int64_t)gridDim.x * blockDim.x) {
    Q4<T> a, b;
    a.x = (T)x[j]; a.y = (T)y[j]; a.z = (T)z[j]; a.w = (T)m[j];
    b.x = b.y = b.z = 0;
    if constexpr (MIXED) {
      b.x = (T)(x[j] - (double)a.x);
      b.y = (T)(y[j] - (double)a.y);
      b.z = (T)(z[j] - (double)a.z);
    }
    b.w = (T)(1.0 / ro[j]);
    A[j] = a;
    B[j] = b;
    if constexpr (VJP) {
      Q4<T> l;
      l.x = (T)lx[j]; l.y = (T)ly[j]; l.z = (T)lz[j]; l.w = 0;
      L[j] = l;
    }
  }
}

template <bool MIXED, bool VJP>
__global__ void __launch_bounds__(kDW * 32, MIXED ? P3T_DIRECT_MINB_MIXED : 1)
    k_direct(int64_t n, int64_t chunk, const Q4<typename DT<MIXED>::T> *__restrict__ PA,
             const Q4<typename DT<MIXED>::T> *__restrict__ PB,
             const Q4<typename DT<MIXED>::T> *__restrict__ PL, double gamma, double *part,
             int32_t *tile_cnt, DOut out) {
  pdl_wait();
  using T = typename DT<MIXED>::T;
  constexpr int NC = VJP ? 4 : 3;
  __shared__ Q4<T> sA[kDW][32];                     // x_hi, y_hi, z_hi, m
  __shared__ Q4<T> sB[kDW][32];                     // x_lo, y_lo, z_lo, 1 / r_out
  __shared__ Q4<T> sL[VJP ? kDW : 1][VJP ? 32 : 1];  // lam
  // the 8 warps' sums: FP64, or (MIXED) float-float pairs added with FP32
  // instructions only (an FP64 instruction costs 64 FP32 issue slots here)
  __shared__ double red[MIXED ? 1 : kDW][NC][MIXED ? 1 : kDTB];
  __shared__ float red_h[MIXED ? kDW : 1][NC][MIXED ? kDTB : 1];
  __shared__ float red_l[MIXED ? kDW : 1][NC][MIXED ? kDTB : 1];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const T g = (T)gamma, i1mg = (T)(1.0 / (1.0 - gamma));

  T txh[kDT], tyh[kDT], tzh[kDT], txl[kDT], tyl[kDT], tzl[kDT];
  T tm[kDT], tiro[kDT], tlx[kDT], tly[kDT], tlz[kDT];
#pragma unroll
  for (int t = 0; t < kDT; ++t) {
    const int64_t k = (int64_t)blockIdx.x * kDTB + t * 32 + lane;
    txh[t] = tyh[t] = tzh[t] = txl[t] = tyl[t] = tzl[t] = 0;
    tm[t] = tiro[t] = tlx[t] = tly[t] = tlz[t] = 0;  // 1/r_out = 0: no pair term
    if (k < n) {
      const Q4<T> a = PA[k], b = PB[k];
      txh[t] = a.x; tyh[t] = a.y; tzh[t] = a.z; tm[t] = a.w;
      txl[t] = b.x; tyl[t] = b.y; tzl[t] = b.z; tiro[t] = b.w;
      if constexpr (VJP) {
        const Q4<T> l = PL[k];
        tlx[t] = l.x; tly[t] = l.y; tlz[t] = l.z;
      }
    }
  }
  struct TP {
    f2 xh, yh, zh, xl, yl, zl, m, iro, lx, ly, lz;
  } P{};
  PairConst2 kc{};
  if constexpr (MIXED) {
    P = TP{f2_pk(txh[0], txh[1]), f2_pk(tyh[0], tyh[1]), f2_pk(tzh[0], tzh[1]),
           f2_pk(txl[0], txl[1]), f2_pk(tyl[0], tyl[1]), f2_pk(tzl[0], tzl[1]),
           f2_pk(tm[0], tm[1]), f2_pk(tiro[0], tiro[1]), f2_pk(tlx[0], tlx[1]),
           f2_pk(tly[0], tly[1]), f2_pk(tlz[0], tlz[1])};
    kc = PairConst2{f2_dup((float)g), f2_dup((float)i1mg), f2_dup(35.f), f2_dup(84.f),
                    f2_dup(70.f), f2_dup(20.f), f2_dup(1.f), f2_dup(3.f),
                    f2_dup((float)(140.0 * (1.0 / (1.0 - gamma))))};
  }
  float fh[kDT][NC], fl[kDT][NC];  // MIXED running sums (float-float)
  double dd[kDT][NC];              // FP64 running sums
#pragma unroll
  for (int t = 0; t < kDT; ++t)
#pragma unroll
    for (int c = 0; c < NC; ++c) fh[t][c] = fl[t][c] = 0.0f, dd[t][c] = 0.0;

  // the split's sources, cut into 8 contiguous, equal (to one source) warp
  // ranges, walked in chunks of 32
  const int64_t b_lo = (int64_t)blockIdx.y * chunk;
  const int64_t b_len = max((int64_t)0, min(n, b_lo + chunk) - b_lo);
  const int64_t s_lo = b_lo + b_len * warp / kDW;
  const int64_t s_hi = b_lo + b_len * (warp + 1) / kDW;
  for (int64_t cb = s_lo; cb < s_hi; cb += 32) {
    const int lim = (int)min((int64_t)32, s_hi - cb);
    __syncwarp();
    if (lane < lim) {
      const int64_t j = cb + lane;
      sA[warp][lane] = PA[j];
      sB[warp][lane] = PB[j];
      if constexpr (VJP) sL[warp][lane] = PL[j];
    }
    __syncwarp();
    T acc[kDT][NC];
#pragma unroll
    for (int t = 0; t < kDT; ++t)
#pragma unroll
      for (int c = 0; c < NC; ++c) acc[t][c] = 0;
    if constexpr (MIXED) {
      // the lane's two targets as the halves of packed pairs
      static_assert(kDT == 2, "two targets per lane");
      f2 a2[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) a2[c] = 0ull;
#pragma unroll 2
      for (int q = 0; q < lim; ++q) {
        const Q4<T> A = sA[warp][q], B = sB[warp][q];
        Q4<T> L{0, 0, 0, 0};
        if constexpr (VJP) L = sL[warp][q];
        const f2 rx = add2(sub2(P.xh, f2_dup(A.x)), sub2(P.xl, f2_dup(B.x)));
        const f2 ry = add2(sub2(P.yh, f2_dup(A.y)), sub2(P.yl, f2_dup(B.y)));
        const f2 rz = add2(sub2(P.zh, f2_dup(A.z)), sub2(P.zl, f2_dup(B.z)));
        pair_term2<VJP>(rx, ry, rz, A, B.w, L, P.m, P.iro, P.lx, P.ly, P.lz, kc, a2);
      }
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        acc[0][c] = f2_lo(a2[c]);
        acc[1][c] = f2_hi(a2[c]);
      }
    } else {
#pragma unroll 4
      for (int q = 0; q < lim; ++q) {
        const Q4<T> A = sA[warp][q], B = sB[warp][q];
        Q4<T> L{0, 0, 0, 0};
        if constexpr (VJP) L = sL[warp][q];
#pragma unroll
        for (int t = 0; t < kDT; ++t) {
          T rx = txh[t] - A.x, ry = tyh[t] - A.y, rz = tzh[t] - A.z;
          pair_term<T, VJP>(rx, ry, rz, A, B.w, L, tm[t], tiro[t], tlx[t], tly[t], tlz[t], g,
                            i1mg, acc[t]);
        }
      }
    }
#pragma unroll
    for (int t = 0; t < kDT; ++t)
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        if constexpr (MIXED) two_sum_acc(fh[t][c], fl[t][c], acc[t][c]);
        else dd[t][c] += acc[t][c];
      }
  }
#pragma unroll
  for (int t = 0; t < kDT; ++t)
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      if constexpr (MIXED) {
        red_h[warp][c][t * 32 + lane] = fh[t][c];
        red_l[warp][c][t * 32 + lane] = fl[t][c];
      } else {
        red[warp][c][t * 32 + lane] = dd[t][c];
      }
    }
  __syncthreads();
  for (int e = threadIdx.x; e < NC * kDTB; e += kDW * 32) {
    const int c = e / kDTB, tt = e - c * kDTB;
    const int64_t k = (int64_t)blockIdx.x * kDTB + tt;
    if (k >= n) continue;
    double s = 0.0;
    if constexpr (MIXED) {
      float h = red_h[0][c][tt], l = red_l[0][c][tt];
      for (int w = 1; w < kDW; ++w) {
        two_sum_acc(h, l, red_h[w][c][tt]);
        l += red_l[w][c][tt];
      }
      s = (double)h + (double)l;
    } else {
      for (int w = 0; w < kDW; ++w) s += red[w][c][tt];
    }
    if (gridDim.y == 1) {
      double *o = c == 0 ? out.o[0] : (c == 1 ? out.o[1] : (c == 2 ? out.o[2] : out.o[3]));
      o[k] = (out.add ? o[k] : 0.0) + out.scale * s;
    } else {
      part[((int64_t)blockIdx.y * NC + c) * n + k] = s;
    }
  }
  if (gridDim.y == 1) return;
  // several splits: the last block of this target tile to arrive adds the
  // splits' sums in split order (the result does not depend on which block
  // that is) and resets the tile's counter for the next call
  __shared__ int last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(&tile_cnt[blockIdx.x], 1) == (int)gridDim.y - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  for (int e = threadIdx.x; e < NC * kDTB; e += kDW * 32) {
    const int c = e / kDTB, tt = e - c * kDTB;
    const int64_t k = (int64_t)blockIdx.x * kDTB + tt;
    if (k >= n) continue;
    double s = 0.0;
#pragma unroll 8
    for (int q = 0; q < (int)gridDim.y; ++q) s += __ldcg(&part[((int64_t)q * NC + c) * n + k]);
    double *o = c == 0 ? out.o[0] : (c == 1 ? out.o[1] : (c == 2 ? out.o[2] : out.o[3]));
    o[k] = (out.add ? o[k] : 0.0) + out.scale * s;
  }
  if (threadIdx.x == 0) tile_cnt[blockIdx.x] = 0;
}

// Work split: blocks of 64 targets x one source split.  With fewer than 8
// waves of target tiles alone, the sources are split so that the grid is at
// least 8 waves of resident blocks (the last, partial wave then costs at most
// an eighth); every split keeps at least 256 sources (a chunk per warp).
// With ns >= 2 splits, (ns - 1) n < 8 slots 64, so the partial sums, C ns n
// doubles, fit in 4 * 2 * 8 * slots * 64 (direct_part_doubles).
template <bool MIXED, bool VJP>
int blocks_per_sm() {
  static int b = 0;
  if (b == 0) {
    int v = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_direct<MIXED, VJP>, kDW * 32, 0) !=
            cudaSuccess || v < 1)
      v = 1;
    b = v;
  }
  return b;
}

int max_blocks_per_sm() {
  int b = blocks_per_sm<true, true>();
  b = b > blocks_per_sm<true, false>() ? b : blocks_per_sm<true, false>();
  b = b > blocks_per_sm<false, true>() ? b : blocks_per_sm<false, true>();
  b = b > blocks_per_sm<false, false>() ? b : blocks_per_sm<false, false>();
  return b;
}

struct Split {
  int64_t tiles, chunk;
  int nsplit;
};
Split split_for(const p3t_ctx *c, int64_t n, int bps) {
  Split s;
  s.tiles = (n + kDTB - 1) / kDTB;
  const int64_t slots = (int64_t)c->num_sms * bps;
  int64_t ns = 1;
  if (s.tiles < 8 * slots) ns = (8 * slots + s.tiles - 1) / s.tiles;
  const int64_t ns_max = (n + kDW * 32 - 1) / (kDW * 32);
  ns = ns > ns_max ? ns_max : ns;
  ns = ns < 1 ? 1 : ns;
  s.chunk = (n + ns - 1) / ns;
  s.chunk = (s.chunk + 31) / 32 * 32;
  s.nsplit = (int)((n + s.chunk - 1) / s.chunk);
  return s;
}

template <bool MIXED, bool VJP>
int launch_direct(p3t_ctx *c, const p3t_particles *p, const double *lx, const double *ly,
                  const double *lz, DOut out, cudaStream_t s) {
  constexpr int NC = VJP ? 4 : 3;
  const int64_t n = p->n;
  const Split sp = split_for(c, n, blocks_per_sm<MIXED, VJP>());
  if (sp.nsplit > 1 && (int64_t)NC * sp.nsplit * n > c->dpart_cap) return P3T_ERR_CAPACITY;
  using T = typename DT<MIXED>::T;
  Q4<T> *A = reinterpret_cast<Q4<T> *>(c->hw);  // 3 n packed 4-vectors <= 96 n bytes
  Q4<T> *B = A + n, *L = B + n;
  pdl_launch(k_direct_pack<MIXED, VJP>, dim3((unsigned)p3t_grid(n, 256, (int64_t)c->num_sms * 4)), dim3(256), 0, s, 
      n, p->x, p->y, p->z, p->m, p->r_out, lx, ly, lz, A, B, L);
  if (sp.nsplit > 1 && sp.tiles > c->dcnt_cap) return P3T_ERR_CAPACITY;
  const dim3 grid((unsigned)sp.tiles, (unsigned)sp.nsplit);
  pdl_launch(k_direct<MIXED, VJP>, dim3(grid), dim3(kDW * 32), 0, s, n, sp.chunk, A, B, L, c->prm.gamma, c->dpart,
                                                c->dcnt, out);
  p3t_note_launches(2);
  return cudaGetLastError() == cudaSuccess ? P3T_OK : P3T_ERR_CUDA;
}

}  // namespace

int64_t p3t_direct_part_doubles(const p3t_ctx *c) {
  return (int64_t)4 * 2 * 8 * c->num_sms * max_blocks_per_sm() * kDTB;
}

// with several splits there are fewer than 8 slots target tiles
int64_t p3t_direct_tile_counters(const p3t_ctx *c) {
  return (int64_t)8 * c->num_sms * max_blocks_per_sm();
}

int p3t_run_soft_force_direct(p3t_ctx *c, const p3t_particles *p, double *ax, double *ay,
                              double *az, cudaStream_t s) {
  if (p->n == 0) return P3T_OK;
  const DOut out{{ax, ay, az, nullptr}, -c->prm.G, 0};
  return c->prm.precision == P3T_MIXED ? launch_direct<true, false>(c, p, nullptr, nullptr,
                                                                    nullptr, out, s)
                                       : launch_direct<false, false>(c, p, nullptr, nullptr,
                                                                     nullptr, out, s);
}

int p3t_run_soft_force_vjp(p3t_ctx *c, const p3t_particles *p, double h, const double *lx,
                           const double *ly, const double *lz, double *gx, double *gy,
                           double *gz, double *gm, cudaStream_t s) {
  if (p->n == 0) return P3T_OK;
  const DOut out{{gx, gy, gz, gm}, h * c->prm.G, 1};
  return c->prm.precision == P3T_MIXED ? launch_direct<true, true>(c, p, lx, ly, lz, out, s)
                                       : launch_direct<false, true>(c, p, lx, ly, lz, out, s);
}

// Soft step: the changeover tree walk (Eq. softforce).
//
// One warp per target group (the highest tree node holding <= group_size
// particles, or a leaf), 32 targets per walk (larger groups are taken 32
// targets at a time; the warps take a group's first 32 targets and its rest
// as separate units of work, each walking with the whole group's box).  A walk of k < 32 targets gives each target r =
// floor(32 / k) lanes, each of which takes every r-th entry of a batch; the
// r partial sums are added at the end, so that lanes are not left idle.  The
// walk pops up to 32 nodes at a time from a per-warp stack, decides opening
// for all of them at once on the integer grid, and compacts accepted nodes,
// opened leaves and children with warp ballots / scans into shared-memory
// lists.  Each batch of 32 list entries is staged into shared memory once
// (one coalesced load per lane) and then read by every lane as a broadcast.
// Targets whose FP32 sum is ill-conditioned are redone in float-float right
// after their walk, all of them on one more traversal of the same list.
//
// Mixed path: positions are float-float (hi + lo) pairs, so a relative
// coordinate (x_i,hi - x_j,hi) + (x_i,lo - x_j,lo) carries the accuracy of an
// FP64 subtraction rounded to FP32, with no FP64 instruction per pair.  Pair
// and quadrupole terms are FP32; each batch's FP32 sum is folded into a
// float-float accumulator.  The mixed evaluators take the entries of a batch
// two at a time with packed FP32 pair instructions (add/sub/mul/fma.f32x2:
// one issue for two lanes' worth of FP32 work per thread), the batch staged
// so that one 16-byte shared load gives one coordinate of both entries;
// replicas split a batch by pairs, and each pair slot keeps its own partial
// sum (even and odd entries) until the batch is folded.  FP64 path:
// everything in FP64.
#include "p3t_internal.cuh"

namespace {

constexpr int kWarps = 4;                 // warps per block
constexpr int kPPCap = 32 * 33;           // p-p list: leftover < 32 + 32 leaves x <= 32
constexpr int kNDCap = 64;                // node list: leftover < 32 + 32 nodes
constexpr int kBigCap = 8;                // opened leaves with more than 32 members
// the FP32 candidate test r^2 < r_search^2 is widened by a factor 1.00001
// (applied to the squared radii in the gather); the exact FP64 test follows

struct WalkArgs {
  const TreeNode *node;
  const Mom64 *mom64;
  const Mom32 *mom32;
  const int32_t *leaf_list;
  const int64_t *d_nleaf;
  const int64_t *d_nnode;
  const double *sx, *sy, *sz, *sm, *sro, *srs;
  const float4 *spA, *spB;
  const float *srs32;
  const float *sml;          // mass lo parts (float-float masses with spA.w)
  const int32_t *idx;        // sorted -> caller
  double *ax, *ay, *az;      // caller order
  int32_t *stack;
  int64_t stack_cap;
  int32_t *cand_i, *cand_j;
  int64_t cand_cap;
  unsigned long long *cand_count;
  unsigned long long *counts;  // [2] n_pp, n_pnode (may be null)
  int64_t *cursor;
  DevStatus *st;
  SegView seg;                     // segments: the root of segment d is node d
  double G, gamma;
  double inv1mg;                   // 1 / (1 - gamma)
  float inv1mg_f, mgi_f;           // 1 / (1 - gamma), -gamma / (1 - gamma)
  float refine_cf;                 // refine when sum|term| > refine_cf * |a|
  int64_t bh[P3T_BITS + 1];
};

// integer box of a target group (a leaf) on the key grid
struct GroupBox {
  int32_t qlo0, qlo1, qlo2, qhi0, qhi1, qhi2, R;
  __device__ void load(const TreeNode &G) {
    qlo0 = G.qlo[0]; qlo1 = G.qlo[1]; qlo2 = G.qlo[2];
    qhi0 = G.qhi[0]; qhi1 = G.qhi[1]; qhi2 = G.qhi[2];
    R = G.R;
  }
};

__device__ __forceinline__ int warp_excl_scan(int v, int *total) {
  const int lane = threadIdx.x & 31;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int t = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += t;
  }
  *total = __shfl_sync(0xffffffffu, x, 31);
  return x - v;
}

__device__ __forceinline__ void two_sum(float &hi, float &lo, float b) {
  const float s = hi + b;
  const float bb = s - hi;
  const float err = (hi - (s - bb)) + (b - bb);
  hi = s;
  lo += err;
}

#ifndef P3T_PAIR_UNROLL
#define P3T_PAIR_UNROLL 1  // pair slots in flight per loop iteration
#endif
constexpr int kPairUnroll = P3T_PAIR_UNROLL;


// ---- per-target state (one lane per target) ---------------------------------
template <bool MIXED> struct Target;

template <> struct Target<true> {
  f2 X, Y, Z, XL, YL, ZL;              // (hi, hi) and (lo, lo) of each coordinate
  float inv_ro, rs2;                   // rs2: r_search^2 with the FP32 margin
  float ahx, ahy, ahz, alx, aly, alz;  // float-float accumulators
  float tabs;                          // sum of term magnitudes (conditioning)
  int32_t self;
  int rep, nrep;                       // this lane's replica of the target, replicas
  bool valid;
  __device__ void load(const WalkArgs &a, int32_t ti, bool v, int r, int nr) {
    valid = v;
    self = ti;
    rep = r;
    nrep = nr;
    ahx = ahy = ahz = alx = aly = alz = 0.f;
    tabs = 0.f;
    if (v) {
      const float4 A = a.spA[ti], B = a.spB[ti];
      X = f2_dup(A.x); Y = f2_dup(A.y); Z = f2_dup(A.z);
      XL = f2_dup(B.x); YL = f2_dup(B.y); ZL = f2_dup(B.z);
      inv_ro = B.w;
      rs2 = a.srs32[ti];
    } else {  // far away: no force, no candidate
      X = Y = Z = f2_dup(3.0e30f);
      XL = YL = ZL = 0ull;
      inv_ro = 0.f;
      rs2 = 0.f;
    }
  }
  __device__ void fold(float bx, float by, float bz) {
    two_sum(ahx, alx, bx); two_sum(ahy, aly, by); two_sum(ahz, alz, bz);
  }
  // adds the partial sums of the other replicas (lanes lane + q k) into the
  // first; nrep and k are warp-uniform
  __device__ void reduce(int k) {
    const int lane = threadIdx.x & 31;
    for (int q = 1; q < nrep; ++q) {
      const int src = lane < k ? lane + q * k : lane;
      const float hx = __shfl_sync(0xffffffffu, ahx, src), lx = __shfl_sync(0xffffffffu, alx, src);
      const float hy = __shfl_sync(0xffffffffu, ahy, src), ly = __shfl_sync(0xffffffffu, aly, src);
      const float hz = __shfl_sync(0xffffffffu, ahz, src), lz = __shfl_sync(0xffffffffu, alz, src);
      const float tb = __shfl_sync(0xffffffffu, tabs, src);
      if (lane < k) {
        two_sum(ahx, alx, hx); alx += lx;
        two_sum(ahy, aly, hy); aly += ly;
        two_sum(ahz, alz, hz); alz += lz;
        tabs += tb;
      }
    }
  }
};

template <> struct Target<false> {
  double x, y, z, iro, rs;  // iro = 1 / r_out
  double ax, ay, az;
  int32_t self;
  int rep, nrep;
  bool valid;
  __device__ void load(const WalkArgs &a, int32_t ti, bool v, int r, int nr) {
    valid = v;
    self = ti;
    rep = r;
    nrep = nr;
    ax = ay = az = 0.0;
    if (v) {
      x = a.sx[ti]; y = a.sy[ti]; z = a.sz[ti]; iro = 1.0 / a.sro[ti]; rs = a.srs[ti];
    } else {
      x = y = z = 1.0e300; iro = 1.0; rs = 0.0;
    }
  }
  __device__ void reduce(int k) {
    const int lane = threadIdx.x & 31;
    for (int q = 1; q < nrep; ++q) {
      const int src = lane < k ? lane + q * k : lane;
      const double x2 = __shfl_sync(0xffffffffu, ax, src);
      const double y2 = __shfl_sync(0xffffffffu, ay, src);
      const double z2 = __shfl_sync(0xffffffffu, az, src);
      if (lane < k) { ax += x2; ay += y2; az += z2; }
    }
  }
};

__device__ __forceinline__ void record_candidate(const WalkArgs &a, int32_t i,
                                                 int32_t j) {
  const unsigned long long slot = atomicAdd(a.cand_count, 1ull);
  if (slot < (unsigned long long)a.cand_cap) {
    a.cand_i[slot] = i;
    a.cand_j[slot] = j;
  }
}

// per-warp staging area for one batch of 32 entries
constexpr int kStageBytes = 32 * 96;
// mixed p-p batch by entry pairs (2p, 2p + 1): each 16-byte word holds one
// component of both entries, e.g. axy[p] = (x_2p, x_2p+1, y_2p, y_2p+1) of
// the hi parts; azw: z and mass; bxy, bzw: lo parts and 1 / r_out
struct StagePP32 {
  ulonglong2 axy[16], azw[16], bxy[16], bzw[16];
  float rs[32];
  int32_t idx[32];
};
// mixed node batch by pairs: centre hi / lo, -M, and the quadrupole
// (q0xy: xx, yy; q0zw: zz, xy; q1xy: xz, yz)
struct StageND32 {
  ulonglong2 hxy[16], hzw[16], lxy[16], lzw[16], q0xy[16], q0zw[16], q1xy[16];
};
struct StagePP64 { double x[32], y[32], z[32], m[32], iro[32], rs[32]; int32_t idx[32]; };
static_assert(sizeof(StagePP32) <= kStageBytes && sizeof(StagePP64) <= kStageBytes &&
              sizeof(StageND32) <= kStageBytes && sizeof(Mom64) * 32 <= kStageBytes,
              "stage area");

// entry s of a pair-staged batch: component c (0..3) of word w
__device__ __forceinline__ void stage_put(ulonglong2 *w, int s, float v0, float v1) {
  float *f = reinterpret_cast<float *>(&w[s >> 1]);
  f[s & 1] = v0;
  f[2 + (s & 1)] = v1;
}

// ---- particle-particle batch ----------------------------------------------
// Changeover pair terms in FP32 on float-float relative coordinates, for the
// two entries of pair slot p at once.  r^2 is kept above 1e-30 for the
// reciprocal square root: a coincident pair (the target itself) has y = 0 <
// gamma, K = 0 and so adds nothing, and f is formed as ((m K) r^-1) r^-2 so
// that no factor overflows.  The candidate test compares r^2 with
// max(r_search^2) (squared and widened in the gather); far-away dummy targets
// and the massless dummy entry that pads an odd batch never pass it.  The
// batch sums are kept negated (B = -sum f dx), which is exact.
__device__ __forceinline__ void pp_pair(const WalkArgs &a, Target<true> &t,
                                        const StagePP32 &S, int p, f2 &BX, f2 &BY, f2 &BZ,
                                        f2 &TB, unsigned &npp) {
  const ulonglong2 axy = S.axy[p], azw = S.azw[p], bxy = S.bxy[p], bzw = S.bzw[p];
  const f2 dx = add2(sub2(t.X, axy.x), sub2(t.XL, bxy.x));
  const f2 dy = add2(sub2(t.Y, axy.y), sub2(t.YL, bxy.y));
  const f2 dz = add2(sub2(t.Z, azw.x), sub2(t.ZL, bzw.x));
  const f2 r2 = fma2(dx, dx, fma2(dy, dy, mul2(dz, dz)));
  const float r2a = f2_lo(r2), r2b = f2_hi(r2);
  const f2 rinv = f2_pk(rsqrtf(fmaxf(r2a, 1e-30f)), rsqrtf(fmaxf(r2b, 1e-30f)));
  const f2 r = mul2(r2, rinv);
  const float ya = f2_lo(r) * fminf(t.inv_ro, f2_lo(bzw.y));
  const float yb = f2_hi(r) * fminf(t.inv_ro, f2_hi(bzw.y));
  const f2 x = f2_pk(__saturatef(fmaf(ya, a.inv1mg_f, a.mgi_f)),
                     __saturatef(fmaf(yb, a.inv1mg_f, a.mgi_f)));
  const f2 x2 = mul2(x, x);
  const f2 poly = fma2(fma2(fma2(f2_dup(-20.f), x, f2_dup(70.f)), x, f2_dup(-84.f)), x,
                       f2_dup(35.f));
  const f2 K = mul2(mul2(x2, x2), poly);
  const f2 f = mul2(mul2(mul2(azw.y, K), rinv), mul2(rinv, rinv));
  BX = fma2(f, dx, BX);
  BY = fma2(f, dy, BY);
  BZ = fma2(f, dz, BZ);
  TB = fma2(f, r, TB);
  if (r2a < fmaxf(t.rs2, S.rs[2 * p])) {
    const int32_t j = S.idx[2 * p];
    if (j != t.self) record_candidate(a, t.self, j);
    else --npp;  // the target itself is not a pair
  }
  if (r2b < fmaxf(t.rs2, S.rs[2 * p + 1])) {
    const int32_t j = S.idx[2 * p + 1];
    if (j != t.self) record_candidate(a, t.self, j);
    else --npp;
  }
}

// The targets' bounding box of one walk (float), the largest max(r_search^2,
// r_out^2) of its targets (widened like the candidate test) and the largest
// coordinate magnitude; per warp, in shared memory.
struct FarBox {
  float lo[3], hi[3], R2, amax;
};

// A source is far from every target of the walk when its distance to the
// box, less a margin that covers the FP32 rounding of the coordinates, is
// beyond max(r_search, r_out) of the source and of every target: then K = 1
// for every pair (y >= 1) and no pair is a neighbour candidate.
__device__ __forceinline__ bool far_from(const FarBox &b, const float4 A, const float4 B,
                                         float rs2s) {
  const float x = A.x + B.x, y = A.y + B.y, z = A.z + B.z;
  const float m = 9.5367431640625e-7f *  // 2^-20 of the coordinates' scale
                  (b.amax + fmaxf(fabsf(x), fmaxf(fabsf(y), fabsf(z))));
  const float gx = fmaxf(fmaxf(b.lo[0] - x, x - b.hi[0]) - m, 0.f);
  const float gy = fmaxf(fmaxf(b.lo[1] - y, y - b.hi[1]) - m, 0.f);
  const float gz = fmaxf(fmaxf(b.lo[2] - z, z - b.hi[2]) - m, 0.f);
  const float d2 = gx * gx + gy * gy + gz * gz;
  const float ro = 1.0f / B.w;  // B.w = 1 / r_out
  const float R2 = fmaxf(b.R2, fmaxf(rs2s, ro * ro * 1.00001f));
  return d2 > 0.f && d2 >= R2;
}

// The FP64 walk's counterpart: the targets' box in FP64 and the largest
// max(r_search, r_out)^2 of its targets.  A source whose distance to the box
// exceeds max(r_search, r_out) of the source and of every target by a
// relative 1e-9 (far above the rounding of the pair's r and y) has y >= 1
// (K = 1 exactly) and r^2 >= r_search,max^2 for every target: the far
// evaluation below then gives the bits of the full one.
struct FarBox64 {
  double lo[3], hi[3], R2;
};
template <bool MIXED> struct BoxOf { using type = FarBox; };
template <> struct BoxOf<false> { using type = FarBox64; };

__device__ __forceinline__ bool far_from64(const FarBox64 &b, double x, double y, double z,
                                           double ro, double rs) {
  const double gx = fmax(fmax(b.lo[0] - x, x - b.hi[0]), 0.0);
  const double gy = fmax(fmax(b.lo[1] - y, y - b.hi[1]), 0.0);
  const double gz = fmax(fmax(b.lo[2] - z, z - b.hi[2]), 0.0);
  const double d2 = gx * gx + gy * gy + gz * gz;
  const double R2 = fmax(b.R2, fmax(rs * rs, ro * ro));
  return d2 > 0.0 && d2 >= R2 * (1.0 + 1e-9);
}

// pair terms with K = 1 and no candidate test (the batch is far, see above):
// the same operations as pp_pair's K = 1 case, so the same bits
__device__ __forceinline__ void pp_pair_far(Target<true> &t, const StagePP32 &S, int p, f2 &BX,
                                            f2 &BY, f2 &BZ, f2 &TB) {
  const ulonglong2 axy = S.axy[p], azw = S.azw[p], bxy = S.bxy[p], bzw = S.bzw[p];
  const f2 dx = add2(sub2(t.X, axy.x), sub2(t.XL, bxy.x));
  const f2 dy = add2(sub2(t.Y, axy.y), sub2(t.YL, bxy.y));
  const f2 dz = add2(sub2(t.Z, azw.x), sub2(t.ZL, bzw.x));
  const f2 r2 = fma2(dx, dx, fma2(dy, dy, mul2(dz, dz)));
  const f2 rinv = f2_pk(rsqrtf(f2_lo(r2)), rsqrtf(f2_hi(r2)));
  const f2 r = mul2(r2, rinv);
  const f2 f = mul2(mul2(azw.y, rinv), mul2(rinv, rinv));
  BX = fma2(f, dx, BX);
  BY = fma2(f, dy, BY);
  BZ = fma2(f, dz, BZ);
  TB = fma2(f, r, TB);
}

// the batch sums of the even and odd slots into the target: the force sums
// negated back (B = -sum), the magnitude sum as it is
__device__ __forceinline__ void fold_pairs(Target<true> &t, f2 BX, f2 BY, f2 BZ, f2 TB) {
  t.fold(-(f2_lo(BX) + f2_hi(BX)), -(f2_lo(BY) + f2_hi(BY)), -(f2_lo(BZ) + f2_hi(BZ)));
  t.tabs += f2_lo(TB) + f2_hi(TB);
}

__device__ __forceinline__ void eval_pp(const WalkArgs &a, Target<true> &t, const int32_t *list,
                                        int nsrc, void *stage, const FarBox &box,
                                        unsigned &npp) {
  StagePP32 &S = *reinterpret_cast<StagePP32 *>(stage);
  const int lane = threadIdx.x & 31;
  bool near = false;
  float4 A = make_float4(1.0e18f, 1.0e18f, 1.0e18f, 0.f), B = make_float4(0.f, 0.f, 0.f, 0.f);
  float rs = 0.f;
  int32_t j = -1;
  if (lane < nsrc) {
    j = list[lane];
    A = __ldg(&a.spA[j]);
    B = __ldg(&a.spB[j]);
    rs = __ldg(&a.srs32[j]);
    near = !far_from(box, A, B, rs);
  }
  // lanes past the batch stage a massless dummy far from everything
  stage_put(S.axy, lane, A.x, A.y);
  stage_put(S.azw, lane, A.z, A.w);
  stage_put(S.bxy, lane, B.x, B.y);
  stage_put(S.bzw, lane, B.z, B.w);
  S.rs[lane] = rs;
  S.idx[lane] = j;
  const bool any_near = __any_sync(0xffffffffu, near);
  __syncwarp();
  f2 BX = 0ull, BY = 0ull, BZ = 0ull, TB = 0ull;
  npp += (t.valid && t.rep == 0) ? (unsigned)nsrc : 0u;
  const int np = (nsrc + 1) >> 1;
  if (any_near) {
#pragma unroll kPairUnroll
    for (int p = t.rep; p < np; p += t.nrep) pp_pair(a, t, S, p, BX, BY, BZ, TB, npp);
  } else {
#pragma unroll kPairUnroll
    for (int p = t.rep; p < np; p += t.nrep) pp_pair_far(t, S, p, BX, BY, BZ, TB);
  }
  __syncwarp();
  fold_pairs(t, BX, BY, BZ, TB);
}

__device__ __forceinline__ void eval_pp(const WalkArgs &a, Target<false> &t, const int32_t *list,
                                        int nsrc, void *stage, const FarBox64 &box,
                                        unsigned &npp) {
  StagePP64 &S = *reinterpret_cast<StagePP64 *>(stage);
  const int lane = threadIdx.x & 31;
  bool near = false;
  if (lane < nsrc) {
    const int32_t j = list[lane];
    const double x = a.sx[j], y = a.sy[j], z = a.sz[j], ro = a.sro[j], rs = a.srs[j];
    S.x[lane] = x; S.y[lane] = y; S.z[lane] = z;
    S.m[lane] = a.sm[j]; S.iro[lane] = 1.0 / ro; S.rs[lane] = rs;
    S.idx[lane] = j;
    near = !far_from64(box, x, y, z, ro, rs);
  }
  const bool any_near = __any_sync(0xffffffffu, near);
  __syncwarp();
  npp += (t.valid && t.rep == 0) ? (unsigned)nsrc : 0u;
  if (!any_near) {
    // K = 1 for every pair and no candidate: the full loop's operations with
    // K = 1 (m K = m exactly)
    for (int s = t.rep; s < nsrc; s += t.nrep) {
      const double dx = t.x - S.x[s], dy = t.y - S.y[s], dz = t.z - S.z[s];
      const double r2 = dx * dx + dy * dy + dz * dz;
      const double rinv = r2 > 0.0 ? rsqrt(r2) : 0.0;
      const double f = S.m[s] * (rinv * rinv * rinv);
      t.ax -= f * dx; t.ay -= f * dy; t.az -= f * dz;
    }
    __syncwarp();
    return;
  }
  for (int s = t.rep; s < nsrc; s += t.nrep) {
    const double dx = t.x - S.x[s], dy = t.y - S.y[s], dz = t.z - S.z[s];
    const double r2 = dx * dx + dy * dy + dz * dz;
    const double rinv = r2 > 0.0 ? rsqrt(r2) : 0.0;
    const double r = r2 * rinv;
    // y = r / max(r_out,i, r_out,j) as r min(1 / r_out): one reciprocal a
    // staged source, not a division a pair
    const double y = r * fmin(t.iro, S.iro[s]);
    double x = (y - a.gamma) * a.inv1mg;
    x = x < 0.0 ? 0.0 : (x > 1.0 ? 1.0 : x);
    const double x2 = x * x;
    const double K = (x2 * x2) * (((-20.0 * x + 70.0) * x - 84.0) * x + 35.0);
    const double f = S.m[s] * K * (rinv * rinv * rinv);
    t.ax -= f * dx; t.ay -= f * dy; t.az -= f * dz;
    const double rsj = fmax(t.rs, S.rs[s]);
    if (r2 < rsj * rsj && t.valid) {
      const int32_t j = S.idx[s];
      if (j != t.self) record_candidate(a, t.self, j);
      else --npp;
    }
  }
  __syncwarp();
}

// ---- particle-node batch (monopole + traceless quadrupole) ---------------
// a += -M r/r^3 + Q.r/r^5 - (5/2)(r.Q.r) r/r^7, r = x_i - com, for the two
// nodes of pair slot p (the stage holds -M)
__device__ __forceinline__ void node_pair(Target<true> &t, const StageND32 &S, int p, f2 &BX,
                                          f2 &BY, f2 &BZ, f2 &TB) {
  const ulonglong2 hxy = S.hxy[p], hzw = S.hzw[p], lxy = S.lxy[p], lzw = S.lzw[p];
  const ulonglong2 q0xy = S.q0xy[p], q0zw = S.q0zw[p], q1xy = S.q1xy[p];
  const f2 dx = add2(sub2(t.X, hxy.x), sub2(t.XL, lxy.x));
  const f2 dy = add2(sub2(t.Y, hxy.y), sub2(t.YL, lxy.y));
  const f2 dz = add2(sub2(t.Z, hzw.x), sub2(t.ZL, lzw.x));
  const f2 r2 = fma2(dx, dx, fma2(dy, dy, mul2(dz, dz)));
  const f2 rinv = f2_pk(rsqrtf(fmaxf(f2_lo(r2), 1e-30f)), rsqrtf(fmaxf(f2_hi(r2), 1e-30f)));
  const f2 rinv2 = mul2(rinv, rinv);
  const f2 rinv3 = mul2(rinv2, rinv);
  const f2 rinv5 = mul2(rinv3, rinv2);
  // q0xy = (xx, yy), q0zw = (zz, xy), q1xy = (xz, yz)
  const f2 qx = fma2(q0xy.x, dx, fma2(q0zw.y, dy, mul2(q1xy.x, dz)));
  const f2 qy = fma2(q0zw.y, dx, fma2(q0xy.y, dy, mul2(q1xy.y, dz)));
  const f2 qz = fma2(q1xy.x, dx, fma2(q1xy.y, dy, mul2(q0zw.x, dz)));
  const f2 rqr = fma2(dx, qx, fma2(dy, qy, mul2(dz, qz)));
  const f2 c = fma2(mul2(f2_dup(-2.5f), rqr), mul2(rinv5, rinv2), mul2(hzw.y, rinv3));
  BX = fma2(c, dx, fma2(qx, rinv5, BX));
  BY = fma2(c, dy, fma2(qy, rinv5, BY));
  BZ = fma2(c, dz, fma2(qz, rinv5, BZ));
  TB = fma2(hzw.y, rinv2, TB);  // -M / r^2
}

__device__ __forceinline__ void eval_nodes(const WalkArgs &a, Target<true> &t,
                                           const int32_t *list, int nnd, void *stage,
                                           unsigned &npn) {
  StageND32 &S = *reinterpret_cast<StageND32 *>(stage);
  const int lane = threadIdx.x & 31;
  // lanes past the batch stage a massless, quadrupole-free dummy far away
  float4 hi = make_float4(1.0e18f, 1.0e18f, 1.0e18f, 0.f), lo = make_float4(0.f, 0.f, 0.f, 0.f);
  float4 q0 = lo, q1 = lo;
  if (lane < nnd) {
    const Mom32 *m = &a.mom32[list[lane]];
    hi = __ldg(&m->hi); lo = __ldg(&m->lo);
    q0 = __ldg(&m->q0); q1 = __ldg(&m->q1);
  }
  stage_put(S.hxy, lane, hi.x, hi.y);
  stage_put(S.hzw, lane, hi.z, -hi.w);
  stage_put(S.lxy, lane, lo.x, lo.y);
  stage_put(S.lzw, lane, lo.z, lo.w);
  stage_put(S.q0xy, lane, q0.x, q0.y);
  stage_put(S.q0zw, lane, q0.z, q0.w);
  stage_put(S.q1xy, lane, q1.x, q1.y);
  __syncwarp();
  f2 BX = 0ull, BY = 0ull, BZ = 0ull, TB = 0ull;
  npn += (t.valid && t.rep == 0) ? (unsigned)nnd : 0u;
  const int np = (nnd + 1) >> 1;
#pragma unroll kPairUnroll
  for (int p = t.rep; p < np; p += t.nrep) node_pair(t, S, p, BX, BY, BZ, TB);
  __syncwarp();
  // force sums as they are; the magnitude sum was of -M / r^2
  t.fold(f2_lo(BX) + f2_hi(BX), f2_lo(BY) + f2_hi(BY), f2_lo(BZ) + f2_hi(BZ));
  t.tabs -= f2_lo(TB) + f2_hi(TB);
}

__device__ __forceinline__ void eval_nodes(const WalkArgs &a, Target<false> &t,
                                           const int32_t *list, int nnd, void *stage,
                                           unsigned &npn) {
  Mom64 *S = reinterpret_cast<Mom64 *>(stage);
  const int lane = threadIdx.x & 31;
  if (lane < nnd) S[lane] = a.mom64[list[lane]];
  __syncwarp();
  npn += (t.valid && t.rep == 0) ? (unsigned)nnd : 0u;
  for (int s = t.rep; s < nnd; s += t.nrep) {
    const Mom64 &m = S[s];
    const double dx = t.x - m.cx, dy = t.y - m.cy, dz = t.z - m.cz;
    const double r2 = dx * dx + dy * dy + dz * dz;
    const double rinv = r2 > 0.0 ? rsqrt(r2) : 0.0;
    const double rinv2 = rinv * rinv, rinv3 = rinv2 * rinv, rinv5 = rinv3 * rinv2;
    const double qx = m.qxx * dx + m.qxy * dy + m.qxz * dz;
    const double qy = m.qxy * dx + m.qyy * dy + m.qyz * dz;
    const double qz = m.qxz * dx + m.qyz * dy + m.qzz * dz;
    const double rqr = dx * qx + dy * qy + dz * qz;
    const double c = -m.M * rinv3 - 2.5 * rqr * rinv5 * rinv2;
    t.ax += c * dx + qx * rinv5;
    t.ay += c * dy + qy * rinv5;
    t.az += c * dz + qz * rinv5;
  }
  __syncwarp();
}

// writes the target's acceleration; returns whether the target is to be
// redone in float-float (mixed path)
template <bool MIXED>
__device__ __forceinline__ bool write_result(const WalkArgs &a, Target<MIXED> &t);

template <>
__device__ __forceinline__ bool write_result<true>(const WalkArgs &a, Target<true> &t) {
  if (!t.valid || t.rep != 0) return false;
  const double x = (double)t.ahx + (double)t.alx;
  const double y = (double)t.ahy + (double)t.aly;
  const double z = (double)t.ahz + (double)t.alz;
  const int32_t i = a.idx[t.self];
  a.ax[i] = a.G * x; a.ay[i] = a.G * y; a.az[i] = a.G * z;
  // FP32 terms carry ~1e-7 relative error each; where they cancel to a sum
  // much smaller than their magnitudes the target is redone in float-float
  const float amag = sqrtf((float)(x * x + y * y + z * z));
  return t.tabs > a.refine_cf * amag;
}

template <>
__device__ __forceinline__ bool write_result<false>(const WalkArgs &a, Target<false> &t) {
  if (!t.valid || t.rep != 0) return false;
  const int32_t i = a.idx[t.self];
  a.ax[i] = a.G * t.ax; a.ay[i] = a.G * t.ay; a.az[i] = a.G * t.az;
  return false;
}

// ---- the traversal, shared by the group walk and the float-float redo ------
// Pops up to 32 nodes per round, decides opening on the integer grid, and
// hands full batches of 32 accepted nodes / leaf members to the evaluator.
// Returns false when the walk had to stop (capacity or round bound).
template <class Ev>
__device__ bool traverse(const WalkArgs &a, const GroupBox &gb, int32_t first, int32_t *stack,
                         int32_t *pp, int32_t *nd, int32_t *big,
                         const int64_t *s_bh, int64_t round_limit, Ev &ev) {
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  int top = 1, npl = 0, nnd = 0, nbig = 0;
  int64_t rounds = 0;
  // sorted order keeps each segment contiguous, and segment d's root (level
  // 0, d-th in key order) is BFS node d: start at the root of the segment
  // that holds sorted particle `first`.  Every box inside the root cube lies
  // within 2^21 half cells of its centre on each axis, so when the root's
  // Barnes-Hut threshold exceeds 3 (2^21)^2 the root is opened for every
  // group: its children then start the stack, where the first round would
  // have pushed them
  const int32_t root = seg_at(a.seg, first);
  const int4 rc = __ldg(reinterpret_cast<const int4 *>(&a.node[root]) + 3);  // child0, nchild
  if (s_bh[0] > (3ll << 42) && rc.y > 0) {
    if (lane < rc.y) stack[lane] = rc.x + lane;
    top = rc.y;
  } else if (lane == 0) {
    stack[0] = root;
  }
  __syncwarp();
  while (top > 0) {
    if (++rounds > round_limit) {
      if (lane == 0) dev_fail(a.st, P3T_ERR_TIMEOUT, 43, 0);
      return false;
    }
    const int k = top < 32 ? top : 32;
    top -= k;
    int32_t id = -1;
    bool acc_node = false, open_leaf = false, open_inner = false;
    int32_t child0 = 0, nchild = 0, first = 0, count = 0;
    if (lane < k) {
      id = stack[top + lane];
      const int4 *r = reinterpret_cast<const int4 *>(&a.node[id]);
      const int4 q0 = __ldg(r), q1 = __ldg(r + 1), q2 = __ldg(r + 2), q3 = __ldg(r + 3);
      // (i) Barnes-Hut on the grid: half units, group cells [2 qlo, 2 qhi + 2]
      int64_t d2 = 0, g2 = 0;
      {
        int32_t d = max(0, max(2 * gb.qlo0 - q2.x, q2.x - (2 * gb.qhi0 + 2)));
        d2 += (int64_t)d * d;
        d = max(0, max(2 * gb.qlo1 - q2.y, q2.y - (2 * gb.qhi1 + 2)));
        d2 += (int64_t)d * d;
        d = max(0, max(2 * gb.qlo2 - q2.z, q2.z - (2 * gb.qhi2 + 2)));
        d2 += (int64_t)d * d;
      }
      // (ii) cut-off reach: lower-bound gap against the larger search reach
      {
        int32_t e = max(0, max(q0.x - gb.qhi0 - 2, gb.qlo0 - q1.x - 2));
        g2 += (int64_t)e * e;
        e = max(0, max(q0.y - gb.qhi1 - 2, gb.qlo1 - q1.y - 2));
        g2 += (int64_t)e * e;
        e = max(0, max(q0.z - gb.qhi2 - 2, gb.qlo2 - q1.z - 2));
        g2 += (int64_t)e * e;
      }
      const int64_t R = max(gb.R, q0.w);
      const bool open = (d2 < s_bh[q1.w]) || (g2 < R * R);
      child0 = q3.x; nchild = q3.y; first = q3.z; count = q3.w;
      acc_node = !open;
      open_leaf = open && nchild == 0;
      open_inner = open && nchild > 0;
    }
    // accepted nodes -> node list
    {
      const unsigned m = __ballot_sync(0xffffffffu, acc_node);
      if (acc_node) nd[nnd + __popc(m & lt)] = id;
      nnd += __popc(m);
    }
    // opened big leaves (> 32 members) -> their own list
    {
      const bool isbig = open_leaf && count > 32;
      const unsigned m = __ballot_sync(0xffffffffu, isbig);
      if (isbig) {
        const int slot = nbig + __popc(m & lt);
        if (slot < kBigCap) big[slot] = id;
      }
      nbig += __popc(m);
      if (isbig) open_leaf = false;
    }
    __syncwarp();  // every lane has read its stack entry before any push
    // children of opened inner nodes -> stack
    {
      int tot;
      const int c = open_inner ? nchild : 0;
      const int off = warp_excl_scan(c, &tot);
      if (top + tot > a.stack_cap) {
        if (lane == 0) dev_fail(a.st, P3T_ERR_CAPACITY, 40, top + tot);
        return false;
      }
      for (int q = 0; q < c; ++q) stack[top + off + q] = child0 + q;
      top += tot;
    }
    // members of opened leaves -> p-p list
    {
      int tot;
      const int c = open_leaf ? count : 0;
      const int off = warp_excl_scan(c, &tot);
      for (int q = 0; q < c; ++q) pp[npl + off + q] = first + q;
      npl += tot;
    }
    __syncwarp();
    if (nbig > kBigCap) {
      if (lane == 0) dev_fail(a.st, P3T_ERR_CAPACITY, 41, nbig);
      return false;
    }
    // evaluate full batches
    int o = 0;
    for (; nnd - o >= 32; o += 32) ev.nodes(nd + o, 32);
    if (o) {
      __syncwarp();
      const int rem = nnd - o;
      const int32_t v = lane < rem ? nd[o + lane] : 0;
      __syncwarp();
      if (lane < rem) nd[lane] = v;
      nnd = rem;
    }
    o = 0;
    for (; npl - o >= 32; o += 32) ev.pp(pp + o, 32);
    if (o) {
      __syncwarp();
      const int rem = npl - o;
      const int32_t v = lane < rem ? pp[o + lane] : 0;
      __syncwarp();
      if (lane < rem) pp[lane] = v;
      npl = rem;
    }
    __syncwarp();
  }
  if (nnd) ev.nodes(nd, nnd);
  if (npl) ev.pp(pp, npl);
  // big leaves, 32 members at a time, straight from their index range
  for (int b = 0; b < nbig; ++b) {
    const TreeNode &B = a.node[big[b]];
    for (int32_t s0 = B.first; s0 < B.first + B.count; s0 += 32) {
      const int ns = min(32, B.first + B.count - s0);
      __syncwarp();
      if (lane < ns) pp[lane] = s0 + lane;
      __syncwarp();
      ev.pp(pp, ns);
    }
  }
  __syncwarp();
  return true;
}

// up to 32 targets of a group (each on nrep lanes), batches staged in shared
// memory
template <bool MIXED> struct GroupEval {
  const WalkArgs &a;
  Target<MIXED> &t;
  void *stage;
  const typename BoxOf<MIXED>::type &box;
  unsigned &npp, &npn;
  __device__ void nodes(const int32_t *list, int n) { eval_nodes(a, t, list, n, stage, npn); }
  __device__ void pp(const int32_t *list, int n) { eval_pp(a, t, list, n, stage, box, npp); }
};

// the walk's FarBox from its (valid) targets, written by lane 0
__device__ __forceinline__ void far_box(const Target<true> &t, FarBox &b) {
  const float x = f2_lo(t.X) + f2_lo(t.XL), y = f2_lo(t.Y) + f2_lo(t.YL),
              z = f2_lo(t.Z) + f2_lo(t.ZL);
  const float inf = __int_as_float(0x7f800000);
  float lo0 = t.valid ? x : inf, lo1 = t.valid ? y : inf, lo2 = t.valid ? z : inf;
  float hi0 = t.valid ? x : -inf, hi1 = t.valid ? y : -inf, hi2 = t.valid ? z : -inf;
  const float ro = 1.0f / t.inv_ro;
  float R2 = t.valid ? fmaxf(t.rs2, ro * ro * 1.00001f) : 0.f;
  float am = t.valid ? fmaxf(fabsf(x), fmaxf(fabsf(y), fabsf(z))) : 0.f;
  for (int o = 16; o > 0; o >>= 1) {
    lo0 = fminf(lo0, __shfl_xor_sync(0xffffffffu, lo0, o));
    lo1 = fminf(lo1, __shfl_xor_sync(0xffffffffu, lo1, o));
    lo2 = fminf(lo2, __shfl_xor_sync(0xffffffffu, lo2, o));
    hi0 = fmaxf(hi0, __shfl_xor_sync(0xffffffffu, hi0, o));
    hi1 = fmaxf(hi1, __shfl_xor_sync(0xffffffffu, hi1, o));
    hi2 = fmaxf(hi2, __shfl_xor_sync(0xffffffffu, hi2, o));
    R2 = fmaxf(R2, __shfl_xor_sync(0xffffffffu, R2, o));
    am = fmaxf(am, __shfl_xor_sync(0xffffffffu, am, o));
  }
  __syncwarp();
  if ((threadIdx.x & 31) == 0) {
    b.lo[0] = lo0; b.lo[1] = lo1; b.lo[2] = lo2;
    b.hi[0] = hi0; b.hi[1] = hi1; b.hi[2] = hi2;
    b.R2 = R2;
    b.amax = am;
  }
  __syncwarp();
}

// the FP64 walk's FarBox64 from its (valid) targets, written by lane 0
__device__ __forceinline__ void far_box64(const Target<false> &t, FarBox64 &b) {
  const double inf = __longlong_as_double(0x7ff0000000000000ll);
  double lo0 = t.valid ? t.x : inf, lo1 = t.valid ? t.y : inf, lo2 = t.valid ? t.z : inf;
  double hi0 = t.valid ? t.x : -inf, hi1 = t.valid ? t.y : -inf, hi2 = t.valid ? t.z : -inf;
  const double ro = 1.0 / t.iro;
  double R2 = t.valid ? fmax(t.rs * t.rs, ro * ro) : 0.0;
  for (int o = 16; o > 0; o >>= 1) {
    lo0 = fmin(lo0, __shfl_xor_sync(0xffffffffu, lo0, o));
    lo1 = fmin(lo1, __shfl_xor_sync(0xffffffffu, lo1, o));
    lo2 = fmin(lo2, __shfl_xor_sync(0xffffffffu, lo2, o));
    hi0 = fmax(hi0, __shfl_xor_sync(0xffffffffu, hi0, o));
    hi1 = fmax(hi1, __shfl_xor_sync(0xffffffffu, hi1, o));
    hi2 = fmax(hi2, __shfl_xor_sync(0xffffffffu, hi2, o));
    R2 = fmax(R2, __shfl_xor_sync(0xffffffffu, R2, o));
  }
  __syncwarp();
  if ((threadIdx.x & 31) == 0) {
    b.lo[0] = lo0; b.lo[1] = lo1; b.lo[2] = lo2;
    b.hi[0] = hi0; b.hi[1] = hi1; b.hi[2] = hi2;
    b.R2 = R2;
  }
  __syncwarp();
}

__device__ __forceinline__ FF ff_shfl(FF a, int src) {
  return {__shfl_sync(0xffffffffu, a.h, src), __shfl_sync(0xffffffffu, a.l, src)};
}

// one target, all 32 lanes, float-float (the refinement of ill-conditioned
// targets): relative coordinates, r^2, 1/r, masses, monopoles and the sums in
// float-float (terms to ~1e-13 of themselves); the changeover factor K and
// the quadrupole correction in FP32 (exact K = 1 beyond r_out)
struct RefineEval {
  const WalkArgs &a;
  float xh, yh, zh, xl, yl, zl, inv_ro;
  FF ax, ay, az;
  int s0, ds;  // this lane's entries of a batch: s0, s0 + ds, ...
  __device__ void term(FF dx, FF dy, FF dz, FF m, float k_inv_ro, bool pp, const float4 q0,
                       const float4 q1) {
    const FF r2 = ff_add(ff_add(ff_mul(dx, dx), ff_mul(dy, dy)), ff_mul(dz, dz));
    if (r2.h == 0.0f) return;  // the target itself
    const FF ri = ff_rsqrt(r2);
    const FF ri3 = ff_mul(ff_mul(ri, ri), ri);
    float K = 1.0f;
    if (pp) {
      const float y = r2.h * ri.h * k_inv_ro;
      const float x = __saturatef(fmaf(y, a.inv1mg_f, a.mgi_f));
      const float x2 = x * x;
      K = (x2 * x2) * fmaf(fmaf(fmaf(-20.f, x, 70.f), x, -84.f), x, 35.f);
      if (K == 0.0f) return;
    }
    const FF f = ff_mul(ff_mulf(m, K), ri3);  // m K / r^3
    ax = ff_add(ax, ff_mul(f, {-dx.h, -dx.l}));
    ay = ff_add(ay, ff_mul(f, {-dy.h, -dy.l}));
    az = ff_add(az, ff_mul(f, {-dz.h, -dz.l}));
    if (!pp) {  // Q.r / r^5 - (5/2) (r.Q.r) r / r^7 in FP32
      const float ddx = dx.h, ddy = dy.h, ddz = dz.h, rinv = ri.h;
      const float rinv2 = rinv * rinv, rinv5 = rinv2 * rinv2 * rinv;
      const float qx = fmaf(q0.x, ddx, fmaf(q0.w, ddy, q1.x * ddz));
      const float qy = fmaf(q0.w, ddx, fmaf(q0.y, ddy, q1.y * ddz));
      const float qz = fmaf(q1.x, ddx, fmaf(q1.y, ddy, q0.z * ddz));
      const float rqr = fmaf(ddx, qx, fmaf(ddy, qy, ddz * qz));
      const float c = -2.5f * rqr * rinv5 * rinv2;
      ax = ff_add(ax, ff_fast(fmaf(c, ddx, qx * rinv5), 0.0f));
      ay = ff_add(ay, ff_fast(fmaf(c, ddy, qy * rinv5), 0.0f));
      az = ff_add(az, ff_fast(fmaf(c, ddz, qz * rinv5), 0.0f));
    }
  }
  __device__ void pp(const int32_t *list, int n) {
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int s = s0; s < n; s += ds) {
      const int32_t j = list[s];
      const float4 A = __ldg(&a.spA[j]), B = __ldg(&a.spB[j]);
      const FF dx = ff_add({xh, xl}, {-A.x, -B.x});
      const FF dy = ff_add({yh, yl}, {-A.y, -B.y});
      const FF dz = ff_add({zh, zl}, {-A.z, -B.z});
      term(dx, dy, dz, ff_fast(A.w, __ldg(&a.sml[j])), fminf(inv_ro, B.w), true, z4, z4);
    }
  }
  __device__ void nodes(const int32_t *list, int n) {
    for (int s = s0; s < n; s += ds) {
      const Mom32 *m = &a.mom32[list[s]];
      const float4 hi = __ldg(&m->hi), lo = __ldg(&m->lo);
      const FF dx = ff_add({xh, xl}, {-hi.x, -lo.x});
      const FF dy = ff_add({yh, yl}, {-hi.y, -lo.y});
      const FF dz = ff_add({zh, zl}, {-hi.z, -lo.z});
      term(dx, dy, dz, ff_fast(hi.w, lo.w), 0.0f, false, __ldg(&m->q0), __ldg(&m->q1));
    }
  }
};

// Float-float redo of the ill-conditioned targets of one walk (lanes with
// `redo` set), right after it: the same group box, hence the same interaction
// list, walked once for all of them.  With k such targets each takes
// floor(32 / k) lanes that split every batch (lane j + q k takes entries q,
// q + 32 / k, ... for target j); the lanes' float-float sums are added in
// replica order.
__device__ bool refine_group(const WalkArgs &a, const GroupBox &gb, bool redo, int32_t self,
                             int32_t first, int32_t *stack, int32_t *pp, int32_t *nd,
                             int32_t *big, const int64_t *s_bh, int64_t round_limit) {
  const int lane = threadIdx.x & 31;
  const unsigned todo = __ballot_sync(0xffffffffu, redo);
  const int k = __popc(todo);
  if (k == 0) return true;
  const int nrep = 32 / k, rep = lane / k, j = lane - rep * k;
  // lane of the j-th flagged target
  unsigned m = todo;
  for (int q = 0; q < j; ++q) m &= m - 1;
  const int32_t ti = __shfl_sync(0xffffffffu, self, __ffs(m) - 1);
  const bool valid = rep < nrep;
  const float4 A = a.spA[ti], B = a.spB[ti];
  RefineEval ev{a, A.x, A.y, A.z, B.x, B.y, B.z, B.w, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f},
                valid ? rep : 32, nrep};
  if (!traverse(a, gb, first, stack, pp, nd, big, s_bh, round_limit, ev)) return false;
  // a target's own entry is skipped (r = 0)
  for (int q = 1; q < nrep; ++q) {
    const int src = lane < k ? lane + q * k : lane;
    const FF bx = ff_shfl(ev.ax, src), by = ff_shfl(ev.ay, src), bz = ff_shfl(ev.az, src);
    if (lane < k) {
      ev.ax = ff_add(ev.ax, bx);
      ev.ay = ff_add(ev.ay, by);
      ev.az = ff_add(ev.az, bz);
    }
  }
  if (lane < k) {
    const int32_t i = a.idx[ti];
    a.ax[i] = a.G * ((double)ev.ax.h + (double)ev.ax.l);
    a.ay[i] = a.G * ((double)ev.ay.h + (double)ev.ay.l);
    a.az[i] = a.G * ((double)ev.az.h + (double)ev.az.l);
  }
  return true;
}

#ifndef P3T_WALK_MINB_MIXED
#define P3T_WALK_MINB_MIXED 6  // resident blocks per SM asked of the mixed walk
#endif

template <bool MIXED>
__global__ void __launch_bounds__(kWarps * 32, MIXED ? P3T_WALK_MINB_MIXED : 1)
    k_walk(const WalkArgs a) {
  pdl_wait();
  __shared__ int32_t s_pp[kWarps][kPPCap];
  __shared__ int32_t s_nd[kWarps][kNDCap];
  __shared__ int32_t s_big[kWarps][kBigCap];
  __shared__ __align__(16) unsigned char s_stage[kWarps][kStageBytes];
  __shared__ int64_t s_bh[P3T_BITS + 1];
  __shared__ typename BoxOf<MIXED>::type s_box[kWarps];
  if (threadIdx.x <= P3T_BITS) s_bh[threadIdx.x] = a.bh[threadIdx.x];
  __syncthreads();

  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int32_t *stack = a.stack + ((int64_t)blockIdx.x * kWarps + w) * a.stack_cap;
  const int64_t nleaf = *a.d_nleaf;
  const int64_t round_limit = *a.d_nnode + 2;  // a node is pushed at most once per walk
  unsigned npp = 0, npn = 0;

  for (;;) {
    // work unit u: target group u / 2, its first 32 targets (u even) or the
    // rest (u odd; empty for a group of at most 32): half-group units keep
    // the warps' finishing times within one such unit of each other
    int64_t u = 0;
    if (lane == 0) u = atomicAdd(reinterpret_cast<unsigned long long *>(a.cursor), 1ull);
    u = __shfl_sync(0xffffffffu, u, 0);
    const int64_t g = u >> 1;
    if (g >= nleaf) break;
    if (*(volatile int32_t *)&a.st->code != 0) break;
    const TreeNode &G = a.node[a.leaf_list[g]];
    const int32_t gfirst = G.first, gcount = G.count;
    const int32_t t0 = (u & 1) ? gfirst + 32 : gfirst;
    const int32_t t1 = (u & 1) ? gfirst + gcount : min(gfirst + gcount, gfirst + 32);
    if (t0 >= t1) continue;
    GroupBox gb;
    gb.load(G);
    bool ok = true;
    for (int32_t tb = t0; tb < t1 && ok; tb += 32) {
      const int k = min(32, t1 - tb);
      const int nrep = 32 / k, rep = lane / k;
      Target<MIXED> t;
      t.load(a, tb + (lane - rep * k), rep < nrep, rep < nrep ? rep : 0, nrep);
      if constexpr (MIXED) far_box(t, s_box[w]); else far_box64(t, s_box[w]);
      GroupEval<MIXED> ev{a, t, s_stage[w], s_box[w], npp, npn};
      ok = traverse(a, gb, gfirst, stack, s_pp[w], s_nd[w], s_big[w], s_bh, round_limit, ev);
      if (ok) {
        t.reduce(k);
        const bool redo = write_result<MIXED>(a, t);
        if constexpr (MIXED)
          ok = refine_group(a, gb, redo, t.self, gfirst, stack, s_pp[w], s_nd[w], s_big[w],
                            s_bh, round_limit);
      }
    }
    if (!ok) break;
  }
  if (a.counts) {
    // a replica lane that met its target's own entry holds npp below zero:
    // the warp sum is taken modulo 2^32, where a warp's true count fits
    unsigned p = npp, q = npn;
    for (int o = 16; o > 0; o >>= 1) {
      p += __shfl_xor_sync(0xffffffffu, p, o);
      q += __shfl_xor_sync(0xffffffffu, q, o);
    }
    if (lane == 0) {
      atomicAdd(&a.counts[0], (unsigned long long)p);
      atomicAdd(&a.counts[1], (unsigned long long)q);
    }
  }
}

// ---- adjoint of the tree walk (FP64 path) -----------------------------------
// The vector-Jacobian product of the soft force of Eq. softforce as the tree
// gives it, with the tree and the interaction lists held fixed: a second walk
// of the same tree from the same group boxes meets the same lists.  With
// L = sum_i lam_i . a_i (lam_i = s times the caller's velocity adjoint):
//   p-p term a_i += -G m_j K(y) r / r^3, r = x_i - x_j, y = r / r_out,ij:
//     dL/dx_i += J lam_i, dL/dx_j -= J lam_i, dL/dm_j += lam_i . (-G K r / r^3),
//     J = -G m_j (phi I + psi r r^T), phi = K / r^3,
//     psi = K'(y) / (r_out,ij r^4) - 3 K / r^5;
//   node term a_i += G [-M r / r^3 + Q r / r^5 - (5/2) (r.Q.r) r / r^7],
//     r = x_i - c: dL/dx_i += g, dL/dc -= g, with g = grad_r (lam_i . a),
//     and dL/dM, dL/dQ accumulated per node;
// the node adjoints then reach the member particles through M = sum m_k,
// c = sum m_k x_k / M, Q = sum m_k (3 d d^T - d^2 I), d = x_k - c (the
// derivative of Q through c vanishes, as sum m_k d_k = 0).  One warp per
// target group, one lane per target (lanes past the group idle); the
// contributions of a walk's targets to one source or node are added by a
// warp reduction and then to the global sums by FP64 atomics (their order
// follows the walks' order, so the last bits can differ from run to run).
struct VjpOut {
  const double *lx, *ly, *lz;  // velocity adjoints, caller order
  double s;                    // scale (the kick's time step)
  double *gx, *gy, *gz, *gm;   // accumulated position and mass adjoints, caller order
  double *nadj;                // per node: dL/dc (3), dL/dM, dL/dQ (xx yy zz xy xz yz)
};

__device__ __forceinline__ double warp_sum_d(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

struct VjpEval {
  const WalkArgs &a;
  const VjpOut &o;
  void *stage;
  bool valid;
  int32_t self;            // sorted index of the lane's target
  double x, y, z, ro;      // target
  double lx, ly, lz;       // s lam
  double gx, gy, gz;       // dL/dx of the target, this walk
  __device__ void nodes(const int32_t *list, int n) {
    Mom64 *S = reinterpret_cast<Mom64 *>(stage);
    int32_t *ids = reinterpret_cast<int32_t *>(S + 32);
    const int lane = threadIdx.x & 31;
    if (lane < n) {
      S[lane] = a.mom64[list[lane]];
      ids[lane] = list[lane];
    }
    __syncwarp();
    for (int q = 0; q < n; ++q) {
      const Mom64 &m = S[q];
      double c[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
      if (valid) {
        const double rx = x - m.cx, ry = y - m.cy, rz = z - m.cz;
        const double r2 = rx * rx + ry * ry + rz * rz;
        const double ri = rsqrt(r2);
        const double ri2 = ri * ri, ri3 = ri2 * ri, ri5 = ri3 * ri2, ri7 = ri5 * ri2,
                     ri9 = ri7 * ri2;
        const double qx = m.qxx * rx + m.qxy * ry + m.qxz * rz;
        const double qy = m.qxy * rx + m.qyy * ry + m.qyz * rz;
        const double qz = m.qxz * rx + m.qyz * ry + m.qzz * rz;
        const double q2 = rx * qx + ry * qy + rz * qz;           // r.Q.r
        const double lr = lx * rx + ly * ry + lz * rz;           // lam.r
        const double lq = lx * qx + ly * qy + lz * qz;           // lam.Q r
        const double Ql_x = m.qxx * lx + m.qxy * ly + m.qxz * lz;  // Q lam
        const double Ql_y = m.qxy * lx + m.qyy * ly + m.qyz * lz;
        const double Ql_z = m.qxz * lx + m.qyz * ly + m.qzz * lz;
        const double G = a.G;
        // g = grad_r lam.a (a the node term)
        const double cr = G * (3.0 * m.M * lr * ri5 - 5.0 * lq * ri7 + 17.5 * q2 * lr * ri9);
        const double cl = G * (-m.M * ri3 - 2.5 * q2 * ri7);
        const double cQ = G * ri5, cQr = -5.0 * G * lr * ri7;
        const double g0 = cl * lx + cr * rx + cQ * Ql_x + cQr * qx;
        const double g1 = cl * ly + cr * ry + cQ * Ql_y + cQr * qy;
        const double g2 = cl * lz + cr * rz + cQ * Ql_z + cQr * qz;
        gx += g0; gy += g1; gz += g2;
        c[0] = -g0; c[1] = -g1; c[2] = -g2;
        c[3] = -G * lr * ri3;
        // d(lam.a)/dQ per stored component (an off-diagonal one stands for ab and ba)
        const double u = G * ri5, v = -2.5 * G * lr * ri7;
        c[4] = u * lx * rx + v * rx * rx;
        c[5] = u * ly * ry + v * ry * ry;
        c[6] = u * lz * rz + v * rz * rz;
        c[7] = u * (lx * ry + ly * rx) + 2.0 * v * rx * ry;
        c[8] = u * (lx * rz + lz * rx) + 2.0 * v * rx * rz;
        c[9] = u * (ly * rz + lz * ry) + 2.0 * v * ry * rz;
      }
      for (int k = 0; k < 10; ++k) c[k] = warp_sum_d(c[k]);
      if (lane == 0)
        for (int k = 0; k < 10; ++k) atomicAdd(&o.nadj[10 * (int64_t)ids[q] + k], c[k]);
    }
    __syncwarp();
  }
  __device__ void pp(const int32_t *list, int n) {
    double *S = reinterpret_cast<double *>(stage);  // x, y, z, m, ro of 32 sources
    int32_t *ids = reinterpret_cast<int32_t *>(S + 5 * 32);
    const int lane = threadIdx.x & 31;
    if (lane < n) {
      const int32_t j = list[lane];
      S[lane] = a.sx[j]; S[32 + lane] = a.sy[j]; S[64 + lane] = a.sz[j];
      S[96 + lane] = a.sm[j]; S[128 + lane] = a.sro[j];
      ids[lane] = j;
    }
    __syncwarp();
    const double i1mg = 1.0 / (1.0 - a.gamma);
    for (int q = 0; q < n; ++q) {
      double c[4] = {0, 0, 0, 0};
      if (valid && ids[q] != self) {
        const double rx = x - S[q], ry = y - S[32 + q], rz = z - S[64 + q];
        const double mj = S[96 + q];
        const double r2 = rx * rx + ry * ry + rz * rz;
        const double r = sqrt(r2);
        const double roij = fmax(ro, S[128 + q]);
        const double yv = r / roij;
        double K = 0.0, dK = 0.0;
        if (yv >= 1.0) {
          K = 1.0;
        } else if (yv > a.gamma) {
          const double xs = (yv - a.gamma) * i1mg;
          const double x2 = xs * xs, x3 = x2 * xs, us = 1.0 - xs;
          K = x2 * x2 * (35.0 - 84.0 * xs + 70.0 * x2 - 20.0 * x3);
          dK = 140.0 * x3 * us * us * us * i1mg;
        }
        if (K != 0.0 || dK != 0.0) {
          const double r3 = r2 * r, r4 = r2 * r2, r5 = r4 * r;
          const double phi = K / r3, psi = dK / (roij * r4) - 3.0 * K / r5;
          const double lr = lx * rx + ly * ry + lz * rz;
          const double f = -a.G * mj;
          const double j0 = f * (phi * lx + psi * lr * rx);
          const double j1 = f * (phi * ly + psi * lr * ry);
          const double j2 = f * (phi * lz + psi * lr * rz);
          gx += j0; gy += j1; gz += j2;
          c[0] = -j0; c[1] = -j1; c[2] = -j2;
          c[3] = -a.G * phi * lr;
        }
      }
      for (int k = 0; k < 4; ++k) c[k] = warp_sum_d(c[k]);
      if (lane == 0) {
        const int32_t i = a.idx[ids[q]];
        atomicAdd(&o.gx[i], c[0]); atomicAdd(&o.gy[i], c[1]); atomicAdd(&o.gz[i], c[2]);
        atomicAdd(&o.gm[i], c[3]);
      }
    }
    __syncwarp();
  }
};

__global__ void __launch_bounds__(kWarps * 32) k_walk_vjp(const WalkArgs a, const VjpOut o) {
  pdl_wait();
  __shared__ int32_t s_pp[kWarps][kPPCap];
  __shared__ int32_t s_nd[kWarps][kNDCap];
  __shared__ int32_t s_big[kWarps][kBigCap];
  // a batch of 32 FP64 moments (or sources) and their 32 ids
  __shared__ __align__(16) unsigned char s_stage[kWarps][32 * sizeof(Mom64) + 32 * 4];
  __shared__ int64_t s_bh[P3T_BITS + 1];
  if (threadIdx.x <= P3T_BITS) s_bh[threadIdx.x] = a.bh[threadIdx.x];
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int32_t *stack = a.stack + ((int64_t)blockIdx.x * kWarps + w) * a.stack_cap;
  const int64_t ngroup = *a.d_nleaf;
  const int64_t round_limit = *a.d_nnode + 2;
  for (;;) {
    int64_t g = 0;
    if (lane == 0) g = atomicAdd(reinterpret_cast<unsigned long long *>(a.cursor), 1ull);
    g = __shfl_sync(0xffffffffu, g, 0);
    if (g >= ngroup) break;
    if (*(volatile int32_t *)&a.st->code != 0) break;
    const TreeNode &G = a.node[a.leaf_list[g]];
    GroupBox gb;
    gb.load(G);
    bool ok = true;
    for (int32_t tb = G.first; tb < G.first + G.count && ok; tb += 32) {
      const bool valid = tb + lane < G.first + G.count;
      VjpEval ev{a, o, s_stage[w], valid, tb + lane, 0, 0, 0, 1, 0, 0, 0, 0, 0, 0};
      if (valid) {
        const int32_t t = tb + lane, i = a.idx[t];
        ev.x = a.sx[t]; ev.y = a.sy[t]; ev.z = a.sz[t]; ev.ro = a.sro[t];
        ev.lx = o.s * o.lx[i]; ev.ly = o.s * o.ly[i]; ev.lz = o.s * o.lz[i];
      }
      ok = traverse(a, gb, G.first, stack, s_pp[w], s_nd[w], s_big[w], s_bh, round_limit, ev);
      if (ok && valid) {
        const int32_t i = a.idx[tb + lane];
        atomicAdd(&o.gx[i], ev.gx); atomicAdd(&o.gy[i], ev.gy); atomicAdd(&o.gz[i], ev.gz);
      }
    }
    if (!ok) break;
  }
}

// node adjoints to the member particles: each particle climbs from its leaf
// to the root (fixed order)
__global__ void k_node_adjoint(const int64_t *d_nleaf, const int32_t *leaf_list,
                               const TreeNode *node, const Mom64 *mom, const double *nadj,
                               const double *sx, const double *sy, const double *sz,
                               const double *sm, const int32_t *idx, double *gx, double *gy,
                               double *gz, double *gm) {
  pdl_wait();
  const int64_t nleaf = *d_nleaf;
  for (int64_t b = blockIdx.x; b < nleaf; b += gridDim.x) {
    const TreeNode &L = node[leaf_list[b]];
    for (int32_t k = L.first + threadIdx.x; k < L.first + L.count; k += blockDim.x) {
      const double xk = sx[k], yk = sy[k], zk = sz[k], mk = sm[k];
      double ax = 0.0, ay = 0.0, az = 0.0, am = 0.0;
      for (int32_t n = leaf_list[b]; n >= 0; n = node[n].parent) {
        const double *A = nadj + 10 * (int64_t)n;
        const Mom64 &M = mom[n];
        const double dx = xk - M.cx, dy = yk - M.cy, dz = zk - M.cz;
        const double d2 = dx * dx + dy * dy + dz * dz;
        const double tr = A[4] + A[5] + A[6];
        // dQ/dx_k and dQ/dm_k with the stored components (xx yy zz xy xz yz)
        ax += mk / M.M * A[0] + mk * (6.0 * A[4] * dx - 2.0 * tr * dx + 3.0 * (A[7] * dy + A[8] * dz));
        ay += mk / M.M * A[1] + mk * (6.0 * A[5] * dy - 2.0 * tr * dy + 3.0 * (A[7] * dx + A[9] * dz));
        az += mk / M.M * A[2] + mk * (6.0 * A[6] * dz - 2.0 * tr * dz + 3.0 * (A[8] * dx + A[9] * dy));
        am += A[3] + (A[0] * dx + A[1] * dy + A[2] * dz) / M.M +
              A[4] * (3.0 * dx * dx - d2) + A[5] * (3.0 * dy * dy - d2) +
              A[6] * (3.0 * dz * dz - d2) +
              3.0 * (A[7] * dx * dy + A[8] * dx * dz + A[9] * dy * dz);
      }
      const int32_t i = idx[k];
      gx[i] += ax; gy[i] += ay; gz[i] += az; gm[i] += am;
    }
  }
}

__global__ void k_walk_prep(int64_t *cursor, unsigned long long *cand_count,
                            unsigned long long *counts) {
  pdl_wait();
  *cursor = 0;
  *cand_count = 0ull;
  if (counts) { counts[0] = 0ull; counts[1] = 0ull; }
}

// candidates found -> device status (for growth on the host) and clamped count
__global__ void k_walk_post(int64_t *cnt, int64_t cand_cap, DevStatus *st) {
  pdl_wait();
  const int64_t nc = cnt[8];
  st->cand_need = nc;
  if (nc > cand_cap) dev_fail(st, P3T_ERR_CAPACITY, 42, nc);
  cnt[9] = nc < cand_cap ? nc : cand_cap;
}

// T M^2 >= 2^K for T < 2^49, M < 2^53, K >= 0: the product formed exactly in
// three 64-bit limbs and compared with the power of two
bool prod_sq_ge_pow2(uint64_t T, uint64_t M, int K) {
  const unsigned __int128 a = (unsigned __int128)T * M;  // < 2^102
  const unsigned __int128 p0 = (unsigned __int128)(uint64_t)a * M;
  const unsigned __int128 p1 = (unsigned __int128)(uint64_t)(a >> 64) * M;
  const unsigned __int128 mid = (p0 >> 64) + (unsigned __int128)(uint64_t)p1;
  const uint64_t w[3] = {(uint64_t)p0, (uint64_t)mid,
                         (uint64_t)(p1 >> 64) + (uint64_t)(mid >> 64)};
  if (K >= 192) return false;
  for (int q = 2; q > K / 64; --q)
    if (w[q]) return true;
  return (w[K / 64] >> (K % 64)) != 0;
}

// Barnes-Hut threshold of a level: the smallest integer T with T theta^2 >=
// side^2, side = 2^(22 - l) half cells, so that the integer test d^2 < T is
// exactly side^2 > theta^2 d^2.  theta = M 2^E with M odd, so the condition
// is T M^2 >= 2^K, K = 2 (22 - l) - 2E.  The FP64 quotient side^2 / theta^2
// gives T to within one, and the exact product settles it.  Thresholds
// beyond 2^47 (above every squared distance on the grid, < 3 * 2^44) are
// clamped to 2^47; theta = 0 opens every node.
int64_t bh_threshold(double theta, int level) {
  const int64_t cap = (int64_t)1 << 47;
  if (!(theta > 0.0)) return cap;
  int e;
  uint64_t M = (uint64_t)ldexp(frexp(theta, &e), 53);
  int E = e - 53;
  while (!(M & 1u)) { M >>= 1; ++E; }
  const int K = 2 * (P3T_BITS + 1 - level) - 2 * E;
  if (K < 0) return 1;
  const double X = ldexp(1.0, 2 * (P3T_BITS + 1 - level)) / (theta * theta);
  if (X > (double)cap + 4.0) return cap;
  uint64_t T = (uint64_t)ceil(X);
  if (T < 1) T = 1;
  while (T > 1 && prod_sq_ge_pow2(T - 1, M, K)) --T;
  while (!prod_sq_ge_pow2(T, M, K)) ++T;
  return (int64_t)T < cap ? (int64_t)T : cap;
}

}  // namespace

// blocks of 4 warps resident per SM: the mixed walk is compiled for 6 (80
// registers; 30.5 KB of shared memory a block)
int p3t_walk_blocks_per_sm() { return P3T_WALK_MINB_MIXED; }

// the walk's arguments for the tree of context c built from particles p
static WalkArgs walk_args(p3t_ctx *c, const p3t_particles *p) {
  WalkArgs a;
  a.node = c->node; a.mom64 = c->mom64; a.mom32 = c->mom32;
  a.leaf_list = c->group_list; a.d_nleaf = &c->counters[15]; a.d_nnode = &c->counters[3];
  a.sx = c->sx; a.sy = c->sy; a.sz = c->sz; a.sm = c->sm; a.sro = c->sro; a.srs = c->srs;
  a.spA = c->spA; a.spB = c->spB; a.srs32 = c->srs32; a.sml = c->sml;
  a.idx = c->idx;
  a.ax = a.ay = a.az = nullptr;
  a.stack = c->walk_stack; a.stack_cap = c->stack_cap;
  a.cand_i = c->cand_i; a.cand_j = c->cand_j; a.cand_cap = c->cand_cap;
  a.cand_count = reinterpret_cast<unsigned long long *>(&c->counters[8]);
  a.counts = nullptr;
  a.cursor = &c->counters[12];
  a.st = c->status;
  a.seg = SegView{c->seg_off, (int)c->nseg, p->n};
  a.refine_cf = 32.0f;
  a.G = c->prm.G;
  a.gamma = c->prm.gamma;
  a.inv1mg = 1.0 / (1.0 - c->prm.gamma);
  a.inv1mg_f = (float)(1.0 / (1.0 - c->prm.gamma));
  a.mgi_f = (float)(-c->prm.gamma / (1.0 - c->prm.gamma));
  for (int l = 0; l <= P3T_BITS; ++l) a.bh[l] = bh_threshold(c->prm.theta, l);
  return a;
}

int p3t_run_soft_force_vjp_tree(p3t_ctx *c, const p3t_particles *p, double s,
                                const double *lx, const double *ly, const double *lz,
                                double *gx, double *gy, double *gz, double *gm,
                                cudaStream_t st) {
  WalkArgs a = walk_args(c, p);
  VjpOut o{lx, ly, lz, s, gx, gy, gz, gm, c->nadj};
  P3T_CUDA_TRY(cudaMemsetAsync(c->nadj, 0, sizeof(double) * 10 * c->node_cap, st));
  P3T_CUDA_TRY(cudaMemsetAsync(a.cursor, 0, sizeof(int64_t), st));
  const unsigned blocks = (unsigned)(c->walk_warps / kWarps);
  pdl_launch(k_walk_vjp, dim3(blocks), dim3(kWarps * 32), 0, st, a, o);
  pdl_launch(k_node_adjoint, dim3((unsigned)(c->num_sms * 8)), dim3(128), 0, st, 
      &c->counters[2], c->leaf_list, c->node, c->mom64, c->nadj, c->sx, c->sy, c->sz, c->sm,
      c->idx, gx, gy, gz, gm);
  p3t_note_launches(3);
  return cudaGetLastError() == cudaSuccess ? P3T_OK : P3T_ERR_CUDA;
}

int p3t_run_soft_force(p3t_ctx *c, const p3t_particles *p, double *ax,
                       double *ay, double *az, uint64_t *counts,
                       cudaStream_t s) {
  WalkArgs a;
  a.node = c->node; a.mom64 = c->mom64; a.mom32 = c->mom32;
  a.leaf_list = c->group_list; a.d_nleaf = &c->counters[15]; a.d_nnode = &c->counters[3];
  a.sx = c->sx; a.sy = c->sy; a.sz = c->sz; a.sm = c->sm; a.sro = c->sro; a.srs = c->srs;
  a.spA = c->spA; a.spB = c->spB; a.srs32 = c->srs32; a.sml = c->sml;
  a.idx = c->idx;
  a.ax = ax; a.ay = ay; a.az = az;
  a.stack = c->walk_stack; a.stack_cap = c->stack_cap;
  a.cand_i = c->cand_i; a.cand_j = c->cand_j; a.cand_cap = c->cand_cap;
  a.cand_count = reinterpret_cast<unsigned long long *>(&c->counters[8]);
  a.counts = reinterpret_cast<unsigned long long *>(counts);
  a.cursor = &c->counters[12];
  a.st = c->status;
  a.seg = SegView{c->seg_off, (int)c->nseg, p->n};
  a.refine_cf = 32.0f;
  a.G = c->prm.G;
  a.gamma = c->prm.gamma;
  a.inv1mg = 1.0 / (1.0 - c->prm.gamma);
  a.inv1mg_f = (float)(1.0 / (1.0 - c->prm.gamma));
  a.mgi_f = (float)(-c->prm.gamma / (1.0 - c->prm.gamma));
  // Barnes-Hut thresholds per level, ceil((2^(22-l))^2 / theta^2) (half units)
  for (int l = 0; l <= P3T_BITS; ++l) a.bh[l] = bh_threshold(c->prm.theta, l);
  pdl_launch(k_walk_prep, dim3(1), dim3(1), 0, s, a.cursor, a.cand_count, a.counts);
  unsigned blocks = (unsigned)(c->walk_warps / kWarps);
  if (c->walk_bps > 0 && (int64_t)c->num_sms * c->walk_bps < (int64_t)blocks)
    blocks = (unsigned)(c->num_sms * c->walk_bps);
  if (c->prm.precision == P3T_MIXED) {
    // one target per lane (or several lanes per target): two targets per
    // lane (a 64-target group walked once) was measured slower than two
    // walks of 32 (register pressure, longer chains)
    pdl_launch(k_walk<true>, dim3(blocks), dim3(kWarps * 32), 0, s, a);
  } else {
    pdl_launch(k_walk<false>, dim3(blocks), dim3(kWarps * 32), 0, s, a);
  }
  pdl_launch(k_walk_post, dim3(1), dim3(1), 0, s, c->counters, c->cand_cap, c->status);
  p3t_note_launches(3);
  (void)p;
  return cudaGetLastError() == cudaSuccess ? P3T_OK : P3T_ERR_CUDA;
}

// persistent walk warps for a context of up to n particles: 6 blocks per SM,
// fewer for small systems (a block for every 256 particles: a group walk
// takes a warp, and a group holds tens of particles)
int64_t p3t_walk_warps(int num_sms, int64_t n) {
  int64_t blocks = (int64_t)num_sms * p3t_walk_blocks_per_sm();
  const int64_t want = n / 256 + 1;
  if (want < blocks) blocks = want;
  return blocks * kWarps;
}

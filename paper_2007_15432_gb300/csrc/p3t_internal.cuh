// Internal declarations of libp3t (CUDA, sm_103a).  Not part of the C ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "p3t.h"

#define P3T_BITS 21           // bits per axis of the Morton grid
#define P3T_QMAX (1 << P3T_BITS)
#define P3T_KMAX 40           // deepest Hermite block level: dt / 2^40
#define P3T_NSM_BLOCKS 8      // resident blocks per SM assumed for grid sizing
#define P3T_MAX_SEGMENTS 4096 // independent systems sharing one context

// ---- segments: the segment of a position, its range --------------------------
// ---- float-float arithmetic (pairs hi + lo of floats, ~2^-44 relative) ------
// Dekker's and Knuth's error-free transformations with fmaf for the product
// error: FP32 instructions only, which on this part cost 1/64 of an FP64 one.
struct FF {
  float h, l;
};
__device__ __forceinline__ FF ff_fast(float a, float b) {  // |a| >= |b|
  const float s = a + b;
  return {s, b - (s - a)};
}
__device__ __forceinline__ FF ff_add(FF a, FF b) {
  const float s = a.h + b.h;
  const float bb = s - a.h;
  const float e = (a.h - (s - bb)) + (b.h - bb) + (a.l + b.l);
  return ff_fast(s, e);
}
__device__ __forceinline__ FF ff_mul(FF a, FF b) {
  const float p = a.h * b.h;
  float e = fmaf(a.h, b.h, -p);
  e = fmaf(a.h, b.l, fmaf(a.l, b.h, e));
  return ff_fast(p, e);
}
__device__ __forceinline__ FF ff_mulf(FF a, float b) {
  const float p = a.h * b;
  const float e = fmaf(a.l, b, fmaf(a.h, b, -p));
  return ff_fast(p, e);
}
__device__ __forceinline__ FF ff_neg(FF a) { return {-a.h, -a.l}; }
// a / b: the FP32 quotient and one correction from the float-float residual
__device__ __forceinline__ FF ff_div(FF a, FF b) {
  const float q1 = a.h / b.h;
  const FF r = ff_add(a, ff_neg(ff_mulf(b, q1)));
  return ff_fast(q1, r.h / b.h);
}

// 1 / sqrt(r2): the FP32 estimate and one Newton step y (3 - r2 y^2) / 2 with
// the residual 1 - r2 y^2 formed in float-float
__device__ __forceinline__ FF ff_rsqrt(FF r2) {
  const float y = rsqrtf(r2.h);
  const float p = y * y;
  const FF yy{p, fmaf(y, y, -p)};
  const FF t = ff_mul(r2, yy);
  const float d = ((1.0f - t.h) - t.l);
  return ff_fast(y, 0.5f * y * d);
}

// ---- packed FP32 pairs ----------------------------------------------------------
// a pair of floats in one 64-bit register (low half: the first value); the
// .f32x2 instructions round each half as the scalar instruction would
typedef unsigned long long f2;
__device__ __forceinline__ f2 f2_pk(float a, float b) {
  f2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ float f2_lo(f2 v) {
  return __uint_as_float((unsigned)(v & 0xffffffffull));
}
__device__ __forceinline__ float f2_hi(f2 v) { return __uint_as_float((unsigned)(v >> 32)); }
__device__ __forceinline__ f2 add2(f2 a, f2 b) {
  f2 d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2 sub2(f2 a, f2 b) {
  f2 d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2 mul2(f2 a, f2 b) {
  f2 d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) {
  f2 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ f2 f2_dup(float a) { return f2_pk(a, a); }

struct SegView {
  const int64_t *off;  // nseg + 1 offsets (unused when nseg == 1)
  int nseg;
  int64_t n;
};
__device__ __forceinline__ int seg_of(const SegView &v, int64_t i) {
  int lo = 0, hi = v.nseg - 1;  // largest d with off[d] <= i
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (v.off[mid] <= i) lo = mid; else hi = mid - 1;
  }
  return lo;
}
__device__ __forceinline__ int64_t seg_lo(const SegView &v, int d) {
  return v.nseg == 1 ? 0 : v.off[d];
}
__device__ __forceinline__ int64_t seg_hi(const SegView &v, int d) {
  return v.nseg == 1 ? v.n : v.off[d + 1];
}
__device__ __forceinline__ int seg_at(const SegView &v, int64_t i) {
  return v.nseg == 1 ? 0 : seg_of(v, i);
}

// ---- device-side status (sticky first error + requested size) ------------
struct DevStatus {
  int32_t code;
  int32_t where;       // id of the kernel that recorded it (diagnostics)
  int64_t required;    // size asked for by a capacity error
  int64_t cand_need;   // neighbour candidates found by the last walk
  int64_t walk_stack_need;
};

__device__ __forceinline__ void dev_fail(DevStatus *st, int code, int where,
                                         int64_t required) {
  if (atomicCAS(&st->code, 0, code) == 0) st->where = where;
  if (required > 0)
    atomicMax(reinterpret_cast<unsigned long long *>(&st->required),
              (unsigned long long)required);
}

// ---- tree node, walk record (64 bytes, breadth-first order) ---------------
// Integer geometry on the 21-bit grid: quantised tight box of the members
// (qlo, qhi), cell centre in half units (c2), search reach R (grid units).
struct __align__(16) TreeNode {
  int32_t qlo[3];
  int32_t R;
  int32_t qhi[3];
  int32_t level;
  int32_t c2[3];
  int32_t parent;
  int32_t child0;   // first child (children contiguous), -1 for a leaf
  int32_t nchild;   // 0 for a leaf
  int32_t first;    // first member in sorted order
  int32_t count;    // number of members
};

// multipole moments in FP64: centre of mass, mass, traceless quadrupole
struct __align__(16) Mom64 {
  double cx, cy, cz, M;
  double qxx, qyy, qzz, qxy;
  double qxz, qyz, pad0, pad1;
};

// the same for the mixed path: centre of mass as float-float, Q in FP32
struct __align__(16) Mom32 {
  float4 hi;  // cx_hi, cy_hi, cz_hi, M
  float4 lo;  // cx_lo, cy_lo, cz_lo, M - (float)M
  float4 q0;  // qxx, qyy, qzz, qxy
  float4 q1;  // qxz, qyz, 0, 0
};

// ---- the context ---------------------------------------------------------
struct p3t_ctx {
  int device = 0;
  int num_sms = 0;
  p3t_params prm{};
  int64_t cap = 0;        // particle capacity
  int64_t node_cap = 0;   // node capacity
  int64_t cand_cap = 0;   // neighbour-candidate capacity (pairs)
  int64_t walk_warps = 0; // resident warps of the walk kernel
  // independent particle systems sharing the arrays (segments): nseg > 1 when
  // set by p3t_set_segments; one segment is [0, n) and reads no table
  int64_t nseg = 1;
  int64_t *seg_off = nullptr;      // device, nseg + 1 offsets
  int64_t *seg_off_h = nullptr;    // host copy
  int32_t *seg_nb = nullptr;       // device, radial bins of each segment (cut-offs)
  int32_t *seg_base = nullptr;     //   and the first global bin of each
  double *seg_l = nullptr;         //   log R_min, log R_max of each (2 nseg)
  unsigned long long *scan_state = nullptr;  // the single-pass scan's tile words
  int64_t scan_words = 0;
  double *dpart = nullptr; // partial sums of the all-pairs kernels (allocated
  int64_t dpart_cap = 0;   //   on their first call; size independent of n)
  int32_t *dcnt = nullptr; // their per-tile arrival counters (zero between calls)
  int64_t dcnt_cap = 0;
  int64_t stack_cap = 0;  // walk stack entries per warp
  // limits of the bounded device loops and the per-member Hermite step
  // record (p3t_set_diag)
  int64_t hermite_limit = (int64_t)1 << 24;  // block times per cluster and hard step
  int64_t poll_limit = (int64_t)1 << 22;     // polls of a waiting scan tile
  int32_t *hermite_rec = nullptr;            // caller's int32[n] or null
  // launch shapes (p3t_set_tuning): largest cluster integrated by one warp,
  // walk blocks per SM
  int hwarp_max = 8;
  int walk_bps = 0;  // 0: as many as fit
  int64_t last_n = -1;    // n of the last tree build
  bool have_tree = false;
  bool have_cand = false;

  DevStatus *status = nullptr;
  // root box {x0, y0, z0, L} and scalar counters
  double *box = nullptr;
  unsigned long long *box_bits = nullptr;  // ordered-bits min/max workspace [6]
  int64_t *counters = nullptr;             // misc device counters [64] (32..53: tree level offsets)

  // sort
  uint64_t *keys = nullptr, *keys_alt = nullptr;
  int32_t *idx = nullptr, *idx_alt = nullptr;
  uint32_t *radix_hist = nullptr;
  int64_t radix_hist_cap = 0;

  // sorted particles (FP64 and mixed packings)
  double *sx = nullptr, *sy = nullptr, *sz = nullptr, *sm = nullptr;
  double *pack = nullptr;  // (x, y, z, m, r_out, r_search) per particle, caller order
  double *sro = nullptr, *srs = nullptr;
  int32_t *sq = nullptr;                   // 3 * cap quantised coordinates
  float4 *spA = nullptr, *spB = nullptr;   // {x_hi,y_hi,z_hi,m}, {x_lo,y_lo,z_lo,1/r_out}
  float *srs32 = nullptr;                  // r_search^2 x 1.00001 in FP32 (walk's candidate test)
  float *sml = nullptr;                    // m - (float)m: the mass as float-float with spA.w

  // tree build scratch (per particle)
  int8_t *lp = nullptr, *lv = nullptr;     // lcp with predecessor, leaf level
  int32_t *ncount = nullptr;               // nodes started by particle
  int64_t *nstart = nullptr;               // exclusive scan of ncount
  // nodes (preorder scratch and breadth-first result)
  int32_t *pre_first = nullptr, *pre_count = nullptr, *pre_level = nullptr;
  uint64_t *lvl_keys = nullptr, *lvl_keys_alt = nullptr;
  int32_t *bfs2pre = nullptr, *bfs2pre_alt = nullptr, *pre2bfs = nullptr;
  TreeNode *node = nullptr;
  Mom64 *mom64 = nullptr;
  Mom32 *mom32 = nullptr;
  double *nrs = nullptr;                   // max r_search per node
  int32_t *node_done = nullptr;            // bottom-up arrival counters
  int32_t *leaf_list = nullptr;            // leaves (BFS ids) in key order
  int32_t *group_list = nullptr;           // target groups (BFS ids) in key order
  int32_t *node_flag = nullptr;            // per preorder node: bit 0 leaf, bit 1 target group
  int64_t *flag_pos = nullptr;             // their prefix counts (leaves bits 0-30, groups from 31)
  int64_t *bh_table = nullptr;             // Barnes-Hut thresholds per level

  // walk
  int32_t *walk_stack = nullptr;
  int32_t *cand_i = nullptr, *cand_j = nullptr;  // sorted indices
  double *acc_sorted = nullptr;            // 3 * cap, sorted order

  // neighbours and clusters
  int32_t *cand_keep = nullptr;
  int32_t *deg = nullptr, *fill = nullptr;
  int32_t *parent = nullptr, *label = nullptr, *csize = nullptr;
  int32_t *flag = nullptr;
  int64_t *pos = nullptr;
  int32_t *singles = nullptr, *cl_mem = nullptr;
  int64_t *cl_off = nullptr;
  int64_t *cl_counts = nullptr;            // [4]
  uint64_t *mkeys = nullptr, *mkeys_alt = nullptr;
  int32_t *mvals = nullptr, *mvals_alt = nullptr;

  // hard step workspace (per cluster member, clusters of more than 128)
  double *hw = nullptr;                    // 33 * cap doubles
  int64_t *ht = nullptr;                   // time in units of dt / 2^40
  int32_t *hl = nullptr;                   // 6 * cap: level, list, sets, partner, flags
  unsigned long long *hsteps = nullptr;    // device counter
  int64_t *hcursor = nullptr;              // [5] cluster cursors of the three Hermite kernels,
                                           // then the lengths of the two lists below
  int32_t *hlist = nullptr;                // clusters of the four-warp kernel, then (from
                                           // hlist_cap on) those of the workspace kernel
  int64_t hlist_cap = 0;

  // composites of colliding particles, from the hard step to the merge
  unsigned long long *coll_ctr = nullptr;  // (records << 32) | entries
  int4 *coll_ent = nullptr;                // cap entries {particle, lowest member, lo, hi}
  int4 *coll_rec = nullptr;                // cap / 2 + 1 records {label, first, count, 0}
  double *coll_rec_e = nullptr;            // dissipation per record
  double *coll_esoft = nullptr;            // kick dissipation per entry
  int32_t *coll_slot = nullptr;            // particle -> entry or -1 (cap)

  // energy
  double *epart = nullptr;                 // per-block partial sums

  // adjoint of the tree walk: per node dL/dc, dL/dM, dL/dQ (allocated on
  // the first call, node_cap entries of 10)
  double *nadj = nullptr;
  int64_t nadj_cap = 0;
  // adjoint of the hard part: the cluster members' adjoints (6 per member,
  // allocated on the first call, cap entries)
  double *hadj = nullptr;
  int64_t hadj_cap = 0;

  // auxiliary streams and events for work that can overlap inside a call
  cudaStream_t aux[2] = {nullptr, nullptr};
  cudaEvent_t ev_fork = nullptr, ev_join[2] = {nullptr, nullptr};
  // the pending-collision count read without a stream synchronisation:
  // pinned host word, the event after its copy, and whether a copy is queued
  unsigned long long *coll_pin = nullptr;
  cudaEvent_t ev_coll = nullptr;
  bool coll_queued = false;
};

// ---- helpers -------------------------------------------------------------
// kernels launched by the library in this process (diagnostics)
void p3t_note_launches(int64_t k);

// ---- programmatic dependent launch ------------------------------------------
// A kernel launched with pdl_launch may be scheduled while its predecessor on
// the stream is still finishing (its blocks are dispatched as the
// predecessor's last blocks exit, the launch latency hidden); it calls
// pdl_wait() before anything else, which returns once the predecessor has
// completed and its writes are visible.  Launched the ordinary way, pdl_wait()
// returns at once.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
template <typename... KArgs, typename... Args>
inline cudaError_t pdl_launch(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                              cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

#define P3T_CUDA_TRY(x)                      \
  do {                                       \
    cudaError_t e_ = (x);                    \
    if (e_ != cudaSuccess) return P3T_ERR_CUDA; \
  } while (0)

static inline int64_t p3t_grid(int64_t n, int block, int64_t max_blocks) {
  int64_t g = (n + block - 1) / block;
  if (g < 1) g = 1;
  if (g > max_blocks) g = max_blocks;
  return g;
}

// ---- primitives (primitives.cu) ------------------------------------------
// Exclusive scan of n (device count *d_n, at most n_cap) non-negative int32
// values into int64; *d_total receives the sum.  Deterministic (one pass,
// decoupled look-back).  state: p3t_scan_state_words(n_cap) words, zero
// before the first call (the scan leaves them zero).
int64_t p3t_scan_state_words(int64_t n_cap);
// poll_limit: polls a tile makes for its predecessors' sums before it gives
// up (P3T_ERR_TIMEOUT recorded, the silent tiles counted as zero).
int p3t_scan_i32_to_i64(const int32_t *in, int64_t *out, const int64_t *d_n,
                        int64_t n_cap, int64_t *d_total, unsigned long long *state,
                        int64_t state_words, DevStatus *st, int64_t poll_limit,
                        cudaStream_t s);
// The same scan of inputs that each hold a 0/1 flag in bit 0 and a
// non-negative value in bits 1-31: out and *d_total hold the prefix count of
// the flag in bits 0-30 and the prefix sum of the values from bit 31 up (each
// sum below 2^31).
int p3t_scan_flag_pairs(const int32_t *in, int64_t *out, const int64_t *d_n, int64_t n_cap,
                        int64_t *d_total, unsigned long long *state, int64_t state_words,
                        DevStatus *st, int64_t poll_limit, cudaStream_t s);
// Stable LSD radix sort of (key, val) on bits [begin_bit, end_bit), n from
// device memory (at most n_cap).  Ping-pongs between the two buffers; on
// return *keys / *vals point at the sorted data.
int p3t_radix_sort(uint64_t **keys, int32_t **vals, uint64_t **keys_alt,
                   int32_t **vals_alt, const int64_t *d_n, int64_t n_cap,
                   int begin_bit, int end_bit, uint32_t *hist,
                   int64_t hist_cap, cudaStream_t s);
int64_t p3t_radix_hist_entries(int64_t n_cap);

// ---- stages (tree.cu, walk.cu, neighbours.cu, hard.cu) -------------------
int p3t_run_cutoffs(p3t_ctx *c, p3t_particles *p, cudaStream_t s);
int p3t_run_build_tree(p3t_ctx *c, const p3t_particles *p, cudaStream_t s);
int p3t_run_tree_stats(p3t_ctx *c, cudaStream_t s);
int p3t_run_soft_force(p3t_ctx *c, const p3t_particles *p, double *ax,
                       double *ay, double *az, uint64_t *counts,
                       cudaStream_t s);
int p3t_run_neighbours(p3t_ctx *c, const p3t_particles *p, int64_t *nb_off,
                       int32_t *nb_idx, int64_t nb_cap, cudaStream_t s);
int p3t_run_hard_step(p3t_ctx *c, p3t_particles *p, const p3t_clusters *cl,
                      double dt, uint64_t *n_steps, cudaStream_t s);
int p3t_run_kick(p3t_ctx *c, p3t_particles *p, const double *ax,
                 const double *ay, const double *az, double h, cudaStream_t s);
int p3t_run_energy(p3t_ctx *c, const p3t_particles *p, double *out,
                   cudaStream_t s);
int p3t_run_merge(p3t_ctx *c, p3t_particles *p, int32_t *new_index, double *e_disp,
                  int64_t *n_merged, cudaStream_t s);
int64_t p3t_direct_part_doubles(const p3t_ctx *c);
int64_t p3t_direct_tile_counters(const p3t_ctx *c);
int p3t_run_kepler_drift(p3t_ctx *c, p3t_particles *p, double dt, cudaStream_t s);
int p3t_run_soft_force_direct(p3t_ctx *c, const p3t_particles *p, double *ax, double *ay,
                              double *az, cudaStream_t s);
int p3t_run_soft_force_vjp(p3t_ctx *c, const p3t_particles *p, double h, const double *lx,
                           const double *ly, const double *lz, double *gx, double *gy,
                           double *gz, double *gm, cudaStream_t s);
int p3t_run_kepler_vjp(p3t_ctx *c, const p3t_particles *p, double dt, double *lx, double *ly,
                       double *lz, double *lvx, double *lvy, double *lvz, cudaStream_t s);
int p3t_run_hard_step_vjp(p3t_ctx *c, const p3t_particles *p, const p3t_clusters *cl, double dt,
                          double *lx, double *ly, double *lz, double *lvx, double *lvy,
                          double *lvz, double *gm, cudaStream_t s);
int p3t_run_soft_force_vjp_tree(p3t_ctx *c, const p3t_particles *p, double s,
                                const double *lx, const double *ly, const double *lz,
                                double *gx, double *gy, double *gz, double *gm,
                                cudaStream_t st);

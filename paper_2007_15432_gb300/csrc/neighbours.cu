// Soft step: neighbour lists and neighbour clusters
// (Sec. 2.3).  Compiled with -fmad=false: the neighbour predicate is decided
// in FP64 with a fixed evaluation order so that membership is bit-exact.
#include "p3t_internal.cuh"

namespace {

constexpr int kBlock = 256;
constexpr int64_t kUFLimit = 1 << 26;  // bound on union-find retries per edge

// Sec. 2.3: candidate j of i (r_ij < max(r_search,i, r_search,j)) stays a
// neighbour iff the closest approach of the linear relative motion over
// [0, dt] (Eq. rsearch1 with the clamped t_min) is within R~s,2 r_out,ij, or
// v_ij < R~s,3 a_ij dt/2 with a_ij = G (m_i + m_j) / r_ij^2.
__device__ __forceinline__ bool neighbour_pair(int32_t i, int32_t j,
                                               const p3t_particles &p,
                                               const p3t_params &prm) {
  const double rx = p.x[i] - p.x[j], ry = p.y[i] - p.y[j], rz = p.z[i] - p.z[j];
  const double r2 = rx * rx + ry * ry + rz * rz;
  const double rs = fmax(p.r_search[i], p.r_search[j]);
  if (!(r2 < rs * rs)) return false;
  const double ux = p.vx[i] - p.vx[j], uy = p.vy[i] - p.vy[j], uz = p.vz[i] - p.vz[j];
  const double v2 = ux * ux + uy * uy + uz * uz;
  const double rv = rx * ux + ry * uy + rz * uz;
  double t = 0.0;
  if (v2 > 0.0) {
    t = -rv / v2;
    if (t < 0.0) t = 0.0;
    if (t >= prm.dt_soft) t = prm.dt_soft;
  }
  const double dx = rx + ux * t, dy = ry + uy * t, dz = rz + uz * t;
  const double d2 = dx * dx + dy * dy + dz * dz;
  const double lim = prm.rs2 * fmax(p.r_out[i], p.r_out[j]);
  if (d2 <= lim * lim) return true;
  const double a = prm.G * (p.m[i] + p.m[j]) / r2;
  const double w = prm.rs3 * a * prm.dt_soft * 0.5;
  return v2 < w * w;
}

__global__ void k_nb_filter(const int64_t *d_ncand, const int32_t *cand_i,
                            const int32_t *cand_j, const int32_t *idx,
                            const p3t_particles p, const p3t_params prm,
                            int32_t *keep, int32_t *deg, const DevStatus *st) {
  pdl_wait();
  if (st->code != 0) return;
  const int64_t nc = *d_ncand;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nc;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int32_t i = idx[cand_i[k]], j = idx[cand_j[k]];
    const bool ok = neighbour_pair(i, j, p, prm);
    keep[k] = ok ? 1 : 0;
    if (ok) atomicAdd(&deg[i], 1);
  }
}

__global__ void k_nb_check(const int64_t *nb_total, int64_t nb_cap, DevStatus *st) {
  pdl_wait();
  if (*nb_total > nb_cap) dev_fail(st, P3T_ERR_CAPACITY, 50, *nb_total);
}

__global__ void k_nb_fill(const int64_t *d_ncand, const int32_t *cand_i,
                          const int32_t *cand_j, const int32_t *idx,
                          const int32_t *keep, const int64_t *nb_off,
                          int32_t *fill, int32_t *nb_idx, const DevStatus *st) {
  pdl_wait();
  if (st->code != 0) return;
  const int64_t nc = *d_ncand;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nc;
       k += (int64_t)gridDim.x * blockDim.x) {
    if (!keep[k]) continue;
    const int32_t i = idx[cand_i[k]], j = idx[cand_j[k]];
    const int32_t q = atomicAdd(&fill[i], 1);
    nb_idx[nb_off[i] + q] = j;
  }
}

// rows are short (<n_b> << 1 in the paper's runs): insertion sort per row
__global__ void k_nb_sort_rows(int64_t n, const int64_t *nb_off, int32_t *nb_idx,
                               const DevStatus *st) {
  pdl_wait();
  if (st->code != 0) return;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = nb_off[i], e = nb_off[i + 1];
    for (int64_t u = b + 1; u < e; ++u) {
      const int32_t v = nb_idx[u];
      int64_t w = u - 1;
      while (w >= b && nb_idx[w] > v) { nb_idx[w + 1] = nb_idx[w]; --w; }
      nb_idx[w + 1] = v;
    }
  }
}

// ---- union-find: a root is the smallest index of its tree -----------------
__device__ __forceinline__ int32_t uf_find(const int32_t *parent, int32_t x) {
  int32_t p = __ldcg(&parent[x]);
  int64_t guard = 0;
  while (p != x && guard++ < kUFLimit) { x = p; p = __ldcg(&parent[x]); }
  return x;
}

__global__ void k_uf_init(int64_t n, int32_t *parent, int32_t *csize) {
  pdl_wait();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    parent[i] = (int32_t)i;
    csize[i] = 0;
  }
}

__global__ void k_uf_union(int64_t n, const int64_t *nb_off, const int32_t *nb_idx,
                           int32_t *parent, DevStatus *st) {
  pdl_wait();
  if (st->code != 0) return;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    for (int64_t q = nb_off[i]; q < nb_off[i + 1]; ++q) {
      const int32_t j = nb_idx[q];
      if (j <= i) continue;
      int64_t tries = 0;
      for (;;) {
        int32_t a = uf_find(parent, (int32_t)i), b = uf_find(parent, j);
        if (a == b) break;
        if (a > b) { int32_t t = a; a = b; b = t; }
        // hook the larger root below the smaller one
        if (atomicCAS(&parent[b], b, a) == b) break;
        if (++tries > kUFLimit) { dev_fail(st, P3T_ERR_TIMEOUT, 51, 0); return; }
      }
    }
  }
}

__global__ void k_uf_label(int64_t n, const int32_t *parent, int32_t *label,
                           int32_t *csize) {
  pdl_wait();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t r = uf_find(parent, (int32_t)i);
    label[i] = r;
    atomicAdd(&csize[r], 1);
  }
}

// flags: [0, n) isolated, [n, 2n) cluster roots, [2n, 3n) root sizes,
// [3n, 4n) members of clusters of >= 2
__global__ void k_cl_flags(int64_t n, const int32_t *label, const int32_t *csize,
                           int32_t *flag, int64_t *counts) {
  pdl_wait();
  unsigned long long mx = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t sz = csize[label[i]];
    const bool root = label[i] == i && csize[i] >= 2;
    // two words a particle, each scanned as (bit 0) + (bits 1-31) 2^31:
    // isolated and cluster member; cluster root and its size
    flag[i] = (sz == 1 ? 1 : 0) | (sz >= 2 ? 2 : 0);
    flag[n + i] = root ? 1 | (csize[i] << 1) : 0;
    if (root) mx = max(mx, (unsigned long long)csize[i]);
  }
  if (mx) atomicMax(reinterpret_cast<unsigned long long *>(&counts[3]), mx);
}

// the singles, each cluster's offset and the members (with their labels, for
// the sort) from the two packed scans (counts in bits 0-30, the second sum
// from bit 31), and the four totals: singles, clusters, members (counts[0..2])
// and members again for the sort (*d_nmem)
__global__ void k_cl_scatter(int64_t n, const int32_t *label, const int32_t *flag,
                             const int64_t *pos, const int64_t *d_tot, int32_t *singles,
                             int64_t *cl_off, uint64_t *mkeys, int32_t *mvals, int64_t *counts,
                             int64_t *d_nmem) {
  pdl_wait();
  constexpr int64_t kLow = (1ll << 31) - 1;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t fa = flag[i], fb = flag[n + i];
    if (fa & 1) singles[pos[i] & kLow] = (int32_t)i;
    if (fb & 1) {
      const int64_t q = pos[n + i];
      cl_off[q & kLow] = q >> 31;
    }
    if (fa & 2) {
      const int64_t q = pos[i] >> 31;
      mkeys[q] = (uint64_t)label[i];
      mvals[q] = (int32_t)i;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const int64_t ta = d_tot[0], tb = d_tot[1];
    counts[0] = ta & kLow;
    counts[1] = tb & kLow;
    counts[2] = tb >> 31;
    *d_nmem = ta >> 31;
    cl_off[tb & kLow] = tb >> 31;
  }
}

// the first *d_n values of src into dst
__global__ void k_copy_i32(const int64_t *d_n, const int32_t *src, int32_t *dst) {
  pdl_wait();
  const int64_t n = *d_n;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = src[i];
}

__global__ void k_zero_i64(int64_t *p, int k) {
  pdl_wait();
  if (threadIdx.x < k) p[threadIdx.x] = 0;
}

}  // namespace

int p3t_run_neighbours(p3t_ctx *c, const p3t_particles *p, int64_t *nb_off,
                       int32_t *nb_idx, int64_t nb_cap, cudaStream_t s) {
  const int64_t n = p->n;
  const int64_t maxb = (int64_t)c->num_sms * P3T_NSM_BLOCKS;
  const int64_t g = p3t_grid(n, kBlock, maxb);
  const int64_t gc = p3t_grid(c->cand_cap, kBlock, maxb);
  int64_t *cnt = c->counters;
  int rc;
  // ---- neighbour lists ----
  P3T_CUDA_TRY(cudaMemsetAsync(c->deg, 0, sizeof(int32_t) * (n + 1), s));
  P3T_CUDA_TRY(cudaMemsetAsync(c->fill, 0, sizeof(int32_t) * (n + 1), s));
  pdl_launch(k_nb_filter, dim3((unsigned)gc), dim3(kBlock), 0, s, &cnt[9], c->cand_i, c->cand_j, c->idx, *p,
                                              c->prm, c->cand_keep, c->deg, c->status);
  rc = p3t_scan_i32_to_i64(c->deg, nb_off, &cnt[0], c->cap, nb_off + n, c->scan_state, c->scan_words, c->status, c->poll_limit, s);
  if (rc) return rc;
  pdl_launch(k_nb_check, dim3(1), dim3(1), 0, s, nb_off + n, nb_cap, c->status);
  pdl_launch(k_nb_fill, dim3((unsigned)gc), dim3(kBlock), 0, s, &cnt[9], c->cand_i, c->cand_j, c->idx,
                                            c->cand_keep, nb_off, c->fill, nb_idx, c->status);
  pdl_launch(k_nb_sort_rows, dim3((unsigned)g), dim3(kBlock), 0, s, n, nb_off, nb_idx, c->status);
  // ---- neighbour clusters ----
  pdl_launch(k_zero_i64, dim3(1), dim3(32), 0, s, c->cl_counts, 4);
  pdl_launch(k_uf_init, dim3((unsigned)g), dim3(kBlock), 0, s, n, c->parent, c->csize);
  pdl_launch(k_uf_union, dim3((unsigned)g), dim3(kBlock), 0, s, n, nb_off, nb_idx, c->parent, c->status);
  pdl_launch(k_uf_label, dim3((unsigned)g), dim3(kBlock), 0, s, n, c->parent, c->label, c->csize);
  pdl_launch(k_cl_flags, dim3((unsigned)g), dim3(kBlock), 0, s, n, c->label, c->csize, c->flag, c->cl_counts);
  // two packed scans: (isolated, members) and (roots, root sizes); their
  // totals in cnt[21], cnt[22]
  for (int q = 0; q < 2; ++q) {
    rc = p3t_scan_flag_pairs(c->flag + q * n, c->pos + q * n, &cnt[0], c->cap, &cnt[21 + q],
                             c->scan_state, c->scan_words, c->status, c->poll_limit, s);
    if (rc) return rc;
  }
  pdl_launch(k_cl_scatter, dim3((unsigned)g), dim3(kBlock), 0, s, n, c->label, c->flag, c->pos,
             &cnt[21], c->singles, c->cl_off, c->mkeys, c->mvals, c->cl_counts, &cnt[11]);
  // filter, check, fill, sort_rows, zero, uf_init, uf_union, uf_label, flags, scatter
  p3t_note_launches(10);
  // members ordered by (label, index): stable sort of the ascending member
  // list on the label's bits (labels are particle indices below n).  The
  // sorted members must land in the buffer they started in, so that the
  // cluster views keep their addresses from step to step (a step captured in
  // a CUDA graph reads the previous step's clusters there): after an odd
  // number of 8-bit passes they are copied back
  const int bits = n <= 65536 ? 16 : (n <= (1 << 24) ? 24 : 32);
  uint64_t *k0 = c->mkeys, *k1 = c->mkeys_alt;
  int32_t *v0 = c->mvals, *v1 = c->mvals_alt;
  rc = p3t_radix_sort(&k0, &v0, &k1, &v1, &cnt[11], c->cap, 0, bits, c->radix_hist,
                      c->radix_hist_cap, s);
  if (rc) return rc;
  if (v0 != c->mvals) {
    pdl_launch(k_copy_i32, dim3((unsigned)p3t_grid(n, kBlock, maxb)), dim3(kBlock), 0, s, &cnt[11],
               v0, c->mvals);
    p3t_note_launches(1);
  }
  c->cl_mem = c->mvals;  // sorted payload buffer
  return cudaGetLastError() == cudaSuccess ? P3T_OK : P3T_ERR_CUDA;
}

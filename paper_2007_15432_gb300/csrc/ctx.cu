// C-ABI entry points of libp3t: context, buffers, argument checks, status.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <atomic>
#include <new>

#include "p3t_internal.cuh"

int64_t p3t_walk_warps(int num_sms, int64_t n);
int p3t_walk_blocks_per_sm();

static std::atomic<long long> g_launches{0};
void p3t_note_launches(int64_t k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

namespace {

constexpr int64_t kStackCap = 8192;  // walk stack entries per warp

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

bool params_ok(const p3t_params *p) {
  if (!p) return false;
  if (!(p->G > 0.0) || !(p->m_star >= 0.0) || !(p->dt_soft > 0.0)) return false;
  if (!(p->gamma > 0.0 && p->gamma < 1.0)) return false;
  if (!(p->rcut0 >= 0.0) || !(p->rcut1 >= 0.0)) return false;
  if (!(p->rs0 >= 1.0) || !(p->rs1 >= 0.0) || !(p->rs2 >= 0.0) || !(p->rs3 >= 0.0)) return false;
  if (!(p->theta >= 0.0) || !(p->eta > 0.0) || !(p->eta0 > 0.0)) return false;
  if (p->leaf_size < 1 || p->leaf_size > 32) return false;
  if (p->precision != P3T_FP64 && p->precision != P3T_MIXED) return false;
  if (p->vran_bins < 0 || p->vran_bins > 4096) return false;
  if (p->group_size < 0 || p->group_size > 64) return false;
  if (!(p->f_radius >= 0.0)) return false;
  if (p->cutoff_mode < P3T_CUT_HILL_VRAN || p->cutoff_mode > P3T_CUT_SHARED) return false;
  return true;
}

bool particles_ok(const p3t_particles *p) {
  if (!p || p->n < 0 || p->n >= ((int64_t)1 << 31)) return false;
  if (p->n == 0) return true;
  return p->x && p->y && p->z && p->vx && p->vy && p->vz && p->m && p->r_out &&
         p->r_search;
}

// with segments set, the particle count must be the segments' total
bool segments_ok(const p3t_ctx *c, const p3t_particles *p) {
  return c->nseg == 1 || p->n == c->seg_off_h[c->nseg];
}

template <typename T> void dfree(T *&ptr) {
  if (ptr) cudaFree((void *)ptr);
  ptr = nullptr;
}

template <typename T> bool dalloc(T *&ptr, int64_t count) {
  dfree(ptr);
  if (count < 1) count = 1;
  return cudaMalloc((void **)&ptr, sizeof(T) * (size_t)count) == cudaSuccess;
}

void free_particle_buffers(p3t_ctx *c) {
  dfree(c->keys); dfree(c->keys_alt); dfree(c->idx); dfree(c->idx_alt);
  dfree(c->radix_hist);
  dfree(c->sx); dfree(c->sy); dfree(c->sz); dfree(c->sm); dfree(c->sro); dfree(c->srs);
  dfree(c->pack);
  dfree(c->sq); dfree(c->spA); dfree(c->spB); dfree(c->srs32); dfree(c->sml);
  dfree(c->lp); dfree(c->lv); dfree(c->ncount); dfree(c->nstart);
  dfree(c->pre_first); dfree(c->pre_count); dfree(c->pre_level);
  dfree(c->lvl_keys); dfree(c->lvl_keys_alt); dfree(c->bfs2pre); dfree(c->bfs2pre_alt);
  dfree(c->pre2bfs); dfree(c->node); dfree(c->mom64); dfree(c->mom32); dfree(c->nrs);
  dfree(c->node_done); dfree(c->leaf_list); dfree(c->node_flag); dfree(c->flag_pos);
  dfree(c->group_list);
  dfree(c->walk_stack); dfree(c->cand_i); dfree(c->cand_j); dfree(c->cand_keep);
  dfree(c->deg); dfree(c->fill); dfree(c->parent); dfree(c->label); dfree(c->csize);
  dfree(c->flag); dfree(c->pos); dfree(c->singles); dfree(c->cl_off); dfree(c->hlist);
  // cl_mem aliases one of the mvals buffers
  c->cl_mem = nullptr;
  dfree(c->mkeys); dfree(c->mkeys_alt); dfree(c->mvals); dfree(c->mvals_alt);
  dfree(c->hw); dfree(c->ht); dfree(c->hl);
  dfree(c->coll_ent); dfree(c->coll_rec); dfree(c->coll_rec_e); dfree(c->coll_esoft);
  dfree(c->coll_slot); dfree(c->scan_state);
  dfree(c->nadj);
  c->nadj_cap = 0;
  dfree(c->hadj);
  c->hadj_cap = 0;
  c->scan_words = 0;
  c->cap = 0;
  c->have_tree = c->have_cand = false;
}

int64_t node_bound(int64_t n, int leaf, int64_t nseg) {
  // internal nodes hold > leaf particles: at most n / (leaf + 1) per level
  // below the roots, 21 levels, plus one root per segment and level;
  // leaves are disjoint non-empty sets: at most n
  return n + (int64_t)P3T_BITS * (n / (leaf + 1) + nseg) + 64;
}

int reserve(p3t_ctx *c, int64_t n, int64_t cand_cap) {
  const int64_t want_nodes = node_bound(n, c->prm.leaf_size, c->nseg);
  if (n <= c->cap && want_nodes <= c->node_cap && cand_cap <= c->cand_cap) return P3T_OK;
  cudaDeviceSynchronize();
  free_particle_buffers(c);
  const int64_t N = n > 1 ? n : 1;
  const int64_t NC = want_nodes;
  c->node_cap = NC;
  c->cand_cap = cand_cap;
  c->walk_warps = p3t_walk_warps(c->num_sms, N);
  c->stack_cap = kStackCap;
  c->radix_hist_cap = p3t_radix_hist_entries(N > NC ? N : NC);
  bool ok = true;
  ok &= dalloc(c->keys, N) && dalloc(c->keys_alt, N) && dalloc(c->idx, N) && dalloc(c->idx_alt, N);
  ok &= dalloc(c->radix_hist, c->radix_hist_cap);
  ok &= dalloc(c->sx, N) && dalloc(c->sy, N) && dalloc(c->sz, N) && dalloc(c->sm, N);
  ok &= dalloc(c->pack, 6 * N);
  ok &= dalloc(c->sro, N) && dalloc(c->srs, N) && dalloc(c->sq, 3 * N);
  ok &= dalloc(c->spA, N) && dalloc(c->spB, N) && dalloc(c->srs32, N) &&
        dalloc(c->sml, N);
  ok &= dalloc(c->lp, N) && dalloc(c->lv, N) && dalloc(c->ncount, N);
  ok &= dalloc(c->nstart, N);
  ok &= dalloc(c->pre_first, NC) && dalloc(c->pre_count, NC) && dalloc(c->pre_level, NC);
  ok &= dalloc(c->lvl_keys, NC) && dalloc(c->lvl_keys_alt, NC);
  ok &= dalloc(c->bfs2pre, NC) && dalloc(c->bfs2pre_alt, NC) && dalloc(c->pre2bfs, NC);
  ok &= dalloc(c->node, NC) && dalloc(c->mom64, NC) && dalloc(c->mom32, NC) && dalloc(c->nrs, NC);
  ok &= dalloc(c->node_done, NC) && dalloc(c->leaf_list, NC) && dalloc(c->node_flag, NC);
  ok &= dalloc(c->flag_pos, NC);
  ok &= dalloc(c->group_list, NC);
  ok &= dalloc(c->walk_stack, c->walk_warps * c->stack_cap);
  ok &= dalloc(c->cand_i, cand_cap) && dalloc(c->cand_j, cand_cap) && dalloc(c->cand_keep, cand_cap);
  ok &= dalloc(c->deg, N + 1) && dalloc(c->fill, N + 1);
  ok &= dalloc(c->parent, N) && dalloc(c->label, N) && dalloc(c->csize, N);
  ok &= dalloc(c->flag, 4 * N) && dalloc(c->pos, 4 * N);
  ok &= dalloc(c->singles, N) && dalloc(c->cl_off, N + 1);
  c->hlist_cap = N / 2 + 1;  // clusters have at least two members
  ok &= dalloc(c->hlist, 2 * c->hlist_cap);
  ok &= dalloc(c->mkeys, N) && dalloc(c->mkeys_alt, N) && dalloc(c->mvals, N) && dalloc(c->mvals_alt, N);
  ok &= dalloc(c->hw, 33 * N) && dalloc(c->ht, N) && dalloc(c->hl, 6 * N);
  ok &= dalloc(c->coll_ent, N) && dalloc(c->coll_rec, N / 2 + 1) && dalloc(c->coll_rec_e, N / 2 + 1);
  ok &= dalloc(c->coll_esoft, N) && dalloc(c->coll_slot, N);
  c->scan_words = p3t_scan_state_words(N > NC ? N : NC);
  ok &= dalloc(c->scan_state, c->scan_words);
  if (ok) ok = cudaMemset(c->scan_state, 0, sizeof(unsigned long long) * c->scan_words) ==
               cudaSuccess;
  // no composites: every slot -1, empty list (composites pending from a
  // smaller context are dropped with it)
  if (ok) ok = cudaMemset(c->coll_slot, 0xff, sizeof(int32_t) * N) == cudaSuccess &&
               cudaMemset(c->coll_ctr, 0, sizeof(unsigned long long)) == cudaSuccess &&
               cudaDeviceSynchronize() == cudaSuccess;
  if (!ok) {
    free_particle_buffers(c);
    cudaGetLastError();
    return P3T_ERR_CUDA;
  }
  c->cl_mem = c->mvals;
  c->cap = N;
  return P3T_OK;
}

int64_t default_cand_cap(int64_t n) { return 8 * n + 65536; }

int ensure(p3t_ctx *c, int64_t n) {
  int64_t cc = c->cand_cap > default_cand_cap(n) ? c->cand_cap : default_cand_cap(n);
  return reserve(c, n, cc);
}

}  // namespace

extern "C" {

int p3t_create(p3t_ctx **ctx, const p3t_params *p, int device) {
  if (!ctx || !params_ok(p)) return P3T_ERR_INVALID;
  *ctx = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return P3T_ERR_CUDA;
  }
  DeviceGuard g(device);
  p3t_ctx *c = new (std::nothrow) p3t_ctx();
  if (!c) return P3T_ERR_CUDA;
  c->device = device;
  c->prm = *p;
  if (cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
    delete c;
    return P3T_ERR_CUDA;
  }
  bool ok = dalloc(c->status, 1) && dalloc(c->box, 5) && dalloc(c->box_bits, 6) &&
            dalloc(c->counters, 64) && dalloc(c->cl_counts, 4) && dalloc(c->hsteps, 1) && dalloc(c->hcursor, 5) &&
            dalloc(c->coll_ctr, 1) &&
            dalloc(c->epart, 8192) && dalloc(c->bh_table, 32);
  for (int q = 0; q < 2 && ok; ++q)
    ok = cudaStreamCreateWithFlags(&c->aux[q], cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&c->ev_join[q], cudaEventDisableTiming) == cudaSuccess;
  if (ok) ok = cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) == cudaSuccess &&
               cudaEventCreateWithFlags(&c->ev_coll, cudaEventDisableTiming) == cudaSuccess &&
               cudaHostAlloc(reinterpret_cast<void **>(&c->coll_pin), sizeof(unsigned long long),
                             cudaHostAllocDefault) == cudaSuccess;
  if (ok) ok = cudaMemset(c->status, 0, sizeof(DevStatus)) == cudaSuccess &&
               cudaMemset(c->counters, 0, 64 * sizeof(int64_t)) == cudaSuccess &&
               cudaMemset(c->coll_ctr, 0, sizeof(unsigned long long)) == cudaSuccess &&
               cudaMemset(c->cl_counts, 0, 4 * sizeof(int64_t)) == cudaSuccess;
  if (!ok) {
    p3t_destroy(c);
    cudaGetLastError();
    return P3T_ERR_CUDA;
  }
  *ctx = c;
  return P3T_OK;
}

void p3t_destroy(p3t_ctx *c) {
  if (!c) return;
  DeviceGuard g(c->device);
  cudaDeviceSynchronize();
  free_particle_buffers(c);
  dfree(c->status); dfree(c->box); dfree(c->box_bits); dfree(c->counters);
  dfree(c->seg_off); dfree(c->seg_nb); dfree(c->seg_base); dfree(c->seg_l);
  delete[] c->seg_off_h;
  dfree(c->cl_counts); dfree(c->hsteps); dfree(c->hcursor); dfree(c->epart);
  dfree(c->coll_ctr);
  dfree(c->bh_table);
  dfree(c->dpart); dfree(c->dcnt);
  for (int q = 0; q < 2; ++q) {
    if (c->aux[q]) cudaStreamDestroy(c->aux[q]);
    if (c->ev_join[q]) cudaEventDestroy(c->ev_join[q]);
  }
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_coll) cudaEventDestroy(c->ev_coll);
  if (c->coll_pin) cudaFreeHost(c->coll_pin);
  cudaGetLastError();
  delete c;
}

int p3t_set_params(p3t_ctx *c, const p3t_params *p) {
  if (!c || !params_ok(p)) return P3T_ERR_INVALID;
  // the tree holds the sorted copies and moments of one precision only
  const bool leaf_changed = p->leaf_size != c->prm.leaf_size ||
                            p->group_size != c->prm.group_size ||
                            p->precision != c->prm.precision;
  c->prm = *p;
  if (leaf_changed) c->have_tree = c->have_cand = false;
  return P3T_OK;
}

int p3t_reserve(p3t_ctx *c, int64_t n) {
  if (!c || n < 0 || n >= ((int64_t)1 << 31)) return P3T_ERR_INVALID;
  DeviceGuard g(c->device);
  return ensure(c, n);
}

int p3t_set_segments(p3t_ctx *c, int64_t nseg, const int64_t *seg_off) {
  if (!c || nseg < 1 || nseg > P3T_MAX_SEGMENTS || !seg_off || seg_off[0] != 0)
    return P3T_ERR_INVALID;
  for (int64_t d = 0; d < nseg; ++d)
    if (seg_off[d + 1] <= seg_off[d]) return P3T_ERR_INVALID;  // no empty segment
  if (seg_off[nseg] >= ((int64_t)1 << 31)) return P3T_ERR_INVALID;
  DeviceGuard g(c->device);
  cudaDeviceSynchronize();
  dfree(c->seg_off); dfree(c->seg_nb); dfree(c->seg_base); dfree(c->seg_l);
  dfree(c->box); dfree(c->box_bits);
  delete[] c->seg_off_h;
  c->seg_off_h = nullptr;
  c->nseg = 1;
  const int64_t S = nseg;
  bool ok = dalloc(c->box, 5 * S) && dalloc(c->box_bits, 6 * S);
  if (ok && nseg > 1) {
    ok = dalloc(c->seg_off, S + 1) && dalloc(c->seg_nb, S) && dalloc(c->seg_base, S) &&
         dalloc(c->seg_l, 2 * S);
    if (ok)
      ok = cudaMemcpy(c->seg_off, seg_off, sizeof(int64_t) * (S + 1),
                      cudaMemcpyHostToDevice) == cudaSuccess;
    if (ok) {
      c->seg_off_h = new (std::nothrow) int64_t[S + 1];
      ok = c->seg_off_h != nullptr;
      if (ok) for (int64_t d = 0; d <= S; ++d) c->seg_off_h[d] = seg_off[d];
    }
  }
  if (!ok) {
    cudaGetLastError();
    return P3T_ERR_CUDA;
  }
  c->nseg = nseg;
  c->have_tree = c->have_cand = false;
  return P3T_OK;
}

int p3t_cutoffs(p3t_ctx *c, p3t_particles *p, void *stream) {
  if (!c || !particles_ok(p) || !segments_ok(c, p)) return P3T_ERR_INVALID;
  DeviceGuard g(c->device);
  int rc = ensure(c, p->n);
  if (rc) return rc;
  return p3t_run_cutoffs(c, p, (cudaStream_t)stream);
}

int p3t_build_tree(p3t_ctx *c, p3t_particles *p, int update_cutoffs, void *stream) {
  if (!c || !particles_ok(p) || !segments_ok(c, p)) return P3T_ERR_INVALID;
  DeviceGuard g(c->device);
  int rc = ensure(c, p->n);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  if (update_cutoffs) {
    rc = p3t_run_cutoffs(c, p, s);
    if (rc) return rc;
  }
  if (p->n == 0) {
    c->have_tree = false;
    c->last_n = 0;
    return P3T_OK;
  }
  rc = p3t_run_build_tree(c, p, s);
  if (rc) return rc;
  c->last_n = p->n;
  c->have_tree = true;
  c->have_cand = false;
  return P3T_OK;
}

int p3t_soft_force(p3t_ctx *c, const p3t_particles *p, double *ax, double *ay,
                   double *az, uint64_t *counts, void *stream) {
  if (!c || !particles_ok(p) || !segments_ok(c, p)) return P3T_ERR_INVALID;
  if (p->n == 0) return P3T_OK;
  if (!ax || !ay || !az || !c->have_tree || p->n != c->last_n) return P3T_ERR_INVALID;
  DeviceGuard g(c->device);
  int rc = p3t_run_soft_force(c, p, ax, ay, az, counts, (cudaStream_t)stream);
  if (rc == P3T_OK) c->have_cand = true;
  return rc;
}

int p3t_neighbours(p3t_ctx *c, const p3t_particles *p, int64_t *nb_off,
                   int32_t *nb_idx, int64_t nb_cap, p3t_clusters *out, void *stream) {
  if (!c || !particles_ok(p) || !nb_off || !out || nb_cap < 0) return P3T_ERR_INVALID;
  if (nb_cap > 0 && !nb_idx) return P3T_ERR_INVALID;
  if (p->n > 0 && (!c->have_cand || p->n != c->last_n)) return P3T_ERR_INVALID;
  DeviceGuard g(c->device);
  int rc = ensure(c, p->n);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  if (p->n == 0) {
    if (cudaMemsetAsync(nb_off, 0, sizeof(int64_t), s) != cudaSuccess ||
        cudaMemsetAsync(c->cl_counts, 0, 4 * sizeof(int64_t), s) != cudaSuccess ||
        cudaMemsetAsync(c->cl_off, 0, sizeof(int64_t), s) != cudaSuccess)
      return P3T_ERR_CUDA;
  } else {
    rc = p3t_run_neighbours(c, p, nb_off, nb_idx, nb_cap, s);
    if (rc) return rc;
  }
  out->label = c->label;
  out->singles = c->singles;
  out->cl_off = c->cl_off;
  out->cl_mem = c->cl_mem;
  out->counts = c->cl_counts;
  return P3T_OK;
}

int p3t_hard_step(p3t_ctx *c, p3t_particles *p, const p3t_clusters *cl, double dt,
                  uint64_t *n_steps, void *stream) {
  if (!c || !particles_ok(p) || !cl || !(dt > 0.0)) return P3T_ERR_INVALID;
  if (p->n == 0) return P3T_OK;
  if (!cl->singles || !cl->cl_off || !cl->cl_mem || !cl->counts) return P3T_ERR_INVALID;
  DeviceGuard g(c->device);
  int rc = ensure(c, p->n);
  if (rc) return rc;
  return p3t_run_hard_step(c, p, cl, dt, n_steps, (cudaStream_t)stream);
}

int p3t_kick(p3t_ctx *c, p3t_particles *p, const double *ax, const double *ay,
             const double *az, double h, void *stream) {
  if (!c || !particles_ok(p)) return P3T_ERR_INVALID;
  if (p->n > 0 && (!ax || !ay || !az)) return P3T_ERR_INVALID;
  DeviceGuard g(c->device);
  return p3t_run_kick(c, p, ax, ay, az, h, (cudaStream_t)stream);
}

int p3t_merge(p3t_ctx *c, p3t_particles *p, int32_t *new_index, double *e_disp,
              int64_t *n_merged, void *stream) {
  if (!c || !particles_ok(p) || c->nseg > 1) return P3T_ERR_INVALID;
  DeviceGuard g(c->device);
  if (p->n > c->cap) return P3T_ERR_INVALID;
  const int64_t n0 = p->n;
  int rc = p3t_run_merge(c, p, new_index, e_disp, n_merged, (cudaStream_t)stream);
  if (rc == P3T_OK && p->n != n0) c->have_tree = c->have_cand = false;
  return rc;
}

int p3t_collisions_pending(p3t_ctx *c, int64_t *n_clusters, void *stream) {
  if (!c || !n_clusters) return P3T_ERR_INVALID;
  DeviceGuard g(c->device);
  const cudaStream_t s = (cudaStream_t)stream;
  unsigned long long ctr = 0;  // (records << 32) | entries
  if (cudaMemcpyAsync(&ctr, c->coll_ctr, sizeof(ctr), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return P3T_ERR_CUDA;
  *n_clusters = (int64_t)(ctr >> 32);
  return P3T_OK;
}

int p3t_collisions_pending_async(p3t_ctx *c, void *stream) {
  if (!c) return P3T_ERR_INVALID;
  DeviceGuard g(c->device);
  const cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemcpyAsync(c->coll_pin, c->coll_ctr, sizeof(unsigned long long),
                      cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaEventRecord(c->ev_coll, s) != cudaSuccess)
    return P3T_ERR_CUDA;
  c->coll_queued = true;
  return P3T_OK;
}

int p3t_collisions_pending_wait(p3t_ctx *c, int64_t *n_clusters) {
  if (!c || !n_clusters || !c->coll_queued) return P3T_ERR_INVALID;
  DeviceGuard g(c->device);
  c->coll_queued = false;
  if (cudaEventSynchronize(c->ev_coll) != cudaSuccess) return P3T_ERR_CUDA;
  *n_clusters = (int64_t)(*c->coll_pin >> 32);
  return P3T_OK;
}

// the all-pairs kernels' scratch: the packed particles in hw (sized by
// ensure) and the partial sums, one allocation of fixed size made on the
// first call (a graph captured after one eager call allocates nothing)
static int direct_scratch(p3t_ctx *c, int64_t n) {
  int rc = ensure(c, n);  // hw holds the packed particles
  if (rc) return rc;
  if (c->dpart) return P3T_OK;
  const int64_t want = p3t_direct_part_doubles(c), tiles = p3t_direct_tile_counters(c);
  if (!dalloc(c->dpart, want) || !dalloc(c->dcnt, tiles)) return P3T_ERR_CUDA;
  if (cudaMemset(c->dcnt, 0, sizeof(int32_t) * tiles) != cudaSuccess) return P3T_ERR_CUDA;
  c->dpart_cap = want;
  c->dcnt_cap = tiles;
  return P3T_OK;
}

int p3t_kepler_drift(p3t_ctx *c, p3t_particles *p, double dt, void *stream) {
  if (!c || !particles_ok(p)) return P3T_ERR_INVALID;
  DeviceGuard g(c->device);
  return p3t_run_kepler_drift(c, p, dt, (cudaStream_t)stream);
}

int p3t_soft_force_direct(p3t_ctx *c, const p3t_particles *p, double *ax, double *ay,
                          double *az, void *stream) {
  if (!c || !particles_ok(p) || c->nseg > 1) return P3T_ERR_INVALID;
  if (p->n > 0 && (!ax || !ay || !az)) return P3T_ERR_INVALID;
  DeviceGuard g(c->device);
  int rc = direct_scratch(c, p->n);
  if (rc) return rc;
  return p3t_run_soft_force_direct(c, p, ax, ay, az, (cudaStream_t)stream);
}

int p3t_soft_force_vjp(p3t_ctx *c, const p3t_particles *p, double h, const double *lx,
                       const double *ly, const double *lz, double *gx, double *gy, double *gz,
                       double *gm, void *stream) {
  if (!c || !particles_ok(p) || c->nseg > 1) return P3T_ERR_INVALID;
  if (p->n > 0 && (!lx || !ly || !lz || !gx || !gy || !gz || !gm)) return P3T_ERR_INVALID;
  DeviceGuard g(c->device);
  int rc = direct_scratch(c, p->n);
  if (rc) return rc;
  return p3t_run_soft_force_vjp(c, p, h, lx, ly, lz, gx, gy, gz, gm, (cudaStream_t)stream);
}

int p3t_soft_force_vjp_tree(p3t_ctx *c, const p3t_particles *p, double h, const double *lx,
                            const double *ly, const double *lz, double *gx, double *gy,
                            double *gz, double *gm, void *stream) {
  if (!c || !particles_ok(p) || !segments_ok(c, p)) return P3T_ERR_INVALID;
  if (p->n == 0) return P3T_OK;
  if (!lx || !ly || !lz || !gx || !gy || !gz || !gm) return P3T_ERR_INVALID;
  if (c->prm.precision != P3T_FP64 || !c->have_tree || p->n != c->last_n) return P3T_ERR_INVALID;
  DeviceGuard g(c->device);
  if (c->nadj_cap < c->node_cap) {
    if (!dalloc(c->nadj, 10 * c->node_cap)) return P3T_ERR_CUDA;
    c->nadj_cap = c->node_cap;
  }
  return p3t_run_soft_force_vjp_tree(c, p, h, lx, ly, lz, gx, gy, gz, gm, (cudaStream_t)stream);
}

int p3t_hard_step_vjp(p3t_ctx *c, const p3t_particles *p, const p3t_clusters *cl, double dt,
                      double *lx, double *ly, double *lz, double *lvx, double *lvy, double *lvz,
                      double *gm, void *stream) {
  if (!c || !particles_ok(p) || !cl || !(dt > 0.0) || c->prm.f_radius > 0.0)
    return P3T_ERR_INVALID;
  if (p->n == 0) return P3T_OK;
  if (!cl->cl_off || !cl->cl_mem || !cl->counts || !lx || !ly || !lz || !lvx || !lvy || !lvz ||
      !gm)
    return P3T_ERR_INVALID;
  DeviceGuard g(c->device);
  if (c->hadj_cap < p->n) {
    if (!dalloc(c->hadj, 6 * p->n)) return P3T_ERR_CUDA;
    c->hadj_cap = p->n;
  }
  return p3t_run_hard_step_vjp(c, p, cl, dt, lx, ly, lz, lvx, lvy, lvz, gm,
                               (cudaStream_t)stream);
}

int p3t_kepler_vjp(p3t_ctx *c, const p3t_particles *p, double dt, double *lx, double *ly,
                   double *lz, double *lvx, double *lvy, double *lvz, void *stream) {
  if (!c || !particles_ok(p)) return P3T_ERR_INVALID;
  if (p->n > 0 && (!lx || !ly || !lz || !lvx || !lvy || !lvz)) return P3T_ERR_INVALID;
  DeviceGuard g(c->device);
  return p3t_run_kepler_vjp(c, p, dt, lx, ly, lz, lvx, lvy, lvz, (cudaStream_t)stream);
}

int p3t_energy(p3t_ctx *c, const p3t_particles *p, double *out, void *stream) {
  if (!c || !particles_ok(p) || !out || c->nseg > 1) return P3T_ERR_INVALID;
  DeviceGuard g(c->device);
  int rc = ensure(c, p->n);
  if (rc) return rc;
  return p3t_run_energy(c, p, out, (cudaStream_t)stream);
}

int p3t_copy_clusters(p3t_ctx *c, const p3t_clusters *cl, int64_t n, int32_t *label,
                      int32_t *singles, int64_t *cl_off, int32_t *cl_mem, int64_t *counts,
                      void *stream) {
  if (!c || !cl || n < 0 || !label || !singles || !cl_off || !cl_mem || !counts)
    return P3T_ERR_INVALID;
  DeviceGuard g(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  const cudaMemcpyKind k = cudaMemcpyDeviceToDevice;
  if (n > 0) {
    P3T_CUDA_TRY(cudaMemcpyAsync(label, cl->label, sizeof(int32_t) * n, k, s));
    P3T_CUDA_TRY(cudaMemcpyAsync(singles, cl->singles, sizeof(int32_t) * n, k, s));
    P3T_CUDA_TRY(cudaMemcpyAsync(cl_mem, cl->cl_mem, sizeof(int32_t) * n, k, s));
  }
  P3T_CUDA_TRY(cudaMemcpyAsync(cl_off, cl->cl_off, sizeof(int64_t) * (n + 1), k, s));
  P3T_CUDA_TRY(cudaMemcpyAsync(counts, cl->counts, sizeof(int64_t) * 4, k, s));
  return P3T_OK;
}

int p3t_set_diag(p3t_ctx *c, const p3t_diag *d) {
  if (!c || !d || d->hermite_block_limit < 0 || d->scan_poll_limit < 0) return P3T_ERR_INVALID;
  c->hermite_limit = d->hermite_block_limit > 0 ? d->hermite_block_limit : (int64_t)1 << 24;
  c->poll_limit = d->scan_poll_limit > 0 ? d->scan_poll_limit : (int64_t)1 << 22;
  c->hermite_rec = d->hermite_steps;
  return P3T_OK;
}

int p3t_set_tuning(p3t_ctx *c, const p3t_tuning *t) {
  if (!c || !t) return P3T_ERR_INVALID;
  if (t->hermite_warp_max != 0 && (t->hermite_warp_max < 2 || t->hermite_warp_max > 32))
    return P3T_ERR_INVALID;
  if (t->walk_blocks_per_sm < 0 || t->walk_blocks_per_sm > p3t_walk_blocks_per_sm())
    return P3T_ERR_INVALID;
  c->hwarp_max = t->hermite_warp_max ? t->hermite_warp_max : 8;
  c->walk_bps = t->walk_blocks_per_sm;
  return P3T_OK;
}

int p3t_status(p3t_ctx *c, int64_t *required) {
  if (!c) return P3T_ERR_INVALID;
  DeviceGuard g(c->device);
  if (cudaDeviceSynchronize() != cudaSuccess) {
    cudaGetLastError();
    return P3T_ERR_CUDA;
  }
  DevStatus st;
  if (cudaMemcpy(&st, c->status, sizeof(st), cudaMemcpyDeviceToHost) != cudaSuccess)
    return P3T_ERR_CUDA;
  if (required) *required = st.required;
  // grow the candidate buffers for the next walk if this one overflowed (the
  // force and neighbour calls of that step must then be repeated)
  if (st.cand_need > c->cand_cap) {
    const int64_t want = st.cand_need + st.cand_need / 4 + 1024;
    if (dalloc(c->cand_i, want) && dalloc(c->cand_j, want) && dalloc(c->cand_keep, want)) {
      c->cand_cap = want;
    } else {
      cudaGetLastError();
      dalloc(c->cand_i, c->cand_cap); dalloc(c->cand_j, c->cand_cap);
      dalloc(c->cand_keep, c->cand_cap);
    }
    c->have_cand = false;
  }
  DevStatus zero;
  memset(&zero, 0, sizeof(zero));
  zero.cand_need = st.cand_need;
  if (cudaMemcpy(c->status, &zero, sizeof(zero), cudaMemcpyHostToDevice) != cudaSuccess)
    return P3T_ERR_CUDA;
  return st.code;
}

int p3t_tree_stats(p3t_ctx *c, int64_t out[4]) {
  if (!c || !out) return P3T_ERR_INVALID;
  DeviceGuard g(c->device);
  if (cudaDeviceSynchronize() != cudaSuccess) return P3T_ERR_CUDA;
  if (c->have_tree) {
    if (p3t_run_tree_stats(c, 0) != P3T_OK) return P3T_ERR_CUDA;
    if (cudaDeviceSynchronize() != cudaSuccess) return P3T_ERR_CUDA;
  }
  int64_t h[8];
  if (cudaMemcpy(h, c->counters, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess)
    return P3T_ERR_CUDA;
  out[0] = h[1];
  out[1] = h[5];
  out[2] = h[6];
  out[3] = h[7];
  return P3T_OK;
}

int64_t p3t_launch_count(void) { return (int64_t)g_launches.load(); }

const char *p3t_strerror(int code) {
  switch (code) {
    case P3T_OK: return "ok";
    case P3T_ERR_INVALID: return "invalid argument, parameter or call order";
    case P3T_ERR_CUDA: return "CUDA runtime error";
    case P3T_ERR_CAPACITY: return "buffer capacity exceeded (see required size)";
    case P3T_ERR_DT_UNDERFLOW: return "Hermite time step below dt / 2^40";
    case P3T_ERR_TIMEOUT: return "bounded device loop gave up";
    default: return "unknown status";
  }
}

}  // extern "C"

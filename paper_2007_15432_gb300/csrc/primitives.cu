// Device-wide primitives of libp3t: exclusive scan and stable LSD radix sort.
// Element counts are read from device memory so that a whole soft step can be
// enqueued (and captured in a CUDA graph) without reading sizes on the host.
#include "p3t_internal.cuh"

namespace {

__device__ __forceinline__ int64_t warp_incl_scan(int64_t v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int64_t t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

// block-wide exclusive scan of one value per thread; returns the block total
__device__ int64_t block_excl_scan(int64_t v, int64_t *excl, int64_t *sh) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int64_t inc = warp_incl_scan(v);
  if (lane == 31) sh[w] = inc;
  __syncthreads();
  if (w == 0) {
    int64_t s = lane < nw ? sh[lane] : 0;
    int64_t si = warp_incl_scan(s);
    if (lane < nw) sh[lane] = si - s;
    if (lane == 31) sh[32] = si;
  }
  __syncthreads();
  *excl = inc - v + sh[w];
  int64_t tot = sh[32];
  __syncthreads();
  return tot;
}

// ---- single-pass exclusive scan (decoupled look-back) -----------------------
// Each block takes the next tile number from a counter in state[0] (so every
// smaller tile belongs to a block that has started and will finish without
// waiting on this one), scans its tile, publishes the tile's sum, adds its
// predecessors' sums by looking back (a warp reads 32 predecessor words at a
// time and stops at the nearest one that holds an inclusive prefix), and
// publishes its own inclusive prefix.  A word holds a flag in bits 63-62 (1:
// the tile's own sum, 2: inclusive prefix) and the value in bits 61-0
// (non-negative inputs).  The grid is sized for the capacity; only as many
// blocks as the count has tiles take one, the rest return at once.  The last
// block to finish (counter state[1]) clears the words it used and both
// counters, so that the next call starts clean with no host involvement.  A bounded number of polls: a predecessor that
// never publishes is reported (P3T_ERR_TIMEOUT) and counted as zero.  With
// PAIRS, every input holds a 0/1 flag in bit 0 and a non-negative value in
// bits 1-31 and counts as flag + value 2^31, so that one scan gives both
// prefix sums (each below 2^31) in one word.
constexpr int kScanThreads = 512;
constexpr int kScanPer = 8;
constexpr int kScanTile = kScanThreads * kScanPer;
constexpr unsigned long long kFlagAgg = 1ull << 62, kFlagInc = 2ull << 62;
constexpr unsigned long long kValMask = (1ull << 62) - 1;
template <bool PAIRS>
__device__ __forceinline__ int64_t scan_value(int32_t v) {
  return PAIRS ? (int64_t)(v & 1) + ((int64_t)((uint32_t)v >> 1) << 31) : (int64_t)v;
}
template <bool PAIRS>
__global__ void __launch_bounds__(kScanThreads)
scan_onepass(const int32_t *in, int64_t *out, const int64_t *d_n, int64_t *d_total,
             unsigned long long *state, DevStatus *st, int64_t poll_limit) {
  pdl_wait();
  __shared__ int64_t sh[33];
  // the tile: first its int32 inputs, then its int64 outputs (staged so that
  // both the loads and the stores are coalesced)
  __shared__ __align__(16) int64_t s_buf[kScanTile];
  int32_t *s_in = reinterpret_cast<int32_t *>(s_buf);
  __shared__ unsigned long long s_tile;
  __shared__ int64_t s_prefix;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int64_t n = *d_n;
  // the grid is sized for the capacity: only the first `used` blocks take
  // tiles (and count themselves out below); the others return at once
  const int64_t used = (n + kScanTile - 1) / kScanTile;
  const int64_t takers = used < 1 ? 1 : (used < (int64_t)gridDim.x ? used : (int64_t)gridDim.x);
  if ((int64_t)blockIdx.x >= takers) return;
  if (t == 0) s_tile = atomicAdd(&state[0], 1ull);
  __syncthreads();
  const int64_t tile = (int64_t)s_tile;
  const int64_t base = tile * kScanTile;
  unsigned long long *ts = state + 2;
  if (base < n) {
    for (int i = 0; i < kScanPer; ++i) {
      const int64_t e = base + (int64_t)i * kScanThreads + t;
      s_in[i * kScanThreads + t] = e < n ? in[e] : 0;
    }
    __syncthreads();
    int32_t v[kScanPer];
    int64_t sum = 0;
    {
      const int4 a = reinterpret_cast<const int4 *>(s_in)[2 * t];
      const int4 b = reinterpret_cast<const int4 *>(s_in)[2 * t + 1];
      v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
      v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
    }
#pragma unroll
    for (int i = 0; i < kScanPer; ++i) sum += scan_value<PAIRS>(v[i]);
    int64_t ex;
    const int64_t agg = block_excl_scan(sum, &ex, sh);
    if (warp == 0) {
      int64_t prefix = 0;
      if (tile == 0) {
        if (lane == 0) {
          __threadfence();
          __stcg(&ts[0], kFlagInc | (unsigned long long)agg);
        }
      } else {
        if (lane == 0) {
          __threadfence();
          __stcg(&ts[tile], kFlagAgg | (unsigned long long)agg);
        }
        int64_t p = tile - 1;  // the window's first (nearest) predecessor
        int64_t polls = 0;
        for (;;) {
          const int64_t q = p - lane;
          unsigned long long w = q >= 0 ? __ldcv(&ts[q]) : kFlagInc;
          while (__any_sync(0xffffffffu, (w >> 62) == 0)) {
            if (++polls > poll_limit) {
              if (lane == 0) dev_fail(st, P3T_ERR_TIMEOUT, 70, 0);
              w = (w >> 62) == 0 ? kFlagAgg : w;  // count the silent tile as zero
              break;
            }
            __nanosleep(64);
            if ((w >> 62) == 0) w = __ldcv(&ts[q]);
          }
          const unsigned inc = __ballot_sync(0xffffffffu, (w >> 62) == 2);
          const int last = inc ? __ffs(inc) - 1 : 31;  // nearest inclusive prefix
          int64_t val = lane <= last ? (int64_t)(w & kValMask) : 0;
          for (int o = 16; o > 0; o >>= 1) val += __shfl_xor_sync(0xffffffffu, val, o);
          prefix += val;
          if (inc) break;
          p -= 32;
        }
        if (lane == 0) {
          __threadfence();
          __stcg(&ts[tile], kFlagInc | (unsigned long long)(prefix + agg));
        }
      }
      if (lane == 0) s_prefix = prefix;
    }
    __syncthreads();  // every thread has read its inputs: s_buf now holds outputs
    int64_t run = s_prefix + ex;
#pragma unroll
    for (int i = 0; i < kScanPer; ++i) {
      s_buf[t * kScanPer + i] = run;
      run += scan_value<PAIRS>(v[i]);
    }
    __syncthreads();
    for (int i = 0; i < kScanPer; ++i) {
      const int64_t e = base + (int64_t)i * kScanThreads + t;
      if (e < n) out[e] = s_buf[i * kScanThreads + t];
    }
    if (t == 0 && base + kScanTile >= n && d_total) *d_total = s_prefix + agg;
  } else if (t == 0 && tile == 0 && d_total) {
    *d_total = 0;  // n = 0
  }
  // the last block out resets the tile words and the counters
  __shared__ bool s_last;
  __syncthreads();
  if (t == 0) {
    __threadfence();
    s_last = atomicAdd(&state[1], 1ull) == (unsigned long long)takers - 1;
  }
  __syncthreads();
  if (s_last) {
    __threadfence();
    for (int64_t k = t; k < used; k += kScanThreads) ts[k] = 0ull;
    if (t == 0) { state[0] = 0ull; state[1] = 0ull; }
  }
}

// ---- radix sort -----------------------------------------------------------
constexpr int kRadixBits = 8;
constexpr int kRadix = 1 << kRadixBits;
constexpr int kSortThreads = 256;
constexpr int kSortItems = 8;
constexpr int kSortTile = kSortThreads * kSortItems;

// The grids are sized for the capacity; the tiles actually holding keys
// (from the count on the device) are dealt grid-stride, so a short sort (a
// few thousand cluster members in a buffer sized for every particle) costs
// little more than its launches.  hist rows keep the capacity's stride.
__device__ __forceinline__ int64_t radix_tiles(const int64_t *d_n) {
  return (*d_n + kSortTile - 1) / kSortTile;
}

__global__ void radix_upsweep(const uint64_t *keys, const int64_t *d_n,
                              int shift, uint32_t *hist, int ntiles) {
  pdl_wait();
  __shared__ uint32_t h[kRadix];
  const int64_t n = *d_n;
  const int64_t used = radix_tiles(d_n);
  for (int64_t tile = blockIdx.x; tile < used; tile += gridDim.x) {
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = tile * kSortTile;
    // every load of the tile issued before the first is used
    uint32_t dig[kSortItems];
#pragma unroll
    for (int k = 0; k < kSortItems; ++k) {
      const int64_t e = base + k * kSortThreads + threadIdx.x;
      dig[k] = e < n ? (uint32_t)((__ldg(&keys[e]) >> shift) & (kRadix - 1)) : kRadix;
    }
    // plain shared atomics: on this part a warp's same-address atomics cost
    // less than matching the lanes' digits first
#pragma unroll
    for (int k = 0; k < kSortItems; ++k)
      if (dig[k] < kRadix) atomicAdd(&h[dig[k]], 1u);
    __syncthreads();
    hist[(int64_t)threadIdx.x * ntiles + tile] = h[threadIdx.x];
    __syncthreads();
  }
}

// exclusive scan of each digit's row of tile counts (one block per digit);
// the row total goes to the last slot of the digit's totals
__global__ void __launch_bounds__(kRadix) radix_row_scan(uint32_t *hist, int ntiles,
                                                         uint32_t *digit_total,
                                                         const int64_t *d_n) {
  pdl_wait();
  __shared__ int64_t sh[33];
  uint32_t *row = hist + (int64_t)blockIdx.x * ntiles;
  const int used = (int)radix_tiles(d_n);
  int64_t carry = 0;
  for (int base = 0; base < used; base += kRadix) {
    const int i = base + threadIdx.x;
    const int64_t v = i < used ? row[i] : 0;
    int64_t ex;
    const int64_t tot = block_excl_scan(v, &ex, sh);
    if (i < used) row[i] = (uint32_t)(carry + ex);
    carry += tot;
  }
  if (threadIdx.x == 0) digit_total[blockIdx.x] = (uint32_t)carry;
}

// The lanes of the warp whose (valid) digit equals this lane's: eight ballots,
// one a bit of the digit (on this part cheaper than __match_any_sync); zero
// for an invalid lane
__device__ __forceinline__ uint32_t match_digit(uint32_t d, bool valid) {
  uint32_t m = __ballot_sync(0xffffffffu, valid);
#pragma unroll
  for (int b = 0; b < kRadixBits; ++b) {
    const uint32_t bb = __ballot_sync(0xffffffffu, (d >> b) & 1u);
    m &= ((d >> b) & 1u) ? bb : ~bb;
  }
  return valid ? m : 0u;
}

// Stable scatter of one tile: the tile's elements are ranked by (digit,
// position), placed digit-ordered in shared memory, then written out so that
// consecutive threads write consecutive addresses of one digit's run.
__global__ void __launch_bounds__(kSortThreads)
radix_downsweep(const uint64_t *keys, const int32_t *vals, uint64_t *okeys,
                int32_t *ovals, const int64_t *d_n, int shift,
                const uint32_t *hist, int ntiles, const uint32_t *digit_total) {
  pdl_wait();
  __shared__ uint32_t s_warp[kSortThreads / 32][kRadix];
  __shared__ uint32_t s_run[kRadix];
  __shared__ uint32_t s_gbase[kRadix];  // first output index of the tile's digit d
  __shared__ uint32_t s_lbase[kRadix];  // first tile position of digit d
  __shared__ int64_t sh[33];
  __shared__ uint64_t s_key[kSortTile];
  __shared__ int32_t s_val[kSortTile];
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const int64_t n = *d_n;
  const int64_t used = radix_tiles(d_n);
  if (blockIdx.x >= used) return;  // no tile of this sort for this block
  int64_t dbase;
  block_excl_scan((int64_t)digit_total[t], &dbase, sh);   // digit bases
  for (int64_t tile = blockIdx.x; tile < used; tile += gridDim.x) {
    __syncthreads();
    s_run[t] = 0;
    s_gbase[t] = (uint32_t)dbase + hist[(int64_t)t * ntiles + tile];
    const int64_t base = tile * kSortTile;
    const uint32_t lt = (1u << lane) - 1u;
    uint64_t key[kSortItems];
    int32_t val[kSortItems];
    uint32_t dig[kSortItems], rk[kSortItems];
    // the tile's loads all issued up front: the ranking rounds below are
    // separated by block barriers, which no load can be moved across
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
      const int64_t e = base + r * kSortThreads + t;
      key[r] = 0;
      val[r] = 0;
      if (e < n) {
        key[r] = __ldg(&keys[e]);
        val[r] = __ldg(&vals[e]);
      }
    }
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
#pragma unroll
      for (int k = 0; k < kSortThreads / 32; ++k) s_warp[k][t] = 0;
      __syncthreads();
      const int64_t e = base + r * kSortThreads + t;
      const bool valid = e < n;
      // invalid lanes belong to no group
      const uint32_t d = valid ? (uint32_t)((key[r] >> shift) & (kRadix - 1)) : kRadix;
      dig[r] = d;
      const uint32_t peers = match_digit(d, valid);
      if (valid && lane == __ffs(peers) - 1) s_warp[w][d] = __popc(peers);
      __syncthreads();
      {
        uint32_t run = s_run[t];
#pragma unroll
        for (int k = 0; k < kSortThreads / 32; ++k) {
          uint32_t c = s_warp[k][t];
          s_warp[k][t] = run;
          run += c;
        }
        s_run[t] = run;
      }
      __syncthreads();
      rk[r] = valid ? s_warp[w][d] + __popc(peers & lt) : 0;  // rank within the tile's digit
      __syncthreads();
    }
    {
      int64_t ex;
      block_excl_scan((int64_t)s_run[t], &ex, sh);
      s_lbase[t] = (uint32_t)ex;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kSortItems; ++r)
      if (dig[r] < kRadix) {
        const uint32_t pos = s_lbase[dig[r]] + rk[r];
        s_key[pos] = key[r];
        s_val[pos] = val[r];
      }
    __syncthreads();
    const int64_t tn = n - base < kSortTile ? n - base : kSortTile;
    for (int i = t; i < tn; i += kSortThreads) {
      const uint64_t k = s_key[i];
      const uint32_t d = (uint32_t)((k >> shift) & (kRadix - 1));
      const uint32_t dst = s_gbase[d] + ((uint32_t)i - s_lbase[d]);
      okeys[dst] = k;
      ovals[dst] = s_val[i];
    }
  }
}

}  // namespace

int64_t p3t_scan_state_words(int64_t n_cap) {
  return 2 + (n_cap + kScanTile - 1) / kScanTile;
}

int p3t_scan_i32_to_i64(const int32_t *in, int64_t *out, const int64_t *d_n,
                        int64_t n_cap, int64_t *d_total, unsigned long long *state,
                        int64_t state_words, DevStatus *st, int64_t poll_limit,
                        cudaStream_t s) {
  int64_t G = (n_cap + kScanTile - 1) / kScanTile;
  if (G < 1) G = 1;
  if (G + 2 > state_words) return P3T_ERR_CAPACITY;
  pdl_launch(scan_onepass<false>, dim3((unsigned)G), dim3(kScanThreads), 0, s, in, out, d_n, d_total,
             state, st, poll_limit);
  p3t_note_launches(1);
  return cudaGetLastError() == cudaSuccess ? P3T_OK : P3T_ERR_CUDA;
}

int p3t_scan_flag_pairs(const int32_t *in, int64_t *out, const int64_t *d_n, int64_t n_cap,
                        int64_t *d_total, unsigned long long *state, int64_t state_words,
                        DevStatus *st, int64_t poll_limit, cudaStream_t s) {
  int64_t G = (n_cap + kScanTile - 1) / kScanTile;
  if (G < 1) G = 1;
  if (G + 2 > state_words) return P3T_ERR_CAPACITY;
  pdl_launch(scan_onepass<true>, dim3((unsigned)G), dim3(kScanThreads), 0, s, in, out, d_n, d_total,
             state, st, poll_limit);
  p3t_note_launches(1);
  return cudaGetLastError() == cudaSuccess ? P3T_OK : P3T_ERR_CUDA;
}

int64_t p3t_radix_hist_entries(int64_t n_cap) {
  int64_t ntiles = (n_cap + kSortTile - 1) / kSortTile;
  if (ntiles < 1) ntiles = 1;
  return ntiles * kRadix + kRadix;  // + the digit totals
}

int p3t_radix_sort(uint64_t **keys, int32_t **vals, uint64_t **keys_alt,
                   int32_t **vals_alt, const int64_t *d_n, int64_t n_cap,
                   int begin_bit, int end_bit, uint32_t *hist,
                   int64_t hist_cap, cudaStream_t s) {
  int64_t ntiles = (n_cap + kSortTile - 1) / kSortTile;
  if (ntiles < 1) ntiles = 1;
  if (ntiles * kRadix + kRadix > hist_cap) return P3T_ERR_CAPACITY;
  uint32_t *digit_total = hist + ntiles * kRadix;
  for (int shift = begin_bit; shift < end_bit; shift += kRadixBits) {
    pdl_launch(radix_upsweep, dim3((unsigned)ntiles), dim3(kSortThreads), 0, s, *keys, d_n, shift,
                                                            hist, (int)ntiles);
    pdl_launch(radix_row_scan, dim3(kRadix), dim3(kRadix), 0, s, hist, (int)ntiles, digit_total, d_n);
    pdl_launch(radix_downsweep, dim3((unsigned)ntiles), dim3(kSortThreads), 0, s, 
        *keys, *vals, *keys_alt, *vals_alt, d_n, shift, hist, (int)ntiles, digit_total);
    p3t_note_launches(3);
    uint64_t *tk = *keys; *keys = *keys_alt; *keys_alt = tk;
    int32_t *tv = *vals; *vals = *vals_alt; *vals_alt = tv;
  }
  return cudaGetLastError() == cudaSuccess ? P3T_OK : P3T_ERR_CUDA;
}

// Device-wide primitives of libp3t: exclusive scan and stable LSD radix sort.
// Element counts are read from device memory so that a whole soft step can be
// enqueued (and captured in a CUDA graph) without reading sizes on the host.
#include "p3t_internal.cuh"

namespace {

constexpr int kScanBlock = 1024;
constexpr int kScanMaxBlocks = 1024;

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

__global__ void scan_reduce_kernel(const int32_t *in, const int64_t *d_n,
                                   int64_t *part) {
  __shared__ int64_t sh[33];
  const int64_t n = *d_n;
  const int64_t G = gridDim.x;
  const int64_t chunk = (n + G - 1) / G;
  const int64_t lo = blockIdx.x * chunk;
  const int64_t hi = min(n, lo + chunk);
  int64_t s = 0;
  for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) s += in[i];
  int64_t ex;
  int64_t tot = block_excl_scan(s, &ex, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

__global__ void scan_partials_kernel(int64_t *part, int G, int64_t *d_total) {
  __shared__ int64_t sh[33];
  int64_t v = threadIdx.x < G ? part[threadIdx.x] : 0;
  int64_t ex;
  int64_t tot = block_excl_scan(v, &ex, sh);
  if (threadIdx.x < G) part[threadIdx.x] = ex;
  if (threadIdx.x == 0 && d_total) *d_total = tot;
}

__global__ void scan_apply_kernel(const int32_t *in, int64_t *out,
                                  const int64_t *d_n, const int64_t *part) {
  __shared__ int64_t sh[33];
  const int64_t n = *d_n;
  const int64_t G = gridDim.x;
  const int64_t chunk = (n + G - 1) / G;
  const int64_t lo = blockIdx.x * chunk;
  const int64_t hi = min(n, lo + chunk);
  int64_t carry = part[blockIdx.x];
  for (int64_t base = lo; base < hi; base += blockDim.x) {
    int64_t i = base + threadIdx.x;
    int64_t v = i < hi ? in[i] : 0;
    int64_t ex;
    int64_t tot = block_excl_scan(v, &ex, sh);
    if (i < hi) out[i] = carry + ex;
    carry += tot;
  }
}

// ---- radix sort -----------------------------------------------------------
constexpr int kRadixBits = 8;
constexpr int kRadix = 1 << kRadixBits;
constexpr int kSortThreads = 256;
constexpr int kSortItems = 8;
constexpr int kSortTile = kSortThreads * kSortItems;

__global__ void radix_upsweep(const uint64_t *keys, const int64_t *d_n,
                              int shift, uint32_t *hist, int ntiles) {
  __shared__ uint32_t h[kRadix];
  h[threadIdx.x] = 0;
  __syncthreads();
  const int64_t n = *d_n;
  const int64_t base = (int64_t)blockIdx.x * kSortTile;
  const int lane = threadIdx.x & 31;
  for (int k = 0; k < kSortItems; ++k) {
    const int64_t e = base + k * kSortThreads + threadIdx.x;
    const uint32_t d = e < n ? (uint32_t)((keys[e] >> shift) & (kRadix - 1)) : kRadix;
    const uint32_t peers = __match_any_sync(0xffffffffu, d);  // one atomic per digit and warp
    if (d < kRadix && lane == __ffs(peers) - 1) atomicAdd(&h[d], (uint32_t)__popc(peers));
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

// exclusive scan of each digit's row of tile counts (one block per digit);
// the row total goes to the last slot of the digit's totals
__global__ void __launch_bounds__(kRadix) radix_row_scan(uint32_t *hist, int ntiles,
                                                         uint32_t *digit_total) {
  __shared__ int64_t sh[33];
  uint32_t *row = hist + (int64_t)blockIdx.x * ntiles;
  int64_t carry = 0;
  for (int base = 0; base < ntiles; base += kRadix) {
    const int i = base + threadIdx.x;
    const int64_t v = i < ntiles ? row[i] : 0;
    int64_t ex;
    const int64_t tot = block_excl_scan(v, &ex, sh);
    if (i < ntiles) row[i] = (uint32_t)(carry + ex);
    carry += tot;
  }
  if (threadIdx.x == 0) digit_total[blockIdx.x] = (uint32_t)carry;
}

// Stable scatter of one tile: the tile's elements are ranked by (digit,
// position), placed digit-ordered in shared memory, then written out so that
// consecutive threads write consecutive addresses of one digit's run.
__global__ void __launch_bounds__(kSortThreads)
radix_downsweep(const uint64_t *keys, const int32_t *vals, uint64_t *okeys,
                int32_t *ovals, const int64_t *d_n, int shift,
                const uint32_t *hist, int ntiles, const uint32_t *digit_total) {
  __shared__ uint32_t s_warp[kSortThreads / 32][kRadix];
  __shared__ uint32_t s_run[kRadix];
  __shared__ uint32_t s_gbase[kRadix];  // first output index of the tile's digit d
  __shared__ uint32_t s_lbase[kRadix];  // first tile position of digit d
  __shared__ int64_t sh[33];
  __shared__ uint64_t s_key[kSortTile];
  __shared__ int32_t s_val[kSortTile];
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  s_run[t] = 0;
  {
    int64_t ex;
    block_excl_scan((int64_t)digit_total[t], &ex, sh);   // digit bases
    s_gbase[t] = (uint32_t)ex + hist[(int64_t)t * ntiles + blockIdx.x];
  }
  const int64_t n = *d_n;
  const int64_t base = (int64_t)blockIdx.x * kSortTile;
  const uint32_t lt = (1u << lane) - 1u;
  uint64_t key[kSortItems];
  int32_t val[kSortItems];
  uint32_t dig[kSortItems], rk[kSortItems];
#pragma unroll
  for (int r = 0; r < kSortItems; ++r) {
#pragma unroll
    for (int k = 0; k < kSortThreads / 32; ++k) s_warp[k][t] = 0;
    __syncthreads();
    const int64_t e = base + r * kSortThreads + t;
    const bool valid = e < n;
    key[r] = 0;
    val[r] = 0;
    uint32_t d = kRadix;  // invalid lanes form their own group
    if (valid) {
      key[r] = keys[e];
      val[r] = vals[e];
      d = (uint32_t)((key[r] >> shift) & (kRadix - 1));
    }
    dig[r] = d;
    const uint32_t peers = __match_any_sync(0xffffffffu, d);
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

}  // namespace

int p3t_scan_i32_to_i64(const int32_t *in, int64_t *out, const int64_t *d_n,
                        int64_t n_cap, int64_t *d_total, int64_t *part,
                        cudaStream_t s) {
  int G = (int)((n_cap + 4 * kScanBlock - 1) / (4 * kScanBlock));
  if (G < 1) G = 1;
  if (G > kScanMaxBlocks) G = kScanMaxBlocks;
  scan_reduce_kernel<<<G, kScanBlock, 0, s>>>(in, d_n, part);
  scan_partials_kernel<<<1, kScanBlock, 0, s>>>(part, G, d_total);
  scan_apply_kernel<<<G, kScanBlock, 0, s>>>(in, out, d_n, part);
  p3t_note_launches(3);
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
    radix_upsweep<<<(unsigned)ntiles, kSortThreads, 0, s>>>(*keys, d_n, shift,
                                                            hist, (int)ntiles);
    radix_row_scan<<<kRadix, kRadix, 0, s>>>(hist, (int)ntiles, digit_total);
    radix_downsweep<<<(unsigned)ntiles, kSortThreads, 0, s>>>(
        *keys, *vals, *keys_alt, *vals_alt, d_n, shift, hist, (int)ntiles, digit_total);
    p3t_note_launches(3);
    uint64_t *tk = *keys; *keys = *keys_alt; *keys_alt = tk;
    int32_t *tv = *vals; *vals = *vals_alt; *vals_alt = tv;
  }
  return cudaGetLastError() == cudaSuccess ? P3T_OK : P3T_ERR_CUDA;
}

// Test program: the exact conversions of the tree build (exact_conv.cuh)
// against the hardware FP64 conversions, and the cell index on the 21-bit
// grid for coordinates read from a file (the test compares those with the
// exact rational floor).
//   exact_conv_check split <count> <seed>      -> prints mismatches
//   exact_conv_check reach <count> <seed>      -> prints mismatches
//   exact_conv_check cells <in.bin> <out.bin>  -> in: n, lo, L, v[n] (double)
//                                                 out: q[n] (uint64)
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "../../paper_2007_15432_gb300/csrc/exact_conv.cuh"

// splitmix64: the test's own input generator
__host__ __device__ inline uint64_t mix64(uint64_t z) {
  z += 0x9e3779b97f4a7c15ull;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

__global__ void k_split(int64_t n, uint64_t seed, unsigned long long *bad, double *first_bad) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t r = mix64(seed + (uint64_t)i);
    double x;
    const int kind = (int)(r & 3);
    if (kind == 0) {
      x = __longlong_as_double((long long)mix64(r));  // any bit pattern
    } else if (kind == 1) {  // magnitudes of the workloads: 1e-15 .. 1e3
      const double m = 1.0 + (double)(mix64(r) >> 11) * 0x1p-53;
      x = ldexp(m, (int)((r >> 8) % 60) - 50) * ((r >> 20) & 1 ? -1.0 : 1.0);
    } else if (kind == 2) {  // halfway and near-halfway mantissas
      const uint64_t b = (mix64(r) & 0xffffffffe0000000ull) | (1ull << 28) |
                         ((r >> 9) & 1 ? 1ull : 0ull);
      x = __longlong_as_double((long long)((b & 0x800fffffffffffffull) |
                                           ((uint64_t)(950 + (r >> 40) % 191) << 52)));
    } else {  // the range edges of the integer path
      const int e = (int)((r >> 3) & 1 ? 949 + (r >> 4) % 3 : 1139 + (r >> 4) % 3);
      x = __longlong_as_double((long long)((mix64(r) & 0x800fffffffffffffull) | ((uint64_t)e << 52)));
    }
    if (x != x) continue;  // NaN
    float hi, lo;
    split_f32(x, hi, lo);
    const float h0 = (float)x;
    const float l0 = (float)(x - (double)h0);
    if (__float_as_int(hi) != __float_as_int(h0) || __float_as_int(lo) != __float_as_int(l0)) {
      if (atomicAdd(bad, 1ull) == 0ull) *first_bad = x;
    }
  }
}

// reach_cells against the FP64 expression, on radii of every magnitude and
// radii within a few ulps of whole and half cells, for boxes of many sides
__global__ void k_reach(int64_t n, uint64_t seed, unsigned long long *bad, double *first_bad) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t r = mix64(seed + (uint64_t)i);
    const double L = ldexp(1.0 + (double)(mix64(r ^ 0x5555ull) >> 11) * 0x1p-53,
                           (int)((r >> 50) % 40) - 20);
    const double u = ldexp(L, -P3T_BITS);
    double rs;
    const int kind = (int)(r & 3);
    if (kind == 0) {  // any magnitude up to beyond the cap
      rs = ldexp(1.0 + (double)(mix64(r) >> 11) * 0x1p-53, (int)((r >> 8) % 64) - 40) * u;
    } else if (kind == 1) {  // a whole number of cells, a few ulps either side
      const double m = (double)(mix64(r) % 5000000ull);
      rs = m * u;
      for (int s = 0; s < (int)((r >> 20) % 4); ++s) rs = nextafter(rs, (r >> 24) & 1 ? 0.0 : 1e300);
    } else if (kind == 2) {  // small multiples
      rs = (double)(mix64(r) % 64ull) * u * (1.0 + ldexp((double)((int)((r >> 30) % 9) - 4), -52));
    } else {  // the range edges
      rs = ldexp(1.0, (int)((r >> 8) % 6) + 19) * u * (1.0 + ldexp((double)((int)((r >> 30) % 9) - 4), -52));
    }
    if (!(rs >= 0.0)) continue;
    const int32_t got = reach_cells(rs, L, cell_scale(L));
    const double rq = ceil(rs / u) + 1.0;
    const int32_t want = rq < 8388608.0 ? (int32_t)rq : 8388608;
    if (got != want && atomicAdd(bad, 1ull) == 0ull) *first_bad = rs / u;
  }
}

__global__ void k_cells(int64_t n, double lo, double L, const double *v, uint64_t *q) {
  const CellScale cs = cell_scale(L);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    q[i] = quantise(v[i], lo, cs);
}

#define CK(x)                                                             \
  do {                                                                    \
    cudaError_t e_ = (x);                                                 \
    if (e_ != cudaSuccess) {                                              \
      fprintf(stderr, "CUDA error %s at line %d\n", cudaGetErrorString(e_), __LINE__); \
      return 2;                                                           \
    }                                                                     \
  } while (0)

int main(int argc, char **argv) {
  if (argc == 4 && !strcmp(argv[1], "split")) {
    const int64_t n = atoll(argv[2]);
    const uint64_t seed = strtoull(argv[3], nullptr, 10);
    unsigned long long *bad;
    double *fb;
    CK(cudaMalloc(&bad, sizeof(*bad)));
    CK(cudaMalloc(&fb, sizeof(*fb)));
    CK(cudaMemset(bad, 0, sizeof(*bad)));
    k_split<<<1024, 256>>>(n, seed, bad, fb);
    CK(cudaGetLastError());
    CK(cudaDeviceSynchronize());
    unsigned long long hb = 0;
    double hf = 0.0;
    CK(cudaMemcpy(&hb, bad, sizeof(hb), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(&hf, fb, sizeof(hf), cudaMemcpyDeviceToHost));
    printf("{\"checked\": %lld, \"mismatches\": %llu, \"first\": %.17g}\n", (long long)n, hb,
           hb ? hf : 0.0);
    return 0;
  }
  if (argc == 4 && !strcmp(argv[1], "reach")) {
    const int64_t n = atoll(argv[2]);
    const uint64_t seed = strtoull(argv[3], nullptr, 10);
    unsigned long long *bad;
    double *fb;
    CK(cudaMalloc(&bad, sizeof(*bad)));
    CK(cudaMalloc(&fb, sizeof(*fb)));
    CK(cudaMemset(bad, 0, sizeof(*bad)));
    k_reach<<<1024, 256>>>(n, seed, bad, fb);
    CK(cudaGetLastError());
    CK(cudaDeviceSynchronize());
    unsigned long long hb = 0;
    double hf = 0.0;
    CK(cudaMemcpy(&hb, bad, sizeof(hb), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(&hf, fb, sizeof(hf), cudaMemcpyDeviceToHost));
    printf("{\"checked\": %lld, \"mismatches\": %llu, \"first\": %.17g}\n", (long long)n, hb,
           hb ? hf : 0.0);
    return 0;
  }
  if (argc == 4 && !strcmp(argv[1], "cells")) {
    FILE *f = fopen(argv[2], "rb");
    if (!f) return 3;
    int64_t n = 0;
    double lo = 0.0, L = 0.0;
    if (fread(&n, 8, 1, f) != 1 || fread(&lo, 8, 1, f) != 1 || fread(&L, 8, 1, f) != 1 || n < 1) return 3;
    std::vector<double> v((size_t)n);
    if (fread(v.data(), 8, (size_t)n, f) != (size_t)n) return 3;
    fclose(f);
    double *dv;
    uint64_t *dq;
    CK(cudaMalloc(&dv, 8 * n));
    CK(cudaMalloc(&dq, 8 * n));
    CK(cudaMemcpy(dv, v.data(), 8 * n, cudaMemcpyHostToDevice));
    k_cells<<<256, 256>>>(n, lo, L, dv, dq);
    CK(cudaGetLastError());
    std::vector<uint64_t> q((size_t)n);
    CK(cudaMemcpy(q.data(), dq, 8 * n, cudaMemcpyDeviceToHost));
    FILE *g = fopen(argv[3], "wb");
    if (!g) return 3;
    fwrite(q.data(), 8, (size_t)n, g);
    fclose(g);
    return 0;
  }
  fprintf(stderr, "usage: exact_conv_check split <count> <seed> | cells <in> <out>\n");
  return 1;
}

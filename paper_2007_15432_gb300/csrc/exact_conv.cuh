// Exact conversions of the tree build done without FP64 arithmetic (FP64
// instructions issue at 1/64 of the FP32 rate on this part): the cell index
// of a coordinate on the 21-bit grid and the float-float split of a double.
// Header-only so that a test program can check them against the hardware
// conversions and the exact rational values.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#ifndef P3T_BITS
#define P3T_BITS 21
#define P3T_QMAX (1 << P3T_BITS)
#endif

// cell index of v: floor(d / u) of d = v - lo (rounded, the one FP64
// operation) and the cell side u = L / 2^21, the quotient taken exactly (the
// largest q with q u <= d), clamped to [0, 2^21).  With d = Md 2^Ed and
// u = Mu 2^Eu (53-bit integer mantissas), q = floor(Md 2^k / Mu), k = Ed - Eu:
// an FP32 quotient of the leading 32 bits of each mantissa is within 3 of it,
// and the remainder Md 2^k - q Mu in 64-bit integers settles it.
struct CellScale {
  uint64_t Mu;  // mantissa of L with the hidden bit
  int eL;       // biased exponent of L
  float rb;     // 1 / (leading 32 bits of Mu), rounded
};
__device__ __forceinline__ CellScale cell_scale(double L) {
  const uint64_t b = (uint64_t)__double_as_longlong(L);
  const uint64_t Mu = (b & 0xfffffffffffffull) | (1ull << 52);
  return {Mu, (int)((b >> 52) & 0x7ff), 1.0f / (float)(uint32_t)(Mu >> 21)};
}
// floor(Md 2^k / Mu) and its remainder for 0 <= k <= 22 (a quotient below
// 2^23): the FP32 estimate is within 3 of the quotient, and the remainder
// Md 2^k - q Mu, below 2^55 in magnitude, is exact modulo 2^64
__device__ __forceinline__ int32_t floor_div_cells(uint64_t Md, int k, const CellScale &cs,
                                                   int64_t &r) {
  int32_t q = (int32_t)((float)(uint32_t)(Md >> 21) * cs.rb * (float)(1u << k));
  r = (int64_t)((Md << k) - (uint64_t)(uint32_t)q * cs.Mu);
  const int64_t mu = (int64_t)cs.Mu;
#pragma unroll
  for (int it = 0; it < 4; ++it)
    if (r < 0) { r += mu; --q; }
#pragma unroll
  for (int it = 0; it < 4; ++it)
    if (r >= mu) { r -= mu; ++q; }
  return q;
}

__device__ __forceinline__ uint64_t quantise(double v, double lo, CellScale cs) {
  const double d = v - lo;
  const uint64_t bd = (uint64_t)__double_as_longlong(d);
  const int ed = (int)(bd >> 52);  // with the sign bit: >= 2048 for d < 0
  // zero or subnormal (below one cell), negative (below the corner), or
  // not finite: cell 0
  if (ed == 0 || ed >= 0x7ff) return 0;
  const uint64_t Md = (bd & 0xfffffffffffffull) | (1ull << 52);
  const int k = ed - cs.eL + P3T_BITS;  // d / u = (Md / Mu) 2^k
  if (k < 0) return 0;                   // Md / Mu < 2: below one cell
  if (k > P3T_BITS + 1) return P3T_QMAX - 1;  // at least 2^22 cells: clamped
  int64_t r;
  const int32_t q = floor_div_cells(Md, k, cs, r);
  return q < P3T_QMAX - 1 ? (uint64_t)(uint32_t)q : (uint64_t)(P3T_QMAX - 1);
}

// A node's search reach in grid cells, R = ceil(rs / u) + 1 with the FP64
// quotient (rounded to nearest) as the definition has it, capped at 2^23.
__device__ __noinline__ int32_t reach_cells_fp64(double rs, double L) {
  const double rq = ceil(rs / ldexp(L, -P3T_BITS)) + 1.0;
  return rq < 8388608.0 ? (int32_t)rq : 8388608;
}
// The same without FP64 arithmetic: the exact quotient is x = q + r / Mu
// (floor_div_cells); its FP64 rounding stays at q exactly when the fraction
// is at most half an ulp of x, 2^(floor(log2 q) - 53) (a tie rounds to the
// even q), i.e. when r <= Mu / 2^(53 - floor(log2 q)); otherwise it lies in
// (q, q + 1] and its ceiling is q + 1.  Outside 2^-900 < x < 2^21 (and for
// rs that is zero, subnormal, negative or not finite) the FP64 expression.
__device__ __forceinline__ int32_t reach_cells(double rs, double L, const CellScale &cs) {
  const uint64_t bd = (uint64_t)__double_as_longlong(rs);
  const int ed = (int)(bd >> 52);
  if (ed == 0 || ed >= 0x7ff) return reach_cells_fp64(rs, L);
  const int k = ed - cs.eL + P3T_BITS;
  if (k > P3T_BITS || k < -900) return reach_cells_fp64(rs, L);
  if (k < 0) return 2;  // 0 < x < 1: the rounded quotient is in (0, 1]
  const uint64_t Md = (bd & 0xfffffffffffffull) | (1ull << 52);
  int64_t r;
  const int32_t q = floor_div_cells(Md, k, cs, r);
  if (r == 0) return q + 1;
  if (q == 0) return 2;
  const int s = 53 - (31 - __clz(q));
  return r <= (int64_t)(cs.Mu >> s) ? q + 1 : q + 2;
}

// x = hi + lo: hi = x rounded to FP32 and lo = (x - hi) rounded to FP32,
// the values of the FP64 conversions (float)x and (float)(x - (double)hi),
// formed with 32-bit integer operations and one 32-bit integer conversion
// (FP64 instructions, and conversions from or to 64-bit integers, issue at a
// small fraction of the FP32 rate on this part).  With x = +-M 2^s (M the
// 53-bit integer mantissa): M is rounded to 24 significant bits, nearest
// even, by integer shifts (q = M / 2^29 rounded, q in [2^23, 2^24]), and hi
// = q 2^(s+29) is written directly as float bits (q = 2^24 carries into the
// exponent); the residual r = M - q 2^29 (|r| <= 2^28) converts, rounded to
// nearest, to lo 2^-s.  Where a result could leave the normal floats (|x|
// below 2^-73 or above 2^117, zero included) the FP64 conversions are taken.
// the FP64 conversions, out of line: inlined, the compiler predicates them
// into every call, and predicated-off FP64 instructions still occupy the
// FP64 pipe
__device__ __noinline__ void split_f32_fp64(double x, float &hi, float &lo) {
  hi = (float)x;
  lo = (float)(x - (double)hi);
}
__device__ __forceinline__ void split_f32(double x, float &hi, float &lo) {
  const uint64_t b = (uint64_t)__double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7ff);
  if (e < 950 || e > 1140) {
    split_f32_fp64(x, hi, lo);
    return;
  }
  const uint64_t M = (b & 0xfffffffffffffull) | (1ull << 52);
  uint32_t q = (uint32_t)(M >> 29);
  const uint32_t rem = (uint32_t)M & 0x1fffffffu;
  const bool up = rem > 0x10000000u || (rem == 0x10000000u && (q & 1u));
  q += up ? 1u : 0u;
  const int32_t r = up ? (int32_t)rem - 0x20000000 : (int32_t)rem;
  const uint32_t sgn = (uint32_t)(b >> 63) << 31;
  hi = __uint_as_float(sgn | ((uint32_t)(e - 896) << 23) + (q - (1u << 23)));
  lo = r == 0 ? 0.0f
              : __int_as_float((__float_as_int(__int2float_rn(r)) + (e - 1075) * (1 << 23)) ^
                               (int)sgn);
}

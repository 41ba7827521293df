// p3t_cutoffs_noalloc: the cut-off and search radii for callers that
// cannot allocate device memory.
//
// Some callers of this library cannot call cudaMalloc: an application that
// owns all device memory through its own pool and forbids other allocations
// (a plugin host, an embedding framework with a fixed memory budget), or a
// latency-critical loop where the device-wide synchronisation that cudaMalloc
// and cudaFree may imply would stall other work.  Such callers cannot create a
// p3t context either, because the context allocates its buffers.  This entry
// point needs no context and allocates nothing: its only scratch (the radial
// bin sums and counts and the range of the cylindrical radius) lives in a
// fixed array in device memory that every GPU loading the library holds until
// the process exits.
//
// The scratch holds at most kMaxBins radial bins.  Every call shares it and
// it keeps the contents of the last call; each call clears the part it uses
// before use.  Calls that overlap on the GPU (on different streams without an
// ordering between them) race on the scratch and must not be issued.
//
// The bin sums of |u|^2 are exact sums of fixed-point terms: each term is cut
// to a multiple of 2^-88 (|u|^2 < 2^40 assumed; a larger term saturates) and
// added as a 128-bit integer, so the order in which threads add them does not
// matter and every run gives the same bits.
#include <math.h>

#include <mutex>

#include "p3t_internal.cuh"

namespace {

constexpr int kMaxBins = 4096;           // largest vran_bins this entry point accepts
// range bits, 128-bit bin sums (low and high words), bin counts
constexpr int kScratchWords = 2 + 3 * kMaxBins;
constexpr int kSharedBins = 2048;        // bins summed per block in shared memory first
constexpr int kMaxDevices = 64;
constexpr int kBlock = 256;

}  // namespace

// 16 + 3 * 4096 * 8 = 98,320 bytes per device
static __device__ __align__(256) unsigned long long p3t_noalloc_scratch[kScratchWords];

namespace {

std::mutex g_mu;
void *g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch on the current device.  Looked up once per
// device (the first call on a device does it) with that device current.
int scratch_address(unsigned long long **out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return P3T_ERR_CUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) return P3T_ERR_INVALID;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_addr[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, p3t_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return P3T_ERR_CUDA;
    }
    g_scratch_addr[dev] = p;
  }
  *out = static_cast<unsigned long long *>(g_scratch_addr[dev]);
  return P3T_OK;
}

__device__ __forceinline__ unsigned long long nz_ord_bits(double v) {
  unsigned long long b = (unsigned long long)__double_as_longlong(v);
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ double nz_ord_double(unsigned long long b) {
  b = (b >> 63) ? (b & 0x7fffffffffffffffull) : ~b;
  return __longlong_as_double((long long)b);
}

// scratch layout: [0] min and [1] max of R_cyl (ordered bits), then per bin
// the low words [2, 2 + nb) and high words [2 + kMaxBins, ...) of the
// fixed-point sums of |u|^2, and the counts [2 + 2 kMaxBins, ...)
__global__ void nz_clear(unsigned long long *sc, int nb) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t == 0) { sc[0] = ~0ull; sc[1] = 0ull; }
  for (int k = t; k < nb; k += gridDim.x * blockDim.x) {
    sc[2 + k] = 0ull;
    sc[2 + kMaxBins + k] = 0ull;
    sc[2 + 2 * kMaxBins + k] = 0ull;
  }
}

__global__ void nz_range(int64_t n, const double *x, const double *y,
                         unsigned long long *sc) {
  unsigned long long lo = ~0ull, hi = 0ull;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long b = nz_ord_bits(sqrt(x[i] * x[i] + y[i] * y[i]));
    lo = b < lo ? b : lo;
    hi = b > hi ? b : hi;
  }
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long a = __shfl_xor_sync(0xffffffffu, lo, o);
    const unsigned long long c = __shfl_xor_sync(0xffffffffu, hi, o);
    lo = a < lo ? a : lo;
    hi = c > hi ? c : hi;
  }
  if ((threadIdx.x & 31) == 0) { atomicMin(&sc[0], lo); atomicMax(&sc[1], hi); }
}

__device__ __forceinline__ int nz_bin(double R, double Rmin, double Rmax,
                                      double lmin, double lmax, int nb) {
  int k = 0;
  if (Rmax > Rmin && R > Rmin) {
    const double t = (log(R) - lmin) / (lmax - lmin);
    const double f = floor(t * (double)nb);
    k = f < 0.0 ? 0 : (f > (double)(nb - 1) ? nb - 1 : (int)f);
  }
  return k;
}

// t >= 0 as a 128-bit count of 2^-88 (truncated; saturated at 2^128 - 1):
// the high word is floor(t 2^24), the low word the next 64 bits (both
// products by powers of two and the fraction t 2^24 - hi are exact)
__device__ __forceinline__ void nz_fixed(double t, unsigned long long &lo,
                                         unsigned long long &hi) {
  const double a = t * 16777216.0;  // t 2^(88 - 64)
  if (!(a < 18446744073709551616.0)) { lo = hi = ~0ull; return; }
  const double h = floor(a);
  hi = (unsigned long long)h;
  lo = (unsigned long long)((a - h) * 18446744073709551616.0);
}

// (lo, hi) += (a_lo, a_hi) with atomics: the carry out of the low word is
// known from its old value, so the 128-bit total is exact in any order
__device__ __forceinline__ void nz_add128(unsigned long long *lo, unsigned long long *hi,
                                          unsigned long long a_lo, unsigned long long a_hi) {
  const unsigned long long old = atomicAdd(lo, a_lo);
  const unsigned long long carry = old + a_lo < old ? 1ull : 0ull;
  if (a_hi + carry) atomicAdd(hi, a_hi + carry);
}

// random velocity u = v - sqrt(G M_* / |x|) phi_hat, |u|^2 summed per bin
// (per block in shared memory first when the bins fit)
__global__ void nz_bins(int64_t n, const double *x, const double *y,
                        const double *z, const double *vx, const double *vy,
                        const double *vz, double mu, int nb,
                        unsigned long long *sc) {
  extern __shared__ unsigned long long s_w[];
  const bool shared = nb <= kSharedBins;
  unsigned long long *s_lo = s_w, *s_hi = s_w + nb, *s_cnt = s_w + 2 * nb;
  if (shared) {
    for (int k = threadIdx.x; k < 3 * nb; k += blockDim.x) s_w[k] = 0ull;
    __syncthreads();
  }
  unsigned long long *g_lo = sc + 2, *g_hi = sc + 2 + kMaxBins, *g_cnt = sc + 2 + 2 * kMaxBins;
  const double Rmin = nz_ord_double(sc[0]), Rmax = nz_ord_double(sc[1]);
  const double lmin = log(Rmin), lmax = log(Rmax);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double R = sqrt(x[i] * x[i] + y[i] * y[i]);
    const double r = sqrt(x[i] * x[i] + y[i] * y[i] + z[i] * z[i]);
    const double vk = sqrt(mu / r);
    double px = 0.0, py = 0.0;
    if (R > 0.0) { px = -y[i] / R; py = x[i] / R; }
    const double ux = vx[i] - vk * px, uy = vy[i] - vk * py, uz = vz[i];
    const int k = nz_bin(R, Rmin, Rmax, lmin, lmax, nb);
    unsigned long long lo, hi;
    nz_fixed(ux * ux + uy * uy + uz * uz, lo, hi);
    if (shared) {
      nz_add128(&s_lo[k], &s_hi[k], lo, hi);
      atomicAdd(&s_cnt[k], 1ull);
    } else {
      nz_add128(&g_lo[k], &g_hi[k], lo, hi);
      atomicAdd(&g_cnt[k], 1ull);
    }
  }
  if (!shared) return;
  __syncthreads();
  for (int k = threadIdx.x; k < nb; k += blockDim.x) {
    if (s_cnt[k]) {
      nz_add128(&g_lo[k], &g_hi[k], s_lo[k], s_hi[k]);
      atomicAdd(&g_cnt[k], s_cnt[k]);
    }
  }
}

// r_out = max(R~cut,0 r_Hill, R~cut,1 v_ran dt), r_search = R~s,0 r_out + R~s,1 v_ran dt
__global__ void nz_final(int64_t n, const double *x, const double *y,
                         const double *z, const double *vx, const double *vy,
                         const double *vz, const double *m, p3t_params prm,
                         int nb, const unsigned long long *sc, double *r_out,
                         double *r_search) {
  const double mu = prm.G * prm.m_star;
  const double Rmin = nz_ord_double(sc[0]), Rmax = nz_ord_double(sc[1]);
  const double lmin = log(Rmin), lmax = log(Rmax);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double R = sqrt(x[i] * x[i] + y[i] * y[i]);
    const double r = sqrt(x[i] * x[i] + y[i] * y[i] + z[i] * z[i]);
    const double v2 = vx[i] * vx[i] + vy[i] * vy[i] + vz[i] * vz[i];
    const double alpha = 2.0 / r - v2 / mu;
    const double a = alpha > 0.0 ? 1.0 / alpha : r;
    const double rhill = cbrt(m[i] / (3.0 * prm.m_star)) * a;
    const int k = nz_bin(R, Rmin, Rmax, lmin, lmax, nb);
    // the bin's 128-bit sum to FP64: hi 2^-24 + lo 2^-88
    const double sum = (double)sc[2 + kMaxBins + k] * 5.9604644775390625e-08 +
                       (double)sc[2 + k] * 3.2311742677852644e-27;
    const double vr = sqrt(sum / (double)sc[2 + 2 * kMaxBins + k]);
    const double ro = prm.cutoff_mode == P3T_CUT_HILL_VRAN
                          ? fmax(prm.rcut0 * rhill, prm.rcut1 * vr * prm.dt_soft)
                          : prm.rcut0 * rhill;
    r_out[i] = ro;
    r_search[i] = prm.rs0 * ro + prm.rs1 * vr * prm.dt_soft;
  }
}

}  // namespace

extern "C" int p3t_cutoffs_noalloc(const p3t_params *prm, p3t_particles *p,
                                   void *stream) {
  if (!prm || !p || p->n < 0 || p->n >= ((int64_t)1 << 31)) return P3T_ERR_INVALID;
  if (!(prm->G > 0.0) || !(prm->m_star > 0.0) || !(prm->dt_soft > 0.0)) return P3T_ERR_INVALID;
  if (prm->vran_bins < 0 || prm->vran_bins > kMaxBins) return P3T_ERR_INVALID;
  // the shared radius needs a maximum over all particles: not offered here
  if (prm->cutoff_mode != P3T_CUT_HILL_VRAN && prm->cutoff_mode != P3T_CUT_HILL)
    return P3T_ERR_INVALID;
  if (p->n == 0) return P3T_OK;
  if (!p->x || !p->y || !p->z || !p->vx || !p->vy || !p->vz || !p->m || !p->r_out ||
      !p->r_search)
    return P3T_ERR_INVALID;
  unsigned long long *sc = nullptr;
  int rc = scratch_address(&sc);
  if (rc != P3T_OK) return rc;
  const int64_t n = p->n;
  int nb = prm->vran_bins;
  if (nb == 0) {
    const int64_t t = n / 1000;
    nb = (int)(t < 1 ? 1 : (t > 1024 ? 1024 : t));
  }
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return P3T_ERR_CUDA;
  }
  cudaStream_t s = (cudaStream_t)stream;
  int64_t g = (n + kBlock - 1) / kBlock;
  if (g > (int64_t)sms * P3T_NSM_BLOCKS) g = (int64_t)sms * P3T_NSM_BLOCKS;
  if (g < 1) g = 1;
  const double mu = prm->G * prm->m_star;
  nz_clear<<<4, kBlock, 0, s>>>(sc, nb);
  nz_range<<<(unsigned)g, kBlock, 0, s>>>(n, p->x, p->y, sc);
  const size_t smem = nb <= kSharedBins ? 3 * sizeof(unsigned long long) * nb : 0;
  nz_bins<<<(unsigned)g, kBlock, smem, s>>>(n, p->x, p->y, p->z, p->vx, p->vy, p->vz, mu,
                                            nb, sc);
  nz_final<<<(unsigned)g, kBlock, 0, s>>>(n, p->x, p->y, p->z, p->vx, p->vy, p->vz,
                                          p->m, *prm, nb, sc, p->r_out, p->r_search);
  return cudaGetLastError() == cudaSuccess ? P3T_OK : P3T_ERR_CUDA;
}

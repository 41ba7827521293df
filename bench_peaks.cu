// Device peak probe for the roofline denominators: FP32 FFMA, FP64 DFMA, FP64
// DADD and FP32 rsqrt throughput from independent dependency chains, and the
// latency of one dependent FMA chain in a single block (1 or 4 warps, 1, 8 or
// 32 active lanes a warp).
// Each thread runs 8 independent chains; one store per thread at the end (in bounds: out has grid*block elems).
#include <cstdio>
#include <cuda_runtime.h>
template<typename T> __global__ void fma_chain(T* out, int iters, T a, T b) {
  T x0 = threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
  for (int k = 0; k < iters; ++k) {
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      x0 = x0 * a + b; x1 = x1 * a + b; x2 = x2 * a + b; x3 = x3 * a + b;
      x4 = x4 * a + b; x5 = x5 * a + b; x6 = x6 * a + b; x7 = x7 * a + b;
    }
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}
__global__ void dadd_chain(double* out, int iters, double b) {
  double x0 = threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
  for (int k = 0; k < iters; ++k) {
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      x0 = x0 + b; x1 = x1 + b; x2 = x2 + b; x3 = x3 + b; x4 = x4 + b; x5 = x5 + b; x6 = x6 + b; x7 = x7 + b;
    }
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}
__global__ void rsqrt_chain(float* out, int iters) {
  float x0 = threadIdx.x + 1.f, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3;
  for (int k = 0; k < iters; ++k) {
#pragma unroll
    for (int u = 0; u < 16; ++u) { x0 = rsqrtf(x0) + 1.f; x1 = rsqrtf(x1) + 1.f; x2 = rsqrtf(x2) + 1.f; x3 = rsqrtf(x3) + 1.f; }
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3;
}
// one dependent FMA per iteration; lanes >= active return at once (out has
// >= blockDim.x elements)
template <typename T> __global__ void latency_chain(T* out, int iters, int active, T a, T b) {
  if ((int)(threadIdx.x & 31) >= active) return;
  T x = (T)threadIdx.x;
  for (int i = 0; i < iters; ++i) x = x * a + b;
  out[threadIdx.x] = x;
}
int main() {
  int dev = 0; cudaDeviceProp p; cudaGetDeviceProperties(&p, dev);
  printf("device %s SMs %d clock? cc %d.%d\n", p.name, p.multiProcessorCount, p.major, p.minor);
  const int blocks = p.multiProcessorCount * 8, threads = 256, n = blocks * threads;
  float* of; double* od; cudaMalloc(&of, n * sizeof(float)); cudaMalloc(&od, n * sizeof(double));
  cudaEvent_t e0, e1; cudaEventCreate(&e0); cudaEventCreate(&e1); float ms;
  for (int rep = 0; rep < 2; ++rep) {
    int it32 = 4096; cudaEventRecord(e0); fma_chain<float><<<blocks, threads>>>(of, it32, 0.999f, 0.001f); cudaEventRecord(e1); cudaEventSynchronize(e1); cudaEventElapsedTime(&ms, e0, e1);
    double fl = 2.0 * 8 * 16 * (double)it32 * n; printf("FP32 FFMA: %.2f TFLOP/s (%.3f ms)\n", fl / ms / 1e9, ms);
    int it64 = 128; cudaEventRecord(e0); fma_chain<double><<<blocks, threads>>>(od, it64, 0.999, 0.001); cudaEventRecord(e1); cudaEventSynchronize(e1); cudaEventElapsedTime(&ms, e0, e1);
    fl = 2.0 * 8 * 16 * (double)it64 * n; printf("FP64 DFMA: %.3f TFLOP/s (%.3f ms)\n", fl / ms / 1e9, ms);
    cudaEventRecord(e0); dadd_chain<<<blocks, threads>>>(od, it64, 0.001); cudaEventRecord(e1); cudaEventSynchronize(e1); cudaEventElapsedTime(&ms, e0, e1);
    fl = 1.0 * 8 * 16 * (double)it64 * n; printf("FP64 DADD: %.3f Gop/s (%.3f ms)\n", fl / ms / 1e6, ms);
    int itr = 1024; cudaEventRecord(e0); rsqrt_chain<<<blocks, threads>>>(of, itr); cudaEventRecord(e1); cudaEventSynchronize(e1); cudaEventElapsedTime(&ms, e0, e1);
    fl = 4.0 * 16 * (double)itr * n; printf("FP32 rsqrt(+add): %.3f Gop/s (%.3f ms)\n", fl / ms / 1e6, ms);
  }
  const int itl = 200000;
  for (int warps = 1; warps <= 4; warps *= 4)
    for (int act : {1, 8, 32}) {
      float m64 = 0.f, m32 = 0.f;
      for (int rep = 0; rep < 2; ++rep) {
        cudaEventRecord(e0); latency_chain<double><<<1, 32 * warps>>>(od, itl, act, 0.999999, 1e-9); cudaEventRecord(e1); cudaEventSynchronize(e1); cudaEventElapsedTime(&m64, e0, e1);
        cudaEventRecord(e0); latency_chain<float><<<1, 32 * warps>>>(of, itl, act, 0.999f, 1e-3f); cudaEventRecord(e1); cudaEventSynchronize(e1); cudaEventElapsedTime(&m32, e0, e1);
      }
      printf("dependent FMA, %d warp(s), %2d active lanes: FP64 %.2f ns, FP32 %.2f ns\n", warps, act,
             m64 * 1e6 / itl, m32 * 1e6 / itl);
    }
  cudaError_t err = cudaDeviceSynchronize(); printf("status %s\n", cudaGetErrorString(err));
  return err == cudaSuccess ? 0 : 1;
}

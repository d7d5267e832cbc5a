// Throughput probes of the FP64 pipes of the current device (the roofline denominators of the
// complex128 path): FP64 tensor-core mma.sync m8n8k4 and scalar FP64 fused multiply-add.
#include <cuda_runtime.h>

#include "ctx.h"

namespace {
constexpr int ITERS = 2048;

__global__ void k_probe_dmma(double* out) {
  double a = 1.0 + threadIdx.x * 1e-9, b = 1.0 - threadIdx.x * 1e-9;
  double c[8];   // distinct starting values: no two accumulator chains are identical
#pragma unroll
  for (int k = 0; k < 8; ++k) c[k] = 1e-3 * (k + 1) + 1e-12 * threadIdx.x;
  for (int i = 0; i < ITERS; ++i) {
#pragma unroll
    for (int k = 0; k < 4; ++k)
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
                   : "+d"(c[2 * k]), "+d"(c[2 * k + 1])
                   : "d"(a), "d"(b));
  }
  double s = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += c[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void k_probe_dfma(double* out, double a, double b) {
  double x[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = threadIdx.x + k;
  for (int i = 0; i < ITERS; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = fma(x[k], a, b);
  }
  double s = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += x[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}
}  // namespace

extern "C" int hsc_device_fp64_peaks(double* dmma_gflops, double* dfma_gflops) {
  if (!dmma_gflops || !dfma_gflops) return hsc_fail(nullptr, HSC_ERR_ARG, "NULL output");
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return hsc_fail(nullptr, HSC_ERR_CUDA, "no CUDA device");
  const int blocks = sms * 8, threads = 256;
  double* buf = nullptr;
  if (cudaMalloc(&buf, sizeof(double) * blocks * threads) != cudaSuccess)
    return hsc_fail(nullptr, HSC_ERR_OOM, "cudaMalloc probe buffer");
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  float best_mma = 1e30f, best_fma = 1e30f, ms = 0;
  for (int rep = 0; rep < 3; ++rep) {
    cudaEventRecord(a);
    k_probe_dmma<<<blocks, threads>>>(buf);
    cudaEventRecord(b);
    cudaEventSynchronize(b);
    cudaEventElapsedTime(&ms, a, b);
    best_mma = ms < best_mma ? ms : best_mma;
    cudaEventRecord(a);
    k_probe_dfma<<<blocks, threads>>>(buf, 0.999, 0.001);
    cudaEventRecord(b);
    cudaEventSynchronize(b);
    cudaEventElapsedTime(&ms, a, b);
    best_fma = ms < best_fma ? ms : best_fma;
  }
  cudaError_t err = cudaGetLastError();
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaFree(buf);
  if (err != cudaSuccess) return hsc_fail(nullptr, HSC_ERR_CUDA, cudaGetErrorString(err));
  const double warps = (double)blocks * (threads / 32);
  *dmma_gflops = 4.0 * ITERS * warps * 512.0 / (best_mma * 1e6);   // 8x8x4 MACs = 512 flops
  *dfma_gflops = 8.0 * ITERS * (double)blocks * threads * 2.0 / (best_fma * 1e6);
  return HSC_OK;
}

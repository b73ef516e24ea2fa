// Measured FP64 rates of the two FP64 instruction paths of the GPU, for the
// roofline of the FP64 kernels: DFMA (one fused multiply-add per thread per
// instruction) and DMMA (mma.sync m8n8k4 f64: 256 multiply-adds per warp per
// instruction). Each warp runs independent accumulator chains on register
// data (no memory traffic), so the rate is the issue / pipe rate alone.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/hqr.h"
#include "ptx.cuh"

namespace {

constexpr int kChains = 8;

__global__ void fp64_dfma_loop(int iters, double seed, double *sink) {
  double a[kChains], b = seed * 0.5 + 1.0, c = seed * 0.25 - 1.0;
#pragma unroll
  for (int q = 0; q < kChains; ++q) a[q] = seed + q + threadIdx.x;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int q = 0; q < kChains; ++q) a[q] = fma(a[q], b, c);
  }
  double s = 0.0;
#pragma unroll
  for (int q = 0; q < kChains; ++q) s += a[q];
  if (s == 12345.678) sink[threadIdx.x] = s;  // keeps the chains alive
}

__global__ void fp64_dmma_loop(int iters, double seed, double *sink) {
  double d[kChains][2];
  const double a = seed + threadIdx.x, b = seed * 0.5 + 1.0;
#pragma unroll
  for (int q = 0; q < kChains; ++q) d[q][0] = d[q][1] = seed * q;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int q = 0; q < kChains; ++q)
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
                   : "+d"(d[q][0]), "+d"(d[q][1])
                   : "d"(a), "d"(b));
  }
  double s = 0.0;
#pragma unroll
  for (int q = 0; q < kChains; ++q) s += d[q][0] + d[q][1];
  if (s == 12345.678) sink[threadIdx.x] = s;
}

__global__ void widen_f32(const float *x, double *y, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = hqr::ptx::to_f64(x[i]);
}

}  // namespace

extern "C" int hqr_widen_f32(const float *x, double *y, long long n, void *stream) {
  if (n < 0) return -3;
  if (n == 0) return HQR_SUCCESS;
  if (!x) return -1;
  if (!y) return -2;
  const long long blocks = (n + 255) / 256;
  widen_f32<<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, (cudaStream_t)stream>>>(x, y, n);
  return cudaGetLastError() == cudaSuccess ? HQR_SUCCESS : HQR_ERR_CUDA;
}

extern "C" int hqr_fp64_pipe_rates(double *dfma_tflops, double *dmma_tflops) {
  if (!dfma_tflops) return -1;
  if (!dmma_tflops) return -2;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return HQR_ERR_CUDA;
  double *sink = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaMalloc(&sink, 1024 * sizeof(double)) != cudaSuccess) return HQR_ERR_NOMEM;
  int st = HQR_SUCCESS;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) st = HQR_ERR_CUDA;
  const int threads = 256, blocks = 4 * sms, iters = 4096;
  for (int kind = 0; kind < 2 && !st; ++kind) {
    float best = 1e30f;
    for (int rep = 0; rep < 4 && !st; ++rep) {  // the first is a warm-up
      cudaEventRecord(e0, 0);
      if (kind == 0)
        fp64_dfma_loop<<<blocks, threads>>>(iters, 1.0 + rep, sink);
      else
        fp64_dmma_loop<<<blocks, threads>>>(iters, 1.0 + rep, sink);
      cudaEventRecord(e1, 0);
      float ms = 0.f;
      if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
        st = HQR_ERR_CUDA;
      else if (rep > 0 && ms < best)
        best = ms;
    }
    // multiply-adds per launch: DFMA one per thread per chain step, DMMA 256 per warp per instruction
    const double fmas = kind == 0 ? (double)blocks * threads * iters * kChains
                                  : (double)blocks * (threads / 32) * iters * kChains * 256.0;
    const double tflops = 2.0 * fmas / (best * 1e-3) / 1e12;
    if (kind == 0)
      *dfma_tflops = tflops;
    else
      *dmma_tflops = tflops;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(sink);
  return st;
}

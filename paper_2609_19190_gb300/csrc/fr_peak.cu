// fr_peak.cu -- measured issue throughput of the SM's 32-bit ALU pipes.
//
// The mapping kernel is bound by plain integer / logic / fp32 instruction
// issue (no tensor cores, little HBM traffic), so its roofline denominator is
// the rate at which the chip retires independent 32-bit lane operations.
// Nominal figures (SMs x lanes x clock) assume every lane issues every cycle;
// these kernels measure it: every thread runs kChains dependency chains of
// one operation (int32 add, int32 multiply-add, or fp32 fused multiply-add),
// with enough warps per SM to hide the pipeline latency, timed by CUDA
// events.  The integer add chains are coupled (each adds its neighbour), so
// no compiler can fold a chain into fewer operations.
#include <cstdint>

#include <cuda_runtime.h>

#include "../../include/flashmap.h"

namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 16;
constexpr int kThreads = 256;
constexpr int kBlocksPerSm = 8;  // 2048 threads per SM

__global__ void __launch_bounds__(kThreads) peak_int_kernel(uint32_t* sink, int iters,
                                                            uint32_t m) {
  uint32_t x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = threadIdx.x * 977u + c * 131u + blockIdx.x;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
#pragma unroll
      for (int c = 0; c < kChains; ++c) x[c] = x[c] * m + (uint32_t)(c + u);
  }
  uint32_t r = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) r ^= x[c];
  if (r == 0x9e3779b9u) sink[0] = r;  // keeps the chains live
}

__global__ void __launch_bounds__(kThreads) peak_add_kernel(uint32_t* sink, int iters) {
  uint32_t x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = threadIdx.x * 977u + c * 131u + blockIdx.x;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
#pragma unroll
      for (int c = 0; c < kChains; ++c) x[c] += x[(c + 1) % kChains];
  }
  uint32_t r = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) r ^= x[c];
  if (r == 0x9e3779b9u) sink[0] = r;
}

__global__ void __launch_bounds__(kThreads) peak_fp_kernel(float* sink, int iters, float m) {
  float x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = 1e-3f * (float)(threadIdx.x + c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
#pragma unroll
      for (int c = 0; c < kChains; ++c) x[c] = fmaf(x[c], m, 1e-7f * (float)(c + 1));
  }
  float r = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) r += x[c];
  if (r == 12345.678f) sink[0] = r;
}

}  // namespace

extern "C" fr_status fr_measure_alu_peak(int32_t device, double* int32_add_per_s,
                                         double* int32_mad_per_s, double* fp32_fma_per_s) {
  if (!int32_add_per_s || !int32_mad_per_s || !fp32_fma_per_s) return FR_ERR_INVALID_ARG;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
    return FR_ERR_UNSUPPORTED;
  if (cudaSetDevice(device) != cudaSuccess) return FR_ERR_CUDA;
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return FR_ERR_CUDA;
  const int grid = prop.multiProcessorCount * kBlocksPerSm;
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  void* sink = nullptr;
  fr_status st = FR_OK;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess ||
      cudaMalloc(&sink, 64) != cudaSuccess) {
    st = FR_ERR_CUDA;
  }
  const int iters = 4096;
  const double ops = (double)grid * kThreads * iters * kUnroll * kChains;
  double* const res[3] = {int32_add_per_s, int32_mad_per_s, fp32_fma_per_s};
  for (int kind = 0; kind < 3 && st == FR_OK; ++kind) {
    float best = 0.f;
    for (int rep = 0; rep < 4 && st == FR_OK; ++rep) {  // the first run warms up
      if (cudaEventRecord(e0, s) != cudaSuccess) st = FR_ERR_CUDA;
      if (kind == 0)
        peak_add_kernel<<<grid, kThreads, 0, s>>>((uint32_t*)sink, iters);
      else if (kind == 1)
        peak_int_kernel<<<grid, kThreads, 0, s>>>((uint32_t*)sink, iters, 0x9e3779b1u);
      else
        peak_fp_kernel<<<grid, kThreads, 0, s>>>((float*)sink, iters, 0.999999f);
      if (cudaGetLastError() != cudaSuccess || cudaEventRecord(e1, s) != cudaSuccess ||
          cudaEventSynchronize(e1) != cudaSuccess) {
        st = FR_ERR_CUDA;
        break;
      }
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) st = FR_ERR_CUDA;
      if (rep > 0 && (best == 0.f || ms < best)) best = ms;
    }
    if (st == FR_OK) *res[kind] = ops / (best * 1e-3);
  }
  if (sink) cudaFree(sink);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (s) cudaStreamDestroy(s);
  return st;
}

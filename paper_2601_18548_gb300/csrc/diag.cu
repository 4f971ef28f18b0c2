// Measurement aids that have no counterpart in the paper: an FP32
// fused-multiply-add loop whose rate is the roofline denominator of the FP32
// CUDA-core paths (the fused FP32 kernel and the FP32 fit GEMM).
#include "gcdf_internal.cuh"

namespace gcdf {

namespace {

constexpr int kChains = 8;   // independent FMA chains per thread (hides the FMA latency)
constexpr int kUnroll = 4;   // chain steps per loop trip: 32 FMAs per trip

__global__ void fma_rate_kernel(float* __restrict__ sink, int iters, float seed) {
  const int gid = blockIdx.x * blockDim.x + threadIdx.x;
  float a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = seed + 1e-7f * (float)(threadIdx.x + k);
  const float m = 0.9999999f, c = 1e-7f;
#pragma unroll 1
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
#pragma unroll
      for (int k = 0; k < kChains; ++k) a[k] = fmaf(a[k], m, c);
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  sink[gid] = s;
}

}  // namespace

cudaError_t launch_fma_rate(int blocks, int threads, int iters, float* sink, cudaStream_t s) {
  fma_rate_kernel<<<blocks, threads, 0, s>>>(sink, iters, 1.0f);
  return cudaGetLastError();
}

long long fma_rate_flops_per_thread(int iters) { return 2LL * kChains * kUnroll * iters; }

}  // namespace gcdf

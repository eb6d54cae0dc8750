// lbm_peak.cu -- measured arithmetic ceilings of the current GPU, used as the
// roofline denominators of ALU-bound kernels: independent FMA chains in FP64,
// FP32 and packed FP32 (two lanes per instruction, fma.rn.f32x2) over a grid of
// 8 blocks per SM, timed with CUDA events.
#include <cuda_runtime.h>

#include "lbm.h"

namespace {

constexpr int kChains = 8;

template <typename T>
__global__ void __launch_bounds__(256) fma_chains(T* out, int iters, T a, T b) {
  T acc[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) acc[c] = (T)(threadIdx.x + c);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc[c] = acc[c] * a + b;
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += acc[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// Packed FP32 chains: each instruction is two FMAs.
__global__ void __launch_bounds__(256) fma2_chains(float2* out, int iters, float2 a, float2 b) {
  float2 acc[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) acc[c] = make_float2((float)(threadIdx.x + c), (float)(threadIdx.x - c));
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc[c] = __ffma2_rn(acc[c], a, b);
  }
  float2 s = make_float2(0.0f, 0.0f);
#pragma unroll
  for (int c = 0; c < kChains; ++c) s = __fadd2_rn(s, acc[c]);
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T> void launch_chains(T* d, int grid, int block, int iters) {
  fma_chains<T><<<grid, block>>>(d, iters, (T)0.999999, (T)1e-7);
}
template <> void launch_chains<float2>(float2* d, int grid, int block, int iters) {
  fma2_chains<<<grid, block>>>(d, iters, make_float2(0.999999f, 0.999998f), make_float2(1e-7f, 2e-7f));
}

template <typename T>
int measure(int iters, double* flops, int lanes = 1) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return LBM_ECUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return LBM_ECUDA;
  const int block = 256, grid = sms * 8;
  T* d = nullptr;
  if (cudaMalloc(&d, sizeof(T) * (size_t)grid * block) != cudaSuccess) return LBM_ENOMEM;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  for (int rep = 0; rep < 4; ++rep) {  // first repetition is warm-up
    cudaEventRecord(e0, 0);
    launch_chains<T>(d, grid, block, iters);
    cudaEventRecord(e1, 0);
    cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && ms < best) best = ms;
  }
  const cudaError_t err = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(d);
  if (err != cudaSuccess) return LBM_ECUDA;
  *flops = 2.0 * lanes * kChains * (double)iters * grid * block / (best * 1e-3);
  return LBM_OK;
}

}  // namespace

extern "C" int lbm_measure_peak(int kind, double* h_flops) {
  if (!h_flops) return LBM_EINVAL;
  if (kind == 0) return measure<double>(4096, h_flops);
  if (kind == 1) return measure<float>(65536, h_flops);
  if (kind == 2) return measure<float2>(65536, h_flops, 2);
  return LBM_EINVAL;
}

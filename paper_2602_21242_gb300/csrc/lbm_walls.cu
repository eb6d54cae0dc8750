// lbm_walls.cu -- fullway bounce-back wall nodes (arXiv 2602.21242, Sec. 5.2's
// shocktube walls) for lattices created through the C ABI.
//
// A wall node does not collide: every population that arrived is sent back the
// way it came, f*_i(x) = f_ibar(x) with c_ibar = -c_i. The step kernels update
// every node; the walls kernel runs after them on the same stream and
// overwrites the wall nodes' outputs with the reversal of their pulled inputs,
// so the bulk kernels carry no per-node branch. With the buffer convention
// B_i(x) = f_i(x + c_i) (the pulled value of node x for population i sits at
// x - c_i), the wall node x writes B'_i(x) = f_ibar(x, t) = B_ibar(x + c_i).
// The reversal is a permutation, so the shifted forms (deviations from the
// rest weights, which are symmetric under c -> -c) reverse the same way, bit
// for bit.
//
// Adjoint: the transposed Jacobian of the reversal is the reversal, so at a
// wall node lambda_j(t)(x) = mu_jbar(x) = lambda_jbar(t + 1)(x - c_j).
#include <cuda_runtime.h>

#include <cstdint>

#include "lbm_device.cuh"
#include "lbm_walls.h"

namespace olbm {

namespace {

constexpr int kWallThreads = 128;

__device__ __forceinline__ int opposite(int i) {
  // Fig. 1a numbering: 1 <-> 3, 2 <-> 4, 5 <-> 7, 6 <-> 8
  return i == 0 ? 0 : (i < 5 ? ((i + 1) & 3) + 1 : ((i - 3) & 3) + 5);
}

__device__ __forceinline__ int wrap(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

// One thread per wall node; E is the element type, copied bit for bit.
// sign = +1: forward, out_i(x) = in_ibar(x + c_i); sign = -1: adjoint, out_i(x) = in_ibar(x - c_i).
template <typename E, int SIGN>
__global__ void __launch_bounds__(kWallThreads) walls_kernel(const E* __restrict__ in, E* __restrict__ out,
                                                             Geometry g, const int2* __restrict__ walls,
                                                             long long n) {
  const long long k = (long long)blockIdx.x * kWallThreads + threadIdx.x;
  if (k >= n) return;
  const int2 w = walls[k];
  const long long here = (long long)w.y * g.pitch + w.x;
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const int xs = wrap(w.x + SIGN * cx_of(i), g.nx), ys = wrap(w.y + SIGN * cy_of(i), g.ny);
    out[i * g.plane + here] = in[opposite(i) * g.plane + (long long)ys * g.pitch + xs];
  }
}

template <int SIGN>
cudaError_t launch(int elem_bytes, const void* in, void* out, const Geometry& g, const int2* walls, long long n,
                   cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const unsigned blocks = (unsigned)((n + kWallThreads - 1) / kWallThreads);
  switch (elem_bytes) {
    case 8:
      walls_kernel<uint64_t, SIGN><<<blocks, kWallThreads, 0, st>>>((const uint64_t*)in, (uint64_t*)out, g, walls, n);
      break;
    case 4:
      walls_kernel<uint32_t, SIGN><<<blocks, kWallThreads, 0, st>>>((const uint32_t*)in, (uint32_t*)out, g, walls, n);
      break;
    case 2:
      walls_kernel<uint16_t, SIGN><<<blocks, kWallThreads, 0, st>>>((const uint16_t*)in, (uint16_t*)out, g, walls, n);
      break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_walls(int elem_bytes, const void* src, void* dst, const Geometry& g, const int2* walls,
                         long long n, cudaStream_t st) {
  return launch<1>(elem_bytes, src, dst, g, walls, n, st);
}

cudaError_t launch_walls_adjoint(int elem_bytes, const void* lam_next, void* lam, const Geometry& g,
                                 const int2* walls, long long n, cudaStream_t st) {
  return launch<-1>(elem_bytes, lam_next, lam, g, walls, n, st);
}

}  // namespace olbm

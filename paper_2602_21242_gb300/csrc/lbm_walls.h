// lbm_walls.h -- fullway bounce-back wall nodes applied after a step (internal
// to liblbm.so; the public entry point is lbm_set_walls in include/lbm.h).
#pragma once

#include <cuda_runtime.h>

#include "lbm_device.cuh"

namespace olbm {

// Overwrite the outputs of the n wall nodes (x, y) of one step with the
// reversal of their pulled inputs: dst_i(x) = src_ibar(x + c_i). elem_bytes is
// the storage element size (8 FP64, 4 FP32, 2 FP16).
cudaError_t launch_walls(int elem_bytes, const void* src, void* dst, const Geometry& g, const int2* walls,
                         long long n, cudaStream_t st);

// The same for one adjoint step: lam_i(x) = lam_next_ibar(x - c_i).
cudaError_t launch_walls_adjoint(int elem_bytes, const void* lam_next, void* lam, const Geometry& g,
                                 const int2* walls, long long n, cudaStream_t st);

}  // namespace olbm

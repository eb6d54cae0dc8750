// lbm_halo.h -- halo rows of a lattice that is one slab of a larger lattice split
// along y (internal to liblbm.so; the public entry points are lbm_halo_bytes,
// lbm_halo_pack and lbm_halo_unpack in include/lbm.h).
#pragma once

#include <cuda_runtime.h>

#include "lbm_device.cuh"

namespace olbm {

// Copy out the populations that leave the slab through its faces: the top row
// (y = ny - 1) of planes 2, 5, 6 into up[3 nx] and the bottom row (y = 0) of
// planes 4, 7, 8 into down[3 nx], plane after plane, x fastest. elem_bytes is
// the storage element size (8 FP64, 4 FP32, 2 FP16); values are copied bit for
// bit.
cudaError_t launch_halo_pack(int elem_bytes, const void* state, const Geometry& g, void* up, void* down,
                             cudaStream_t st);

// The reverse: from_below[3 nx] into the top row of planes 2, 5, 6 and
// from_above[3 nx] into the bottom row of planes 4, 7, 8.
cudaError_t launch_halo_unpack(int elem_bytes, void* state, const Geometry& g, const void* from_below,
                               const void* from_above, cudaStream_t st);

}  // namespace olbm

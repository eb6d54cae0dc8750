// lbm_halo.cu -- halo rows of a slab of a lattice split along y (Eq. 1's
// streaming across the faces between slabs).
//
// A context that holds rows [y0, y1) of a larger periodic lattice steps them
// as if they were periodic on their own. Its buffer holds, at node x, the
// post-collision values that the next step pulls to x + c_i. A population with
// c_y = +1 (planes 2, 5, 6) that sits in the top row is pulled, through the
// slab's own periodic wrap, into its bottom row; in the whole lattice it
// belongs to the slab above, and the bottom row should receive the values of
// the slab below's top row instead. Likewise for c_y = -1 (planes 4, 7, 8) in
// the bottom row. So after each step every slab sends those 3 nx values per
// face to its neighbours and overwrites the same slots with what it receives:
// the next step then pulls the whole lattice's values, and so do the moments,
// state copies and diagnostics of the context, which read through the same
// pull. Only these slots move; no row is duplicated and no extra row is
// stepped.
#include <cuda_runtime.h>

#include <cstdint>

#include "lbm_halo.h"

namespace olbm {

namespace {

constexpr int kHaloThreads = 256;

// Plane of the k-th value of a face: up face 2, 5, 6; down face 4, 7, 8.
__device__ __forceinline__ int face_plane(int face, int k) {
  return face == 0 ? (k == 0 ? 2 : 4 + k) : (k == 0 ? 4 : 6 + k);
}

// One thread per value of both faces (6 nx values). PACK: state -> face
// buffers; otherwise face buffers -> state.
template <typename E, bool PACK>
__global__ void __launch_bounds__(kHaloThreads) halo_kernel(E* __restrict__ state, Geometry g, E* __restrict__ a,
                                                            E* __restrict__ b) {
  const long long n = 3LL * g.nx;
  const long long j = (long long)blockIdx.x * kHaloThreads + threadIdx.x;
  if (j >= 2 * n) return;
  const int face = j >= n;
  const long long r = face ? j - n : j;
  const int k = (int)(r / g.nx);
  const int x = (int)(r - (long long)k * g.nx);
  const int y = face == 0 ? g.ny - 1 : 0;
  E* s = state + face_plane(face, k) * g.plane + (long long)y * g.pitch + x;
  E* q = (face == 0 ? a : b) + r;
  if constexpr (PACK)
    *q = *s;
  else
    *s = *q;
}

template <bool PACK>
cudaError_t launch(int elem_bytes, void* state, const Geometry& g, void* a, void* b, cudaStream_t st) {
  const long long n = 6LL * g.nx;
  const unsigned blocks = (unsigned)((n + kHaloThreads - 1) / kHaloThreads);
  switch (elem_bytes) {
    case 8:
      halo_kernel<uint64_t, PACK><<<blocks, kHaloThreads, 0, st>>>((uint64_t*)state, g, (uint64_t*)a, (uint64_t*)b);
      break;
    case 4:
      halo_kernel<uint32_t, PACK><<<blocks, kHaloThreads, 0, st>>>((uint32_t*)state, g, (uint32_t*)a, (uint32_t*)b);
      break;
    case 2:
      halo_kernel<uint16_t, PACK><<<blocks, kHaloThreads, 0, st>>>((uint16_t*)state, g, (uint16_t*)a, (uint16_t*)b);
      break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_halo_pack(int elem_bytes, const void* state, const Geometry& g, void* up, void* down,
                             cudaStream_t st) {
  return launch<true>(elem_bytes, const_cast<void*>(state), g, up, down, st);
}

cudaError_t launch_halo_unpack(int elem_bytes, void* state, const Geometry& g, const void* from_below,
                               const void* from_above, cudaStream_t st) {
  return launch<false>(elem_bytes, state, g, const_cast<void*>(from_below), const_cast<void*>(from_above), st);
}

}  // namespace olbm

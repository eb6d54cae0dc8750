// lbm_stream.cuh -- bulk-copy pipelined step kernel for the shifted storage
// forms (arXiv 2602.21242, Eq. 1; same per-node arithmetic as the column
// kernels).
//
// Work is cut into tiles: strips of W = 2 * NC node columns [x0, x0 + W) by
// blocks of H rows; a persistent grid of CTAs takes tiles round robin. A
// producer warp streams, row by row, the nine plane segments each output row
// pulls (plane i: row y - c_iy, columns x0 - c_ix ..) into a ring of STAGES
// shared-memory slots with cp.async.bulk (TMA bulk copies, tracked by mbarrier
// transaction counts); NC consumer threads (node pairs, packed f32x2 collision)
// read the slot, collide, store the pair to global memory and release the slot.
// Each slot holds, per plane, the W-node row segment plus one 16-byte chunk on
// each side that carries the x -+ 1 neighbours (periodic in x and y: the
// producer computes the wrapped source row and the wrapped edge chunks). The
// copies need 16-byte aligned starts and sizes: nx a multiple of 8.
//
// Waits are bounded: an mbarrier wait that does not complete within ~1 s
// records an error flag and the CTA stops issuing work; the producer first
// waits (bounded as well) for the copies it already issued.
#pragma once

#include "lbm_device.cuh"

namespace olbm {

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx_arrive(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned long long* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
constexpr long long kMbarCycles = 2000000000LL;  // ~1 s at GB300 clocks
// Bounded wait for the phase with the given parity; false (and *err set) on timeout.
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity, int* err) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (clock64() - t0 < kMbarCycles)
    if (mbar_try_wait(bar, parity)) return true;
  atomicExch(err, 1);
  return false;
}
// Global -> shared bulk copy of `bytes` (multiple of 16, both addresses 16-byte aligned).
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// Grid barrier with bounded waits. count/gen/err live in device memory zeroed
// before the launch. Returns false (in every thread of the block) once any
// block has given up.
struct GridBarrier {
  unsigned count;
  unsigned gen;
  int err;
  int pad;
};
constexpr long long kBarrierCycles = 2000000000LL;  // ~1 s at GB300 clocks

__device__ __forceinline__ bool grid_sync(GridBarrier* b, unsigned nblocks) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    ok = 1;
    volatile unsigned* vgen = &b->gen;
    volatile int* verr = &b->err;
    const unsigned g = *vgen;  // generation before this block arrives
    __threadfence();           // this block's stores before its arrival
    const unsigned arrived = atomicAdd(&b->count, 1u) + 1u;
    if (arrived == nblocks) {
      b->count = 0;
      __threadfence();
      atomicAdd(&b->gen, 1u);
    } else {
      const long long t0 = clock64();
      while (*vgen == g) {
        if (*verr != 0 || clock64() - t0 > kBarrierCycles) {
          atomicExch(&b->err, 1);
          ok = 0;
          break;
        }
        __nanosleep(100);
      }
    }
    __threadfence();
    if (*verr != 0) ok = 0;
  }
  __syncthreads();
  return ok != 0;
}

__device__ __forceinline__ f32x2 lds_pair(const float* p) { return f32x2(*reinterpret_cast<const float2*>(p)); }
__device__ __forceinline__ f32x2 lds_pair(const __half* p) {
  return f32x2(__half22float2(*reinterpret_cast<const __half2*>(p)));
}
__device__ __forceinline__ f32x2 lds_two(const float* p0, const float* p1) { return f32x2(make_float2(*p0, *p1)); }
__device__ __forceinline__ f32x2 lds_two(const __half* p0, const __half* p1) {
  return f32x2(make_float2(__half2float(*p0), __half2float(*p1)));
}

// Shared-memory footprint of the ring (bytes).
template <int PREC, int NC, int STAGES> struct StreamShape {
  using S = typename Form<PREC>::S;
  static constexpr int kChunk = 16 / (int)sizeof(S);   // elements in one 16-byte chunk
  static constexpr int kW = 2 * NC;                     // nodes per row segment
  static constexpr int kSeg = kW + 2 * kChunk;          // elements per plane per slot
  static constexpr int kSlotBytes = 9 * kSeg * (int)sizeof(S);
  static constexpr int kRingBytes = STAGES * kSlotBytes;
  static constexpr int kBarBytes = 2 * STAGES * 8;
  static constexpr int kSmemBytes = kRingBytes + kBarBytes;
};

template <int MODEL, int PREC, bool DIAG, int NC, int STAGES>
__global__ void __launch_bounds__(NC + 32) step_stream_persistent_kernel(const typename Form<PREC>::S* __restrict__ src,
                                                             typename Form<PREC>::S* __restrict__ dst, Geometry g,
                                                             Coef<f32x2> c, double* __restrict__ partials, int H,
                                                             int* __restrict__ err) {
  using S = typename Form<PREC>::S;
  using Shape = StreamShape<PREC, NC, STAGES>;
  constexpr int CH = Shape::kChunk, SEG = Shape::kSeg;
  extern __shared__ __align__(128) unsigned char smem[];
  S* ring = reinterpret_cast<S*>(smem);
  unsigned long long* full = reinterpret_cast<unsigned long long*>(smem + Shape::kRingBytes);
  unsigned long long* empty = full + STAGES;

  // Persistent form. Tiles: strips of W columns x blocks of H rows, numbered
  // strip-fastest. CTA b takes tiles b, b + gridDim.x, ...; the ring's item
  // counter runs on across tiles, so a CTA fills the pipeline once.
  const int nstrips = (g.nx + Shape::kW - 1) / Shape::kW;
  const int ntiles = nstrips * ((g.ny + H - 1) / H);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int kConsumerWarps = NC / 32;
  const bool producer = warp == kConsumerWarps;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], kConsumerWarps);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  DiagAcc<f32x2> acc;
  if (producer) {
    bool ok = true;
    int k = 0;  // items (rows) issued by this CTA
    for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
      const int x0 = (tile % nstrips) * Shape::kW, y0 = (tile / nstrips) * H;
      const int w = min(Shape::kW, g.nx - x0);  // a multiple of 8
      const int rows = min(H, g.ny - y0);
      // Copy plan per plane: main segment [x0, x0 + w) always; the left chunk (ending
      // at x0 - 1, periodic) for c_ix = +1, the right chunk (starting at x0 + w) for c_ix = -1.
      const int xl = (x0 == 0) ? g.nx - CH : x0 - CH;
      const int xr = (x0 + w >= g.nx) ? 0 : x0 + w;
      const unsigned main_bytes = (unsigned)(w * sizeof(S));
      const unsigned stage_bytes = 9u * main_bytes + 6u * 16u;
      for (int r = 0; r < rows; ++r, ++k) {
        const int s = k % STAGES;
        if (k >= STAGES) ok = mbar_wait(&empty[s], (unsigned)((k / STAGES - 1) & 1), err);
        ok = __all_sync(0xffffffffu, ok);  // the whole warp leaves together
        if (!ok) break;
        const int y = y0 + r;
        S* slot = ring + (size_t)s * 9 * SEG;
        if (lane == 0) mbar_expect_tx_arrive(&full[s], stage_bytes);
        __syncwarp();
        // lanes 0..8: main segments; lanes 9..14: edge chunks of the planes with c_ix != 0
        if (lane < 15) {
          int i, part;  // part 0: main, 1: left chunk, 2: right chunk
          if (lane < 9) {
            i = lane;
            part = 0;
          } else {
            const int e = lane - 9;  // planes 1, 5, 8 take the left chunk; 3, 6, 7 the right one
            i = e == 0 ? 1 : e == 1 ? 5 : e == 2 ? 8 : e == 3 ? 3 : e == 4 ? 6 : 7;
            part = e < 3 ? 1 : 2;
          }
          int ys = y - cy_of(i);
          ys = ys < 0 ? ys + g.ny : (ys >= g.ny ? ys - g.ny : ys);
          const S* row = src + i * g.plane + (long long)ys * g.pitch;
          S* seg = slot + i * SEG;
          if (part == 0)
            bulk_g2s(seg + CH, row + x0, main_bytes, &full[s]);
          else if (part == 1)
            bulk_g2s(seg, row + xl, 16u, &full[s]);
          else
            bulk_g2s(seg + CH + w, row + xr, 16u, &full[s]);
        }
      }
    }
    // Before leaving, every copy issued must have landed (bounded).
    for (int j = (k > STAGES ? k - STAGES : 0); j < k; ++j)
      if (!__all_sync(0xffffffffu, mbar_wait(&full[j % STAGES], (unsigned)((j / STAGES) & 1), err))) break;
  } else if (threadIdx.x < NC) {
    const int xl = 2 * (int)threadIdx.x;  // local node index of the pair's first node
    bool ok = true;
    int k = 0;
    for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
      const int x0 = (tile % nstrips) * Shape::kW, y0 = (tile / nstrips) * H;
      const int w = min(Shape::kW, g.nx - x0);
      const int rows = min(H, g.ny - y0);
      const bool active = xl < w;
      for (int r = 0; r < rows; ++r, ++k) {
        const int s = k % STAGES;
        ok = __all_sync(0xffffffffu, mbar_wait(&full[s], (unsigned)((k / STAGES) & 1), err));
        if (!ok) break;
        const S* slot = ring + (size_t)s * 9 * SEG;
        f32x2 f[9];
        if (active) {
          // plane i, node x0 + xl + q: element CH + xl + q - c_ix of the plane's segment
          f[0] = lds_pair(slot + 0 * SEG + CH + xl);
          f[1] = lds_two(slot + 1 * SEG + CH + xl - 1, slot + 1 * SEG + CH + xl);
          f[2] = lds_pair(slot + 2 * SEG + CH + xl);
          f[3] = lds_two(slot + 3 * SEG + CH + xl + 1, slot + 3 * SEG + CH + xl + 2);
          f[4] = lds_pair(slot + 4 * SEG + CH + xl);
          f[5] = lds_two(slot + 5 * SEG + CH + xl - 1, slot + 5 * SEG + CH + xl);
          f[6] = lds_two(slot + 6 * SEG + CH + xl + 1, slot + 6 * SEG + CH + xl + 2);
          f[7] = lds_two(slot + 7 * SEG + CH + xl + 1, slot + 7 * SEG + CH + xl + 2);
          f[8] = lds_two(slot + 8 * SEG + CH + xl - 1, slot + 8 * SEG + CH + xl);
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);
        if (active) {
          NodeMoments<f32x2> m;
          collide<MODEL, true, f32x2>(f, c, m);
          S* q = dst + (long long)(y0 + r) * g.pitch + x0 + xl;
#pragma unroll
          for (int i = 0; i < 9; ++i) st_pair(q + i * g.plane, f[i]);
          if constexpr (DIAG) acc.add(m);
        }
      }
    }
  }
  if constexpr (DIAG) block_diag_acc(acc, partials + (long long)blockIdx.x * 5);
}

// One CTA per tile: strip blockIdx.x of W columns, rows [blockIdx.y H, + H).
// (Measured faster than the persistent form when registers allow only two
// resident CTAs per SM: overlapping CTA lifetimes hide the ring's fill.)
template <int MODEL, int PREC, bool DIAG, int NC, int STAGES>
__global__ void __launch_bounds__(NC + 32) step_stream_kernel(const typename Form<PREC>::S* __restrict__ src,
                                                             typename Form<PREC>::S* __restrict__ dst, Geometry g,
                                                             Coef<f32x2> c, double* __restrict__ partials, int H,
                                                             int* __restrict__ err) {
  using S = typename Form<PREC>::S;
  using Shape = StreamShape<PREC, NC, STAGES>;
  constexpr int CH = Shape::kChunk, SEG = Shape::kSeg;
  extern __shared__ __align__(128) unsigned char smem[];
  S* ring = reinterpret_cast<S*>(smem);
  unsigned long long* full = reinterpret_cast<unsigned long long*>(smem + Shape::kRingBytes);
  unsigned long long* empty = full + STAGES;

  const int x0 = blockIdx.x * Shape::kW;
  const int y0 = blockIdx.y * H;
  const int w = min(Shape::kW, g.nx - x0);       // nodes of this strip (a multiple of 8)
  const int rows = min(H, g.ny - y0);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int kConsumerWarps = NC / 32;
  const bool producer = warp == kConsumerWarps;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], kConsumerWarps);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  DiagAcc<f32x2> acc;
  if (producer) {
    // Copy plan per plane: main segment [x0, x0 + w) always; the left chunk (ending
    // at x0 - 1, periodic) for c_ix = +1, the right chunk (starting at x0 + w) for c_ix = -1.
    const int xl = (x0 == 0) ? g.nx - CH : x0 - CH;
    const int xr = (x0 + w >= g.nx) ? 0 : x0 + w;
    const unsigned main_bytes = (unsigned)(w * sizeof(S));
    const unsigned stage_bytes = 9u * main_bytes + 6u * 16u;
    bool ok = true;
    int issued = 0;
    for (int k = 0; k < rows && ok; ++k) {
      const int s = k % STAGES;
      if (k >= STAGES) ok = mbar_wait(&empty[s], (unsigned)((k / STAGES - 1) & 1), err);
      ok = __all_sync(0xffffffffu, ok);  // the whole warp leaves together
      if (!ok) break;
      const int y = y0 + k;
      S* slot = ring + (size_t)s * 9 * SEG;
      if (lane == 0) mbar_expect_tx_arrive(&full[s], stage_bytes);
      __syncwarp();
      // lanes 0..8: main segments; lanes 9..14: edge chunks of the planes with c_ix != 0
      if (lane < 15) {
        int i, part;  // part 0: main, 1: left chunk, 2: right chunk
        if (lane < 9) {
          i = lane;
          part = 0;
        } else {
          const int e = lane - 9;  // planes 1, 5, 8 take the left chunk; 3, 6, 7 the right one
          const int planes[6] = {1, 5, 8, 3, 6, 7};
          i = planes[e];
          part = e < 3 ? 1 : 2;
        }
        int ys = y - cy_of(i);
        ys = ys < 0 ? ys + g.ny : (ys >= g.ny ? ys - g.ny : ys);
        const S* row = src + i * g.plane + (long long)ys * g.pitch;
        S* seg = slot + i * SEG;
        if (part == 0)
          bulk_g2s(seg + CH, row + x0, main_bytes, &full[s]);
        else if (part == 1)
          bulk_g2s(seg, row + xl, 16u, &full[s]);
        else
          bulk_g2s(seg + CH + w, row + xr, 16u, &full[s]);
      }
      ++issued;
    }
    // Before leaving, every copy issued must have landed (bounded).
    for (int k = (issued > STAGES ? issued - STAGES : 0); k < issued; ++k)
      if (!__all_sync(0xffffffffu, mbar_wait(&full[k % STAGES], (unsigned)((k / STAGES) & 1), err))) break;
  } else if (threadIdx.x < NC) {
    const int t = threadIdx.x;
    const int xl = 2 * t;  // local node index of the pair's first node
    const bool active = xl < w;
    for (int k = 0; k < rows; ++k) {
      const int s = k % STAGES;
      if (!__all_sync(0xffffffffu, mbar_wait(&full[s], (unsigned)((k / STAGES) & 1), err))) break;
      const S* slot = ring + (size_t)s * 9 * SEG;
      f32x2 f[9];
      if (active) {
        // plane i, node x0 + xl + q: element CH + xl + q - c_ix of the plane's segment
        f[0] = lds_pair(slot + 0 * SEG + CH + xl);
        f[1] = lds_two(slot + 1 * SEG + CH + xl - 1, slot + 1 * SEG + CH + xl);
        f[2] = lds_pair(slot + 2 * SEG + CH + xl);
        f[3] = lds_two(slot + 3 * SEG + CH + xl + 1, slot + 3 * SEG + CH + xl + 2);
        f[4] = lds_pair(slot + 4 * SEG + CH + xl);
        f[5] = lds_two(slot + 5 * SEG + CH + xl - 1, slot + 5 * SEG + CH + xl);
        f[6] = lds_two(slot + 6 * SEG + CH + xl + 1, slot + 6 * SEG + CH + xl + 2);
        f[7] = lds_two(slot + 7 * SEG + CH + xl + 1, slot + 7 * SEG + CH + xl + 2);
        f[8] = lds_two(slot + 8 * SEG + CH + xl - 1, slot + 8 * SEG + CH + xl);
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[s]);
      if (active) {
        NodeMoments<f32x2> m;
        collide<MODEL, true, f32x2>(f, c, m);
        S* q = dst + (long long)(y0 + k) * g.pitch + x0 + xl;
#pragma unroll
        for (int i = 0; i < 9; ++i) st_pair(q + i * g.plane, f[i]);
        if constexpr (DIAG) acc.add(m);
      }
    }
  }
  if constexpr (DIAG) block_diag_acc(acc, partials + (long long)(blockIdx.y * gridDim.x + blockIdx.x) * 5);
}

}  // namespace olbm

// lbm_stream.cuh -- bulk-copy pipelined step kernel for the shifted storage
// forms (arXiv 2602.21242, Eq. 1; same per-node arithmetic as the column
// kernels).
//
// Work is cut into tiles: strips of W = 2 * NC node columns [x0, x0 + W) (FP64:
// W = NC) by blocks of H rows, one CTA per tile or a persistent grid whose CTAs
// take the next tile from a counter. A
// producer warp streams, row by row, the nine plane segments each output row
// pulls (plane i: row y - c_iy, columns x0 - c_ix ..) into a ring of STAGES
// shared-memory slots with cp.async.bulk (TMA bulk copies, tracked by mbarrier
// transaction counts); NC consumer threads (node pairs, packed f32x2 collision;
// FP64: single nodes) read the slot, collide, store to global memory and
// release the slot.
// Each slot holds, per plane, the row segment plus one 16-byte chunk on each
// side that carries the x -+ 1 neighbours (periodic in x and y: the producer
// computes the wrapped source row and the wrapped edge chunks). Bulk copies
// need 16-byte aligned starts and sizes; any nx works: tiles start on multiples
// of W, the main copy is rounded up to whole chunks (the layout's row padding
// holds the overhang, which no node reads), the chunk left of column 0 is the
// aligned chunk holding column nx - 1, and a pair whose second node lies past
// the strip stores and reduces its first node only.
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

// Programmatic dependent launch (sm_90 and later). A step kernel launched with
// the programmatic-serialization attribute may be scheduled while the previous
// kernel of its stream is finishing; every CTA of a step kernel signals at its
// start that the next grid may launch (launch_dependents), and the next grid's
// producer waits for the previous grid to complete, its writes visible, before
// it reads anything that grid wrote (griddepcontrol.wait, a no-op for a kernel
// launched without the attribute). The consumers touch global memory only
// after the producer's copies, so they follow the wait. What overlaps is the
// next grid's launch and set-up (CTA placement, mbarrier initialisation) with
// the previous grid's last CTAs.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

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

// Resident CTAs per SM the pipeline kernels ask the compiler to allow for:
// three when a CTA of NC + 32 threads at 72 registers a thread fits three
// times in the register file (NC = 256: the ring then also fits three times).
// Without the bound the FP16 form's diagnostics variant took 78 registers and
// ran two CTAs a SM (measured at 4096^2: 113.7 GLUPS, against 118.8 with it).
#ifndef OLBM_STREAM_MINB256
#define OLBM_STREAM_MINB256 3
#endif
template <int NC> constexpr int stream_min_blocks() {
  return (NC + 32) * 3 * 72 <= 65536 && NC >= 256 ? OLBM_STREAM_MINB256 : 1;
}

// Shared-memory footprint of the ring (bytes).
template <int PREC, int NC, int STAGES> struct StreamShape {
  using S = typename Form<PREC>::S;
  static constexpr int kChunk = 16 / (int)sizeof(S);   // elements in one 16-byte chunk
  static constexpr int kW = PREC == 0 ? NC : 2 * NC;    // nodes per row segment (FP64: one per consumer)
  static constexpr int kSeg = kW + 2 * kChunk;          // elements per plane per slot
  static constexpr int kSlotBytes = 9 * kSeg * (int)sizeof(S);
  static constexpr int kRingBytes = STAGES * kSlotBytes;
  static constexpr int kBarBytes = 2 * STAGES * 8;
  static constexpr int kSmemBytes = kRingBytes + kBarBytes;
};

// Copy plan of one tile: columns [x0, x0 + w) of a lattice of any width. A
// row's plane segment holds the main copy (wr = w rounded up to whole 16-byte
// chunks) at elements [CH, CH + wr), the left chunk at [0, CH) and the right
// chunk at [CH + wr, CH + wr + CH): sub = wr + 2 CH elements. A slot's plane
// segment (SEG elements) holds R = SEG / sub consecutive rows side by side, so
// narrow strips (the last strip of a lattice, small domains of a batch) still
// fill the ring's slots.
template <int CH> struct TilePlan {
  int w, wr, sub, R;
  int src_l, src_r;  // first source column of the left / right chunk
  int lidx;          // element of a row's segment holding column x0 - 1 (periodic)
  __device__ __forceinline__ TilePlan(const Geometry& g, int x0, int W, int SEG) {
    w = min(W, g.nx - x0);
    wr = (w + CH - 1) / CH * CH;
    sub = wr + 2 * CH;
    R = max(1, SEG / sub);
    if (x0 == 0) {
      src_l = (g.nx - 1) / CH * CH;  // the aligned chunk holding column nx - 1
      lidx = g.nx - 1 - src_l;
    } else {
      src_l = x0 - CH;
      lidx = CH - 1;
    }
    src_r = (x0 + w >= g.nx) ? 0 : x0 + w;
  }
};

// The ring of one CTA: STAGES slots, a full and an empty mbarrier per slot, and
// the count of ring items this thread has issued (producer) or consumed.
template <int PREC, int NC, int STAGES> struct Pipeline {
  using S = typename Form<PREC>::S;
  using Shape = StreamShape<PREC, NC, STAGES>;
  static constexpr int CH = Shape::kChunk, SEG = Shape::kSeg, W = Shape::kW;
  static constexpr int kConsumerWarps = NC / 32;
  S* ring;
  unsigned long long* full;
  unsigned long long* empty;
  int k = 0;

  __device__ __forceinline__ explicit Pipeline(unsigned char* smem)
      : ring(reinterpret_cast<S*>(smem)),
        full(reinterpret_cast<unsigned long long*>(smem + Shape::kRingBytes)),
        empty(reinterpret_cast<unsigned long long*>(smem + Shape::kRingBytes) + STAGES) {}

  // Thread 0 initialises the barriers; the caller synchronises the block after.
  __device__ __forceinline__ void init() {
    if (threadIdx.x == 0) {
      for (int s = 0; s < STAGES; ++s) {
        mbar_init(&full[s], 1);
        mbar_init(&empty[s], kConsumerWarps);
      }
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
  }

  // Producer warp: stream rows [y0, y0 + rows) of the tile at column x0, R rows
  // a slot. With tags, each slot's entry tags[s] is set to `tag` before the slot
  // is armed (the consumers read it once the slot is full). Returns false (in the
  // whole warp) once a bounded wait gave up.
  __device__ __forceinline__ bool produce(const S* __restrict__ src, const Geometry& g, int x0, int y0, int rows,
                                          int lane, int* err, volatile int* tags = nullptr, int tag = 0) {
    const TilePlan<CH> p(g, x0, W, SEG);
    const unsigned main_bytes = (unsigned)(p.wr * (int)sizeof(S));
    const unsigned row_bytes = 9u * main_bytes + 6u * 16u;
    for (int r0 = 0; r0 < rows; r0 += p.R, ++k) {
      const int nr = min(p.R, rows - r0);
      const int s = k % STAGES;
      bool ok = true;
      if (k >= STAGES) ok = mbar_wait(&empty[s], (unsigned)((k / STAGES - 1) & 1), err);
      if (!__all_sync(0xffffffffu, ok)) return false;  // the whole warp leaves together
      S* slot = ring + (size_t)s * 9 * SEG;
      if (lane == 0) {
        if (tags != nullptr) tags[s] = tag;
        mbar_expect_tx_arrive(&full[s], (unsigned)nr * row_bytes);
      }
      __syncwarp();
      // 15 copies per row: the main segments of the nine planes, then the edge chunks of
      // the planes with c_ix != 0 (planes 1, 5, 8 the left chunk, 3, 6, 7 the right one).
      // Operands are selected without branches; a slot of one row (full strips) takes
      // one copy per lane without a loop, so the ring fills as fast as it can.
      auto copy = [&](int j, int c) {
        const int e = c - 9;
        const bool main = c < 9, left = e < 3;
        const int i = main ? c : (int)((0x763851u >> (4 * e)) & 15u);
        int ys = y0 + r0 + j - cy_of(i);
        ys = ys < 0 ? ys + g.ny : (ys >= g.ny ? ys - g.ny : ys);
        const int dst_off = j * p.sub + (main ? CH : (left ? 0 : CH + p.wr));
        const int src_col = main ? x0 : (left ? p.src_l : p.src_r);
        const unsigned bytes = main ? main_bytes : 16u;
        bulk_g2s(slot + i * SEG + dst_off, src + i * g.plane + (long long)ys * g.pitch + src_col, bytes, &full[s]);
      };
      if (nr == 1) {
        if (lane < 15) copy(0, lane);
      } else {
        for (int q = lane; q < 15 * nr; q += 32) copy(q / 15, q % 15);
      }
    }
    return true;
  }

  // Producer warp, before leaving: every copy issued must have landed (bounded).
  __device__ __forceinline__ void drain(int* err) {
    for (int j = (k > STAGES ? k - STAGES : 0); j < k; ++j)
      if (!__all_sync(0xffffffffu, mbar_wait(&full[j % STAGES], (unsigned)((j / STAGES) & 1), err))) break;
  }

  // Consumer thread t: the pair of local nodes xl, xl + 1 of row j of each slot
  // (t = j * ceil(w / 2) + xl / 2); collide the tile's rows.
  template <int MODEL, bool DIAG>
  __device__ __forceinline__ bool consume(S* __restrict__ dst, const Geometry& g, const Coef<f32x2>& c, int x0,
                                          int y0, int rows, int t, int lane, DiagAcc<f32x2>& acc, int* err) {
    // A full strip (one row a slot, every consumer thread a whole pair) takes a
    // path without the per-pair tests of partial strips.
    const TilePlan<CH> p(g, x0, W, SEG);
    if (p.w == W && p.R == 1) return consume_tile<MODEL, DIAG, true>(dst, g, c, p, x0, y0, rows, t, lane, acc, err);
    return consume_tile<MODEL, DIAG, false>(dst, g, c, p, x0, y0, rows, t, lane, acc, err);
  }

  template <int MODEL, bool DIAG, bool FULL>
  __device__ __forceinline__ bool consume_tile(S* __restrict__ dst, const Geometry& g, const Coef<f32x2>& c,
                                               const TilePlan<CH>& p, int x0, int y0, int rows, int t, int lane,
                                               DiagAcc<f32x2>& acc, int* err) {
    const int ppr = FULL ? NC : (p.w + 1) / 2;  // pairs per row
    const int j = FULL ? 0 : t / ppr;
    const int xl = 2 * (t - j * ppr);
    const bool whole = FULL || xl + 1 < p.w;  // both nodes of the pair lie in the strip
    // segment elements of the pair's nodes and of their x -+ 1 neighbours
    const int base = j * p.sub;
    const int iM = base + CH + xl;
    const int iL = xl == 0 ? base + p.lidx : iM - 1;
    const int iR0 = whole ? iM + 1 : base + CH + p.wr;
    const int iR1 = xl + 2 < p.w ? iM + 2 : base + CH + p.wr;
    for (int r0 = 0; r0 < rows; r0 += (FULL ? 1 : p.R), ++k) {
      const bool active = FULL || j < min(p.R, rows - r0);
      const int s = k % STAGES;
      if (!__all_sync(0xffffffffu, mbar_wait(&full[s], (unsigned)((k / STAGES) & 1), err))) return false;
      const S* slot = ring + (size_t)s * 9 * SEG;
      f32x2 f[9];
      if (active) {
        f[0] = lds_pair(slot + 0 * SEG + iM);
        f[1] = lds_two(slot + 1 * SEG + iL, slot + 1 * SEG + iM);
        f[2] = lds_pair(slot + 2 * SEG + iM);
        f[3] = lds_two(slot + 3 * SEG + iR0, slot + 3 * SEG + iR1);
        f[4] = lds_pair(slot + 4 * SEG + iM);
        f[5] = lds_two(slot + 5 * SEG + iL, slot + 5 * SEG + iM);
        f[6] = lds_two(slot + 6 * SEG + iR0, slot + 6 * SEG + iR1);
        f[7] = lds_two(slot + 7 * SEG + iR0, slot + 7 * SEG + iR1);
        f[8] = lds_two(slot + 8 * SEG + iL, slot + 8 * SEG + iM);
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[s]);
      if (active) {
        collide<MODEL, true, f32x2>(f, c, [&](NodeMoments<f32x2> m) {
          if constexpr (DIAG) {
            if (!whole) {  // the pair's second node lies past the strip
              m.m0.v.y = 0.0f;
              m.jx.v.y = 0.0f;
              m.jy.v.y = 0.0f;
              m.ux.v.y = 0.0f;
              m.uy.v.y = 0.0f;
            }
            acc.add(m);
          }
        });
        S* q = dst + (long long)(y0 + r0 + j) * g.pitch + x0 + xl;
        if (whole) {
#pragma unroll
          for (int i = 0; i < 9; ++i) st_pair(q + i * g.plane, f[i]);
        } else {
#pragma unroll
          for (int i = 0; i < 9; ++i) st_t(q + i * g.plane, f[i].v.x);
        }
      }
    }
    return true;
  }

  // FP64 storage (PREC 0): consumer thread t updates local node xl of row j of
  // each slot (t = j w + xl) in FP64, one node a thread.
  template <int MODEL, bool DIAG>
  __device__ __forceinline__ bool consume_f64(double* __restrict__ dst, const Geometry& g, const Coef<double>& c,
                                              int x0, int y0, int rows, int t, int lane, DiagAcc<double>& acc,
                                              int* err) {
    static_assert(PREC == 0, "one node a consumer thread is the FP64 layout");
    const TilePlan<CH> p(g, x0, W, SEG);
    const int j = t / p.w;
    const int xl = t - j * p.w;
    const int base = j * p.sub;
    const int iM = base + CH + xl;
    const int iL = xl == 0 ? base + p.lidx : iM - 1;
    const int iR = xl + 1 < p.w ? iM + 1 : base + CH + p.wr;
    int mode = 0;  // which products this warp's nodes take (see collide)
    for (int r0 = 0; r0 < rows; r0 += p.R, ++k) {
      const bool active = j < min(p.R, rows - r0);
      const int s = k % STAGES;
      if (!__all_sync(0xffffffffu, mbar_wait(&full[s], (unsigned)((k / STAGES) & 1), err))) return false;
      const double* slot = ring + (size_t)s * 9 * SEG;
      double f[9];
      if (active) {
        f[0] = slot[0 * SEG + iM];
        f[1] = slot[1 * SEG + iL];
        f[2] = slot[2 * SEG + iM];
        f[3] = slot[3 * SEG + iR];
        f[4] = slot[4 * SEG + iM];
        f[5] = slot[5 * SEG + iL];
        f[6] = slot[6 * SEG + iR];
        f[7] = slot[7 * SEG + iR];
        f[8] = slot[8 * SEG + iL];
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[s]);
      if (active) {
        collide<MODEL, false, double>(
            f, c,
            [&](const NodeMoments<double>& m) {
              if constexpr (DIAG) acc.add(m);
            },
            KeepInputs(), &mode);
        double* q = dst + (long long)(y0 + r0 + j) * g.pitch + x0 + xl;
#pragma unroll
        for (int i = 0; i < 9; ++i) q[i * g.plane] = f[i];
      }
    }
    return true;
  }
};

// Persistent form over one lattice. Tiles: strips of W columns x blocks of H
// rows, numbered strip-fastest. A CTA's producer takes the next tile from the
// counter sched[0] when it has issued the last one, tags the ring slots with it
// and closes with a slot tagged -1; the consumers follow the tags. The ring's
// item counter runs on across tiles, so a CTA fills the pipeline once. The
// last CTA to finish (counted in sched[1]) zeroes both counters for the next
// launch.
template <int MODEL, int PREC, bool DIAG, int NC, int STAGES>
__global__ void __launch_bounds__(NC + 32, stream_min_blocks<NC>()) step_stream_persistent_kernel(const typename Form<PREC>::S* __restrict__ src,
                                                                         typename Form<PREC>::S* __restrict__ dst,
                                                                         Geometry g, Coef<f32x2> c,
                                                                         double* __restrict__ partials, int H,
                                                                         int* __restrict__ err, int* sched) {
  using P = Pipeline<PREC, NC, STAGES>;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ int tags[STAGES];
  P pipe(smem);
  pipe.init();
  __syncthreads();
  pdl_launch_dependents();
  const int nstrips = (g.nx + P::W - 1) / P::W;
  const int ntiles = nstrips * ((g.ny + H - 1) / H);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  DiagAcc<f32x2> acc;
  if (warp == P::kConsumerWarps) {
    pdl_wait();  // the tile counter and src belong to the previous step until it completes
    for (;;) {
      int tile = 0;
      if (lane == 0) tile = atomicAdd(&sched[0], 1);
      tile = __shfl_sync(0xffffffffu, tile, 0);
      if (tile >= ntiles) {  // close: a slot without data, tagged -1
        const int q = pipe.k % STAGES;
        bool ok = true;
        if (pipe.k >= STAGES) ok = mbar_wait(&pipe.empty[q], (unsigned)((pipe.k / STAGES - 1) & 1), err);
        if (__all_sync(0xffffffffu, ok) && lane == 0) {
          tags[q] = -1;
          mbar_arrive(&pipe.full[q]);
        }
        ++pipe.k;
        break;
      }
      const int x0 = (tile % nstrips) * P::W, y0 = (tile / nstrips) * H;
      if (!pipe.produce(src, g, x0, y0, min(H, g.ny - y0), lane, err, tags, tile)) break;
    }
    pipe.drain(err);
  } else if (threadIdx.x < NC) {
    for (;;) {
      const int q = pipe.k % STAGES;
      if (!__all_sync(0xffffffffu, mbar_wait(&pipe.full[q], (unsigned)((pipe.k / STAGES) & 1), err))) break;
      const int tile = *(volatile int*)&tags[q];
      if (tile < 0) {
        __syncwarp();
        if (lane == 0) mbar_arrive(&pipe.empty[q]);
        ++pipe.k;
        break;
      }
      const int x0 = (tile % nstrips) * P::W, y0 = (tile / nstrips) * H;
      if (!pipe.template consume<MODEL, DIAG>(dst, g, c, x0, y0, min(H, g.ny - y0), threadIdx.x, lane, acc, err))
        break;
    }
  }
  if constexpr (DIAG) block_diag_acc(acc, partials + (long long)blockIdx.x * 5);
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(&sched[1], 1) == (int)gridDim.x - 1) {
      atomicExch(&sched[0], 0);
      atomicExch(&sched[1], 0);
    }
  }
}

// One CTA per tile: strip blockIdx.x of W columns, rows [blockIdx.y H, + H).
// (Measured faster than the persistent form when registers allow only two
// resident CTAs per SM: overlapping CTA lifetimes hide the ring's fill.)
template <int MODEL, int PREC, bool DIAG, int NC, int STAGES>
__global__ void __launch_bounds__(NC + 32, stream_min_blocks<NC>()) step_stream_kernel(const typename Form<PREC>::S* __restrict__ src,
                                                             typename Form<PREC>::S* __restrict__ dst, Geometry g,
                                                             Coef<f32x2> c, double* __restrict__ partials, int H,
                                                             int* __restrict__ err) {
  using P = Pipeline<PREC, NC, STAGES>;
  extern __shared__ __align__(128) unsigned char smem[];
  P pipe(smem);
  pipe.init();
  __syncthreads();
  pdl_launch_dependents();
  const int x0 = blockIdx.x * P::W, y0 = blockIdx.y * H;
  const int rows = min(H, g.ny - y0);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  DiagAcc<f32x2> acc;
  if (warp == P::kConsumerWarps) {
    pdl_wait();
    pipe.produce(src, g, x0, y0, rows, lane, err);
    pipe.drain(err);
  } else if (threadIdx.x < NC) {
    pipe.template consume<MODEL, DIAG>(dst, g, c, x0, y0, rows, threadIdx.x, lane, acc, err);
  }
  if constexpr (DIAG) block_diag_acc(acc, partials + (long long)(blockIdx.y * gridDim.x + blockIdx.x) * 5);
}

// FP64 storage, one CTA per tile of W = NC columns: the same producer, one
// node a consumer thread (compiled for four resident CTAs: 96 registers).
template <int MODEL, bool DIAG, int NC, int STAGES>
__global__ void __launch_bounds__(NC + 32, 4) step_stream_f64_kernel(const double* __restrict__ src,
                                                                      double* __restrict__ dst, Geometry g,
                                                                      Coef<double> c, double* __restrict__ partials,
                                                                      int H, int* __restrict__ err) {
  using P = Pipeline<0, NC, STAGES>;
  extern __shared__ __align__(128) unsigned char smem[];
  P pipe(smem);
  pipe.init();
  __syncthreads();
  pdl_launch_dependents();
  const int x0 = blockIdx.x * P::W, y0 = blockIdx.y * H;
  const int rows = min(H, g.ny - y0);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  DiagAcc<double> acc;
  if (warp == P::kConsumerWarps) {
    pdl_wait();
    pipe.produce(src, g, x0, y0, rows, lane, err);
    pipe.drain(err);
  } else if (threadIdx.x < NC) {
    pipe.template consume_f64<MODEL, DIAG>(dst, g, c, x0, y0, rows, threadIdx.x, lane, acc, err);
  }
  if constexpr (DIAG) block_diag_acc(acc, partials + (long long)(blockIdx.y * gridDim.x + blockIdx.x) * 5);
}

}  // namespace olbm

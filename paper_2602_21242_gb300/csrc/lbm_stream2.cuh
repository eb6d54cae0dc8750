// lbm_stream2.cuh -- two steps of Eq. 1 per launch for the shifted storage
// forms (temporal blocking of the bulk-copy pipeline; same per-node arithmetic
// and the same rounding to the storage type between the steps, so the result is
// bit-identical to two single steps).
//
// A CTA owns output columns [x0, x0 + w) and rows [y0, y0 + H) of step t + 1.
// They pull step t's post-collision values s1 at rows y0 - 1 .. y0 + H and
// columns x0 - 1 .. x0 + w, which pull the stored state at rows y0 - 2 ..
// y0 + H + 1 and columns x0 - 2 .. x0 + w + 1. The producer warp streams, for
// each s1 row, the nine pulled plane rows of those columns into a ring of
// STAGES slots: per plane the columns inside the lattice from the 16-byte
// aligned chunk at or left of x0 - 2 (rounded up into the row padding at the
// right end), and, where the range wraps around the lattice, the aligned
// chunk(s) holding columns nx - 2 and nx - 1 (left of column 0) and the chunk
// of columns 0 .. into two halo areas after the main part, so any width works.
// Consumer thread t computes the s1 node pair (x0 - 1 + 2t, x0 + 2t), rounds it
// to the storage type into a four-row window in shared memory and, once every
// consumer warp has written s1 row r, the output pair (x0 + 2t, x0 + 2t + 1) of
// row r - 1 from the window. The window's four rows need one wait a row: s1 row
// r + 1 overwrites row r - 3, which the last read (output row r - 2) finished
// before its warp wrote s1 row r.
//
// With NC consumers a full strip is w = 2 NC - 2 columns (the s1 range is two
// columns wider). The consumer pairs whose columns wrap (the first pair of the
// first strip, the last ones of the strip that reaches nx) read element by
// element through the halo areas; the others read aligned pairs from the main
// part. On odd widths the last s1 and output pairs carry a node past the range
// in their second lane, which is neither stored nor counted. s1 rows and
// columns outside the tile are computed in every tile that needs them (2 rows
// and 2 columns of each tile, about 1/H + 1/w more collisions) and counted in
// the diagnostics of step t once, by the tile that owns them.
//
// Every wait is bounded (ring mbarriers and the window's mbarriers). A warp
// whose wait gave up records the error and stops waiting and computing; the
// other warps then give up at their next wait. No named barrier is used, so no
// warp can be left waiting for one that has left.
#pragma once

#include "lbm_kernels.cuh"

namespace olbm {

template <int PREC, int NC, int STAGES> struct Stream2Shape {
  using S = typename Form<PREC>::S;
  static constexpr int CH = 16 / (int)sizeof(S);                // elements in one 16-byte chunk
  static constexpr int W = 2 * NC - 2;                          // output columns of a full strip
  static constexpr int kMain = (W + 4 + CH - 1) / CH * CH + CH;  // main part: columns from an aligned start
  static constexpr int kSeg = kMain + 3 * CH;                    // + left halo (two chunks) + right halo (one)
  static constexpr int kWin = 2 * NC;                           // window elements per plane (s1 columns)
  static constexpr int kSlotBytes = 9 * kSeg * (int)sizeof(S);
  static constexpr int kRingBytes = STAGES * kSlotBytes;
  static constexpr int kWinBytes = 4 * 9 * kWin * (int)sizeof(S);
  static constexpr int kBarBytes = (2 * STAGES + 4) * 8;
  static constexpr int kSmemBytes = kRingBytes + kWinBytes + kBarBytes;
  static_assert(kSlotBytes % 16 == 0 && kWinBytes % 16 == 0, "16-byte aligned ring and window");
};

__device__ __forceinline__ int floor_div(int a, int b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }

template <int PREC, int NC, int STAGES> struct Pipeline2 {
  using S = typename Form<PREC>::S;
  using Shape = Stream2Shape<PREC, NC, STAGES>;
  static constexpr int CH = Shape::CH, SEG = Shape::kSeg, MAIN = Shape::kMain, WIN = Shape::kWin, W = Shape::W;
  static constexpr int kConsumerWarps = NC / 32;
  S* ring;
  S* win;
  unsigned long long* full;
  unsigned long long* empty;
  unsigned long long* wbar;  // [4]: s1 row of window slot q written by every consumer warp
  int k = 0;                 // ring items issued (producer) or consumed
  int kw = 0;                // window rows written by this CTA's consumers before the current tile

  __device__ __forceinline__ explicit Pipeline2(unsigned char* smem)
      : ring(reinterpret_cast<S*>(smem)),
        win(reinterpret_cast<S*>(smem + Shape::kRingBytes)),
        full(reinterpret_cast<unsigned long long*>(smem + Shape::kRingBytes + Shape::kWinBytes)),
        empty(full + STAGES),
        wbar(full + 2 * STAGES) {}

  __device__ __forceinline__ void init() {
    if (threadIdx.x == 0) {
      for (int s = 0; s < STAGES; ++s) {
        mbar_init(&full[s], 1);
        mbar_init(&empty[s], kConsumerWarps);
      }
      for (int q = 0; q < 4; ++q) mbar_init(&wbar[q], kConsumerWarps);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
  }

  // Producer warp: the pulled rows of s1 rows y0 - 1 .. y0 + rows, one slot each.
  // CONTIG (nx a multiple of the chunk): per plane the columns [xa, xe) from the
  // aligned chunk at or left of x0 - 2 to past x0 + w + 1, contiguous, the parts
  // left of 0 and right of nx copied from the other end of the row (aligned there
  // too). Otherwise: the main part [m0, m1) of the columns inside the lattice
  // (clipped at 0 and at the padded row end), then, if x0 == 0, the chunks
  // [a0, a1 + CH) holding columns nx - 2 and nx - 1 at element MAIN, and, if the
  // range passes nx, the chunk of columns 0 .. CH - 1 at element MAIN + 2 CH.
  // With tags (a CTA taking several tiles), each slot's tags entry is set to `tag`
  // before the slot is armed.
  template <bool CONTIG>
  __device__ __forceinline__ bool produce(const S* __restrict__ src, const Geometry& g, int x0, int w, int y0,
                                          int rows, int lane, int* err, volatile int* tags = nullptr,
                                          int tag = 0) {
    const int xa = floor_div(x0 - 2, CH) * CH;
    const int xe = (x0 + w + 2 + CH - 1) / CH * CH;
    const int nxr = (g.nx + CH - 1) / CH * CH;  // row padding holds the overhang
    const int m0 = xa < 0 ? 0 : xa, m1 = min(xe, CONTIG ? g.nx : nxr);
    // (a lattice one column wide has no other columns: its main part holds column 0)
    const bool left = xa < 0 && g.nx > 1, right = (CONTIG ? xe > g.nx : x0 + w + 2 > g.nx) && g.nx > 1;
    const int a0 = CONTIG ? xa + g.nx : floor_div(g.nx - 2, CH) * CH;
    const int a1 = CONTIG ? g.nx - CH : (g.nx - 1) / CH * CH;
    const int llen = a1 + CH - a0, rlen = CONTIG ? xe - g.nx : CH;
    const int lcol = CONTIG ? 0 : MAIN, rcol = CONTIG ? g.nx - xa : MAIN + 2 * CH;
    const int np = 1 + (left ? 1 : 0) + (right ? 1 : 0);
    const unsigned plane_elems = (unsigned)(m1 - m0) + (left ? (unsigned)llen : 0u) + (right ? (unsigned)rlen : 0u);
    const unsigned row_bytes = 9u * plane_elems * (unsigned)sizeof(S);
    for (int it = 0; it < rows + 2; ++it, ++k) {
      const int s = k % STAGES;
      bool ok = true;
      if (k >= STAGES) ok = mbar_wait(&empty[s], (unsigned)((k / STAGES - 1) & 1), err);
      if (!__all_sync(0xffffffffu, ok)) return false;
      S* slot = ring + (size_t)s * 9 * SEG;
      if (lane == 0) {
        if (tags != nullptr) tags[s] = tag;
        mbar_expect_tx_arrive(&full[s], row_bytes);
      }
      __syncwarp();
      if (lane < 9 * np) {
        const int i = lane / np;
        int p = lane - i * np;  // piece 0 the main part, 1 the left part (if any), 2 the right part
        if (p == 1 && !left) p = 2;
        const int gcol = p == 0 ? m0 : (p == 1 ? a0 : 0);
        const int scol = p == 0 ? m0 - xa : (p == 1 ? lcol : rcol);
        const int len = p == 0 ? m1 - m0 : (p == 1 ? llen : rlen);
        int ys = (y0 - 1 + it - cy_of(i)) % g.ny;
        if (ys < 0) ys += g.ny;
        bulk_g2s(slot + i * SEG + scol, src + i * g.plane + (long long)ys * g.pitch + gcol,
                 (unsigned)len * (unsigned)sizeof(S), &full[s]);
      }
    }
    return true;
  }

  __device__ __forceinline__ void drain(int* err) {
    for (int j = (k > STAGES ? k - STAGES : 0); j < k; ++j)
      if (!__all_sync(0xffffffffu, mbar_wait(&full[j % STAGES], (unsigned)((j / STAGES) & 1), err))) break;
  }

  // The nine pulled values of a node pair whose first node's c_ix = 0 value sits
  // at the odd element e0 of each plane (stride `plane` elements): planes with
  // c_ix = 0 at e0, e0 + 1 (they straddle a pair boundary and are read element by
  // element), c_ix = +1 at e0 - 1, e0 and c_ix = -1 at e0 + 1, e0 + 2 (aligned
  // pairs). From the window (WINDOW), plane i comes from the slot of s1 row
  // it - 1 - c_iy; from the ring, all planes from the one slot at base.
  template <bool WINDOW>
  __device__ static __forceinline__ void pull9(const S* base, int plane, int it, int e0, f32x2 (&f)[9]) {
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      const int slot = WINDOW ? ((it - 1 - cy_of(i)) & 3) * 9 * WIN : 0;
      const S* p = base + slot + i * plane + e0 - cx_of(i);
      if (cx_of(i) == 0)
        f[i] = lds_two(p, p + 1);
      else
        f[i] = lds_pair(p);
    }
  }

  // The same for a pair whose columns wrap around the lattice, element by element:
  // column c of the main part at c - xa, columns -2, -1 in the left halo, columns
  // nx, nx + 1, .. in the right halo (for nx >= 2 the pairs read no column below
  // -2 or from 2 nx on).
  __device__ static __forceinline__ void pull9_edge(const S* base, const Geometry& g, int xs, int xa,
                                                    f32x2 (&f)[9]) {
    const int a0 = floor_div(g.nx - 2, CH) * CH;
    auto at = [&](int c) {
      if (g.nx == 1) return -xa;  // every column is column 0
      return c < 0 ? MAIN + (c + g.nx - a0) : (c >= g.nx ? MAIN + 2 * CH + (c - g.nx) : c - xa);
    };
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      const S* p = base + i * SEG;
      f[i] = lds_two(p + at(xs - cx_of(i)), p + at(xs + 1 - cx_of(i)));
    }
  }

  // CONTIG: the ring holds every column contiguously (produce<true>); otherwise the
  // pairs whose columns wrap read through the halo areas. The window rows of a CTA's
  // tiles are numbered on (kw): a tile's first row takes the slot after the previous
  // tile's last, and before its second row overwrites a slot that the previous tile's
  // last output row may still be reading, every warp must have written the first.
  // Returns false once a bounded wait gave up.
  template <int MODEL, int DIAGS, bool CONTIG>
  __device__ __forceinline__ bool consume(S* __restrict__ dst, const Geometry& g, const Coef<f32x2>& c, int x0,
                                          int w, int y0, int rows, int t, int lane, DiagAcc<f32x2>& acc1,
                                          DiagAcc<f32x2>& acc2, int* err) {
    const int xa = floor_div(x0 - 2, CH) * CH;
    const int e1 = 2 * t + 1 + (x0 - 2 - xa);  // ring element of s1 node x0 - 1 + 2t (c_ix = 0; odd)
    // (with nx a multiple of the chunk every strip's width is even: whole output pairs)
    const bool act1 = 2 * t < w + 2, act2 = 2 * t < w, pair2 = CONTIG || 2 * t + 1 < w;
    // the pair's columns wrap around the lattice
    const bool edge = !CONTIG && ((x0 == 0 && t == 0) || x0 + 2 * t + 1 >= g.nx);
    // s1 nodes outside [x0, x0 + w) (the border, and a node past the range on odd widths)
    const bool mask_lo = !(t >= 1 && 2 * t <= w), mask_hi = !(2 * t < w);
    bool failed = false;
    for (int it = 0; it < rows + 2; ++it, ++k) {
      // ---- s1 row y0 - 1 + it
      const int s = k % STAGES;
      if (!failed) failed = !__all_sync(0xffffffffu, mbar_wait(&full[s], (unsigned)((k / STAGES) & 1), err));
      f32x2 f[9];
      if (!failed && act1) {
        if (edge)
          pull9_edge(ring + (size_t)s * 9 * SEG, g, x0 - 1 + 2 * t, xa, f);
        else
          pull9<false>(ring + (size_t)s * 9 * SEG, SEG, it, e1, f);
      }
      __syncwarp();
      if (!failed && lane == 0) mbar_arrive(&empty[s]);
      const int a = kw + it;  // this s1 row's number in the window
      const int q = a & 3;
      if (it == 1 && kw > 0 && !failed)  // the previous tile's last reads are done once every warp wrote row kw
        failed = !__all_sync(0xffffffffu, mbar_wait(&wbar[kw & 3], (unsigned)((kw >> 2) & 1), err));
      if (!failed && act1) {
        collide<MODEL, true, f32x2>(f, c, [&](NodeMoments<f32x2> m) {
          if constexpr ((DIAGS & 1) != 0) {
            if (it >= 1 && it <= rows) {
              if (mask_lo) m.m0.v.x = m.jx.v.x = m.jy.v.x = m.ux.v.x = m.uy.v.x = 0.0f;
              if (mask_hi) m.m0.v.y = m.jx.v.y = m.jy.v.y = m.ux.v.y = m.uy.v.y = 0.0f;
              acc1.add(m);
            }
          }
        });
        S* wq = win + (size_t)q * 9 * WIN + 2 * t;
#pragma unroll
        for (int i = 0; i < 9; ++i) st_pair(wq + i * WIN, f[i]);
      }
      __syncwarp();
      if (!failed && lane == 0) mbar_arrive(&wbar[q]);
      if (it < 2) continue;
      // ---- output row y0 + it - 2 from s1 rows it - 2, it - 1, it of the window
      if (!failed) failed = !__all_sync(0xffffffffu, mbar_wait(&wbar[q], (unsigned)((a >> 2) & 1), err));
      if (failed || !act2) continue;
      pull9<true>(win, WIN, a, 2 * t + 1, f);
      collide<MODEL, true, f32x2>(f, c, [&](NodeMoments<f32x2> m) {
        if constexpr ((DIAGS & 2) != 0) {
          if (!pair2) m.m0.v.y = m.jx.v.y = m.jy.v.y = m.ux.v.y = m.uy.v.y = 0.0f;  // past the strip
          acc2.add(m);
        }
      });
      S* o = dst + (long long)(y0 + it - 2) * g.pitch + x0 + 2 * t;
      if (pair2) {
#pragma unroll
        for (int i = 0; i < 9; ++i) st_pair(o + i * g.plane, f[i]);
      } else {
#pragma unroll
        for (int i = 0; i < 9; ++i) st_t(o + i * g.plane, f[i].v.x);
      }
    }
    kw += rows + 2;
    return !failed;
  }
};

// One CTA per tile: strip blockIdx.x (w = W columns, the last strip the rest),
// output rows [blockIdx.y H, + H). DIAGS bit 0: diagnostics of step t into
// partials1; bit 1: of step t + 1 into partials2.
template <int MODEL, int PREC, int DIAGS, int NC, int STAGES>
__global__ void __launch_bounds__(NC + 32, NC <= 128 ? 4 : 3)
    step2_stream_kernel(const typename Form<PREC>::S* __restrict__ src,
                                                                   typename Form<PREC>::S* __restrict__ dst,
                                                                   Geometry g, Coef<f32x2> c,
                                                                   double* __restrict__ partials1,
                                                                   double* __restrict__ partials2, int H,
                                                                   int* __restrict__ err) {
  using P = Pipeline2<PREC, NC, STAGES>;
  extern __shared__ __align__(128) unsigned char smem[];
  P pipe(smem);
  pipe.init();
  __syncthreads();
  pdl_launch_dependents();
  const int x0 = blockIdx.x * P::W, y0 = blockIdx.y * H;
  const int w = min(P::W, g.nx - x0), rows = min(H, g.ny - y0);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  DiagAcc<f32x2> acc1, acc2;
  if (warp == P::kConsumerWarps) {
    pdl_wait();
    if (g.nx % P::CH == 0)
      pipe.template produce<true>(src, g, x0, w, y0, rows, lane, err);
    else
      pipe.template produce<false>(src, g, x0, w, y0, rows, lane, err);
    pipe.drain(err);
  } else if (threadIdx.x < NC) {
    if (g.nx % P::CH == 0)
      pipe.template consume<MODEL, DIAGS, true>(dst, g, c, x0, w, y0, rows, threadIdx.x, lane, acc1, acc2, err);
    else
      pipe.template consume<MODEL, DIAGS, false>(dst, g, c, x0, w, y0, rows, threadIdx.x, lane, acc1, acc2, err);
  }
  const long long b = (long long)(blockIdx.y * gridDim.x + blockIdx.x) * 5;
  if constexpr ((DIAGS & 1) != 0) block_diag_acc(acc1, partials1 + b);
  if constexpr (DIAGS == 3) __syncthreads();  // block_diag's shared scratch is reused
  if constexpr ((DIAGS & 2) != 0) block_diag_acc(acc2, partials2 + b);
}

// ------------------------------------------------------------------ launcher
// Two ring slots: the ring (2 x 9.5 KB) and the window (36 KB) let four FP32 CTAs
// share an SM (measured at 4096^2, complete model, diagnostics every step: 2 slots
// 142.0 GLUPS, 3 slots 133.6, 4 slots 134.3, 6 slots 113.3).
#ifndef OLBM_STREAM2_STAGES
#define OLBM_STREAM2_STAGES 2
#endif
constexpr int kStream2Stages = OLBM_STREAM2_STAGES;

template <int PREC> struct Launch2 {
  using S = typename Form<PREC>::S;
  static constexpr int NC = PREC == 1 ? kStream2NC32 : kStream2NC16;
  using Shape = Stream2Shape<PREC, NC, kStream2Stages>;
  static_assert(Shape::W == 2 * NC - 2, "tile width of the launcher");

  template <int MODEL, int DIAGS>
  static cudaError_t run(const StepArgs& a, cudaStream_t st) {
    auto kernel = step2_stream_kernel<MODEL, PREC, DIAGS, NC, kStream2Stages>;
    // once per device: opt in to the large shared-memory carve-out
    constexpr int kMaxDev = 64;
    static bool ready[kMaxDev] = {false};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDev) return cudaErrorInvalidDevice;
    if (!ready[dev]) {
      e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, Shape::kSmemBytes);
      if (e != cudaSuccess) return e;
      ready[dev] = true;
    }
    const dim3 grid = step2_grid(a.g, a.cfg, PREC);
    if (a.parts_used) *a.parts_used = (long long)grid.x * grid.y;
    const Coef<f32x2> c = make_coef<f32x2>(a.theta, a.tau, a.rho_ref);
    return launch_step_kernel(kernel, grid, dim3(NC + 32), Shape::kSmemBytes, st, (const S*)a.src, (S*)a.dst, a.g,
                              c, a.partials, a.partials2, a.cfg.rows, a.err);
  }

  template <int MODEL>
  static cudaError_t run_m(const StepArgs& a, cudaStream_t st) {
    switch ((a.diag ? 1 : 0) | (a.diag2 ? 2 : 0)) {
      case 0: return run<MODEL, 0>(a, st);
      case 1: return run<MODEL, 1>(a, st);
      case 2: return run<MODEL, 2>(a, st);
      default: return run<MODEL, 3>(a, st);
    }
  }

  static cudaError_t step2(const StepArgs& a, cudaStream_t st) {
    if (!step2_applies(PREC, a.g, a.cfg) || a.err == nullptr) return cudaErrorInvalidConfiguration;
    if ((a.diag && a.partials == nullptr) || (a.diag2 && a.partials2 == nullptr)) return cudaErrorInvalidValue;
    switch (a.model) {
      case 0: return run_m<0>(a, st);
      case 1: return run_m<1>(a, st);
      case 2: return run_m<2>(a, st);
      case 3: return run_m<3>(a, st);
      case 4: return run_m<4>(a, st);
      case 5: return run_m<5>(a, st);
      default: return cudaErrorInvalidValue;
    }
  }
};

}  // namespace olbm

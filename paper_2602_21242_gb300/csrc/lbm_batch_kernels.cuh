// lbm_batch_kernels.cuh -- kernels and launchers of the batched form for one
// storage form (arXiv 2602.21242, Eq. 1 applied per domain); instantiated once
// per form by lbm_batch_f64.cu, lbm_batch_f32.cu and lbm_batch_f16.cu.
//
// Launch kind 0: one thread block per tile of (bx or 2 bx) columns x (by x
// rows) rows with the single-lattice column routine. Launch kind 1 (shifted
// forms): one CTA per tile of 2 NC columns x `rows` rows with the single-lattice
// bulk-copy pipeline (NC consumer threads: 32, 64 or 128 for FP32, 64, 128 or 256
// for FP16; narrower tiles waste less of a strip on narrow domains). Graph mode
// launches one tile kernel per step; persistent mode one cooperative kernel
// for all steps, tiles strided over the grid, a bounded grid barrier between
// steps.
#pragma once

#include <algorithm>
#include <atomic>

#include "lbm_batch.h"

namespace olbm {

// Update one tile (d, x0, y0) from buffer `parity` into buffer parity ^ 1.
template <int MODEL, int PREC, bool DIAG, bool CG>
__device__ __forceinline__ void update_tile(const Desc<typename Form<PREC>::T>& d, int x0, int y0, int parity,
                                            int rows, double* __restrict__ out5) {
  using S = typename Form<PREC>::S;
  const S* src = static_cast<const S*>(d.buf[parity]);
  S* dst = static_cast<S*>(d.buf[parity ^ 1]);
  const int y = y0 + threadIdx.y, dy = blockDim.y;
  if constexpr (PREC != 0) {
    if (d.pairs) {
      using Col = Column<MODEL, PREC, DIAG, true, CG>;
      DiagAcc<f32x2> acc;
      Col::run(src, dst, d.g, broadcast(d.c), x0 + 2 * threadIdx.x, y, dy, rows, acc);
      if constexpr (DIAG) block_diag_acc(acc, out5);
      return;
    }
  }
  using Col = Column<MODEL, PREC, DIAG, false, CG>;
  DiagAcc<typename Col::CT> acc;
  Col::run(src, dst, d.g, d.c, x0 + threadIdx.x, y, dy, rows, acc);
  if constexpr (DIAG) block_diag_acc(acc, out5);
}

// One time step of every domain: block b updates tile b.
template <int MODEL, int PREC, bool DIAG>
__global__ void __launch_bounds__(512) batch_step_kernel(const Desc<typename Form<PREC>::T>* __restrict__ desc,
                                                         const int4* __restrict__ tiles, int parity,
                                                         double* __restrict__ partials, int rows) {
  const int4 tl = tiles[blockIdx.x];
  const Desc<typename Form<PREC>::T> d = desc[tl.x];
  update_tile<MODEL, PREC, DIAG, false>(d, tl.y, tl.z, parity, rows, partials + (long long)blockIdx.x * 5);
}

// n steps of every domain in one launch; tiles strided over the grid.
template <int MODEL, int PREC>
__global__ void __launch_bounds__(512) batch_persistent_kernel(const Desc<typename Form<PREC>::T>* __restrict__ desc,
                                                               const int4* __restrict__ tiles, int ntiles,
                                                               int parity0, int nsteps, int rows, GridBarrier* bar) {
  for (int s = 0; s < nsteps; ++s) {
    const int parity = (parity0 + s) & 1;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
      const int4 tl = tiles[t];
      const Desc<typename Form<PREC>::T> d = desc[tl.x];
      update_tile<MODEL, PREC, false, true>(d, tl.y, tl.z, parity, rows, nullptr);
    }
    if (!grid_sync(bar, gridDim.x)) return;
  }
}

// Pull-only diagnostics of one tile (FP64), as diag_kernel for one lattice.
// A tile spans cols1 columns (cols2 for node-pair domains) x trows rows; the
// block's threads stride over its nodes.
template <int PREC>
__global__ void __launch_bounds__(512) batch_diag_kernel(const Desc<typename Form<PREC>::T>* __restrict__ desc,
                                                         const int4* __restrict__ tiles, int parity, int cols1,
                                                         int cols2, int trows, double rho_ref,
                                                         double* __restrict__ partials) {
  using S = typename Form<PREC>::S;
  const int4 tl = tiles[blockIdx.x];
  const Desc<typename Form<PREC>::T> d = desc[tl.x];
  const S* src = static_cast<const S*>(d.buf[parity]);
  const int w = min(d.pairs ? cols2 : cols1, d.g.nx - tl.y);
  const int h = min(trows, d.g.ny - tl.z);
  const int nthreads = blockDim.x * blockDim.y, tid = threadIdx.y * blockDim.x + threadIdx.x;
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  int bad = 0;
  for (int j = tid; j < w * h; j += nthreads) {
    const int x = tl.y + j % w, y = tl.z + j / w;
    double m0, jx, jy;
    pulled_moments<PREC>(src, d.g, x, y, m0, jx, jy);
    if (finite_bits(m0)) {
      v[0] += m0;
      v[1] += jx;
      v[2] += jy;
      v[3] = fma(0.5 * fma(jx, jx, jy * jy), recip(rho_ref + m0), v[3]);
    } else {
      ++bad;
    }
  }
  block_diag<double>(v, bad, partials + (long long)blockIdx.x * 5);
}

// Pipelined tile step (launch kind 1, shifted forms): one CTA per tile of W
// columns x H rows of one domain, the single-lattice pipeline on that tile.
template <int MODEL, int PREC, bool DIAG, int NC, int STAGES>
__global__ void __launch_bounds__(NC + 32) batch_stream_kernel(const Desc<float>* __restrict__ desc,
                                                              const int4* __restrict__ tiles, int parity,
                                                              double* __restrict__ partials, int H,
                                                              int* __restrict__ err) {
  using P = Pipeline<PREC, NC, STAGES>;
  using S = typename Form<PREC>::S;
  extern __shared__ __align__(128) unsigned char smem[];
  P pipe(smem);
  pipe.init();
  __syncthreads();
  const int4 tl = tiles[blockIdx.x];
  const Desc<float>* d = desc + tl.x;
  const Geometry g = d->g;
  const int rows = min(H, g.ny - tl.z);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  DiagAcc<f32x2> acc;
  if (warp == P::kConsumerWarps) {
    pipe.produce(static_cast<const S*>(d->buf[parity]), g, tl.y, tl.z, rows, lane, err);
    pipe.drain(err);
  } else if (threadIdx.x < NC) {
    pipe.template consume<MODEL, DIAG>(static_cast<S*>(d->buf[parity ^ 1]), g, broadcast(d->c), tl.y, tl.z, rows,
                                       threadIdx.x, lane, acc, err);
  }
  if constexpr (DIAG) block_diag_acc(acc, partials + (long long)blockIdx.x * 5);
}

__device__ __forceinline__ void fence_proxy_async_global() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
}

// n steps of every domain in one cooperative launch of pipelined CTAs, a
// bounded grid barrier between steps. Tiles are handed out in list (domain)
// order by an atomic counter per step, ctr[s & 1]: a CTA's producer takes the
// next tile when it has issued the previous one, so CTAs that finish early take
// more, and tiles that run together stay neighbours (their halo rows meet in
// L2). The producer tags every ring slot with its tile and closes the step with
// a slot tagged -1; the consumers follow the tags. The counter of the step
// after next is reset at the start of a step (it was last used two barriers
// ago). The consumers' stores (generic proxy) reach the next step's bulk copies
// (async proxy) through a proxy fence on both sides of the barrier. A bounded
// wait that gives up sets the barrier's error flag, so every CTA leaves at the
// next barrier.
template <int MODEL, int PREC, int NC, int STAGES>
__global__ void __launch_bounds__(NC + 32) batch_stream_persistent_kernel(const Desc<float>* __restrict__ desc,
                                                                         const int4* __restrict__ tiles, int ntiles,
                                                                         int parity0, int nsteps, int H,
                                                                         GridBarrier* bar, int* ctr) {
  using P = Pipeline<PREC, NC, STAGES>;
  using S = typename Form<PREC>::S;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ int tags[STAGES];
  P pipe(smem);
  pipe.init();
  __syncthreads();
  int* err = &bar->err;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const bool producer = warp == P::kConsumerWarps;
  DiagAcc<f32x2> acc;  // no fused diagnostics in this mode
  for (int s = 0; s < nsteps; ++s) {
    const int parity = (parity0 + s) & 1;
    if (producer) {
      if (blockIdx.x == 0 && lane == 0) atomicExch(&ctr[(s + 1) & 1], 0);
      fence_proxy_async_global();
      bool ok = true;
      for (;;) {
        int t = 0;
        if (lane == 0) t = atomicAdd(&ctr[s & 1], 1);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= ntiles) {  // close the step: a slot without data, tagged -1
          const int q = pipe.k % STAGES;
          if (pipe.k >= STAGES) ok = mbar_wait(&pipe.empty[q], (unsigned)((pipe.k / STAGES - 1) & 1), err);
          ok = __all_sync(0xffffffffu, ok);
          if (ok && lane == 0) {
            tags[q] = -1;
            mbar_arrive(&pipe.full[q]);
          }
          ++pipe.k;
          break;
        }
        const int4 tl = tiles[t];
        const Desc<float>* d = desc + tl.x;
        if (!pipe.produce(static_cast<const S*>(d->buf[parity]), d->g, tl.y, tl.z, min(H, d->g.ny - tl.z), lane,
                          err, tags, t)) {
          ok = false;
          break;
        }
      }
      (void)ok;
    } else if (threadIdx.x < NC) {
      for (;;) {
        const int q = pipe.k % STAGES;
        if (!__all_sync(0xffffffffu, mbar_wait(&pipe.full[q], (unsigned)((pipe.k / STAGES) & 1), err))) break;
        const int t = *(volatile int*)&tags[q];
        if (t < 0) {  // end of the step
          __syncwarp();
          if (lane == 0) mbar_arrive(&pipe.empty[q]);
          ++pipe.k;
          break;
        }
        const int4 tl = tiles[t];
        const Desc<float>* d = desc + tl.x;
        if (!pipe.template consume<MODEL, false>(static_cast<S*>(d->buf[parity ^ 1]), d->g, broadcast(d->c), tl.y,
                                                 tl.z, min(H, d->g.ny - tl.z), threadIdx.x, lane, acc, err))
          break;
      }
      fence_proxy_async_global();
    }
    if (!grid_sync(bar, gridDim.x)) break;
  }
  if (producer) pipe.drain(err);
}

// ------------------------------------------------------------------ launchers of one storage form
template <int PREC> struct BatchOps {
  using T = typename Form<PREC>::T;
  // pipelined consumer widths instantiated for this form
  static constexpr int kNcA = PREC == 1 ? 32 : 64, kNcB = PREC == 1 ? 64 : 128, kNcC = PREC == 1 ? 128 : 256;
  static constexpr int kStages = kStreamStages;

  // The shared-memory opt-in is a per-device attribute: set once per kernel and device.
  template <auto K> static cudaError_t allow_ring(int bytes) {
    static std::atomic<unsigned long long> done{0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    const unsigned long long bit = 1ull << dev;
    if (done.load() & bit) return cudaSuccess;
    e = cudaFuncSetAttribute(K, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) done.fetch_or(bit);
    return e;
  }

  template <int MODEL, int NC> static cudaError_t prepare_nc() {
    constexpr int bytes = StreamShape<PREC, NC, kStages>::kSmemBytes;
    cudaError_t e = allow_ring<batch_stream_kernel<MODEL, PREC, true, NC, kStages>>(bytes);
    if (e == cudaSuccess) e = allow_ring<batch_stream_kernel<MODEL, PREC, false, NC, kStages>>(bytes);
    if (e == cudaSuccess) e = allow_ring<batch_stream_persistent_kernel<MODEL, PREC, NC, kStages>>(bytes);
    return e;
  }

  template <int MODEL, int NC>
  static cudaError_t step_stream(const BatchLaunch& b, bool diag, int parity, cudaStream_t st) {
    constexpr int bytes = StreamShape<PREC, NC, kStages>::kSmemBytes;
    const auto* desc = static_cast<const Desc<float>*>(b.desc);
    if (diag)
      batch_stream_kernel<MODEL, PREC, true, NC, kStages><<<b.ntiles, NC + 32, bytes, st>>>(
          desc, b.tiles, parity, b.partials, b.cfg.rows, b.perr);
    else
      batch_stream_kernel<MODEL, PREC, false, NC, kStages><<<b.ntiles, NC + 32, bytes, st>>>(
          desc, b.tiles, parity, b.partials, b.cfg.rows, b.perr);
    return cudaGetLastError();
  }

  template <int MODEL, int NC>
  static cudaError_t persistent_stream(const BatchLaunch& b, int n, int parity0, cudaStream_t st) {
    constexpr int bytes = StreamShape<PREC, NC, kStages>::kSmemBytes;
    auto kernel = batch_stream_persistent_kernel<MODEL, PREC, NC, kStages>;
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, NC + 32, bytes);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int grid = std::min(b.ntiles, per_sm * b.sms);
    const auto* desc = static_cast<const Desc<float>*>(b.desc);
    const int4* tiles = b.tiles;
    int ntiles = b.ntiles, rows = b.cfg.rows;
    GridBarrier* bar = b.bar;
    int* ctr = b.ctr;
    void* args[] = {(void*)&desc, (void*)&tiles, (void*)&ntiles, (void*)&parity0, (void*)&n, (void*)&rows,
                    (void*)&bar, (void*)&ctr};
    e = cudaMemsetAsync(b.bar, 0, b.keep_err ? 2 * sizeof(unsigned) : sizeof(GridBarrier), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(b.ctr, 0, 2 * sizeof(int), st);
    if (e != cudaSuccess) return e;
    return cudaLaunchCooperativeKernel((const void*)kernel, dim3(grid), dim3(NC + 32), args, (size_t)bytes, st);
  }

  template <int MODEL> static cudaError_t prepare_m(const BatchLaunch& b) {
    if constexpr (PREC != 0) {
      if (b.cfg.kind == 1) {
        switch (batch_stream_nc(PREC, b.cfg.bx)) {
          case kNcA: return prepare_nc<MODEL, kNcA>();
          case kNcB: return prepare_nc<MODEL, kNcB>();
          case kNcC: return prepare_nc<MODEL, kNcC>();
          default: return cudaErrorInvalidConfiguration;
        }
      }
    }
    return cudaSuccess;
  }

  template <int MODEL> static cudaError_t step_m(const BatchLaunch& b, bool diag, int parity, cudaStream_t st) {
    if constexpr (PREC != 0) {
      if (b.cfg.kind == 1) {
        switch (batch_stream_nc(PREC, b.cfg.bx)) {
          case kNcA: return step_stream<MODEL, kNcA>(b, diag, parity, st);
          case kNcB: return step_stream<MODEL, kNcB>(b, diag, parity, st);
          case kNcC: return step_stream<MODEL, kNcC>(b, diag, parity, st);
          default: return cudaErrorInvalidConfiguration;
        }
      }
    }
    const auto* desc = static_cast<const Desc<T>*>(b.desc);
    const dim3 block(b.cfg.bx, b.cfg.by);
    if (diag)
      batch_step_kernel<MODEL, PREC, true><<<b.ntiles, block, 0, st>>>(desc, b.tiles, parity, b.partials, b.cfg.rows);
    else
      batch_step_kernel<MODEL, PREC, false><<<b.ntiles, block, 0, st>>>(desc, b.tiles, parity, b.partials, b.cfg.rows);
    return cudaGetLastError();
  }

  template <int MODEL> static cudaError_t persistent_m(const BatchLaunch& b, int n, int parity0, cudaStream_t st) {
    if constexpr (PREC != 0) {
      if (b.cfg.kind == 1) {
        switch (batch_stream_nc(PREC, b.cfg.bx)) {
          case kNcA: return persistent_stream<MODEL, kNcA>(b, n, parity0, st);
          case kNcB: return persistent_stream<MODEL, kNcB>(b, n, parity0, st);
          case kNcC: return persistent_stream<MODEL, kNcC>(b, n, parity0, st);
          default: return cudaErrorInvalidConfiguration;
        }
      }
    }
    auto kernel = batch_persistent_kernel<MODEL, PREC>;
    const int threads = b.cfg.bx * b.cfg.by;
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int grid = std::min(b.ntiles, per_sm * b.sms);
    const auto* desc = static_cast<const Desc<T>*>(b.desc);
    const int4* tiles = b.tiles;
    int ntiles = b.ntiles, rows = b.cfg.rows;
    GridBarrier* bar = b.bar;
    void* args[] = {(void*)&desc, (void*)&tiles, (void*)&ntiles, (void*)&parity0, (void*)&n, (void*)&rows,
                    (void*)&bar};
    e = cudaMemsetAsync(b.bar, 0, b.keep_err ? 2 * sizeof(unsigned) : sizeof(GridBarrier), st);
    if (e != cudaSuccess) return e;
    return cudaLaunchCooperativeKernel((const void*)kernel, dim3(grid), dim3(b.cfg.bx, b.cfg.by), args, 0, st);
  }

  static cudaError_t prepare(const BatchLaunch& b) {
    switch (b.model) {
      case 0: return prepare_m<0>(b);
      case 1: return prepare_m<1>(b);
      case 2: return prepare_m<2>(b);
      case 3: return prepare_m<3>(b);
      case 4: return prepare_m<4>(b);
      case 5: return prepare_m<5>(b);
      default: return cudaErrorInvalidValue;
    }
  }

  static cudaError_t step(const BatchLaunch& b, bool diag, int parity, cudaStream_t st) {
    switch (b.model) {
      case 0: return step_m<0>(b, diag, parity, st);
      case 1: return step_m<1>(b, diag, parity, st);
      case 2: return step_m<2>(b, diag, parity, st);
      case 3: return step_m<3>(b, diag, parity, st);
      case 4: return step_m<4>(b, diag, parity, st);
      case 5: return step_m<5>(b, diag, parity, st);
      default: return cudaErrorInvalidValue;
    }
  }

  static cudaError_t persistent(const BatchLaunch& b, int n, int parity0, cudaStream_t st) {
    switch (b.model) {
      case 0: return persistent_m<0>(b, n, parity0, st);
      case 1: return persistent_m<1>(b, n, parity0, st);
      case 2: return persistent_m<2>(b, n, parity0, st);
      case 3: return persistent_m<3>(b, n, parity0, st);
      case 4: return persistent_m<4>(b, n, parity0, st);
      case 5: return persistent_m<5>(b, n, parity0, st);
      default: return cudaErrorInvalidValue;
    }
  }

  static cudaError_t diag(const BatchLaunch& b, int parity, double rho_ref, cudaStream_t st) {
    const auto* desc = static_cast<const Desc<T>*>(b.desc);
    if (b.cfg.kind == 1) {
      const int w = 2 * batch_stream_nc(PREC, b.cfg.bx);
      batch_diag_kernel<PREC><<<b.ntiles, 256, 0, st>>>(desc, b.tiles, parity, w, w, b.cfg.rows, rho_ref, b.partials);
    } else {
      batch_diag_kernel<PREC><<<b.ntiles, dim3(b.cfg.bx, b.cfg.by), 0, st>>>(
          desc, b.tiles, parity, b.cfg.bx, 2 * b.cfg.bx, b.cfg.by * b.cfg.rows, rho_ref, b.partials);
    }
    return cudaGetLastError();
  }
};

#define OLBM_DEFINE_BATCH(SUFFIX, PREC)                                                                 \
  cudaError_t batch_prepare_##SUFFIX(const BatchLaunch& b) { return BatchOps<PREC>::prepare(b); }      \
  cudaError_t batch_step_##SUFFIX(const BatchLaunch& b, bool diag, int parity, cudaStream_t st) {       \
    return BatchOps<PREC>::step(b, diag, parity, st);                                                   \
  }                                                                                                     \
  cudaError_t batch_persistent_##SUFFIX(const BatchLaunch& b, int n, int parity0, cudaStream_t st) {    \
    return BatchOps<PREC>::persistent(b, n, parity0, st);                                               \
  }                                                                                                     \
  cudaError_t batch_diag_##SUFFIX(const BatchLaunch& b, int parity, double rho_ref, cudaStream_t st) {   \
    return BatchOps<PREC>::diag(b, parity, rho_ref, st);                                                \
  }

}  // namespace olbm

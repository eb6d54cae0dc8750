// lbm_batch_stream2.cuh -- two steps per launch for batched domains (launch kind 2
// of lbm_batch_set_launch_ex; shifted storage forms): the two-step tile routine of
// lbm_stream2.cuh on a list of tiles of 2 NC - 2 columns x H rows of any domain,
// one CTA per tile, each domain's geometry, buffers and coefficients from its
// descriptor. Results equal two single steps of every domain bit for bit.
#pragma once

#include <algorithm>
#include <atomic>

#include "lbm_batch.h"
#include "lbm_batch_kernels.cuh"
#include "lbm_stream2.cuh"

namespace olbm {

template <int MODEL, int PREC, int DIAGS, int NC, int STAGES>
__global__ void __launch_bounds__(NC + 32, NC <= 128 ? 4 : 3) batch_step2_kernel(const Desc<float>* __restrict__ desc,
                                                                                const int4* __restrict__ tiles,
                                                                                int parity,
                                                                                double* __restrict__ partials1,
                                                                                double* __restrict__ partials2, int H,
                                                                                int* __restrict__ err) {
  using P = Pipeline2<PREC, NC, STAGES>;
  using S = typename Form<PREC>::S;
  extern __shared__ __align__(128) unsigned char smem[];
  P pipe(smem);
  pipe.init();
  __syncthreads();
  const int4 tl = tiles[blockIdx.x];
  const Desc<float>* d = desc + tl.x;
  const Geometry g = d->g;
  const int x0 = tl.y, y0 = tl.z;
  const int w = min(P::W, g.nx - x0), rows = min(H, g.ny - y0);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  DiagAcc<f32x2> acc1, acc2;
  if (warp == P::kConsumerWarps) {
    const S* src = static_cast<const S*>(d->buf[parity]);
    if (g.nx % P::CH == 0)
      pipe.template produce<true>(src, g, x0, w, y0, rows, lane, err);
    else
      pipe.template produce<false>(src, g, x0, w, y0, rows, lane, err);
    pipe.drain(err);
  } else if (threadIdx.x < NC) {
    S* dst = static_cast<S*>(d->buf[parity ^ 1]);
    const Coef<f32x2> c = broadcast(d->c);
    if (g.nx % P::CH == 0)
      pipe.template consume<MODEL, DIAGS, true>(dst, g, c, x0, w, y0, rows, threadIdx.x, lane, acc1, acc2, err);
    else
      pipe.template consume<MODEL, DIAGS, false>(dst, g, c, x0, w, y0, rows, threadIdx.x, lane, acc1, acc2, err);
  }
  const long long b = (long long)blockIdx.x * 5;
  if constexpr ((DIAGS & 1) != 0) block_diag_acc(acc1, partials1 + b);
  if constexpr (DIAGS == 3) __syncthreads();  // block_diag's shared scratch is reused
  if constexpr ((DIAGS & 2) != 0) block_diag_acc(acc2, partials2 + b);
}

// npairs pairs of steps of every domain in one cooperative launch (persistent mode
// with launch kind 2): per pair, the CTAs take two-step tiles from the counter
// ctr[pair & 1] in list order (as the single-step persistent kernel does), the
// producer tags each ring slot with its tile and closes the pair with a slot
// tagged -1, and a bounded grid barrier separates the pairs (with proxy fences on
// both sides: the consumers' stores reach the next pair's bulk copies). No fused
// diagnostics. A bounded wait that gives up sets the barrier's error flag, so
// every CTA leaves at the next barrier.
// Three resident CTAs a SM: its tile hand-out takes registers that a bound of four
// turns into spills (256 domains, 32-row tiles: 106.2 GLUPS against 100.3).
#ifndef OLBM_BATCH2_PERSISTENT_MINB
#define OLBM_BATCH2_PERSISTENT_MINB 3
#endif
template <int MODEL, int PREC, int NC, int STAGES>
__global__ void __launch_bounds__(NC + 32, NC <= 128 ? OLBM_BATCH2_PERSISTENT_MINB : 3)
    batch_step2_persistent_kernel(const Desc<float>* __restrict__ desc, const int4* __restrict__ tiles, int ntiles,
                                  int parity0, int npairs, int H, GridBarrier* bar, int* ctr) {
  using P = Pipeline2<PREC, NC, STAGES>;
  using S = typename Form<PREC>::S;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ int tags[STAGES];
  P pipe(smem);
  pipe.init();
  __syncthreads();
  int* err = &bar->err;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const bool producer = warp == P::kConsumerWarps;
  DiagAcc<f32x2> acc1, acc2;  // no fused diagnostics in this mode
  for (int s = 0; s < npairs; ++s) {
    const int parity = (parity0 + s) & 1;
    if (producer) {
      if (blockIdx.x == 0 && lane == 0) atomicExch(&ctr[(s + 1) & 1], 0);
      fence_proxy_async_global();
      for (;;) {
        int t = 0;
        if (lane == 0) t = atomicAdd(&ctr[s & 1], 1);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= ntiles) {  // close the pair: a slot without data, tagged -1
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
        const int4 tl = tiles[t];
        const Desc<float>* d = desc + tl.x;
        const Geometry g = d->g;
        const S* src = static_cast<const S*>(d->buf[parity]);
        const int w = min(P::W, g.nx - tl.y), rows = min(H, g.ny - tl.z);
        const bool ok = g.nx % P::CH == 0
                            ? pipe.template produce<true>(src, g, tl.y, w, tl.z, rows, lane, err, tags, t)
                            : pipe.template produce<false>(src, g, tl.y, w, tl.z, rows, lane, err, tags, t);
        if (!ok) break;
      }
    } else if (threadIdx.x < NC) {
      for (;;) {
        const int q = pipe.k % STAGES;
        if (!__all_sync(0xffffffffu, mbar_wait(&pipe.full[q], (unsigned)((pipe.k / STAGES) & 1), err))) break;
        const int t = *(volatile int*)&tags[q];
        if (t < 0) {  // end of the pair
          __syncwarp();
          if (lane == 0) mbar_arrive(&pipe.empty[q]);
          ++pipe.k;
          break;
        }
        const int4 tl = tiles[t];
        const Desc<float>* d = desc + tl.x;
        const Geometry g = d->g;
        S* dst = static_cast<S*>(d->buf[parity ^ 1]);
        const Coef<f32x2> c = broadcast(d->c);
        const int w = min(P::W, g.nx - tl.y), rows = min(H, g.ny - tl.z);
        const bool ok = g.nx % P::CH == 0
                            ? pipe.template consume<MODEL, 0, true>(dst, g, c, tl.y, w, tl.z, rows, threadIdx.x, lane,
                                                                    acc1, acc2, err)
                            : pipe.template consume<MODEL, 0, false>(dst, g, c, tl.y, w, tl.z, rows, threadIdx.x, lane,
                                                                     acc1, acc2, err);
        if (!ok) break;
      }
      fence_proxy_async_global();
    }
    if (!grid_sync(bar, gridDim.x)) break;
  }
  if (producer) pipe.drain(err);
}

template <int PREC> struct BatchOps2 {
  static constexpr int NC = PREC == 1 ? kStream2NC32 : kStream2NC16;
  using Shape = Stream2Shape<PREC, NC, kStream2Stages>;

  template <auto K> static cudaError_t allow() {
    static std::atomic<unsigned long long> done{0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    const unsigned long long bit = 1ull << dev;
    if (done.load() & bit) return cudaSuccess;
    e = cudaFuncSetAttribute(K, cudaFuncAttributeMaxDynamicSharedMemorySize, Shape::kSmemBytes);
    if (e == cudaSuccess) done.fetch_or(bit);
    return e;
  }

  template <int MODEL> static cudaError_t prepare_m() {
    cudaError_t e = allow<batch_step2_kernel<MODEL, PREC, 0, NC, kStream2Stages>>();
    if (e == cudaSuccess) e = allow<batch_step2_kernel<MODEL, PREC, 1, NC, kStream2Stages>>();
    if (e == cudaSuccess) e = allow<batch_step2_kernel<MODEL, PREC, 2, NC, kStream2Stages>>();
    if (e == cudaSuccess) e = allow<batch_step2_kernel<MODEL, PREC, 3, NC, kStream2Stages>>();
    if (e == cudaSuccess) e = allow<batch_step2_persistent_kernel<MODEL, PREC, NC, kStream2Stages>>();
    return e;
  }

  template <int MODEL> static cudaError_t persistent_m(const BatchLaunch& b, int npairs, int parity0, cudaStream_t st) {
    auto kernel = batch_step2_persistent_kernel<MODEL, PREC, NC, kStream2Stages>;
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, NC + 32, Shape::kSmemBytes);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int grid = std::min(b.ntiles2, per_sm * b.sms);
    const auto* desc = static_cast<const Desc<float>*>(b.desc);
    const int4* tiles = b.tiles2;
    int ntiles = b.ntiles2, rows = b.cfg.rows;
    GridBarrier* bar = b.bar;
    int* ctr = b.ctr;
    void* args[] = {(void*)&desc, (void*)&tiles, (void*)&ntiles, (void*)&parity0, (void*)&npairs, (void*)&rows,
                    (void*)&bar, (void*)&ctr};
    e = cudaMemsetAsync(b.bar, 0, b.keep_err ? 2 * sizeof(unsigned) : sizeof(GridBarrier), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(b.ctr, 0, 2 * sizeof(int), st);
    if (e != cudaSuccess) return e;
    return cudaLaunchCooperativeKernel((const void*)kernel, dim3(grid), dim3(NC + 32), args,
                                       (size_t)Shape::kSmemBytes, st);
  }

  static cudaError_t persistent(const BatchLaunch& b, int npairs, int parity0, cudaStream_t st) {
    if (b.tiles2 == nullptr || b.bar == nullptr || b.ctr == nullptr) return cudaErrorInvalidValue;
    switch (b.model) {
      case 0: return persistent_m<0>(b, npairs, parity0, st);
      case 1: return persistent_m<1>(b, npairs, parity0, st);
      case 2: return persistent_m<2>(b, npairs, parity0, st);
      case 3: return persistent_m<3>(b, npairs, parity0, st);
      case 4: return persistent_m<4>(b, npairs, parity0, st);
      case 5: return persistent_m<5>(b, npairs, parity0, st);
      default: return cudaErrorInvalidValue;
    }
  }

  template <int MODEL, int DIAGS> static cudaError_t run(const BatchLaunch& b, int parity, cudaStream_t st) {
    batch_step2_kernel<MODEL, PREC, DIAGS, NC, kStream2Stages><<<b.ntiles2, NC + 32, Shape::kSmemBytes, st>>>(
        static_cast<const Desc<float>*>(b.desc), b.tiles2, parity, b.partials, b.partials2, b.cfg.rows, b.perr);
    return cudaGetLastError();
  }

  template <int MODEL>
  static cudaError_t step_m(const BatchLaunch& b, bool diag1, bool diag2, int parity, cudaStream_t st) {
    switch ((diag1 ? 1 : 0) | (diag2 ? 2 : 0)) {
      case 0: return run<MODEL, 0>(b, parity, st);
      case 1: return run<MODEL, 1>(b, parity, st);
      case 2: return run<MODEL, 2>(b, parity, st);
      default: return run<MODEL, 3>(b, parity, st);
    }
  }

  static cudaError_t prepare(const BatchLaunch& b) {
    switch (b.model) {
      case 0: return prepare_m<0>();
      case 1: return prepare_m<1>();
      case 2: return prepare_m<2>();
      case 3: return prepare_m<3>();
      case 4: return prepare_m<4>();
      case 5: return prepare_m<5>();
      default: return cudaErrorInvalidValue;
    }
  }

  static cudaError_t step(const BatchLaunch& b, bool diag1, bool diag2, int parity, cudaStream_t st) {
    if (b.tiles2 == nullptr || b.perr == nullptr) return cudaErrorInvalidValue;
    switch (b.model) {
      case 0: return step_m<0>(b, diag1, diag2, parity, st);
      case 1: return step_m<1>(b, diag1, diag2, parity, st);
      case 2: return step_m<2>(b, diag1, diag2, parity, st);
      case 3: return step_m<3>(b, diag1, diag2, parity, st);
      case 4: return step_m<4>(b, diag1, diag2, parity, st);
      case 5: return step_m<5>(b, diag1, diag2, parity, st);
      default: return cudaErrorInvalidValue;
    }
  }
};

}  // namespace olbm

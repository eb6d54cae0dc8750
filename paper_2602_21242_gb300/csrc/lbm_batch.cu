// lbm_batch.cu -- many independent periodic lattices of uneven size, theta and
// tau, advanced together (the batched form of the D2Q9 OReg-GEq step,
// arXiv 2602.21242, Eq. 1 applied per domain).
//
// Layout: one device arena holds every domain's two population buffers (each
// in the single-lattice layout of lbm_layout). A descriptor table gives each
// domain's geometry, buffers and collision coefficients in the compute type. A
// tile work-list cuts every domain into tiles; one thread block updates one
// tile with a single-lattice routine, so a tile's results equal those of a
// single lattice run with the same launch kind. Launch kind 0: tiles of
// (bx or 2 bx) columns x (by x rows) rows, the column routine. Launch kind 1
// (shifted forms): tiles of W columns (256 FP32, 512 FP16) x `rows` rows, the
// bulk-copy pipeline (producer warp, shared-memory ring, consumer warps), any
// domain width.
//
// Two execution modes for lbm_batch_step(n):
//   LBM_BATCH_GRAPH       n launches of the tile kernel (one per time step),
//                         captured once into a CUDA graph and replayed as one
//                         graph launch; fused diagnostics as for one lattice.
//   LBM_BATCH_PERSISTENT  one cooperative launch of a persistent kernel that
//                         loops over the n steps, tiles strided over the grid,
//                         separated by a grid barrier whose waits are bounded:
//                         a barrier that does not complete within ~1 s sets an
//                         error flag, every block leaves, and the call reports
//                         LBM_ETIMEOUT. Loads bypass L1 (data written by other
//                         blocks earlier in the same launch). No fused
//                         diagnostics; lbm_batch_diagnostics computes them.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <new>
#include <vector>

#include "lbm.h"
#include "lbm_kernels.cuh"

namespace olbm {

// Per-domain descriptor; CT is the scalar compute type (double or float).
template <typename CT> struct Desc {
  Geometry g;
  void* buf[2];
  Coef<CT> c;
  int pairs;  // 1: node pairs (shifted forms, even nx)
  int pad;
};

__host__ __device__ inline Coef<f32x2> broadcast(const Coef<float>& a) {
  Coef<f32x2> c;
  c.theta = a.theta;
  c.one_m_theta = a.one_m_theta;
  c.half_theta = a.half_theta;
  c.omega = a.omega;
  c.one_m_omega = a.one_m_omega;
  c.k1 = a.k1;
  c.k2 = a.k2;
  c.c3 = a.c3;
  c.tt = a.tt;
  c.inv2t2 = a.inv2t2;
  c.mq_inv2t2 = a.mq_inv2t2;
  c.rho_ref = a.rho_ref;
  c.w[0] = a.w[0];
  c.w[1] = a.w[1];
  c.w[2] = a.w[2];
  return c;
}

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
    long long o[9];
    pull_offsets(x, y, d.g, o);
    double m0 = 0.0, jx = 0.0, jy = 0.0;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      const double f = to_double(src[i * d.g.plane + o[i]]);
      m0 += f;
      jx += (double)cx_of(i) * f;
      jy += (double)cy_of(i) * f;
    }
    if (finite_bits(m0)) {
      v[0] += m0;
      v[1] += jx;
      v[2] += jy;
      v[3] += 0.5 * (jx * jx + jy * jy) / (rho_ref + m0);
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

// n steps of every domain in one cooperative launch of pipelined CTAs: tiles
// strided over the grid, a bounded grid barrier between steps. The consumers'
// stores (generic proxy) reach the next step's bulk copies (async proxy)
// through a proxy fence on both sides of the barrier. A bounded wait that gives
// up sets the barrier's error flag, so every CTA leaves at the next barrier.
template <int MODEL, int PREC, int NC, int STAGES>
__global__ void __launch_bounds__(NC + 32) batch_stream_persistent_kernel(const Desc<float>* __restrict__ desc,
                                                                         const int4* __restrict__ tiles, int ntiles,
                                                                         int parity0, int nsteps, int H,
                                                                         GridBarrier* bar) {
  using P = Pipeline<PREC, NC, STAGES>;
  using S = typename Form<PREC>::S;
  extern __shared__ __align__(128) unsigned char smem[];
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
      fence_proxy_async_global();
      for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int4 tl = tiles[t];
        const Desc<float>* d = desc + tl.x;
        if (!pipe.produce(static_cast<const S*>(d->buf[parity]), d->g, tl.y, tl.z, min(H, d->g.ny - tl.z), lane,
                          err))
          break;
      }
    } else if (threadIdx.x < NC) {
      for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
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

// Per-domain fixed-order sums of the tile partials: out[d * 5 + k].
__global__ void __launch_bounds__(256) batch_finalize_kernel(const double* __restrict__ partials,
                                                             const int2* __restrict__ ranges,
                                                             const long long* __restrict__ nodes, double rho_ref,
                                                             double* __restrict__ out,
                                                             unsigned long long* __restrict__ sticky) {
  const int2 r = ranges[blockIdx.x];
  double v[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  for (int j = r.x + threadIdx.x; j < r.x + r.y; j += 256)
#pragma unroll
    for (int k = 0; k < 5; ++k) v[k] += partials[(long long)j * 5 + k];
  double tot[5];
  block_sum<5, 256>(v, tot);
  if (threadIdx.x == 0) {
    double* o = out + (long long)blockIdx.x * 5;
    const double bad = tot[4];
    o[0] = tot[0] + rho_ref * ((double)nodes[blockIdx.x] - bad);
    o[1] = tot[1];
    o[2] = tot[2];
    o[3] = tot[3];
    o[4] = bad;
    if (bad > 0.0 && sticky != nullptr) atomicAdd(sticky, (unsigned long long)bad);
  }
}

}  // namespace olbm

// ============================================================================ host side

struct lbm_batch {
  int device = 0, sms = 1;
  int n = 0, model = 0, prec = 0, mode = LBM_BATCH_GRAPH;
  double rho_ref = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t capture = nullptr;  // private non-blocking stream used only for graph capture
  std::vector<olbm::Geometry> geo;
  std::vector<double> theta, tau;
  std::vector<long long> node0;  // offset of each domain in packed field arrays
  std::vector<size_t> off;       // byte offset of each domain's first buffer in the arena
  long long total_nodes = 0;
  char* arena = nullptr;
  size_t arena_bytes = 0;
  void* d_desc = nullptr;
  int4* d_tiles = nullptr;
  int2* d_ranges = nullptr;
  long long* d_nodes = nullptr;
  int ntiles = 0;
  double* d_partials = nullptr;
  double* d_diag = nullptr;  // n * 5, latest fused diagnostics
  double* d_diag_now = nullptr;
  unsigned long long* d_sticky = nullptr;
  olbm::GridBarrier* d_bar = nullptr;
  int* d_perr = nullptr;  // set by a bounded wait of the pipelined tile kernel that gave up
  olbm::LaunchCfg cfg{};
  int cur = 0;
  long long t = 0;
  bool initialised = false;
  int diag_every = 0;
  long long last_diag_t = -1;
  cudaGraphExec_t graph = nullptr;
  long long graph_key[4] = {-1, -1, -1, -1};
  char err[320] = {0};
};

namespace {

int bfail(lbm_batch* b, int status, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  if (b) {
    vsnprintf(b->err, sizeof(b->err), fmt, ap);
  } else {
    char msg[320];
    vsnprintf(msg, sizeof(msg), fmt, ap);
    olbm::set_thread_error(status, "%s", msg);
  }
  va_end(ap);
  return status;
}

int bcuda(lbm_batch* b, cudaError_t e, const char* what) {
  return bfail(b, e == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

template <typename CT> void fill_desc(lbm_batch* b, std::vector<olbm::Desc<CT>>& out) {
  out.resize(b->n);
  for (int k = 0; k < b->n; ++k) {
    olbm::Desc<CT>& d = out[k];
    d.g = b->geo[k];
    long long bytes = 0;
    lbm_layout(d.g.nx, d.g.ny, b->prec, nullptr, nullptr, &bytes);
    d.buf[0] = b->arena + b->off[k];
    d.buf[1] = b->arena + b->off[k] + (size_t)bytes;
    d.c = olbm::make_coef<CT>(b->theta[k], b->tau[k], b->rho_ref);
    d.pairs = olbm::uses_pairs(b->prec, d.g) ? 1 : 0;
    d.pad = 0;
  }
}

// Rebuild the tile list for the current launch shape.
int build_tiles(lbm_batch* b) {
  std::vector<int4> tiles;
  std::vector<int2> ranges(b->n);
  for (int k = 0; k < b->n; ++k) {
    const olbm::Geometry& g = b->geo[k];
    int cols, trows;
    if (b->cfg.kind == 1) {
      cols = olbm::stream_width(b->prec);
      trows = b->cfg.rows;
    } else {
      cols = olbm::uses_pairs(b->prec, g) ? 2 * b->cfg.bx : b->cfg.bx;
      trows = b->cfg.by * b->cfg.rows;
    }
    ranges[k].x = (int)tiles.size();
    for (int y0 = 0; y0 < g.ny; y0 += trows)
      for (int x0 = 0; x0 < g.nx; x0 += cols) tiles.push_back(make_int4(k, x0, y0, 0));
    ranges[k].y = (int)tiles.size() - ranges[k].x;
  }
  if (tiles.size() > (size_t)0x7fffffff) return bfail(b, LBM_EINVAL, "too many tiles");
  cudaError_t e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return bcuda(b, e, "lbm_batch tiles sync");
  cudaFree(b->d_tiles);
  cudaFree(b->d_ranges);
  cudaFree(b->d_partials);
  b->d_tiles = nullptr;
  b->d_ranges = nullptr;
  b->d_partials = nullptr;
  b->ntiles = (int)tiles.size();
  if ((e = cudaMalloc(&b->d_tiles, sizeof(int4) * tiles.size())) != cudaSuccess ||
      (e = cudaMalloc(&b->d_ranges, sizeof(int2) * ranges.size())) != cudaSuccess ||
      (e = cudaMalloc(&b->d_partials, sizeof(double) * 5 * tiles.size())) != cudaSuccess)
    return bcuda(b, e, "lbm_batch tile allocation");
  if ((e = cudaMemcpy(b->d_tiles, tiles.data(), sizeof(int4) * tiles.size(), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(b->d_ranges, ranges.data(), sizeof(int2) * ranges.size(), cudaMemcpyHostToDevice)) !=
          cudaSuccess)
    return bcuda(b, e, "lbm_batch tile upload");
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  return LBM_OK;
}

void free_batch(lbm_batch* b) {
  if (!b) return;
  if (b->graph) cudaGraphExecDestroy(b->graph);
  if (b->capture) cudaStreamDestroy(b->capture);
  cudaFree(b->arena);
  cudaFree(b->d_desc);
  cudaFree(b->d_tiles);
  cudaFree(b->d_ranges);
  cudaFree(b->d_nodes);
  cudaFree(b->d_partials);
  cudaFree(b->d_diag);
  cudaFree(b->d_diag_now);
  cudaFree(b->d_sticky);
  cudaFree(b->d_bar);
  cudaFree(b->d_perr);
  delete b;
}

int check_batch(lbm_batch* b) {
  if (!b) return LBM_EINVAL;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != b->device)
    return bfail(b, LBM_EINVAL, "the current CUDA device (%d) is not the batch's device (%d)", dev, b->device);
  return LBM_OK;
}

// Pipeline shape of a shifted storage form (the single-lattice one).
template <int PREC> struct StreamCfg {
  static constexpr int NC = PREC == 1 ? olbm::kStreamNC32 : olbm::kStreamNC16;
  static constexpr int STAGES = olbm::kStreamStages;
  using Shape = olbm::StreamShape<PREC, NC, STAGES>;
};

// Opt a pipelined kernel in to its shared-memory ring, once per kernel. Called
// before any launch or graph capture of the kernel (not during a capture).
template <auto K> cudaError_t allow_ring(int bytes) {
  static bool done = false;
  if (done) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(K, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) done = true;
  return e;
}

template <int PREC, int MODEL> cudaError_t allow_rings() {
  if constexpr (PREC == 0) {
    return cudaSuccess;
  } else {
    using C = StreamCfg<PREC>;
    constexpr int bytes = C::Shape::kSmemBytes;
    cudaError_t e = allow_ring<olbm::batch_stream_kernel<MODEL, PREC, true, C::NC, C::STAGES>>(bytes);
    if (e == cudaSuccess) e = allow_ring<olbm::batch_stream_kernel<MODEL, PREC, false, C::NC, C::STAGES>>(bytes);
    if (e == cudaSuccess) e = allow_ring<olbm::batch_stream_persistent_kernel<MODEL, PREC, C::NC, C::STAGES>>(bytes);
    return e;
  }
}

template <int PREC> cudaError_t allow_rings_p(int model) {
  switch (model) {
    case 0: return allow_rings<PREC, 0>();
    case 1: return allow_rings<PREC, 1>();
    case 2: return allow_rings<PREC, 2>();
    case 3: return allow_rings<PREC, 3>();
    default: return allow_rings<PREC, 4>();
  }
}

cudaError_t prepare_launch(const lbm_batch* b) {
  if (b->cfg.kind != 1) return cudaSuccess;
  switch (b->prec) {
    case LBM_F32_SHIFT: return allow_rings_p<1>(b->model);
    case LBM_F16_SHIFT: return allow_rings_p<2>(b->model);
    default: return cudaSuccess;
  }
}

template <int PREC, int MODEL>
cudaError_t launch_batch_stream(const lbm_batch* b, bool diag, int parity, cudaStream_t st) {
  if constexpr (PREC == 0) {
    return cudaErrorInvalidConfiguration;
  } else {
    using C = StreamCfg<PREC>;
    const auto* desc = static_cast<const olbm::Desc<float>*>(b->d_desc);
    auto k1 = olbm::batch_stream_kernel<MODEL, PREC, true, C::NC, C::STAGES>;
    auto k0 = olbm::batch_stream_kernel<MODEL, PREC, false, C::NC, C::STAGES>;
    auto kernel = diag ? k1 : k0;
    kernel<<<b->ntiles, C::NC + 32, C::Shape::kSmemBytes, st>>>(desc, b->d_tiles, parity, b->d_partials, b->cfg.rows,
                                                                 b->d_perr);
    return cudaGetLastError();
  }
}

template <int PREC, int MODEL>
cudaError_t launch_batch_step(const lbm_batch* b, bool diag, int parity, cudaStream_t st) {
  if (b->cfg.kind == 1) return launch_batch_stream<PREC, MODEL>(b, diag, parity, st);
  using T = typename olbm::Form<PREC>::T;
  const auto* desc = static_cast<const olbm::Desc<T>*>(b->d_desc);
  const dim3 block(b->cfg.bx, b->cfg.by);
  if (diag)
    olbm::batch_step_kernel<MODEL, PREC, true><<<b->ntiles, block, 0, st>>>(desc, b->d_tiles, parity, b->d_partials,
                                                                            b->cfg.rows);
  else
    olbm::batch_step_kernel<MODEL, PREC, false><<<b->ntiles, block, 0, st>>>(desc, b->d_tiles, parity,
                                                                             b->d_partials, b->cfg.rows);
  return cudaGetLastError();
}

template <int PREC>
cudaError_t launch_batch_step_p(const lbm_batch* b, bool diag, int parity, cudaStream_t st) {
  switch (b->model) {
    case 0: return launch_batch_step<PREC, 0>(b, diag, parity, st);
    case 1: return launch_batch_step<PREC, 1>(b, diag, parity, st);
    case 2: return launch_batch_step<PREC, 2>(b, diag, parity, st);
    case 3: return launch_batch_step<PREC, 3>(b, diag, parity, st);
    default: return launch_batch_step<PREC, 4>(b, diag, parity, st);
  }
}

cudaError_t launch_one_step(const lbm_batch* b, bool diag, int parity, cudaStream_t st) {
  switch (b->prec) {
    case LBM_F64: return launch_batch_step_p<0>(b, diag, parity, st);
    case LBM_F32_SHIFT: return launch_batch_step_p<1>(b, diag, parity, st);
    default: return launch_batch_step_p<2>(b, diag, parity, st);
  }
}

cudaError_t launch_finalize(const lbm_batch* b, double* out, unsigned long long* sticky, cudaStream_t st) {
  olbm::batch_finalize_kernel<<<b->n, 256, 0, st>>>(b->d_partials, b->d_ranges, b->d_nodes, b->rho_ref, out, sticky);
  return cudaGetLastError();
}

template <int PREC, int MODEL>
cudaError_t launch_persistent_stream(lbm_batch* b, int n, int parity0, cudaStream_t st) {
  if constexpr (PREC == 0) {
    return cudaErrorInvalidConfiguration;
  } else {
    using C = StreamCfg<PREC>;
    auto kernel = olbm::batch_stream_persistent_kernel<MODEL, PREC, C::NC, C::STAGES>;
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, C::NC + 32, C::Shape::kSmemBytes);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int grid = std::min(b->ntiles, per_sm * b->sms);
    const auto* desc = static_cast<const olbm::Desc<float>*>(b->d_desc);
    const int4* tiles = b->d_tiles;
    int ntiles = b->ntiles, rows = b->cfg.rows;
    olbm::GridBarrier* bar = b->d_bar;
    void* args[] = {(void*)&desc, (void*)&tiles, (void*)&ntiles, (void*)&parity0, (void*)&n, (void*)&rows,
                    (void*)&bar};
    e = cudaMemsetAsync(b->d_bar, 0, sizeof(olbm::GridBarrier), st);
    if (e != cudaSuccess) return e;
    return cudaLaunchCooperativeKernel((const void*)kernel, dim3(grid), dim3(C::NC + 32), args,
                                       (size_t)C::Shape::kSmemBytes, st);
  }
}

template <int PREC, int MODEL>
cudaError_t launch_persistent(lbm_batch* b, int n, int parity0, cudaStream_t st) {
  if (b->cfg.kind == 1) return launch_persistent_stream<PREC, MODEL>(b, n, parity0, st);
  using T = typename olbm::Form<PREC>::T;
  auto kernel = olbm::batch_persistent_kernel<MODEL, PREC>;
  const int threads = b->cfg.bx * b->cfg.by;
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const int grid = std::min(b->ntiles, per_sm * b->sms);
  const auto* desc = static_cast<const olbm::Desc<T>*>(b->d_desc);
  const int4* tiles = b->d_tiles;
  int ntiles = b->ntiles, rows = b->cfg.rows;
  olbm::GridBarrier* bar = b->d_bar;
  void* args[] = {(void*)&desc, (void*)&tiles, (void*)&ntiles, (void*)&parity0, (void*)&n, (void*)&rows, (void*)&bar};
  e = cudaMemsetAsync(b->d_bar, 0, sizeof(olbm::GridBarrier), st);
  if (e != cudaSuccess) return e;
  return cudaLaunchCooperativeKernel((const void*)kernel, dim3(grid), dim3(b->cfg.bx, b->cfg.by), args, 0, st);
}

template <int PREC>
cudaError_t launch_persistent_p(lbm_batch* b, int n, int parity0, cudaStream_t st) {
  switch (b->model) {
    case 0: return launch_persistent<PREC, 0>(b, n, parity0, st);
    case 1: return launch_persistent<PREC, 1>(b, n, parity0, st);
    case 2: return launch_persistent<PREC, 2>(b, n, parity0, st);
    case 3: return launch_persistent<PREC, 3>(b, n, parity0, st);
    default: return launch_persistent<PREC, 4>(b, n, parity0, st);
  }
}

template <int PREC>
cudaError_t launch_batch_diag(const lbm_batch* b, cudaStream_t st) {
  using T = typename olbm::Form<PREC>::T;
  const auto* desc = static_cast<const olbm::Desc<T>*>(b->d_desc);
  if (b->cfg.kind == 1) {
    const int w = olbm::stream_width(b->prec);
    olbm::batch_diag_kernel<PREC><<<b->ntiles, 256, 0, st>>>(desc, b->d_tiles, b->cur, w, w, b->cfg.rows, b->rho_ref,
                                                             b->d_partials);
  } else {
    olbm::batch_diag_kernel<PREC><<<b->ntiles, dim3(b->cfg.bx, b->cfg.by), 0, st>>>(
        desc, b->d_tiles, b->cur, b->cfg.bx, 2 * b->cfg.bx, b->cfg.by * b->cfg.rows, b->rho_ref, b->d_partials);
  }
  return cudaGetLastError();
}

}  // namespace

extern "C" {

int lbm_batch_create(int n, const int* nx, const int* ny, const double* theta, const double* tau, int model,
                     int prec, void* stream, lbm_batch** out) {
  if (!out || n < 1 || !nx || !ny || !theta || !tau) return bfail(nullptr, LBM_EINVAL, "lbm_batch_create: bad arguments");
  if (model < LBM_LBGK || model > LBM_OREG_COMPLETE_NEQ) return bfail(nullptr, LBM_EINVAL, "unknown model %d", model);
  if (prec < LBM_F64 || prec > LBM_F16_SHIFT) return bfail(nullptr, LBM_EINVAL, "unknown storage form %d", prec);
  lbm_batch* b = new (std::nothrow) lbm_batch();
  if (!b) return bfail(nullptr, LBM_ENOMEM, "host allocation failed");
  b->n = n;
  b->model = model;
  b->prec = prec;
  b->rho_ref = prec == LBM_F64 ? 0.0 : 1.0;
  b->stream = static_cast<cudaStream_t>(stream);
  size_t arena = 0;
  for (int k = 0; k < n; ++k) {
    long long pitch, plane, bytes;
    if (lbm_layout(nx[k], ny[k], prec, &pitch, &plane, &bytes) != LBM_OK) {
      delete b;
      return bfail(nullptr, LBM_EINVAL, "domain %d: invalid size %d x %d", k, nx[k], ny[k]);
    }
    if (!(theta[k] > 0.0 && theta[k] < 1.0) || !(tau[k] > 0.5) || !std::isfinite(tau[k])) {
      delete b;
      return bfail(nullptr, LBM_EINVAL, "domain %d: theta must lie in (0, 1) and tau exceed 1/2", k);
    }
    b->geo.push_back(olbm::Geometry{nx[k], ny[k], pitch, plane});
    b->theta.push_back(theta[k]);
    b->tau.push_back(tau[k]);
    b->node0.push_back(b->total_nodes);
    b->total_nodes += (long long)nx[k] * ny[k];
    b->off.push_back(arena);
    arena = align_up(arena + 2 * (size_t)bytes, 256);
  }
  cudaError_t e = cudaGetDevice(&b->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->device);
  if (e != cudaSuccess) {
    delete b;
    return bfail(nullptr, LBM_ECUDA, "lbm_batch_create: %s", cudaGetErrorString(e));
  }
  b->arena_bytes = arena;
  std::vector<long long> nodes(n);
  for (int k = 0; k < n; ++k) nodes[k] = (long long)nx[k] * ny[k];
  const size_t desc_bytes =
      (size_t)n * (prec == LBM_F64 ? sizeof(olbm::Desc<double>) : sizeof(olbm::Desc<float>));
  if ((e = cudaMalloc(&b->arena, arena)) != cudaSuccess || (e = cudaMalloc(&b->d_desc, desc_bytes)) != cudaSuccess ||
      (e = cudaMalloc(&b->d_nodes, sizeof(long long) * n)) != cudaSuccess ||
      (e = cudaMalloc(&b->d_diag, sizeof(double) * 5 * n)) != cudaSuccess ||
      (e = cudaMalloc(&b->d_diag_now, sizeof(double) * 5 * n)) != cudaSuccess ||
      (e = cudaMalloc(&b->d_sticky, sizeof(unsigned long long))) != cudaSuccess ||
      (e = cudaMalloc(&b->d_bar, sizeof(olbm::GridBarrier))) != cudaSuccess ||
      (e = cudaMalloc(&b->d_perr, sizeof(int))) != cudaSuccess) {
    free_batch(b);
    cudaGetLastError();
    return bfail(nullptr, LBM_ENOMEM, "lbm_batch_create: %s", cudaGetErrorString(e));
  }
  if (prec == LBM_F64) {
    std::vector<olbm::Desc<double>> d;
    fill_desc(b, d);
    e = cudaMemcpy(b->d_desc, d.data(), desc_bytes, cudaMemcpyHostToDevice);
  } else {
    std::vector<olbm::Desc<float>> d;
    fill_desc(b, d);
    e = cudaMemcpy(b->d_desc, d.data(), desc_bytes, cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess) e = cudaMemcpy(b->d_nodes, nodes.data(), sizeof(long long) * n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(b->arena, 0, arena);
  if (e == cudaSuccess) e = cudaMemset(b->d_sticky, 0, sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMemset(b->d_perr, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(b->d_diag, 0, sizeof(double) * 5 * n);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    free_batch(b);
    return bfail(nullptr, LBM_ECUDA, "lbm_batch_create: %s", cudaGetErrorString(e));
  }
  // Default tiles: FP64 the column routine with 64 x 2 threads and 16 rows; the
  // shifted forms the bulk-copy pipeline on tiles of 32 rows.
  if (prec == LBM_F64) {
    b->cfg.bx = 64, b->cfg.by = 2, b->cfg.rows = 16;
  } else {
    b->cfg.kind = 1, b->cfg.bx = 0, b->cfg.by = 1, b->cfg.rows = 32;
  }
  int s = build_tiles(b);
  if (s != LBM_OK) {
    char msg[320];
    snprintf(msg, sizeof(msg), "%s", b->err);
    free_batch(b);
    return bfail(nullptr, s, "%s", msg);
  }
  *out = b;
  return LBM_OK;
}

int lbm_batch_destroy(lbm_batch* b) {
  if (!b) return LBM_OK;
  cudaStreamSynchronize(b->stream);
  free_batch(b);
  return LBM_OK;
}

int lbm_batch_set_launch(lbm_batch* b, int bx, int by, int rows) {
  int s = check_batch(b);
  if (s != LBM_OK) return s;
  olbm::LaunchCfg k;
  k.bx = bx;
  k.by = by;
  k.rows = rows;
  if (!olbm::valid_cfg(k))
    return bfail(b, LBM_EINVAL, "tile shape %dx%d x %d rows invalid (bx a multiple of 32, bx*by <= 512, rows 1..64)",
                 bx, by, rows);
  b->cfg = k;
  return build_tiles(b);
}

int lbm_batch_set_launch_ex(lbm_batch* b, int kind, int bx, int by, int rows) {
  int s = check_batch(b);
  if (s != LBM_OK) return s;
  if (kind == 0) return lbm_batch_set_launch(b, bx, by, rows);
  if (kind != 1 || b->prec == LBM_F64 || rows < 1 || rows > 4096)
    return bfail(b, LBM_EINVAL,
                 "launch kind %d with %d rows invalid (kind 1: shifted storage forms only, rows 1..4096)", kind, rows);
  olbm::LaunchCfg k;
  k.kind = 1;
  k.bx = 0;
  k.by = 1;
  k.rows = rows;
  b->cfg = k;
  return build_tiles(b);
}

int lbm_batch_get_launch_ex(const lbm_batch* b, int* kind, int* bx, int* by, int* rows, int* ntiles) {
  if (!b || !kind) return LBM_EINVAL;
  *kind = b->cfg.kind;
  return lbm_batch_get_launch(b, bx, by, rows, ntiles);
}

int lbm_batch_get_launch(const lbm_batch* b, int* bx, int* by, int* rows, int* ntiles) {
  if (!b) return LBM_EINVAL;
  if (bx) *bx = b->cfg.bx;
  if (by) *by = b->cfg.by;
  if (rows) *rows = b->cfg.rows;
  if (ntiles) *ntiles = b->ntiles;
  return LBM_OK;
}

int lbm_batch_set_mode(lbm_batch* b, int mode) {
  if (!b) return LBM_EINVAL;
  if (mode != LBM_BATCH_GRAPH && mode != LBM_BATCH_PERSISTENT) return bfail(b, LBM_EINVAL, "unknown mode %d", mode);
  b->mode = mode;
  return LBM_OK;
}

int lbm_batch_set_diagnostics_interval(lbm_batch* b, int every) {
  if (!b || every < 0) return LBM_EINVAL;
  b->diag_every = every;
  return LBM_OK;
}

int lbm_batch_init(lbm_batch* b, const double* d_rho, const double* d_ux, const double* d_uy) {
  int s = check_batch(b);
  if (s != LBM_OK) return s;
  if (!d_rho || !d_ux || !d_uy) return bfail(b, LBM_EINVAL, "lbm_batch_init: NULL field pointer");
  for (int k = 0; k < b->n; ++k) {
    long long bytes = 0;
    lbm_layout(b->geo[k].nx, b->geo[k].ny, b->prec, nullptr, nullptr, &bytes);
    void* dst = b->arena + b->off[k] + (size_t)(b->cur ? bytes : 0);
    const long long o = b->node0[k];
    cudaError_t e;
    switch (b->prec) {
      case LBM_F64: e = olbm::launch_init_f64(d_rho + o, d_ux + o, d_uy + o, b->geo[k], b->theta[k], b->rho_ref, dst, b->stream); break;
      case LBM_F32_SHIFT: e = olbm::launch_init_f32(d_rho + o, d_ux + o, d_uy + o, b->geo[k], b->theta[k], b->rho_ref, dst, b->stream); break;
      default: e = olbm::launch_init_f16(d_rho + o, d_ux + o, d_uy + o, b->geo[k], b->theta[k], b->rho_ref, dst, b->stream); break;
    }
    if (e != cudaSuccess) return bcuda(b, e, "lbm_batch_init");
  }
  cudaError_t e = cudaMemsetAsync(b->d_sticky, 0, sizeof(unsigned long long), b->stream);
  if (e != cudaSuccess) return bcuda(b, e, "lbm_batch_init reset");
  b->initialised = true;
  b->t = 0;
  b->last_diag_t = -1;
  return LBM_OK;
}

static void* domain_buffer(lbm_batch* b, int k, int which) {
  long long bytes = 0;
  lbm_layout(b->geo[k].nx, b->geo[k].ny, b->prec, nullptr, nullptr, &bytes);
  return b->arena + b->off[k] + (size_t)(which ? bytes : 0);
}

int lbm_batch_get_state(lbm_batch* b, int k, double* d_f) {
  int s = check_batch(b);
  if (s != LBM_OK) return s;
  if (k < 0 || k >= b->n || !d_f) return bfail(b, LBM_EINVAL, "lbm_batch_get_state: bad domain or pointer");
  const void* src = domain_buffer(b, k, b->cur);
  cudaError_t e;
  switch (b->prec) {
    case LBM_F64: e = olbm::launch_get_state_f64(src, b->geo[k], b->theta[k], b->rho_ref, d_f, b->stream); break;
    case LBM_F32_SHIFT: e = olbm::launch_get_state_f32(src, b->geo[k], b->theta[k], b->rho_ref, d_f, b->stream); break;
    default: e = olbm::launch_get_state_f16(src, b->geo[k], b->theta[k], b->rho_ref, d_f, b->stream); break;
  }
  return e == cudaSuccess ? LBM_OK : bcuda(b, e, "lbm_batch_get_state");
}

int lbm_batch_set_state(lbm_batch* b, int k, const double* d_f) {
  int s = check_batch(b);
  if (s != LBM_OK) return s;
  if (k < 0 || k >= b->n || !d_f) return bfail(b, LBM_EINVAL, "lbm_batch_set_state: bad domain or pointer");
  void* dst = domain_buffer(b, k, b->cur);
  cudaError_t e;
  switch (b->prec) {
    case LBM_F64: e = olbm::launch_set_state_f64(d_f, b->geo[k], b->theta[k], b->rho_ref, dst, b->stream); break;
    case LBM_F32_SHIFT: e = olbm::launch_set_state_f32(d_f, b->geo[k], b->theta[k], b->rho_ref, dst, b->stream); break;
    default: e = olbm::launch_set_state_f16(d_f, b->geo[k], b->theta[k], b->rho_ref, dst, b->stream); break;
  }
  if (e != cudaSuccess) return bcuda(b, e, "lbm_batch_set_state");
  b->initialised = true;
  return LBM_OK;
}

int lbm_batch_moments(lbm_batch* b, double* d_rho, double* d_ux, double* d_uy) {
  int s = check_batch(b);
  if (s != LBM_OK) return s;
  if (!d_rho || !d_ux || !d_uy) return bfail(b, LBM_EINVAL, "lbm_batch_moments: NULL field pointer");
  for (int k = 0; k < b->n; ++k) {
    const void* src = domain_buffer(b, k, b->cur);
    const long long o = b->node0[k];
    cudaError_t e;
    switch (b->prec) {
      case LBM_F64: e = olbm::launch_moments_f64(src, b->geo[k], b->rho_ref, d_rho + o, d_ux + o, d_uy + o, b->stream); break;
      case LBM_F32_SHIFT: e = olbm::launch_moments_f32(src, b->geo[k], b->rho_ref, d_rho + o, d_ux + o, d_uy + o, b->stream); break;
      default: e = olbm::launch_moments_f16(src, b->geo[k], b->rho_ref, d_rho + o, d_ux + o, d_uy + o, b->stream); break;
    }
    if (e != cudaSuccess) return bcuda(b, e, "lbm_batch_moments");
  }
  return LBM_OK;
}

int lbm_batch_step(lbm_batch* b, int n) {
  int s = check_batch(b);
  if (s != LBM_OK) return s;
  if (n < 0) return bfail(b, LBM_EINVAL, "lbm_batch_step: n must be >= 0");
  if (!b->initialised) return bfail(b, LBM_ESTATE, "lbm_batch_step before lbm_batch_init");
  if (n == 0) return LBM_OK;
  cudaError_t e = prepare_launch(b);
  if (e != cudaSuccess) return bcuda(b, e, "lbm_batch_step kernel attributes");
  if (b->mode == LBM_BATCH_PERSISTENT) {
    switch (b->prec) {
      case LBM_F64: e = launch_persistent_p<0>(b, n, b->cur, b->stream); break;
      case LBM_F32_SHIFT: e = launch_persistent_p<1>(b, n, b->cur, b->stream); break;
      default: e = launch_persistent_p<2>(b, n, b->cur, b->stream); break;
    }
    if (e != cudaSuccess) return bcuda(b, e, "lbm_batch_step persistent launch");
    int timed_out = 0;
    e = cudaMemcpyAsync(&timed_out, &b->d_bar->err, sizeof(int), cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "lbm_batch_step persistent");
    b->cur = (int)((b->cur + n) & 1);
    b->t += n;
    if (timed_out) return bfail(b, LBM_ETIMEOUT, "a grid barrier of the persistent batch kernel timed out");
    return LBM_OK;
  }
  // Graph mode: capture the n launches once per (n, parity, diagnostics phase), replay.
  const long long phase = b->diag_every > 0 ? b->t % b->diag_every : -1;
  const long long key[4] = {n, b->cur, b->diag_every, phase};
  if (!b->graph || !std::equal(key, key + 4, b->graph_key)) {
    if (b->graph) {
      cudaGraphExecDestroy(b->graph);
      b->graph = nullptr;
    }
    cudaGraph_t g = nullptr;
    e = cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return bcuda(b, e, "lbm_batch_step capture");
    cudaError_t le = cudaSuccess;
    for (int k = 0; k < n && le == cudaSuccess; ++k) {
      const long long tk = b->t + k;
      const bool diag = b->diag_every > 0 && (tk % b->diag_every) == 0;
      le = launch_one_step(b, diag, (int)((b->cur + k) & 1), b->capture);
      if (le == cudaSuccess && diag) le = launch_finalize(b, b->d_diag, b->d_sticky, b->capture);
    }
    e = cudaStreamEndCapture(b->capture, &g);
    if (le != cudaSuccess || e != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return bcuda(b, le != cudaSuccess ? le : e, "lbm_batch_step capture");
    }
    e = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      b->graph = nullptr;
      return bcuda(b, e, "lbm_batch_step graph instantiate");
    }
    std::copy(key, key + 4, b->graph_key);
  }
  e = cudaGraphLaunch(b->graph, b->stream);
  if (e != cudaSuccess) return bcuda(b, e, "lbm_batch_step graph launch");
  if (b->diag_every > 0) {
    const long long last = b->t + n - 1;
    const long long ld = last - (last % b->diag_every);  // latest fused pass in [t, t + n), if any
    if (ld >= b->t) b->last_diag_t = ld;
  }
  b->cur = (int)((b->cur + n) & 1);
  b->t += n;
  return LBM_OK;
}

int lbm_batch_step_diagnostics(lbm_batch* b, double* h_out, long long* h_time) {
  int s = check_batch(b);
  if (s != LBM_OK) return s;
  if (!h_out) return bfail(b, LBM_EINVAL, "lbm_batch_step_diagnostics: NULL output");
  unsigned long long bad = 0;
  int timed_out = 0;
  cudaError_t e = cudaMemcpyAsync(h_out, b->d_diag, sizeof(double) * 5 * b->n, cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, b->d_sticky, sizeof(bad), cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&timed_out, b->d_perr, sizeof(int), cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return bcuda(b, e, "lbm_batch_step_diagnostics");
  if (timed_out) return bfail(b, LBM_ETIMEOUT, "a bounded device-side wait of the pipelined tile kernel gave up");
  if (h_time) *h_time = b->last_diag_t;
  if (bad > 0) return bfail(b, LBM_ENONFINITE, "%llu non-finite node(s) met by fused diagnostics", bad);
  return LBM_OK;
}

int lbm_batch_diagnostics(lbm_batch* b, double* h_out) {
  int s = check_batch(b);
  if (s != LBM_OK) return s;
  if (!h_out) return bfail(b, LBM_EINVAL, "lbm_batch_diagnostics: NULL output");
  if (!b->initialised) return bfail(b, LBM_ESTATE, "lbm_batch_diagnostics before lbm_batch_init");
  cudaError_t e;
  switch (b->prec) {
    case LBM_F64: e = launch_batch_diag<0>(b, b->stream); break;
    case LBM_F32_SHIFT: e = launch_batch_diag<1>(b, b->stream); break;
    default: e = launch_batch_diag<2>(b, b->stream); break;
  }
  if (e == cudaSuccess) e = launch_finalize(b, b->d_diag_now, nullptr, b->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h_out, b->d_diag_now, sizeof(double) * 5 * b->n, cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return bcuda(b, e, "lbm_batch_diagnostics");
  for (int k = 0; k < b->n; ++k)
    if (h_out[5 * k + 4] > 0) return bfail(b, LBM_ENONFINITE, "domain %d holds non-finite populations", k);
  return LBM_OK;
}

int lbm_batch_info(const lbm_batch* b, long long* total_nodes, long long* arena_bytes, long long* t) {
  if (!b) return LBM_EINVAL;
  if (total_nodes) *total_nodes = b->total_nodes;
  if (arena_bytes) *arena_bytes = (long long)b->arena_bytes;
  if (t) *t = b->t;
  return LBM_OK;
}

int lbm_batch_sync(lbm_batch* b) {
  int s = check_batch(b);
  if (s != LBM_OK) return s;
  cudaError_t e = cudaStreamSynchronize(b->stream);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return bcuda(b, e, "lbm_batch_sync");
  unsigned long long bad = 0;
  int timed_out = 0;
  e = cudaMemcpyAsync(&bad, b->d_sticky, sizeof(bad), cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&timed_out, b->d_perr, sizeof(int), cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return bcuda(b, e, "lbm_batch_sync");
  if (timed_out) return bfail(b, LBM_ETIMEOUT, "a bounded device-side wait of the pipelined tile kernel gave up");
  if (bad > 0) return bfail(b, LBM_ENONFINITE, "%llu non-finite node(s) met by fused diagnostics", bad);
  return LBM_OK;
}

const char* lbm_batch_last_error(const lbm_batch* b) { return b ? b->err : lbm_last_error(nullptr); }

}  // extern "C"

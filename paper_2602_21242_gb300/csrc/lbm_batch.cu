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
//                         loops over the n steps (captured with its barrier
//                         reset into a CUDA graph once per n and buffer parity,
//                         and replayed), tiles strided over the grid,
//                         separated by a grid barrier whose waits are bounded:
//                         a barrier that does not complete within ~1 s sets an
//                         error flag, every block leaves, and the call reports
//                         LBM_ETIMEOUT. Loads bypass L1 (data written by other
//                         blocks earlier in the same launch). No fused
//                         diagnostics; lbm_batch_diagnostics computes them.
// With launch kind 2 (shifted forms) both modes take two steps a launch: the
// graph holds n / 2 two-step launches, the persistent kernel loops over n / 2
// pairs of steps (barrier between pairs); an odd last step is a single-step
// launch of the kind 1 tiles (in persistent mode a second cooperative launch in
// the same graph, which keeps the first one's error flag).
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <new>
#include <vector>

#include "lbm.h"
#include "lbm_batch.h"

namespace olbm {

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
  // Fused diagnostics in graph mode: diagnosed steps take four partials buffers in
  // turn (a two-step launch takes two) and each step's final sum is a branch of the
  // graph (captured from a second stream) beside the following steps.
  static constexpr int kParts = 4;
  cudaStream_t capture_side = nullptr;
  cudaEvent_t ev_step[kParts] = {};
  cudaEvent_t ev_fin[kParts] = {};
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
  // launch kind 2: the two-step tiles (2 NC - 2 columns) and their per-domain ranges;
  // the single steps of an odd count take the kind 1 tiles above
  int4* d_tiles2 = nullptr;
  int2* d_ranges2 = nullptr;
  int ntiles2 = 0;
  double* d_parts[kParts] = {};  // per-tile partials, max(ntiles, ntiles2) each
  double* d_diag = nullptr;  // n * 5, latest fused diagnostics
  double* d_diag_now = nullptr;
  unsigned long long* d_sticky = nullptr;
  olbm::GridBarrier* d_bar = nullptr;
  int* d_perr = nullptr;
  int* d_ctr = nullptr;  // tile counters of the persistent pipelined kernel  // set by a bounded wait of the pipelined tile kernel that gave up
  olbm::LaunchCfg cfg{};
  int cur = 0;
  long long t = 0;
  bool initialised = false;
  int diag_every = 0;
  long long last_diag_t = -1;
  cudaGraphExec_t graph = nullptr;
  long long graph_key[4] = {-1, -1, -1, -1};
  int graph_parity_end = 0;  // buffer holding the state after a replay of `graph`
  // Persistent mode: the barrier reset and the cooperative launch of n steps,
  // captured once per (n, buffer parity) and replayed.
  cudaGraphExec_t pgraph = nullptr;
  long long pgraph_key[2] = {-1, -1};
  int pgraph_parity_end = 0;  // buffer holding the state after a replay of `pgraph`
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

// Tiles of cols x trows of every domain, domain after domain, and each domain's range.
void cut_tiles(const lbm_batch* b, int cols, int trows, std::vector<int4>& tiles, std::vector<int2>& ranges) {
  tiles.clear();
  ranges.assign(b->n, make_int2(0, 0));
  for (int k = 0; k < b->n; ++k) {
    const olbm::Geometry& g = b->geo[k];
    ranges[k].x = (int)tiles.size();
    for (int y0 = 0; y0 < g.ny; y0 += trows)
      for (int x0 = 0; x0 < g.nx; x0 += cols) tiles.push_back(make_int4(k, x0, y0, 0));
    ranges[k].y = (int)tiles.size() - ranges[k].x;
  }
}

// Rebuild the tile lists for the current launch shape.
int build_tiles(lbm_batch* b) {
  std::vector<int4> tiles, tiles2;
  std::vector<int2> ranges, ranges2;
  if (b->cfg.kind == 1 || b->cfg.kind == 2) {
    const int nc = olbm::batch_stream_nc(b->prec, b->cfg.kind == 2 ? 0 : b->cfg.bx);
    cut_tiles(b, 2 * nc, b->cfg.rows, tiles, ranges);
    if (b->cfg.kind == 2) cut_tiles(b, olbm::stream2_width(b->prec), b->cfg.rows, tiles2, ranges2);
  } else {
    // kind 0: (bx or 2 bx) columns per domain, by x rows rows
    tiles.clear();
    ranges.assign(b->n, make_int2(0, 0));
    for (int k = 0; k < b->n; ++k) {
      const olbm::Geometry& g = b->geo[k];
      const int cols = olbm::uses_pairs(b->prec, g) ? 2 * b->cfg.bx : b->cfg.bx, trows = b->cfg.by * b->cfg.rows;
      ranges[k].x = (int)tiles.size();
      for (int y0 = 0; y0 < g.ny; y0 += trows)
        for (int x0 = 0; x0 < g.nx; x0 += cols) tiles.push_back(make_int4(k, x0, y0, 0));
      ranges[k].y = (int)tiles.size() - ranges[k].x;
    }
  }
  if (tiles.size() > (size_t)0x7fffffff || tiles2.size() > (size_t)0x7fffffff)
    return bfail(b, LBM_EINVAL, "too many tiles");
  cudaError_t e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return bcuda(b, e, "lbm_batch tiles sync");
  cudaFree(b->d_tiles);
  cudaFree(b->d_ranges);
  cudaFree(b->d_tiles2);
  cudaFree(b->d_ranges2);
  b->d_tiles = nullptr;
  b->d_ranges = nullptr;
  b->d_tiles2 = nullptr;
  b->d_ranges2 = nullptr;
  for (int q = 0; q < lbm_batch::kParts; ++q) {
    cudaFree(b->d_parts[q]);
    b->d_parts[q] = nullptr;
  }
  b->ntiles = (int)tiles.size();
  b->ntiles2 = (int)tiles2.size();
  const size_t nparts = std::max(tiles.size(), tiles2.size());
  e = cudaMalloc(&b->d_tiles, sizeof(int4) * tiles.size());
  if (e == cudaSuccess) e = cudaMalloc(&b->d_ranges, sizeof(int2) * ranges.size());
  if (e == cudaSuccess && !tiles2.empty()) e = cudaMalloc(&b->d_tiles2, sizeof(int4) * tiles2.size());
  if (e == cudaSuccess && !tiles2.empty()) e = cudaMalloc(&b->d_ranges2, sizeof(int2) * ranges2.size());
  for (int q = 0; q < lbm_batch::kParts && e == cudaSuccess; ++q)
    e = cudaMalloc(&b->d_parts[q], sizeof(double) * 5 * nparts);
  if (e != cudaSuccess) return bcuda(b, e, "lbm_batch tile allocation");
  e = cudaMemcpy(b->d_tiles, tiles.data(), sizeof(int4) * tiles.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(b->d_ranges, ranges.data(), sizeof(int2) * ranges.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !tiles2.empty())
    e = cudaMemcpy(b->d_tiles2, tiles2.data(), sizeof(int4) * tiles2.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !tiles2.empty())
    e = cudaMemcpy(b->d_ranges2, ranges2.data(), sizeof(int2) * ranges2.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return bcuda(b, e, "lbm_batch tile upload");
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  if (b->pgraph) {
    cudaGraphExecDestroy(b->pgraph);
    b->pgraph = nullptr;
  }
  return LBM_OK;
}

void free_batch(lbm_batch* b) {
  if (!b) return;
  if (b->graph) cudaGraphExecDestroy(b->graph);
  if (b->pgraph) cudaGraphExecDestroy(b->pgraph);
  if (b->capture) cudaStreamDestroy(b->capture);
  if (b->capture_side) cudaStreamDestroy(b->capture_side);
  for (int k = 0; k < lbm_batch::kParts; ++k) {
    if (b->ev_step[k]) cudaEventDestroy(b->ev_step[k]);
    if (b->ev_fin[k]) cudaEventDestroy(b->ev_fin[k]);
    cudaFree(b->d_parts[k]);
  }
  cudaFree(b->arena);
  cudaFree(b->d_desc);
  cudaFree(b->d_tiles);
  cudaFree(b->d_ranges);
  cudaFree(b->d_tiles2);
  cudaFree(b->d_ranges2);
  cudaFree(b->d_nodes);
  cudaFree(b->d_diag);
  cudaFree(b->d_diag_now);
  cudaFree(b->d_sticky);
  cudaFree(b->d_bar);
  cudaFree(b->d_perr);
  cudaFree(b->d_ctr);
  delete b;
}

int check_batch(lbm_batch* b) {
  if (!b) return LBM_EINVAL;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != b->device)
    return bfail(b, LBM_EINVAL, "the current CUDA device (%d) is not the batch's device (%d)", dev, b->device);
  return LBM_OK;
}

olbm::BatchLaunch view(const lbm_batch* b) {
  olbm::BatchLaunch v;
  v.model = b->model;
  v.cfg = b->cfg;
  if (b->cfg.kind == 2) v.cfg.kind = 1, v.cfg.bx = 0;  // single steps: the kind 1 tiles
  v.desc = b->d_desc;
  v.tiles = b->d_tiles;
  v.ntiles = b->ntiles;
  v.tiles2 = b->d_tiles2;
  v.ntiles2 = b->ntiles2;
  v.partials = b->d_parts[0];
  v.perr = b->d_perr;
  v.bar = b->d_bar;
  v.ctr = b->d_ctr;
  v.sms = b->sms;
  return v;
}

// Shared-memory opt-in of the pipelined kernels; before any launch or capture.
cudaError_t prepare_launch(const lbm_batch* b) {
  cudaError_t e;
  switch (b->prec) {
    case LBM_F64: return olbm::batch_prepare_f64(view(b));
    case LBM_F32_SHIFT: e = olbm::batch_prepare_f32(view(b)); break;
    default: e = olbm::batch_prepare_f16(view(b)); break;
  }
  if (e != cudaSuccess || b->cfg.kind != 2) return e;
  return b->prec == LBM_F32_SHIFT ? olbm::batch_prepare2_f32(view(b)) : olbm::batch_prepare2_f16(view(b));
}

// Two steps of every domain in one launch (kind 2) from buffer `parity`.
cudaError_t launch_two_steps(const lbm_batch* b, bool diag1, bool diag2, int parity, cudaStream_t st,
                             double* partials1, double* partials2) {
  olbm::BatchLaunch v = view(b);
  v.partials = partials1;
  v.partials2 = partials2;
  return b->prec == LBM_F32_SHIFT ? olbm::batch_step2_f32(v, diag1, diag2, parity, st)
                                  : olbm::batch_step2_f16(v, diag1, diag2, parity, st);
}

cudaError_t launch_one_step(const lbm_batch* b, bool diag, int parity, cudaStream_t st, double* partials) {
  olbm::BatchLaunch v = view(b);
  v.partials = partials;
  switch (b->prec) {
    case LBM_F64: return olbm::batch_step_f64(v, diag, parity, st);
    case LBM_F32_SHIFT: return olbm::batch_step_f32(v, diag, parity, st);
    default: return olbm::batch_step_f16(v, diag, parity, st);
  }
}

cudaError_t launch_persistent(const lbm_batch* b, int n, int parity0, cudaStream_t st, bool keep_err = false) {
  olbm::BatchLaunch v = view(b);
  v.keep_err = keep_err;
  switch (b->prec) {
    case LBM_F64: return olbm::batch_persistent_f64(v, n, parity0, st);
    case LBM_F32_SHIFT: return olbm::batch_persistent_f32(v, n, parity0, st);
    default: return olbm::batch_persistent_f16(v, n, parity0, st);
  }
}

// Persistent mode with launch kind 2: n / 2 pairs of steps in one cooperative launch,
// then, for odd n, the last step in a single-step one. Returns the parity after them.
cudaError_t launch_persistent_pairs(const lbm_batch* b, int n, int parity0, cudaStream_t st, int& parity_end) {
  const int pairs = n / 2;
  olbm::BatchLaunch v = view(b);
  cudaError_t e = b->prec == LBM_F32_SHIFT ? olbm::batch_persistent2_f32(v, pairs, parity0, st)
                                           : olbm::batch_persistent2_f16(v, pairs, parity0, st);
  int parity = parity0 ^ (pairs & 1);
  if (e == cudaSuccess && (n & 1)) {
    e = launch_persistent(b, 1, parity, st, true);
    parity ^= 1;
  }
  parity_end = parity;
  return e;
}

cudaError_t launch_diag(const lbm_batch* b, cudaStream_t st) {
  switch (b->prec) {
    case LBM_F64: return olbm::batch_diag_f64(view(b), b->cur, b->rho_ref, st);
    case LBM_F32_SHIFT: return olbm::batch_diag_f32(view(b), b->cur, b->rho_ref, st);
    default: return olbm::batch_diag_f16(view(b), b->cur, b->rho_ref, st);
  }
}

// Per-domain sums of one launch's partials; ranges: the tile ranges of that launch's list.
cudaError_t launch_finalize(const lbm_batch* b, const double* partials, double* out, unsigned long long* sticky,
                            cudaStream_t st, const int2* ranges = nullptr) {
  olbm::batch_finalize_kernel<<<b->n, 256, 0, st>>>(partials, ranges ? ranges : b->d_ranges, b->d_nodes,
                                                    b->rho_ref, out, sticky);
  return cudaGetLastError();
}

}  // namespace

extern "C" {

int lbm_batch_create(int n, const int* nx, const int* ny, const double* theta, const double* tau, int model,
                     int prec, void* stream, lbm_batch** out) {
  if (!out || n < 1 || !nx || !ny || !theta || !tau) return bfail(nullptr, LBM_EINVAL, "lbm_batch_create: bad arguments");
  if (model < LBM_LBGK || model > LBM_LBGK_POLY) return bfail(nullptr, LBM_EINVAL, "unknown model %d", model);
  if (prec < LBM_F64 || prec > LBM_F16_SHIFT)
    return bfail(nullptr, LBM_EINVAL, "storage form %d not available for batches (LBM_F64, LBM_F32_SHIFT, LBM_F16_SHIFT)",
                 prec);
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
      (e = cudaMalloc(&b->d_perr, sizeof(int))) != cudaSuccess ||
      (e = cudaMalloc(&b->d_ctr, 2 * sizeof(int))) != cudaSuccess) {
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
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->capture_side, cudaStreamNonBlocking);
  for (int k = 0; k < lbm_batch::kParts && e == cudaSuccess; ++k) {
    e = cudaEventCreateWithFlags(&b->ev_step[k], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_fin[k], cudaEventDisableTiming);
  }
  if (e != cudaSuccess) {
    free_batch(b);
    return bfail(nullptr, LBM_ECUDA, "lbm_batch_create: %s", cudaGetErrorString(e));
  }
  // Default tiles: FP64 the column routine with 64 x 2 threads and 16 rows; FP16
  // the bulk-copy pipeline on tiles of 32 rows; FP32 two steps a launch on tiles of
  // 32 rows (256 Taylor-Green domains N ~ U{64..512}, diagnostics every step: 113.3
  // GLUPS in graph mode against 83.3 for the single-step pipeline; the persistent
  // mode takes single steps either way).
  if (prec == LBM_F64) {
    b->cfg.bx = 64, b->cfg.by = 2, b->cfg.rows = 16;
  } else {
    b->cfg.kind = prec == LBM_F32_SHIFT ? 2 : 1, b->cfg.bx = 0, b->cfg.by = 1, b->cfg.rows = 32;
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
  if ((kind != 1 && kind != 2) || b->prec == LBM_F64 || rows < 1 || rows > 4096 ||
      !olbm::batch_stream_nc_valid(b->prec, bx) || (kind == 2 && bx != 0))
    return bfail(b, LBM_EINVAL,
                 "launch kind %d, bx %d, %d rows invalid (kinds 1 and 2: shifted storage forms only, bx = consumer "
                 "threads 0 (default), 32, 64 or 128 for FP32, 64, 128 or 256 for FP16 (kind 2: 0), rows 1..4096)",
                 kind, bx, rows);
  olbm::LaunchCfg k;
  k.kind = kind;
  k.bx = bx;
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
  if (ntiles) *ntiles = b->cfg.kind == 2 ? b->ntiles2 : b->ntiles;
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
    // One persistent cooperative launch for the n steps, captured with its barrier
    // reset into a CUDA graph once per (n, buffer parity) and replayed.
    const long long pkey[2] = {n, b->cur};
    if (!b->pgraph || !std::equal(pkey, pkey + 2, b->pgraph_key)) {
      if (b->pgraph) {
        cudaGraphExecDestroy(b->pgraph);
        b->pgraph = nullptr;
      }
      cudaGraph_t g = nullptr;
      e = cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal);
      if (e != cudaSuccess) return bcuda(b, e, "lbm_batch_step persistent capture");
      int parity_end = (b->cur + n) & 1;
      const cudaError_t le = b->cfg.kind == 2 && n >= 2
                                 ? launch_persistent_pairs(b, n, b->cur, b->capture, parity_end)
                                 : launch_persistent(b, n, b->cur, b->capture);
      b->pgraph_parity_end = parity_end;
      e = cudaStreamEndCapture(b->capture, &g);
      if (le != cudaSuccess || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return bcuda(b, le != cudaSuccess ? le : e, "lbm_batch_step persistent capture");
      }
      e = cudaGraphInstantiate(&b->pgraph, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) {
        b->pgraph = nullptr;
        return bcuda(b, e, "lbm_batch_step persistent graph instantiate");
      }
      std::copy(pkey, pkey + 2, b->pgraph_key);
    }
    e = cudaGraphLaunch(b->pgraph, b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "lbm_batch_step persistent launch");
    int timed_out = 0;
    e = cudaMemcpyAsync(&timed_out, &b->d_bar->err, sizeof(int), cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "lbm_batch_step persistent");
    b->cur = b->pgraph_parity_end;
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
    bool pending[lbm_batch::kParts] = {};
    int pb = 0, last = -1;
    // the next free partials buffer (after its previous final sum) for a diagnosed step
    auto take = [&](bool diag, int& q) {
      q = -1;
      if (!diag || le != cudaSuccess) return;
      q = pb;
      pb = (pb + 1) % lbm_batch::kParts;
      if (pending[q]) le = cudaStreamWaitEvent(b->capture, b->ev_fin[q], 0);
    };
    // the final sum of buffer q (tile ranges of the launch that wrote it) beside the next steps
    auto finish = [&](int q, const int2* ranges) {
      if (q < 0 || le != cudaSuccess) return;
      le = cudaEventRecord(b->ev_step[q], b->capture);
      if (le == cudaSuccess) le = cudaStreamWaitEvent(b->capture_side, b->ev_step[q], 0);
      if (le == cudaSuccess) le = launch_finalize(b, b->d_parts[q], b->d_diag, b->d_sticky, b->capture_side, ranges);
      if (le == cudaSuccess) le = cudaEventRecord(b->ev_fin[q], b->capture_side);
      pending[q] = true;
      last = q;
    };
    auto due = [&](long long tk) { return b->diag_every > 0 && (tk % b->diag_every) == 0; };
    int parity = b->cur;
    for (int k = 0; k < n && le == cudaSuccess;) {
      const long long tk = b->t + k;
      int q1 = -1, q2 = -1;
      if (b->cfg.kind == 2 && k + 1 < n) {  // two steps in one launch
        take(due(tk), q1);
        take(due(tk + 1), q2);
        if (le == cudaSuccess)
          le = launch_two_steps(b, q1 >= 0, q2 >= 0, parity, b->capture, b->d_parts[q1 < 0 ? 0 : q1],
                                b->d_parts[q2 < 0 ? 0 : q2]);
        finish(q1, b->d_ranges2);
        finish(q2, b->d_ranges2);
        k += 2;
      } else {
        take(due(tk), q1);
        if (le == cudaSuccess)
          le = launch_one_step(b, q1 >= 0, parity, b->capture, b->d_parts[q1 < 0 ? 0 : q1]);
        finish(q1, b->d_ranges);
        k += 1;
      }
      parity ^= 1;
    }
    b->graph_parity_end = parity;
    if (le == cudaSuccess && last >= 0) le = cudaStreamWaitEvent(b->capture, b->ev_fin[last], 0);  // join
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
  b->cur = b->graph_parity_end;
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
  cudaError_t e = launch_diag(b, b->stream);
  if (e == cudaSuccess) e = launch_finalize(b, b->d_parts[0], b->d_diag_now, nullptr, b->stream);
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

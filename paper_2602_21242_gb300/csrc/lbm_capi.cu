// lbm_capi.cu -- implementation of the C ABI declared in include/lbm.h.
//
// A lattice (lbm_ctx) owns two population buffers (ping-pong), the per-block
// diagnostics partials and a few device scalars. Each call validates its
// arguments on the host, enqueues kernels on the lattice's stream and returns a
// status; only the calls documented as synchronous wait for the device.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdint>
#include <cstring>
#include <algorithm>
#include <new>

#include "lbm.h"
#include "lbm_ctx.h"
#include "lbm_launch.h"
#include "lbm_halo.h"
#include "lbm_walls.h"

namespace {

thread_local char g_create_err[320] = "";

int fail(lbm_ctx* ctx, int status, const char* fmt, ...) {
  char* dst = ctx ? ctx->err : g_create_err;
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(dst, sizeof(g_create_err), fmt, ap);
  va_end(ap);
  return status;
}

int cuda_fail(lbm_ctx* ctx, cudaError_t e, const char* what) {
  return fail(ctx, LBM_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

long long elem_size(int prec) { return (prec == LBM_F64 || prec == LBM_F64_DF) ? 8 : (prec == LBM_F32_SHIFT ? 4 : 2); }

long long round_up(long long v, long long m) { return (v + m - 1) / m * m; }

bool layout_of(int nx, int ny, int prec, long long* pitch, long long* plane, long long* bytes) {
  if (nx < 1 || ny < 1 || prec < LBM_F64 || prec > LBM_F64_DF) return false;
  const long long es = elem_size(prec);
  const long long p = round_up(nx, 128 / es);         // 128-byte rows
  const long long pl = round_up(p * (long long)ny, 256 / es);  // 256-byte planes
  const long long b = 9 * pl * es;
  if (p > (1LL << 31) || b > (1LL << 40)) return false;
  if (pitch) *pitch = p;
  if (plane) *plane = pl;
  if (bytes) *bytes = b;
  return true;
}

long long nodes_of(const lbm_ctx* c) { return (long long)c->nx * c->ny; }

// Default launch of the step kernel per storage form, chosen by timing on GB300
// at the 4096^2 benchmark size: FP64 the column kernel with 64 x 2 threads and
// 32 rows per thread; the shifted forms the bulk-copy pipeline with one CTA per
// tile of 32 rows (refined per form below), except on lattices narrower than 32
// columns, where the column kernel with 128 x 4 threads and 16 rows wastes fewer
// threads. On smaller lattices the rows are halved until the grid has at least
// 4 CTAs per SM.
// lbm_set_launch[_ex] (and the autotuner built on it) overrides the choice.
olbm::LaunchCfg default_cfg(int prec, const olbm::Geometry& g, int sms) {
  olbm::LaunchCfg k;
  if (prec == LBM_F64 || prec == LBM_F64_DF) {
    k.bx = 64, k.by = 2, k.rows = 32;
  } else if (g.nx >= 32) {
    k.kind = 1, k.bx = 0, k.by = 1, k.rows = 32;
  } else {
    k.bx = 128, k.by = 4, k.rows = 16;
  }
  if (k.kind == 1 && prec == LBM_F16_SHIFT) {
    // One CTA per tile: the tile height whose last wave of CTAs is fullest,
    // preferring taller tiles unless a shorter one wastes 2 % less of a wave
    // (4096^2: 24 rows, 3.0 waves, +2-4 % over 32 rows; 8192^2: 48 rows).
    const long long strips = (g.nx + olbm::stream_tile_width(prec) - 1) / olbm::stream_tile_width(prec);
    const double resident = (double)olbm::stream_ctas_per_sm(prec) * sms;
    double best_waste = 2.0;
    for (int rows : {48, 40, 32, 24, 16}) {
      const double waves = (double)(strips * ((g.ny + rows - 1) / rows)) / resident;
      const double full = std::ceil(waves);
      const double waste = (full - waves) / full;
      if (waste < best_waste - 0.02) best_waste = waste, k.rows = rows;
    }
  }
  while (k.rows > 1 && olbm::step_blocks(g, k, prec) < 4LL * sms) k.rows /= 2;
  // FP32: two steps a launch (kind 2) on 24-row tiles, 48 from 8192^2 (diagnostics
  // every step: 143.6 GLUPS at 4096^2 against 92.6 for single steps, heights 16 to
  // 58 within 3 %; 161.6 at 8192^2 against 96.7); where it does not apply, the persistent pipeline over all
  // resident CTAs on 4-row tiles (measured 3-5 % above one CTA per tile at 4096^2
  // and 8192^2). FP16 is bound by its arithmetic, not by memory, and keeps single
  // steps on one CTA per tile (two steps: 136.7 against 152 GLUPS at 4096^2).
  if (k.kind == 1 && prec == LBM_F32_SHIFT) {
    olbm::LaunchCfg k2 = k;
    k2.kind = 2, k2.bx = 0, k2.rows = g.nx >= 8192 && g.ny >= 8192 ? 48 : 24;
    if (olbm::uses_step2(prec, g, k2)) {
      while (k2.rows > 1 && olbm::step2_blocks(g, k2, prec) < 4LL * sms) k2.rows /= 2;
      return k2;
    }
    k.bx = 64, k.rows = k.rows < 4 ? k.rows : 4;
  }
  return k;
}

cudaError_t launch_step(const olbm::StepArgs& a, int prec, cudaStream_t st) {
  switch (prec) {
    case LBM_F64: return olbm::launch_step_f64(a, st);
    case LBM_F32_SHIFT: return olbm::launch_step_f32(a, st);
    case LBM_F64_DF: return olbm::launch_step_f64df(a, st);
    default: return olbm::launch_step_f16(a, st);
  }
}

cudaError_t launch_step2(const olbm::StepArgs& a, int prec, cudaStream_t st) {
  switch (prec) {
    case LBM_F32_SHIFT: return olbm::launch_step2_f32(a, st);
    case LBM_F16_SHIFT: return olbm::launch_step2_f16(a, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_diag(const lbm_ctx* c, cudaStream_t st) {
  const void* src = c->buf[c->cur];
  switch (c->prec) {
    case LBM_F64:
    case LBM_F64_DF: return olbm::launch_diag_f64(src, c->g, c->rho_ref, c->d_parts[0], st);
    case LBM_F32_SHIFT: return olbm::launch_diag_f32(src, c->g, c->rho_ref, c->d_parts[0], st);
    default: return olbm::launch_diag_f16(src, c->g, c->rho_ref, c->d_parts[0], st);
  }
}

int check_ctx(lbm_ctx* ctx) {
  if (!ctx) return LBM_EINVAL;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != ctx->device)
    return fail(ctx, LBM_EINVAL, "the current CUDA device (%d) is not the lattice's device (%d)", dev, ctx->device);
  return LBM_OK;
}

void free_ctx(lbm_ctx* c) {
  if (!c) return;
  if (c->own_buffers) {
    cudaFree(c->buf[0]);
    cudaFree(c->buf[1]);
  }
  for (int b = 0; b < lbm_ctx::kParts; ++b) {
    cudaFree(c->d_parts[b]);
    if (c->ev_step[b]) cudaEventDestroy(c->ev_step[b]);
    if (c->ev_fin[b]) cudaEventDestroy(c->ev_fin[b]);
  }
  if (c->ev_io) cudaEventDestroy(c->ev_io);
  if (c->ev_rebind) cudaEventDestroy(c->ev_rebind);
  if (c->side) cudaStreamDestroy(c->side);
  cudaFree(c->d_diag);
  cudaFree(c->d_diag_now);
  cudaFree(c->d_sticky);
  cudaFree(c->d_err);
  cudaFree(c->d_sched);
  cudaFree(c->d_stage);
  cudaFree(c->d_vjp);
  cudaFree(c->d_walls);
  delete c;
}

}  // namespace

int olbm::set_thread_error(int status, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_create_err, sizeof(g_create_err), fmt, ap);
  va_end(ap);
  return status;
}

extern "C" {

int lbm_version(void) { return (1 << 16) | 1; }

int lbm_layout(int nx, int ny, int prec, long long* pitch, long long* plane, long long* state_bytes) {
  return layout_of(nx, ny, prec, pitch, plane, state_bytes) ? LBM_OK : LBM_EINVAL;
}

int lbm_create_ex(int nx, int ny, double theta, double tau, int model, int prec, void* stream,
                  void* d_pop_buffers, lbm_ctx** out) {
  if (!out) return fail(nullptr, LBM_EINVAL, "out is NULL");
  long long pitch, plane, bytes;
  if (!layout_of(nx, ny, prec, &pitch, &plane, &bytes))
    return fail(nullptr, LBM_EINVAL, "invalid size or precision (nx=%d ny=%d prec=%d)", nx, ny, prec);
  if (!(theta > 0.0 && theta < 1.0)) return fail(nullptr, LBM_EINVAL, "theta must lie in (0, 1), got %g", theta);
  if (!(tau > 0.5) || !std::isfinite(tau))
    return fail(nullptr, LBM_EINVAL, "tau must exceed 1/2 (positive viscosity), got %g", tau);
  if (model < LBM_LBGK || model > LBM_LBGK_POLY)
    return fail(nullptr, LBM_EINVAL, "unknown collision model %d", model);
  if (d_pop_buffers && (reinterpret_cast<uintptr_t>(d_pop_buffers) % 256) != 0)
    return fail(nullptr, LBM_EINVAL, "population buffers must be 256-byte aligned");

  lbm_ctx* c = new (std::nothrow) lbm_ctx();
  if (!c) return fail(nullptr, LBM_ENOMEM, "host allocation failed");
  cudaError_t e = cudaGetDevice(&c->device);
  if (e != cudaSuccess) {
    delete c;
    return fail(nullptr, LBM_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  }
  c->nx = nx;
  c->ny = ny;
  c->model = model;
  c->prec = prec;
  c->theta = theta;
  c->tau = tau;
  c->rho_ref = (prec == LBM_F64 || prec == LBM_F64_DF) ? 0.0 : 1.0;
  c->g = olbm::Geometry{nx, ny, pitch, plane};
  c->state_bytes = bytes;
  c->stream = static_cast<cudaStream_t>(stream);
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess || sms < 1) sms = 1;
  c->cfg = default_cfg(prec, c->g, sms);
  c->nparts = olbm::step_blocks(c->g, c->cfg, prec);
  c->parts_cap = std::max(c->nparts, olbm::node_blocks(c->g));

  if (d_pop_buffers) {
    c->own_buffers = false;
    c->buf[0] = d_pop_buffers;
    c->buf[1] = static_cast<char*>(d_pop_buffers) + bytes;
  } else {
    for (int k = 0; k < 2; ++k) {
      e = cudaMalloc(&c->buf[k], (size_t)bytes);
      if (e != cudaSuccess) {
        free_ctx(c);
        cudaGetLastError();
        return fail(nullptr, LBM_ENOMEM, "cudaMalloc of %lld bytes: %s", bytes, cudaGetErrorString(e));
      }
    }
  }
  for (int b = 0; b < lbm_ctx::kParts && e == cudaSuccess; ++b)
    e = cudaMalloc(&c->d_parts[b], sizeof(double) * 5 * (size_t)c->parts_cap);
  if (e != cudaSuccess ||
      (e = cudaMalloc(&c->d_diag, sizeof(double) * 6)) != cudaSuccess ||
      (e = cudaMalloc(&c->d_diag_now, sizeof(double) * 6)) != cudaSuccess ||
      (e = cudaMalloc(&c->d_sticky, sizeof(unsigned long long))) != cudaSuccess ||
      (e = cudaMalloc(&c->d_err, sizeof(int))) != cudaSuccess ||
      (e = cudaMalloc(&c->d_sched, 2 * sizeof(int))) != cudaSuccess) {
    free_ctx(c);
    cudaGetLastError();
    return fail(nullptr, LBM_ENOMEM, "cudaMalloc: %s", cudaGetErrorString(e));
  }
  e = cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking);
  for (int b = 0; b < lbm_ctx::kParts && e == cudaSuccess; ++b) {
    e = cudaEventCreateWithFlags(&c->ev_step[b], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_fin[b], cudaEventDisableTiming);
  }
  if (e != cudaSuccess || (e = cudaEventCreateWithFlags(&c->ev_io, cudaEventDisableTiming)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&c->ev_rebind, cudaEventDisableTiming)) != cudaSuccess) {
    free_ctx(c);
    cudaGetLastError();
    return fail(nullptr, LBM_ECUDA, "stream/event creation: %s", cudaGetErrorString(e));
  }
  // Defined contents everywhere, including row and plane padding.
  if ((e = cudaMemsetAsync(c->buf[0], 0, (size_t)bytes, c->stream)) != cudaSuccess ||
      (e = cudaMemsetAsync(c->buf[1], 0, (size_t)bytes, c->stream)) != cudaSuccess ||
      (e = cudaMemsetAsync(c->d_diag, 0, sizeof(double) * 6, c->stream)) != cudaSuccess ||
      (e = cudaMemsetAsync(c->d_sticky, 0, sizeof(unsigned long long), c->stream)) != cudaSuccess ||
      (e = cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream)) != cudaSuccess ||
      (e = cudaMemsetAsync(c->d_sched, 0, 2 * sizeof(int), c->stream)) != cudaSuccess) {
    free_ctx(c);
    return fail(nullptr, LBM_ECUDA, "cudaMemsetAsync: %s", cudaGetErrorString(e));
  }
  *out = c;
  return LBM_OK;
}

int lbm_create(int nx, int ny, double theta, double tau, int model, lbm_ctx** out) {
  return lbm_create_ex(nx, ny, theta, tau, model, LBM_F64, nullptr, nullptr, out);
}

int lbm_destroy(lbm_ctx* ctx) {
  if (!ctx) return LBM_OK;
  cudaStreamSynchronize(ctx->stream);
  if (ctx->side) cudaStreamSynchronize(ctx->side);
  free_ctx(ctx);
  return LBM_OK;
}

int lbm_set_stream(lbm_ctx* ctx, void* stream) {
  int s = check_ctx(ctx);
  if (s != LBM_OK) return s;
  cudaStream_t next = static_cast<cudaStream_t>(stream);
  if (next == ctx->stream) return LBM_OK;
  // Everything enqueued so far (lbm_step joins the side stream's final sums into
  // the old stream before it returns) precedes the next call's work.
  cudaError_t e = cudaEventRecord(ctx->ev_rebind, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(next, ctx->ev_rebind, 0);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "lbm_set_stream");
  ctx->stream = next;
  return LBM_OK;
}

int lbm_init(lbm_ctx* ctx, const double* d_rho, const double* d_ux, const double* d_uy) {
  int s = check_ctx(ctx);
  if (s != LBM_OK) return s;
  if (!d_rho || !d_ux || !d_uy) return fail(ctx, LBM_EINVAL, "lbm_init: NULL field pointer");
  cudaError_t e;
  void* dst = ctx->buf[ctx->cur];
  switch (ctx->prec) {
    case LBM_F64:
    case LBM_F64_DF: e = olbm::launch_init_f64(d_rho, d_ux, d_uy, ctx->g, ctx->theta, ctx->rho_ref, dst, ctx->stream); break;
    case LBM_F32_SHIFT: e = olbm::launch_init_f32(d_rho, d_ux, d_uy, ctx->g, ctx->theta, ctx->rho_ref, dst, ctx->stream); break;
    default: e = olbm::launch_init_f16(d_rho, d_ux, d_uy, ctx->g, ctx->theta, ctx->rho_ref, dst, ctx->stream); break;
  }
  if (e != cudaSuccess) return cuda_fail(ctx, e, "lbm_init launch");
  e = cudaMemsetAsync(ctx->d_sticky, 0, sizeof(unsigned long long), ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "lbm_init reset");
  ctx->initialised = true;
  ctx->t = 0;
  ctx->halo_t = 0;
  ctx->packed_t = -1;
  ctx->last_diag_t = -1;
  ++ctx->state_gen;
  return LBM_OK;
}

int lbm_set_walls(lbm_ctx* ctx, const unsigned char* h_mask, long long* h_count) {
  int s = check_ctx(ctx);
  if (s != LBM_OK) return s;
  ++ctx->state_gen;
  const long long nodes = nodes_of(ctx);
  long long n = 0;
  int2* list = nullptr;
  if (h_mask) {
    for (long long k = 0; k < nodes; ++k) n += h_mask[k] != 0;
    if (n > 0) {
      list = new (std::nothrow) int2[n];
      if (!list) return fail(ctx, LBM_ENOMEM, "lbm_set_walls: host list");
      long long j = 0;
      for (int y = 0; y < ctx->ny; ++y)
        for (int x = 0; x < ctx->nx; ++x)
          if (h_mask[(long long)y * ctx->nx + x]) list[j++] = make_int2(x, y);
    }
  }
  // the previous list may still be read by queued steps
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) {
    delete[] list;
    return cuda_fail(ctx, e, "lbm_set_walls sync");
  }
  cudaFree(ctx->d_walls);
  ctx->d_walls = nullptr;
  ctx->n_walls = 0;
  if (n > 0) {
    e = cudaMalloc(&ctx->d_walls, sizeof(int2) * (size_t)n);
    if (e == cudaSuccess)
      e = cudaMemcpy(ctx->d_walls, list, sizeof(int2) * (size_t)n, cudaMemcpyHostToDevice);
    delete[] list;
    if (e != cudaSuccess) {
      cudaGetLastError();
      cudaFree(ctx->d_walls);
      ctx->d_walls = nullptr;
      return fail(ctx, e == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA, "lbm_set_walls: %s",
                  cudaGetErrorString(e));
    }
    ctx->n_walls = n;
  }
  if (h_count) *h_count = n;
  return LBM_OK;
}

int lbm_halo_bytes(const lbm_ctx* ctx, long long* h_bytes) {
  if (!ctx || !h_bytes) return LBM_EINVAL;
  *h_bytes = 3LL * ctx->nx * elem_size(ctx->prec);
  return LBM_OK;
}

namespace {

int halo_check(lbm_ctx* ctx, const void* a, const void* b, const char* what) {
  int s = check_ctx(ctx);
  if (s != LBM_OK) return s;
  if (!a || !b) return fail(ctx, LBM_EINVAL, "%s: NULL pointer", what);
  const uintptr_t es = (uintptr_t)elem_size(ctx->prec);
  if ((uintptr_t)a % es || (uintptr_t)b % es)
    return fail(ctx, LBM_EINVAL, "%s: face buffers must be aligned to %d bytes", what, (int)es);
  if (!ctx->initialised) return fail(ctx, LBM_ESTATE, "%s before lbm_init / lbm_set_state", what);
  return LBM_OK;
}

}  // namespace

int lbm_halo_pack(lbm_ctx* ctx, void* d_up, void* d_down) {
  int s = halo_check(ctx, d_up, d_down, "lbm_halo_pack");
  if (s != LBM_OK) return s;
  if (ctx->t != ctx->halo_t + 1)
    return fail(ctx, LBM_ESTATE,
                "lbm_halo_pack: %lld step(s) since the last lbm_halo_unpack / lbm_init / lbm_set_state (needs 1)",
                ctx->t - ctx->halo_t);
  cudaError_t e = olbm::launch_halo_pack((int)elem_size(ctx->prec), ctx->buf[ctx->cur], ctx->g, d_up, d_down,
                                         ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "lbm_halo_pack launch");
  ctx->packed_t = ctx->t;
  return LBM_OK;
}

int lbm_halo_unpack(lbm_ctx* ctx, const void* d_from_below, const void* d_from_above) {
  int s = halo_check(ctx, d_from_below, d_from_above, "lbm_halo_unpack");
  if (s != LBM_OK) return s;
  if (ctx->packed_t != ctx->t)
    return fail(ctx, LBM_ESTATE, "lbm_halo_unpack: no lbm_halo_pack since the last step");
  cudaError_t e = olbm::launch_halo_unpack((int)elem_size(ctx->prec), ctx->buf[ctx->cur], ctx->g, d_from_below,
                                           d_from_above, ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "lbm_halo_unpack launch");
  ctx->halo_t = ctx->t;
  ctx->packed_t = -1;
  ++ctx->state_gen;
  return LBM_OK;
}

int lbm_set_diagnostics_interval(lbm_ctx* ctx, int every) {
  if (!ctx) return LBM_EINVAL;
  if (every < 0) return fail(ctx, LBM_EINVAL, "diagnostics interval must be >= 0");
  ctx->diag_every = every;
  return LBM_OK;
}

int lbm_step(lbm_ctx* ctx, int n) {
  int s = check_ctx(ctx);
  if (s != LBM_OK) return s;
  if (n < 0) return fail(ctx, LBM_EINVAL, "lbm_step: n must be >= 0");
  if (!ctx->initialised) return fail(ctx, LBM_ESTATE, "lbm_step before lbm_init / lbm_set_state");
  if (n > 0) ++ctx->state_gen;
  olbm::StepArgs a;
  a.model = ctx->model;
  a.g = ctx->g;
  a.theta = ctx->theta;
  a.tau = ctx->tau;
  a.rho_ref = ctx->rho_ref;
  a.partials = ctx->d_parts[0];
  a.cfg = ctx->cfg;
  a.err = ctx->d_err;
  a.sched = ctx->d_sched;
  long long used = ctx->nparts;
  a.parts_used = &used;
  int joined = -1;  // partials buffer whose final sum was launched last (-1: none in this call)
  // The next free partials buffer (waiting for its previous final sum), or null.
  auto take = [&](bool diag, int& b) -> cudaError_t {
    b = -1;
    if (!diag) return cudaSuccess;
    b = ctx->pbuf;
    ctx->pbuf = (ctx->pbuf + 1) % lbm_ctx::kParts;
    return ctx->fin_pending[b] ? cudaStreamWaitEvent(ctx->stream, ctx->ev_fin[b], 0) : cudaSuccess;
  };
  // The final sum of buffer b's partials (step time t) on the side stream, beside the next step.
  auto finish = [&](int b, long long t) -> cudaError_t {
    cudaError_t e;
    if ((e = cudaEventRecord(ctx->ev_step[b], ctx->stream)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(ctx->side, ctx->ev_step[b], 0)) != cudaSuccess ||
        (e = olbm::launch_finalize(ctx->d_parts[b], (int)used, ctx->rho_ref, nodes_of(ctx), t, ctx->d_diag,
                                   ctx->d_sticky, ctx->side)) != cudaSuccess ||
        (e = cudaEventRecord(ctx->ev_fin[b], ctx->side)) != cudaSuccess)
      return e;
    ctx->fin_pending[b] = true;
    joined = b;
    ctx->last_diag_t = t;
    return cudaSuccess;
  };
  auto due = [&](long long t) { return ctx->diag_every > 0 && (t % ctx->diag_every) == 0; };
  for (int k = 0; k < n;) {
    // launch kind 2: two steps in one launch where two remain (no walls: they act after every step)
    const bool two = k + 1 < n && ctx->n_walls == 0 && olbm::uses_step2(ctx->prec, ctx->g, ctx->cfg);
    a.diag = due(ctx->t);
    a.diag2 = two && due(ctx->t + 1);
    a.src = ctx->buf[ctx->cur];
    a.dst = ctx->buf[ctx->cur ^ 1];
    used = ctx->nparts;
    int b1 = -1, b2 = -1;
    cudaError_t e = take(a.diag, b1);
    if (e == cudaSuccess) e = take(a.diag2, b2);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "lbm_step event wait");
    a.partials = ctx->d_parts[b1 < 0 ? 0 : b1];
    a.partials2 = ctx->d_parts[b2 < 0 ? 0 : b2];
    e = two ? launch_step2(a, ctx->prec, ctx->stream) : launch_step(a, ctx->prec, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "lbm_step launch");
    if (ctx->n_walls > 0) {
      e = olbm::launch_walls((int)elem_size(ctx->prec), a.src, a.dst, ctx->g, ctx->d_walls, ctx->n_walls,
                             ctx->stream);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "lbm_step walls launch");
    }
    if (b1 >= 0 && (e = finish(b1, ctx->t)) != cudaSuccess) return cuda_fail(ctx, e, "lbm_step diagnostics launch");
    if (b2 >= 0 && (e = finish(b2, ctx->t + 1)) != cudaSuccess)
      return cuda_fail(ctx, e, "lbm_step diagnostics launch");
    ctx->cur ^= 1;
    const int done = two ? 2 : 1;
    ctx->t += done;
    k += done;
  }
  if (joined >= 0) {  // everything queued on `stream` after this call follows the final sums
    cudaError_t e = cudaStreamWaitEvent(ctx->stream, ctx->ev_fin[joined], 0);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "lbm_step join");
  }
  return LBM_OK;
}

int lbm_step_diagnostics(lbm_ctx* ctx, double* h_out5, long long* h_time) {
  int s = check_ctx(ctx);
  if (s != LBM_OK) return s;
  if (!h_out5) return fail(ctx, LBM_EINVAL, "lbm_step_diagnostics: NULL output");
  double d[6];
  unsigned long long bad = 0;
  int timed_out = 0;
  cudaError_t e = cudaMemcpyAsync(d, ctx->d_diag, sizeof(d), cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, ctx->d_sticky, sizeof(bad), cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&timed_out, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "lbm_step_diagnostics");
  if (timed_out) return fail(ctx, LBM_ETIMEOUT, "a bounded device-side wait of the step kernel gave up");
  for (int k = 0; k < 5; ++k) h_out5[k] = ctx->last_diag_t >= 0 ? d[k] : 0.0;
  if (h_time) *h_time = ctx->last_diag_t;
  if (bad > 0) return fail(ctx, LBM_ENONFINITE, "%llu non-finite node(s) met by fused diagnostics", bad);
  return LBM_OK;
}

int lbm_moments(lbm_ctx* ctx, double* d_rho, double* d_ux, double* d_uy) {
  int s = check_ctx(ctx);
  if (s != LBM_OK) return s;
  if (!d_rho || !d_ux || !d_uy) return fail(ctx, LBM_EINVAL, "lbm_moments: NULL field pointer");
  if (!ctx->initialised) return fail(ctx, LBM_ESTATE, "lbm_moments before lbm_init / lbm_set_state");
  const void* src = ctx->buf[ctx->cur];
  cudaError_t e;
  switch (ctx->prec) {
    case LBM_F64:
    case LBM_F64_DF: e = olbm::launch_moments_f64(src, ctx->g, ctx->rho_ref, d_rho, d_ux, d_uy, ctx->stream); break;
    case LBM_F32_SHIFT: e = olbm::launch_moments_f32(src, ctx->g, ctx->rho_ref, d_rho, d_ux, d_uy, ctx->stream); break;
    default: e = olbm::launch_moments_f16(src, ctx->g, ctx->rho_ref, d_rho, d_ux, d_uy, ctx->stream); break;
  }
  return e == cudaSuccess ? LBM_OK : cuda_fail(ctx, e, "lbm_moments launch");
}

int lbm_diagnostics(lbm_ctx* ctx, double* h_out5) {
  int s = check_ctx(ctx);
  if (s != LBM_OK) return s;
  if (!h_out5) return fail(ctx, LBM_EINVAL, "lbm_diagnostics: NULL output");
  if (!ctx->initialised) return fail(ctx, LBM_ESTATE, "lbm_diagnostics before lbm_init / lbm_set_state");
  cudaError_t e = launch_diag(ctx, ctx->stream);
  if (e == cudaSuccess)
    e = olbm::launch_finalize(ctx->d_parts[0], (int)olbm::diag_blocks(ctx->g), ctx->rho_ref, nodes_of(ctx), ctx->t,
                              ctx->d_diag_now, nullptr, ctx->stream);
  double d[6];
  if (e == cudaSuccess) e = cudaMemcpyAsync(d, ctx->d_diag_now, sizeof(d), cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "lbm_diagnostics");
  for (int k = 0; k < 5; ++k) h_out5[k] = d[k];
  if (d[4] > 0) return fail(ctx, LBM_ENONFINITE, "%.0f node(s) hold non-finite populations", d[4]);
  return LBM_OK;
}

int lbm_get_state(lbm_ctx* ctx, double* d_f) {
  int s = check_ctx(ctx);
  if (s != LBM_OK) return s;
  if (!d_f) return fail(ctx, LBM_EINVAL, "lbm_get_state: NULL pointer");
  if (!ctx->initialised) return fail(ctx, LBM_ESTATE, "lbm_get_state before lbm_init / lbm_set_state");
  const void* src = ctx->buf[ctx->cur];
  cudaError_t e;
  switch (ctx->prec) {
    case LBM_F64:
    case LBM_F64_DF: e = olbm::launch_get_state_f64(src, ctx->g, ctx->theta, ctx->rho_ref, d_f, ctx->stream); break;
    case LBM_F32_SHIFT: e = olbm::launch_get_state_f32(src, ctx->g, ctx->theta, ctx->rho_ref, d_f, ctx->stream); break;
    default: e = olbm::launch_get_state_f16(src, ctx->g, ctx->theta, ctx->rho_ref, d_f, ctx->stream); break;
  }
  return e == cudaSuccess ? LBM_OK : cuda_fail(ctx, e, "lbm_get_state launch");
}

int lbm_set_state(lbm_ctx* ctx, const double* d_f) {
  int s = check_ctx(ctx);
  if (s != LBM_OK) return s;
  if (!d_f) return fail(ctx, LBM_EINVAL, "lbm_set_state: NULL pointer");
  void* dst = ctx->buf[ctx->cur];
  cudaError_t e;
  switch (ctx->prec) {
    case LBM_F64:
    case LBM_F64_DF: e = olbm::launch_set_state_f64(d_f, ctx->g, ctx->theta, ctx->rho_ref, dst, ctx->stream); break;
    case LBM_F32_SHIFT: e = olbm::launch_set_state_f32(d_f, ctx->g, ctx->theta, ctx->rho_ref, dst, ctx->stream); break;
    default: e = olbm::launch_set_state_f16(d_f, ctx->g, ctx->theta, ctx->rho_ref, dst, ctx->stream); break;
  }
  if (e != cudaSuccess) return cuda_fail(ctx, e, "lbm_set_state launch");
  e = cudaMemsetAsync(ctx->d_sticky, 0, sizeof(unsigned long long), ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "lbm_set_state reset");
  ctx->initialised = true;
  ctx->t = 0;
  ctx->halo_t = 0;
  ctx->packed_t = -1;
  ctx->last_diag_t = -1;
  ++ctx->state_gen;
  return LBM_OK;
}

int lbm_time(const lbm_ctx* ctx, long long* h_t) {
  if (!ctx || !h_t) return LBM_EINVAL;
  *h_t = ctx->t;
  return LBM_OK;
}

int lbm_run_host(lbm_ctx* ctx, const double* h_rho0, const double* h_ux0, const double* h_uy0, int n, double* h_rho,
                 double* h_ux, double* h_uy, double* h_diag5) {
  int s = check_ctx(ctx);
  if (s != LBM_OK) return s;
  if (!h_rho0 || !h_ux0 || !h_uy0) return fail(ctx, LBM_EINVAL, "lbm_run_host: NULL input");
  if (n < 0) return fail(ctx, LBM_EINVAL, "lbm_run_host: n must be >= 0");
  const size_t N = (size_t)nodes_of(ctx);
  cudaError_t e;
  if (!ctx->d_stage) {
    e = cudaMalloc(&ctx->d_stage, sizeof(double) * 6 * N);
    if (e != cudaSuccess) {
      ctx->d_stage = nullptr;
      cudaGetLastError();
      return fail(ctx, LBM_ENOMEM, "lbm_run_host staging: %s", cudaGetErrorString(e));
    }
  }
  double* in = ctx->d_stage;
  double* outp = ctx->d_stage + 3 * N;
  const size_t fb = sizeof(double) * N;
  if ((e = cudaMemcpyAsync(in, h_rho0, fb, cudaMemcpyHostToDevice, ctx->stream)) != cudaSuccess ||
      (e = cudaMemcpyAsync(in + N, h_ux0, fb, cudaMemcpyHostToDevice, ctx->stream)) != cudaSuccess ||
      (e = cudaMemcpyAsync(in + 2 * N, h_uy0, fb, cudaMemcpyHostToDevice, ctx->stream)) != cudaSuccess)
    return cuda_fail(ctx, e, "lbm_run_host upload");
  if ((s = lbm_init(ctx, in, in + N, in + 2 * N)) != LBM_OK) return s;
  if ((s = lbm_step(ctx, n)) != LBM_OK) return s;
  if (h_rho || h_ux || h_uy) {
    // The downloads run on the side stream, beside the diagnostics pass on the main one.
    if ((s = lbm_moments(ctx, outp, outp + N, outp + 2 * N)) != LBM_OK) return s;
    if ((e = cudaEventRecord(ctx->ev_io, ctx->stream)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(ctx->side, ctx->ev_io, 0)) != cudaSuccess)
      return cuda_fail(ctx, e, "lbm_run_host download");
    if (h_rho && (e = cudaMemcpyAsync(h_rho, outp, fb, cudaMemcpyDeviceToHost, ctx->side)) != cudaSuccess)
      return cuda_fail(ctx, e, "lbm_run_host download");
    if (h_ux && (e = cudaMemcpyAsync(h_ux, outp + N, fb, cudaMemcpyDeviceToHost, ctx->side)) != cudaSuccess)
      return cuda_fail(ctx, e, "lbm_run_host download");
    if (h_uy && (e = cudaMemcpyAsync(h_uy, outp + 2 * N, fb, cudaMemcpyDeviceToHost, ctx->side)) != cudaSuccess)
      return cuda_fail(ctx, e, "lbm_run_host download");
  }
  s = h_diag5 ? lbm_diagnostics(ctx, h_diag5) : LBM_OK;  // synchronises the main stream
  if ((e = cudaStreamSynchronize(ctx->side)) != cudaSuccess) return cuda_fail(ctx, e, "lbm_run_host download");
  if (s != LBM_OK) return s;
  e = cudaStreamSynchronize(ctx->stream);
  return e == cudaSuccess ? LBM_OK : cuda_fail(ctx, e, "lbm_run_host sync");
}

int lbm_set_launch(lbm_ctx* ctx, int bx, int by, int rows) { return lbm_set_launch_ex(ctx, 0, bx, by, rows); }

int lbm_set_launch_ex(lbm_ctx* ctx, int kind, int bx, int by, int rows) {
  int s = check_ctx(ctx);
  if (s != LBM_OK) return s;
  olbm::LaunchCfg k;
  k.kind = kind;
  k.bx = bx;
  k.by = by;
  k.rows = rows;
  if (!olbm::valid_cfg(k))
    return fail(ctx, LBM_EINVAL,
                "launch kind %d shape %dx%d x %d rows invalid (kind 0: bx a multiple of 32, bx*by <= 512, rows 1..64; "
                "kind 1: rows 1..4096; kind 2: rows 1..4096, bx = 0)",
                kind, bx, by, rows);
  if (ctx->prec == LBM_F64_DF && (k.kind != 0 || bx * by > 256))
    return fail(ctx, LBM_EINVAL, "storage form LBM_F64_DF takes launch kind 0 with at most 256 threads a block");
  if (k.kind == 2 && ctx->prec != LBM_F32_SHIFT && ctx->prec != LBM_F16_SHIFT)
    return fail(ctx, LBM_EINVAL, "launch kind 2 (two steps a launch) applies to the shifted storage forms");
  if (ctx->prec == LBM_F64 && k.kind == 1 && bx != 0)
    return fail(ctx, LBM_EINVAL, "storage form LBM_F64 takes launch kind 1 with one CTA per tile (bx = 0)");
  const long long need = olbm::step_blocks(ctx->g, k, ctx->prec);
  if (need > ctx->parts_cap) {
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->side);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "lbm_set_launch sync");
    double* p[lbm_ctx::kParts] = {};
    for (int b = 0; b < lbm_ctx::kParts && e == cudaSuccess; ++b)
      e = cudaMalloc(&p[b], sizeof(double) * 5 * (size_t)need);
    if (e != cudaSuccess) {
      for (int b = 0; b < lbm_ctx::kParts; ++b) cudaFree(p[b]);
      cudaGetLastError();
      return fail(ctx, LBM_ENOMEM, "lbm_set_launch: %s", cudaGetErrorString(e));
    }
    for (int b = 0; b < lbm_ctx::kParts; ++b) {
      cudaFree(ctx->d_parts[b]);
      ctx->d_parts[b] = p[b];
    }
    ctx->parts_cap = need;
  }
  ctx->cfg = k;
  ctx->nparts = need;
  return LBM_OK;
}

int lbm_get_launch_ex(const lbm_ctx* ctx, int* kind, int* bx, int* by, int* rows) {
  if (!ctx || !kind) return LBM_EINVAL;
  *kind = ctx->cfg.kind;
  return lbm_get_launch(ctx, bx, by, rows);
}

int lbm_get_launch(const lbm_ctx* ctx, int* bx, int* by, int* rows) {
  if (!ctx || !bx || !by || !rows) return LBM_EINVAL;
  *bx = ctx->cfg.bx;
  *by = ctx->cfg.by;
  *rows = ctx->cfg.rows;
  return LBM_OK;
}

int lbm_sync(lbm_ctx* ctx) {
  int s = check_ctx(ctx);
  if (s != LBM_OK) return s;
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(ctx, e, "lbm_sync");
  unsigned long long bad = 0;
  int timed_out = 0;
  e = cudaMemcpyAsync(&bad, ctx->d_sticky, sizeof(bad), cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&timed_out, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "lbm_sync flag read");
  if (timed_out) return fail(ctx, LBM_ETIMEOUT, "a bounded device-side wait of the step kernel gave up");
  if (bad > 0) return fail(ctx, LBM_ENONFINITE, "%llu non-finite node(s) met by fused diagnostics", bad);
  return LBM_OK;
}

const char* lbm_last_error(const lbm_ctx* ctx) { return ctx ? ctx->err : g_create_err; }

}  // extern "C"

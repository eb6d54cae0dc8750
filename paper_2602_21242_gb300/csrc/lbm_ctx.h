// lbm_ctx.h -- the lattice object behind the opaque lbm_ctx handle of the C
// ABI (internal to liblbm.so).
#pragma once

#include <cuda_runtime.h>

#include "lbm_launch.h"

struct lbm_ctx {
  int device = 0;
  int nx = 0, ny = 0, model = 0, prec = 0;
  double theta = 0, tau = 0, rho_ref = 0;
  olbm::Geometry g{};
  long long state_bytes = 0;
  void* buf[2] = {nullptr, nullptr};
  int cur = 0;  // buffer holding the current state
  bool own_buffers = true;
  bool initialised = false;
  cudaStream_t stream = nullptr;
  olbm::LaunchCfg cfg{};
  // Per-block diagnostics partials, kParts buffers of parts_cap blocks each (d_parts[0]
  // also serves lbm_diagnostics). Consecutive diagnosed steps take the buffers in turn,
  // and the final sum of step t runs on a second stream while later steps run; lbm_step
  // joins that stream back into `stream` before it returns. A two-step launch takes two
  // buffers at once, so the next launch's buffers are never the ones still being summed.
  static constexpr int kParts = 4;
  double* d_parts[kParts] = {nullptr, nullptr, nullptr, nullptr};
  long long nparts = 0;      // partials the step kernel writes under cfg
  long long parts_cap = 0;   // partials allocated (each buffer)
  cudaStream_t side = nullptr;
  cudaEvent_t ev_step[kParts] = {};  // partials of buffer b written (on `stream`)
  cudaEvent_t ev_fin[kParts] = {};   // partials of buffer b summed (on `side`)
  cudaEvent_t ev_io = nullptr;                  // lbm_run_host: moments written (on `stream`)
  cudaEvent_t ev_rebind = nullptr;              // lbm_set_stream: end of the old stream's work
  bool fin_pending[kParts] = {};
  int pbuf = 0;  // partials buffer of the next diagnosed step (0 .. kParts - 1)
  double* d_diag = nullptr;      // [6] latest fused diagnostics (out5 + time)
  double* d_diag_now = nullptr;  // [6] scratch of lbm_diagnostics
  unsigned long long* d_sticky = nullptr;
  int* d_err = nullptr;  // set by a bounded device-side wait that gave up
  int* d_sched = nullptr;  // [next tile, CTAs done] of the persistent pipeline kernel; zero between launches
  int diag_every = 0;
  long long t = 0;
  long long last_diag_t = -1;
  double* d_stage = nullptr;  // lbm_run_host staging, 6 * nodes doubles
  // lbm_vjp work memory: checkpoints, recompute ring, adjoint fields (grown on demand)
  void* d_vjp = nullptr;
  size_t vjp_bytes = 0;
  // Count of calls that changed the state or the dynamics (init, set_state, step,
  // walls); the forward pass of lbm_vjp_forward records it with its (n, ckpt_every)
  // so that lbm_vjp_ex can tell whether its checkpoints still describe the lattice.
  long long state_gen = 0;
  long long vjp_gen = -1;
  int vjp_n = -1, vjp_k = -1;
  // fullway bounce-back wall nodes (x, y), applied after every step (lbm_set_walls)
  int2* d_walls = nullptr;
  long long n_walls = 0;
  // Slab halo trade (lbm_halo_pack / lbm_halo_unpack): the time of the last
  // unpack, or of lbm_init / lbm_set_state (a pack needs exactly one step
  // since), and the time of the last pack (an unpack needs one at this time).
  long long halo_t = 0;
  long long packed_t = -1;
  char err[320] = {0};
};


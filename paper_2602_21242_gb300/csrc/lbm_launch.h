// lbm_launch.h -- host-side entry points into the kernels of one storage form
// (internal to liblbm.so; the public ABI is include/lbm.h).
#pragma once

#include <cuda_runtime.h>

#include "lbm_device.cuh"

namespace olbm {

// Launch shape of the step kernel. kind 0: bx x by threads (bx a multiple of
// 32, bx * by <= 512), each thread updating `rows` nodes of one column.
// kind 1 (shifted forms and FP64, any nx): the bulk-copy pipeline over
// tiles of stream_width(prec) columns by `rows` rows; bx = 0 launches one CTA
// per tile, bx > 0 (shifted forms) a persistent grid of bx CTAs per SM (at
// most the resident count) looping over the tiles; by unused. kind 2 (shifted
// forms): two steps per launch (step2_stream_kernel, one CTA per tile of
// 2 NC - 2 columns by `rows` rows) wherever two steps follow each other and no
// walls are set (any nx); a single step (the last of an odd count) takes the
// kind 1 pipeline with the same rows; bx = 0.
struct LaunchCfg {
  int bx = 32, by = 8, rows = 1, kind = 0;
  int cap = 0;  // kind 1: most CTAs launched (a multiple of the SM count); 0 = one CTA per tile
};

inline bool valid_cfg(const LaunchCfg& k) {
  if (k.kind == 1) return k.rows >= 1 && k.rows <= 4096 && k.bx >= 0 && k.bx <= 64;
  if (k.kind == 2) return k.rows >= 1 && k.rows <= 4096 && k.bx == 0;
  return k.kind == 0 && k.bx >= 32 && k.bx % 32 == 0 && k.by >= 1 && k.bx * k.by <= 512 && k.rows >= 1 &&
         k.rows <= 64;
}

struct StepArgs {
  int model;         // 0..3, enum lbm_model
  bool diag;         // fuse the diagnostics reduction into this step
  const void* src;   // buffer holding f*(t - 1) at source nodes
  void* dst;         // buffer receiving f*(t)
  Geometry g;
  double theta, tau;
  double rho_ref;    // 0 for absolute storage, 1 for the shifted forms
  double* partials;  // grid blocks * 5 doubles when diag
  LaunchCfg cfg;
  int* err = nullptr;  // device flag set by a bounded wait that gave up (pipeline kernel)
  int* sched = nullptr;  // two ints, zero between launches: tile counter of the persistent pipeline kernel
  long long* parts_used = nullptr;  // out: diagnostics partials the launch wrote (its grid size)
  // two-step launches (kind 2): diagnostics of the second step into partials2
  bool diag2 = false;
  double* partials2 = nullptr;
};

// Number of thread blocks of the auxiliary node-parallel kernels and of the
// step kernel under a launch shape (= diagnostics partials they write).
long long node_blocks(const Geometry& g);
// Blocks (= diagnostics partials) of the diagnostics kernel, at most node_blocks.
long long diag_blocks(const Geometry& g);
long long step_blocks(const Geometry& g, const LaunchCfg& k, int prec);
// Columns of one bulk-copy pipeline tile and the CTAs of that kernel resident
// on one SM (launch kind 1) for a shifted storage form.
int stream_tile_width(int prec);
int stream_ctas_per_sm(int prec);
// Whether a launch of kind 2 runs two steps (the shifted forms), and
// the blocks (= diagnostics partials) of that two-step launch.
bool uses_step2(int prec, const Geometry& g, const LaunchCfg& k);
long long step2_blocks(const Geometry& g, const LaunchCfg& k, int prec);

#define OLBM_DECLARE_LAUNCHERS(SUFFIX)                                                                        \
  cudaError_t launch_step_##SUFFIX(const StepArgs& a, cudaStream_t st);                                       \
  cudaError_t launch_diag_##SUFFIX(const void* src, const Geometry& g, double rho_ref, double* partials,      \
                                   cudaStream_t st);                                                          \
  cudaError_t launch_init_##SUFFIX(const double* rho, const double* ux, const double* uy, const Geometry& g,  \
                                   double theta, double rho_ref, void* dst, cudaStream_t st);                 \
  cudaError_t launch_moments_##SUFFIX(const void* src, const Geometry& g, double rho_ref, double* rho,        \
                                      double* ux, double* uy, cudaStream_t st);                               \
  cudaError_t launch_get_state_##SUFFIX(const void* src, const Geometry& g, double theta, double rho_ref,     \
                                        double* out, cudaStream_t st);                                        \
  cudaError_t launch_set_state_##SUFFIX(const double* in, const Geometry& g, double theta, double rho_ref,    \
                                        void* dst, cudaStream_t st);

OLBM_DECLARE_LAUNCHERS(f64)
OLBM_DECLARE_LAUNCHERS(f32)
OLBM_DECLARE_LAUNCHERS(f16)
// storage form 3 (FP64 storage, double-float arithmetic): its own step kernel; the
// other kernels are the FP64 form's (same storage)
cudaError_t launch_step_f64df(const StepArgs& a, cudaStream_t st);
// two steps per launch (kind 2) for the shifted forms
cudaError_t launch_step2_f32(const StepArgs& a, cudaStream_t st);
cudaError_t launch_step2_f16(const StepArgs& a, cudaStream_t st);

// Record a message for lbm_last_error(NULL) on this thread; returns status.
int set_thread_error(int status, const char* fmt, ...);

cudaError_t launch_finalize(const double* partials, int nparts, double rho_ref, long long nodes, long long t,
                            double* out, unsigned long long* sticky, cudaStream_t st);

}  // namespace olbm

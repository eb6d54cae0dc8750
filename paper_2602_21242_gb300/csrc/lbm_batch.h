// lbm_batch.h -- batched domains (internal to liblbm.so; the public entry
// points are the lbm_batch_* calls of include/lbm.h): the per-domain
// descriptor, the launch view the host side hands to the per-storage-form
// kernel translation units, and their entry points.
#pragma once

#include <cuda_runtime.h>

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

__host__ __device__ inline Coef<f32x2> broadcast(const Coef<float>& a) { return coef_cast<f32x2>(a); }

// Consumer threads of a pipelined batch tile (launch kind 1): bx, or the
// single-lattice default when bx = 0. Tiles are 2 NC columns wide.
inline int batch_stream_nc(int prec, int bx) { return bx != 0 ? bx : (prec == 1 ? kStreamNC32 : kStreamNC16); }
inline bool batch_stream_nc_valid(int prec, int bx) {
  const int nc = batch_stream_nc(prec, bx);
  if (prec == 1) return nc == 32 || nc == 64 || nc == 128;
  if (prec == 2) return nc == 64 || nc == 128 || nc == 256;
  return false;
}

// What a kernel launch needs to know of a batch.
struct BatchLaunch {
  int model = 0;
  LaunchCfg cfg{};           // kind 0: bx x by threads, rows; kind 1: bx = NC selector, rows = tile rows
                             // (a batch of kind 2 hands its single steps to kind 1 with bx = 0)
  const void* desc = nullptr;  // Desc<double> (FP64) or Desc<float> (shifted forms), one per domain
  const int4* tiles = nullptr;  // (domain, x0, y0, 0)
  int ntiles = 0;
  double* partials = nullptr;  // 5 doubles per tile
  int* perr = nullptr;         // bounded-wait flag of the pipelined tile kernel
  GridBarrier* bar = nullptr;  // persistent mode
  int* ctr = nullptr;          // persistent pipelined mode: two tile counters
  int sms = 1;
  // two steps a launch (kind 2): tiles of 2 NC - 2 columns and the second step's partials
  const int4* tiles2 = nullptr;
  int ntiles2 = 0;
  double* partials2 = nullptr;
  // persistent launches: reset only the barrier's count and generation, keeping an
  // error flag that an earlier launch of the same call set
  bool keep_err = false;
};

#define OLBM_DECLARE_BATCH(SUFFIX)                                                                          \
  cudaError_t batch_prepare_##SUFFIX(const BatchLaunch& b);                                                 \
  cudaError_t batch_step_##SUFFIX(const BatchLaunch& b, bool diag, int parity, cudaStream_t st);           \
  cudaError_t batch_persistent_##SUFFIX(const BatchLaunch& b, int n, int parity0, cudaStream_t st);        \
  cudaError_t batch_diag_##SUFFIX(const BatchLaunch& b, int parity, double rho_ref, cudaStream_t st);

OLBM_DECLARE_BATCH(f64)
OLBM_DECLARE_BATCH(f32)
OLBM_DECLARE_BATCH(f16)

// Two steps a launch (kind 2, shifted forms): the tiles2 list, step t's diagnostics
// into partials (diag1), step t + 1's into partials2 (diag2).
cudaError_t batch_prepare2_f32(const BatchLaunch& b);
cudaError_t batch_prepare2_f16(const BatchLaunch& b);
cudaError_t batch_step2_f32(const BatchLaunch& b, bool diag1, bool diag2, int parity, cudaStream_t st);
cudaError_t batch_step2_f16(const BatchLaunch& b, bool diag1, bool diag2, int parity, cudaStream_t st);
// npairs two-step pairs of every domain in one cooperative launch (persistent mode, kind 2)
cudaError_t batch_persistent2_f32(const BatchLaunch& b, int npairs, int parity0, cudaStream_t st);
cudaError_t batch_persistent2_f16(const BatchLaunch& b, int npairs, int parity0, cudaStream_t st);

}  // namespace olbm

// lbm_reduce.cu -- final, fixed-order reduction of the per-block diagnostics
// partials written by the step and diagnostics kernels, and the shared grid
// shape of the node-parallel kernels.
#include "lbm_kernels.cuh"

namespace olbm {

long long node_blocks(const Geometry& g) {
  const dim3 gr = grid_of(g);
  return (long long)gr.x * gr.y;
}

long long diag_blocks(const Geometry& g) {
  const dim3 gr = diag_grid(g);
  return (long long)gr.x * gr.y;
}

long long step_blocks(const Geometry& g, const LaunchCfg& k, int prec) {
  const dim3 gr = step_grid(g, k, prec);
  const long long one = (long long)gr.x * gr.y;
  if (!step2_applies(prec, g, k)) return one;
  const dim3 g2 = step2_grid(g, k, prec);
  return std::max(one, (long long)g2.x * g2.y);  // kind 2 also launches single steps
}

int stream_tile_width(int prec) { return stream_width(prec); }

bool uses_step2(int prec, const Geometry& g, const LaunchCfg& k) { return step2_applies(prec, g, k); }

long long step2_blocks(const Geometry& g, const LaunchCfg& k, int prec) {
  const dim3 gr = step2_grid(g, k, prec);
  return (long long)gr.x * gr.y;
}

// The ring fits three times in an SM's shared memory for both shifted forms;
// FP16 is compiled for three CTAs (registers), FP32 (160 threads) fits them.
#ifndef OLBM_STREAM_CTAS
#define OLBM_STREAM_CTAS 3
#endif
int stream_ctas_per_sm(int) { return OLBM_STREAM_CTAS; }

// Fixed-order final sum of the block partials: out[0..4] as in lbm_diagnostics
// (mass gets rho_ref for every finite node), out[5] = t; non-finite nodes are
// added to *sticky.
constexpr int kFinalThreads = 256;
__global__ void __launch_bounds__(kFinalThreads) finalize_kernel(const double* __restrict__ partials, int nparts,
                                                                 double rho_ref, long long nodes, long long t,
                                                                 double* __restrict__ out,
                                                                 unsigned long long* __restrict__ sticky) {
  double v[kNDiag] = {0.0, 0.0, 0.0, 0.0, 0.0};
  for (int j = threadIdx.x; j < nparts; j += kFinalThreads)
#pragma unroll
    for (int k = 0; k < kNDiag; ++k) v[k] += partials[(long long)j * kNDiag + k];
  double tot[kNDiag];
  block_sum<kNDiag, kFinalThreads>(v, tot);
  if (threadIdx.x == 0) {
    const double bad = tot[4];
    out[0] = tot[0] + rho_ref * (double)(nodes - (long long)bad);
    out[1] = tot[1];
    out[2] = tot[2];
    out[3] = tot[3];
    out[4] = bad;
    out[5] = (double)t;
    if (bad > 0.0 && sticky != nullptr) *sticky += (unsigned long long)bad;
  }
}

cudaError_t launch_finalize(const double* partials, int nparts, double rho_ref, long long nodes, long long t,
                            double* out, unsigned long long* sticky, cudaStream_t st) {
  finalize_kernel<<<1, kFinalThreads, 0, st>>>(partials, nparts, rho_ref, nodes, t, out, sticky);
  return cudaGetLastError();
}

}  // namespace olbm

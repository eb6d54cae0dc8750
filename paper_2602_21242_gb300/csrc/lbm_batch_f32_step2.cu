// lbm_batch_f32_step2.cu -- two-step batch kernels (launch kind 2) for storage
// form 1 (FP32 deviations; see lbm_batch_stream2.cuh).
#include <atomic>

#include "lbm_batch_stream2.cuh"

namespace olbm {
cudaError_t batch_prepare2_f32(const BatchLaunch& b) { return BatchOps2<1>::prepare(b); }
cudaError_t batch_step2_f32(const BatchLaunch& b, bool diag1, bool diag2, int parity, cudaStream_t st) {
  return BatchOps2<1>::step(b, diag1, diag2, parity, st);
}
cudaError_t batch_persistent2_f32(const BatchLaunch& b, int npairs, int parity0, cudaStream_t st) {
  return BatchOps2<1>::persistent(b, npairs, parity0, st);
}
}  // namespace olbm

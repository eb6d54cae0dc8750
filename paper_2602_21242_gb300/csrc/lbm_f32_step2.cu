// lbm_f32_step2.cu -- instantiation of the two-step kernels (launch kind 2)
// for storage form 1 (FP32 deviations; see lbm_stream2.cuh).
#include "lbm_stream2.cuh"

namespace olbm {
cudaError_t launch_step2_f32(const StepArgs& a, cudaStream_t st) { return Launch2<1>::step2(a, st); }
}  // namespace olbm

// lbm_f16_step2.cu -- instantiation of the two-step kernels (launch kind 2)
// for storage form 2 (FP16 deviations; see lbm_stream2.cuh).
#include "lbm_stream2.cuh"

namespace olbm {
cudaError_t launch_step2_f16(const StepArgs& a, cudaStream_t st) { return Launch2<2>::step2(a, st); }
}  // namespace olbm

// lbm_f64df.cu -- the step kernel of storage form 3: FP64 populations,
// collision in double-float arithmetic on the FP32 pipes (lbm_df64.cuh).
#include "lbm_kernels.cuh"

namespace olbm {
cudaError_t launch_step_f64df(const StepArgs& a, cudaStream_t st) { return Launch<3>::step(a, st); }
}  // namespace olbm

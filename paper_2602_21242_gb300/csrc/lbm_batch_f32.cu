// lbm_batch_f32.cu -- batched-form kernels for FP32 shifted storage.
#include "lbm_batch_kernels.cuh"

namespace olbm {
OLBM_DEFINE_BATCH(f32, 1)
}  // namespace olbm

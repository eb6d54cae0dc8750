// lbm_batch_f16.cu -- batched-form kernels for FP16 shifted storage.
#include "lbm_batch_kernels.cuh"

namespace olbm {
OLBM_DEFINE_BATCH(f16, 2)
}  // namespace olbm

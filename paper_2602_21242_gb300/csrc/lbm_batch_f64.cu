// lbm_batch_f64.cu -- batched-form kernels for FP64 storage.
#include "lbm_batch_kernels.cuh"

namespace olbm {
OLBM_DEFINE_BATCH(f64, 0)
}  // namespace olbm

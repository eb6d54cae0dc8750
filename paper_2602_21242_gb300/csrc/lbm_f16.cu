// lbm_f16.cu -- instantiation of the step, diagnostics, init, moments and
// state-copy kernels for storage form 2 (see lbm_device.cuh, Form<2>).
#include "lbm_kernels.cuh"

OLBM_DEFINE_LAUNCHERS(2, f16)

// lbm_f32.cu -- instantiation of the step, diagnostics, init, moments and
// state-copy kernels for storage form 1 (see lbm_device.cuh, Form<1>).
#include "lbm_kernels.cuh"

OLBM_DEFINE_LAUNCHERS(1, f32)

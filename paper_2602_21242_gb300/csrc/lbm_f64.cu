// lbm_f64.cu -- instantiation of the step, diagnostics, init, moments and
// state-copy kernels for storage form 0 (see lbm_device.cuh, Form<0>).
#include "lbm_kernels.cuh"

OLBM_DEFINE_LAUNCHERS(0, f64)

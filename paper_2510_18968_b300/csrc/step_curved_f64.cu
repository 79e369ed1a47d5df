// step_curved_f64.cu -- step sequencing and kernels for the curved metric, FP64 path.
#include "step_impl.cuh"

RMHD_INSTANTIATE_STEP(false, double)

// step_flat_f64.cu -- step sequencing and kernels for the flat metric, FP64 path.
#include "step_impl.cuh"

RMHD_INSTANTIATE_STEP(true, double)

// step_flat_f32.cu -- step sequencing and kernels for the flat metric, mixed path (FP32 stencil).
#include "step_impl.cuh"

RMHD_INSTANTIATE_STEP(true, float)

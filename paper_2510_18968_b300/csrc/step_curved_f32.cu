// step_curved_f32.cu -- step sequencing and kernels for the curved metric, mixed path (FP32 stencil).
#include "step_impl.cuh"

RMHD_INSTANTIATE_STEP(false, float)

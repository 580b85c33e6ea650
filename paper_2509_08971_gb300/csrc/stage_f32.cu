// FP32 instantiation of the stage, rate and totals kernels.
#define HH_T float
#define HH_SUFFIX f32
#include "kernels_impl.cuh"

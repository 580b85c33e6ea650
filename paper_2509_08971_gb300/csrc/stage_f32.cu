// FP32 instantiation of the stage, rate and totals kernels.  Built with
// --fmad=false: multiply-adds are fused only where the source calls fmaf.
#define HH_T float
#define HH_WS 1
#define HH_SUFFIX f32
#include "kernels_impl.cuh"

// FP32 instantiation of the WENO5-Z + HLL stage kernel.  Built with
// --fmad=false: multiply-adds are fused only where the source calls fmaf.
#define HH_T float
#define HH_SUFFIX f32
#include "weno_impl.cuh"

// FP64 instantiation of the stage, rate and totals kernels.  Built with
// --fmad=false: every operation is a separately rounded IEEE operation, in the
// same order as the FP64 CPU oracle of the scheme.
#define HH_T double
#define HH_SUFFIX f64
#include "kernels_impl.cuh"

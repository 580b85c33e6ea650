// FP64 instantiation of the WENO5-Z + HLL stage kernel, one IEEE rounding per
// source operation (--fmad=false), the oracle's order of evaluation.
#define HH_T double
#define HH_SUFFIX f64
#include "weno_impl.cuh"

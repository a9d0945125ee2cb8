// SpMV kernels instantiated for storage float, x/y float, accumulation float.
#include "spmv_kernels.cuh"

SPMV_DEFINE_SET(f32_ff, float, float, float)

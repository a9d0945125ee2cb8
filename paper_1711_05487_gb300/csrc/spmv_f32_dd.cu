// SpMV kernels instantiated for storage float, x/y double, accumulation double.
#include "spmv_kernels.cuh"

SPMV_DEFINE_SET(f32_dd, float, double, double)

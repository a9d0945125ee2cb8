// SpMV kernels instantiated for storage double, x/y double, accumulation double.
#include "spmv_kernels.cuh"

SPMV_DEFINE_SET(f64_dd, double, double, double)

// SpMV kernels instantiated for storage __nv_bfloat16, x/y double, accumulation double.
#include "spmv_kernels.cuh"

SPMV_DEFINE_SET(bf16_dd, __nv_bfloat16, double, double)

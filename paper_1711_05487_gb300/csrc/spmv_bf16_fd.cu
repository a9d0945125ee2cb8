// SpMV kernels instantiated for storage __nv_bfloat16, x/y float, accumulation double.
#include "spmv_kernels.cuh"

SPMV_DEFINE_SET(bf16_fd, __nv_bfloat16, float, double)

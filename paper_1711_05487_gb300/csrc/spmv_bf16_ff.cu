// SpMV kernels instantiated for storage __nv_bfloat16, x/y float, accumulation float.
#include "spmv_kernels.cuh"

SPMV_DEFINE_SET(bf16_ff, __nv_bfloat16, float, float)

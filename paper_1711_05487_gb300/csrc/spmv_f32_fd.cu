// SpMV kernels instantiated for storage float, x/y float, accumulation double.
#include "spmv_kernels.cuh"

SPMV_DEFINE_SET(f32_fd, float, float, double)

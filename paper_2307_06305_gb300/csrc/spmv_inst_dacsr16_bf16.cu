// SpMV kernels for dacsr16 indices and bf16 values (see spmv_launch.cuh).
#include "spmv_launch.cuh"

DAMN_SPMV_INSTANCE(spmv_launch_dacsr16_bf16, __nv_bfloat16, int16_t)

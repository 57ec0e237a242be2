// SpMV kernels for dacsr16 indices and f32 values (see spmv_launch.cuh).
#include "spmv_launch.cuh"

DAMN_SPMV_INSTANCE(spmv_launch_dacsr16_f32, float, int16_t)

// SpMV kernels for dacsr8 indices and f32 values (see spmv_launch.cuh).
#include "spmv_launch.cuh"

DAMN_SPMV_INSTANCE(spmv_launch_dacsr8_f32, float, int8_t)

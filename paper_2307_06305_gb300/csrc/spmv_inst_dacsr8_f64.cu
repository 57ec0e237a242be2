// SpMV kernels for dacsr8 indices and f64 values (see spmv_launch.cuh).
#include "spmv_launch.cuh"

DAMN_SPMV_INSTANCE(spmv_launch_dacsr8_f64, double, int8_t)

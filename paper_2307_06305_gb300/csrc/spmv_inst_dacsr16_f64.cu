// SpMV kernels for dacsr16 indices and f64 values (see spmv_launch.cuh).
#include "spmv_launch.cuh"

DAMN_SPMV_INSTANCE(spmv_launch_dacsr16_f64, double, int16_t)

// Kernel module: populations stored as double.
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#define RLBM_S double
#define RLBM_OPS ops_f64
#define RLBM_STEP_MIN_BLOCKS 1
#define RLBM_NAME "f64"
#include "prec_impl.cuh"

// Kernel module: populations stored as __half.
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#define RLBM_S __half
#define RLBM_OPS ops_f16
#define RLBM_STEP_MIN_BLOCKS 7
#define RLBM_NAME "f16"
#include "prec_impl.cuh"

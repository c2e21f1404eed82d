// Kernel module: populations stored as __nv_bfloat16.
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#define RLBM_S __nv_bfloat16
#define RLBM_OPS ops_bf16
#define RLBM_STEP_MIN_BLOCKS 7
#define RLBM_NAME "bf16"
#include "prec_impl.cuh"

// Kernel module: populations stored as float.
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#define RLBM_S float
#define RLBM_OPS ops_f32
#define RLBM_STEP_MIN_BLOCKS 6
#define RLBM_NAME "f32"
#include "prec_impl.cuh"

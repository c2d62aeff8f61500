// Kernels for M = 5 species, FP32 arithmetic with BF16 storage.
#include "lbm_inst.cuh"
LBM_INSTANTIATE(5, bf16, float, __nv_bfloat16)

// Kernels for M = 3 species, FP32 arithmetic with BF16 storage.
#include "lbm_inst.cuh"
LBM_INSTANTIATE(3, bf16, float, __nv_bfloat16)

// Kernels for M = 1 species, FP32 arithmetic with FP16 storage.
#include "lbm_inst.cuh"
LBM_INSTANTIATE(1, f16, float, __half)

// Kernels for M = 2 species, FP32 arithmetic with FP16 storage.
#include "lbm_inst.cuh"
LBM_INSTANTIATE(2, f16, float, __half)

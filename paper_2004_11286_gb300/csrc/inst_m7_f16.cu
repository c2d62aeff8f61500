// Kernels for M = 7 species, FP32 arithmetic with FP16 storage.
#include "lbm_inst.cuh"
LBM_INSTANTIATE(7, f16, float, __half)

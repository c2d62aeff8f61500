// Kernels for M = 8 species, FP32 arithmetic with FP16 storage.
#include "lbm_inst.cuh"
LBM_INSTANTIATE(8, f16, float, __half)

// Kernels for M = 4 species, FP32 arithmetic with FP16 storage.
#include "lbm_inst.cuh"
LBM_INSTANTIATE(4, f16, float, __half)

// Kernels for M = 6 species, FP32 arithmetic with FP16 storage.
#include "lbm_inst.cuh"
LBM_INSTANTIATE(6, f16, float, __half)

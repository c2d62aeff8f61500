// Kernels for M = 3 species, FP32 arithmetic with FP16 storage.
#include "lbm_inst.cuh"
LBM_INSTANTIATE(3, f16, float, __half)

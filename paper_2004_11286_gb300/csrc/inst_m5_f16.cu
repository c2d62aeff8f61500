// Kernels for M = 5 species, FP32 arithmetic with FP16 storage.
#include "lbm_inst.cuh"
LBM_INSTANTIATE(5, f16, float, __half)

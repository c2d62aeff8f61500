// Kernels for M = 1 species, FP32.
#include "lbm_inst.cuh"
LBM_INSTANTIATE(1, f32, float, float)

// Kernels for M = 2 species, FP32.
#include "lbm_inst.cuh"
LBM_INSTANTIATE(2, f32, float, float)

// Kernels for M = 7 species, FP32.
#include "lbm_inst.cuh"
LBM_INSTANTIATE(7, f32, float, float)

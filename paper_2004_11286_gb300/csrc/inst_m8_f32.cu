// Kernels for M = 8 species, FP32.
#include "lbm_inst.cuh"
LBM_INSTANTIATE(8, f32, float, float)

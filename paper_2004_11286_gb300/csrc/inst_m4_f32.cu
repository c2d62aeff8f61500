// Kernels for M = 4 species, FP32.
#include "lbm_inst.cuh"
LBM_INSTANTIATE(4, f32, float, float)

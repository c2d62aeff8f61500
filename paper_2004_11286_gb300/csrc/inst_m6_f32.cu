// Kernels for M = 6 species, FP32.
#include "lbm_inst.cuh"
LBM_INSTANTIATE(6, f32, float, float)

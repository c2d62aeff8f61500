// Kernels for M = 3 species, FP32.
#include "lbm_inst.cuh"
LBM_INSTANTIATE(3, f32, float, float)

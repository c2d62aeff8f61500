// Kernels for M = 5 species, FP32.
#include "lbm_inst.cuh"
LBM_INSTANTIATE(5, f32, float, float)

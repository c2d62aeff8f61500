// Kernels for M = 8 species, FP64.
#include "lbm_inst.cuh"
LBM_INSTANTIATE(8, f64, double, double)

// Kernels for M = 1 species, FP64.
#include "lbm_inst.cuh"
LBM_INSTANTIATE(1, f64, double, double)

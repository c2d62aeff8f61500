// Kernels for M = 2 species, FP64.
#include "lbm_inst.cuh"
LBM_INSTANTIATE(2, f64, double, double)

// Kernels for M = 7 species, FP64.
#include "lbm_inst.cuh"
LBM_INSTANTIATE(7, f64, double, double)

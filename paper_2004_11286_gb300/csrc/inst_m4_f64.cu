// Kernels for M = 4 species, FP64.
#include "lbm_inst.cuh"
LBM_INSTANTIATE(4, f64, double, double)

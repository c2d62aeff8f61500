// Kernels for M = 6 species, FP64.
#include "lbm_inst.cuh"
LBM_INSTANTIATE(6, f64, double, double)

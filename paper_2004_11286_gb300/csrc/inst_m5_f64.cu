// Kernels for M = 5 species, FP64.
#include "lbm_inst.cuh"
LBM_INSTANTIATE(5, f64, double, double)

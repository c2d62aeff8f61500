// Kernels for M = 3 species, FP64.
#include "lbm_inst.cuh"
LBM_INSTANTIATE(3, f64, double, double)

// Kernels for M = 1 species.
#include "lbm_inst.cuh"
LBM_INSTANTIATE(1)

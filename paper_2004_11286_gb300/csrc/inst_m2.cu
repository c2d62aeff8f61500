// Kernels for M = 2 species.
#include "lbm_inst.cuh"
LBM_INSTANTIATE(2)

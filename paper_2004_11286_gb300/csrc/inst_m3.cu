// Kernels for M = 3 species.
#include "lbm_inst.cuh"
LBM_INSTANTIATE(3)

// Kernels for M = 4 species.
#include "lbm_inst.cuh"
LBM_INSTANTIATE(4)

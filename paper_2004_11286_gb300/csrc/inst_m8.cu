// Kernels for M = 8 species.
#include "lbm_inst.cuh"
LBM_INSTANTIATE(8)

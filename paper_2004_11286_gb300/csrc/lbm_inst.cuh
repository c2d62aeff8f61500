// lbm_inst.cuh -- explicit instantiation of one launcher table (one species
// count and one precision per translation unit keeps builds parallel).
#pragma once

#include "lbm_kernels.cuh"

#define LBM_INSTANTIATE(MM, TAG, REAL, STORE)                                \
  namespace lbm {                                                            \
  const KernelSet* kernel_set_m##MM##_##TAG() {                              \
    static const KernelSet s = Launch<MM, REAL, STORE>::make();              \
    return &s;                                                               \
  }                                                                          \
  }

// lbm_inst.cuh -- explicit instantiation of the launcher table for one
// species count (one translation unit per M keeps builds parallel).
#pragma once

#include "lbm_kernels.cuh"

#define LBM_INSTANTIATE(MM)                                                   \
  namespace lbm {                                                             \
  const KernelSet* kernel_set_m##MM(int prec) {                               \
    static const KernelSet s64 = Launch<MM, double, double>::make();          \
    static const KernelSet s32 = Launch<MM, float, float>::make();            \
    switch (prec) {                                                           \
      case 0: return &s64;                                                    \
      case 1: return &s32;                                                    \
      default: return nullptr;                                                \
    }                                                                         \
  }                                                                           \
  }

// lbm_train.h -- host entry points of the closure-network training kernels
// (lbm_train.cu), called by the C-ABI layer.
#pragma once

#include <cuda_runtime.h>

namespace lbm {

struct MlpShape {
  int H, F, O;   // hidden width, padded feature and output counts
  int valid;     // outputs that enter the loss (3M)
};

// Device scratch for one mini-batch of `rows` samples: [rows][H] for the
// hidden pre-activations, activations and their gradients, [rows][O] for the
// outputs and their gradients.
struct MlpScratch {
  float *h1, *a1, *h2, *a2, *d1, *d2, *out, *dout;
};

// Gradient of the mean-squared loss at weights w over `rows` samples
// (features X [rows][F], targets T [rows][O]) into g (packed like w); the loss
// into *d_loss (device).
cudaError_t mlp_train_grad(cudaStream_t s, const MlpShape& sh, const float* w, const float* X, const float* T,
                           int rows, const MlpScratch& z, float* g, double* d_loss);
// FP32 forward pass only (outputs in z.out).
cudaError_t mlp_train_forward(cudaStream_t s, const MlpShape& sh, const float* w, const float* X, int rows,
                              const MlpScratch& z);
// One Adam step (step number t >= 1, beta1 0.9, beta2 0.999, eps 1e-8).
cudaError_t mlp_adam(cudaStream_t s, float* w, const float* g, float* m, float* v, long long count, float lr, int t);

}  // namespace lbm

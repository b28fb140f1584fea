// Learned cost model: MLP kernels (mlp.cu) and the model around them
// (learned.cpp).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>

namespace wt {

constexpr int kMlpFeatures = 18;  // launch features (learned.cpp)
constexpr int kMlpHidden = 64;
constexpr int kMlpParams = kMlpHidden * kMlpFeatures + kMlpHidden + kMlpHidden * kMlpHidden + kMlpHidden +
                           kMlpHidden + 1;
constexpr int kMlpMaxBatch = 128;

size_t mlp_train_smem(int batch);
// `steps` Adam steps (t0 taken before) over mini-batches idx[steps][batch]
// of (X, Y); all pointers device memory; loss[step] = batch mean squared
// error before the step's update.
cudaError_t mlp_train_launch(float *params, float *m, float *v, int t0, const float *X, const float *Y,
                             const int *idx, int steps, int batch, float lr, float beta1, float beta2, float eps,
                             float wd, float *loss, cudaStream_t stream);
cudaError_t mlp_forward_launch(const float *params, const float *X, int n, float *Y, cudaStream_t stream);

}  // namespace wt

// Learned cost model (learned.cpp): launch features, the trained MLP and
// its use by the scheduler.
#pragma once

#include <cuda_runtime.h>

#include <string>

#include "wt_sched.hpp"

namespace wt {

// Features of one launch (a fused group, or the per-stage kernel of one
// stage when !fused) at image size W0 x H0; false if infeasible.
bool launch_features(const Pipeline &p, const std::vector<int> &seg, const GroupParams &prm, bool fused, int W0,
                     int H0, int dtype, const GpuConfig &cfg, const std::vector<StageStats> &st, float *f);

// The MLP kernels on host arrays (copies in and out).
void mlp_train_steps(float *params, float *m, float *v, int t0, const float *x, const float *y, int n,
                     const int32_t *idx, int steps, int batch, float lr, float wd, float *loss, cudaStream_t s);
void mlp_forward(const float *params, const float *x, int n, float *y, cudaStream_t s);

// The process-wide model: trained on (features, log ms) or loaded.
float costmodel_train(const float *features, const float *log_ms, int n, int epochs, int batch, float lr,
                      uint64_t seed);
void costmodel_predict(const float *features, int n, float *log_ms, cudaStream_t s);
void costmodel_reset();
void costmodel_save(const std::string &path);
void costmodel_load(const std::string &path);

}  // namespace wt

// Scheduling: cost models and DP-Fusion (sched.cpp), batched runtime.
#pragma once

#include <cuda_runtime.h>

#include "wt_internal.hpp"

namespace wt {

Schedule auto_schedule(const Pipeline &p, int W, int H, int dtype, int model);
void run_batch(Pipeline &p, const wt_image *in, const wt_image *out, int n_images, cudaStream_t stream);

}  // namespace wt

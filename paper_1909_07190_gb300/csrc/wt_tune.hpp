// Measured schedule search (tune.cpp).
#pragma once

#include <cuda_runtime.h>

#include "wt_internal.hpp"

namespace wt {

// Kernel time (ms per run) of the installed schedule: min over 3 samples of
// the mean of `reps` runs; n_images >= 1 times wt_run_batch.  Infinity if a
// run raised the device error word.
double time_installed(Pipeline &p, const wt_image *in, int n_in, const wt_image *out, int n_out, int n_images,
                      cudaStream_t s, int reps);
// Per-launch kernel times of one run of the installed schedule (each launch
// repeated `reps` times alone; min over 3 samples of the mean).
struct LaunchTime {
  int first_stage = 0, n_stages = 0;
  bool fused = false;
  double ms = 0;
};
std::vector<LaunchTime> time_launches(Pipeline &p, const wt_image *in, int n_in, const wt_image *out, int n_out,
                                      cudaStream_t s, int reps);
// Compiles the kernels of candidate schedules in parallel host threads.
void precompile(Pipeline &p, const std::vector<Schedule> &cands, const wt_image *in, int n_in, const wt_image *out,
                int n_out, bool persistent);

struct TuneResult {
  double best_ms = 0;
  int timed = 0;
};
TuneResult tune(Pipeline &p, const wt_image *in, int n_in, const wt_image *out, int n_out, int n_images,
                int max_variants, int reps, cudaStream_t stream);

}  // namespace wt

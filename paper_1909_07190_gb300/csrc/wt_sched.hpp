// Scheduling: cost models and DP-Fusion (sched.cpp), learned model
// (learned.cpp).
#pragma once

#include <cuda_runtime.h>

#include <cmath>
#include <functional>

#include "wt_internal.hpp"

namespace wt {

// The GPU quantities Alg. 2 uses (Table 1), filled from the device.
struct GpuConfig {
  int nsms = 0, cores_per_sm = 0;
  double glmem_bw = 0;  // bytes/s
  int max_smem_per_tb = 0, smem_per_sm = 0, max_warps_per_sm = 0, max_tb_per_sm = 0;
  int regs_per_sm = 0, max_regs_per_th = 0, warp_size = 32, max_th_per_sm = 0;
};
GpuConfig default_gb300();
GpuConfig device_config(int dev);

// Sec. 4 OTPW geometry.
void otpw_warp_sizes(const int B[3], int warp_size, int W[3]);
int64_t otpw_scratchpad_points(const int B[3], const int W[3], const int T[3], const int O[3]);
// Alg. 2 occupancy lines (shared memory, registers).
double alg2_occupancy(const GpuConfig &g, int64_t smem_per_tb, int warps_per_tb, int regs_per_th,
                      int *max_tb_per_sm, int *warps_per_sm);
// Minimum number of txn-byte transactions covering the accesses (A17).
int64_t min_gl_txs(const int64_t *addr, int n, int access_bytes, int txn);

// Sec. 6 preprocessing: per-stage time per iteration and registers.
struct StageStats {
  double ns_per_iter = 1.0;
  int regs = 24;
  bool measured = false;
};
std::vector<StageStats> stage_stats(const Pipeline &p, bool measure);

extern const char *kTermNames[7];
struct CostWeights {
  double w[7];
};
CostWeights default_weights();
CostWeights current_weights();
void set_weights(const CostWeights &w);

struct CostInfo {
  double t[7] = {0, 0, 0, 0, 0, 0, 0};
  double cost = INFINITY;
  bool feasible = false;
  int regs = 0, smem_per_tb = 0;
  double occupancy = 0, waves = 0, work = 0;
  int64_t tiles = 0;
};
double work_share(const Pipeline &p, const std::vector<int> &stages, int W0, int H0);
double pipeline_bytes(const Pipeline &p, int W0, int H0, int dtype);
int estimate_regs(const GroupGeom &g, int V, const std::vector<StageStats> &st);
CostInfo cost_group(const Pipeline &p, const std::vector<int> &stages, const GroupParams &prm, int txn, int W0,
                    int H0, int dtype, const GpuConfig &cfg, const std::vector<StageStats> &st,
                    const CostWeights &w, double pipeline_bytes, const GroupGeom *pre = nullptr);
CostInfo cost_plain(const Pipeline &p, int s, int W0, int H0, int dtype, const CostWeights &w, double pbytes);

// Alternative scorer of a candidate (the learned model); lower is better.
using CandidateScorer = std::function<double(const std::vector<int> &, const GroupParams &, const CostInfo &)>;

// HBM bytes of a reduction chain across levels run as one kernel.
double chain_bytes(const Pipeline &p, const std::vector<int> &seg, int W0, int H0);
// HBM bytes of a group of down-sampling stages run as cascade launches
// (cascade_units): each pair's first stage is not read back.
double cascade_bytes(const Pipeline &p, const std::vector<int> &seg, int W0, int H0);
struct SegmentChoice {
  double cost = INFINITY;
  bool fused = false;
  GroupParams prm;
  CostInfo info;
};
SegmentChoice best_for_segment(const Pipeline &p, const std::vector<int> &seg, int W, int H, int dtype,
                               const GpuConfig &cfg, const std::vector<StageStats> &st, const CostWeights &w,
                               double pbytes, const CandidateScorer *scorer);
Schedule dp_fusion(const Pipeline &p, int W, int H, int dtype, const GpuConfig &cfg,
                   const std::vector<StageStats> &st, const CostWeights &w, const CandidateScorer *scorer,
                   int max_group);
// Longest group DP-Fusion forms (stages).
constexpr int kMaxGroupStages = 16;
Schedule auto_schedule(const Pipeline &p, int W, int H, int dtype, int model);
// The analytic model's choice for stages [first, first + n) as
// wt_schedule_auto's DP-Fusion weighs that group.
SegmentChoice auto_segment(const Pipeline &p, int first, int n, int W, int H, int dtype);

// learned.cpp (see wt_learned.hpp)
bool costmodel_ready();
Schedule learned_schedule(const Pipeline &p, int W, int H, int dtype, const GpuConfig &cfg,
                          const std::vector<StageStats> &st, int max_group);

}  // namespace wt

// Learned cost model (placeholder until the MLP lands): the analytic cost.
#include "wt_sched.hpp"

namespace wt {

CandidateScorer learned_scorer(const Pipeline &p, int W, int H, int dtype, const GpuConfig &cfg,
                               const std::vector<StageStats> &st) {
  (void)p; (void)W; (void)H; (void)dtype; (void)cfg; (void)st;
  return [](const std::vector<int> &, const GroupParams &, const CostInfo &ci) { return ci.cost; };
}

}  // namespace wt

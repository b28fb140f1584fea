// Scheduling (placeholder until the cost models land): one fused group.
#include "wt_sched.hpp"

namespace wt {

Schedule auto_schedule(const Pipeline &p, int W, int H, int dtype, int model) {
  (void)W; (void)H; (void)dtype; (void)model;
  Schedule s;
  s.exec = WT_EXEC_FUSED;
  s.n_groups = 1;
  s.group_of_stage.assign(p.stages.size(), 0);
  s.params.assign(1, GroupParams());
  s.installed = true;
  return s;
}

void run_batch(Pipeline &p, const wt_image *in, const wt_image *out, int n_images, cudaStream_t stream) {
  (void)p; (void)in; (void)out; (void)n_images; (void)stream;
  fail(WT_EUNSUPPORTED, "batched runs are not implemented yet");
}

}  // namespace wt

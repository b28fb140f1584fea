// Batched runtime (placeholder until the persistent batched launch lands).
#include "wt_sched.hpp"

namespace wt {

void run_batch(Pipeline &p, const wt_image *in, const wt_image *out, int n_images, cudaStream_t stream) {
  (void)p; (void)in; (void)out; (void)n_images; (void)stream;
  fail(WT_EUNSUPPORTED, "batched runs are not implemented yet");
}

}  // namespace wt

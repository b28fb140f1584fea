// wt_run_static: a pipeline run that allocates no device memory.
//
// Some callers cannot let a library call cudaMalloc: processes that hand
// all device memory to their own allocator up front and run under a fixed
// budget (a late cudaMalloc would fail or fragment it), and latency-critical
// paths where cudaMalloc/cudaFree may synchronize the whole device.  For
// them this entry point runs the installed schedule with the intermediates
// between groups and the device status word placed in one file-scope static
// device array instead of the pipeline's workspace.
#include <cuda_runtime.h>

#include <mutex>

#include "wt.h"
#include "wt_jit.hpp"
#include "wt_runtime.hpp"

namespace {

// Scratch of every wt_run_static call on a device: the first kCtrlBytes
// hold the status word the kernels' bounded waits write and the tile-queue
// counters, the rest the plan's intermediates.  Every GPU that loads the
// library holds it until exit.
constexpr size_t kStaticScratchBytes = size_t(32) << 20;
constexpr size_t kStatusBytes = wt::kCtrlBytes;
static __device__ __align__(256) unsigned char g_wt_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
char *g_base[kMaxDevices] = {};

// Device address of the scratch on the current device.  The name of a
// __device__ array in host code is only a host-side stand-in, so the
// address is taken once per device with cudaGetSymbolAddress.
char *scratch_address(int dev) {
  if (dev < 0 || dev >= kMaxDevices) wt::fail(WT_EUNSUPPORTED, "device index beyond 63");
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_base[dev]) {
    void *ptr = nullptr;
    cudaError_t rc = cudaGetSymbolAddress(&ptr, g_wt_static_scratch);
    if (rc != cudaSuccess || !ptr)
      wt::fail(WT_ECUDA, std::string("cudaGetSymbolAddress(static scratch): ") + cudaGetErrorString(rc));
    g_base[dev] = (char *)ptr;
  }
  return g_base[dev];
}

}  // namespace

namespace wt {

int32_t *static_status_word(int dev) {
  if (dev < 0 || dev >= kMaxDevices) return nullptr;
  std::lock_guard<std::mutex> lk(g_mu);
  return (int32_t *)g_base[dev];
}

// Launches a plan whose workspace is `base` and whose status word is `err`;
// every kernel must already be loaded (loading code allocates device memory).
static void run_plan_at(Pipeline &p, RunPlan &plan, char *base, int32_t *err, cudaStream_t stream, int dev) {
  if ((int)plan.launches.size() > kMaxLaunches) fail(WT_EUNSUPPORTED, "more than 500 launches per run");
  int li = 0;
  for (Launch &L : plan.launches) {
    Kernel *k = find_kernel(p, L, dev);
    if (!k)
      fail(WT_EUNSUPPORTED,
           "group kernel " + L.kname + " is not loaded on this device; run the pipeline once with wt_run "
           "(same schedule, image sizes and dtypes) first, since loading kernel code allocates device memory");
    KernelArgs a = launch_args(p, plan, L, *k, base, err, li++, dev);
    launch(L, *k, a, stream);
  }
}

}  // namespace wt

struct wt_pipeline : wt::Pipeline {};

extern "C" wt_status wt_run_static(wt_pipeline *p, const wt_image *inputs, int32_t n_inputs,
                                   const wt_image *outputs, int32_t n_outputs, void *stream) {
  try {
    if (!p) wt::fail(WT_EINVAL, "null pipeline");
    if (!inputs || !outputs) wt::fail(WT_EINVAL, "null image array");
    std::lock_guard<std::mutex> lk(p->mu);
    wt::RunPlan plan = wt::build_plan(*p, inputs, n_inputs, outputs, n_outputs);
    if (plan.ws_bytes > (int64_t)(kStaticScratchBytes - kStatusBytes))
      wt::fail(WT_EINVAL, "this run needs " + std::to_string(plan.ws_bytes) +
                              " bytes of intermediates; wt_run_static holds at most " +
                              std::to_string(kStaticScratchBytes - kStatusBytes) +
                              " (use fewer groups, smaller images, or wt_run)");
    int dev = 0;
    wt::check_rt(cudaGetDevice(&dev), "cudaGetDevice");
    char *base = scratch_address(dev);
    cudaStream_t st = (cudaStream_t)stream;
    // the status word and the tile-queue counters must start at zero;
    // intermediates need no clearing
    wt::check_rt(cudaMemsetAsync(base, 0, kStatusBytes, st), "cudaMemsetAsync(status word)");
    wt::run_plan_at(*p, plan, base + kStatusBytes, (int32_t *)base, st, dev);
    if (dev < 64) p->static_devs |= uint64_t(1) << dev;
    wt::set_last_error("");
    return WT_OK;
  } catch (const wt::Error &e) {
    wt::set_last_error(e.msg);
    return e.code;
  } catch (const std::exception &e) {
    wt::set_last_error(e.what());
    return WT_EINVAL;
  }
}

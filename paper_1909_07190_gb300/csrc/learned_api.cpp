// C ABI of the learned cost model and per-launch timing (include/wt.h).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "wt.h"
#include "wt_jit.hpp"
#include "wt_learned.hpp"
#include "wt_mlp.hpp"
#include "wt_runtime.hpp"
#include "wt_tune.hpp"

struct wt_pipeline : wt::Pipeline {};

namespace {

template <class F>
wt_status guard(F &&f) {
  try {
    f();
    wt::set_last_error("");
    return WT_OK;
  } catch (const wt::Error &e) {
    wt::set_last_error(e.msg);
    return e.code;
  } catch (const std::bad_alloc &) {
    wt::set_last_error("host allocation failed");
    return WT_ENOMEM;
  } catch (const std::exception &e) {
    wt::set_last_error(e.what());
    return WT_EINVAL;
  }
}

static_assert(WT_COSTMODEL_FEATURES == wt::kMlpFeatures, "feature count");
static_assert(WT_COSTMODEL_HIDDEN == wt::kMlpHidden, "hidden width");
static_assert(WT_MLP_PARAMS == wt::kMlpParams, "parameter count");

}  // namespace

extern "C" {

wt_status wt_schedule_time_launches(wt_pipeline *p, const wt_image *inputs, int32_t n_inputs,
                                    const wt_image *outputs, int32_t n_outputs, int32_t reps, void *stream,
                                    double *ms, int32_t *info, int32_t cap, int32_t *n_launches) {
  return guard([&] {
    if (!p || !inputs || !outputs || reps < 1 || cap < 0) wt::fail(WT_EINVAL, "bad arguments");
    std::lock_guard<std::mutex> lk(p->mu);
    auto t = wt::time_launches(*p, inputs, n_inputs, outputs, n_outputs, (cudaStream_t)stream, reps);
    if (n_launches) *n_launches = (int32_t)t.size();
    if ((int)t.size() > cap && (ms || info)) wt::fail(WT_EINVAL, "arrays too small for the launches");
    for (size_t i = 0; i < t.size(); i++) {
      if (ms) ms[i] = t[i].ms;
      if (info) {
        info[3 * i] = t[i].first_stage;
        info[3 * i + 1] = t[i].n_stages;
        info[3 * i + 2] = t[i].fused ? 1 : 0;
      }
    }
  });
}

wt_status wt_costmodel_features(wt_pipeline *p, int32_t first_stage, int32_t n_stages, const wt_group_params *prm,
                                int32_t fused, int32_t width, int32_t height, int32_t dtype, float *features) {
  return guard([&] {
    if (!p || !features) wt::fail(WT_EINVAL, "bad arguments");
    if (first_stage < 0 || n_stages < 1 || first_stage + n_stages > (int)p->stages.size())
      wt::fail(WT_EINVAL, "stage range");
    if (width < 1 || height < 1 || dtype < WT_F32 || dtype > WT_BF16) wt::fail(WT_EINVAL, "bad size or dtype");
    if (fused && !prm) wt::fail(WT_EINVAL, "a fused launch needs its group parameters");
    wt::GroupParams q;
    if (prm) {
      q.tile_h = prm->tile_h;
      q.warps_per_block = prm->warps_per_block;
      q.frac_reg = prm->frac_reg;
      q.vec = prm->vec ? prm->vec : 4;
      q.chunk_rows = prm->chunk_rows ? prm->chunk_rows : 8;
      q.n_buffers = prm->n_buffers ? prm->n_buffers : 2;
      if (q.tile_h < 1 || q.warps_per_block < 1 || q.warps_per_block > 16 || !(q.frac_reg >= 0 && q.frac_reg <= 1))
        wt::fail(WT_EINVAL, "bad group parameters");
    }
    std::vector<int> seg;
    for (int s = first_stage; s < first_stage + n_stages; s++) seg.push_back(s);
    int dev = -1;
    bool gpu = cudaGetDevice(&dev) == cudaSuccess;
    cudaGetLastError();
    wt::GpuConfig cfg = gpu ? wt::device_config(dev) : wt::default_gb300();
    auto st = wt::stage_stats(*p, false);
    if (!wt::launch_features(*p, seg, q, fused != 0, width, height, dtype, cfg, st, features))
      wt::fail(WT_EUNSUPPORTED, "launch is infeasible (group does not fuse or does not fit)");
  });
}

wt_status wt_costmodel_collect(wt_pipeline *p, const wt_image *inputs, int32_t n_inputs,
                               const wt_image *outputs, int32_t n_outputs, int32_t reps, void *stream,
                               float *features, float *log_ms, int32_t *stages, int32_t cap, int32_t *n_rows) {
  return guard([&] {
    if (!p || !inputs || !outputs || reps < 1 || cap < 0) wt::fail(WT_EINVAL, "bad arguments");
    std::lock_guard<std::mutex> lk(p->mu);
    auto t = wt::time_launches(*p, inputs, n_inputs, outputs, n_outputs, (cudaStream_t)stream, reps);
    wt::RunPlan plan = wt::build_plan(*p, inputs, n_inputs, outputs, n_outputs);
    if (plan.launches.size() != t.size()) wt::fail(WT_EUNSUPPORTED, "run plan changed");
    const auto groups = wt::schedule_groups(*p);
    int dev = 0;
    wt::check_rt(cudaGetDevice(&dev), "cudaGetDevice");
    const wt::GpuConfig cfg = wt::device_config(dev);
    const auto st = wt::stage_stats(*p, false);
    const int W = inputs[0].width, H = inputs[0].height, dtype = inputs[0].dtype;
    int rows = 0;
    for (size_t i = 0; i < t.size(); i++) {
      const wt::Launch &L = plan.launches[i];
      const bool warp_tile = L.fused && !L.key.otptb;
      const bool per_stage = !L.fused && L.key.plain && !L.key.down && !L.key.cascade && !L.key.chain && !L.key.vol;
      if (!warp_tile && !per_stage) continue;
      std::vector<int> seg(L.stages.begin(), L.stages.end());
      wt::GroupParams q;
      if (warp_tile) {
        // the schedule parameters of the group this launch runs
        for (size_t gi = 0; gi < groups.size(); gi++)
          if (!groups[gi].empty() && groups[gi][0] == seg[0]) q = wt::group_params(*p, (int)gi);
        q.vec = L.key.vec;  // the pixels per lane the kernel was generated for
      }
      float f[WT_COSTMODEL_FEATURES];
      if (!wt::launch_features(*p, seg, q, warp_tile, W, H, dtype, cfg, st, f)) continue;
      if (rows < cap) {
        if (features) std::memcpy(features + (size_t)rows * WT_COSTMODEL_FEATURES, f, sizeof f);
        if (log_ms) log_ms[rows] = (float)std::log(std::max(t[i].ms, 1e-9));
        if (stages) {
          stages[2 * rows] = seg[0];
          stages[2 * rows + 1] = (int32_t)seg.size();
        }
      } else if (features || log_ms || stages) {
        wt::fail(WT_EINVAL, "arrays too small for the launches");
      }
      rows++;
    }
    if (n_rows) *n_rows = rows;
  });
}

wt_status wt_mlp_train_steps(float *params, float *adam_m, float *adam_v, int32_t t0, const float *x,
                             const float *y, int32_t n, const int32_t *idx, int32_t steps, int32_t batch, float lr,
                             float weight_decay, float *loss, void *stream) {
  return guard([&] {
    if (!params || !adam_m || !adam_v || !x || !y || (steps > 0 && !idx) || t0 < 0)
      wt::fail(WT_EINVAL, "bad arguments");
    if (!(lr > 0) || !(weight_decay >= 0)) wt::fail(WT_EINVAL, "bad learning rate or weight decay");
    wt::mlp_train_steps(params, adam_m, adam_v, t0, x, y, n, idx, steps, batch, lr, weight_decay, loss,
                        (cudaStream_t)stream);
  });
}

wt_status wt_mlp_forward(const float *params, const float *x, int32_t n, float *y, void *stream) {
  return guard([&] {
    if (!params || (n > 0 && (!x || !y))) wt::fail(WT_EINVAL, "bad arguments");
    wt::mlp_forward(params, x, n, y, (cudaStream_t)stream);
  });
}

wt_status wt_costmodel_train(const float *features, const float *log_ms, int32_t n, int32_t epochs, int32_t batch,
                             float lr, uint64_t seed, float *final_loss) {
  return guard([&] {
    if (!features || !log_ms) wt::fail(WT_EINVAL, "bad arguments");
    if (!(lr > 0)) wt::fail(WT_EINVAL, "bad learning rate");
    float l = wt::costmodel_train(features, log_ms, n, epochs, batch, lr, seed);
    if (final_loss) *final_loss = l;
  });
}

wt_status wt_costmodel_predict(const float *features, int32_t n, float *log_ms) {
  return guard([&] {
    if (n < 0 || (n > 0 && (!features || !log_ms))) wt::fail(WT_EINVAL, "bad arguments");
    wt::costmodel_predict(features, n, log_ms, nullptr);
  });
}

int32_t wt_costmodel_ready(void) { return wt::costmodel_ready() ? 1 : 0; }

wt_status wt_costmodel_reset(void) {
  return guard([&] { wt::costmodel_reset(); });
}

wt_status wt_costmodel_save(const char *path) {
  return guard([&] {
    if (!path) wt::fail(WT_EINVAL, "null path");
    wt::costmodel_save(path);
  });
}

wt_status wt_costmodel_load(const char *path) {
  return guard([&] {
    if (!path) wt::fail(WT_EINVAL, "null path");
    wt::costmodel_load(path);
  });
}

}  // extern "C"

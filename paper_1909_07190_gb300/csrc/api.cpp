// C ABI entry points (include/wt.h, include/wt_debug.h).  Every entry point
// converts internal errors to a wt_status and a thread-local message.
#include <functional>
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>

#include "wt.h"
#include "wt_debug.h"
#include "wt_jit.hpp"
#include "wt_runtime.hpp"
#include "wt_sched.hpp"
#include "wt_tune.hpp"

struct wt_pipeline : wt::Pipeline {};

namespace wt {
void inject_alloc_failure(int kind, int after);
void live_objects(long long *pipelines, long long *device_bytes);
}  // namespace wt

namespace {
using wt::fail;
thread_local std::string g_err;

template <class F>
wt_status guard(F &&f) {
  try {
    f();
    g_err.clear();
    return WT_OK;
  } catch (const wt::Error &e) {
    g_err = e.msg;
    return e.code;
  } catch (const std::bad_alloc &) {
    g_err = "host allocation failed";
    return WT_ENOMEM;
  } catch (const std::exception &e) {
    g_err = e.what();
    return WT_EINVAL;
  }
}

void default_schedule(wt::Pipeline &p) {
  p.sched = wt::Schedule();
  p.sched.exec = WT_EXEC_FUSED;
  p.sched.n_groups = 1;
  p.sched.group_of_stage.assign(p.stages.size(), 0);
  p.sched.params.assign(1, wt::GroupParams());
  p.sched.installed = true;
}

wt::Schedule to_schedule(const wt::Pipeline &p, const wt_schedule_desc *d) {
  wt::Schedule s;
  if (!d) fail(WT_EINVAL, "null schedule");
  if (d->exec != WT_EXEC_FUSED && d->exec != WT_EXEC_PLAIN) fail(WT_EINVAL, "bad exec mode");
  s.exec = d->exec;
  s.intermediate_dtype = d->intermediate_dtype;
  if (s.intermediate_dtype < -1 || s.intermediate_dtype > WT_BF16) fail(WT_EINVAL, "bad intermediate dtype");
  const int n = (int)p.stages.size();
  if (s.exec == WT_EXEC_FUSED) {
    if (d->n_groups < 1 || d->n_groups > n) fail(WT_EINVAL, "n_groups out of range");
    if (!d->group_of_stage) fail(WT_EINVAL, "group_of_stage is required");
    s.n_groups = d->n_groups;
    s.group_of_stage.assign(d->group_of_stage, d->group_of_stage + n);
    // contiguous runs in topological order, numbered 0..n_groups-1
    int cur = 0;
    for (int i = 0; i < n; i++) {
      int g = s.group_of_stage[i];
      if (g < 0 || g >= s.n_groups) fail(WT_EINVAL, "group index out of range");
      if (i == 0 && g != 0) fail(WT_EINVAL, "groups must be numbered in topological order");
      if (g == cur) continue;
      if (g != cur + 1) fail(WT_EINVAL, "every group must be a contiguous run of stages");
      cur = g;
    }
    if (cur != s.n_groups - 1) fail(WT_EINVAL, "empty group");
    s.params.assign(s.n_groups, wt::GroupParams());
    if (d->params)
      for (int g = 0; g < s.n_groups; g++) {
        const wt_group_params &q = d->params[g];
        wt::GroupParams &r = s.params[g];
        if (q.tile_h < 1 || q.tile_h > 4096) fail(WT_EINVAL, "tile_h out of range");
        if (q.warps_per_block < 1 || q.warps_per_block > 16) fail(WT_EINVAL, "warps_per_block out of range");
        if (!(q.frac_reg >= 0.f && q.frac_reg <= 1.f)) fail(WT_EINVAL, "frac_reg out of [0,1]");
        bool zgroup = false;  // the group has a plane-offset tap: a 3-D group
        for (int i = 0; i < n; i++)
          if (s.group_of_stage[i] == g && p.stages[i].has_z) zgroup = true;
        if (q.vec != 0 && q.vec != 4 && q.vec != 8 &&
            !((q.flags & WT_FLAG_OTPTB) && (q.vec == 1 || q.vec == 2)) && !(zgroup && (q.vec == 1 || q.vec == 2)))
          fail(WT_EINVAL, "vec must be 0, 4 or 8 (1 or 2 with WT_FLAG_OTPTB or in 3-D groups)");
        if (q.tile_o < 0 || q.tile_o > 64) fail(WT_EINVAL, "tile_o out of range");
        if (q.max_regs < 0 || q.max_regs > 255) fail(WT_EINVAL, "max_regs out of range");
        if (q.chunk_rows < 0 || q.chunk_rows > 64) fail(WT_EINVAL, "chunk_rows out of range");
        if (q.n_buffers < 0 || q.n_buffers > 8) fail(WT_EINVAL, "n_buffers out of range");
        r.tile_h = q.tile_h;
        r.warps_per_block = q.warps_per_block;
        r.frac_reg = q.frac_reg;
        r.vec = q.vec;
        r.max_regs = q.max_regs;
        r.chunk_rows = q.chunk_rows ? q.chunk_rows : 8;
        r.n_buffers = q.n_buffers ? q.n_buffers : 2;
        if (q.flags & ~(WT_FLAG_NO_PAIRS | WT_FLAG_NO_TILE_SPLIT | WT_FLAG_PLAIN | WT_FLAG_OTPTB | WT_FLAG_SMEM16 |
                        WT_FLAG_ZSTREAM | WT_FLAG_TEST_STALL | WT_FLAG_TILE_QUEUE |
                        WT_FLAG_ONE_STREAM | WT_FLAG_NO_FOLD))
          fail(WT_EINVAL, "unknown flags");
        r.tile_o = q.tile_o;
        r.zstream = (q.flags & WT_FLAG_ZSTREAM) ? 1 : 0;
        r.smem16 = (q.flags & WT_FLAG_SMEM16) ? 1 : 0;
        r.plain = (q.flags & WT_FLAG_PLAIN) ? 1 : 0;
        r.otptb = (q.flags & WT_FLAG_OTPTB) ? 1 : 0;
        r.pairs = (q.flags & WT_FLAG_NO_PAIRS) ? 0 : 1;
        r.tile_split = (q.flags & WT_FLAG_NO_TILE_SPLIT) ? 0 : 1;
        r.test_stall = (q.flags & WT_FLAG_TEST_STALL) ? 1 : 0;
        r.tile_queue = (q.flags & WT_FLAG_TILE_QUEUE) ? 1 : 0;
        r.one_stream = (q.flags & WT_FLAG_ONE_STREAM) ? 1 : 0;
        r.fold = (q.flags & WT_FLAG_NO_FOLD) ? 0 : 1;
      }
  } else {
    s.n_groups = n;
    s.group_of_stage.resize(n);
    for (int i = 0; i < n; i++) s.group_of_stage[i] = i;
    s.params.assign(n, wt::GroupParams());
  }
  s.installed = true;
  return s;
}

void install(wt::Pipeline &p, const wt_schedule_desc *d) {
  p.sched = to_schedule(p, d);
  p.sched_version++;
}

int64_t image_bytes(const wt_image &im) {
  return im.pitch_bytes * (int64_t)im.height * im.channels;
}
}  // namespace

namespace wt {
// Sets the message wt_last_error() returns on this thread.
void set_last_error(const std::string &msg) { g_err = msg; }
}  // namespace wt

extern "C" {

const char *wt_last_error(void) { return g_err.c_str(); }

int32_t wt_version(void) { return 100; }

wt_status wt_pipeline_create(const wt_stage *stages, int32_t n_stages, const int32_t *input_channels,
                             int32_t n_inputs, const int32_t *outputs, int32_t n_outputs, int32_t boundary,
                             wt_pipeline **out) {
  return guard([&] {
    if (!out) wt::fail(WT_EINVAL, "null out");
    if (boundary != WT_BOUNDARY_CLAMP) wt::fail(WT_EUNSUPPORTED, "only the clamp-to-edge boundary is supported");
    wt::host_alloc_point();
    auto p = std::make_unique<wt_pipeline>();
    wt::build_pipeline(*p, stages, n_stages, input_channels, n_inputs, outputs, n_outputs);
    wt::host_alloc_point();
    default_schedule(*p);
    *out = p.release();
  });
}

wt_status wt_pipeline_destroy(wt_pipeline *p) {
  return guard([&] { delete p; });
}

wt_status wt_schedule(wt_pipeline *p, const wt_schedule_desc *desc) {
  return guard([&] {
    if (!p) wt::fail(WT_EINVAL, "null pipeline");
    std::lock_guard<std::mutex> lk(p->mu);
    install(*p, desc);
  });
}

wt_status wt_schedule_auto(wt_pipeline *p, int32_t width, int32_t height, int32_t dtype, int32_t model) {
  return guard([&] {
    if (!p) wt::fail(WT_EINVAL, "null pipeline");
    if (width < 1 || height < 1) wt::fail(WT_EINVAL, "bad size");
    if (dtype < WT_F32 || dtype > WT_BF16) wt::fail(WT_EINVAL, "bad dtype");
    if (model != WT_MODEL_ANALYTIC && model != WT_MODEL_LEARNED) wt::fail(WT_EINVAL, "bad model");
    std::lock_guard<std::mutex> lk(p->mu);
    wt::Schedule s = wt::auto_schedule(*p, width, height, dtype, model);
    p->sched = s;
    p->sched_version++;
  });
}

wt_status wt_schedule_get(const wt_pipeline *p, int32_t *exec, int32_t *n_groups, int32_t *group_of_stage,
                          wt_group_params *params) {
  return guard([&] {
    if (!p) wt::fail(WT_EINVAL, "null pipeline");
    const wt::Schedule &s = p->sched;
    if (exec) *exec = s.exec;
    if (n_groups) *n_groups = s.n_groups;
    if (group_of_stage)
      for (size_t i = 0; i < p->stages.size(); i++) group_of_stage[i] = s.group_of_stage[i];
    if (params)
      for (int g = 0; g < s.n_groups; g++) {
        const wt::GroupParams &r = s.params[g];
        params[g].tile_h = r.tile_h;
        params[g].warps_per_block = r.warps_per_block;
        params[g].frac_reg = r.frac_reg;
        params[g].vec = r.vec;
        params[g].max_regs = r.max_regs;
        params[g].chunk_rows = r.chunk_rows;
        params[g].n_buffers = r.n_buffers;
        params[g].flags = (r.pairs ? 0 : WT_FLAG_NO_PAIRS) | (r.tile_split ? 0 : WT_FLAG_NO_TILE_SPLIT) |
                          (r.plain ? WT_FLAG_PLAIN : 0) | (r.otptb ? WT_FLAG_OTPTB : 0) |
                          (r.smem16 ? WT_FLAG_SMEM16 : 0) | (r.zstream ? WT_FLAG_ZSTREAM : 0) |
                          (r.test_stall ? WT_FLAG_TEST_STALL : 0) | (r.tile_queue ? WT_FLAG_TILE_QUEUE : 0) |
                          (r.one_stream ? WT_FLAG_ONE_STREAM : 0) | (r.fold ? 0 : WT_FLAG_NO_FOLD);
        params[g].tile_o = r.tile_o;
      }
  });
}

wt_status wt_run(wt_pipeline *p, const wt_image *inputs, int32_t n_inputs, const wt_image *outputs,
                 int32_t n_outputs, void *stream) {
  return guard([&] {
    if (!p) wt::fail(WT_EINVAL, "null pipeline");
    if (!inputs || !outputs) wt::fail(WT_EINVAL, "null image array");
    std::lock_guard<std::mutex> lk(p->mu);
    wt::run(*p, inputs, n_inputs, outputs, n_outputs, (cudaStream_t)stream);
  });
}

namespace {

// Rows above (and below) an output row that the pipeline reads from its
// inputs, over every path of same-level taps (Sec. 2.3 footprints summed
// along the DAG); -1 when some stage is not at level 0.
int pipeline_row_halo(const wt::Pipeline &p) {
  const int n = (int)p.stages.size();
  for (const wt::Stage &st : p.stages)
    if (st.level != 0) return -1;
  std::vector<int> top(n, 0), bot(n, 0);
  int h = 0;
  for (int c = n - 1; c >= 0; c--)
    for (const wt::Edge &e : p.stages[c].edges) {
      if (e.mode != WT_TAP_SAME) return -1;
      const int t = top[c] + std::max(0, -e.dymin), b = bot[c] + std::max(0, e.dymax);
      if (e.producer >= 0) {
        top[e.producer] = std::max(top[e.producer], t);
        bot[e.producer] = std::max(bot[e.producer], b);
      } else {
        h = std::max(h, std::max(t, b));
      }
    }
  return h;
}

// Row bands of a banded host run: band b keeps output rows [y0, y1) and
// runs the pipeline on input rows [ys, ye), its rows and the pipeline's row
// halo.  ys is even, so a program reading the output row's parity
// (WT_OP_YPAR) sees the same parity in the band's sub-image as in the
// whole image.  Empty when the call runs the whole image at once: a stage
// off level 0, a multi-plane input, inputs and outputs of different
// heights, or an image too small to split.
struct HostBand {
  int y0, y1, ys, ye;
};

std::vector<HostBand> plan_host_bands(const wt::Pipeline &p, const wt_image *inputs, int n_in,
                                      const wt_image *outputs, int n_out) {
  const int h = pipeline_row_halo(p);
  if (h < 0) return {};
  const int H = inputs[0].height;
  for (int j = 0; j < n_in; j++)
    if (inputs[j].height != H || inputs[j].channels != 1) return {};
  for (int k = 0; k < n_out; k++)
    if (outputs[k].height != H) return {};
  // Up to 8 bands (pipeline fill and drain cost one band's copies), none
  // shorter than 64 rows or 4 halos, and none copying less than 8 MiB in
  // (every band adds copies, events and a launch of a short image; on a
  // GB300 the corner response at 4096^2 ran 6% faster end to end with 8
  // bands of 8 MiB than with 16 of 4 MiB, and at 2048^2 and 8192^2 no slower).
  int64_t in_bytes = 0;
  for (int j = 0; j < n_in; j++) in_bytes += image_bytes(inputs[j]);
  const int min_rows = std::max(64, 4 * h);
  const int kBands = (int)std::min<int64_t>({8, H / min_rows, in_bytes / (8 << 20)});
  if (kBands < 2) return {};
  const int rows = (H + kBands - 1) / kBands;
  std::vector<HostBand> bands;
  for (int y0 = 0; y0 < H; y0 += rows) {
    HostBand B;
    B.y0 = y0;
    B.y1 = std::min(H, y0 + rows);
    B.ys = std::max(0, y0 - h) & ~1;
    B.ye = std::min(H, B.y1 + h);
    bands.push_back(B);
  }
  return bands;
}

// wt_run_host in row bands for single-level pipelines: band b's input rows
// (with the pipeline's halo) are copied in on one stream while band b-1
// computes on a second and band b-2's output rows are copied out on a
// third.  A band runs the pipeline on its sub-image; clamp-to-edge at a
// band edge only changes rows within the halo of that edge, which the band
// does not keep (its neighbour computes them), so the result equals the
// whole-image run.  Returns false when the pipeline or the images do not
// qualify (then the caller runs the whole image at once).
bool run_host_banded(wt::Pipeline &p, const wt_image *inputs, int n_in, const wt_image *outputs, int n_out,
                     cudaStream_t user, wt::Workspace &w, const std::function<void *(int, const wt_image &)> &stage) {
  const std::vector<HostBand> plan = plan_host_bands(p, inputs, n_in, outputs, n_out);
  if (plan.empty()) return false;
  const int H = inputs[0].height;
  const int nb = (int)plan.size();
  for (int i = 0; i < 3; i++)
    if (!w.band_stream[i])
      wt::check_rt(cudaStreamCreateWithFlags(&w.band_stream[i], cudaStreamNonBlocking), "cudaStreamCreate");
  while ((int)w.band_events.size() < 3 * nb + 4) {
    cudaEvent_t e;
    wt::check_rt(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "cudaEventCreate");
    w.band_events.push_back(e);
  }
  cudaStream_t sin = w.band_stream[0], scomp = w.band_stream[1], sout = w.band_stream[2];
  cudaEvent_t *ev = w.band_events.data();
  // device copies: whole inputs; per output two band-sized scratch images
  // (allocated here, never while a graph is being captured)
  std::vector<wt_image> din(inputs, inputs + n_in);
  for (int j = 0; j < n_in; j++) din[j].data = stage(j, inputs[j]);
  int brows = 0;
  for (const HostBand &B : plan) brows = std::max(brows, B.ye - B.ys);
  std::vector<wt_image> scratch[2];
  for (int q = 0; q < 2; q++)
    for (int k = 0; k < n_out; k++) {
      wt_image sc = outputs[k];
      sc.height = brows;
      sc.data = stage(200 + 16 * q + k, sc);
      scratch[q].push_back(sc);
    }
  struct Band {
    int y0, y1, ys, ye;
    std::vector<wt_image> in, out;
  };
  std::vector<Band> bands;
  for (int b = 0; b < nb; b++) {
    Band B;
    B.y0 = plan[b].y0;
    B.y1 = plan[b].y1;
    B.ys = plan[b].ys;
    B.ye = plan[b].ye;
    B.in = din;
    B.out = scratch[b % 2];
    for (int j = 0; j < n_in; j++) {
      B.in[j].data = (char *)din[j].data + (int64_t)B.ys * din[j].pitch_bytes;
      B.in[j].height = B.ye - B.ys;
    }
    // (a row range of a one-plane input is itself an image; multi-plane
    // inputs were excluded)
    for (int k = 0; k < n_out; k++) B.out[k].height = B.ye - B.ys;
    bands.push_back(B);
  }
  // Work of one call, forked from and joined back to `origin`.
  auto submit = [&](cudaStream_t origin) {
    wt::check_rt(cudaEventRecord(ev[0], origin), "cudaEventRecord");
    for (int i = 0; i < 3; i++)
      if (w.band_stream[i] != origin)
        wt::check_rt(cudaStreamWaitEvent(w.band_stream[i], ev[0], 0), "cudaStreamWaitEvent");
    int copied = 0;  // input rows [0, copied) are on the device
    for (int b = 0; b < nb; b++) {
      const Band &B = bands[b];
      // copy in the rows this band needs that are not there yet
      if (B.ye > copied) {
        for (int j = 0; j < n_in; j++) {
          const int64_t off = copied * inputs[j].pitch_bytes;
          wt::check_rt(cudaMemcpyAsync((char *)din[j].data + off, (const char *)inputs[j].data + off,
                                       (size_t)((B.ye - copied) * inputs[j].pitch_bytes), cudaMemcpyHostToDevice,
                                       sin),
                       "cudaMemcpyAsync(H2D band)");
        }
        copied = B.ye;
      }
      cudaEvent_t in_done = ev[1 + 3 * b], comp_done = ev[2 + 3 * b], out_done = ev[3 + 3 * b];
      wt::check_rt(cudaEventRecord(in_done, sin), "cudaEventRecord");
      wt::check_rt(cudaStreamWaitEvent(scomp, in_done, 0), "cudaStreamWaitEvent");
      // the scratch this band writes was copied out two bands ago
      if (b >= 2) wt::check_rt(cudaStreamWaitEvent(scomp, ev[3 + 3 * (b - 2)], 0), "cudaStreamWaitEvent");
      wt::run(p, B.in.data(), n_in, B.out.data(), n_out, scomp);
      wt::check_rt(cudaEventRecord(comp_done, scomp), "cudaEventRecord");
      wt::check_rt(cudaStreamWaitEvent(sout, comp_done, 0), "cudaStreamWaitEvent");
      for (int k = 0; k < n_out; k++)
        for (int c = 0; c < outputs[k].channels; c++) {
          const int64_t hp = outputs[k].pitch_bytes * (int64_t)H;
          const int64_t sp = outputs[k].pitch_bytes * (int64_t)(B.ye - B.ys);
          wt::check_rt(
              cudaMemcpyAsync((char *)outputs[k].data + c * hp + (int64_t)B.y0 * outputs[k].pitch_bytes,
                              (const char *)B.out[k].data + c * sp + (int64_t)(B.y0 - B.ys) * outputs[k].pitch_bytes,
                              (size_t)((B.y1 - B.y0) * outputs[k].pitch_bytes), cudaMemcpyDeviceToHost, sout),
              "cudaMemcpyAsync(D2H band)");
        }
      wt::check_rt(cudaEventRecord(out_done, sout), "cudaEventRecord");
    }
    // join
    cudaEvent_t jc = ev[1 + 3 * nb], jo = ev[2 + 3 * nb];
    wt::check_rt(cudaEventRecord(jc, scomp), "cudaEventRecord");
    wt::check_rt(cudaEventRecord(jo, sout), "cudaEventRecord");
    wt::check_rt(cudaStreamWaitEvent(origin, jc, 0), "cudaStreamWaitEvent");
    wt::check_rt(cudaStreamWaitEvent(origin, jo, 0), "cudaStreamWaitEvent");
    if (origin != sin) {
      cudaEvent_t ji = ev[3 + 3 * nb];
      wt::check_rt(cudaEventRecord(ji, sin), "cudaEventRecord");
      wt::check_rt(cudaStreamWaitEvent(origin, ji, 0), "cudaStreamWaitEvent");
    }
  };
  // The same images again: replay the captured call (one launch instead of
  // some ten API calls per band); the second time: capture it.
  std::string key((const char *)inputs, sizeof(wt_image) * n_in);
  key.append((const char *)outputs, sizeof(wt_image) * n_out);
  key += "|" + std::to_string(p.sched_version) + "|" + std::to_string(w.generation);
  auto it = w.host_graphs.find(key);
  if (it != w.host_graphs.end() && it->second) {
    wt::check_rt(cudaGraphLaunch(it->second, user), "cudaGraphLaunch");
    wt::check_rt(cudaStreamSynchronize(user), "cudaStreamSynchronize");
    return true;
  }
  bool cached = true;  // every band's launches planned: nothing but launches to capture
  for (const Band &B : bands) cached = cached && wt::cached_run(p, B.in.data(), n_in, B.out.data(), n_out);
  if (it != w.host_graphs.end() && cached) {
    wt::check_rt(cudaStreamBeginCapture(sin, cudaStreamCaptureModeRelaxed), "cudaStreamBeginCapture");
    try {
      submit(sin);
    } catch (...) {
      cudaGraph_t g = nullptr;
      cudaStreamEndCapture(sin, &g);
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      throw;
    }
    cudaGraph_t g = nullptr;
    wt::check_rt(cudaStreamEndCapture(sin, &g), "cudaStreamEndCapture");
    cudaGraphExec_t ex = nullptr;
    const cudaError_t ie = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    wt::check_rt(ie, "cudaGraphInstantiate");
    it->second = ex;
    wt::check_rt(cudaGraphLaunch(ex, user), "cudaGraphLaunch");
    wt::check_rt(cudaStreamSynchronize(user), "cudaStreamSynchronize");
    return true;
  }
  submit(user);
  wt::check_rt(cudaStreamSynchronize(user), "cudaStreamSynchronize");
  if (w.host_graphs.size() >= 64) w.clear_host_graphs();
  w.host_graphs.emplace(key, nullptr);
  return true;
}

}  // namespace

wt_status wt_run_host(wt_pipeline *p, const wt_image *inputs, int32_t n_inputs, const wt_image *outputs,
                      int32_t n_outputs, void *stream) {
  return guard([&] {
    if (!p) wt::fail(WT_EINVAL, "null pipeline");
    if (!inputs || !outputs || n_inputs < 1 || n_outputs < 1 || n_inputs > 16 || n_outputs > 16)
      wt::fail(WT_EINVAL, "bad image arrays");
    std::lock_guard<std::mutex> lk(p->mu);
    cudaStream_t st = (cudaStream_t)stream;
    wt::Workspace &w = wt::workspace(*p, 0);
    std::vector<wt_image> din(inputs, inputs + n_inputs), dout(outputs, outputs + n_outputs);
    auto stage = [&](int key, const wt_image &h) -> void * {
      int64_t need = image_bytes(h);
      wt::Staging &s = w.staging[key];
      if (s.bytes < need) {
        w.clear_host_graphs();  // captured calls use the old buffers
        if (s.ptr) {
          wt::check_rt(cudaStreamSynchronize(st), "cudaStreamSynchronize");
          wt::dev_free(s.ptr, (size_t)s.bytes);
          s.ptr = nullptr;
          s.bytes = 0;
        }
        if (wt::dev_alloc(&s.ptr, (size_t)need) != cudaSuccess) {
          cudaGetLastError();
          wt::fail(WT_ENOMEM, "cannot allocate staging buffer");
        }
        s.bytes = need;
      }
      return s.ptr;
    };
    for (int j = 0; j < n_inputs; j++)
      if (!inputs[j].data) wt::fail(WT_EINVAL, "null host input");
    for (int k = 0; k < n_outputs; k++)
      if (!outputs[k].data) wt::fail(WT_EINVAL, "null host output");
    if (run_host_banded(*p, inputs, n_inputs, outputs, n_outputs, st, w, stage)) return;
    for (int j = 0; j < n_inputs; j++) {
      din[j].data = stage(j, inputs[j]);
      wt::check_rt(cudaMemcpyAsync(din[j].data, inputs[j].data, (size_t)image_bytes(inputs[j]),
                                   cudaMemcpyHostToDevice, st),
                   "cudaMemcpyAsync(H2D)");
    }
    for (int k = 0; k < n_outputs; k++) {
      if (!outputs[k].data) wt::fail(WT_EINVAL, "null host output");
      dout[k].data = stage(100 + k, outputs[k]);
    }
    wt::run(*p, din.data(), n_inputs, dout.data(), n_outputs, st);
    for (int k = 0; k < n_outputs; k++)
      wt::check_rt(cudaMemcpyAsync(outputs[k].data, dout[k].data, (size_t)image_bytes(outputs[k]),
                                   cudaMemcpyDeviceToHost, st),
                   "cudaMemcpyAsync(D2H)");
    wt::check_rt(cudaStreamSynchronize(st), "cudaStreamSynchronize");
  });
}

wt_status wt_run_batch(wt_pipeline *p, const wt_image *inputs, const wt_image *outputs, int32_t n_images,
                       void *stream) {
  return guard([&] {
    if (!p) wt::fail(WT_EINVAL, "null pipeline");
    if (!inputs || !outputs || n_images < 1) wt::fail(WT_EINVAL, "bad batch");
    std::lock_guard<std::mutex> lk(p->mu);
    wt::run_batch(*p, inputs, outputs, n_images, (cudaStream_t)stream);
  });
}

wt_status wt_schedule_time(wt_pipeline *p, const wt_image *inputs, int32_t n_inputs, const wt_image *outputs,
                           int32_t n_outputs, int32_t n_images, int32_t reps, void *stream, double *ms) {
  return guard([&] {
    if (!p || !inputs || !outputs || !ms || n_images < 0 || reps < 1) wt::fail(WT_EINVAL, "bad arguments");
    std::lock_guard<std::mutex> lk(p->mu);
    *ms = wt::time_installed(*p, inputs, n_inputs, outputs, n_outputs, n_images, (cudaStream_t)stream, reps);
    if (!std::isfinite(*ms)) wt::fail(WT_EDEVICE, "a timed run raised the device error word");
  });
}

wt_status wt_schedule_tune(wt_pipeline *p, const wt_image *inputs, int32_t n_inputs, const wt_image *outputs,
                           int32_t n_outputs, int32_t n_images, int32_t max_variants, int32_t reps, void *stream,
                           double *best_ms, int32_t *n_timed) {
  return guard([&] {
    if (!p || !inputs || !outputs || n_images < 0) wt::fail(WT_EINVAL, "bad arguments");
    std::lock_guard<std::mutex> lk(p->mu);
    const wt::Schedule user = p->sched;
    try {
      wt::TuneResult r = wt::tune(*p, inputs, n_inputs, outputs, n_outputs, n_images, max_variants, reps,
                                  (cudaStream_t)stream);
      if (best_ms) *best_ms = r.best_ms;
      if (n_timed) *n_timed = r.timed;
    } catch (...) {
      p->sched = user;
      p->sched_version++;
      throw;
    }
  });
}

wt_status wt_prepare(wt_pipeline *p, const wt_schedule_desc *descs, int32_t n_descs, const wt_image *inputs,
                     int32_t n_inputs, const wt_image *outputs, int32_t n_outputs, int32_t batched) {
  return guard([&] {
    if (!p || (n_descs > 0 && !descs) || n_descs < 0 || !inputs || !outputs) wt::fail(WT_EINVAL, "bad arguments");
    std::lock_guard<std::mutex> lk(p->mu);
    std::vector<wt::Schedule> c;
    for (int i = 0; i < n_descs; i++) c.push_back(to_schedule(*p, &descs[i]));
    wt::precompile(*p, c, inputs, n_inputs, outputs, n_outputs, batched != 0);
  });
}

wt_status wt_check(wt_pipeline *p, void *stream) {
  wt_status st = WT_OK;
  wt_status rc = guard([&] {
    if (!p) wt::fail(WT_EINVAL, "null pipeline");
    wt::check_rt(cudaStreamSynchronize((cudaStream_t)stream), "cudaStreamSynchronize");
    // the workspace's error word (wt_run, wt_run_batch, wt_run_host) and,
    // after wt_run_static on this device, the static scratch's status word
    int dev = 0;
    wt::check_rt(cudaGetDevice(&dev), "cudaGetDevice");
    int32_t *words[2] = {p->ws ? p->ws->err : nullptr,
                         dev < 64 && (p->static_devs >> dev & 1) ? wt::static_status_word(dev) : nullptr};
    for (int32_t *w : words) {
      if (!w) continue;
      int32_t v = 0;
      wt::check_rt(cudaMemcpy(&v, w, sizeof v, cudaMemcpyDeviceToHost), "cudaMemcpy(error word)");
      if (v != 0) {
        wt::check_rt(cudaMemset(w, 0, sizeof v), "cudaMemset");
        if (st == WT_OK) st = v == 1 ? WT_ETIMEOUT : WT_EDEVICE;
      }
    }
  });
  if (rc != WT_OK) return rc;
  if (st != WT_OK) g_err = st == WT_ETIMEOUT ? "a device-side bounded wait gave up" : "device-side check failed";
  return st;
}

int32_t wt_launches_per_run(const wt_pipeline *p) {
  if (!p) return -1;
  int32_t n = 0;
  wt_status rc = guard([&] {
    auto groups = wt::schedule_groups(*p);
    for (size_t gi = 0; gi < groups.size(); gi++) {
      const wt::GroupParams gp = wt::group_params(*p, (int)gi);
      bool zgroup = false;
      for (int s : groups[gi]) zgroup = zgroup || p->stages[s].has_z;
      bool fused = p->sched.exec == WT_EXEC_FUSED && !gp.plain &&
                   (zgroup ? wt::vol_analyze(*p, groups[gi], gp.zstream, gp.tile_o > 0 ? gp.tile_o : 4,
                                             std::max(1, gp.tile_h), gp.vec > 0 ? gp.vec : 2, gp.frac_reg < 1.f,
                                             gp.n_buffers).ok
                           : ((!gp.otptb && wt::chain_form(*p, groups[gi]).ok) ||
                              wt::analyze_group(*p, groups[gi], 4, 1.f, 4).fusable));
      const std::vector<wt::CascadeUnit> cu =
          p->sched.exec == WT_EXEC_FUSED && !gp.plain && !gp.otptb && !zgroup && !wt::chain_form(*p, groups[gi]).ok
              ? wt::cascade_units(*p, groups[gi])
              : std::vector<wt::CascadeUnit>();
      if (!cu.empty()) {
        for (const wt::CascadeUnit &u : cu)
          if (u.s2 >= 0 || !p->consumers[u.s1].empty() || p->is_output[u.s1]) n++;
      } else if (fused) {
        n++;
      } else {
        for (int s : groups[gi])
          if (!p->consumers[s].empty() || p->is_output[s]) n++;
      }
    }
  });
  return rc == WT_OK ? n : -1;
}

// ------------------------------------------------------------- debug API

int64_t wt_debug_args_size(void) { return (int64_t)sizeof(wt::KernelArgs); }

wt_status wt_debug_kernel_ws(wt_pipeline *p, int32_t launch_index, const wt_image *inputs, int32_t n_inputs,
                             const wt_image *outputs, int32_t n_outputs, void *workspace, int64_t ws_cap,
                             char *src, int64_t src_cap, int64_t *src_len, void *args, int64_t args_cap,
                             int32_t *launch, char *kname, int64_t kname_cap, int64_t *ws_bytes) {
  return guard([&] {
    if (!p) wt::fail(WT_EINVAL, "null pipeline");
    std::lock_guard<std::mutex> lk(p->mu);
    wt::RunPlan plan = wt::build_plan(*p, inputs, n_inputs, outputs, n_outputs);
    if (launch_index < 0 || launch_index >= (int)plan.launches.size()) wt::fail(WT_EINVAL, "launch index");
    const wt::Launch &L = plan.launches[launch_index];
    if (ws_bytes) *ws_bytes = plan.ws_bytes;
    if (workspace && ws_cap < plan.ws_bytes) wt::fail(WT_EINVAL, "workspace buffer too small");
    std::string s = wt::launch_source(*p, L);
    if (src_len) *src_len = (int64_t)s.size();
    if (src && src_cap > 0) {
      size_t n = std::min((size_t)src_cap - 1, s.size());
      memcpy(src, s.data(), n);
      src[n] = 0;
    }
    wt::KernelArgs a;
    // the argument block (with the caller's workspace when asked for it;
    // otherwise any base: only the tile counts are used)
    static char no_ws;
    wt::fill_args(*p, plan, L, args || workspace ? (char *)workspace : &no_ws, a, false);
    unsigned gx = L.grid[0];
    // as on the GPU with few resident warps: exercises both tile heights
    if (L.fused && !L.key.otptb) {
      wt::split_tiles(L, a, 4 * L.key.nw);
      a.direct = L.params.tile_queue ? 0 : 1;
      if (a.direct) gx = (unsigned)((a.n_tiles + L.key.nw - 1) / L.key.nw);
    }
    if (args) {
      if (args_cap < (int64_t)sizeof(wt::KernelArgs)) wt::fail(WT_EINVAL, "args buffer too small");
      memcpy(args, &a, sizeof a);
    }
    if (launch) {
      launch[0] = (int32_t)gx;
      launch[1] = (int32_t)L.grid[1];
      launch[2] = (int32_t)L.grid[2];
      launch[3] = L.block;
      launch[4] = L.smem;
      launch[5] = L.fused ? 1 : 0;
      launch[6] = (int32_t)plan.launches.size();
      launch[7] = L.fused ? L.geom.unroll : 0;
    }
    if (kname && kname_cap > 0) {
      size_t n = std::min((size_t)kname_cap - 1, L.kname.size());
      memcpy(kname, L.kname.data(), n);
      kname[n] = 0;
    }
  });
}

wt_status wt_debug_kernel(wt_pipeline *p, int32_t launch_index, const wt_image *inputs, int32_t n_inputs,
                          const wt_image *outputs, int32_t n_outputs, char *src, int64_t src_cap,
                          int64_t *src_len, void *args, int64_t args_cap, int32_t *launch, char *kname,
                          int64_t kname_cap) {
  return wt_debug_kernel_ws(p, launch_index, inputs, n_inputs, outputs, n_outputs, nullptr, 0, src, src_cap,
                            src_len, args, args_cap, launch, kname, kname_cap, nullptr);
}

wt_status wt_debug_batch(wt_pipeline *p, int32_t launch_index, const wt_image *inputs, const wt_image *outputs,
                         int32_t n_images, char *src, int64_t src_cap, int64_t *src_len, void *args,
                         void *img_tab, int64_t img_tab_cap, int32_t *tiles, int64_t tiles_cap,
                         int64_t *n_tiles, int32_t *launch, char *kname, int64_t kname_cap) {
  return guard([&] {
    if (!p) wt::fail(WT_EINVAL, "null pipeline");
    if (!inputs || !outputs || n_images < 1) wt::fail(WT_EINVAL, "bad batch");
    std::lock_guard<std::mutex> lk(p->mu);
    wt::BatchPlan b = wt::build_batch(*p, inputs, outputs, n_images);
    if (launch_index < 0 || launch_index >= (int)b.launches.size()) wt::fail(WT_EINVAL, "launch index");
    const wt::Launch &L = b.launches[launch_index];
    const std::vector<int32_t> &t = b.tiles[launch_index];
    if (n_tiles) *n_tiles = (int64_t)t.size() / 4;
    if (src_len || src) {
      std::string s = wt::launch_source(*p, L);
      if (src_len) *src_len = (int64_t)s.size();
      if (src && src_cap > 0) {
        size_t n = std::min((size_t)src_cap - 1, s.size());
        memcpy(src, s.data(), n);
        src[n] = 0;
      }
    }
    if (img_tab) {
      if (img_tab_cap < (int64_t)n_images * (int64_t)sizeof(wt::KernelArgs)) wt::fail(WT_EINVAL, "img_tab too small");
      for (int i = 0; i < n_images; i++) {
        wt::KernelArgs a = wt::batch_image_args(*p, b, launch_index, i, nullptr, false);
        memcpy((char *)img_tab + (size_t)i * sizeof a, &a, sizeof a);
      }
    }
    if (tiles) {
      if (tiles_cap < (int64_t)t.size()) wt::fail(WT_EINVAL, "tile buffer too small");
      memcpy(tiles, t.data(), t.size() * 4);
    }
    if (args) {
      wt::KernelArgs a;
      memset(&a, 0, sizeof a);
      a.n_tiles = L.n_tiles;
      a.n_images = n_images;
      memcpy(args, &a, sizeof a);
    }
    if (launch) {
      launch[0] = (int32_t)L.grid[0];
      launch[1] = 1;
      launch[2] = 1;
      launch[3] = L.block;
      launch[4] = L.smem;
      launch[5] = 1;
      launch[6] = (int32_t)b.launches.size();
      launch[7] = L.geom.unroll;
    }
    if (kname && kname_cap > 0) {
      size_t n = std::min((size_t)kname_cap - 1, L.kname.size());
      memcpy(kname, L.kname.data(), n);
      kname[n] = 0;
    }
  });
}

wt_status wt_debug_compile(wt_pipeline *p, int32_t launch_index, const wt_image *inputs, int32_t n_inputs,
                           const wt_image *outputs, int32_t n_outputs, int64_t *cubin_bytes) {
  return guard([&] {
    if (!p) wt::fail(WT_EINVAL, "null pipeline");
    std::lock_guard<std::mutex> lk(p->mu);
    wt::RunPlan plan = wt::build_plan(*p, inputs, n_inputs, outputs, n_outputs);
    if (launch_index < 0 || launch_index >= (int)plan.launches.size()) wt::fail(WT_EINVAL, "launch index");
    const wt::Launch &L = plan.launches[launch_index];
    std::string cubin = wt::compile_cubin(wt::launch_source(*p, L), L.kname, L.key.max_regs);
    if (cubin_bytes) *cubin_bytes = (int64_t)cubin.size();
  });
}

wt_status wt_debug_layout(wt_pipeline *p, int32_t launch_index, const wt_image *inputs, int32_t n_inputs,
                          const wt_image *outputs, int32_t n_outputs, int32_t *out, int32_t cap, int32_t *n_out) {
  return guard([&] {
    if (!p) wt::fail(WT_EINVAL, "null pipeline");
    std::lock_guard<std::mutex> lk(p->mu);
    wt::RunPlan plan = wt::build_plan(*p, inputs, n_inputs, outputs, n_outputs);
    if (launch_index < 0 || launch_index >= (int)plan.launches.size()) wt::fail(WT_EINVAL, "launch index");
    const wt::Launch &L = plan.launches[launch_index];
    if (!L.fused || L.key.otptb) wt::fail(WT_EINVAL, "not a warp-tiled group launch");
    const wt::FusedLayout &F = L.layout;
    std::vector<int32_t> v = {F.warp_bytes, F.bar_off, F.chunk, F.nbuf, F.V, F.out_w, (int32_t)F.boxw.size()};
    for (size_t s = 0; s < F.boxw.size(); s++) {
      v.push_back(F.ring_off[s]);
      v.push_back(F.bufb[s]);
      v.push_back(F.boxw[s]);
      v.push_back(F.esz[s]);
    }
    if (n_out) *n_out = (int32_t)v.size();
    if (out)
      for (int i = 0; i < (int)v.size() && i < cap; i++) out[i] = v[i];
  });
}

wt_status wt_debug_lanes(wt_pipeline *p, const wt_image *inputs, int32_t n_inputs, const wt_image *outputs,
                         int32_t n_outputs, int32_t *out, int32_t cap, int32_t *n_out) {
  return guard([&] {
    if (!p) wt::fail(WT_EINVAL, "null pipeline");
    std::lock_guard<std::mutex> lk(p->mu);
    wt::RunPlan plan = wt::build_plan(*p, inputs, n_inputs, outputs, n_outputs);
    std::vector<int32_t> v = {(int32_t)plan.launches.size(), plan.n_lanes};
    for (const wt::Launch &L : plan.launches) {
      v.push_back(L.lane);
      v.push_back((int32_t)L.waits.size());
      v.insert(v.end(), L.waits.begin(), L.waits.end());
      v.push_back((int32_t)L.stages.size());
      v.insert(v.end(), L.stages.begin(), L.stages.end());
    }
    if (n_out) *n_out = (int32_t)v.size();
    if (out)
      for (int i = 0; i < (int)v.size() && i < cap; i++) out[i] = v[i];
  });
}

wt_status wt_debug_host_bands(wt_pipeline *p, const wt_image *inputs, int32_t n_inputs, const wt_image *outputs,
                              int32_t n_outputs, int32_t *bands, int32_t cap, int32_t *n_bands) {
  return guard([&] {
    if (!p) wt::fail(WT_EINVAL, "null pipeline");
    if (!inputs || !outputs || n_inputs < 1 || n_outputs < 1 || n_inputs > 16 || n_outputs > 16)
      wt::fail(WT_EINVAL, "bad image arrays");
    std::lock_guard<std::mutex> lk(p->mu);
    const std::vector<HostBand> plan = plan_host_bands(*p, inputs, n_inputs, outputs, n_outputs);
    if (n_bands) *n_bands = (int32_t)plan.size();
    if (bands)
      for (int b = 0; b < (int)plan.size() && b < cap; b++) {
        bands[4 * b] = plan[b].y0;
        bands[4 * b + 1] = plan[b].y1;
        bands[4 * b + 2] = plan[b].ys;
        bands[4 * b + 3] = plan[b].ye;
      }
  });
}

wt_status wt_debug_segment_cost(wt_pipeline *p, int32_t first, int32_t n, int32_t width, int32_t height,
                                int32_t dtype, double *cost, int32_t *fused) {
  return guard([&] {
    if (!p || !cost) wt::fail(WT_EINVAL, "null argument");
    if (first < 0 || n < 1 || n > wt::kMaxGroupStages || first + n > (int)p->stages.size())
      wt::fail(WT_EINVAL, "stage range");
    if (width < 1 || height < 1) wt::fail(WT_EINVAL, "bad size");
    if (dtype < WT_F32 || dtype > WT_BF16) wt::fail(WT_EINVAL, "bad dtype");
    std::lock_guard<std::mutex> lk(p->mu);
    const wt::SegmentChoice c = wt::auto_segment(*p, first, n, width, height, dtype);
    *cost = c.cost;
    if (fused) *fused = c.fused ? 1 : 0;
  });
}

wt_status wt_debug_group_geometry(wt_pipeline *p, int32_t group, int32_t vec, float frac_reg, int32_t *out,
                                  int32_t cap, int32_t *n_out) {
  return guard([&] {
    if (!p) wt::fail(WT_EINVAL, "null pipeline");
    auto groups = wt::schedule_groups(*p);
    if (group < 0 || group >= (int)groups.size()) wt::fail(WT_EINVAL, "group index");
    wt::GroupGeom g = wt::analyze_group(*p, groups[group], vec, frac_reg, 4);
    std::vector<int32_t> v = {g.fusable ? 1 : 0, g.halo_l, g.halo_r, g.halo_t, g.halo_b, g.unroll,
                              (int32_t)g.nodes.size()};
    for (const wt::Node &n : g.nodes) {
      int32_t rec[10] = {n.id, n.src_chan, n.is_source, n.is_liveout, n.top, n.bot, n.delay, n.window,
                         n.xl * 1000 + n.xr, n.in_smem};
      v.insert(v.end(), rec, rec + 10);
    }
    if (n_out) *n_out = (int32_t)v.size();
    if (out)
      for (int i = 0; i < (int)v.size() && i < cap; i++) out[i] = v[i];
  });
}

wt_status wt_debug_inject_alloc_failure(int32_t kind, int32_t after) {
  return guard([&] {
    if (kind != wt::kAllocHost && kind != wt::kAllocDevice) wt::fail(WT_EINVAL, "kind must be 0 or 1");
    wt::inject_alloc_failure(kind, after);
  });
}

wt_status wt_debug_live_objects(int64_t *pipelines, int64_t *device_bytes) {
  return guard([&] {
    long long a = 0, b = 0;
    wt::live_objects(&a, &b);
    if (pipelines) *pipelines = a;
    if (device_bytes) *device_bytes = b;
  });
}

}  // extern "C"

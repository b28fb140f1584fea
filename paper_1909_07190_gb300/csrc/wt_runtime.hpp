// Run plans and launches (runtime.cpp).
#pragma once

#include <cuda_runtime.h>

#include "wt_internal.hpp"

namespace wt {

// Where a stage's (or input's) values live in HBM.
struct Loc {
  const void *ptr = nullptr;
  int64_t pitch = 0, plane = 0;
  int W = 0, H = 0, C = 0, dtype = WT_F32;
  bool user = false;     // caller's output image
  bool ws = false;       // lives in the workspace at ws_off
  int64_t ws_off = 0, ws_bytes = 0;
};

struct Launch {
  bool fused = true;
  std::vector<int> stages;
  GroupParams params;
  GroupGeom geom;
  FusedLayout layout;
  CodegenKey key;
  VolGeom vol;  // 3-D group (key.vol)
  std::string kname;
  std::vector<int> src, src_chan, dst;
  int n_ring = 0;  // staged (TMA) sources: src[0, n_ring); gather sources after
  int W = 0, H = 0;
  int tiles_x = 0, tiles_y = 0, n_tiles = 0;
  unsigned grid[3] = {1, 1, 1};
  int block = 128;
  int smem = 0;
  int resident_blocks_per_sm = 0;
  int resident_warps = 0;  // fused launches: resident warps on the device
  // Stream lane (0: the caller's stream), the earlier launches on other
  // lanes it waits for, and whether an event is recorded after it (another
  // lane waits for it, or it ends a side lane).
  int lane = 0;
  std::vector<int> waits;
  bool record = false;
};

// Most stream lanes a run uses: the caller's stream and three side streams.
constexpr int kMaxLanes = 4;

struct RunPlan {
  int W = 0, H = 0;
  int mid_dtype = WT_F32;
  std::vector<Loc> loc;     // per stage
  std::vector<Loc> in_loc;  // per pipeline input
  std::vector<Launch> launches;
  int64_t ws_bytes = 0;
  int n_lanes = 1;
};

// Lanes of a plan's launches: a launch that reads no stage an earlier launch
// writes may run beside it.  Greedy in plan order: a launch continues the
// lane whose last launch it depends on, else opens a new lane (at most
// kMaxLanes), else joins the lane idle longest; it waits by event for its
// dependencies on other lanes.  Stages never share workspace memory, so
// reads after writes are the only hazards within a run.
void assign_lanes(RunPlan &plan);

// Device control block of a workspace: the error word at byte 0 and, from
// kCtrlQueueOffset, two tile-queue counters per launch (next tile, warps
// finished) that the last warp of each launch resets to zero.
constexpr int kCtrlBytes = 4096;
constexpr int kCtrlQueueOffset = 64;
constexpr int kMaxLaunches = (kCtrlBytes - kCtrlQueueOffset) / 8;
int32_t *queue_counters(int32_t *ctrl, int launch_index);
void split_tiles(const Launch &L, KernelArgs &a, int resident_warps);

struct Staging {
  void *ptr = nullptr;
  int64_t bytes = 0;
};

struct Workspace {
  int device = -1;
  char *base = nullptr;
  int64_t bytes = 0;
  int32_t *err = nullptr;
  uint64_t generation = 1;         // bumped when `base` is reallocated
  std::map<int, Staging> staging;  // wt_run_host device copies
  // wt_run_host row bands: copy-in, compute and copy-out streams, and
  // events (created on first use)
  cudaStream_t band_stream[3] = {nullptr, nullptr, nullptr};
  std::vector<cudaEvent_t> band_events;
  // side streams of concurrent launch lanes (lanes 1..), the fork event and
  // one event per launch of a run (created by the first run that needs them)
  cudaStream_t lane_stream[kMaxLanes - 1] = {};
  cudaEvent_t fork_event = nullptr;
  std::vector<cudaEvent_t> launch_events;
  // banded host runs captured as CUDA graphs, by image descriptors (null:
  // seen once, captured at the next call)
  std::map<std::string, cudaGraphExec_t> host_graphs;
  void clear_host_graphs();
  ~Workspace();
};

std::vector<std::vector<int>> schedule_groups(const Pipeline &p);
GroupParams group_params(const Pipeline &p, int gi);
// batched: one image of a batch (tile heights are not shortened for small
// images: the batch's tiles share the resident warps)
RunPlan build_plan(Pipeline &p, const wt_image *in, int n_in, const wt_image *out, int n_out,
                   bool batched = false);
std::string launch_source(const Pipeline &p, const Launch &L);
// Entry-point name of a generated kernel (a hash of the pipeline, the
// codegen key and the generator version).
std::string kernel_name(const Pipeline &p, const CodegenKey &key, bool fused, bool gather = false);
void fill_args(const Pipeline &p, const RunPlan &plan, const Launch &L, char *ws, KernelArgs &a,
               bool encode_tmaps);
Kernel &get_kernel(const Pipeline &p, const Launch &L, int device);
// The loaded kernel of a launch, or null (never compiles or loads).
Kernel *find_kernel(const Pipeline &p, const Launch &L, int device);
void set_last_error(const std::string &msg);
void launch(const Launch &L, Kernel &k, KernelArgs &a, cudaStream_t stream);
// Per-launch set-up shared by every path that launches a plan (grid of the
// persistent kernels, tensor maps, tile split, status word, queue counters).
KernelArgs launch_args(Pipeline &p, const RunPlan &plan, Launch &L, Kernel &k, char *ws, int32_t *err, int li,
                       int dev);
Workspace &workspace(Pipeline &p, int64_t bytes);
// Status word of wt_run_static's scratch on device `dev` (noalloc.cu), or
// null if no wt_run_static call has set it up there.
int32_t *static_status_word(int dev);
void run_plan(Pipeline &p, RunPlan &plan, cudaStream_t stream, const std::string *cache_key = nullptr);
// The cached launches of an earlier run with these images, or null.
const CachedRun *cached_run(const Pipeline &p, const wt_image *in, int n_in, const wt_image *out, int n_out);
// wt_run: reuses the cached launches when schedule and images are unchanged.
void run(Pipeline &p, const wt_image *in, int n_in, const wt_image *out, int n_out, cudaStream_t stream);

// Batched runs (batch.cpp): per-image plans (same kernels), each image's
// slice of the workspace, and per group the persistent launch with its tile
// list (4 ints per tile: image, tile column, tile row, channel).
struct BatchPlan {
  std::vector<RunPlan> img;
  std::vector<int64_t> ws_off;
  int64_t ws_bytes = 0;
  std::vector<Launch> launches;
  std::vector<std::vector<int32_t>> tiles;
};
BatchPlan build_batch(Pipeline &p, const wt_image *in, const wt_image *out, int n);
KernelArgs batch_image_args(const Pipeline &p, const BatchPlan &b, int l, int i, char *ws, bool encode_tmaps);
void run_batch(Pipeline &p, const wt_image *in, const wt_image *out, int n_images, cudaStream_t stream);

}  // namespace wt

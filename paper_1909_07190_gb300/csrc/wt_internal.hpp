// Internal types of the warp-tiled pipeline library (host side).
#pragma once

#include <array>
#include <cstdint>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "wt.h"

namespace wt {

// Tap modes (wt_tapmode): 0 same level; 2s - 1 down by 2^s (producer s
// levels finer, P(2^s x + dx)); 2s up by 2^s (producer s levels coarser,
// P(floor(x / 2^s) + dx)).
inline int tap_shift(int mode) { return (mode + 1) / 2; }
inline bool tap_is_down(int mode) { return mode > 0 && (mode & 1); }
inline bool tap_is_up(int mode) { return mode > 0 && !(mode & 1); }
inline int tap_level_delta(int mode) { return tap_is_down(mode) ? tap_shift(mode) : -tap_shift(mode); }

constexpr int kMaxSrc = 8;     // TMA-staged sources per group kernel
constexpr int kMaxAllSrc = 24; // all external sources (staged and gathered)
constexpr int kMaxDst = 8;     // liveouts per group kernel
constexpr int kMaxOps = 256;   // ops per stage program
constexpr int kMaxStack = 32;  // postfix stack depth

// Thrown inside the library, converted to a wt_status at the C boundary.
struct Error {
  wt_status code;
  std::string msg;
};
[[noreturn]] void fail(wt_status code, const std::string &msg);

// Tile height single-image runs use for requested height T on a level of
// height H with tiles_x tile columns (runtime.cpp).
struct GroupGeom;
// Steps of a warp tile beyond its output rows (codegen.cpp).
int stream_extra_steps(const GroupGeom &g);
int effective_tile_h(int T, int H, int tiles_x, int channels, const GroupGeom &g);

// Allocation points (runtime.cpp).  A test can make the n-th allocation of
// one kind fail (wt_debug_inject_alloc_failure): host points throw
// std::bad_alloc (WT_ENOMEM at the C boundary), device allocations go
// through dev_alloc/dev_free, which also count the device bytes the
// library holds.
constexpr int kAllocHost = 0, kAllocDevice = 1;
void host_alloc_point();
int dev_alloc(void **ptr, size_t bytes);  // cudaError_t
void dev_free(void *ptr, size_t bytes);
// Live pipelines (a count kept for leak tests).
struct LiveCounter {
  LiveCounter();
  ~LiveCounter();
  LiveCounter(const LiveCounter &) = delete;
  LiveCounter &operator=(const LiveCounter &) = delete;
};

struct Op {
  int op = 0, slot = 0, dx = 0, dy = 0, chan = -1, mode = 0;
  float value = 0.f;
};

// Footprint of one producer as read by one consumer (Sec. 2.3: the set of
// dependence vectors, summarised as a box per tap mode).
struct Edge {
  int producer = 0;  // stage id or -(j+1)
  int mode = 0;      // wt_tapmode (one mode per edge; checked)
  int dxmin = 0, dxmax = 0, dymin = 0, dymax = 0;
  std::vector<int> chans;  // distinct channel specs used (-1 or fixed)
  bool zrel = false;       // some tap is a plane-offset (3-D) tap
  int dzmin = 0, dzmax = 0;
};

struct Stage {
  int channels = 1;
  std::vector<int> inputs;
  std::vector<Op> ops;
  // derived
  int level = 0;
  std::vector<Edge> edges;  // one per input slot that is tapped
  bool has_z = false;       // a plane-offset (WT_OP_TAPZ) tap in its program
};

struct GroupParams {
  int tile_h = 40;
  int warps_per_block = 1;
  float frac_reg = 1.f;
  int vec = 0;
  int max_regs = 0;
  int chunk_rows = 8;
  int n_buffers = 2;
  int tile_split = 1;  // short tiles for the last round of the tile queue
  int pairs = 1;       // packed f32x2 arithmetic where taps align
  int plain = 0;       // run the group's stages as per-stage kernels
  int smem16 = 0;      // shared-memory windows in the 16-bit storage type
  int otptb = 0;       // one overlapped tile per thread block (the baseline
                       // tiling the paper compares against)
  int tile_o = 0;      // 3-D groups: planes (rows when streaming planes) per tile
  int zstream = 0;     // 3-D groups: stream along planes instead of rows
  int test_stall = 0;  // test only: every tile's first staging wait gives up
  int tile_queue = 0;  // persistent warps pull tiles from a device queue
  int fold = 1;        // deferred constant scales in warp-tile groups
  int one_stream = 0;  // the run's launches in plan order on the caller's stream
};

struct Schedule {
  int exec = WT_EXEC_FUSED;
  std::vector<int> group_of_stage;
  std::vector<GroupParams> params;
  int n_groups = 0;
  int intermediate_dtype = -1;
  bool installed = false;
  double predicted_cost = 0;  // model cost of the schedule (auto schedules)
};

// Geometry of one fused group (Sec. 4 OTPW and Sec. 5 hybrid tiling, in the
// streaming form used here: split dimension y, one lane row per warp).
// One op of a kernel node's postfix program; taps name kernel nodes.
struct KOp {
  int op = 0;
  int node = -1;  // WT_OP_TAP: producer node index
  int dx = 0, dy = 0;
  float value = 0.f;
};

struct Node {
  int id = 0;             // stage id, or -(j+1) for a pipeline input
  bool synthetic = false; // row pass of a split separable stencil (no stage)
  std::vector<KOp> prog;  // stages and synthetic nodes: program over nodes
  int src_chan = -1;      // sources: channel spec (-1 = tile channel)
  bool is_source = false; // read from memory (pipeline input or earlier group)
  bool is_liveout = false;
  int channels = 1;
  int top = 0, bot = 0;   // rows needed above/below the output rows
  int left = 0, right = 0;// columns needed left/right of the output columns
  int delay = 0;          // e_n: stage n computes row y_top + k - e_n at step k
  int window = 1;         // rows kept (rotation window)
  int xl = 0, xr = 0;     // extra columns each lane needs from its neighbours
  bool in_smem = false;   // window lives in shared memory (else registers)
  bool rotate = true;     // rotating slot names (window divides unroll)
  int src_index = -1;     // sources: index into the kernel's source table
  int dst_index = -1;     // liveouts: index into the kernel's dst table
  // Gather source: a producer outside the group read through a down- or
  // up-sampling tap (another level).  It has no window and is not staged:
  // each tap loads the clamped pixel it names from memory.
  int gather_mode = 0;    // WT_TAP_DOWN2 / WT_TAP_UP2, 0 = not a gather source
};

struct NodeEdge {
  int c = 0, p = 0;  // consumer and producer node
  int dxmin = 0, dxmax = 0, dymin = 0, dymax = 0;
};

struct GroupGeom {
  std::vector<int> stages;     // stage ids (topological)
  std::vector<Node> nodes;     // stable indices: sources, stages, synthetic
  std::vector<int> order;      // evaluation order (sources first)
  std::vector<NodeEdge> edges;
  int n_split = 0;             // separable stencils split into two passes
  std::vector<int> liveouts;   // stage ids
  bool fusable = true;         // else: per-stage kernel
  std::string why_not;         // reason when !fusable
  int level = 0;
  int channels = 1;            // tile channels (max over stages)
  int halo_l = 0, halo_r = 0;  // x halo (pixels) over all sources
  int halo_t = 0, halo_b = 0;  // y halo (rows) over all sources
  int max_delay = 0;
  int unroll = 1;
  int max_src_window = 1;
  bool uses_ypar = false;      // some node selects on the row parity
  int node_of(int id, int chan) const;
  int gather_of(int id, int chan, int mode) const;
  int n_gather = 0;            // gather sources (after the staged sources)
};

struct Pipeline;

// Per-device compiled module cache entry.
struct Kernel {
  void *module = nullptr;    // CUmodule
  void *function = nullptr;  // CUfunction
  int regs = 0;
  int static_smem = 0;
  std::string name;
};

struct Workspace;   // runtime buffers (defined in runtime.cpp)
struct BatchCache;  // batched-run launches and tables (batch.cpp)

// Launch-argument block shared by every generated kernel (device layout is
// mirrored in the device source).
struct alignas(64) TmapBytes {
  uint64_t v[16];
};
// What wt_debug_kernel stores in a tensor-map slot (no driver involved).
struct DebugTmap {
  const void *ptr;
  int32_t W, H, C, esz;
  int64_t pitch, plane;
  int32_t boxw, boxh;
};
struct SrcDesc {
  const void *ptr;
  int32_t W, H, C, dtype;
  int64_t pitch, plane;
};
struct DstDesc {
  void *ptr;
  int32_t W, H, C, dtype;
  int64_t pitch, plane;
};
struct alignas(64) KernelArgs {
  TmapBytes tmap[kMaxSrc];
  SrcDesc src[kMaxAllSrc];
  DstDesc dst[kMaxDst];
  int32_t W, H;            // domain of the group's level
  int32_t tile_h, tiles_x, tiles_y, n_tiles;
  int32_t chunk, nbuf;
  int32_t out_w;           // output columns per warp tile
  int32_t channels;
  int32_t *err;            // device error word
  // persistent batched mode
  const int32_t *tile_table;  // 4 ints per tile: image, tx, ty, c
  int32_t *queue;             // atomic tile counter
  int32_t n_images;
  int32_t direct;          // warp-tile kernels: 1 = one tile per warp by block index
  const void *img_tab;        // per-image SrcDesc/DstDesc/tmaps
  // two tile heights: tiles [0, n_big) have tile_h rows and cover tile
  // rows [0, ty1); the rest have tile_h2 rows (short tiles end the run)
  int32_t tile_h2, ty1, ty2, n_big;
};


// Launches of earlier runs, reused while the schedule, the device, the
// workspace and the image descriptors stay the same (no re-planning, no
// tensor-map re-encoding).
struct CachedRun {
  std::vector<void *> functions;   // CUfunction per launch
  std::vector<KernelArgs> args;
  std::vector<unsigned> grid;      // 3 per launch
  std::vector<int> block, smem;
  // stream lanes of the launches (empty: one lane, the caller's stream)
  std::vector<int> lane;
  std::vector<std::vector<int>> waits;
  std::vector<char> record;
  int n_lanes = 1;
};
struct RunCache {
  int device = -1;
  uint64_t sched_version = 0;
  uint64_t ws_generation = 0;
  std::map<std::string, CachedRun> runs;  // key: raw bytes of the descriptors
};

struct Pipeline {
  std::vector<Stage> stages;
  std::vector<int> in_channels;
  std::vector<int> outputs;
  std::vector<std::vector<int>> consumers;
  std::vector<char> is_output;
  Schedule sched;
  uint64_t sched_version = 1;
  RunCache cache;
  std::mutex mu;
  std::shared_ptr<Workspace> ws;
  std::shared_ptr<BatchCache> batch;
  uint64_t hash = 0;
  bool has_z = false;  // some stage has a plane-offset (3-D) tap
  // Sec. 6 preprocessing results (wt_preprocess): per stage, ns per
  // iteration of its body alone and registers; empty until measured
  std::vector<double> pre_ns;
  std::vector<int> pre_regs;
  // devices (bit d) on which wt_run_static ran this pipeline: wt_check then
  // also reads the status word of the library's static scratch there
  uint64_t static_devs = 0;
  LiveCounter live;
};

// ir.cpp
void build_pipeline(Pipeline &p, const wt_stage *st, int n, const int32_t *in_ch,
                    int n_in, const int32_t *outs, int n_out);
void level_dims(int W, int H, int level, int *w, int *h);
uint64_t fnv1a(const void *data, size_t n, uint64_t h = 1469598103934665603ull);

// analysis.cpp
GroupGeom analyze_group(const Pipeline &p, const std::vector<int> &stages, int vec,
                        float frac_reg, int dtype_bytes, bool split_separable = true);
int elem_bytes(int dtype);

// codegen.cpp
// Register cap of warp-tile group kernels whose schedule sets none (launch
// bounds for 14 one-warp blocks per SM).  Measured on a GB300: the corner
// response's group then takes 128 registers instead of 154, 16 warps per SM
// instead of 12, and runs 12% faster; kernels that need more registers
// than the cap leaves spill under it and are rebuilt without it.
constexpr int kSoftRegCap = 144;

struct CodegenKey {
  std::vector<int> stages;
  int vec = 4;
  std::vector<int> src_dtypes, dst_dtypes;
  float frac_reg = 1.f;
  int max_regs = 0;
  int nw = 4;        // warps per block (launch bound)
  int chunk = 8;     // TMA rows per chunk
  int nbuf = 2;      // TMA buffers per source
  bool plain = false;
  bool persistent = false;
  bool pairs = true;  // packed f32x2 arithmetic
  // warp-tile groups: constant factors of stage programs deferred to the
  // consumers (register values hold the value over a compile-time scale)
  bool fold = false;
  // max_regs is the library's soft cap (the schedule set none): get_kernel
  // rebuilds the kernel uncapped if it spills under it
  bool soft_cap = false;
  // per-stage kernel reading several fixed planes of one producer through
  // taps up by 4 or 8: the planes share one row address and column clamps
  bool shared_planes = false;
  // test only (WT_FLAG_TEST_STALL): the first chunk of every tile is armed
  // for bytes no copy delivers, and waits give up after a few polls
  bool test_stall = false;
  // every tile starts on an even row and the unroll is even: the row parity
  // of each unrolled step is a compile-time constant
  bool even_rows = false;
  // storage type of the intermediates' shared-memory windows (FP32, or the
  // group's 16-bit storage type; arithmetic stays FP32)
  int win_dtype = WT_F32;
  // one overlapped tile of tbx x tby outputs per thread block, stages in
  // shared memory between block barriers
  bool otptb = false;
  int tbx = 0, tby = 0;
  // per-stage kernel of a separable down-sampling stage, streamed at two
  // rates (scaled.cpp): vec outputs per lane, tby output rows per warp
  bool down = false;
  // reduction chain across levels (chain.cpp)
  bool chain = false;
  // two-level down-sampling cascade (cascade.cpp): vec S1 values per lane,
  // tby S2 rows per warp
  bool cascade = false;
  // 3-D group (vol.cpp): split (streamed) axis 0 = rows, 1 = planes; vol_to
  // points of the other non-x axis per warp tile; tby streamed points
  bool vol = false;
  int vol_split = 0, vol_to = 0;
  std::string str() const;
};

// Shared-memory layout and tile geometry of a fused group kernel.
struct FusedLayout {
  int V = 4;
  int lpad = 0, rpad = 0, out_w = 0;  // x halo (multiples of V), output columns
  int chunk = 8, nbuf = 3, ring = 24; // ring = chunk * nbuf rows
  int issue_blk = 0;                  // block offset in a chunk that refills a buffer
  int nsx = 0;                        // nsteps = halo_t + tile_h + nsx
  int src_rows_extra = 0;             // source rows = halo_t + tile_h + halo_b
  std::vector<int> boxw;              // per source: TMA box width (elements)
  std::vector<int> bufb;              // per source: bytes per staging buffer (128-multiple)
  std::vector<int> esz;               // per source: element bytes
  std::vector<int> ring_off;          // per source: byte offset in the warp slice
  std::vector<int> win_off;           // per node: smem window offset (-1 = regs)
  int bar_off = 0;
  int warp_bytes = 0;
  int chunk_bytes = 0;                // expect_tx per chunk (all sources)
};
FusedLayout fused_layout(const GroupGeom &g, const CodegenKey &key);
std::string emit_fused(const Pipeline &p, const GroupGeom &g, const CodegenKey &key,
                       const std::string &kname);
std::string emit_plain(const Pipeline &p, int sid, const CodegenKey &key,
                       const std::string &kname);
// otptb.cpp: block-tile kernel of a fused group.  Per node, its region
// relative to the tile origin (rx, ry, rw x rh points) and its FP32 buffer's
// byte offset in dynamic shared memory (buffers of dead nodes are reused).
struct OtptbLayout {
  int tbx = 128, tby = 16;
  std::vector<int> rx, ry, rw, rh, off;
  int smem = 0;
};
OtptbLayout otptb_layout(const GroupGeom &g, const CodegenKey &key);
std::string emit_otptb(const Pipeline &p, const GroupGeom &g, const CodegenKey &key,
                       const std::string &kname);
// scaled.cpp: a stage whose taps all read one producer one level finer
// (DOWN2) in a rank-one linear pattern: sum_ij wy[j] wx[i] P(2x + dx0 + i,
// 2y + dy0 + j) + c.
struct DownForm {
  bool ok = false;
  int slot = 0, chan = 0;  // producer input slot and channel spec
  int dx0 = 0, dy0 = 0;
  std::vector<double> wx, wy;
  double c = 0;
};
DownForm down_form(const Pipeline &p, int sid);
// The streaming kernel handles the form with `vo` outputs per lane.
bool down_streamable(const DownForm &f, int vo);
std::string emit_down(const Pipeline &p, int sid, const CodegenKey &key,
                      const std::string &kname);
// Dynamic shared memory of the down-sampling kernel (its cp.async ring).
int down_smem(const Pipeline &p, int sid, const CodegenKey &key);
// cascade.cpp: S2 reduces S1 one level further (centred form), S1 a
// streamable down-sampling stage; one kernel streams S1's producer and
// writes both.
bool cascade_pair_ok(const Pipeline &p, int s1, int s2);
struct CascadeUnit {
  int s1, s2;  // s2 = -1: s1 alone (the single-level streaming kernel)
};
// Launch units of a group of down-sampling stages (pairs and singles, in
// launch order); empty unless every stage is a streamable down-sampling
// stage and at least one pair forms.
std::vector<CascadeUnit> cascade_units(const Pipeline &p, const std::vector<int> &seg);
std::string emit_cascade(const Pipeline &p, int s1, int s2, const CodegenKey &key, const std::string &kname);
int cascade_smem(const Pipeline &p, int s1, const CodegenKey &key);
// chain.cpp: a group S1..Sk, each stage one level coarser: S1 a program of
// one one-plane producer's DOWN2 taps inside its 2x2 block, every later
// stage a weighted 2x2 sum of the one before (w[m][i + 2 j] for S(m+2));
// only Sk leaves the group.
struct ChainForm {
  bool ok = false;
  int producer = 0;
  int C = 1;
  std::vector<std::array<double, 4>> w;
};
ChainForm chain_form(const Pipeline &p, const std::vector<int> &stages);
std::string emit_chain(const Pipeline &p, const std::vector<int> &stages, const CodegenKey &key,
                       const std::string &kname);
// Code-generation helpers shared by the kernel generators (codegen.cpp):
// the device helpers' dtype suffix ("f32", "f16", "bf16"), and an FP32
// literal of v (NaN and infinities by bit pattern, integral values with a
// point).
const char *dtype_name(int dtype);
std::string float_literal(float v);
// Source table of a plain (per-stage) kernel: distinct (slot, channel spec).
struct PlainSrc {
  int slot, chan;
};
std::vector<PlainSrc> plain_sources(const Pipeline &p, int sid);
// Whether stage sid's per-stage kernel reads two or more fixed planes of
// one producer through taps up by 4 or 8 (they then share row addressing).
bool plain_shares_planes(const Pipeline &p, int sid);
extern const char *kDeviceSource;  // device_src.cpp

// vol.cpp: a fused group over a volume (App. A, generalised hybrid
// tiling).  A D x H x W volume is an image of D planes.  Warp tiles stream
// along the split axis s (rows, or planes), lanes cover x (V points each),
// and the third axis o is a register tile of vol_to points plus halos: each
// node keeps, per o point of its range, a window of its last `window`
// streamed rows, V values per lane.  Producer reads along o are
// same-thread register reads; along x, shuffles from the lane that holds
// the column; along s, older window slots.
struct VolNode {
  int id = 0;            // stage id, or -(j+1) for a pipeline input
  bool source = false;   // read from memory (outside the group)
  int lead = 0;          // rows ahead of the output row
  int window = 1;        // streamed rows kept
  int olo = 0, ohi = 0;  // o points below/above the tile's range
  int xl = 0, xr = 0;    // neighbour values stored per lane (kept 0: x
                         // neighbours come by shuffle at the tap)
  int need_lo = 0;       // first needed row relative to the tile (<= 0)
  int src_index = -1, dst_index = -1;
  int planes = 1;        // planes of the image (sources: 1 or D)
  bool rotate = true;    // slots rotate by unrolling (window divides U)
};
struct VolGeom {
  bool ok = false;
  bool staged = false;         // sources staged in shared memory (else registers)
  int prefetch = 2;            // rows a source is loaded ahead of its first use
  std::string why;
  int split = 0, To = 4, Ts = 32, V = 2;
  int D = 1, level = 0;
  std::vector<VolNode> nodes;  // sources first, then the group's stages
  std::vector<int> liveouts;   // stage ids
  int hxl = 0, hxlp = 0, hxr = 0, ow = 0;  // x halo, V-rounded left halo, outputs
  int xml = 0, xmr = 0;        // source columns read left/right of a lane's V
  int pro = 0;                 // prologue steps
  int U = 1;                   // unrolled steps per loop iteration
  int regs = 0;                // window registers per thread
  int node_of(int id) const;
};
// Geometry of a 3-D group, or ok = false with the reason.
// `staged`: sources in the warp's shared memory (frac_reg < 1), else in
// registers like the stages' windows; `prefetch`: rows a source is loaded
// ahead of its first use (1..8).
VolGeom vol_analyze(const Pipeline &p, const std::vector<int> &stages, int split, int To, int Ts, int V,
                    bool staged, int prefetch);
std::string emit_vol(const Pipeline &p, const VolGeom &g, const CodegenKey &key, const std::string &kname);
// Shared memory per warp of a 3-D group kernel (its sources' staged rows);
// `offs` (optional) receives each source node's byte offset.
int vol_warp_smem(const VolGeom &g, const CodegenKey &key, std::vector<int> *offs);

}  // namespace wt

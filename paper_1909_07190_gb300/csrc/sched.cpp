// Scheduling: grouping, tile shapes and the hybrid split (Sec. 6).
//
//  * OTPW geometry of Sec. 4 (warp sizes, warp overlapped tile, scratchpad
//    size) as the paper states it, used to pin the formulas;
//  * per-stage preprocessing of Sec. 6: each stage's register use (the
//    compiled per-stage kernel) and time per iteration (a one-thread
//    micro-kernel looping over the stage body with shared-memory taps);
//  * the cost function of Alg. 2, evaluated on this implementation's
//    kernels (their real shared-memory layout, register windows, tiles);
//  * DP-Fusion (Sec. 2.4) over contiguous groupings of the topological
//    order, each group taking the argmin of the cost over tile height,
//    warps per block, pixels per lane, fracReg and transaction size.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <map>
#include <set>
#include <sstream>

#include "wt_jit.hpp"
#include "wt_runtime.hpp"
#include "wt_sched.hpp"

namespace wt {

// ------------------------------------------------------ GPU configuration

GpuConfig default_gb300() {
  GpuConfig c;
  c.nsms = 152;
  c.cores_per_sm = 128;
  c.glmem_bw = 6781.4e9;
  c.max_smem_per_tb = 227 * 1024;
  c.smem_per_sm = 228 * 1024;
  c.max_warps_per_sm = 64;
  c.max_tb_per_sm = 32;
  c.regs_per_sm = 65536;
  c.max_regs_per_th = 255;
  c.warp_size = 32;
  c.max_th_per_sm = 2048;
  return c;
}

GpuConfig device_config(int dev) {
  GpuConfig c = default_gb300();
  cudaDeviceProp pr;
  if (cudaGetDeviceProperties(&pr, dev) != cudaSuccess) {
    cudaGetLastError();
    return c;
  }
  c.nsms = pr.multiProcessorCount;
  c.max_smem_per_tb = (int)pr.sharedMemPerBlockOptin;
  c.smem_per_sm = (int)pr.sharedMemPerMultiprocessor;
  c.max_warps_per_sm = pr.maxThreadsPerMultiProcessor / pr.warpSize;
  c.max_tb_per_sm = pr.maxBlocksPerMultiProcessor;
  c.regs_per_sm = pr.regsPerMultiprocessor;
  c.warp_size = pr.warpSize;
  c.max_th_per_sm = pr.maxThreadsPerMultiProcessor;
  int mem_khz = 0, bus_bits = 0;
  cudaDeviceGetAttribute(&mem_khz, cudaDevAttrMemoryClockRate, dev);
  cudaDeviceGetAttribute(&bus_bits, cudaDevAttrGlobalMemoryBusWidth, dev);
  const char *env = getenv("WT_HBM_GBS");  // a measured copy bandwidth, if known
  if (env && atof(env) > 0) c.glmem_bw = atof(env) * 1e9;
  else if (mem_khz > 0 && bus_bits > 0) c.glmem_bw = 2.0 * mem_khz * 1e3 * bus_bits / 8.0;
  cudaGetLastError();
  return c;
}

// --------------------------------------------------- Sec. 4 OTPW geometry

void otpw_warp_sizes(const int B[3], int warp_size, int W[3]) {
  W[0] = std::min(B[0], warp_size);
  W[1] = std::min(B[1], std::max(1, warp_size / W[0]));
  W[2] = std::min(B[2], std::max(1, warp_size / (W[0] * W[1])));
}

int64_t otpw_scratchpad_points(const int B[3], const int W[3], const int T[3], const int O[3]) {
  int64_t n = 1;
  for (int i = 0; i < 3; i++) n *= (int64_t)((B[i] + W[i] - 1) / W[i]) * ((int64_t)T[i] * W[i] + O[i]);
  return n;
}

// ----------------------------------------------- Alg. 2 occupancy lines

double alg2_occupancy(const GpuConfig &g, int64_t smem_per_tb, int warps_per_tb, int regs_per_th,
                      int *max_tb_per_sm, int *warps_per_sm) {
  int tb = g.max_tb_per_sm;
  if (smem_per_tb > 0) tb = (int)std::min<int64_t>(g.smem_per_sm / smem_per_tb, g.max_tb_per_sm);
  int sh_occ = std::min(tb * warps_per_tb, g.max_warps_per_sm);
  int th = std::min(g.regs_per_sm / std::max(1, regs_per_th), g.max_th_per_sm);
  // registers are granted per warp: whole warps only
  int reg_occ = th / g.warp_size;
  // and per block
  int reg_tb = reg_occ / std::max(1, warps_per_tb);
  int warps = std::min(sh_occ, std::min(reg_occ, reg_tb * warps_per_tb));
  if (max_tb_per_sm) *max_tb_per_sm = std::min(tb, reg_tb);
  if (warps_per_sm) *warps_per_sm = warps;
  return (double)warps / g.max_warps_per_sm;
}

// ----------------------------------- A17: coalescing into transactions

int64_t min_gl_txs(const int64_t *addr, int n, int access_bytes, int txn) {
  std::set<int64_t> segs;
  for (int i = 0; i < n; i++) {
    int64_t a0 = addr[i] / txn, a1 = (addr[i] + access_bytes - 1) / txn;
    for (int64_t s = a0; s <= a1; s++) segs.insert(s);
  }
  return (int64_t)segs.size();
}

// ------------------------------------------- Sec. 6 preprocessing (A16)

namespace {

std::string micro_source(const Pipeline &p, int sid, const std::string &name) {
  const Stage &S = p.stages[sid];
  std::ostringstream o;
  o << "extern \"C\" __global__ void " << name << "(float *out, int iters) {\n"
       "__shared__ float sm[1024];\n"
       "for (int i = threadIdx.x; i < 1024; i += blockDim.x) sm[i] = 0.001f * (float)(i & 63) + 0.5f;\n"
       "__syncthreads();\nfloat acc = 0.f;\nint base = threadIdx.x;\n"
       "for (int it = 0; it < iters; it++) {\n";
  std::vector<std::string> st;
  int tap = 0;
  for (const Op &op : S.ops) {
    char b[64];
    switch (op.op) {
      case WT_OP_CONST: {
        // a valid FP32 literal for every value (integral ones need a point)
        if (std::isnan(op.value)) {
          st.push_back("__int_as_float(0x7fc00000)");
        } else if (std::isinf(op.value)) {
          st.push_back(op.value > 0 ? "__int_as_float(0x7f800000)" : "__int_as_float(0xff800000)");
        } else {
          snprintf(b, sizeof b, "%.9g", (double)op.value);
          std::string v(b);
          if (v.find_first_of(".e") == std::string::npos) v += ".0";
          st.push_back("(" + v + "f)");
        }
      } break;
      case WT_OP_XPAR: st.push_back("((float)(it & 1))"); break;
      case WT_OP_YPAR: st.push_back("((float)((it >> 1) & 1))"); break;
      case WT_OP_CHAN: st.push_back("((float)((it >> 2) & 7))"); break;
      case WT_OP_TAP:
        snprintf(b, sizeof b, "sm[(base + %d) & 1023]", 37 * tap++ + 11 * op.dx + 101 * op.dy);
        st.push_back(b);
        break;
      case WT_OP_NEG: st.back() = "(-" + st.back() + ")"; break;
      case WT_OP_ABS: st.back() = "fabsf(" + st.back() + ")"; break;
      case WT_OP_SQRT: st.back() = "sqrtf(" + st.back() + ")"; break;
      default: {
        std::string bb = st.back();
        st.pop_back();
        std::string aa = st.back();
        st.pop_back();
        const char *f = op.op == WT_OP_ADD ? "+" : op.op == WT_OP_SUB ? "-" : op.op == WT_OP_MUL ? "*" : "/";
        if (op.op == WT_OP_MIN) st.push_back("fminf(" + aa + ", " + bb + ")");
        else if (op.op == WT_OP_MAX) st.push_back("fmaxf(" + aa + ", " + bb + ")");
        else st.push_back("(" + aa + " " + f + " " + bb + ")");
      }
    }
  }
  o << "acc += " << st.back() << ";\nbase = (base + 7) & 1023;\n}\nout[threadIdx.x] = acc;\n}\n";
  return o.str();
}

}  // namespace

std::vector<StageStats> stage_stats(const Pipeline &p, bool measure) {
  std::vector<StageStats> r(p.stages.size());
  const bool have = p.pre_ns.size() == p.stages.size() && p.pre_regs.size() == p.stages.size();
  for (size_t s = 0; s < p.stages.size(); s++) {
    int ops = 0;
    for (const Op &op : p.stages[s].ops)
      if (op.op != WT_OP_TAP && op.op != WT_OP_CONST) ops++;
    r[s].ns_per_iter = 0.5 + 0.5 * ops;  // estimate when not measured
    r[s].regs = 24;
    r[s].measured = false;
    if (have) {  // measured by an earlier preprocessing run
      r[s].ns_per_iter = p.pre_ns[s];
      r[s].regs = p.pre_regs[s];
      r[s].measured = true;
    }
  }
  if (!measure) return r;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return r;
  }
  const Driver &drv = driver();
  // device buffer, events and the current module are released on every
  // exit, errors included
  struct Res {
    float *out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CUmodule mod = nullptr;
    ~Res() {
      if (mod) driver().moduleUnload(mod);
      if (e0) cudaEventDestroy(e0);
      if (e1) cudaEventDestroy(e1);
      dev_free(out, 256 * sizeof(float));
    }
  } res;
  if (dev_alloc((void **)&res.out, 256 * sizeof(float)) != cudaSuccess) {
    cudaGetLastError();
    fail(WT_ENOMEM, "cannot allocate the preprocessing buffer");
  }
  float *out = res.out;
  check_rt(cudaEventCreate(&res.e0), "cudaEventCreate");
  check_rt(cudaEventCreate(&res.e1), "cudaEventCreate");
  cudaEvent_t e0 = res.e0, e1 = res.e1;
  for (size_t s = 0; s < p.stages.size(); s++) {
    char nm[64];
    snprintf(nm, sizeof nm, "wt_micro_%016llx_%zu", (unsigned long long)p.hash, s);
    std::string cubin = compile_cubin(micro_source(p, (int)s, nm), nm, 0);
    check_cu(drv.moduleLoadData(&res.mod, cubin.data()), "cuModuleLoadData(micro)");
    CUfunction f;
    check_cu(drv.moduleGetFunction(&f, res.mod, nm), "cuModuleGetFunction(micro)");
    int iters = 1 << 16;
    void *args[] = {&out, &iters};
    // one block, one thread (Sec. 6): the time of one stage iteration
    check_cu(drv.launchKernel(f, 1, 1, 1, 1, 1, 1, 0, nullptr, args, nullptr), "cuLaunchKernel(micro)");
    cudaEventRecord(e0, nullptr);
    check_cu(drv.launchKernel(f, 1, 1, 1, 1, 1, 1, 0, nullptr, args, nullptr), "cuLaunchKernel(micro)");
    cudaEventRecord(e1, nullptr);
    check_rt(cudaEventSynchronize(e1), "cudaEventSynchronize(micro)");
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    r[s].ns_per_iter = (double)ms * 1e6 / iters;
    int regs = 0;
    if (drv.funcGetAttribute(&regs, CU_FUNC_ATTRIBUTE_NUM_REGS, f) == CUDA_SUCCESS && regs > 0) r[s].regs = regs;
    drv.moduleUnload(res.mod);
    res.mod = nullptr;
    r[s].measured = true;
  }
  return r;
}

// ------------------------------------------------------ Alg. 2 cost terms

const char *kTermNames[7] = {"gl_traffic", "one_minus_occupancy", "mem_over_compute",
                             "unallocated_smem", "unused_regs", "frac_overlap", "extra_tbs"};

CostWeights default_weights() {
  CostWeights w;
  // Table 3's Tesla V100 weights as the starting point (re-fit on GB300 by
  // fit_weights from measured runtimes).
  const double v100[7] = {50, 0.5, 60, 10, 2, 100, 1};
  for (int i = 0; i < 7; i++) w.w[i] = v100[i];
  return w;
}

static CostWeights g_weights = default_weights();
static std::mutex g_wmu;

CostWeights current_weights() {
  std::lock_guard<std::mutex> lk(g_wmu);
  return g_weights;
}

void set_weights(const CostWeights &w) {
  std::lock_guard<std::mutex> lk(g_wmu);
  g_weights = w;
}

int estimate_regs(const GroupGeom &g, int V, const std::vector<StageStats> &st) {
  // registers of the rotating windows (the register tile) plus the live
  // temporaries of the largest stage (stages run one after another in the
  // streaming kernel, so the max rather than the sum of Alg. 2's RegUsage)
  int tile = 0;
  for (const Node &n : g.nodes)
    if (!n.in_smem) tile += n.window * (V + n.xl + n.xr);
  int stage = 0;
  for (int s : g.stages) stage = std::max(stage, st[s].regs);
  return std::min(255, 24 + tile + stage / 2);
}

double work_share(const Pipeline &p, const std::vector<int> &stages, int W0, int H0) {
  auto pts = [&](int s) {
    int w, h;
    level_dims(W0, H0, p.stages[s].level, &w, &h);
    return (double)w * h * p.stages[s].channels;
  };
  double g = 0, t = 0;
  for (int s : stages) g += pts(s);
  for (size_t s = 0; s < p.stages.size(); s++) t += pts((int)s);
  return g / std::max(1.0, t);
}

double pipeline_bytes(const Pipeline &p, int W0, int H0, int dtype) {
  double b = 0;
  for (size_t j = 0; j < p.in_channels.size(); j++) b += (double)W0 * H0 * p.in_channels[j];
  for (int o : p.outputs) {
    int w, h;
    level_dims(W0, H0, p.stages[o].level, &w, &h);
    b += (double)w * h * p.stages[o].channels;
  }
  return b * elem_bytes(dtype);
}

// Cost of one stage run alone by the per-stage kernel: its HBM traffic.
CostInfo cost_plain(const Pipeline &p, int s, int W0, int H0, int dtype, const CostWeights &w, double pbytes) {
  CostInfo ci;
  int wl, hl;
  level_dims(W0, H0, p.stages[s].level, &wl, &hl);
  double bytes = (double)wl * hl * p.stages[s].channels * 4;
  for (const Edge &e : p.stages[s].edges) {
    int pl = e.producer >= 0 ? p.stages[e.producer].level : 0;
    int pw, ph;
    level_dims(W0, H0, pl, &pw, &ph);
    // channels read: every producer channel for per-channel taps (-1),
    // else the distinct fixed ones
    const int pc = e.producer >= 0 ? p.stages[e.producer].channels : p.in_channels[-e.producer - 1];
    const bool per_channel = std::find(e.chans.begin(), e.chans.end(), -1) != e.chans.end();
    bytes += (double)pw * ph * (per_channel ? pc : (int)e.chans.size()) * 4;
  }
  (void)dtype;
  ci.t[0] = bytes / std::max(1.0, pbytes);
  ci.cost = w.w[0] * ci.t[0];
  ci.feasible = true;
  ci.work = work_share(p, {s}, W0, H0);
  return ci;
}

CostInfo cost_group(const Pipeline &p, const std::vector<int> &stages, const GroupParams &prm, int txn, int W0,
                    int H0, int dtype, const GpuConfig &cfg, const std::vector<StageStats> &st,
                    const CostWeights &w, double pipeline_bytes, const GroupGeom *pre) {
  CostInfo ci;
  GroupGeom g = pre ? *pre : analyze_group(p, stages, prm.vec ? prm.vec : 4, prm.frac_reg, 4);
  // Alg. 2 line 1: dependence vectors must be constant (here: one level,
  // same-level taps); other groups run as per-stage kernels instead.
  if (!g.fusable) return ci;
  const int V = prm.vec ? prm.vec : 4;
  CodegenKey key;
  key.vec = V;
  key.nw = prm.warps_per_block;
  key.chunk = prm.chunk_rows;
  key.nbuf = prm.n_buffers;
  int n_src = 0;
  for (const Node &n : g.nodes)
    if (n.is_source) n_src++;
  key.src_dtypes.assign(n_src, dtype);
  key.dst_dtypes.assign(g.liveouts.size(), dtype);
  FusedLayout L;
  try {
    L = fused_layout(g, key);
  } catch (const Error &) {
    return ci;
  }
  int Wl, Hl;
  level_dims(W0, H0, g.level, &Wl, &Hl);
  const int T = prm.tile_h;
  const int esz = elem_bytes(dtype);
  const int64_t tiles = (int64_t)((Wl + L.out_w - 1) / L.out_w) * ((Hl + T - 1) / T) * g.channels;
  const int nw = prm.warps_per_block;
  const int64_t smem_tb = (int64_t)nw * L.warp_bytes;
  if (smem_tb > cfg.max_smem_per_tb) return ci;
  const int regs = estimate_regs(g, V, st);
  if (regs > cfg.max_regs_per_th) return ci;
  // global memory transactions per warp tile (A17 on the warp's rows)
  const int nsteps = g.halo_t + T + L.nsx;
  const int src_rows = g.halo_t + T + g.halo_b;
  int64_t tx_tile = 0;
  std::vector<int64_t> addr;
  for (int s = 0; s < n_src; s++) {
    addr.clear();
    // TMA box row: boxw contiguous elements starting on a 16-byte boundary
    for (int e = 0; e < L.boxw[s]; e += 4) addr.push_back((int64_t)e * esz);
    tx_tile += src_rows * min_gl_txs(addr.data(), (int)addr.size(), 4 * esz, txn);
  }
  for (size_t d = 0; d < g.liveouts.size(); d++) {
    addr.clear();
    for (int l = L.lpad / V; l < 32 - L.rpad / V; l++) addr.push_back((int64_t)(L.lpad + (l - L.lpad / V) * V) * esz);
    tx_tile += T * min_gl_txs(addr.data(), (int)addr.size(), V * esz, txn);
  }
  // gather sources (another level, read by plain loads, not staged): the
  // source rows and columns under the tile, at the source's scale
  for (const Node &n : g.nodes) {
    if (!n.gather_mode) continue;
    const bool down = n.gather_mode == WT_TAP_DOWN2;
    const int cols = down ? 2 * 32 * V + 4 : 32 * V / 2 + 2;
    const int rows = down ? 2 * src_rows + 3 : src_rows / 2 + 2;
    tx_tile += (int64_t)rows * ((cols * esz + txn - 1) / txn + 1);
  }
  const double total_tx = (double)tx_tile * tiles;
  int tb_per_sm = 0, warps_sm = 0;
  const double occ = alg2_occupancy(cfg, smem_tb, nw, regs, &tb_per_sm, &warps_sm);
  if (warps_sm < 1) return ci;
  const double mem_time = txn * total_tx / cfg.glmem_bw;
  double iter_ns = 0;
  int64_t useful = 0, computed = 0;
  for (const Node &n : g.nodes) {
    if (n.is_source || n.gather_mode) continue;  // read, not computed
    double ns = n.synthetic ? 0.5 + 0.5 * (double)n.prog.size() / 3 : st[n.id].ns_per_iter;
    iter_ns += ns;
    computed += (int64_t)32 * V * nsteps;
    useful += (int64_t)L.out_w * T;
  }
  const double compute_time =
      iter_ns * 1e-9 * (double)computed / (32 * V) * tiles * V / ((double)cfg.nsms * cfg.cores_per_sm);
  const double active = (double)warps_sm * cfg.nsms;
  const double waves = tiles / active;
  ci.t[0] = txn * total_tx / std::max(1.0, pipeline_bytes);
  ci.t[1] = 1.0 - occ;
  ci.t[2] = mem_time / std::max(1e-12, compute_time);
  ci.t[3] = 1.0 - (double)smem_tb * tb_per_sm / cfg.smem_per_sm;
  ci.t[4] = 1.0 - (double)regs * (occ * cfg.max_warps_per_sm * cfg.warp_size) / cfg.regs_per_sm;
  ci.t[5] = (double)(computed - useful) / std::max<int64_t>(1, useful);
  ci.t[6] = (std::ceil(waves) - waves) / std::max(1.0, std::ceil(waves));
  // intensive terms count in proportion to the group's share of the
  // pipeline's points (a small group adds a small occupancy penalty)
  ci.work = work_share(p, stages, W0, H0);
  double cost = w.w[0] * ci.t[0];
  for (int i = 1; i < 7; i++) cost += w.w[i] * ci.t[i] * ci.work;
  ci.cost = cost;
  ci.feasible = true;
  ci.regs = regs;
  ci.smem_per_tb = (int)smem_tb;
  ci.occupancy = occ;
  ci.tiles = tiles;
  ci.waves = waves;
  return ci;
}

}  // namespace wt

namespace wt {

// ------------------------------------------------------------ DP-Fusion

static const int kTileH[] = {8, 12, 16, 20, 24, 32, 48, 64};
static const int kWarps[] = {2, 4, 8};
static const int kVec[] = {4, 8};
static const int kTxn[] = {32, 128};

// HBM bytes of a reduction chain across levels run as one kernel (its
// producer read once, only its last stage written), FP32 like the per-stage
// kernels' estimate.
double chain_bytes(const Pipeline &p, const std::vector<int> &seg, int W0, int H0) {
  const ChainForm f = chain_form(p, seg);
  const int pl = f.producer >= 0 ? p.stages[f.producer].level : 0;
  int pw, ph, lw, lh;
  level_dims(W0, H0, pl, &pw, &ph);
  level_dims(W0, H0, p.stages[seg.back()].level, &lw, &lh);
  return ((double)pw * ph + (double)lw * lh * p.stages[seg.back()].channels) * 4;
}

// HBM bytes of a group of down-sampling stages run as cascade launches:
// each pair reads its first stage's producer once and writes both stages,
// each other stage reads its producer and writes itself (FP32, like the
// per-stage kernels' estimate).
double cascade_bytes(const Pipeline &p, const std::vector<int> &seg, int W0, int H0) {
  double bytes = 0;
  for (const CascadeUnit &u : cascade_units(p, seg)) {
    const DownForm f = down_form(p, u.s1);
    const int pid = p.stages[u.s1].inputs[f.slot];
    const int pl = pid >= 0 ? p.stages[pid].level : 0;
    const int pc = pid >= 0 ? p.stages[pid].channels : p.in_channels[-pid - 1];
    int w, h;
    level_dims(W0, H0, pl, &w, &h);
    bytes += (double)w * h * (f.chan >= 0 ? 1 : pc) * 4;
    for (int s : {u.s1, u.s2}) {
      if (s < 0) continue;
      level_dims(W0, H0, p.stages[s].level, &w, &h);
      bytes += (double)w * h * p.stages[s].channels * 4;
    }
  }
  return bytes;
}

SegmentChoice best_for_segment(const Pipeline &p, const std::vector<int> &seg, int W, int H, int dtype,
                               const GpuConfig &cfg, const std::vector<StageStats> &st, const CostWeights &w,
                               double pbytes, const CandidateScorer *scorer) {
  SegmentChoice best;
  best.cost = INFINITY;
  if (chain_form(p, seg).ok) {
    // a group spanning levels: the reduction chain kernel (Sec. 5's scaled
    // groups), costed by its traffic like a per-stage kernel
    CostInfo ci;
    ci.t[0] = chain_bytes(p, seg, W, H) / std::max(1.0, pbytes);
    ci.cost = w.w[0] * ci.t[0];
    ci.feasible = true;
    ci.work = work_share(p, seg, W, H);
    best.cost = ci.cost;
    best.fused = true;
    best.prm = GroupParams();
    best.info = ci;
    return best;
  }
  if (!cascade_units(p, seg).empty()) {
    // down-sampling stages of two levels: cascade launches (Sec. 5's
    // scaled groups, each pair's first level kept on chip), costed by
    // their traffic like a per-stage kernel
    CostInfo ci;
    ci.t[0] = cascade_bytes(p, seg, W, H) / std::max(1.0, pbytes);
    ci.cost = w.w[0] * ci.t[0];
    ci.feasible = true;
    ci.work = work_share(p, seg, W, H);
    best.cost = ci.cost;
    best.fused = true;
    best.prm = GroupParams();
    // S2 rows per warp: taller where the coarser level is tall (fewer
    // re-streamed halo rows), short where it is small (more warps)
    int lv = 0, w2, h2;
    for (int s : seg) lv = std::max(lv, p.stages[s].level);
    level_dims(W, H, lv, &w2, &h2);
    best.prm.tile_h = std::max(4, std::min(16, h2 / 128));
    best.info = ci;
    return best;
  }
  for (int V : kVec) {
    std::set<std::vector<char>> seen;
    for (int fi = 0; fi <= 10; fi++) {
      float frac = fi / 10.f;
      GroupGeom g = analyze_group(p, seg, V, frac, 4);
      if (!g.fusable) break;
      std::vector<char> sig;
      for (const Node &n : g.nodes) sig.push_back(n.in_smem);
      if (!seen.insert(sig).second) continue;  // same placement as an earlier fracReg
      for (int T : kTileH)
        for (int nw : kWarps)
          for (int txn : kTxn) {
            GroupParams prm;
            prm.tile_h = T;
            prm.warps_per_block = nw;
            prm.vec = V;
            prm.frac_reg = frac;
            CostInfo ci = cost_group(p, seg, prm, txn, W, H, dtype, cfg, st, w, pbytes, &g);
            if (!ci.feasible) continue;
            double c = scorer ? (*scorer)(seg, prm, ci) : ci.cost;
            if (c < best.cost) {
              best.cost = c;
              best.fused = true;
              best.prm = prm;
              best.info = ci;
            }
          }
    }
  }
  if (seg.size() == 1) {
    CostInfo ci = cost_plain(p, seg[0], W, H, dtype, w, pbytes);
    double c = scorer ? (*scorer)(seg, GroupParams(), ci) : ci.cost;
    if (c < best.cost) {
      best.cost = c;
      best.fused = false;
      best.info = ci;
    }
  }
  return best;
}

Schedule dp_fusion(const Pipeline &p, int W, int H, int dtype, const GpuConfig &cfg,
                   const std::vector<StageStats> &st, const CostWeights &w, const CandidateScorer *scorer,
                   int max_group) {
  const int n = (int)p.stages.size();
  const double pbytes = pipeline_bytes(p, W, H, dtype);
  std::vector<double> best(n + 1, INFINITY);
  std::vector<int> from(n + 1, -1);
  std::vector<SegmentChoice> choice(n + 1);
  best[0] = 0;
  for (int j = 1; j <= n; j++)
    for (int i = std::max(0, j - max_group); i < j; i++) {
      if (!std::isfinite(best[i])) continue;
      std::vector<int> seg;
      for (int s = i; s < j; s++) seg.push_back(s);
      SegmentChoice c = best_for_segment(p, seg, W, H, dtype, cfg, st, w, pbytes, scorer);
      if (best[i] + c.cost < best[j]) {
        best[j] = best[i] + c.cost;
        from[j] = i;
        choice[j] = c;
      }
    }
  if (!std::isfinite(best[n])) fail(WT_EUNSUPPORTED, "no feasible schedule");
  std::vector<std::pair<int, int>> segs;
  for (int j = n; j > 0; j = from[j]) segs.push_back({from[j], j});
  std::reverse(segs.begin(), segs.end());
  Schedule s;
  s.exec = WT_EXEC_FUSED;
  s.n_groups = (int)segs.size();
  s.group_of_stage.assign(n, 0);
  for (size_t g = 0; g < segs.size(); g++) {
    for (int k = segs[g].first; k < segs[g].second; k++) s.group_of_stage[k] = (int)g;
    GroupParams prm = choice[segs[g].second].prm;
    if (!choice[segs[g].second].fused) {
      prm = GroupParams();
      prm.plain = 1;
    }
    s.params.push_back(prm);
  }
  s.installed = true;
  s.predicted_cost = best[n];
  return s;
}

// What the automatic schedule costs groups with: the current device (the
// GB300 description without one), the stage statistics and the weights.
static GpuConfig auto_config() {
  int dev = -1;
  bool gpu = cudaGetDevice(&dev) == cudaSuccess;
  cudaGetLastError();
  return gpu ? device_config(dev) : default_gb300();
}

Schedule auto_schedule(const Pipeline &p, int W, int H, int dtype, int model) {
  GpuConfig cfg = auto_config();
  std::vector<StageStats> st = stage_stats(p, false);
  CostWeights w = current_weights();
  // the learned model when one is trained or loaded, else the analytic one
  if (model == WT_MODEL_LEARNED && costmodel_ready()) return learned_schedule(p, W, H, dtype, cfg, st, kMaxGroupStages);
  return dp_fusion(p, W, H, dtype, cfg, st, w, nullptr, kMaxGroupStages);
}

SegmentChoice auto_segment(const Pipeline &p, int first, int n, int W, int H, int dtype) {
  std::vector<int> seg;
  for (int s = first; s < first + n; s++) seg.push_back(s);
  return best_for_segment(p, seg, W, H, dtype, auto_config(), stage_stats(p, false), current_weights(),
                          pipeline_bytes(p, W, H, dtype), nullptr);
}

}  // namespace wt

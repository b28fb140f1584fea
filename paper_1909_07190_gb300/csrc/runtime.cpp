// Runtime: run plans, device workspace, kernel cache and launches.
//
// A run plan turns the installed schedule into launches: one fused
// warp-tile kernel per fusable group, one per-stage kernel for every stage
// of a non-fusable group (or of every stage under WT_EXEC_PLAIN).  Values
// crossing group boundaries live in HBM: pipeline inputs/outputs in the
// caller's images, other stages in the pipeline's workspace.
#include "wt_runtime.hpp"

#include <atomic>
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "wt_jit.hpp"

namespace wt {

// ------------------------------------------------------------- validation

static void check_image(const wt_image &im, const char *what) {
  if (!im.data) fail(WT_EINVAL, std::string(what) + ": null data");
  if (im.width < 1 || im.height < 1 || im.channels < 1)
    fail(WT_EINVAL, std::string(what) + ": empty image (width, height and channels must be >= 1)");
  if (im.dtype < WT_F32 || im.dtype > WT_BF16) fail(WT_EINVAL, std::string(what) + ": bad dtype");
  if (im.pitch_bytes % 16 != 0) fail(WT_EINVAL, std::string(what) + ": pitch_bytes must be a multiple of 16");
  if (im.pitch_bytes < (int64_t)im.width * elem_bytes(im.dtype))
    fail(WT_EINVAL, std::string(what) + ": pitch_bytes smaller than a row");
  if (((uintptr_t)im.data) % 16 != 0) fail(WT_EINVAL, std::string(what) + ": data must be 16-byte aligned");
}

std::vector<std::vector<int>> schedule_groups(const Pipeline &p) {
  std::vector<std::vector<int>> groups;
  const Schedule &s = p.sched;
  if (s.exec == WT_EXEC_PLAIN) {
    for (size_t i = 0; i < p.stages.size(); i++) groups.push_back({(int)i});
    return groups;
  }
  groups.resize(s.n_groups);
  for (size_t i = 0; i < p.stages.size(); i++) groups[s.group_of_stage[i]].push_back((int)i);
  return groups;
}

GroupParams group_params(const Pipeline &p, int gi) {
  const Schedule &s = p.sched;
  if (gi < (int)s.params.size()) return s.params[gi];
  return GroupParams();
}

static int pick_vec(const GroupParams &gp, const std::vector<int> &src_dtypes) {
  if (gp.vec == 4 || gp.vec == 8) return gp.vec;
  (void)src_dtypes;
  return 4;
}

// -------------------------------------------------------------- planning

// Images too small to give each resident warp (12 per SM) about 1.5 warp
// tiles of height T (single-image runs) use shorter tiles of the same parity (the
// kernel's row-parity folding depends on it), so that every warp has work.
int effective_tile_h(int T, int H, int tiles_x, int channels, const GroupGeom &g) {
  static int nsm = 0;
  if (!nsm) {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) ==
                                                  cudaSuccess && v > 0)
      nsm = v;
    else
      nsm = 152;
    cudaGetLastError();
  }
  T = std::max(1, T);
  const int64_t want = 3ll * nsm * 12 / 2;  // tiles: about 1.5 per resident warp
  const int64_t cols = (int64_t)std::max(1, tiles_x) * std::max(1, channels);
  const int fit = (int)std::max<int64_t>(4, (int64_t)H * cols / want);
  if (fit >= T) return T;
  // the tallest height up to `fit` whose steps (the rows plus the group's
  // streaming halo) fill whole unrolled blocks, so no block computes rows
  // past the tile's end; the same parity as T when the kernel folds the
  // row parity
  const int U = std::max(1, g.unroll), extra = stream_extra_steps(g);
  const bool parity = g.uses_ypar;
  for (int t = fit; t >= std::max(3, fit / 2); t--) {
    if (parity && (t - T) % 2) continue;
    if ((t + extra) % U == 0) return t;
  }
  int t = fit;
  if (parity && (t - T) % 2) t--;
  return std::max(T % 2 && parity ? 3 : 4, t);
}

RunPlan build_plan(Pipeline &p, const wt_image *in, int n_in, const wt_image *out, int n_out, bool batched) {
  host_alloc_point();
  if (n_in != (int)p.in_channels.size())
    fail(WT_EINVAL, "expected " + std::to_string(p.in_channels.size()) + " inputs");
  if (n_out != (int)p.outputs.size())
    fail(WT_EINVAL, "expected " + std::to_string(p.outputs.size()) + " outputs");
  for (int j = 0; j < n_in; j++) {
    check_image(in[j], "input");
    if (in[j].channels != p.in_channels[j]) fail(WT_EINVAL, "input " + std::to_string(j) + ": channels");
    if (in[j].width != in[0].width || in[j].height != in[0].height)
      fail(WT_EINVAL, "all inputs must have the same width and height");
  }
  RunPlan plan;
  plan.W = in[0].width;
  plan.H = in[0].height;
  const int n = (int)p.stages.size();
  plan.loc.assign(n, Loc());
  plan.in_loc.resize(n_in);
  for (int j = 0; j < n_in; j++) {
    Loc &l = plan.in_loc[j];
    l.ptr = in[j].data; l.pitch = in[j].pitch_bytes;
    l.plane = in[j].pitch_bytes * in[j].height;
    l.W = in[j].width; l.H = in[j].height; l.C = in[j].channels; l.dtype = in[j].dtype;
  }
  for (int k = 0; k < n_out; k++) {
    check_image(out[k], "output");
    int s = p.outputs[k];
    int w, h;
    level_dims(plan.W, plan.H, p.stages[s].level, &w, &h);
    if (out[k].width != w || out[k].height != h || out[k].channels != p.stages[s].channels)
      fail(WT_EINVAL, "output " + std::to_string(k) + ": expected " + std::to_string(w) + "x" +
                          std::to_string(h) + "x" + std::to_string(p.stages[s].channels));
    Loc &l = plan.loc[s];
    l.ptr = out[k].data; l.pitch = out[k].pitch_bytes; l.plane = out[k].pitch_bytes * out[k].height;
    l.W = w; l.H = h; l.C = out[k].channels; l.dtype = out[k].dtype; l.user = true;
  }
  int mid = p.sched.intermediate_dtype;
  if (mid < 0) mid = p.sched.exec == WT_EXEC_PLAIN ? WT_F32 : in[0].dtype;
  plan.mid_dtype = mid;
  auto groups = schedule_groups(p);
  std::vector<int> group_of(n, 0);
  for (size_t gi = 0; gi < groups.size(); gi++)
    for (int s : groups[gi]) group_of[s] = (int)gi;
  // Stages needing an HBM buffer: read by a later group (or every stage in
  // plain mode), unless they are pipeline outputs.
  auto materialize = [&](int s, bool need) {
    if (!need || plan.loc[s].ptr || plan.loc[s].user) return;
    Loc &l = plan.loc[s];
    int w, h;
    level_dims(plan.W, plan.H, p.stages[s].level, &w, &h);
    l.W = w; l.H = h; l.C = p.stages[s].channels; l.dtype = mid;
    l.pitch = ((int64_t)w * elem_bytes(mid) + 127) / 128 * 128;
    l.plane = l.pitch * h;
    l.ws_bytes = l.plane * l.C;
    l.ws = true;
  };
  for (size_t gi = 0; gi < groups.size(); gi++) {
    const auto &G = groups[gi];
    GroupParams gp = group_params(p, (int)gi);
    bool fused = p.sched.exec == WT_EXEC_FUSED && !gp.plain;
    bool zgroup = false;
    for (int s : G) zgroup = zgroup || p.stages[s].has_z;
    if (fused && zgroup) {
      // plane-offset taps: a 3-D group (App. A), else per-stage kernels
      const int V = gp.vec > 0 ? gp.vec : 2;
      VolGeom vg = vol_analyze(p, G, gp.zstream, gp.tile_o > 0 ? gp.tile_o : 4, std::max(1, gp.tile_h), V,
                               gp.frac_reg < 1.f, gp.n_buffers);
      if (vg.ok) {
        for (int s : vg.liveouts) materialize(s, !p.consumers[s].empty());
        Launch L;
        L.fused = false;
        L.stages = G;
        L.params = gp;
        L.key.vol = true;
        L.vol = vg;
        plan.launches.push_back(L);
        continue;
      }
      fused = false;
    }
    if (fused && !gp.otptb && chain_form(p, G).ok) {
      // a reduction chain across levels: one launch, only its last stage
      // written
      materialize(G.back(), !p.consumers[G.back()].empty());
      Launch L;
      L.fused = false;
      L.stages = G;
      L.params = gp;
      L.key.chain = true;
      plan.launches.push_back(L);
      continue;
    }
    if (fused && !gp.otptb) {
      const std::vector<CascadeUnit> cu = cascade_units(p, G);
      if (!cu.empty()) {
        // down-sampling stages of two levels: each pair one cascade launch
        // writing both stages, every other stage its streaming kernel
        for (const CascadeUnit &u : cu) {
          if (u.s2 < 0 && p.consumers[u.s1].empty() && !p.is_output[u.s1]) continue;  // dead stage
          materialize(u.s1, true);
          if (u.s2 >= 0) materialize(u.s2, true);
          Launch L;
          L.fused = false;
          L.stages = u.s2 < 0 ? std::vector<int>{u.s1} : std::vector<int>{u.s1, u.s2};
          L.params = gp;
          L.key.cascade = u.s2 >= 0;
          plan.launches.push_back(L);
        }
        continue;
      }
    }
    GroupGeom geom;
    if (fused) {
      geom = analyze_group(p, G, 4, gp.frac_reg, 4);
      fused = geom.fusable;
    }
    if (!fused) {
      for (int s : G) {
        if (p.consumers[s].empty() && !p.is_output[s]) continue;  // dead stage
        materialize(s, !p.consumers[s].empty());
        Launch L;
        L.fused = false;
        L.stages = {s};
        L.params = gp;
        plan.launches.push_back(L);
      }
      continue;
    }
    for (int s : geom.liveouts) materialize(s, true);
    Launch L;
    L.fused = true;
    L.stages = G;
    L.params = gp;
    L.geom = geom;
    plan.launches.push_back(L);
  }
  // Workspace offsets (256-byte aligned).
  int64_t off = 0;
  for (int s = 0; s < n; s++) {
    if (!plan.loc[s].ws) continue;
    off = (off + 255) / 256 * 256;
    plan.loc[s].ws_off = off;
    off += plan.loc[s].ws_bytes;
  }
  plan.ws_bytes = off;
  // Resolve sources, destinations and keys.
  for (Launch &L : plan.launches) {
    CodegenKey &key = L.key;
    key.stages = L.stages;
    key.frac_reg = L.params.frac_reg;
    key.max_regs = L.params.max_regs;
    if (L.fused && !L.params.otptb && key.max_regs == 0) {
      key.max_regs = kSoftRegCap;
      key.soft_cap = true;
    }
    key.nw = std::max(1, std::min(16, L.params.warps_per_block));
    key.chunk = L.params.chunk_rows > 0 ? L.params.chunk_rows : 8;
    key.nbuf = L.params.n_buffers > 0 ? L.params.n_buffers : 2;
    key.pairs = L.params.pairs != 0;
    key.fold = L.fused && !L.params.otptb && L.params.fold != 0;
    key.test_stall = L.params.test_stall != 0;
    key.even_rows = L.fused && L.geom.uses_ypar && L.params.tile_h % 2 == 0;
    L.src.clear();
    L.dst.clear();
    auto loc_of = [&](int pid) -> const Loc & { return pid >= 0 ? plan.loc[pid] : plan.in_loc[-pid - 1]; };
    if (L.fused) {
      for (const Node &nd : L.geom.nodes)
        if (nd.is_source) {
          L.src.push_back(nd.id);
          L.src_chan.push_back(nd.src_chan);
          key.src_dtypes.push_back(loc_of(nd.id).dtype);
        }
      L.n_ring = (int)L.src.size();
      // gather sources (other levels) after the staged ones
      for (const Node &nd : L.geom.nodes)
        if (nd.gather_mode) {
          L.src.push_back(nd.id);
          L.src_chan.push_back(nd.src_chan);
          key.src_dtypes.push_back(loc_of(nd.id).dtype);
        }
      for (int s : L.geom.liveouts) {
        L.dst.push_back(s);
        key.dst_dtypes.push_back(plan.loc[s].dtype);
      }
      if (L.params.otptb) {
        // one block per overlapped tile of (32 vec) x tile_h outputs
        if (L.geom.n_gather > 0) fail(WT_EUNSUPPORTED, "block tiling of groups that read other levels");
        key.otptb = true;
        key.vec = L.params.vec > 0 ? L.params.vec : 4;
        key.tbx = 32 * key.vec;
        key.tby = std::max(1, L.params.tile_h);
        key.frac_reg = 1.f;
        key.chunk = key.nbuf = 0;
        key.pairs = key.even_rows = false;
        level_dims(plan.W, plan.H, L.geom.level, &L.W, &L.H);
        const int64_t gx = (L.W + key.tbx - 1) / key.tbx, gy = (L.H + key.tby - 1) / key.tby;
        if (gy > 65535 || L.geom.channels > 65535) fail(WT_EUNSUPPORTED, "too many block tiles");
        L.tiles_x = (int)gx; L.tiles_y = (int)gy;
        L.n_tiles = (int)(gx * gy * L.geom.channels);
        L.block = 32 * key.nw;
        L.grid[0] = (unsigned)gx;
        L.grid[1] = (unsigned)gy;
        L.grid[2] = (unsigned)L.geom.channels;
        L.smem = otptb_layout(L.geom, key).smem;
        if (L.smem > 227 * 1024) fail(WT_EUNSUPPORTED, "block tile needs more than 227 KB of shared memory");
        L.kname = kernel_name(p, key, true);
        continue;
      }
      key.vec = pick_vec(L.params, key.src_dtypes);
      if (key.vec != 4) L.geom = analyze_group(p, L.stages, key.vec, L.params.frac_reg, 4);
      // 16-bit windows when asked for and the group's storage is 16-bit
      if (L.params.smem16 && !key.src_dtypes.empty() && key.src_dtypes[0] != WT_F32)
        key.win_dtype = key.src_dtypes[0];
      L.layout = fused_layout(L.geom, key);
      level_dims(plan.W, plan.H, L.geom.level, &L.W, &L.H);
      int th = std::max(1, L.params.tile_h);
      int tiles_x = (L.W + L.layout.out_w - 1) / L.layout.out_w;
      if (!batched) {
        th = effective_tile_h(th, L.H, tiles_x, L.geom.channels, L.geom);
        L.params.tile_h = th;
      }
      int tiles_y = (L.H + th - 1) / th;
      int64_t nt = (int64_t)tiles_x * tiles_y * L.geom.channels;
      if (nt > (1ll << 30)) fail(WT_EUNSUPPORTED, "too many tiles");
      L.tiles_x = tiles_x; L.tiles_y = tiles_y; L.n_tiles = (int)nt;
      L.block = 32 * key.nw;
      L.grid[0] = (unsigned)((nt + key.nw - 1) / key.nw);
      L.grid[1] = L.grid[2] = 1;
      L.smem = key.nw * L.layout.warp_bytes;
      if (L.smem > 227 * 1024) fail(WT_EUNSUPPORTED, "group needs more than 227 KB of shared memory per block");
    } else if (key.vol) {
      const VolGeom &vg = L.vol;
      key.plain = true;
      key.vec = vg.V;
      key.tby = vg.Ts;
      key.vol_split = vg.split;
      key.vol_to = vg.To;
      key.pairs = false;
      key.chunk = 0;
      key.nbuf = vg.prefetch;
      key.frac_reg = vg.staged ? 0.f : 1.f;
      for (const VolNode &nd : vg.nodes)
        if (nd.source) {
          L.src.push_back(nd.id);
          L.src_chan.push_back(-1);
          key.src_dtypes.push_back(loc_of(nd.id).dtype);
        }
      for (int s : vg.liveouts) {
        L.dst.push_back(s);
        key.dst_dtypes.push_back(plan.loc[s].dtype);
      }
      level_dims(plan.W, plan.H, vg.level, &L.W, &L.H);
      const int NS = vg.split == 0 ? L.H : vg.D, NO = vg.split == 0 ? vg.D : L.H;
      const int64_t tx = (L.W + vg.ow - 1) / vg.ow, ts = (NS + vg.Ts - 1) / vg.Ts, to = (NO + vg.To - 1) / vg.To;
      const int64_t nt = tx * ts * to;
      if (nt * 32 >= (1ll << 31)) fail(WT_EUNSUPPORTED, "too many 3-D tiles");
      L.tiles_x = (int)tx;
      L.tiles_y = (int)ts;
      L.n_tiles = (int)nt;
      L.block = 32 * key.nw;
      L.grid[0] = (unsigned)((nt + key.nw - 1) / key.nw);
      L.grid[1] = L.grid[2] = 1;
      L.smem = key.nw * vol_warp_smem(vg, key, nullptr);
      if (L.smem > 227 * 1024) fail(WT_EUNSUPPORTED, "3-D group needs more than 227 KB of shared memory per block");
      L.kname = kernel_name(p, key, false);
      continue;
    } else if (key.cascade) {
      const int s1 = L.stages[0], s2 = L.stages[1];
      const DownForm f1 = down_form(p, s1);
      const int src = p.stages[s1].inputs[f1.slot];
      key.plain = true;
      key.vec = L.params.vec == 8 ? 8 : 4;
      key.nw = 4;
      key.tby = std::max(1, L.params.tile_h);
      key.max_regs = L.params.max_regs;
      L.src.push_back(src);
      L.src_chan.push_back(0);
      key.src_dtypes.push_back(loc_of(src).dtype);
      for (int s : {s1, s2}) {
        L.dst.push_back(s);
        key.dst_dtypes.push_back(plan.loc[s].dtype);
      }
      int W1, H1;
      level_dims(plan.W, plan.H, p.stages[s1].level, &W1, &H1);
      level_dims(plan.W, plan.H, p.stages[s2].level, &L.W, &L.H);
      L.block = 32 * key.nw;
      const int64_t wy = (L.H + key.tby - 1) / key.tby;
      L.grid[0] = (unsigned)((W1 + 30 * key.vec - 1) / (30 * key.vec));
      L.grid[1] = (unsigned)((wy + key.nw - 1) / key.nw);
      L.grid[2] = (unsigned)p.stages[s1].channels;
      if (L.grid[1] > 65535 || L.grid[2] > 65535) fail(WT_EUNSUPPORTED, "image too tall for the cascade kernel");
      L.smem = cascade_smem(p, s1, key);
      if (L.smem > 227 * 1024) fail(WT_EUNSUPPORTED, "cascade ring needs more than 227 KB of shared memory");
      L.kname = kernel_name(p, key, false);
      continue;
    } else if (key.chain) {
      const ChainForm cf = chain_form(p, L.stages);
      const int last = L.stages.back();
      key.plain = true;
      key.vec = 1;
      key.nw = 4;
      L.src.push_back(cf.producer);
      L.src_chan.push_back(0);
      key.src_dtypes.push_back(loc_of(cf.producer).dtype);
      L.dst.push_back(last);
      key.dst_dtypes.push_back(plan.loc[last].dtype);
      level_dims(plan.W, plan.H, p.stages[last].level, &L.W, &L.H);
      L.block = 128;
      L.grid[0] = (unsigned)((L.W + 127) / 128);
      L.grid[1] = (unsigned)L.H;
      L.grid[2] = 1;
      if (L.H > 65535) fail(WT_EUNSUPPORTED, "image too tall for the reduction-chain kernel");
      L.smem = 0;
      L.kname = kernel_name(p, key, false);
      continue;
    } else {
      int s = L.stages[0];
      key.plain = true;
      key.vec = 4;
      key.nw = 4;
      for (const PlainSrc &ps : plain_sources(p, s)) {
        int pid = p.stages[s].inputs[ps.slot];
        L.src.push_back(pid);
        L.src_chan.push_back(ps.chan);
        key.src_dtypes.push_back(loc_of(pid).dtype);
      }
      L.dst.push_back(s);
      key.dst_dtypes.push_back(plan.loc[s].dtype);
      key.shared_planes = plain_shares_planes(p, s);
      level_dims(plan.W, plan.H, p.stages[s].level, &L.W, &L.H);
      const int vo = L.params.vec == 8 ? 8 : 4;  // outputs per lane (default 4)
      if (p.sched.exec == WT_EXEC_FUSED && down_streamable(down_form(p, s), vo)) {
        // separable down-sampling: producer rows streamed through warps
        key.down = true;
        key.vec = vo;
        key.tby = std::max(1, L.params.tile_h);
        L.block = 32 * key.nw;
        const int64_t wy = (L.H + key.tby - 1) / key.tby;
        L.grid[0] = (unsigned)((L.W + 32 * vo - 1) / (32 * vo));
        L.grid[1] = (unsigned)((wy + key.nw - 1) / key.nw);
        L.grid[2] = (unsigned)p.stages[s].channels;
        if (L.grid[1] > 65535 || L.grid[2] > 65535) fail(WT_EUNSUPPORTED, "image too tall for the down-sampling kernel");
        L.smem = down_smem(p, s, key);
        if (L.smem > 227 * 1024) fail(WT_EUNSUPPORTED, "down-sampling ring needs more than 227 KB of shared memory");
        L.kname = kernel_name(p, key, false);
        continue;
      }
      L.block = 128;
      L.grid[0] = (unsigned)(((L.W + 7) / 8 + 127) / 128);
      L.grid[1] = (unsigned)L.H;
      L.grid[2] = (unsigned)p.stages[s].channels;
      if (L.H > 65535 || L.grid[2] > 65535) fail(WT_EUNSUPPORTED, "image too tall for the per-stage kernel");
      L.smem = 0;
    }
    L.kname = kernel_name(p, key, L.fused, L.fused && L.geom.n_gather > 0);
  }
  if (!batched) assign_lanes(plan);
  return plan;
}

void assign_lanes(RunPlan &plan) {
  const int n = (int)plan.launches.size();
  bool one = false;
  for (const Launch &L : plan.launches) one = one || L.params.one_stream != 0;
  plan.n_lanes = 1;
  for (Launch &L : plan.launches) {
    L.lane = 0;
    L.waits.clear();
    L.record = false;
  }
  if (one || n < 2) return;
  std::vector<int> tail;  // last launch of each lane
  std::vector<std::vector<int>> vc(n);
  for (int j = 0; j < n; j++) {
    Launch &Lj = plan.launches[j];
    std::vector<int> deps;  // earlier launches writing a stage this one reads
    for (int i = 0; i < j; i++) {
      const std::vector<int> &w = plan.launches[i].dst;
      for (int s : Lj.src)
        if (s >= 0 && std::find(w.begin(), w.end(), s) != w.end()) {
          deps.push_back(i);
          break;
        }
    }
    int lane = -1;
    for (int k = (int)deps.size() - 1; k >= 0 && lane < 0; k--)
      if (tail[plan.launches[deps[k]].lane] == deps[k]) lane = plan.launches[deps[k]].lane;
    if (lane < 0 && (int)tail.size() < kMaxLanes) {
      lane = (int)tail.size();
      tail.push_back(-1);
    }
    if (lane < 0) {
      lane = 0;
      for (int l = 1; l < (int)tail.size(); l++)
        if (tail[l] < tail[lane]) lane = l;
    }
    Lj.lane = lane;
    // vector clock: per lane, the latest launch known complete when this
    // one starts (its lane's previous launch and what that waited for);
    // a dependency already covered needs no wait
    vc[j] = tail[lane] >= 0 ? vc[tail[lane]] : std::vector<int>(kMaxLanes, -1);
    for (int k = (int)deps.size() - 1; k >= 0; k--) {
      const int d = deps[k], l = plan.launches[d].lane;
      if (vc[j][l] >= d) continue;
      Lj.waits.push_back(d);
      plan.launches[d].record = true;
      for (int m = 0; m < kMaxLanes; m++) vc[j][m] = std::max(vc[j][m], vc[d][m]);
    }
    vc[j][lane] = j;
    tail[lane] = j;
  }
  plan.n_lanes = (int)tail.size();
  // side lanes end with an event the caller's stream joins
  for (int l = 1; l < plan.n_lanes; l++) plan.launches[tail[l]].record = true;
}

std::string kernel_name(const Pipeline &p, const CodegenKey &key, bool fused, bool gather) {
  char hx[24];
  // the generator's version is part of the name: a kernel whose code
  // changes gets a new name (profiles and caches never mix versions)
  static const char kCodegenVersion[] = "wt-codegen-22";
  static const char kPlainVersion[] = "wt-plain-2";  // the per-stage kernel's own changes
  static const char kBatchVersion[] = "wt-batch-15";  // the persistent variant's own changes
  const std::string ks = key.str();
  uint64_t h = fnv1a(ks.data(), ks.size(), p.hash);
  h = fnv1a(kCodegenVersion, sizeof kCodegenVersion, h);
  if (key.persistent) h = fnv1a(kBatchVersion, sizeof kBatchVersion, h);
  if (!fused) h = fnv1a(kPlainVersion, sizeof kPlainVersion, h);
  static const char kGatherVersion[] = "wt-gather-4";  // kernels reading other levels
  if (gather) h = fnv1a(kGatherVersion, sizeof kGatherVersion, h);
  static const char kOtptbVersion[] = "wt-otptb-2";  // the block-tile kernel's own changes
  if (key.otptb) h = fnv1a(kOtptbVersion, sizeof kOtptbVersion, h);
  static const char kDownVersion[] = "wt-down-5";  // the down-sampling kernel's own changes
  if (key.down) h = fnv1a(kDownVersion, sizeof kDownVersion, h);
  static const char kChainVersion[] = "wt-chain-1";  // the reduction-chain kernel's own changes
  if (key.chain) h = fnv1a(kChainVersion, sizeof kChainVersion, h);
  static const char kCascadeVersion[] = "wt-cascade-3";  // the two-level down-sampling kernel's own changes
  if (key.cascade) h = fnv1a(kCascadeVersion, sizeof kCascadeVersion, h);
  static const char kVolVersion[] = "wt-vol-7";  // the 3-D group kernel's own changes
  if (key.vol) h = fnv1a(kVolVersion, sizeof kVolVersion, h);
  snprintf(hx, sizeof hx, "%012llx", (unsigned long long)(h & 0xffffffffffffull));
  if (key.otptb) return std::string("wt_otptb_") + hx;
  if (key.down) return std::string("wt_down_") + hx;
  if (key.chain) return std::string("wt_chain_") + hx;
  if (key.cascade) return std::string("wt_down2_") + hx;
  if (key.vol) return std::string("wt_vol_") + hx;
  return std::string(fused ? (key.persistent ? "wt_batch_" : "wt_fused_") : "wt_plain_") + hx;
}

std::string launch_source(const Pipeline &p, const Launch &L) {
  if (L.key.otptb) return emit_otptb(p, L.geom, L.key, L.kname);
  if (L.key.down) return emit_down(p, L.stages[0], L.key, L.kname);
  if (L.key.chain) return emit_chain(p, L.stages, L.key, L.kname);
  if (L.key.cascade) return emit_cascade(p, L.stages[0], L.stages[1], L.key, L.kname);
  if (L.key.vol) return emit_vol(p, L.vol, L.key, L.kname);
  if (L.fused) return emit_fused(p, L.geom, L.key, L.kname);
  return emit_plain(p, L.stages[0], L.key, L.kname);
}

// Fills the argument block of a launch.  `ws` is the workspace base (may be
// null when every source/destination is a caller image).
void fill_args(const Pipeline &p, const RunPlan &plan, const Launch &L, char *ws, KernelArgs &a,
               bool encode_tmaps) {
  memset(&a, 0, sizeof a);
  auto loc_of = [&](int pid) -> const Loc & { return pid >= 0 ? plan.loc[pid] : plan.in_loc[-pid - 1]; };
  auto ptr_of = [&](const Loc &l) -> char * {
    if (l.ws) {
      if (!ws) fail(WT_EUNSUPPORTED, "launch reads or writes the workspace");
      return ws + l.ws_off;
    }
    return (char *)l.ptr;
  };
  for (size_t i = 0; i < L.src.size(); i++) {
    const Loc &l = loc_of(L.src[i]);
    SrcDesc &d = a.src[i];
    d.ptr = ptr_of(l);
    d.W = l.W; d.H = l.H; d.C = l.C; d.dtype = l.dtype; d.pitch = l.pitch; d.plane = l.plane;
    if (L.key.otptb) continue;                    // block tiles: plain loads
    if (L.fused && (int)i >= L.n_ring) continue;  // gather source: plain loads, no tensor map
    if (L.fused && !encode_tmaps) {
      // Introspection only: a plain description of the box in place of the
      // opaque tensor map (layout: struct DebugTmap in wt_internal.hpp).
      DebugTmap t;
      t.ptr = d.ptr; t.W = l.W; t.H = l.H; t.C = l.C; t.esz = elem_bytes(l.dtype);
      t.pitch = l.pitch; t.plane = l.plane;
      t.boxw = L.layout.boxw[i]; t.boxh = L.layout.chunk;
      static_assert(sizeof(DebugTmap) <= sizeof(TmapBytes), "debug tensor map size");
      memcpy(&a.tmap[i], &t, sizeof t);
    }
    if (L.fused && encode_tmaps) {
      const Driver &drv = driver();
      CUtensorMapDataType t = l.dtype == WT_F32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                              : l.dtype == WT_F16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                                  : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
      cuuint64_t dims[3] = {(cuuint64_t)l.W, (cuuint64_t)l.H, (cuuint64_t)l.C};
      cuuint64_t strides[2] = {(cuuint64_t)l.pitch, (cuuint64_t)l.plane};
      cuuint32_t box[3] = {(cuuint32_t)L.layout.boxw[i], (cuuint32_t)L.layout.chunk, 1};
      cuuint32_t es[3] = {1, 1, 1};
      static_assert(sizeof(CUtensorMap) == sizeof(TmapBytes), "tensor map size");
      check_cu(drv.tensorMapEncodeTiled((CUtensorMap *)&a.tmap[i], t, 3, (void *)d.ptr, dims, strides, box,
                                        es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE),
               "cuTensorMapEncodeTiled");
    }
  }
  for (size_t i = 0; i < L.dst.size(); i++) {
    const Loc &l = plan.loc[L.dst[i]];
    DstDesc &d = a.dst[i];
    d.ptr = ptr_of(l);
    d.W = l.W; d.H = l.H; d.C = l.C; d.dtype = l.dtype; d.pitch = l.pitch; d.plane = l.plane;
  }
  a.W = L.W;
  a.H = L.H;
  a.tile_h = std::max(1, L.params.tile_h);
  a.tiles_x = L.tiles_x;
  a.tiles_y = L.tiles_y;
  a.n_tiles = L.n_tiles;
  // one tile height unless split_tiles() assigns a short last round
  a.tile_h2 = a.tile_h;
  a.ty1 = L.tiles_y;
  a.ty2 = 0;
  a.n_big = L.n_tiles;
  a.chunk = L.layout.chunk;
  a.nbuf = L.layout.nbuf;
  a.out_w = L.layout.out_w;
  a.channels = L.fused ? L.geom.channels : (L.key.vol ? L.vol.D : 1);
  (void)p;
}

// ---------------------------------------------------------- kernel cache

struct CacheEntry {
  Kernel k;
  int smem_set = 0;
};
static std::mutex g_cache_mu;
static std::map<std::string, CacheEntry> g_cache;

Kernel &get_kernel(const Pipeline &p, const Launch &L, int device) {
  std::string key = L.kname + "@" + std::to_string(device);
  {
    std::lock_guard<std::mutex> lk(g_cache_mu);
    auto it = g_cache.find(key);
    if (it != g_cache.end()) return it->second.k;
  }
  const Driver &drv = driver();
  std::string src = launch_source(p, L);
  std::string cubin = compile_cubin(src, L.kname, L.key.max_regs);
  CUmodule mod;
  check_cu(drv.moduleLoadData(&mod, cubin.data()), "cuModuleLoadData");
  CUfunction f;
  check_cu(drv.moduleGetFunction(&f, mod, L.kname.c_str()), "cuModuleGetFunction");
  if (L.key.soft_cap) {
    int local = 0;
    drv.funcGetAttribute(&local, CU_FUNC_ATTRIBUTE_LOCAL_SIZE_BYTES, f);
    if (local > 0) {
      // spills under the library's soft register cap: the uncapped kernel
      // serves this launch (kept under both names)
      drv.moduleUnload(mod);
      Launch U = L;
      U.key.max_regs = 0;
      U.key.soft_cap = false;
      U.kname = kernel_name(p, U.key, true, U.geom.n_gather > 0);
      Kernel k = get_kernel(p, U, device);
      std::lock_guard<std::mutex> lk(g_cache_mu);
      CacheEntry e;
      e.k = k;
      auto ins = g_cache.emplace(key, e);
      return ins.first->second.k;
    }
  }
  CacheEntry e;
  e.k.module = mod;
  e.k.function = f;
  e.k.name = L.kname;
  drv.funcGetAttribute(&e.k.regs, CU_FUNC_ATTRIBUTE_NUM_REGS, f);
  drv.funcGetAttribute(&e.k.static_smem, CU_FUNC_ATTRIBUTE_SHARED_SIZE_BYTES, f);
  std::lock_guard<std::mutex> lk(g_cache_mu);
  auto ins = g_cache.emplace(key, e);
  return ins.first->second.k;
}

Kernel *find_kernel(const Pipeline &p, const Launch &L, int device) {
  (void)p;
  std::lock_guard<std::mutex> lk(g_cache_mu);
  auto it = g_cache.find(L.kname + "@" + std::to_string(device));
  return it == g_cache.end() ? nullptr : &it->second.k;
}

void launch(const Launch &L, Kernel &k, KernelArgs &a, cudaStream_t stream) {
  const Driver &drv = driver();
  if (L.smem > 48 * 1024)
    check_cu(drv.funcSetAttribute((CUfunction)k.function, CU_FUNC_ATTRIBUTE_MAX_DYNAMIC_SHARED_SIZE_BYTES,
                                  L.smem),
             "cuFuncSetAttribute");
  void *params[] = {&a};
  check_cu(drv.launchKernel((CUfunction)k.function, L.grid[0], L.grid[1], L.grid[2], (unsigned)L.block, 1, 1,
                            (unsigned)L.smem, (CUstream)stream, params, nullptr),
           "cuLaunchKernel");
}

// ------------------------------------------------ allocation accounting

namespace {
std::atomic<int> g_inject_kind{-1};
std::atomic<int> g_inject_after{-1};
std::atomic<long long> g_device_bytes{0};
std::atomic<long long> g_live_pipelines{0};

// true once for the injected failure: the (after+1)-th point of that kind
bool injected(int kind) {
  if (g_inject_kind.load() != kind) return false;
  if (g_inject_after.fetch_sub(1) != 0) return false;
  g_inject_kind.store(-1);
  return true;
}
}  // namespace

void host_alloc_point() {
  if (injected(kAllocHost)) throw std::bad_alloc();
}

int dev_alloc(void **ptr, size_t bytes) {
  *ptr = nullptr;
  if (injected(kAllocDevice)) return (int)cudaErrorMemoryAllocation;
  cudaError_t rc = cudaMalloc(ptr, bytes);
  if (rc == cudaSuccess) g_device_bytes += (long long)bytes;
  else *ptr = nullptr;
  return (int)rc;
}

void dev_free(void *ptr, size_t bytes) {
  if (!ptr) return;
  cudaFree(ptr);
  g_device_bytes -= (long long)bytes;
}

LiveCounter::LiveCounter() { g_live_pipelines++; }
LiveCounter::~LiveCounter() { g_live_pipelines--; }

void inject_alloc_failure(int kind, int after) {
  g_inject_after.store(after);
  g_inject_kind.store(after < 0 ? -1 : kind);
}

void live_objects(long long *pipelines, long long *device_bytes) {
  if (pipelines) *pipelines = g_live_pipelines.load();
  if (device_bytes) *device_bytes = g_device_bytes.load();
}

// ------------------------------------------------------------- workspace

void Workspace::clear_host_graphs() {
  for (auto &kv : host_graphs)
    if (kv.second) cudaGraphExecDestroy(kv.second);
  host_graphs.clear();
}

Workspace::~Workspace() {
  clear_host_graphs();
  dev_free(base, (size_t)bytes);
  dev_free(err, kCtrlBytes);
  for (auto &kv : staging) dev_free(kv.second.ptr, (size_t)kv.second.bytes);
  for (cudaStream_t s : band_stream)
    if (s) cudaStreamDestroy(s);
  for (cudaEvent_t e : band_events) cudaEventDestroy(e);
  for (cudaStream_t s : lane_stream)
    if (s) cudaStreamDestroy(s);
  if (fork_event) cudaEventDestroy(fork_event);
  for (cudaEvent_t e : launch_events) cudaEventDestroy(e);
}

Workspace &workspace(Pipeline &p, int64_t bytes) {
  int dev = 0;
  check_rt(cudaGetDevice(&dev), "cudaGetDevice");
  if (!p.ws || p.ws->device != dev) {
    auto w = std::make_shared<Workspace>();
    w->device = dev;
    // control block: error word at [0], then two tile-queue counters per
    // launch of a plan (zero between launches: the kernels reset them)
    if (dev_alloc((void **)&w->err, kCtrlBytes) != cudaSuccess) {
      cudaGetLastError();
      fail(WT_ENOMEM, "cannot allocate the device control block");
    }
    check_rt(cudaMemset(w->err, 0, kCtrlBytes), "cudaMemset");
    p.ws = w;
  }
  Workspace &w = *p.ws;
  if (bytes > w.bytes) {
    if (w.base) {
      check_rt(cudaDeviceSynchronize(), "cudaDeviceSynchronize");
      dev_free(w.base, (size_t)w.bytes);
      w.base = nullptr;
      w.bytes = 0;
    }
    if (dev_alloc((void **)&w.base, (size_t)bytes) != cudaSuccess) {
      cudaGetLastError();
      fail(WT_ENOMEM, "cannot allocate " + std::to_string(bytes) + " bytes of workspace");
    }
    w.bytes = bytes;
    w.generation++;
  }
  return w;
}

// Two-level tile heights (load balance of the persistent warps): the last
// round of tiles handed out is short, about one tile per resident warp, so
// warps finish within one short tile of each other.  The short tiles form a
// band of ty2 rows of tile_h2 at the top of the image, the tall tiles the
// ty1 rows below it (the last one clipped by the image).
void split_tiles(const Launch &L, KernelArgs &a, int resident_warps) {
  const int T1 = std::max(1, L.params.tile_h);
  // tiles of groups folding the row parity start on even rows: even heights
  const int T2 = std::max(4, L.key.even_rows ? T1 / 2 / 2 * 2 : T1 / 2);
  if (!L.fused || T2 >= T1 || L.params.tile_split == 0) return;
  const int C = L.geom.channels;
  const int per_row = std::max(1, L.tiles_x * C);
  const int ty2 = (resident_warps + per_row - 1) / per_row;
  if (L.H - ty2 * T2 < T1) return;  // too small to split
  const int ty1 = (L.H - ty2 * T2 + T1 - 1) / T1;
  a.tile_h2 = T2;
  a.ty1 = ty1;
  a.ty2 = ty2;
  a.n_big = L.tiles_x * ty1 * C;
  a.n_tiles = a.n_big + L.tiles_x * ty2 * C;
}

int32_t *queue_counters(int32_t *ctrl, int launch_index) {
  return ctrl + kCtrlQueueOffset / 4 + 2 * launch_index;
}

static std::string cache_key(const wt_image *in, int n_in, const wt_image *out, int n_out) {
  std::string k((const char *)in, sizeof(wt_image) * n_in);
  k.append((const char *)out, sizeof(wt_image) * n_out);
  return k;
}

// Per-launch set-up that every path launching a plan shares: a warp-tile
// kernel (persistent warps) gets no more blocks than can be resident at
// once, its tensor maps and its two-level tile split; a block-tile kernel
// keeps one block per tile.  Then the status word and the launch's queue
// counters.
KernelArgs launch_args(Pipeline &p, const RunPlan &plan, Launch &L, Kernel &k, char *ws, int32_t *err, int li,
                       int dev) {
  const bool persistent = L.fused && !L.key.otptb;
  if (L.fused) {
    const Driver &drv = driver();
    if (L.smem > 48 * 1024)
      check_cu(drv.funcSetAttribute((CUfunction)k.function, CU_FUNC_ATTRIBUTE_MAX_DYNAMIC_SHARED_SIZE_BYTES,
                                    L.smem),
               "cuFuncSetAttribute");
    int per_sm = 0, sms = 0;
    check_cu(drv.occupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (CUfunction)k.function, L.block,
                                                           (size_t)L.smem),
             "cuOccupancyMaxActiveBlocksPerMultiprocessor");
    check_rt(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "cudaDeviceGetAttribute");
    if (per_sm < 1) fail(WT_EUNSUPPORTED, "group kernel cannot be resident (registers/shared memory)");
    // one warp per tile in block-index order, or (tile queue) no more
    // blocks than can be resident at once
    if (persistent && L.params.tile_queue) L.grid[0] = std::min<unsigned>(L.grid[0], (unsigned)(per_sm * sms));
    L.resident_blocks_per_sm = per_sm;
    L.resident_warps = per_sm * sms * L.key.nw;
  }
  KernelArgs a;
  fill_args(p, plan, L, ws, a, persistent);
  if (persistent) {
    split_tiles(L, a, L.resident_warps);
    a.direct = L.params.tile_queue ? 0 : 1;
    // one warp per tile: the grid covers every tile of the split
    if (a.direct) L.grid[0] = (unsigned)((a.n_tiles + L.key.nw - 1) / L.key.nw);
  }
  a.err = err;
  a.queue = queue_counters(err, li);
  return a;
}

// Streams and events of a run on `n_lanes` lanes with `n` launches; false
// if they cannot be made now (the caller's stream is being captured: the
// run then goes on one stream).
static bool lanes_ready(Workspace &w, cudaStream_t user, int n_lanes, int n) {
  bool have = w.fork_event != nullptr && (int)w.launch_events.size() >= n;
  for (int l = 1; l < n_lanes; l++) have = have && w.lane_stream[l - 1] != nullptr;
  if (have) return true;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  check_rt(cudaStreamIsCapturing(user, &cs), "cudaStreamIsCapturing");
  if (cs != cudaStreamCaptureStatusNone) return false;
  for (int l = 1; l < n_lanes; l++)
    if (!w.lane_stream[l - 1])
      check_rt(cudaStreamCreateWithFlags(&w.lane_stream[l - 1], cudaStreamNonBlocking), "cudaStreamCreate");
  if (!w.fork_event) check_rt(cudaEventCreateWithFlags(&w.fork_event, cudaEventDisableTiming), "cudaEventCreate");
  while ((int)w.launch_events.size() < n) {
    cudaEvent_t e;
    check_rt(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "cudaEventCreate");
    w.launch_events.push_back(e);
  }
  return true;
}

// Issues a run's launches on their lanes: lane 0 is the caller's stream,
// lanes 1.. the workspace's side streams, which wait for the fork event
// (everything the caller queued before the run) before their first launch;
// each launch first waits for the events of its dependencies on other
// lanes; the caller's stream finally waits for every side lane's last
// launch.  launch_on(i, stream) issues launch i.
template <class F>
static void issue_lanes(Workspace &w, cudaStream_t user, int n_lanes, const std::vector<int> &lane,
                        const std::vector<std::vector<int>> &waits, const std::vector<char> &record, F &&launch_on) {
  const int n = (int)lane.size();
  if (n_lanes <= 1 || !lanes_ready(w, user, n_lanes, n)) {
    for (int i = 0; i < n; i++) launch_on(i, user);
    return;
  }
  check_rt(cudaEventRecord(w.fork_event, user), "cudaEventRecord");
  bool forked[kMaxLanes] = {};
  int last[kMaxLanes];
  for (int l = 0; l < kMaxLanes; l++) last[l] = -1;
  for (int i = 0; i < n; i++) {
    const int l = lane[i];
    cudaStream_t s = l == 0 ? user : w.lane_stream[l - 1];
    if (l != 0 && !forked[l]) {
      check_rt(cudaStreamWaitEvent(s, w.fork_event, 0), "cudaStreamWaitEvent");
      forked[l] = true;
    }
    for (int d : waits[i]) check_rt(cudaStreamWaitEvent(s, w.launch_events[d], 0), "cudaStreamWaitEvent");
    launch_on(i, s);
    if (record[i]) check_rt(cudaEventRecord(w.launch_events[i], s), "cudaEventRecord");
    last[l] = i;
  }
  for (int l = 1; l < n_lanes; l++)
    if (last[l] >= 0) check_rt(cudaStreamWaitEvent(user, w.launch_events[last[l]], 0), "cudaStreamWaitEvent");
}

void run_plan(Pipeline &p, RunPlan &plan, cudaStream_t stream, const std::string *key) {
  Workspace &w = workspace(p, plan.ws_bytes);
  int dev = w.device;
  CachedRun c;
  if ((int)plan.launches.size() > kMaxLaunches) fail(WT_EUNSUPPORTED, "more than 500 launches per run");
  // load every kernel and set up every launch before issuing any
  std::vector<Kernel *> ks;
  int li = 0;
  for (Launch &L : plan.launches) {
    Kernel &k = get_kernel(p, L, dev);
    KernelArgs a = launch_args(p, plan, L, k, w.base, w.err, li++, dev);
    ks.push_back(&k);
    c.functions.push_back(k.function);
    c.args.push_back(a);
    c.grid.insert(c.grid.end(), {L.grid[0], L.grid[1], L.grid[2]});
    c.block.push_back(L.block);
    c.smem.push_back(L.smem);
    c.lane.push_back(L.lane);
    c.waits.push_back(L.waits);
    c.record.push_back(L.record ? 1 : 0);
  }
  c.n_lanes = plan.n_lanes;
  issue_lanes(w, stream, c.n_lanes, c.lane, c.waits, c.record,
              [&](int i, cudaStream_t s) { launch(plan.launches[i], *ks[i], c.args[i], s); });
  if (!key) return;
  RunCache &rc = p.cache;
  if (rc.device != dev || rc.sched_version != p.sched_version || rc.ws_generation != w.generation) {
    rc.runs.clear();
    rc.device = dev;
    rc.sched_version = p.sched_version;
    rc.ws_generation = w.generation;
  }
  if (rc.runs.size() >= 256) rc.runs.clear();
  rc.runs[*key] = std::move(c);
}

const CachedRun *cached_run(const Pipeline &p, const wt_image *in, int n_in, const wt_image *out, int n_out) {
  int dev = 0;
  check_rt(cudaGetDevice(&dev), "cudaGetDevice");
  const RunCache &rc = p.cache;
  if (!(in && out && n_in >= 1 && n_out >= 1 && n_in <= 64 && n_out <= 64)) return nullptr;
  if (rc.device != dev || rc.sched_version != p.sched_version || !p.ws || p.ws->device != dev ||
      rc.ws_generation != p.ws->generation)
    return nullptr;
  auto it = rc.runs.find(cache_key(in, n_in, out, n_out));
  return it == rc.runs.end() ? nullptr : &it->second;
}

void run(Pipeline &p, const wt_image *in, int n_in, const wt_image *out, int n_out, cudaStream_t stream) {
  int dev = 0;
  check_rt(cudaGetDevice(&dev), "cudaGetDevice");
  RunCache &rc = p.cache;
  std::string key;
  if (in && out && n_in >= 1 && n_out >= 1 && n_in <= 64 && n_out <= 64) {
    key = cache_key(in, n_in, out, n_out);
    if (rc.device == dev && rc.sched_version == p.sched_version && p.ws && p.ws->device == dev &&
        rc.ws_generation == p.ws->generation) {
      auto it = rc.runs.find(key);
      if (it != rc.runs.end()) {
        const Driver &drv = driver();
        CachedRun &c = it->second;
        issue_lanes(*p.ws, stream, c.n_lanes, c.lane, c.waits, c.record, [&](int i, cudaStream_t s) {
          void *params[] = {&c.args[i]};
          check_cu(drv.launchKernel((CUfunction)c.functions[i], c.grid[3 * i], c.grid[3 * i + 1],
                                    c.grid[3 * i + 2], (unsigned)c.block[i], 1, 1, (unsigned)c.smem[i],
                                    (CUstream)s, params, nullptr),
                   "cuLaunchKernel");
        });
        return;
      }
    }
  }
  RunPlan plan = build_plan(p, in, n_in, out, n_out);
  run_plan(p, plan, stream, key.empty() ? nullptr : &key);
}

}  // namespace wt

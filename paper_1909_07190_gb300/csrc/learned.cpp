// Learned cost model: the analytic cost of Alg. 2 is a hand-weighted sum
// whose weights need fitting per GPU (Sec. 6, Table 3).  Here a 3-layer FP32
// MLP (features -> 64 -> 64 -> 1, ReLU) predicts the log runtime of one
// launch -- a fused group, or one stage's per-stage kernel -- from
// quantities the method already computes: image size, stage and node
// counts, operations and bytes per pixel, footprint growth, tile shape,
// register and shared-memory use, Alg. 2 occupancy, redundant-compute and
// tail fractions.  It is trained on launch times measured by the library
// itself (wt_schedule_time_launches) with the hand-written kernels of
// mlp.cu; a schedule's predicted time is the sum over its launches and
// DP-Fusion minimises it.  Without a trained model, schedules come from the
// analytic model.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <mutex>
#include <set>
#include <sstream>

#include "wt_jit.hpp"
#include "wt_learned.hpp"
#include "wt_mlp.hpp"
#include "wt_sched.hpp"

namespace wt {

// ------------------------------------------------------------ features

static int prog_len(const Stage &s) { return (int)s.ops.size(); }

bool launch_features(const Pipeline &p, const std::vector<int> &seg, const GroupParams &prm, bool fused, int W0,
                     int H0, int dtype, const GpuConfig &cfg, const std::vector<StageStats> &st, float *f) {
  std::fill(f, f + kMlpFeatures, 0.f);
  const int level = p.stages[seg[0]].level;
  int Wl, Hl;
  level_dims(W0, H0, level, &Wl, &Hl);
  int C = 1;
  for (int s : seg) C = std::max(C, p.stages[s].channels);
  f[0] = (float)std::log2((double)Wl * Hl * C);
  f[1] = (float)seg.size();
  if (fused) {
    const int V = prm.vec ? prm.vec : 4;
    GroupGeom g = analyze_group(p, seg, V, prm.frac_reg, 4);
    if (!g.fusable) return false;
    // the tile height the run will use (shortened for small images)
    GroupParams prm_in = prm;
    {
      const int lp = V * ((g.halo_l + V - 1) / V), rp = V * ((g.halo_r + V - 1) / V);
      const int ow = std::max(V, 32 * V - lp - rp);
      prm_in.tile_h = effective_tile_h(prm.tile_h, Hl, (Wl + ow - 1) / ow, g.channels, g);
    }
    const GroupParams &prm = prm_in;
    CostInfo ci = cost_group(p, seg, prm, 128, W0, H0, dtype, cfg, st, current_weights(),
                             pipeline_bytes(p, W0, H0, dtype), &g);
    if (!ci.feasible) return false;
    int nodes = 0, ops = 0, nsrc = 0;
    for (const Node &n : g.nodes) {
      if (n.is_source) {
        nsrc++;
        continue;
      }
      nodes++;
      ops += (int)n.prog.size();
    }
    const int esz = elem_bytes(dtype);
    f[2] = (float)nodes;
    f[3] = (float)ops;
    f[4] = (float)(nsrc * esz);
    f[5] = (float)(g.liveouts.size() * esz);
    f[6] = (float)(g.halo_t + g.halo_b);
    f[7] = (float)(g.halo_l + g.halo_r);
    f[8] = (float)std::log2((double)std::max(1, prm.tile_h));
    f[9] = (float)V;
    f[10] = (float)prm.warps_per_block;
    f[11] = prm.frac_reg;
    f[12] = ci.regs / 255.f;
    f[13] = ci.smem_per_tb / (227.f * 1024.f);
    f[14] = (float)ci.occupancy;
    f[15] = (float)ci.t[5];
    f[16] = (float)ci.t[6];
    f[17] = 1.f;
    return true;
  }
  if (seg.size() != 1) return false;
  const int s = seg[0];
  const Stage &S = p.stages[s];
  int in_b = 0, ey = 0, ex = 0;
  for (const Edge &e : S.edges) {
    in_b += (int)e.chans.size() * 4;
    ey = std::max(ey, e.dymax - e.dymin);
    ex = std::max(ex, e.dxmax - e.dxmin);
  }
  const double blocks = std::ceil(std::ceil(Wl / 4.0) / 128.0) * Hl * S.channels;
  const double waves = blocks / ((double)cfg.nsms * std::max(1, cfg.max_th_per_sm / 128));
  f[2] = 1.f;
  f[3] = (float)prog_len(S);
  f[4] = (float)in_b;
  f[5] = (float)(S.channels * 4);
  f[6] = (float)ey;
  f[7] = (float)ex;
  f[8] = 0.f;
  f[9] = 4.f;
  f[10] = 4.f;
  f[11] = 1.f;
  f[12] = std::min(255, st[s].regs) / 255.f;
  f[13] = 0.f;
  f[14] = 1.f;
  f[15] = 0.f;
  f[16] = (float)((std::ceil(waves) - waves) / std::max(1.0, std::ceil(waves)));
  f[17] = 0.f;
  return true;
}

// --------------------------------------------------------------- model

namespace {

struct Model {
  bool ready = false;
  float mean[kMlpFeatures], sd[kMlpFeatures];
  float ymean = 0, ysd = 1;
  std::vector<float> params;
};
std::mutex g_mu;
Model g_model;

// splitmix64 (Steele, Lea & Flood 2014) for weight initialisation and the
// mini-batch order
uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
struct Rng {
  uint64_t s;
  uint64_t next() { return mix64(s += 0x9E3779B97F4A7C15ull); }
  double uniform() { return (next() >> 11) * (1.0 / 9007199254740992.0); }
  double normal() {  // Box-Muller
    double u1 = std::max(uniform(), 1e-300), u2 = uniform();
    return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
  }
};

struct DevBuf {
  void *p = nullptr;
  size_t bytes = 0;
  explicit DevBuf(size_t n) : bytes(n) {
    if (n && dev_alloc(&p, n) != cudaSuccess) {
      cudaGetLastError();
      fail(WT_ENOMEM, "cannot allocate " + std::to_string(n) + " bytes for the cost model");
    }
  }
  ~DevBuf() { dev_free(p, bytes); }
  float *f() const { return (float *)p; }
  int *i() const { return (int *)p; }
};

}  // namespace

void mlp_train_steps(float *params, float *m, float *v, int t0, const float *x, const float *y, int n,
                     const int32_t *idx, int steps, int batch, float lr, float wd, float *loss, cudaStream_t s) {
  if (batch < 1 || batch > kMlpMaxBatch) fail(WT_EINVAL, "batch must be in [1, 128]");
  if (n < 1 || steps < 0) fail(WT_EINVAL, "bad sample or step count");
  for (int64_t k = 0; k < (int64_t)steps * batch; k++)
    if (idx[k] < 0 || idx[k] >= n) fail(WT_EINVAL, "mini-batch index out of range");
  DevBuf P(sizeof(float) * kMlpParams), M(sizeof(float) * kMlpParams), V(sizeof(float) * kMlpParams);
  DevBuf X(sizeof(float) * (size_t)n * kMlpFeatures), Y(sizeof(float) * n);
  DevBuf I(sizeof(int) * (size_t)std::max(1, steps) * batch), L(sizeof(float) * std::max(1, steps));
  check_rt(cudaMemcpyAsync(P.p, params, sizeof(float) * kMlpParams, cudaMemcpyHostToDevice, s), "cudaMemcpyAsync");
  check_rt(cudaMemcpyAsync(M.p, m, sizeof(float) * kMlpParams, cudaMemcpyHostToDevice, s), "cudaMemcpyAsync");
  check_rt(cudaMemcpyAsync(V.p, v, sizeof(float) * kMlpParams, cudaMemcpyHostToDevice, s), "cudaMemcpyAsync");
  check_rt(cudaMemcpyAsync(X.p, x, sizeof(float) * (size_t)n * kMlpFeatures, cudaMemcpyHostToDevice, s),
           "cudaMemcpyAsync");
  check_rt(cudaMemcpyAsync(Y.p, y, sizeof(float) * n, cudaMemcpyHostToDevice, s), "cudaMemcpyAsync");
  if (steps > 0)
    check_rt(cudaMemcpyAsync(I.p, idx, sizeof(int) * (size_t)steps * batch, cudaMemcpyHostToDevice, s),
             "cudaMemcpyAsync");
  // launches of at most 512 steps (one block each; the state stays on the
  // device between them)
  for (int s0 = 0; s0 < steps; s0 += 512) {
    const int k = std::min(512, steps - s0);
    check_rt(mlp_train_launch(P.f(), M.f(), V.f(), t0 + s0, X.f(), Y.f(), I.i() + (size_t)s0 * batch, k, batch, lr,
                              0.9f, 0.999f, 1e-8f, wd, L.f() + s0, s),
             "mlp training kernel");
  }
  check_rt(cudaMemcpyAsync(params, P.p, sizeof(float) * kMlpParams, cudaMemcpyDeviceToHost, s), "cudaMemcpyAsync");
  check_rt(cudaMemcpyAsync(m, M.p, sizeof(float) * kMlpParams, cudaMemcpyDeviceToHost, s), "cudaMemcpyAsync");
  check_rt(cudaMemcpyAsync(v, V.p, sizeof(float) * kMlpParams, cudaMemcpyDeviceToHost, s), "cudaMemcpyAsync");
  if (loss && steps > 0)
    check_rt(cudaMemcpyAsync(loss, L.p, sizeof(float) * steps, cudaMemcpyDeviceToHost, s), "cudaMemcpyAsync");
  check_rt(cudaStreamSynchronize(s), "cudaStreamSynchronize");
}

void mlp_forward(const float *params, const float *x, int n, float *y, cudaStream_t s) {
  if (n < 0) fail(WT_EINVAL, "bad sample count");
  if (n == 0) return;
  DevBuf P(sizeof(float) * kMlpParams), X(sizeof(float) * (size_t)n * kMlpFeatures), Y(sizeof(float) * n);
  check_rt(cudaMemcpyAsync(P.p, params, sizeof(float) * kMlpParams, cudaMemcpyHostToDevice, s), "cudaMemcpyAsync");
  check_rt(cudaMemcpyAsync(X.p, x, sizeof(float) * (size_t)n * kMlpFeatures, cudaMemcpyHostToDevice, s),
           "cudaMemcpyAsync");
  check_rt(mlp_forward_launch(P.f(), X.f(), n, Y.f(), s), "mlp inference kernel");
  check_rt(cudaMemcpyAsync(y, Y.p, sizeof(float) * n, cudaMemcpyDeviceToHost, s), "cudaMemcpyAsync");
  check_rt(cudaStreamSynchronize(s), "cudaStreamSynchronize");
}

float costmodel_train(const float *features, const float *log_ms, int n, int epochs, int batch, float lr,
                      uint64_t seed) {
  if (n < 2 || epochs < 1) fail(WT_EINVAL, "need at least 2 samples and 1 epoch");
  if (batch < 1 || batch > kMlpMaxBatch) fail(WT_EINVAL, "batch must be in [1, 128]");
  Model md;
  // standardise features and targets over the training set
  for (int f = 0; f < kMlpFeatures; f++) {
    double s = 0, s2 = 0;
    for (int i = 0; i < n; i++) s += features[(size_t)i * kMlpFeatures + f];
    const double mu = s / n;
    for (int i = 0; i < n; i++) {
      const double d = features[(size_t)i * kMlpFeatures + f] - mu;
      s2 += d * d;
    }
    const double sd = std::sqrt(s2 / n);
    md.mean[f] = (float)mu;
    md.sd[f] = sd > 1e-6 ? (float)sd : 1.f;
  }
  {
    double s = 0, s2 = 0;
    for (int i = 0; i < n; i++) s += log_ms[i];
    const double mu = s / n;
    for (int i = 0; i < n; i++) s2 += (log_ms[i] - mu) * (log_ms[i] - mu);
    md.ymean = (float)mu;
    md.ysd = std::sqrt(s2 / n) > 1e-6 ? (float)std::sqrt(s2 / n) : 1.f;
  }
  std::vector<float> X((size_t)n * kMlpFeatures), Y(n);
  for (int i = 0; i < n; i++) {
    for (int f = 0; f < kMlpFeatures; f++)
      X[(size_t)i * kMlpFeatures + f] = (features[(size_t)i * kMlpFeatures + f] - md.mean[f]) / md.sd[f];
    Y[i] = (log_ms[i] - md.ymean) / md.ysd;
  }
  // He initialisation of the weights, zero biases
  Rng rng{seed};
  md.params.assign(kMlpParams, 0.f);
  const int F = kMlpFeatures, H = kMlpHidden;
  for (int q = 0; q < H * F; q++) md.params[q] = (float)(rng.normal() * std::sqrt(2.0 / F));
  for (int q = 0; q < H * H; q++) md.params[H * F + H + q] = (float)(rng.normal() * std::sqrt(2.0 / H));
  for (int q = 0; q < H; q++) md.params[H * F + H + H * H + H + q] = (float)(rng.normal() * std::sqrt(1.0 / H));
  // mini-batches: a fresh permutation per epoch
  const int per_epoch = (n + batch - 1) / batch;
  const int steps = epochs * per_epoch;
  std::vector<int32_t> idx((size_t)steps * batch);
  std::vector<int32_t> perm(n);
  for (int e = 0; e < epochs; e++) {
    for (int i = 0; i < n; i++) perm[i] = i;
    for (int i = n - 1; i > 0; i--) std::swap(perm[i], perm[rng.next() % (uint64_t)(i + 1)]);
    for (int k = 0; k < per_epoch * batch; k++) idx[(size_t)e * per_epoch * batch + k] = perm[k % n];
  }
  std::vector<float> m(kMlpParams, 0.f), v(kMlpParams, 0.f), loss(steps);
  mlp_train_steps(md.params.data(), m.data(), v.data(), 0, X.data(), Y.data(), n, idx.data(), steps, batch, lr,
                  1e-4f, loss.data(), nullptr);
  md.ready = true;
  float last = 0;
  const int tail = std::min(steps, per_epoch);
  for (int k = steps - tail; k < steps; k++) last += loss[k] / tail;
  std::lock_guard<std::mutex> lk(g_mu);
  g_model = md;
  return last;
}

bool costmodel_ready() {
  std::lock_guard<std::mutex> lk(g_mu);
  return g_model.ready;
}

void costmodel_predict(const float *features, int n, float *log_ms, cudaStream_t s) {
  Model md;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    md = g_model;
  }
  if (!md.ready) fail(WT_EUNSUPPORTED, "no learned cost model (train or load one)");
  std::vector<float> X((size_t)n * kMlpFeatures);
  for (int i = 0; i < n; i++)
    for (int f = 0; f < kMlpFeatures; f++)
      X[(size_t)i * kMlpFeatures + f] = (features[(size_t)i * kMlpFeatures + f] - md.mean[f]) / md.sd[f];
  mlp_forward(md.params.data(), X.data(), n, log_ms, s);
  for (int i = 0; i < n; i++) log_ms[i] = log_ms[i] * md.ysd + md.ymean;
}

void costmodel_reset() {
  std::lock_guard<std::mutex> lk(g_mu);
  g_model = Model();
}

void costmodel_save(const std::string &path) {
  Model md;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    md = g_model;
  }
  if (!md.ready) fail(WT_EUNSUPPORTED, "no learned cost model to save");
  std::ofstream o(path);
  if (!o) fail(WT_EINVAL, "cannot write " + path);
  o << "wt-mlp 1 " << kMlpFeatures << " " << kMlpHidden << "\n";
  char b[32];
  auto put = [&](float x) {
    snprintf(b, sizeof b, "%.9g ", x);
    o << b;
  };
  for (int f = 0; f < kMlpFeatures; f++) put(md.mean[f]);
  o << "\n";
  for (int f = 0; f < kMlpFeatures; f++) put(md.sd[f]);
  o << "\n";
  put(md.ymean);
  put(md.ysd);
  o << "\n";
  for (int q = 0; q < kMlpParams; q++) put(md.params[q]);
  o << "\n";
  if (!o) fail(WT_EINVAL, "cannot write " + path);
}

void costmodel_load(const std::string &path) {
  std::ifstream in(path);
  if (!in) fail(WT_EINVAL, "cannot read " + path);
  std::string tag;
  int ver = 0, nf = 0, nh = 0;
  in >> tag >> ver >> nf >> nh;
  if (tag != "wt-mlp" || ver != 1 || nf != kMlpFeatures || nh != kMlpHidden)
    fail(WT_EINVAL, path + ": not a cost model of this library version");
  Model md;
  for (int f = 0; f < kMlpFeatures; f++) in >> md.mean[f];
  for (int f = 0; f < kMlpFeatures; f++) in >> md.sd[f];
  in >> md.ymean >> md.ysd;
  md.params.resize(kMlpParams);
  for (int q = 0; q < kMlpParams; q++) in >> md.params[q];
  if (!in) fail(WT_EINVAL, path + ": truncated cost model");
  md.ready = true;
  std::lock_guard<std::mutex> lk(g_mu);
  g_model = md;
}

// --------------------------------------------------- DP-Fusion, learned

// Every candidate launch of every contiguous segment (the analytic search
// space, plus the per-stage kernel of single stages) is scored in one
// batched inference; a segment costs its best candidate's predicted time
// and the DP minimises the schedule's predicted time.
Schedule learned_schedule(const Pipeline &p, int W, int H, int dtype, const GpuConfig &cfg,
                          const std::vector<StageStats> &st, int max_group) {
  const int n = (int)p.stages.size();
  struct Cand {
    int i, j;  // segment [i, j)
    bool fused;
    GroupParams prm;
  };
  std::vector<Cand> cands;
  std::vector<float> feats;
  float fv[kMlpFeatures];
  // reduction chains and down-sampling cascades across levels (no
  // features: the model was trained on warp-tile and per-stage launches):
  // their traffic at the device's copy bandwidth, in ms
  std::vector<std::pair<std::pair<int, int>, double>> chains;
  for (int j = 1; j <= n; j++)
    for (int i = std::max(0, j - max_group); i < j; i++) {
      std::vector<int> seg;
      for (int s = i; s < j; s++) seg.push_back(s);
      if (chain_form(p, seg).ok)
        chains.push_back({{i, j}, chain_bytes(p, seg, W, H) / cfg.glmem_bw * 1e3});
      else if (!cascade_units(p, seg).empty())
        chains.push_back({{i, j}, cascade_bytes(p, seg, W, H) / cfg.glmem_bw * 1e3});
    }
  for (int j = 1; j <= n; j++)
    for (int i = std::max(0, j - max_group); i < j; i++) {
      std::vector<int> seg;
      for (int s = i; s < j; s++) seg.push_back(s);
      if (seg.size() == 1 && launch_features(p, seg, GroupParams(), false, W, H, dtype, cfg, st, fv)) {
        cands.push_back({i, j, false, GroupParams()});
        feats.insert(feats.end(), fv, fv + kMlpFeatures);
      }
      for (int V : {4, 8}) {
        std::set<std::vector<char>> seen;
        for (int fi = 10; fi >= 0; fi -= 5) {
          GroupGeom g = analyze_group(p, seg, V, fi / 10.f, 4);
          if (!g.fusable) break;
          std::vector<char> sig;
          for (const Node &nd : g.nodes) sig.push_back(nd.in_smem);
          if (!seen.insert(sig).second) continue;
          for (int T : {8, 16, 24, 32, 40, 56})
            for (int nw : {1, 2}) {
              GroupParams q;
              q.tile_h = T;
              q.warps_per_block = nw;
              q.vec = V;
              q.frac_reg = fi / 10.f;
              if (!launch_features(p, seg, q, true, W, H, dtype, cfg, st, fv)) continue;
              cands.push_back({i, j, true, q});
              feats.insert(feats.end(), fv, fv + kMlpFeatures);
            }
        }
      }
    }
  std::vector<float> pred(cands.size());
  costmodel_predict(feats.data(), (int)cands.size(), pred.data(), nullptr);
  // best candidate per segment
  std::vector<std::vector<double>> seg_cost(n + 1, std::vector<double>(n + 1, INFINITY));
  std::vector<std::vector<int>> seg_best(n + 1, std::vector<int>(n + 1, -1));
  for (size_t k = 0; k < cands.size(); k++) {
    const double t = std::exp((double)pred[k]);
    if (t < seg_cost[cands[k].i][cands[k].j]) {
      seg_cost[cands[k].i][cands[k].j] = t;
      seg_best[cands[k].i][cands[k].j] = (int)k;
    }
  }
  for (auto &c : chains) {
    const int i = c.first.first, j = c.first.second;
    if (c.second < seg_cost[i][j]) {
      seg_cost[i][j] = c.second;
      seg_best[i][j] = (int)cands.size();  // a chain or cascade: installed as a fused group
      cands.push_back({i, j, true, GroupParams()});
    }
  }
  std::vector<double> best(n + 1, INFINITY);
  std::vector<int> from(n + 1, -1);
  best[0] = 0;
  for (int j = 1; j <= n; j++)
    for (int i = std::max(0, j - max_group); i < j; i++)
      if (std::isfinite(best[i]) && best[i] + seg_cost[i][j] < best[j]) {
        best[j] = best[i] + seg_cost[i][j];
        from[j] = i;
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
    const Cand &c = cands[seg_best[segs[g].first][segs[g].second]];
    GroupParams q = c.prm;
    if (!c.fused) {
      q = GroupParams();
      q.plain = 1;
    }
    s.params.push_back(q);
  }
  s.installed = true;
  s.predicted_cost = best[n];
  return s;
}

}  // namespace wt

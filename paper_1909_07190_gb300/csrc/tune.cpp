// Measured schedule search: the grouping and tile search of the method with
// device timings of candidate schedules in place of (or after) the cost
// model's estimates.
//
// Timing protocol (Sec. 7): kernel time only, 3 samples of `reps`
// back-to-back runs on the caller's stream, the minimum of the sample
// means.  Candidate kernels are compiled in parallel host threads first.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <set>
#include <thread>

#include "wt_jit.hpp"
#include "wt_runtime.hpp"
#include "wt_sched.hpp"
#include "wt_tune.hpp"

namespace wt {

namespace {

struct Runner {
  Pipeline &p;
  const wt_image *in;
  int n_in;
  const wt_image *out;
  int n_out;
  int n_images;  // >= 1: batched run of n_images images; 0: one run
  cudaStream_t s;
  void once() const {
    if (n_images >= 1) run_batch(p, in, out, n_images, s);
    else run(p, in, n_in, out, n_out, s);
  }
};

}  // namespace

double time_installed(Pipeline &p, const wt_image *in, int n_in, const wt_image *out, int n_out, int n_images,
                      cudaStream_t s, int reps) {
  Runner r{p, in, n_in, out, n_out, n_images, s};
  r.once();  // plans, compiles, uploads tables
  r.once();
  check_rt(cudaStreamSynchronize(s), "cudaStreamSynchronize");
  cudaEvent_t e0, e1;
  check_rt(cudaEventCreate(&e0), "cudaEventCreate");
  check_rt(cudaEventCreate(&e1), "cudaEventCreate");
  double best = INFINITY;
  for (int t = 0; t < 3; t++) {
    check_rt(cudaEventRecord(e0, s), "cudaEventRecord");
    for (int i = 0; i < reps; i++) r.once();
    check_rt(cudaEventRecord(e1, s), "cudaEventRecord");
    check_rt(cudaEventSynchronize(e1), "cudaEventSynchronize");
    float ms = 0;
    check_rt(cudaEventElapsedTime(&ms, e0, e1), "cudaEventElapsedTime");
    best = std::min(best, (double)ms / reps);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  // a run that raised the device error word (a wait that gave up) does not count
  int32_t word = 0;
  if (p.ws && p.ws->err) {
    check_rt(cudaMemcpy(&word, p.ws->err, 4, cudaMemcpyDeviceToHost), "cudaMemcpy(error word)");
    if (word != 0) {
      check_rt(cudaMemset(p.ws->err, 0, 4), "cudaMemset");
      return INFINITY;
    }
  }
  return best;
}

std::vector<LaunchTime> time_launches(Pipeline &p, const wt_image *in, int n_in, const wt_image *out, int n_out,
                                      cudaStream_t s, int reps) {
  run(p, in, n_in, out, n_out, s);
  run(p, in, n_in, out, n_out, s);
  check_rt(cudaStreamSynchronize(s), "cudaStreamSynchronize");
  const CachedRun *c = cached_run(p, in, n_in, out, n_out);
  if (!c) fail(WT_EUNSUPPORTED, "launches of this run are not cached");
  RunPlan plan = build_plan(p, in, n_in, out, n_out);
  if (plan.launches.size() != c->functions.size()) fail(WT_EUNSUPPORTED, "run plan changed");
  const Driver &drv = driver();
  cudaEvent_t e0, e1;
  check_rt(cudaEventCreate(&e0), "cudaEventCreate");
  check_rt(cudaEventCreate(&e1), "cudaEventCreate");
  std::vector<LaunchTime> res(c->functions.size());
  for (size_t i = 0; i < c->functions.size(); i++) {
    const Launch &L = plan.launches[i];
    res[i].first_stage = L.stages.front();
    res[i].n_stages = (int)L.stages.size();
    res[i].fused = L.fused;
    res[i].ms = INFINITY;
    KernelArgs a = c->args[i];
    void *params[] = {&a};
    // launch i alone, `reps` times (it reads what earlier launches wrote
    // and rewrites the same outputs): 3 samples, the minimum of the means
    for (int t = 0; t < 3; t++) {
      check_rt(cudaEventRecord(e0, s), "cudaEventRecord");
      for (int r = 0; r < reps; r++)
        check_cu(drv.launchKernel((CUfunction)c->functions[i], c->grid[3 * i], c->grid[3 * i + 1],
                                  c->grid[3 * i + 2], (unsigned)c->block[i], 1, 1, (unsigned)c->smem[i],
                                  (CUstream)s, params, nullptr),
                 "cuLaunchKernel");
      check_rt(cudaEventRecord(e1, s), "cudaEventRecord");
      check_rt(cudaEventSynchronize(e1), "cudaEventSynchronize");
      float ms = 0;
      check_rt(cudaEventElapsedTime(&ms, e0, e1), "cudaEventElapsedTime");
      res[i].ms = std::min(res[i].ms, (double)ms / reps);
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return res;
}

void precompile(Pipeline &p, const std::vector<Schedule> &cands, const wt_image *in, int n_in, const wt_image *out,
                int n_out, bool persistent) {
  struct Job {
    std::string src, name;
    int max_regs;
  };
  std::vector<Job> jobs;
  std::set<std::string> names;
  const Schedule saved = p.sched;
  for (const Schedule &c : cands) {
    p.sched = c;
    try {
      RunPlan plan = build_plan(p, in, n_in, out, n_out);
      for (Launch &L : plan.launches) {
        if (persistent && L.fused && !L.key.otptb) {
          L.key.persistent = true;
          L.kname = kernel_name(p, L.key, true, L.geom.n_gather > 0);
        }
        if (!names.insert(L.kname).second) continue;
        jobs.push_back({launch_source(p, L), L.kname, L.key.max_regs});
      }
    } catch (const Error &) {
      // an infeasible candidate: timing reports it
    }
  }
  p.sched = saved;
  if (jobs.empty()) return;
  unsigned hw = std::max(1u, std::thread::hardware_concurrency());
  const unsigned nt = std::min<unsigned>(std::min<unsigned>(hw, 32u), (unsigned)jobs.size());
  std::atomic<size_t> next{0};
  std::vector<std::thread> th;
  for (unsigned t = 0; t < nt; t++)
    th.emplace_back([&] {
      for (;;) {
        size_t i = next.fetch_add(1);
        if (i >= jobs.size()) return;
        try {
          compile_cubin(jobs[i].src, jobs[i].name, jobs[i].max_regs);
        } catch (...) {
          // reported when the candidate is loaded
        }
      }
    });
  for (auto &t : th) t.join();
}

namespace {

double try_time(Pipeline &p, const Schedule &s, const Runner &r, int reps) {
  p.sched = s;
  p.sched.installed = true;
  p.sched_version++;
  try {
    return time_installed(p, r.in, r.n_in, r.out, r.n_out, r.n_images, r.s, reps);
  } catch (const Error &e) {
    if (e.code == WT_ECUDA) throw;  // the context may be unusable: stop
    cudaGetLastError();
    return INFINITY;
  }
}

// Distinct register/shared placements of a group over fracReg in [0, 1]:
// the largest fracReg of each placement, at most three (all registers, all
// shared, and the one in the middle).
std::vector<float> placements(const Pipeline &p, const std::vector<int> &seg, int V) {
  std::vector<float> fr;
  std::set<std::vector<char>> seen;
  for (int fi = 10; fi >= 0; fi--) {
    GroupGeom g = analyze_group(p, seg, V, fi / 10.f, 4);
    if (!g.fusable) return fr;
    std::vector<char> sig;
    for (const Node &n : g.nodes) sig.push_back(n.in_smem);
    if (seen.insert(sig).second) fr.push_back(fi / 10.f);
  }
  if (fr.size() > 3) fr = {fr.front(), fr[fr.size() / 2], fr.back()};
  return fr;
}

}  // namespace

TuneResult tune(Pipeline &p, const wt_image *in, int n_in, const wt_image *out, int n_out, int n_images,
                int max_variants, int reps, cudaStream_t stream) {
  if (max_variants < 1) max_variants = 12;
  if (reps < 1) reps = 20;
  const int n_pipe_in = (int)p.in_channels.size(), n_pipe_out = (int)p.outputs.size();
  const wt_image *in0 = in;
  const wt_image *out0 = out;
  const int W = in0[0].width, H = in0[0].height, dtype = in0[0].dtype;
  int dev = 0;
  check_rt(cudaGetDevice(&dev), "cudaGetDevice");
  const GpuConfig cfg = device_config(dev);
  const std::vector<StageStats> st = stage_stats(p, false);
  const CostWeights w = current_weights();
  const double pbytes = pipeline_bytes(p, W, H, dtype);
  Runner r{p, in, n_in, out, n_out, n_images, stream};
  const bool batched = n_images >= 1;
  // precompiling uses the first image's plan (the kernels of a batch are
  // the same for every image)
  auto pre = [&](const std::vector<Schedule> &c) {
    precompile(p, c, in0, batched ? n_pipe_in : n_in, out0, batched ? n_pipe_out : n_out, batched);
  };
  const Schedule user = p.sched;
  TuneResult res;
  // 1. grouping: the cost model's DP-Fusion choice, and all stages in one
  //    group when that group fuses; default tile parameters
  std::vector<Schedule> groupings;
  Schedule dp = dp_fusion(p, W, H, dtype, cfg, st, w, nullptr, kMaxGroupStages);
  for (auto &g : dp.params) g = GroupParams();
  groupings.push_back(dp);
  std::vector<int> all((size_t)p.stages.size());
  for (size_t i = 0; i < all.size(); i++) all[i] = (int)i;
  // the DP choice with every longest run of stages that forms a reduction
  // chain across levels merged into one group (the DP never proposes
  // groups that span levels); other stages keep their DP groups
  {
    const size_t n = p.stages.size();
    std::vector<int> g(n);
    int ng = 0, prev_dp = -1;
    bool any = false;
    for (size_t s = 0; s < n;) {
      size_t end = s;
      for (size_t e = s + 1; e < n && e - s < 6; e++) {
        std::vector<int> run;
        for (size_t q = s; q <= e; q++) run.push_back((int)q);
        if (chain_form(p, run).ok) end = e;
      }
      if (end > s) {
        for (size_t q = s; q <= end; q++) g[q] = ng;
        ng++;
        any = true;
        prev_dp = -1;
        s = end + 1;
        continue;
      }
      g[s] = (prev_dp >= 0 && dp.group_of_stage[s] == prev_dp) ? ng - 1 : ng++;
      prev_dp = dp.group_of_stage[s];
      s++;
    }
    if (any) {
      Schedule ch = dp;
      ch.n_groups = ng;
      ch.group_of_stage = g;
      ch.params.assign(ng, GroupParams());
      groupings.push_back(ch);
    }
  }
  if (dp.n_groups != 1 && all.size() <= 24 && analyze_group(p, all, 4, 1.f, 4).fusable) {
    Schedule one;
    one.exec = WT_EXEC_FUSED;
    one.n_groups = 1;
    one.group_of_stage.assign(all.size(), 0);
    one.params.assign(1, GroupParams());
    groupings.push_back(one);
  }
  pre(groupings);
  Schedule best;
  double best_ms = INFINITY;
  for (const Schedule &s : groupings) {
    double ms = try_time(p, s, r, reps);
    res.timed++;
    if (ms < best_ms) {
      best_ms = ms;
      best = s;
    }
  }
  if (!std::isfinite(best_ms)) {
    p.sched = user;
    p.sched_version++;
    fail(WT_EUNSUPPORTED, "no candidate schedule ran");
  }
  // 2. per group: kernel variants (warps per block, pixels per lane,
  //    placement, staging buffers) ranked by the cost model, the best
  //    max_variants timed; 3. tile heights for the two fastest variants
  std::vector<std::vector<int>> groups(best.n_groups);
  for (size_t i = 0; i < best.group_of_stage.size(); i++) groups[best.group_of_stage[i]].push_back((int)i);
  for (int gi = 0; gi < best.n_groups; gi++) {
    const std::vector<int> &seg = groups[gi];
    if (!analyze_group(p, seg, 4, 1.f, 4).fusable) continue;
    int gw, gh;
    level_dims(W, H, p.stages[seg[0]].level, &gw, &gh);
    struct Cand {
      GroupParams prm;
      double model;
    };
    std::vector<Cand> cands;
    for (int V : {4, 8})
      for (float fr : placements(p, seg, V))
        for (int nw : {2, 4})
          for (int nb : {2, 3}) {
            GroupParams q = best.params[gi];
            q.vec = V;
            q.frac_reg = fr;
            q.warps_per_block = nw;
            q.n_buffers = nb;
            CostInfo ci = cost_group(p, seg, q, 128, W, H, dtype, cfg, st, w, pbytes);
            if (!ci.feasible) continue;
            cands.push_back({q, ci.cost});
          }
    std::stable_sort(cands.begin(), cands.end(), [](const Cand &a, const Cand &b) { return a.model < b.model; });
    if ((int)cands.size() > max_variants) cands.resize(max_variants);
    std::vector<Schedule> vs;
    for (const Cand &c : cands) {
      Schedule s = best;
      s.params[gi] = c.prm;
      vs.push_back(s);
    }
    // the group's stages as per-stage kernels (single images only: batched
    // runs need every group fused); a down-sampling stage then runs the
    // streaming down-sampling kernel
    if (!batched) {
      Schedule s = best;
      s.params[gi] = GroupParams();
      s.params[gi].plain = 1;
      vs.push_back(s);
    }
    pre(vs);
    std::vector<std::pair<double, GroupParams>> timed;
    for (const Schedule &s : vs) {
      double ms = try_time(p, s, r, reps);
      res.timed++;
      timed.push_back({ms, s.params[gi]});
      if (ms < best_ms) {
        best_ms = ms;
        best = s;
      }
    }
    std::stable_sort(timed.begin(), timed.end(),
                     [](const std::pair<double, GroupParams> &a, const std::pair<double, GroupParams> &b) {
                       return a.first < b.first;
                     });
    bool has_down = false;  // per-stage kernels whose rows per warp matter
    for (int sid : seg) has_down = has_down || down_streamable(down_form(p, sid), 4);
    for (size_t k = 0; k < std::min<size_t>(2, timed.size()); k++) {
      if (!std::isfinite(timed[k].first)) continue;
      if (timed[k].second.plain && !has_down) continue;
      for (int T : {4, 8, 11, 14, 17, 20, 23, 26, 32, 40, 48, 64}) {
        if (T > std::max(8, gh) || T == timed[k].second.tile_h) continue;
        Schedule s = best;
        s.params[gi] = timed[k].second;
        s.params[gi].tile_h = T;
        double ms = try_time(p, s, r, reps);
        res.timed++;
        if (ms < best_ms) {
          best_ms = ms;
          best = s;
        }
      }
    }
  }
  best.installed = true;
  best.predicted_cost = 0;
  p.sched = best;
  p.sched_version++;
  res.best_ms = best_ms;
  return res;
}

}  // namespace wt

// C ABI of the scheduler: GPU configuration, the paper's OTPW geometry and
// Alg. 2 quantities, group costs, cost weights (include/wt.h).
#include <cuda_runtime.h>

#include <cstring>

#include "wt.h"
#include "wt_runtime.hpp"
#include "wt_sched.hpp"

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
  } catch (const std::exception &e) {
    wt::set_last_error(e.what());
    return WT_EINVAL;
  }
}

wt::GpuConfig from_c(const wt_gpu_config &c) {
  wt::GpuConfig g;
  g.nsms = c.nsms;
  g.cores_per_sm = c.cores_per_sm;
  g.glmem_bw = c.glmem_bw_gbs * 1e9;
  g.max_smem_per_tb = c.max_smem_per_block;
  g.smem_per_sm = c.smem_per_sm;
  g.max_warps_per_sm = c.max_warps_per_sm;
  g.max_tb_per_sm = c.max_blocks_per_sm;
  g.regs_per_sm = c.regs_per_sm;
  g.max_regs_per_th = c.max_regs_per_thread;
  g.warp_size = c.warp_size;
  g.max_th_per_sm = c.max_threads_per_sm;
  if (g.nsms < 1 || g.warp_size < 1 || g.max_warps_per_sm < 1 || g.regs_per_sm < 1 || g.smem_per_sm < 1)
    wt::fail(WT_EINVAL, "incomplete GPU configuration");
  return g;
}

void to_c(const wt::GpuConfig &g, wt_gpu_config *c) {
  c->nsms = g.nsms;
  c->cores_per_sm = g.cores_per_sm;
  c->glmem_bw_gbs = g.glmem_bw / 1e9;
  c->max_smem_per_block = g.max_smem_per_tb;
  c->smem_per_sm = g.smem_per_sm;
  c->max_warps_per_sm = g.max_warps_per_sm;
  c->max_blocks_per_sm = g.max_tb_per_sm;
  c->regs_per_sm = g.regs_per_sm;
  c->max_regs_per_thread = g.max_regs_per_th;
  c->warp_size = g.warp_size;
  c->max_threads_per_sm = g.max_th_per_sm;
}

}  // namespace

extern "C" {

wt_status wt_gpu_config_get(int32_t device, wt_gpu_config *out) {
  return guard([&] {
    if (!out) wt::fail(WT_EINVAL, "null out");
    to_c(device < 0 ? wt::default_gb300() : wt::device_config(device), out);
  });
}

wt_status wt_otpw_warp_sizes(const int32_t block[3], int32_t warp_size, int32_t warp[3]) {
  return guard([&] {
    if (!block || !warp || warp_size < 1) wt::fail(WT_EINVAL, "bad arguments");
    int B[3] = {block[0], block[1], block[2]}, W[3];
    for (int i = 0; i < 3; i++)
      if (B[i] < 1) wt::fail(WT_EINVAL, "block sizes must be >= 1");
    wt::otpw_warp_sizes(B, warp_size, W);
    for (int i = 0; i < 3; i++) warp[i] = W[i];
  });
}

wt_status wt_otpw_scratchpad(const int32_t block[3], const int32_t warp[3], const int32_t tile[3],
                             const int32_t overlap[3], int64_t *points) {
  return guard([&] {
    if (!block || !warp || !tile || !overlap || !points) wt::fail(WT_EINVAL, "bad arguments");
    int B[3], W[3], T[3], O[3];
    for (int i = 0; i < 3; i++) {
      B[i] = block[i]; W[i] = warp[i]; T[i] = tile[i]; O[i] = overlap[i];
      if (B[i] < 1 || W[i] < 1 || T[i] < 1 || O[i] < 0) wt::fail(WT_EINVAL, "bad sizes");
    }
    *points = wt::otpw_scratchpad_points(B, W, T, O);
  });
}

wt_status wt_cost_occupancy(const wt_gpu_config *cfg, int64_t smem_per_block, int32_t warps_per_block,
                            int32_t regs_per_thread, double *occupancy, int32_t *blocks_per_sm) {
  return guard([&] {
    if (!cfg || !occupancy || warps_per_block < 1 || regs_per_thread < 1 || smem_per_block < 0)
      wt::fail(WT_EINVAL, "bad arguments");
    int tb = 0;
    *occupancy = wt::alg2_occupancy(from_c(*cfg), smem_per_block, warps_per_block, regs_per_thread, &tb, nullptr);
    if (blocks_per_sm) *blocks_per_sm = tb;
  });
}

wt_status wt_min_transactions(const int64_t *byte_addresses, int32_t n, int32_t access_bytes, int32_t txn_bytes,
                              int64_t *txns) {
  return guard([&] {
    if (!txns || n < 0 || (n > 0 && !byte_addresses) || access_bytes < 1 || txn_bytes < 1)
      wt::fail(WT_EINVAL, "bad arguments");
    *txns = wt::min_gl_txs(byte_addresses, n, access_bytes, txn_bytes);
  });
}

wt_status wt_cost_group(wt_pipeline *p, int32_t first_stage, int32_t n_stages, const wt_group_params *prm,
                        int32_t txn_bytes, int32_t width, int32_t height, int32_t dtype, const wt_gpu_config *cfg,
                        wt_cost_info *out) {
  return guard([&] {
    if (!p || !prm || !out) wt::fail(WT_EINVAL, "bad arguments");
    if (first_stage < 0 || n_stages < 1 || first_stage + n_stages > (int)p->stages.size())
      wt::fail(WT_EINVAL, "stage range");
    if (width < 1 || height < 1 || dtype < WT_F32 || dtype > WT_BF16 || (txn_bytes != 32 && txn_bytes != 128))
      wt::fail(WT_EINVAL, "bad size, dtype or transaction size");
    std::vector<int> seg;
    for (int s = first_stage; s < first_stage + n_stages; s++) seg.push_back(s);
    wt::GpuConfig g = cfg ? from_c(*cfg) : wt::default_gb300();
    wt::GroupParams q;
    q.tile_h = prm->tile_h;
    q.warps_per_block = prm->warps_per_block;
    q.frac_reg = prm->frac_reg;
    q.vec = prm->vec ? prm->vec : 4;
    q.chunk_rows = prm->chunk_rows ? prm->chunk_rows : 8;
    q.n_buffers = prm->n_buffers ? prm->n_buffers : 2;
    if (q.tile_h < 1 || q.warps_per_block < 1 || q.warps_per_block > 16) wt::fail(WT_EINVAL, "bad params");
    auto st = wt::stage_stats(*p, false);
    wt::CostInfo ci = wt::cost_group(*p, seg, q, txn_bytes, width, height, dtype, g, st, wt::current_weights(),
                                     wt::pipeline_bytes(*p, width, height, dtype));
    memset(out, 0, sizeof *out);
    for (int i = 0; i < 7; i++) out->terms[i] = ci.t[i];
    out->cost = ci.cost;
    out->feasible = ci.feasible ? 1 : 0;
    out->regs_per_thread = ci.regs;
    out->smem_per_block = ci.smem_per_tb;
    out->occupancy = ci.occupancy;
    out->waves = ci.waves;
    out->work = ci.work;
  });
}

wt_status wt_preprocess(wt_pipeline *p, double *ns_per_iter, int32_t *regs) {
  return guard([&] {
    if (!p) wt::fail(WT_EINVAL, "null pipeline");
    std::lock_guard<std::mutex> lk(p->mu);
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
      cudaGetLastError();
      wt::fail(WT_ECUDA, "preprocessing needs a GPU");
    }
    auto st = wt::stage_stats(*p, true);
    p->pre_ns.resize(st.size());
    p->pre_regs.resize(st.size());
    for (size_t s = 0; s < st.size(); s++) {
      if (!st[s].measured) wt::fail(WT_ECUDA, "a stage's micro-kernel did not run");
      p->pre_ns[s] = st[s].ns_per_iter;
      p->pre_regs[s] = st[s].regs;
      if (ns_per_iter) ns_per_iter[s] = st[s].ns_per_iter;
      if (regs) regs[s] = st[s].regs;
    }
  });
}

wt_status wt_cost_weights(const double *set7, double *get7) {
  return guard([&] {
    if (set7) {
      wt::CostWeights w;
      for (int i = 0; i < 7; i++) {
        if (!(set7[i] >= 0)) wt::fail(WT_EINVAL, "weights must be >= 0");
        w.w[i] = set7[i];
      }
      wt::set_weights(w);
    }
    if (get7) {
      wt::CostWeights w = wt::current_weights();
      for (int i = 0; i < 7; i++) get7[i] = w.w[i];
    }
  });
}

}  // extern "C"

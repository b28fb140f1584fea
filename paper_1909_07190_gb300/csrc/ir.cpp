// Stage-DAG IR: validation, levels and per-edge footprints.
//
// A pipeline is a DAG of stages, each a per-point function of producer
// values at constant offsets (Sec. 2.2 Fig. 2).  Each tap is a dependence
// vector (Sec. 2.3); after alignment and scaling (Sec. 5) a tap is one of
// three constant maps: same level, DOWN2 (2x+d) or UP2 (x/2+d).  This file
// checks the DAG, assigns every stage its level and summarises each
// producer->consumer edge as a footprint box (used by the halo analysis).
#include <algorithm>
#include <climits>
#include <cstring>

#include "wt_internal.hpp"

namespace wt {

[[noreturn]] void fail(wt_status code, const std::string &msg) { throw Error{code, msg}; }

uint64_t fnv1a(const void *data, size_t n, uint64_t h) {
  const unsigned char *b = static_cast<const unsigned char *>(data);
  for (size_t i = 0; i < n; i++) {
    h ^= b[i];
    h *= 1099511628211ull;
  }
  return h;
}

void level_dims(int W, int H, int level, int *w, int *h) {
  int a = W, b = H;
  for (int l = 0; l < level; l++) {
    a = (a + 1) / 2;
    b = (b + 1) / 2;
  }
  *w = a;
  *h = b;
}

void build_pipeline(Pipeline &p, const wt_stage *st, int n, const int32_t *in_ch,
                    int n_in, const int32_t *outs, int n_out) {
  if (n < 1 || !st) fail(WT_EINVAL, "pipeline needs at least one stage");
  if (n_in < 1 || !in_ch) fail(WT_EINVAL, "pipeline needs at least one input");
  if (n_out < 1 || !outs) fail(WT_EINVAL, "pipeline needs at least one output");
  p.in_channels.assign(in_ch, in_ch + n_in);
  for (int c : p.in_channels)
    if (c < 1) fail(WT_EINVAL, "input channels must be >= 1");
  p.stages.resize(n);
  uint64_t h = fnv1a(in_ch, sizeof(int32_t) * n_in);
  for (int s = 0; s < n; s++) {
    const wt_stage &S = st[s];
    Stage &T = p.stages[s];
    if (S.channels < 1) fail(WT_EINVAL, "stage " + std::to_string(s) + ": channels < 1");
    if (S.n_ops < 1 || S.n_ops > kMaxOps || !S.ops)
      fail(WT_EINVAL, "stage " + std::to_string(s) + ": program must have 1.." +
                          std::to_string(kMaxOps) + " ops");
    if (S.n_inputs < 0 || (S.n_inputs > 0 && !S.inputs))
      fail(WT_EINVAL, "stage " + std::to_string(s) + ": bad inputs");
    T.channels = S.channels;
    T.inputs.assign(S.inputs, S.inputs + S.n_inputs);
    for (int pid : T.inputs) {
      if (pid >= s) fail(WT_EINVAL, "stage " + std::to_string(s) + " reads stage " +
                                        std::to_string(pid) + ": not topological (cycle?)");
      if (pid < -n_in) fail(WT_EINVAL, "stage " + std::to_string(s) + " reads missing input");
    }
    T.ops.resize(S.n_ops);
    int depth = 0, lv = INT_MIN;
    std::vector<int> slot_mode(T.inputs.size(), -1);
    std::vector<Edge> edges(T.inputs.size());
    std::vector<char> used(T.inputs.size(), 0);
    for (int i = 0; i < S.n_ops; i++) {
      const wt_op &o = S.ops[i];
      Op &q = T.ops[i];
      q.op = o.op; q.slot = o.slot; q.dx = o.dx; q.dy = o.dy;
      q.chan = o.chan; q.mode = o.mode; q.value = o.value;
      switch (o.op) {
        case WT_OP_CONST: case WT_OP_XPAR: case WT_OP_YPAR: case WT_OP_CHAN:
          depth++;
          break;
        case WT_OP_TAP: case WT_OP_TAPZ: {
          if (o.slot < 0 || o.slot >= (int)T.inputs.size())
            fail(WT_EINVAL, "stage " + std::to_string(s) + ": tap slot out of range");
          if (o.mode < WT_TAP_SAME || o.mode > WT_TAP_UP8)
            fail(WT_EINVAL, "stage " + std::to_string(s) + ": bad tap mode");
          if (o.dx < -64 || o.dx > 64 || o.dy < -64 || o.dy > 64)
            fail(WT_EINVAL, "stage " + std::to_string(s) + ": tap offset beyond +-64");
          int pid = T.inputs[o.slot];
          int pl = pid >= 0 ? p.stages[pid].level : 0;
          int pc = pid >= 0 ? p.stages[pid].channels : p.in_channels[-pid - 1];
          if (o.op == WT_OP_TAPZ) {
            // plane offset in `chan`; planes of the same depth, same level
            if (o.mode != WT_TAP_SAME) fail(WT_EINVAL, "stage " + std::to_string(s) + ": plane tap with a scaling mode");
            if (o.chan < -16 || o.chan > 16)
              fail(WT_EINVAL, "stage " + std::to_string(s) + ": plane offset beyond +-16");
            if (pc != 1 && pc != S.channels)
              fail(WT_EINVAL, "stage " + std::to_string(s) + ": plane tap of a producer with another plane count");
            T.has_z = true;
          } else {
            if (o.chan >= pc) fail(WT_EINVAL, "stage " + std::to_string(s) + ": tap channel out of range");
            if (o.chan < 0 && pc != 1 && pc != S.channels)
              fail(WT_EINVAL, "stage " + std::to_string(s) +
                                  ": same-channel tap of a producer with a different channel count");
          }
          int implied = pl + tap_level_delta(o.mode);
          if (lv == INT_MIN) lv = implied;
          else if (lv != implied)
            fail(WT_EINVAL, "stage " + std::to_string(s) + ": taps imply different levels");
          if (slot_mode[o.slot] >= 0 && slot_mode[o.slot] != o.mode)
            fail(WT_EINVAL, "stage " + std::to_string(s) + ": one producer read in two tap modes");
          slot_mode[o.slot] = o.mode;
          Edge &e = edges[o.slot];
          const int dz = o.op == WT_OP_TAPZ ? o.chan : 0;
          if (!used[o.slot]) {
            used[o.slot] = 1;
            e.producer = pid; e.mode = o.mode;
            e.dxmin = e.dxmax = o.dx; e.dymin = e.dymax = o.dy;
            e.dzmin = e.dzmax = dz;
          } else {
            e.dxmin = std::min(e.dxmin, o.dx); e.dxmax = std::max(e.dxmax, o.dx);
            e.dymin = std::min(e.dymin, o.dy); e.dymax = std::max(e.dymax, o.dy);
            e.dzmin = std::min(e.dzmin, dz); e.dzmax = std::max(e.dzmax, dz);
          }
          if (o.op == WT_OP_TAPZ) e.zrel = true;
          const int spec = o.op == WT_OP_TAPZ ? -1 : o.chan;
          if (std::find(e.chans.begin(), e.chans.end(), spec) == e.chans.end())
            e.chans.push_back(spec);
          depth++;
        } break;
        case WT_OP_ADD: case WT_OP_SUB: case WT_OP_MUL: case WT_OP_DIV:
        case WT_OP_MIN: case WT_OP_MAX:
          if (depth < 2) fail(WT_EINVAL, "stage " + std::to_string(s) + ": stack underflow");
          depth--;
          break;
        case WT_OP_NEG: case WT_OP_ABS: case WT_OP_SQRT:
          if (depth < 1) fail(WT_EINVAL, "stage " + std::to_string(s) + ": stack underflow");
          break;
        default:
          fail(WT_EINVAL, "stage " + std::to_string(s) + ": unknown opcode " + std::to_string(o.op));
      }
      if (depth > kMaxStack) fail(WT_EINVAL, "stage " + std::to_string(s) + ": stack too deep");
    }
    if (depth != 1) fail(WT_EINVAL, "stage " + std::to_string(s) + ": program must leave one value");
    if (lv == INT_MIN) lv = 0;
    if (lv < 0) fail(WT_EINVAL, "stage " + std::to_string(s) + ": level below the input level");
    T.level = lv;
    T.edges.clear();
    for (size_t k = 0; k < edges.size(); k++)
      if (used[k]) T.edges.push_back(edges[k]);
    h = fnv1a(&S.channels, sizeof(S.channels), h);
    h = fnv1a(S.inputs, sizeof(int32_t) * S.n_inputs, h);
    for (const Op &q : T.ops) {
      int v[6] = {q.op, q.slot, q.dx, q.dy, q.chan, q.mode};
      h = fnv1a(v, sizeof(v), h);
      h = fnv1a(&q.value, sizeof(float), h);
    }
  }
  p.has_z = false;
  for (const Stage &T : p.stages) p.has_z = p.has_z || T.has_z;
  p.outputs.assign(outs, outs + n_out);
  p.is_output.assign(n, 0);
  for (int o : p.outputs) {
    if (o < 0 || o >= n) fail(WT_EINVAL, "output id out of range");
    p.is_output[o] = 1;
  }
  h = fnv1a(outs, sizeof(int32_t) * n_out, h);
  p.consumers.assign(n, {});
  for (int s = 0; s < n; s++)
    for (const Edge &e : p.stages[s].edges)
      if (e.producer >= 0) p.consumers[e.producer].push_back(s);
  p.hash = h;
}

}  // namespace wt

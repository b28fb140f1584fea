// Reduction chain across levels: a group S1 -> S2 -> ... -> Sk where S1 is
// any program of one producer P read through down-sampling taps inside the
// 2x2 block of its point (P(2x + i, 2y + j), i, j in {0, 1}; a histogram's
// splat and first sum), and every later stage is a weighted 2x2 sum of the
// one before (Sm(x, y) = sum_ij w_ij S(m-1)(2x + i, 2y + j)).  The group
// spans k levels (Sec. 2.3 scaling: each stage one level coarser), and one
// kernel computes Sk directly from P: a thread owns one level-k cell and
// sums, over the cell's 2^(k-1) x 2^(k-1) level-1 positions, S1's values
// times the products of the per-level weights, with the clamp-to-edge rule
// applied at every level as the stage-by-stage evaluation does.  No
// intermediate level is written to memory; all channels of a cell are
// accumulated by its thread from one read of P.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <functional>
#include <map>
#include <memory>
#include <sstream>

#include "wt_internal.hpp"

namespace wt {

namespace {


// Expression of S1 for one channel: the postfix program with the channel
// index a constant, folded (operations on constants evaluated in FP32 as
// the device would; x * 0, x * 1, x + 0, x - 0 simplified: exact for the
// finite values stages carry).
struct Ex {
  bool k = false;
  float v = 0.f;
  std::string s;
};

Ex konst(float v) {
  Ex e;
  e.k = true;
  e.v = v;
  e.s = float_literal(v);
  return e;
}

Ex fold_program(const std::vector<Op> &ops, int chan, const std::function<std::string(const Op &)> &tap) {
  std::vector<Ex> st;
  for (const Op &op : ops) {
    switch (op.op) {
      case WT_OP_CONST: st.push_back(konst(op.value)); break;
      case WT_OP_CHAN: st.push_back(konst((float)chan)); break;
      case WT_OP_TAP: {
        Ex e;
        e.s = tap(op);
        st.push_back(e);
      } break;
      case WT_OP_NEG: case WT_OP_ABS: case WT_OP_SQRT: {
        Ex a = st.back();
        if (a.k) {
          const float r = op.op == WT_OP_NEG ? -a.v : op.op == WT_OP_ABS ? std::fabs(a.v) : std::sqrt(a.v);
          st.back() = konst(r);
        } else {
          st.back().s = op.op == WT_OP_NEG ? "(-" + a.s + ")" : op.op == WT_OP_ABS ? "fabsf(" + a.s + ")"
                                                                                  : "sqrtf(" + a.s + ")";
        }
      } break;
      default: {
        Ex b = st.back();
        st.pop_back();
        Ex a = st.back();
        st.pop_back();
        if (a.k && b.k) {
          float r = 0.f;
          switch (op.op) {
            case WT_OP_ADD: r = a.v + b.v; break;
            case WT_OP_SUB: r = a.v - b.v; break;
            case WT_OP_MUL: r = a.v * b.v; break;
            case WT_OP_DIV: r = a.v / b.v; break;
            case WT_OP_MIN: r = std::fmin(a.v, b.v); break;
            case WT_OP_MAX: r = std::fmax(a.v, b.v); break;
            default: fail(WT_EINVAL, "internal: opcode");
          }
          st.push_back(konst(r));
          break;
        }
        Ex e;
        switch (op.op) {
          case WT_OP_ADD:
            if (a.k && a.v == 0.f) e = b;
            else if (b.k && b.v == 0.f) e = a;
            else e.s = "(" + a.s + " + " + b.s + ")";
            break;
          case WT_OP_SUB:
            if (b.k && b.v == 0.f) e = a;
            else e.s = "(" + a.s + " - " + b.s + ")";
            break;
          case WT_OP_MUL:
            if ((a.k && a.v == 0.f) || (b.k && b.v == 0.f)) e = konst(0.f);
            else if (a.k && a.v == 1.f) e = b;
            else if (b.k && b.v == 1.f) e = a;
            else e.s = "(" + a.s + " * " + b.s + ")";
            break;
          case WT_OP_DIV: e.s = "(" + a.s + " / " + b.s + ")"; break;
          case WT_OP_MIN: e.s = "fminf(" + a.s + ", " + b.s + ")"; break;
          case WT_OP_MAX: e.s = "fmaxf(" + a.s + ", " + b.s + ")"; break;
          default: fail(WT_EINVAL, "internal: opcode");
        }
        st.push_back(e);
      }
    }
  }
  return st.back();
}

int pchannels(const Pipeline &p, int pid) { return pid >= 0 ? p.stages[pid].channels : p.in_channels[-pid - 1]; }

}  // namespace

ChainForm chain_form(const Pipeline &p, const std::vector<int> &stages) {
  for (int sid : stages)
    if (p.stages[sid].has_z) return ChainForm();
  ChainForm f;
  const int k = (int)stages.size();
  if (k < 2 || k > 6) return f;
  for (int m = 1; m < k; m++)
    if (stages[m] != stages[m - 1] + 1) return f;
  const Stage &S1 = p.stages[stages[0]];
  const int C = S1.channels;
  if (C > 32) return f;
  int slot = -1;
  for (const Op &op : S1.ops) {
    if (op.op == WT_OP_XPAR || op.op == WT_OP_YPAR) return f;
    if (op.op != WT_OP_TAP) continue;
    if (op.mode != WT_TAP_DOWN2 || op.dx < 0 || op.dx > 1 || op.dy < 0 || op.dy > 1) return f;
    if (slot >= 0 && op.slot != slot) return f;
    slot = op.slot;
  }
  if (slot < 0) return f;
  f.producer = S1.inputs[slot];
  const int pc = pchannels(p, f.producer);
  if (pc != 1) return f;  // one-plane producer: every channel reads the same taps
  f.C = C;
  for (int m = 1; m < k; m++) {
    const int s = stages[m];
    const Stage &S = p.stages[s];
    if (S.channels != C) return f;
    // a weighted 2x2 sum of the stage before: linear in its DOWN2 taps
    std::array<double, 4> w{0, 0, 0, 0};
    struct L {
      bool ok = true, is_c = true;
      double c = 0;
      std::map<int, double> t;
    };
    std::vector<L> st;
    for (const Op &op : S.ops) {
      if (op.op == WT_OP_CONST) {
        L l;
        l.c = op.value;
        st.push_back(l);
      } else if (op.op == WT_OP_TAP) {
        if (op.mode != WT_TAP_DOWN2 || S.inputs[op.slot] != stages[m - 1] || op.chan >= 0 || op.dx < 0 ||
            op.dx > 1 || op.dy < 0 || op.dy > 1)
          return f;
        L l;
        l.is_c = false;
        l.t[op.dx + 2 * op.dy] = 1.0;
        st.push_back(l);
      } else if (op.op == WT_OP_ADD || op.op == WT_OP_SUB) {
        L b = st.back();
        st.pop_back();
        L &a = st.back();
        const double sg = op.op == WT_OP_ADD ? 1.0 : -1.0;
        a.ok = a.ok && b.ok;
        a.is_c = a.is_c && b.is_c;
        a.c += sg * b.c;
        for (auto &kv : b.t) a.t[kv.first] += sg * kv.second;
      } else if (op.op == WT_OP_MUL || op.op == WT_OP_DIV) {
        L b = st.back();
        st.pop_back();
        L &a = st.back();
        if (op.op == WT_OP_DIV) {
          if (!b.is_c || b.c == 0) return f;
          b.c = 1.0 / b.c;
        }
        if (b.is_c) {
          a.c *= b.c;
          for (auto &kv : a.t) kv.second *= b.c;
        } else if (a.is_c && op.op == WT_OP_MUL) {
          const double s0 = a.c;
          a = b;
          a.c *= s0;
          for (auto &kv : a.t) kv.second *= s0;
        } else {
          return f;
        }
      } else if (op.op == WT_OP_NEG) {
        L &a = st.back();
        a.c = -a.c;
        for (auto &kv : a.t) kv.second = -kv.second;
      } else {
        return f;
      }
    }
    if (st.size() != 1 || st[0].is_c || st[0].c != 0) return f;
    for (auto &kv : st[0].t) w[kv.first] = kv.second;
    f.w.push_back(w);
  }
  // only the last stage leaves the group
  for (int m = 0; m + 1 < k; m++) {
    const int s = stages[m];
    if (p.is_output[s]) return f;
    for (int c : p.consumers[s])
      if (c != stages[m + 1]) return f;
  }
  f.ok = true;
  return f;
}

std::string emit_chain(const Pipeline &p, const std::vector<int> &stages, const CodegenKey &key,
                       const std::string &kname) {
  const ChainForm f = chain_form(p, stages);
  if (!f.ok) fail(WT_EINVAL, "internal: not a reduction chain");
  const int k = (int)stages.size();
  const Stage &S1 = p.stages[stages[0]];
  const int C = f.C;
  const int sdt = key.src_dtypes.at(0), ddt = key.dst_dtypes.at(0);
  const int sesz = elem_bytes(sdt), desz = elem_bytes(ddt);
  std::ostringstream o;
  o << kDeviceSource;
  o << "static_assert(sizeof(WtArgs) == " << sizeof(KernelArgs) << ", \"WtArgs layout\");\n";
  o << "extern \"C\" __global__ void __launch_bounds__(128) " << kname << "(const __grid_constant__ WtArgs a) {\n";
  o << "const int X = blockIdx.x * 128 + threadIdx.x, Y = blockIdx.y;\n";
  o << "const int W = a.W, H = a.H;\nif (X >= W || Y >= H) return;\n";
  o << "const int Ws = a.src[0].W, Hs = a.src[0].H;\n";
  o << "const unsigned char *sp = (const unsigned char *)a.src[0].ptr;\nconst wt_i64 pitch = a.src[0].pitch;\n";
  // dims of the levels between: level m (1 = S1's) of the producer's grid
  o << "int Wl[" << k + 1 << "], Hl[" << k + 1 << "];\nWl[0] = Ws; Hl[0] = Hs;\n";
  o << "for (int m = 1; m <= " << k << "; m++) { Wl[m] = (Wl[m - 1] + 1) >> 1; Hl[m] = (Hl[m - 1] + 1) >> 1; }\n";
  o << "float";
  for (int c = 0; c < C; c++) o << (c ? ", " : " ") << "acc" << c << " = 0.f";
  o << ";\n";
  // the thread's block of the producer lies inside it: no clamps needed
  const int B = 1 << k;
  o << "const bool inner = (X + 1) * " << B << " <= Ws && (Y + 1) * " << B << " <= Hs;\n";
  // Leaves: level-1 positions of the cell with their weights (products of
  // the per-level 2x2 weights), enumerated at compile time.
  struct Leaf {
    std::vector<int> ix, iy;  // per level from k down to 2: the 2x2 offsets
    double w;
  };
  std::vector<Leaf> leaves{{{}, {}, 1.0}};
  for (int m = k - 1; m >= 1; m--) {  // S(m+1) sums S(m): weights f.w[m-1]
    std::vector<Leaf> nx;
    for (const Leaf &l : leaves)
      for (int j = 0; j < 2; j++)
        for (int i = 0; i < 2; i++) {
          const double wij = f.w[m - 1][i + 2 * j];
          if (wij == 0) continue;
          Leaf q = l;
          q.ix.push_back(i);
          q.iy.push_back(j);
          q.w *= wij;
          nx.push_back(q);
        }
    leaves = nx;
  }
  // S1's value per channel at a level-1 point from its four taps
  auto tapname = [](const Op &op) { return "t" + std::to_string(op.dx + 2 * op.dy); };
  std::vector<std::string> s1(C);
  for (int c = 0; c < C; c++) s1[c] = fold_program(S1.ops, c, tapname).s;
  auto leaf_body = [&](bool inner) {
    for (const Leaf &l : leaves) {
      // level-1 coordinates: x_m = clamp(2 x_(m+1) + i, 0, W_m - 1), from X at level k
      std::string x = "X", y = "Y";
      for (size_t d = 0; d < l.ix.size(); d++) {
        const int lvl = k - 1 - (int)d;  // level of the index produced
        x = "(2 * " + x + " + " + std::to_string(l.ix[d]) + ")";
        y = "(2 * " + y + " + " + std::to_string(l.iy[d]) + ")";
        if (!inner) {
          x = "wt_clampi(" + x + ", 0, Wl[" + std::to_string(lvl) + "] - 1)";
          y = "wt_clampi(" + y + ", 0, Hl[" + std::to_string(lvl) + "] - 1)";
        }
      }
      o << "{ const int x1 = " << x << ", y1 = " << y << ";\n";
      if (inner) {
        o << "float t0, t1, t2, t3;\n";
        o << "wt_ld2_" << dtype_name(sdt) << "(sp + (wt_i64)(2 * y1) * pitch + (wt_i64)(2 * x1) * " << sesz << ", t0, t1);\n";
        o << "wt_ld2_" << dtype_name(sdt) << "(sp + (wt_i64)(2 * y1 + 1) * pitch + (wt_i64)(2 * x1) * " << sesz
          << ", t2, t3);\n";
      } else {
        o << "const int xa = wt_clampi(2 * x1, 0, Ws - 1), xb = wt_clampi(2 * x1 + 1, 0, Ws - 1);\n";
        o << "const int ya = wt_clampi(2 * y1, 0, Hs - 1), yb = wt_clampi(2 * y1 + 1, 0, Hs - 1);\n";
        o << "const float t0 = wt_ld1_" << dtype_name(sdt) << "(sp + (wt_i64)ya * pitch + (wt_i64)xa * " << sesz << ");\n";
        o << "const float t1 = wt_ld1_" << dtype_name(sdt) << "(sp + (wt_i64)ya * pitch + (wt_i64)xb * " << sesz << ");\n";
        o << "const float t2 = wt_ld1_" << dtype_name(sdt) << "(sp + (wt_i64)yb * pitch + (wt_i64)xa * " << sesz << ");\n";
        o << "const float t3 = wt_ld1_" << dtype_name(sdt) << "(sp + (wt_i64)yb * pitch + (wt_i64)xb * " << sesz << ");\n";
      }
      o << "(void)t0; (void)t1; (void)t2; (void)t3;\n";
      for (int c = 0; c < C; c++) {
        if (l.w == 1.0) o << "acc" << c << " += " << s1[c] << ";\n";
        else o << "acc" << c << " += " << float_literal(l.w) << " * " << s1[c] << ";\n";
      }
      o << "}\n";
    }
  };
  o << "if (inner) {\n";
  leaf_body(true);
  o << "} else {\n";
  leaf_body(false);
  o << "}\n";
  o << "unsigned char *dp = (unsigned char *)a.dst[0].ptr + (wt_i64)Y * a.dst[0].pitch + (wt_i64)X * " << desz
    << ";\n";
  for (int c = 0; c < C; c++)
    o << "wt_st1_" << dtype_name(ddt) << "(dp + (wt_i64)" << c << " * a.dst[0].plane, acc" << c << ");\n";
  o << "}\n";
  return o.str();
}

}  // namespace wt

// Overlapped tiling per thread block (OTPTB): the scheme the paper compares
// against (Sec. 3, Fig. 3; the tiling of PolyMage-GPU and Halide).  One
// thread block computes one output tile of a fused group: the sources'
// tile-plus-halo regions are loaded into shared memory, then every stage is
// computed over its own region (the tile plus the halo its consumers still
// need) into a shared-memory buffer, with a block barrier between stages;
// liveouts are written from their tile.  It reuses the group analysis of
// the warp-tile kernel (halos, separable split) so the two differ only in
// the tiling.
//
// Clamp-to-edge per stage: a region point outside the image holds the value
// of the clamped point, so every point evaluates its program at the clamped
// coordinates; the producer points that reads stay inside the producer's
// region (its region is the consumer's grown by the footprint, and the
// clamped point lies between the consumer region's edge and the tile).
#include <algorithm>
#include <functional>
#include <map>
#include <cmath>
#include <cstdio>
#include <sstream>

#include "wt_internal.hpp"

namespace wt {

namespace {


}  // namespace

OtptbLayout otptb_layout(const GroupGeom &g, const CodegenKey &key) {
  OtptbLayout L;
  L.tbx = key.tbx;
  L.tby = key.tby;
  if (L.tbx < 1 || L.tby < 1) fail(WT_EINVAL, "internal: block tile size");
  const int n = (int)g.nodes.size();
  L.rx.assign(n, 0);
  L.ry.assign(n, 0);
  L.rw.assign(n, 0);
  L.rh.assign(n, 0);
  L.off.assign(n, -1);
  for (int i = 0; i < n; i++) {
    const Node &nd = g.nodes[i];
    if (nd.gather_mode) continue;
    L.rx[i] = -nd.left;
    L.ry[i] = -nd.top;
    L.rw[i] = L.tbx + nd.left + nd.right;
    L.rh[i] = L.tby + nd.top + nd.bot;
  }
  // last use of every node in evaluation order; buffers are reused once
  // their node is dead (first fit over byte offsets)
  std::vector<int> pos(n, -1), last(n, -1);
  for (size_t k = 0; k < g.order.size(); k++) pos[g.order[k]] = (int)k;
  for (int ci : g.order)
    for (const KOp &op : g.nodes[ci].prog)
      if (op.op == WT_OP_TAP) last[op.node] = std::max(last[op.node], pos[ci]);
  struct Blk {
    int off, size, free_after;
  };
  std::vector<Blk> blocks;
  int top = 0;
  for (size_t k = 0; k < g.order.size(); k++) {
    const int i = g.order[k];
    const int bytes = (L.rw[i] * L.rh[i] * 4 + 127) / 128 * 128;
    int off = -1;
    for (Blk &b : blocks)
      if (b.free_after < (int)k && b.size >= bytes) {
        off = b.off;
        b.free_after = std::max(last[i], (int)k);
        break;
      }
    if (off < 0) {
      off = top;
      top += bytes;
      blocks.push_back({off, bytes, std::max(last[i], (int)k)});
    }
    L.off[i] = off;
  }
  L.smem = top;
  return L;
}

std::string emit_otptb(const Pipeline &p, const GroupGeom &g, const CodegenKey &key, const std::string &kname) {
  (void)p;
  for (const Node &n : g.nodes)
    if (n.gather_mode) fail(WT_EUNSUPPORTED, "block tiling of groups that read other levels");
  const OtptbLayout L = otptb_layout(g, key);
  std::ostringstream o;
  o << kDeviceSource;
  o << "static_assert(sizeof(WtArgs) == " << sizeof(KernelArgs) << ", \"WtArgs layout\");\n";
  o << "extern \"C\" __global__ void __launch_bounds__(" << 32 * key.nw << ") " << kname
    << "(const __grid_constant__ WtArgs a) {\n";
  o << "extern __shared__ __align__(128) unsigned char wt_smem[];\n";
  o << "const int W = a.W, H = a.H;\nconst int x0 = blockIdx.x * " << L.tbx << ", y0 = blockIdx.y * " << L.tby
    << ";\nconst int ch = blockIdx.z;\n(void)ch;\n";
  const int nt = 32 * key.nw;
  int src_i = 0, dst_i = 0;
  std::vector<int> sidx(g.nodes.size(), -1), didx(g.nodes.size(), -1);
  int mx_l = 0, mx_r = 0, mx_t = 0, mx_b = 0;
  for (size_t i = 0; i < g.nodes.size(); i++) {
    if (g.nodes[i].is_source) sidx[i] = src_i++;
    else if (g.nodes[i].is_liveout) didx[i] = dst_i++;
    mx_l = std::max(mx_l, g.nodes[i].left);
    mx_r = std::max(mx_r, g.nodes[i].right);
    mx_t = std::max(mx_t, g.nodes[i].top);
    mx_b = std::max(mx_b, g.nodes[i].bot);
  }
  // Every region inside the image: no clamping, and a region point's tap is
  // a constant offset in the producer's buffer from the point's own row and
  // column there (block-uniform).
  o << "const bool inner = x0 - " << mx_l << " >= 0 && x0 + " << L.tbx + mx_r << " <= W && y0 - " << mx_t
    << " >= 0 && y0 + " << L.tby + mx_b << " <= H;\n";
  auto buf = [&](int i) { return "((float *)(wt_smem + " + std::to_string(L.off[i]) + "))"; };
  // the value expression of node i; tap(q, dx, dy) gives a producer read
  auto expr_of = [&](const Node &n, const std::string &xp, const std::string &yp,
                     const std::function<std::string(const KOp &)> &tap) {
    std::vector<std::string> st;
    for (const KOp &op : n.prog) {
      switch (op.op) {
        case WT_OP_CONST: st.push_back(float_literal(op.value)); break;
        case WT_OP_XPAR: st.push_back("((float)(" + xp + " & 1))"); break;
        case WT_OP_YPAR: st.push_back("((float)(" + yp + " & 1))"); break;
        case WT_OP_CHAN: st.push_back(n.channels == 1 ? "(0.0f)" : "((float)ch)"); break;
        case WT_OP_TAP: st.push_back(tap(op)); break;
        case WT_OP_NEG: st.back() = "(-" + st.back() + ")"; break;
        case WT_OP_ABS: st.back() = "fabsf(" + st.back() + ")"; break;
        case WT_OP_SQRT: st.back() = "sqrtf(" + st.back() + ")"; break;
        default: {
          std::string b = st.back();
          st.pop_back();
          std::string a = st.back();
          st.pop_back();
          switch (op.op) {
            case WT_OP_ADD: st.push_back("(" + a + " + " + b + ")"); break;
            case WT_OP_SUB: st.push_back("(" + a + " - " + b + ")"); break;
            case WT_OP_MUL: st.push_back("(" + a + " * " + b + ")"); break;
            case WT_OP_DIV: st.push_back("(" + a + " / " + b + ")"); break;
            case WT_OP_MIN: st.push_back("fminf(" + a + ", " + b + ")"); break;
            case WT_OP_MAX: st.push_back("fmaxf(" + a + ", " + b + ")"); break;
            default: fail(WT_EINVAL, "internal: opcode");
          }
        }
      }
    }
    return st.back();
  };
  auto store_liveout = [&](const Node &n, int i) {
    if (!n.is_liveout) return;
    const int d = didx[i];
    const int dt = key.dst_dtypes.at(d);
    const std::string D = "a.dst[" + std::to_string(d) + "]";
    o << "if (x >= x0 && x < x0 + " << L.tbx << " && y >= y0 && y < y0 + " << L.tby << " && x < W && y < H"
      << (n.channels == 1 && g.channels > 1 ? " && ch == 0" : "") << ")\n";
    o << "wt_st1_" << dtype_name(dt) << "((unsigned char *)" << D << ".ptr + (wt_i64)" << (n.channels > 1 ? "ch" : "0")
      << " * " << D << ".plane + (wt_i64)y * " << D << ".pitch + (wt_i64)x * " << elem_bytes(dt) << ", v_);\n";
  };
  for (int pass = 0; pass < 2; pass++) {
    const bool fast = pass == 0;
    o << (fast ? "if (inner) {\n" : "} else {\n");
    for (int i : g.order) {
      const Node &n = g.nodes[i];
      const std::string RW = std::to_string(L.rw[i]), NP = std::to_string(L.rw[i] * L.rh[i]);
      if (fast) {
        // rows of the region by warp, columns by lane: no division
        o << "for (int ly = threadIdx.x >> 5; ly < " << L.rh[i] << "; ly += " << key.nw << ")\n";
        o << "for (int lx = threadIdx.x & 31; lx < " << L.rw[i] << "; lx += 32) {\n";
        o << "const int t_ = ly * " << RW << " + lx;\n";
        o << "const int x = x0 + (" << L.rx[i] << ") + lx, y = y0 + (" << L.ry[i] << ") + ly;\n(void)x;\n(void)y;\n";
      } else {
        o << "for (int t_ = threadIdx.x; t_ < " << NP << "; t_ += " << nt << ") {\n";
        o << "const int x = x0 + (" << L.rx[i] << ") + t_ % " << RW << ", y = y0 + (" << L.ry[i] << ") + t_ / "
          << RW << ";\n";
        o << "const int xc = wt_clampi(x, 0, W - 1), yc = wt_clampi(y, 0, H - 1);\n(void)xc;\n(void)yc;\n";
      }
      if (n.is_source) {
        const int s = sidx[i];
        const int dt = key.src_dtypes.at(s);
        const std::string S = "a.src[" + std::to_string(s) + "]";
        const std::string chan = n.src_chan >= 0 ? std::to_string(n.src_chan) : "ch";
        o << "wt_sst(" << buf(i) << ", t_, " << NP << ", wt_ld1_" << dtype_name(dt) << "((const unsigned char *)"
          << S << ".ptr + (wt_i64)" << chan << " * " << S << ".plane + (wt_i64)" << (fast ? "y" : "yc") << " * " << S
          << ".pitch + (wt_i64)" << (fast ? "x" : "xc") << " * " << elem_bytes(dt) << "));\n";
      } else {
        std::string e;
        if (fast) {
          // producer index = ly * RWq + lx + constant
          std::map<int, std::string> base;  // per producer region width
          e = expr_of(n, "x", "y", [&](const KOp &op) {
            const int q = op.node;
            const int off = (op.dy + L.ry[i] - L.ry[q]) * L.rw[q] + (op.dx + L.rx[i] - L.rx[q]);
            return "wt_sld(" + buf(q) + ", ly * " + std::to_string(L.rw[q]) + " + lx + (" + std::to_string(off) +
                   "), " + std::to_string(L.rw[q] * L.rh[q]) + ")";
          });
        } else {
          e = expr_of(n, "xc", "yc", [&](const KOp &op) {
            const int q = op.node;
            return "wt_sld(" + buf(q) + ", (yc + (" + std::to_string(op.dy) + ") - y0 - (" + std::to_string(L.ry[q]) +
                   ")) * " + std::to_string(L.rw[q]) + " + (xc + (" + std::to_string(op.dx) + ") - x0 - (" +
                   std::to_string(L.rx[q]) + ")), " + std::to_string(L.rw[q] * L.rh[q]) + ")";
          });
        }
        o << "const float v_ = " << e << ";\n";
        o << "wt_sst(" << buf(i) << ", t_, " << NP << ", v_);\n";
        store_liveout(n, i);
      }
      o << "}\n__syncthreads();\n";
    }
  }
  o << "}\n}\n";
  return o.str();
}

}  // namespace wt

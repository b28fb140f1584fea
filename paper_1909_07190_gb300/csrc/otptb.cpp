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
  for (size_t i = 0; i < g.nodes.size(); i++) {
    if (g.nodes[i].is_source) sidx[i] = src_i++;
    else if (g.nodes[i].is_liveout) didx[i] = dst_i++;
  }
  auto buf = [&](int i) { return "((float *)(wt_smem + " + std::to_string(L.off[i]) + "))"; };
  for (int i : g.order) {
    const Node &n = g.nodes[i];
    const std::string RW = std::to_string(L.rw[i]), NP = std::to_string(L.rw[i] * L.rh[i]);
    o << "for (int t_ = threadIdx.x; t_ < " << NP << "; t_ += " << nt << ") {\n";
    o << "const int x = x0 + (" << L.rx[i] << ") + t_ % " << RW << ", y = y0 + (" << L.ry[i] << ") + t_ / " << RW
      << ";\n";
    o << "const int xc = wt_clampi(x, 0, W - 1), yc = wt_clampi(y, 0, H - 1);\n(void)xc;\n(void)yc;\n";
    if (n.is_source) {
      const int s = sidx[i];
      const int dt = key.src_dtypes.at(s);
      const std::string S = "a.src[" + std::to_string(s) + "]";
      const std::string chan = n.src_chan >= 0 ? std::to_string(n.src_chan) : "ch";
      o << "wt_sst(" << buf(i) << ", t_, " << NP << ", wt_ld1_" << dtype_name(dt) << "((const unsigned char *)" << S
        << ".ptr + (wt_i64)" << chan << " * " << S << ".plane + (wt_i64)yc * " << S << ".pitch + (wt_i64)xc * "
        << elem_bytes(dt) << "));\n";
    } else {
      std::vector<std::string> st;
      for (const KOp &op : n.prog) {
        switch (op.op) {
          case WT_OP_CONST: st.push_back(float_literal(op.value)); break;
          case WT_OP_XPAR: st.push_back("((float)(xc & 1))"); break;
          case WT_OP_YPAR: st.push_back("((float)(yc & 1))"); break;
          case WT_OP_CHAN: st.push_back(n.channels == 1 ? "(0.0f)" : "((float)ch)"); break;
          case WT_OP_TAP: {
            const int q = op.node;
            st.push_back("wt_sld(" + buf(q) + ", (yc + (" + std::to_string(op.dy) + ") - y0 - (" +
                         std::to_string(L.ry[q]) + ")) * " + std::to_string(L.rw[q]) + " + (xc + (" +
                         std::to_string(op.dx) + ") - x0 - (" + std::to_string(L.rx[q]) + ")), " +
                         std::to_string(L.rw[q] * L.rh[q]) + ")");
          } break;
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
      o << "const float v_ = " << st.back() << ";\n";
      o << "wt_sst(" << buf(i) << ", t_, " << NP << ", v_);\n";
      if (n.is_liveout) {
        const int d = didx[i];
        const int dt = key.dst_dtypes.at(d);
        const std::string D = "a.dst[" + std::to_string(d) + "]";
        o << "if (x >= x0 && x < x0 + " << L.tbx << " && y >= y0 && y < y0 + " << L.tby
          << " && x < W && y < H" << (n.channels == 1 && g.channels > 1 ? " && ch == 0" : "") << ")\n";
        o << "wt_st1_" << dtype_name(dt) << "((unsigned char *)" << D << ".ptr + (wt_i64)" << (n.channels > 1 ? "ch" : "0")
          << " * " << D << ".plane + (wt_i64)y * " << D << ".pitch + (wt_i64)x * " << elem_bytes(dt) << ", v_);\n";
      }
    }
    o << "}\n__syncthreads();\n";
  }
  o << "}\n";
  return o.str();
}

}  // namespace wt

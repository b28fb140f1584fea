// Scaled streaming kernel of a down-sampling stage: a stage whose taps all
// read one producer one level finer (P(2x + dx, 2y + dy), Sec. 2.3) with a
// rank-one (separable) linear weight pattern, the pyramids' reduce step.
//
// A warp owns a strip of 32 VO output columns and T output rows and streams
// the producer's rows through it at twice the output rate (the streaming of
// Sec. 4 with the consumer one level coarser): each producer row is loaded
// once, as 2 VO coalesced values per lane, filtered along x at stride 2 (the
// taps left and right of a lane's segment come from its neighbours by warp
// shuffles), and added, weighted, into the accumulators of the output rows
// it contributes to; an output row is stored once its last row is in.  The
// accumulators form a ring whose slots are fixed at compile time by
// unrolling the step loop by the ring length.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <map>
#include <sstream>

#include "wt_internal.hpp"

namespace wt {

namespace {


struct Lin {
  bool ok = true, is_const = true;
  double c = 0;
  std::map<std::pair<int, int>, double> t;  // (dx, dy) -> weight
};

Lin add(const Lin &a, const Lin &b, double s) {
  Lin r;
  r.ok = a.ok && b.ok;
  r.is_const = a.is_const && b.is_const;
  r.c = a.c + s * b.c;
  r.t = a.t;
  for (auto &kv : b.t) r.t[kv.first] += s * kv.second;
  return r;
}

Lin scale(Lin a, double s) {
  a.c *= s;
  for (auto &kv : a.t) kv.second *= s;
  return a;
}

}  // namespace

DownForm down_form(const Pipeline &p, int sid) {
  if (p.stages[sid].has_z) return DownForm();
  DownForm f;
  const Stage &S = p.stages[sid];
  if (S.level < 1) return f;
  int slot = -1, chan = -2;
  Lin bad;
  bad.ok = false;
  std::vector<Lin> st;
  for (const Op &op : S.ops) {
    switch (op.op) {
      case WT_OP_CONST: {
        Lin l;
        l.c = op.value;
        st.push_back(l);
      } break;
      case WT_OP_TAP: {
        if (op.mode != WT_TAP_DOWN2) return f;
        const int pid = S.inputs[op.slot];
        const int pc = pid >= 0 ? p.stages[pid].channels : p.in_channels[-pid - 1];
        const int spec = pc == 1 ? 0 : op.chan;
        if (slot < 0) {
          slot = op.slot;
          chan = spec;
        } else if (slot != op.slot || chan != spec) {
          return f;
        }
        Lin l;
        l.is_const = false;
        l.t[{op.dx, op.dy}] = 1.0;
        st.push_back(l);
      } break;
      case WT_OP_ADD: case WT_OP_SUB: {
        Lin b = st.back(); st.pop_back();
        Lin a = st.back(); st.pop_back();
        st.push_back(add(a, b, op.op == WT_OP_ADD ? 1.0 : -1.0));
      } break;
      case WT_OP_MUL: {
        Lin b = st.back(); st.pop_back();
        Lin a = st.back(); st.pop_back();
        if (!a.ok || !b.ok) st.push_back(bad);
        else if (a.is_const) st.push_back(scale(b, a.c));
        else if (b.is_const) st.push_back(scale(a, b.c));
        else st.push_back(bad);
      } break;
      case WT_OP_DIV: {
        Lin b = st.back(); st.pop_back();
        Lin a = st.back(); st.pop_back();
        if (!a.ok || !b.ok || !b.is_const || b.c == 0) st.push_back(bad);
        else st.push_back(scale(a, 1.0 / b.c));
      } break;
      case WT_OP_NEG: st.back() = scale(st.back(), -1.0); break;
      default: return f;  // min, max, abs, sqrt, parities: not linear in the taps
    }
  }
  if (st.size() != 1 || !st.back().ok || st.back().is_const) return f;
  const Lin &l = st.back();
  int x0 = 1 << 20, x1 = -(1 << 20), y0 = 1 << 20, y1 = -(1 << 20);
  double wmax = 0, pv = 0;
  int pi = 0, pj = 0;
  for (auto &kv : l.t) {
    if (kv.second == 0) continue;
    x0 = std::min(x0, kv.first.first);
    x1 = std::max(x1, kv.first.first);
    y0 = std::min(y0, kv.first.second);
    y1 = std::max(y1, kv.first.second);
    wmax = std::max(wmax, std::fabs(kv.second));
  }
  if (wmax == 0) return f;
  const int nx = x1 - x0 + 1, ny = y1 - y0 + 1;
  std::vector<double> Wm((size_t)nx * ny, 0.0);
  for (auto &kv : l.t) {
    if (kv.second == 0) continue;
    const int i = kv.first.first - x0, j = kv.first.second - y0;
    Wm[(size_t)j * nx + i] = kv.second;
    if (std::fabs(kv.second) > std::fabs(pv)) {
      pv = kv.second;
      pi = i;
      pj = j;
    }
  }
  std::vector<double> v(nx), u(ny);
  for (int i = 0; i < nx; i++) v[i] = Wm[(size_t)pj * nx + i];
  for (int j = 0; j < ny; j++) u[j] = Wm[(size_t)j * nx + pi] / pv;
  for (int j = 0; j < ny; j++)
    for (int i = 0; i < nx; i++)
      if (std::fabs(Wm[(size_t)j * nx + i] - u[j] * v[i]) > 1e-9 * wmax) return f;  // rank > 1
  f.ok = true;
  f.slot = slot;
  f.chan = chan;
  f.dx0 = x0;
  f.dy0 = y0;
  f.wx = v;
  f.wy = u;
  f.c = l.c;
  return f;
}

bool down_streamable(const DownForm &f, int vo) {
  if (!f.ok) return false;
  const int dx1 = f.dx0 + (int)f.wx.size() - 1;
  // neighbour taps come from the adjacent lane only
  return -f.dx0 <= 2 * vo && dx1 - 1 <= 2 * vo && (int)f.wy.size() <= 16;
}

namespace {

// Shared-memory ring of the fast path: per warp RL steps x 2 producer rows,
// each row segment [left halo chunks | 32 x 2 VO own values | right halo
// chunks] in the storage type (16-byte chunks).
struct DownRing {
  int che = 8;         // elements per 16-byte chunk
  int ncl = 0, ncr = 0;  // halo chunks left / right of the warp's columns
  int sege = 0, segb = 0;  // row segment: elements, bytes
  int rl = 3;          // ring length in steps (multiple of NA)
  int pd = 2;          // prefetch distance in steps (rl - 1)
  int warp_bytes = 0;
};

DownRing down_ring(const DownForm &f, const CodegenKey &key) {
  DownRing r;
  const int esz = elem_bytes(key.src_dtypes.at(0));
  const int VO = key.vec;
  const int NX = (int)f.wx.size(), NY = (int)f.wy.size();
  const int LH = std::max(0, -f.dx0), RH = std::max(0, f.dx0 + NX - 2);
  const int NA = (NY - 1) / 2 + 1;
  r.che = 16 / esz;
  r.ncl = (LH + r.che - 1) / r.che;
  r.ncr = (RH + r.che - 1) / r.che;
  r.sege = (r.ncl + r.ncr) * r.che + 64 * VO;
  r.segb = r.sege * esz;
  const int depth = std::max(1, key.nbuf);  // requested prefetch distance (steps)
  r.rl = NA * ((depth + 1 + NA - 1) / NA);
  r.pd = r.rl - 1;
  r.warp_bytes = r.rl * 2 * r.segb;
  return r;
}

}  // namespace

int down_smem(const Pipeline &p, int sid, const CodegenKey &key) {
  return key.nw * down_ring(down_form(p, sid), key).warp_bytes;
}

std::string emit_down(const Pipeline &p, int sid, const CodegenKey &key, const std::string &kname) {
  const Stage &S = p.stages[sid];
  const DownForm f = down_form(p, sid);
  const int VO = key.vec, T = key.tby, NW = key.nw;
  if (!down_streamable(f, VO) || T < 1) fail(WT_EINVAL, "internal: stage is not a streamable down-sampling stencil");
  const int NX = (int)f.wx.size(), NY = (int)f.wy.size();
  const int DX0 = f.dx0, DY0 = f.dy0, DY1 = f.dy0 + NY - 1;
  const int DX1 = DX0 + NX - 1;
  const int LH = std::max(0, -DX0);     // values left of the lane's own 2 VO
  const int RH = std::max(0, DX1 - 1);  // values right of them
  const int NV = LH + 2 * VO + RH;
  const int NA = (DY1 - DY0) / 2 + 1;   // output rows open at once (ring)
  // steps: step m loads producer rows DY0 + 2m and DY0 + 2m + 1 (relative
  // to 2 yo0); output row j is complete after step j + NA - 1
  const int M = T + NA - 1;
  const int sdt = key.src_dtypes.at(0), ddt = key.dst_dtypes.at(0);
  const int sesz = elem_bytes(sdt), desz = elem_bytes(ddt);
  std::ostringstream o;
  o << kDeviceSource;
  o << "static_assert(sizeof(WtArgs) == " << sizeof(KernelArgs) << ", \"WtArgs layout\");\n";
  o << "extern \"C\" __global__ void __launch_bounds__(" << 32 * NW << ") " << kname
    << "(const __grid_constant__ WtArgs a) {\n";
  const DownRing R = down_ring(f, key);
  o << "extern __shared__ __align__(128) unsigned char wt_smem[];\n";
  o << "const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;\n";
  o << "const int W = a.W, H = a.H;\n";
  o << "const int xo0 = blockIdx.x * " << 32 * VO << ";\n";
  o << "const int yo0 = (blockIdx.y * " << NW << " + wid) * " << T << ";\n";
  o << "const int ch = blockIdx.z;\n(void)ch;\n";
  o << "if (yo0 >= H) return;\n";
  o << "const int Ws = a.src[0].W, Hs = a.src[0].H;\n";
  o << "const unsigned char *sp = (const unsigned char *)a.src[0].ptr + (wt_i64)"
    << (f.chan >= 0 ? std::to_string(f.chan) : std::string("ch")) << " * a.src[0].plane;\n";
  o << "const wt_i64 pitch = a.src[0].pitch;\n";
  o << "const int xs = 2 * (xo0 + lane * " << VO << ");\n";
  o << "unsigned char *dp = (unsigned char *)a.dst[0].ptr + (wt_i64)" << (S.channels > 1 ? "ch" : "0")
    << " * a.dst[0].plane;\n";
  o << "const int xo = xo0 + lane * " << VO << ";\n";
  // every column the warp reads (taps and the lanes' own segments, relative
  // to lane 0's and lane 31's xs) lies inside the row: 16-byte loads and
  // shuffles; else clamped scalar loads.  Warp-uniform.
  // The fast path copies the warp's columns and whole 16-byte halo chunks
  // on both sides: all of them must lie inside the row.
  o << "const bool fast = 2 * xo0 - " << R.ncl * R.che << " >= 0 && 2 * xo0 + " << 64 * VO + R.ncr * R.che
    << " <= Ws;\n";
  o << "unsigned char *wb = wt_smem + wid * " << R.warp_bytes << ";\n";
  o << "const wt_u32 wbs = wt_smem_u32(wb);\n(void)wbs;\n";
  // accumulators as packed FP32 pairs (outputs 2k, 2k + 1 of the lane)
  o << "wt_u64";
  for (int s = 0; s < NA; s++)
    for (int k = 0; k < VO / 2; k++) o << (s || k ? ", " : " ") << "acc" << s << "_" << k << " = 0";
  o << ";\n";
  // the column weights as packed pairs
  for (int dy = DY0; dy <= DY1; dy++)
    o << "const wt_u64 wy" << dy - DY0 << " = wt_pk(" << float_literal(f.wy[dy - DY0]) << ", "
      << float_literal(f.wy[dy - DY0]) << ");\n";
  // per-lane copy offsets of the fast path: the lane's own 2 VO values, and
  // the halo chunks left (lane 0) and right (lane 31) of the warp's columns
  o << "const wt_u32 mdo = (" << R.ncl * R.che << " + lane * " << 2 * VO << ") * " << sesz << ";\n";
  o << "const wt_i64 mso = (wt_i64)xs * " << sesz << ";\n";
  o << "const wt_u32 hdo = lane == 0 ? 0u : " << (R.ncl * R.che + 64 * VO) * sesz << "u;\n";
  o << "const wt_i64 hso = (wt_i64)(lane == 0 ? 2 * xo0 - " << R.ncl * R.che << " : 2 * xo0 + " << 64 * VO << ") * "
    << sesz << ";\n";
  for (int c = 0; c < std::max(R.ncl, R.ncr); c++)
    o << "const bool hp" << c << " = " << (c < R.ncl ? "lane == 0" : "false") << " || "
      << (c < R.ncr ? "lane == 31" : "false") << ";\n";
  o << "(void)mdo; (void)mso; (void)hdo; (void)hso;\n";
  auto vn = [](int q, int i) { return "v" + std::to_string(q) + "_" + std::to_string(i); };
  // cp.async of both producer rows of step `mexpr` into ring slot `slot`
  auto issue = [&](int slot, const std::string &mexpr) {
    for (int q = 0; q < 2; q++) {
      o << "{ const unsigned char *gp = sp + (wt_i64)wt_clampi(2 * yo0 + (" << DY0 + q << ") + 2 * (" << mexpr
        << "), 0, Hs - 1) * pitch;\n";
      o << "const wt_u32 sb = wbs + " << (slot * 2 + q) * R.segb << ";\n";
      for (int c = 0; c < 2 * VO * sesz / 16; c++)
        o << "wt_cp_async16(sb + mdo + " << 16 * c << ", gp + mso + " << 16 * c << ");\n";
      for (int c = 0; c < std::max(R.ncl, R.ncr); c++)
        o << "wt_cp_async16_if(hp" << c << ", sb + hdo + " << 16 * c << ", gp + hso + " << 16 * c << ");\n";
      o << "}\n";
    }
  };
  // one step: slot base u (compile time), step index expression mexpr
  auto step = [&](bool fast, int u, const std::string &mexpr) {
    o << "{\nconst int m = " << mexpr << ";\n";
    // both rows' loads first (in flight together)
    if (fast) {
      // refill the slot freed by the previous step with the rows of step
      // m + PD, then wait until this step's rows have landed
      o << "if (m + " << R.pd << " < " << M << ") {\n";
      issue(((u + R.pd) % R.rl), "m + " + std::to_string(R.pd));
      o << "}\nwt_cp_async_commit();\nWT_CP_ASYNC_WAIT(" << R.pd << ");\n__syncwarp();\n";
    }
    for (int q = 0; q < 2; q++) {
      if (!fast)
        o << "const unsigned char *rp" << q << " = sp + (wt_i64)wt_clampi(2 * yo0 + (" << DY0 + q
          << ") + 2 * m, 0, Hs - 1) * pitch;\n";
      o << "float";
      for (int i = 0; i < NV; i++) o << (i ? ", " : " ") << vn(q, i);
      o << ";\n";
      if (fast) {
        // this step's rows from the ring slot (copies waited for above)
        const int row = (u % R.rl) * 2 + q;
        o << "const unsigned char *sb" << q << " = wb + " << row * R.segb << " + (" << R.ncl * R.che << " + lane * "
          << 2 * VO << ") * " << sesz << ";\n";
        for (int b = 0; b < 2 * VO; b += 8) {
          o << "wt_lds8_" << dtype_name(sdt) << "(sb" << q << " + " << b * sesz;
          for (int t = 0; t < 8; t++) o << ", " << vn(q, LH + b + t);
          o << ");\n";
        }
        for (int k = 0; k < LH; k++)
          o << vn(q, k) << " = wt_lds1_" << dtype_name(sdt) << "(sb" << q << " - " << (LH - k) * sesz << ");\n";
        for (int k = 0; k < RH; k++)
          o << vn(q, LH + 2 * VO + k) << " = wt_lds1_" << dtype_name(sdt) << "(sb" << q << " + " << (2 * VO + k) * sesz
            << ");\n";
      } else {
        for (int i = 0; i < NV; i++)
          o << vn(q, i) << " = wt_ld1_" << dtype_name(sdt) << "(rp" << q << " + (wt_i64)wt_clampi(xs + (" << i - LH
            << "), 0, Ws - 1) * " << sesz << ");\n";
      }
    }
    for (int q = 0; q < 2; q++) {
      // row pass at stride 2
      for (int k = 0; k < VO; k++) {
        o << "const float h" << q << "_" << k << " = ";
        bool first = true;
        for (int i = 0; i < NX; i++) {
          if (f.wx[i] == 0) continue;
          o << (first ? "" : " + ") << float_literal(f.wx[i]) << " * " << vn(q, LH + 2 * k + DX0 + i);
          first = false;
        }
        o << ";\n";
      }
      // column pass: this row is tap dy of output j = m + delta
      for (int dy = DY0; dy <= DY1; dy++) {
        if (((DY0 + q - dy) % 2 + 2) % 2 != 0) continue;
        const double w = f.wy[dy - DY0];
        const int delta = (DY0 + q - dy) / 2;  // <= 0
        const int slot = ((u + delta) % NA + NA) % NA;
        if (w == 0 && dy != DY0) continue;
        for (int k = 0; k < VO / 2; k++) {
          const std::string hp = "wt_pk(h" + std::to_string(q) + "_" + std::to_string(2 * k) + ", h" +
                                 std::to_string(q) + "_" + std::to_string(2 * k + 1) + ")";
          const std::string acc = "acc" + std::to_string(slot) + "_" + std::to_string(k);
          if (dy == DY0)
            o << acc << " = wt_mul2(wy" << dy - DY0 << ", " << hp << ");\n";
          else
            o << acc << " = wt_fma2(wy" << dy - DY0 << ", " << hp << ", " << acc << ");\n";
        }
        if (dy != DY1) continue;
        // output row j is complete (rows j < 0 and j >= T are not stored)
        o << "{ const int j = m + (" << delta << "), yo = yo0 + j;\n";
        o << "if (j >= 0 && j < " << T << " && yo < H) {\n";
        o << "unsigned char *op_ = dp + (wt_i64)yo * a.dst[0].pitch;\n";
        std::vector<std::string> outv;
        o << "float";
        for (int k = 0; k < VO; k++) o << (k ? ", " : " ") << "o" << k;
        o << ";\n";
        for (int k = 0; k < VO / 2; k++)
          o << "wt_upk(acc" << slot << "_" << k << ", o" << 2 * k << ", o" << 2 * k + 1 << ");\n";
        for (int k = 0; k < VO; k++) {
          std::string e = "o" + std::to_string(k);
          if (f.c != 0) e = "(" + e + " + " + float_literal(f.c) + ")";
          outv.push_back(e);
        }
        o << "if (xo + " << VO << " <= W) {\n";
        for (int b = 0; b < VO; b += 4)
          o << "wt_st4_" << dtype_name(ddt) << "(op_ + (wt_i64)(xo + " << b << ") * " << desz << ", " << outv[b] << ", "
            << outv[b + 1] << ", " << outv[b + 2] << ", " << outv[b + 3] << ");\n";
        o << "} else {\n";
        for (int k = 0; k < VO; k++)
          o << "if (xo + " << k << " < W) wt_st1_" << dtype_name(ddt) << "(op_ + (wt_i64)(xo + " << k << ") * " << desz
            << ", " << outv[k] << ");\n";
        o << "}\n}\n}\n";
      }
    }
    if (fast) o << "__syncwarp();\n";  // slot read by all lanes before its refill
    o << "}\n";
  };
  // whole rounds of NA steps (ring slots fixed per unrolled step), then the
  // remaining M mod NA steps; both paths, chosen once per warp
  for (int fpath = 1; fpath >= 0; fpath--) {
    // rounds of `un` steps: a multiple of NA (accumulator slots) and, on
    // the fast path, of the ring length (ring slots)
    const int un = fpath ? R.rl : NA;
    const int full = M / un * un;
    o << (fpath ? "if (fast) {\n" : "} else {\n");
    if (fpath) {
      for (int m = 0; m < R.pd; m++) {
        if (m < M) issue(m % R.rl, std::to_string(m));
        o << "wt_cp_async_commit();\n";
      }
    }
    if (full > 0) {
      o << "#pragma unroll 1\nfor (int m0 = 0; m0 < " << full << "; m0 += " << un << ") {\n";
      for (int u = 0; u < un; u++) step(fpath != 0, u, "m0 + " + std::to_string(u));
      o << "}\n";
    }
    for (int u = 0; u < M - full; u++) step(fpath != 0, u, std::to_string(full + u));
    if (fpath) o << "WT_CP_ASYNC_WAIT(0);\n";
  }
  o << "}\n}\n";
  return o.str();
}

}  // namespace wt

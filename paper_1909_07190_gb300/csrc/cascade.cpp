// Two-level down-sampling cascade: a group spanning two pyramid levels
// (Sec. 5: after alignment and scaling every dependence vector of the group
// is constant).  Stage S1 reduces its producer P one level (S1(x, y) =
// sum_{dx,dy} w1 P(2x + dx, 2y + dy)) and stage S2 reduces S1 one level
// further with a centred form.  Scaled to P's grid, S1's points sit at even
// and S2's at multiples of four, so one warp can stream P's rows and
// complete S1's rows at half and S2's at a quarter of P's row rate; S1's
// rows go to memory and on into S2's accumulators without being read back.
//
// Warp geometry (x): lane l holds VO1 consecutive S1 columns starting at
// b0 + l VO1, and its S2 outputs are the VO2 = VO1 / 2 columns whose taps
// start there.  S2's taps reach into the neighbouring lanes' S1 columns, so
// lanes 0 and 31 only compute halo: lanes 1..30 write 30 VO1 S1 columns
// and 30 VO2 S2 columns per warp, and neighbouring warps overlap by two
// lanes.  A completed S1 row is exchanged through a per-warp shared row
// (read with clamped columns in the warps at the image's left and right
// edges, where S2 reads S1 clamped to the edge).
//
// Warp geometry (y): a warp owns T2 rows of S2 and the 2 T2 rows of S1
// under them, and streams the S1 rows from R2 above to R2 below its S2 rows
// (R2 = S2's vertical tap radius); at the image's top and bottom, S2's taps
// of S1 rows outside the image take the edge row (clamp-to-edge), added
// when the edge row completes.
#include <algorithm>
#include <sstream>

#include "wt_internal.hpp"

namespace wt {

// S2 = a centred reduce of S1 (odd tap counts, radius at most 2 along y,
// x taps inside a lane's neighbours at 4 S1 values per lane), per channel
// of S1 (or both one-channel).
bool cascade_pair_ok(const Pipeline &p, int s1, int s2) {
  if (s1 < 0 || s2 < 0 || s1 >= (int)p.stages.size() || s2 >= (int)p.stages.size()) return false;
  const DownForm f1 = down_form(p, s1), f2 = down_form(p, s2);
  if (!f1.ok || !f2.ok || !down_streamable(f1, 4)) return false;
  if (p.stages[s2].inputs[f2.slot] != s1) return false;
  const int C1 = p.stages[s1].channels, C2 = p.stages[s2].channels;
  if (C1 != C2 || (C1 > 1 && f2.chan >= 0)) return false;
  const int NY2 = (int)f2.wy.size(), NX2 = (int)f2.wx.size();
  if (NY2 % 2 == 0 || f2.dy0 != -(NY2 - 1) / 2 || (NY2 - 1) / 2 > 2) return false;
  if (-f2.dx0 > 4 || f2.dx0 + NX2 - 1 > 5) return false;
  return true;
}

// Launch units of a cascade group: in stage order, each stage pairs with
// the first later stage of the segment that it produces and that can
// follow it; unpaired stages run alone.  Empty unless every stage is a
// streamable down-sampling stage, the group spans two consecutive levels
// and at least one pair forms.
std::vector<CascadeUnit> cascade_units(const Pipeline &p, const std::vector<int> &seg) {
  std::vector<CascadeUnit> u;
  if (seg.size() < 2) return u;
  int lo = 1 << 20, hi = -1;
  for (int s : seg) {
    if (s < 0 || s >= (int)p.stages.size()) return {};
    const DownForm f = down_form(p, s);
    if (!down_streamable(f, 4)) return {};
    lo = std::min(lo, p.stages[s].level);
    hi = std::max(hi, p.stages[s].level);
  }
  if (hi != lo + 1) return {};
  std::vector<int> role(seg.size(), 0);  // 0 open, 1 first of a pair, 2 second
  bool any = false;
  for (size_t i = 0; i < seg.size(); i++) {
    if (role[i] != 0) continue;
    for (size_t k = i + 1; k < seg.size(); k++)
      if (role[k] == 0 && cascade_pair_ok(p, seg[i], seg[k])) {
        role[i] = 1;
        role[k] = 2;
        u.push_back({seg[i], seg[k]});
        any = true;
        break;
      }
    if (role[i] == 0) u.push_back({seg[i], -1});
  }
  if (!any) return {};
  // launch order: a unit runs at its last stage's position (its producers
  // come earlier in stage order)
  std::stable_sort(u.begin(), u.end(), [](const CascadeUnit &a, const CascadeUnit &b) {
    return std::max(a.s1, a.s2) < std::max(b.s1, b.s2);
  });
  return u;
}

namespace {

struct CasRing {
  int che = 8;             // elements per 16-byte chunk
  int ncl = 0, ncr = 0;    // halo chunks left / right of the warp's P columns
  int sege = 0, segb = 0;  // one P row segment: elements, bytes
  int rl = 3, pd = 2;      // ring length and prefetch distance in steps
  int ring_bytes = 0;
  int xr = 0;              // floats per exchange row
  int warp_bytes = 0;
};

constexpr int kLP = 4, kRP = 4;  // exchange-row pads (floats) left / right

CasRing cas_ring(const DownForm &f1, const CodegenKey &key) {
  CasRing r;
  const int esz = elem_bytes(key.src_dtypes.at(0));
  const int VO1 = key.vec;
  const int NX = (int)f1.wx.size(), NY = (int)f1.wy.size();
  const int LH = std::max(0, -f1.dx0), RH = std::max(0, f1.dx0 + NX - 2);
  const int NA = (NY - 1) / 2 + 1;
  r.che = 16 / esz;
  r.ncl = (LH + r.che - 1) / r.che;
  r.ncr = (RH + r.che - 1) / r.che;
  r.sege = (r.ncl + r.ncr) * r.che + 64 * VO1;
  r.segb = r.sege * esz;
  const int depth = std::max(1, key.nbuf);
  r.rl = NA * ((depth + 1 + NA - 1) / NA);
  r.pd = r.rl - 1;
  r.ring_bytes = r.rl * 2 * r.segb;
  r.xr = kLP + 32 * VO1 + kRP;
  r.warp_bytes = (r.ring_bytes + 15) / 16 * 16 + 2 * r.xr * 4;
  return r;
}

int gcd_(int a, int b) { return b ? gcd_(b, a % b) : a; }
int lcm_(int a, int b) { return a / gcd_(a, b) * b; }

}  // namespace

int cascade_smem(const Pipeline &p, int s1, const CodegenKey &key) {
  return key.nw * cas_ring(down_form(p, s1), key).warp_bytes;
}

std::string emit_cascade(const Pipeline &p, int s1, int s2, const CodegenKey &key, const std::string &kname) {
  if (!cascade_pair_ok(p, s1, s2)) fail(WT_EINVAL, "internal: not a two-level down-sampling cascade");
  const DownForm f1 = down_form(p, s1), f2 = down_form(p, s2);
  const int VO1 = key.vec, VO2 = VO1 / 2, T2 = key.tby, NW = key.nw;
  if ((VO1 != 4 && VO1 != 8) || T2 < 1 || !down_streamable(f1, VO1))
    fail(WT_EINVAL, "internal: cascade kernel parameters");
  // S1 from P (as the single-level streaming kernel)
  const int NX1 = (int)f1.wx.size(), NY1 = (int)f1.wy.size();
  const int DX0 = f1.dx0, DY0 = f1.dy0, DY1 = f1.dy0 + NY1 - 1, DX1 = DX0 + NX1 - 1;
  const int LH = std::max(0, -DX0), RH = std::max(0, DX1 - 1);
  const int NV = LH + 2 * VO1 + RH;
  const int NA1 = (DY1 - DY0) / 2 + 1;
  // S2 from S1: centred, radius R2 along y; exchange taps EX0..EX1 relative
  // to a lane's first S1 column
  const int NX2 = (int)f2.wx.size(), NY2 = (int)f2.wy.size();
  const int R2 = (NY2 - 1) / 2, NA2 = R2 + 1;
  const int EX0 = f2.dx0, EX1 = VO1 - 2 + f2.dx0 + NX2 - 1;
  // S1 rows streamed per warp: R2 above to R2 below the 2 T2 owned rows;
  // step m completes S1 row j = m - (NA1 - 1)
  const int J1 = 2 * T2 + 2 * R2 - 1;
  const int M = J1 + NA1 - 1;
  const int sdt = key.src_dtypes.at(0), d1 = key.dst_dtypes.at(0), d2 = key.dst_dtypes.at(1);
  const int sesz = elem_bytes(sdt), e1 = elem_bytes(d1), e2 = elem_bytes(d2);
  const CasRing R = cas_ring(f1, key);
  const Stage &S1 = p.stages[s1], &S2 = p.stages[s2];
  std::ostringstream o;
  o << kDeviceSource;
  o << "static_assert(sizeof(WtArgs) == " << sizeof(KernelArgs) << ", \"WtArgs layout\");\n";
  // register cap through the launch bounds: enough resident blocks that
  // each thread gets at most max_regs
  const int min_blocks = key.max_regs > 0 ? std::max(1, 65536 / (key.max_regs * 32 * NW)) : 1;
  o << "extern \"C\" __global__ void __launch_bounds__(" << 32 * NW << ", " << min_blocks << ") " << kname
    << "(const __grid_constant__ WtArgs a) {\n";
  o << "extern __shared__ __align__(128) unsigned char wt_smem[];\n";
  o << "const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;\n";
  o << "const int W1 = a.dst[0].W, H1 = a.dst[0].H, W2 = a.dst[1].W, H2 = a.dst[1].H;\n";
  o << "const int y2_0 = ((int)blockIdx.y * " << NW << " + wid) * " << T2 << ";\n";
  o << "if (y2_0 >= H2) return;\n";
  o << "const int b0 = (int)blockIdx.x * " << 30 * VO1 << " - " << VO1 << ";\n";
  o << "const int x2_0 = (int)blockIdx.x * " << 15 * VO1 << ";\n";
  o << "const int ch = blockIdx.z;\n(void)ch;\n";
  o << "const int R1s = 2 * y2_0 - " << R2 << ";\n";
  o << "const int Ws = a.src[0].W, Hs = a.src[0].H;\n";
  o << "const unsigned char *sp = (const unsigned char *)a.src[0].ptr + (wt_i64)"
    << (f1.chan >= 0 ? std::to_string(f1.chan) : std::string("ch")) << " * a.src[0].plane;\n";
  o << "const wt_i64 pitch = a.src[0].pitch;\n";
  o << "const int c1 = b0 + lane * " << VO1 << ";\n";
  o << "const int xs = 2 * c1;\n";
  o << "unsigned char *dp1 = (unsigned char *)a.dst[0].ptr + (wt_i64)" << (S1.channels > 1 ? "ch" : "0")
    << " * a.dst[0].plane;\n";
  o << "unsigned char *dp2 = (unsigned char *)a.dst[1].ptr + (wt_i64)" << (S2.channels > 1 ? "ch" : "0")
    << " * a.dst[1].plane;\n";
  o << "const bool own = lane >= 1 && lane <= 30;\n";
  o << "const int x2 = x2_0 + (lane - 1) * " << VO2 << ";\n";
  // P columns of the warp and its halo chunks inside the row: 16-byte
  // copies into the ring; else clamped scalar loads.  Warp-uniform.
  o << "const bool fast = 2 * b0 - " << R.ncl * R.che << " >= 0 && 2 * b0 + " << 64 * VO1 + R.ncr * R.che
    << " <= Ws;\n";
  // S2's taps of lanes 1..30 reach outside S1's columns: clamped exchange
  // reads.  Warp-uniform.
  o << "const bool xedge = b0 + " << VO1 + EX0 << " < 0 || b0 + " << 30 * VO1 + EX1 << " > W1 - 1;\n";
  o << "unsigned char *wb = wt_smem + wid * " << R.warp_bytes << ";\n";
  o << "const wt_u32 wbs = wt_smem_u32(wb);\n(void)wbs;\n";
  o << "float *xb = (float *)(wb + " << (R.ring_bytes + 15) / 16 * 16 << ");\n";
  o << "if (lane < " << 2 * (kLP + kRP) << ") xb[(lane >> 3) * " << R.xr << " + ((lane & 7) < " << kLP
    << " ? (lane & 7) : " << kLP + 32 * VO1 - kLP << " + (lane & 7))] = 0.f;\n";
  // S1 accumulators as packed FP32 pairs, the column weights as pairs
  o << "wt_u64";
  for (int s = 0; s < NA1; s++)
    for (int k = 0; k < VO1 / 2; k++) o << (s || k ? ", " : " ") << "acc" << s << "_" << k << " = 0";
  o << ";\n";
  for (int dy = DY0; dy <= DY1; dy++)
    o << "const wt_u64 wy" << dy - DY0 << " = wt_pk(" << float_literal(f1.wy[dy - DY0]) << ", "
      << float_literal(f1.wy[dy - DY0]) << ");\n";
  // per-lane copy offsets: the lane's own 2 VO1 values, and the halo
  // chunks left (lane 0) and right (lane 31) of the warp's columns
  o << "const wt_u32 mdo = (" << R.ncl * R.che << " + lane * " << 2 * VO1 << ") * " << sesz << ";\n";
  o << "const wt_i64 mso = (wt_i64)xs * " << sesz << ";\n";
  o << "const wt_u32 hdo = lane == 0 ? 0u : " << (R.ncl * R.che + 64 * VO1) * sesz << "u;\n";
  o << "const wt_i64 hso = (wt_i64)(lane == 0 ? 2 * b0 - " << R.ncl * R.che << " : 2 * b0 + " << 64 * VO1 << ") * "
    << sesz << ";\n";
  for (int c = 0; c < std::max(R.ncl, R.ncr); c++)
    o << "const bool hp" << c << " = " << (c < R.ncl ? "lane == 0" : "false") << " || "
      << (c < R.ncr ? "lane == 31" : "false") << ";\n";
  o << "(void)mdo; (void)mso; (void)hdo; (void)hso;\n";
  o << "float";
  for (int s = 0; s < NA2; s++)
    for (int k = 0; k < VO2; k++) o << (s || k ? ", " : " ") << "bcc" << s << "_" << k << " = 0.f";
  o << ";\n";
  auto vn = [](int q, int i) { return "v" + std::to_string(q) + "_" + std::to_string(i); };
  auto mod = [](int a, int b) { return ((a % b) + b) % b; };
  // cp.async of both P rows of step `mexpr` into ring slot `slot`
  auto issue = [&](int slot, const std::string &mexpr) {
    for (int q = 0; q < 2; q++) {
      o << "{ const unsigned char *gp = sp + (wt_i64)wt_clampi(2 * R1s + (" << DY0 + q << ") + 2 * (" << mexpr
        << "), 0, Hs - 1) * pitch;\n";
      o << "const wt_u32 sb = wbs + " << (slot * 2 + q) * R.segb << ";\n";
      for (int c = 0; c < 2 * VO1 * sesz / 16; c++)
        o << "wt_cp_async16(sb + mdo + " << 16 * c << ", gp + mso + " << 16 * c << ");\n";
      for (int c = 0; c < std::max(R.ncl, R.ncr); c++)
        o << "wt_cp_async16_if(hp" << c << ", sb + hdo + " << 16 * c << ", gp + hso + " << 16 * c << ");\n";
      o << "}\n";
    }
  };
  // S2 accumulation of h2 as the value of S1 row j (jr = j modulo 2 NA2):
  // tap dy2 of S2 row i = (j - R2 - dy2) / 2, held in slot i modulo NA2
  auto add2 = [&](int jr, int dy2, const std::string &pre) {
    if (mod(jr - R2 - dy2, 2) != 0) return;
    const double w = f2.wy[dy2 + R2];
    if (w == 0) return;
    const int slot = mod((jr - R2 - dy2) / 2, NA2);  // (jr - R2 - dy2) is even
    for (int k = 0; k < VO2; k++)
      o << pre << "bcc" << slot << "_" << k << " += " << float_literal(w) << " * h2_" << k << ";\n";
  };
  // S1 row j complete in accumulator slot `slot1`; jr = j modulo U
  auto row_done = [&](int slot1, int jr, const std::string &jexpr) {
    o << "{ const int j = " << jexpr << ";\nif (j >= 0) {\nconst int r1 = R1s + j;\n";
    o << "float";
    for (int k = 0; k < VO1; k++) o << (k ? ", " : " ") << "g" << k;
    o << ";\n";
    for (int k = 0; k < VO1 / 2; k++)
      o << "wt_upk(acc" << slot1 << "_" << k << ", g" << 2 * k << ", g" << 2 * k + 1 << ");\n";
    if (f1.c != 0)
      for (int k = 0; k < VO1; k++) o << "g" << k << " += " << float_literal(f1.c) << ";\n";
    // S1 to memory: owned lanes and rows inside the image
    o << "if (own && (unsigned)(j - " << R2 << ") < " << 2 * T2 << "u && r1 < H1 && c1 < W1) {\n";
    o << "unsigned char *op_ = dp1 + (wt_i64)r1 * a.dst[0].pitch;\n";
    o << "if (c1 + " << VO1 << " <= W1) {\n";
    for (int b = 0; b < VO1; b += 4)
      o << "wt_st4_" << dtype_name(d1) << "(op_ + (wt_i64)(c1 + " << b << ") * " << e1 << ", g" << b << ", g" << b + 1
        << ", g" << b + 2 << ", g" << b + 3 << ");\n";
    o << "} else {\n";
    for (int k = 0; k < VO1; k++)
      o << "if (c1 + " << k << " < W1) wt_st1_" << dtype_name(d1) << "(op_ + (wt_i64)(c1 + " << k << ") * " << e1
        << ", g" << k << ");\n";
    o << "}\n}\n";
    // S2's taps of S1: the lane's own values and its neighbours' by warp
    // shuffles; at the image's left and right edges through the exchange
    // row (double-buffered by row parity), columns clamped to the image
    o << "float";
    for (int t = EX0; t <= EX1; t++) o << (t == EX0 ? " " : ", ") << "e" << t - EX0;
    o << ";\nif (!xedge) {\n";
    for (int t = EX0; t <= EX1; t++) {
      if (t < 0)
        o << "e" << t - EX0 << " = __shfl_up_sync(0xffffffffu, g" << VO1 + t << ", 1);\n";
      else if (t < VO1)
        o << "e" << t - EX0 << " = g" << t << ";\n";
      else
        o << "e" << t - EX0 << " = __shfl_down_sync(0xffffffffu, g" << t - VO1 << ", 1);\n";
    }
    o << "} else {\n";
    o << "float *xr = xb + " << mod(jr, 2) * R.xr << ";\n";
    for (int b = 0; b < VO1; b += 4)
      o << "*(float4 *)(xr + " << kLP + b << " + lane * " << VO1 << ") = make_float4(g" << b << ", g" << b + 1
        << ", g" << b + 2 << ", g" << b + 3 << ");\n";
    o << "__syncwarp();\n";
    for (int t = EX0; t <= EX1; t++)
      o << "e" << t - EX0 << " = xr[" << kLP << " + wt_clampi(c1 + (" << t << "), 0, W1 - 1) - b0];\n";
    o << "}\n";
    // S2 row pass at stride 2
    for (int k = 0; k < VO2; k++) {
      o << "const float h2_" << k << " = ";
      bool first = true;
      for (int i = 0; i < NX2; i++) {
        if (f2.wx[i] == 0) continue;
        o << (first ? "" : " + ") << float_literal(f2.wx[i]) << " * e" << 2 * k + i;
        first = false;
      }
      if (first) o << "0.f";
      o << ";\n";
    }
    // S2 taps of this row (rows of S1 inside the image)
    o << "if ((unsigned)r1 < (unsigned)H1) {\n";
    for (int dy2 = -R2; dy2 <= R2; dy2++) add2(jr, dy2, "");
    o << "}\n";
    // the S2 row whose last tap this is: store, then free its slot
    if (mod(jr - 2 * R2, 2) == 0) {
      const int slot = mod((jr - 2 * R2) / 2, NA2);
      o << "{ const int i2 = (j - " << 2 * R2 << ") >> 1, y2 = y2_0 + i2;\n";
      o << "if (j >= " << 2 * R2 << " && i2 < " << T2 << " && y2 < H2 && own && x2 < W2) {\n";
      o << "unsigned char *op_ = dp2 + (wt_i64)y2 * a.dst[1].pitch;\n";
      std::vector<std::string> ov;
      for (int k = 0; k < VO2; k++) {
        std::string e = "bcc" + std::to_string(slot) + "_" + std::to_string(k);
        if (f2.c != 0) e = "(" + e + " + " + float_literal(f2.c) + ")";
        ov.push_back(e);
      }
      if (VO2 % 4 == 0) {
        o << "if (x2 + " << VO2 << " <= W2) {\n";
        for (int b = 0; b < VO2; b += 4)
          o << "wt_st4_" << dtype_name(d2) << "(op_ + (wt_i64)(x2 + " << b << ") * " << e2 << ", " << ov[b] << ", "
            << ov[b + 1] << ", " << ov[b + 2] << ", " << ov[b + 3] << ");\n";
        o << "} else {\n";
      } else {
        o << "{\n";
      }
      for (int k = 0; k < VO2; k++)
        o << "if (x2 + " << k << " < W2) wt_st1_" << dtype_name(d2) << "(op_ + (wt_i64)(x2 + " << k << ") * " << e2
          << ", " << ov[k] << ");\n";
      o << "}\n}\n";
      for (int k = 0; k < VO2; k++) o << "bcc" << slot << "_" << k << " = 0.f;\n";
      o << "}\n";
    }
    // clamp-to-edge of S2's taps: S1 rows above the image take row 0 (top
    // warp, when row 0 completes), rows below take row H1 - 1
    if (mod(jr - R2, 2 * NA2) == 0) {
      o << "if (y2_0 == 0 && j == " << R2 << ") {\n";
      for (int t = 1; t <= R2; t++)
        for (int dy2 = -R2; dy2 <= -t; dy2++) add2(mod(jr - t, 2 * NA2), dy2, "");
      o << "}\n";
    }
    o << "if (r1 == H1 - 1) {\n";
    for (int t = 1; t <= R2; t++)
      for (int dy2 = -R2; dy2 <= R2; dy2++) add2(mod(jr + t, 2 * NA2), dy2, "");
    o << "}\n";
    o << "}\n}\n";
  };
  // one step: P rows DY0 + 2m and DY0 + 2m + 1 (relative to 2 R1s), ring
  // slot base u (compile time), step index expression mexpr
  auto step = [&](bool fast, int u, const std::string &mexpr) {
    std::pair<int, int> done{0, 0};  // slot and delta of the S1 row completed by this step
    o << "{\nconst int m = " << mexpr << ";\n";
    if (fast) {
      o << "if (m + " << R.pd << " < " << M << ") {\n";
      issue(mod(u + R.pd, R.rl), "m + " + std::to_string(R.pd));
      o << "}\nwt_cp_async_commit();\nWT_CP_ASYNC_WAIT(" << R.pd << ");\n__syncwarp();\n";
    }
    for (int q = 0; q < 2; q++) {
      if (!fast)
        o << "const unsigned char *rp" << q << " = sp + (wt_i64)wt_clampi(2 * R1s + (" << DY0 + q
          << ") + 2 * m, 0, Hs - 1) * pitch;\n";
      o << "float";
      for (int i = 0; i < NV; i++) o << (i ? ", " : " ") << vn(q, i);
      o << ";\n";
      if (fast) {
        const int row = mod(u, R.rl) * 2 + q;
        o << "const unsigned char *sb" << q << " = wb + " << row * R.segb << " + (" << R.ncl * R.che << " + lane * "
          << 2 * VO1 << ") * " << sesz << ";\n";
        for (int b = 0; b < 2 * VO1; b += 8) {
          o << "wt_lds8_" << dtype_name(sdt) << "(sb" << q << " + " << b * sesz;
          for (int t = 0; t < 8; t++) o << ", " << vn(q, LH + b + t);
          o << ");\n";
        }
        for (int k = 0; k < LH; k++)
          o << vn(q, k) << " = wt_lds1_" << dtype_name(sdt) << "(sb" << q << " - " << (LH - k) * sesz << ");\n";
        for (int k = 0; k < RH; k++)
          o << vn(q, LH + 2 * VO1 + k) << " = wt_lds1_" << dtype_name(sdt) << "(sb" << q << " + "
            << (2 * VO1 + k) * sesz << ");\n";
      } else {
        for (int i = 0; i < NV; i++)
          o << vn(q, i) << " = wt_ld1_" << dtype_name(sdt) << "(rp" << q << " + (wt_i64)wt_clampi(xs + (" << i - LH
            << "), 0, Ws - 1) * " << sesz << ");\n";
      }
      // S1 row pass at stride 2 (one P row at a time: fewer live values)
      for (int k = 0; k < VO1; k++) {
        o << "const float h" << q << "_" << k << " = ";
        bool first = true;
        for (int i = 0; i < NX1; i++) {
          if (f1.wx[i] == 0) continue;
          o << (first ? "" : " + ") << float_literal(f1.wx[i]) << " * " << vn(q, LH + 2 * k + DX0 + i);
          first = false;
        }
        o << ";\n";
      }
      // S1 column pass: this P row is tap dy of S1 row j = m + delta
      for (int dy = DY0; dy <= DY1; dy++) {
        if (mod(DY0 + q - dy, 2) != 0) continue;
        const double w = f1.wy[dy - DY0];
        const int delta = (DY0 + q - dy) / 2;  // <= 0
        const int slot = mod(u + delta, NA1);
        if (w == 0 && dy != DY0 && dy != DY1) continue;
        for (int k = 0; k < VO1 / 2; k++) {
          const std::string hp = "wt_pk(h" + std::to_string(q) + "_" + std::to_string(2 * k) + ", h" +
                                 std::to_string(q) + "_" + std::to_string(2 * k + 1) + ")";
          const std::string acc = "acc" + std::to_string(slot) + "_" + std::to_string(k);
          if (dy == DY0)
            o << acc << " = wt_mul2(wy" << dy - DY0 << ", " << hp << ");\n";
          else
            o << acc << " = wt_fma2(wy" << dy - DY0 << ", " << hp << ", " << acc << ");\n";
        }
        if (dy == DY1) done = {slot, delta};
      }
    }
    if (fast) o << "__syncwarp();\n";  // ring slot read by all lanes before its refill
    // the completed S1 row (its slot is not touched by the other P row of
    // the step), after both P rows' values are dead
    row_done(done.first, mod(u + done.second, 2 * NA2), "m + (" + std::to_string(done.second) + ")");
    o << "}\n";
  };
  for (int fpath = 1; fpath >= 0; fpath--) {
    // rounds of `un` steps: a multiple of NA1 (S1 slots), of 2 NA2 (S2
    // slots and row parity) and, on the fast path, of the ring length
    const int un = fpath ? lcm_(R.rl, lcm_(NA1, 2 * NA2)) : lcm_(NA1, 2 * NA2);
    const int full = M / un * un;
    o << (fpath ? "if (fast) {\n" : "} else {\n");
    if (fpath) {
      for (int m = 0; m < R.pd; m++) {
        if (m < M) issue(mod(m, R.rl), std::to_string(m));
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

// CUDA source generation for group kernels (Fig. 4 "CUDA Code Generation").
//
// Fused groups (OTPW + hybrid tiling, Sec. 4-5, Alg. 1 / Alg. 3 in the
// streaming form described in analysis.cpp):
//   * one warp = one overlapped tile: 32 lanes along x, V pixels per lane
//     (128-bit accesses), tile_h output rows; warps never synchronise with
//     each other, and a warp only uses __syncwarp / shuffles (Sec. 4);
//   * the tile's source rows (tile + halo) are staged by TMA into the warp's
//     shared-memory ring, chunk by chunk, completion on per-buffer
//     mbarriers, with bounded waits;
//   * the warp walks the parallelogram tiles (skewed rows) in order; each
//     stage keeps its last `window` rows either in registers (explicitly
//     named scalars, rotated by unrolling: D4 of the paper) or in a
//     shared-memory ring (the hybrid split, fracReg);
//   * producer loads become the four load types of Sec. 5 / Fig. 5: own
//     register (1), shared memory (2), another lane's register of the same
//     parallelogram row via __shfl (3), another lane's register of an
//     earlier parallelogram row (4: the neighbour values shuffled when that
//     row was produced);
//   * clamp-to-edge at every producer read: border tiles replicate edge
//     rows/columns of each stage (and clamp ring reads), interior tiles run
//     a guard-free body in the steady state.
// Plain groups: one simple kernel per stage reading producers from global
// memory with clamped scalar loads (the unfused baseline).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <map>
#include <set>
#include <functional>
#include <sstream>

#include "wt_internal.hpp"

namespace wt {

const char *dtype_name(int dtype) { return dtype == WT_F32 ? "f32" : (dtype == WT_F16 ? "f16" : "bf16"); }

std::string float_literal(float v) {
  if (std::isnan(v)) return "__int_as_float(0x7fc00000)";
  if (std::isinf(v)) return v > 0 ? "__int_as_float(0x7f800000)" : "__int_as_float(0xff800000)";
  char b[64];
  snprintf(b, sizeof b, "%.9g", (double)v);
  std::string s(b);
  if (s.find_first_of(".e") == std::string::npos) s += ".0";
  return "(" + s + "f)";
}


std::string CodegenKey::str() const {
  std::ostringstream s;
  s << (plain ? "P" : "F") << (persistent ? "b" : "") << (pairs ? "x2" : "") << (even_rows ? "e" : "") << "|v" << vec
    << "|f" << frac_reg
    << "|r" << max_regs << "|w" << nw << "|c" << chunk << "|n" << nbuf << "|s";
  for (int x : stages) s << x << ",";
  s << "|i";
  for (int x : src_dtypes) s << x;
  s << "|o";
  for (int x : dst_dtypes) s << x;
  if (otptb) s << "|B" << tbx << "x" << tby;
  if (win_dtype != WT_F32) s << "|W" << win_dtype;
  if (down) s << "|D" << tby;
  if (chain) s << "|R";
  if (cascade) s << "|K" << tby;
  if (vol) s << "|Z" << vol_split << "x" << vol_to << "x" << tby;
  if (test_stall) s << "|STALL";
  if (fold) s << "|S";
  if (soft_cap) s << "|soft";
  if (shared_planes) s << "|SP";
  return s.str();
}


static int align_up(int v, int a) { return (v + a - 1) / a * a; }

// Steps of a warp tile beyond its output rows: the top halo (rows streamed
// before the first output row) plus the rows after the last output row that
// a node of the group still computes (its bottom halo and delay).
int stream_extra_steps(const GroupGeom &g) {
  int nsx = g.halo_b;
  for (const Node &n : g.nodes)
    if (!n.is_source) nsx = std::max(nsx, n.bot + n.delay);
  return g.halo_t + nsx;
}

FusedLayout fused_layout(const GroupGeom &g, const CodegenKey &key) {
  FusedLayout L;
  L.V = key.vec;
  const int V = L.V;
  L.lpad = V * ((g.halo_l + V - 1) / V);
  L.rpad = V * ((g.halo_r + V - 1) / V);
  L.out_w = 32 * V - L.lpad - L.rpad;
  if (L.out_w < V)
    fail(WT_EUNSUPPORTED, "group halo (" + std::to_string(g.halo_l) + "+" +
                              std::to_string(g.halo_r) + " px) too wide for a warp tile");
  // Chunks hold a multiple of the unroll factor U so that waits and issues
  // happen only at the start of an unrolled block (branch-free blocks).
  const int U = std::max(1, g.unroll);
  L.issue_blk = ((g.max_src_window - 1) + U - 1) / U * U;
  int ch = std::max({key.chunk, g.halo_t + 1, g.max_src_window, L.issue_blk + U});
  L.chunk = (ch + U - 1) / U * U;
  L.nbuf = std::max(2, key.nbuf);
  L.ring = L.chunk * L.nbuf;
  L.nsx = stream_extra_steps(g) - g.halo_t;
  L.src_rows_extra = g.halo_b;
  int off = 0;
  int n_src = 0;
  for (const Node &n : g.nodes)
    if (n.is_source) n_src++;
  L.chunk_bytes = 0;
  for (int s = 0; s < n_src; s++) {
    int dt = key.src_dtypes.at(s);
    int esz = elem_bytes(dt);
    int A = 16 / esz;
    int boxw = 32 * V + ((V % A) ? A : 0);
    if (boxw > 256) fail(WT_EUNSUPPORTED, "TMA box wider than 256 elements");
    // every TMA destination (each staging buffer) starts on a 128-byte
    // boundary: buffers are padded to a multiple of 128 bytes
    off = align_up(off, 128);
    L.boxw.push_back(boxw);
    L.esz.push_back(esz);
    L.ring_off.push_back(off);
    L.bufb.push_back(align_up(L.chunk * boxw * esz, 128));
    off += L.nbuf * L.bufb.back();
    L.chunk_bytes += L.chunk * boxw * esz;
  }
  L.win_off.assign(g.nodes.size(), -1);
  for (size_t i = 0; i < g.nodes.size(); i++) {
    const Node &n = g.nodes[i];
    if (n.is_source || !n.in_smem) continue;
    off = align_up(off, 16);
    L.win_off[i] = off;
    off += n.window * 32 * V * elem_bytes(key.win_dtype);
  }
  off = align_up(off, 8);
  L.bar_off = off;
  off += 8 * L.nbuf;
  L.warp_bytes = align_up(off, 128);
  return L;
}

namespace {

struct Ctx {
  const Pipeline &p;
  const GroupGeom &g;
  const CodegenKey &key;
  const FusedLayout &L;
  std::ostringstream o;
  int V, U, n_src;
  std::vector<int> ks;   // per node: first active step (constant)
  std::vector<int> kec;  // per node: last active step minus tile_h
  // gather-source values loaded for the stage being emitted:
  // (gather node, element, dx, dy) -> variable
  std::map<std::tuple<int, int, int, int>, std::string> gvar;
  // blocks choose their body by their rows (groups without gather sources):
  // STEADY or XEDGE where every row the block touches is inside the image
  bool rowsafe_blocks = false;
  // clamp-to-edge along x at the reads (every node's halo at most one
  // lane wide): edge tiles keep garbage in columns outside the image and
  // redirect each horizontal read that crosses the edge to the edge column
  bool edge_reads = false;
  Ctx(const Pipeline &p_, const GroupGeom &g_, const CodegenKey &k_, const FusedLayout &L_)
      : p(p_), g(g_), key(k_), L(L_) {}
};

// Step bodies of the fused kernel.  STEADY: no guards (every row the block
// touches is inside the image, the tile inside it along x).  XEDGE: rows
// inside the image, the tile crossing the left or right image edge: edge
// columns replicated (clamp-to-edge along x) and stores checked against W.
// GUARDED: rows may leave the image (top and bottom tiles, steps past the
// tile): per-node step ranges, row clamps and edge-row replication too.
enum { STEADY = 0, XEDGE = 1, GUARDED = 2 };

std::string reg(int ni, int slot, int j) {
  return "R" + std::to_string(ni) + "_" + std::to_string(slot) + "_" + std::to_string(j);
}
std::string tmp(int ni, int a, int j) {
  return "T" + std::to_string(ni) + "_" + std::to_string(a) + "_" + std::to_string(j);
}

int slot_of(const Node &n, int u, int a) {
  if (a < 0 || a >= n.window) fail(WT_EINVAL, "internal: window age out of range");
  if (n.rotate) return ((u - a) % n.window + n.window) % n.window;
  return n.window - 1 - a;
}

int width_of(const Node &n, int V) { return V + n.xl + n.xr; }

// x-fixup of the values `v` (clamp-to-edge along x inside border tiles):
// columns left of 0 take column 0's value, columns right of W - 1 take
// column W - 1's.  The tile's constants (xl0_: lanes left of column 0;
// xrl_, xre_: lane and element of column W - 1; fixr_: this lane's
// elements right of it) are computed once per tile; both branches are
// uniform across the warp and the replacements are selects.
void emit_xfix(Ctx &c, const std::vector<std::string> &v) {
  const int V = c.V;
  auto &o = c.o;
  o << "if (xl0_ > 0) { const float b0_ = __shfl_sync(WT_FULL, " << v[0] << ", xl0_);";
  for (int e = 0; e < V; e++) o << " " << v[e] << " = lane < xl0_ ? b0_ : " << v[e] << ";";
  o << " }\n";
  o << "if (xrl_ < 32) { float s_ = " << v[0] << ";";
  for (int e = 1; e < V; e++) o << " s_ = xre_ == " << e << " ? " << v[e] << " : s_;";
  o << " const float bl_ = __shfl_sync(WT_FULL, s_, xrl_);";
  for (int e = 0; e < V; e++) o << " " << v[e] << " = (fixr_ >> " << e << ") & 1 ? bl_ : " << v[e] << ";";
  o << " }\n";
}

// Neighbour columns by warp shuffles: type (3) loads of Sec. 5.  In edge
// tiles with reads redirected at the edge (edge = true): the lane holding
// column 0 takes its own column 0 for every column left of it, the lane
// holding column W - 1 its own column W - 1 (edge_v_) for every column
// right of it; other lanes' out-of-image columns are never read.
void emit_extend(Ctx &c, const Node &n, const std::vector<std::string> &v,
                 const std::function<std::string(int)> &tgt, bool edge = false) {
  const int V = c.V;
  for (int off = -n.xl; off < 0; off++) {
    int q = -((-off + V - 1) / V);
    int el = off - q * V;
    if (edge)  // every lane takes part in the shuffle, then selects
      c.o << "{ const float t_ = __shfl_up_sync(WT_FULL, " << v[el] << ", " << -q << "); " << tgt(n.xl + off)
          << " = fxl_ ? " << v[0] << " : t_; }\n";
    else
      c.o << tgt(n.xl + off) << " = __shfl_up_sync(WT_FULL, " << v[el] << ", " << -q << ");\n";
  }
  for (int off = V; off < V + n.xr; off++) {
    int q = off / V;
    int el = off - q * V;
    if (edge)
      c.o << "{ const float t_ = __shfl_down_sync(WT_FULL, " << v[el] << ", " << q << "); " << tgt(n.xl + off)
          << " = fxr_ ? edge_v_ : t_; }\n";
    else
      c.o << tgt(n.xl + off) << " = __shfl_down_sync(WT_FULL, " << v[el] << ", " << q << ");\n";
  }
  for (int e = 0; e < V; e++) c.o << tgt(n.xl + e) << " = " << v[e] << ";\n";
}

// Right image edge inside a lane: the elements of the lane holding column
// W - 1 past that column take its value (edge_v_, also the lane's right
// halo), so that reads across the edge see the edge column.  Opens a scope
// that the caller closes after emit_extend.
void emit_edge_open(Ctx &c, const Node &n, const std::vector<std::string> &v) {
  const int V = c.V;
  auto &o = c.o;
  // column W - 1 at a lane's last element (W a multiple of V): no element
  // of that lane lies past it, only its right halo does
  o << "{ float edge_v_ = " << v[V - 1] << ";\n";
  if (n.xr <= 0) return;
  o << "if (xrl_ < 32 && xre_ != " << V - 1 << ") {";
  for (int e = 0; e < V - 1; e++) o << " edge_v_ = xre_ == " << e << " ? " << v[e] << " : edge_v_;";
  for (int e = 0; e < V; e++) o << " " << v[e] << " = (fixr_ >> " << e << ") & 1 ? edge_v_ : " << v[e] << ";";
  o << " }\n";
}

void emit_load_vec(Ctx &c, int dtype, const std::string &addr, const std::vector<std::string> &v,
                   int esz) {
  for (int b = 0; b < c.V; b += 4)
    c.o << "wt_ld4_" << dtype_name(dtype) << "((const void *)(" << addr << " + " << b * esz << "), "
        << v[b] << ", " << v[b + 1] << ", " << v[b + 2] << ", " << v[b + 3] << ");\n";
}

std::vector<std::string> names(const std::string &base, int n) {
  std::vector<std::string> r;
  for (int i = 0; i < n; i++) r.push_back(base + std::to_string(i));
  return r;
}

// Shift register windows (non-rotating nodes) by one row.
void emit_shift(Ctx &c, int ni) {
  const Node &n = c.g.nodes[ni];
  if (n.in_smem || n.rotate || n.window < 2) return;
  int wd = width_of(n, c.V);
  for (int s = 0; s + 1 < n.window; s++)
    for (int j = 0; j < wd; j++) c.o << reg(ni, s, j) << " = " << reg(ni, s + 1, j) << ";\n";
}

// Address of the lane's pixels of ring row `ri` of source s.
std::string ring_row(int s, const std::string &ri) {
  std::string S = std::to_string(s);
  // chunk c of the current tile sits in buffer (cbase + c) % NB, where cbase
  // counts the chunks of the warp's earlier tiles.  Rows above the tile's
  // first row (ri down to -(window - 1), read only for rows that are never
  // stored) map into the ring too: ri + NB * CH selects the same buffer and
  // row for ri >= 0 and a stale row of the ring for negative ri, so every
  // address stays inside the warp's staging buffers.
  const std::string rr = "(" + ri + " + NB * CH)";
  return "lp" + S + " + ((cbase + " + rr + " / CH) % NB) * BUFB" + S + " + (" + rr + " % CH) * ROWB" + S;
}

// Row of a register-resident source, loaded from the TMA ring.
void emit_source_row(Ctx &c, int ni, int mode, int u) {
  const Node &n = c.g.nodes[ni];
  auto &o = c.o;
  const int V = c.V;
  int s = n.src_index;
  const bool rows = mode == GUARDED;
  emit_shift(c, ni);
  o << "{\n";
  if (rows) o << "if (k < nsrc) {\n";
  if (rows) o << "const int ri = wt_clampi(y_top + k, 0, H - 1) - y_top;\n";
  std::vector<std::string> v = names("e", V);
  o << "float";
  for (int e = 0; e < V; e++) o << (e ? ", " : " ") << v[e];
  o << ";\n";
  // unguarded steps read row kb + u of the chunk that block kb starts
  // (chunks are a multiple of U rows): the block's row pointer plus u rows
  const std::string S = std::to_string(s);
  emit_load_vec(c, c.key.src_dtypes[s], rows ? ring_row(s, "ri") : "rp" + S + " + " + std::to_string(u) + " * ROWB" + S,
                v, c.L.esz[s]);
  int sl = slot_of(n, u, 0);
  if (mode != STEADY && c.edge_reads) {
    emit_edge_open(c, n, v);
    emit_extend(c, n, v, [&](int j) { return reg(ni, sl, j); }, true);
    o << "}\n";
  } else {
    if (mode != STEADY) emit_xfix(c, v);
    emit_extend(c, n, v, [&](int j) { return reg(ni, sl, j); });
  }
  if (rows) o << "}\n";
  o << "}\n";
}

// Loads row (age a) of a shared-memory node into temporaries T<ni>_<a>_*.
void emit_load_tmp(Ctx &c, int ni, int a, int mode) {
  const Node &n = c.g.nodes[ni];
  auto &o = c.o;
  const int V = c.V;
  const bool rows = mode == GUARDED;
  o << "{\n";
  std::vector<std::string> v = names("q", V);
  o << "float";
  for (int e = 0; e < V; e++) o << (e ? ", " : " ") << v[e];
  o << ";\n";
  if (n.is_source) {
    int s = n.src_index;
    o << "int ri = k - " << a << ";\n";
    if (rows) o << "ri = wt_clampi(y_top + ri, 0, H - 1) - y_top;\n";
    emit_load_vec(c, c.key.src_dtypes[s], ring_row(s, "ri"), v, c.L.esz[s]);
    if (mode != STEADY && !c.edge_reads) emit_xfix(c, v);
  } else {
    o << "int kk = k - " << a << ";\n";
    if (rows)
      o << "{ const int rr = wt_clampi(y_top + kk - (" << n.delay << "), 0, H - 1); kk = rr - y_top + ("
        << n.delay << "); }\n";
    o << "const int sl = ((kk % " << n.window << ") + " << n.window << ") % " << n.window << ";\n";
    emit_load_vec(c, c.key.win_dtype, "sp" + std::to_string(ni) + " + sl * " +
                      std::to_string(32 * V * elem_bytes(c.key.win_dtype)), v, elem_bytes(c.key.win_dtype));
  }
  if (mode != STEADY && c.edge_reads) {
    emit_edge_open(c, n, v);
    emit_extend(c, n, v, [&](int j) { return tmp(ni, a, j); }, true);
    o << "}\n";
  } else {
    emit_extend(c, n, v, [&](int j) { return tmp(ni, a, j); });
  }
  o << "}\n";
}

// A tap of a gather source for element e of the consumer: a variable
// loaded by the stage's gather prologue.
std::string gather_tap(Ctx &c, int gi, int e, int dx, int dy) {
  auto it = c.gvar.find(std::make_tuple(gi, e, dx, dy));
  if (it == c.gvar.end()) fail(WT_EINVAL, "internal: gather tap without a load");
  return it->second;
}

// Gather prologue of a stage: every distinct pixel its taps of other levels
// read, loaded once, with one clamped row address per distinct row and one
// clamped column per distinct column.  The lane's first column X0 = xs +
// lane * V is even (xs and V are), so element e's source column is a
// constant offset from X0 / 2 (up-sampling: floor((X0 + e) / 2) + dx) or
// from 2 X0 (down-sampling: 2 (X0 + e) + dx); rows likewise from r.
// Column of a gather tap relative to the lane's base column: element e of
// the lane, tap offset dx.  Down by 2^s: base (xs + lane V) 2^s, offset
// e 2^s + dx.  Up by 2^s: base (xs + lane V) >> s, offset (e >> s) + dx,
// exact because xs + lane V is a multiple of V (a power of two): either
// 2^s divides it, or the lane's V columns lie in one 2^s-column cell.
int gather_off(int mode, int e, int dx) {
  const int s = tap_shift(mode);
  return tap_is_down(mode) ? (e << s) + dx : (e >> s) + dx;
}
// The lane's base column and a row's producer row, as expressions.
std::string gather_base(int mode, int V) {
  const int s = tap_shift(mode);
  const std::string b = "(xs + lane * " + std::to_string(V) + ")";
  return tap_is_down(mode) ? "(" + b + " * " + std::to_string(1 << s) + ")" : "(" + b + " >> " + std::to_string(s) + ")";
}
std::string gather_row(int mode, const std::string &r) {
  const int s = tap_shift(mode);
  return tap_is_down(mode) ? "(" + r + " * " + std::to_string(1 << s) + ")" : "(" + r + " >> " + std::to_string(s) + ")";
}
// Aligned pair loads need an even base column: every down mode, and up by 2.
bool gather_pairs(int mode) { return tap_is_down(mode) || tap_shift(mode) == 1; }

// Interior tiles: every gather row and column the guard-free body touches
// lies inside the gather source (the tile's border test includes these
// margins), so the loads need no clamps and read aligned pairs.
void emit_gather_prologue_fast(Ctx &c, int ni) {
  const Node &n = c.g.nodes[ni];
  auto &o = c.o;
  c.gvar.clear();
  struct Tap { int gi, dx, dy; };
  std::vector<Tap> taps;
  for (const KOp &op : n.prog)
    if (op.op == WT_OP_TAP && c.g.nodes[op.node].gather_mode) taps.push_back({op.node, op.dx, op.dy});
  if (taps.empty()) return;
  std::map<std::pair<int, int>, std::string> rows;
  std::map<std::tuple<int, int, int>, std::string> vals;  // (gi, dy, pair start) -> first of two names
  std::set<int> modes;
  int id = 0;
  for (const Tap &t : taps) modes.insert(c.g.nodes[t.gi].gather_mode);
  for (int m : modes) o << "const int gcb" << m << " = " << gather_base(m, c.V) << ";\n";
  for (const Tap &t : taps) {
    const Node &pn = c.g.nodes[t.gi];
    const int m = pn.gather_mode;
    const std::string S = "ia.src[" + std::to_string(pn.src_index) + "]";
    const int dt = c.key.src_dtypes.at(pn.src_index);
    const int esz = elem_bytes(dt);
    auto rk = std::make_pair(t.gi, t.dy);
    if (!rows.count(rk)) {
      std::string v = "gr" + std::to_string(id++);
      const std::string chan = pn.src_chan >= 0 ? std::to_string(pn.src_chan) : "ch";
      o << "const unsigned char *" << v << " = (const unsigned char *)" << S << ".ptr + (wt_i64)" << chan << " * "
        << S << ".plane + (wt_i64)(" << gather_row(m, "r") << " + (" << t.dy << ")) * " << S
        << ".pitch + (wt_i64)gcb" << m << " * " << esz << ";\n";
      rows[rk] = v;
    }
    for (int e = 0; e < c.V; e++) {
      const int off = gather_off(m, e, t.dx);
      if (!gather_pairs(m)) {
        // up by 4 or 8: one value per (row, offset), scalar loads
        auto vk = std::make_tuple(t.gi, t.dy, off);
        if (!vals.count(vk)) {
          std::string v = "gv" + std::to_string(id++);
          o << "const float " << v << " = wt_ld1_" << dtype_name(dt) << "(" << rows[rk] << " + (" << off * esz << "));\n";
          vals[vk] = v;
        }
        c.gvar[std::make_tuple(t.gi, e, t.dx, t.dy)] = vals[vk];
        continue;
      }
      const int p0 = off - (((off % 2) + 2) % 2);  // the aligned pair holding it
      auto vk = std::make_tuple(t.gi, t.dy, p0);
      if (!vals.count(vk)) {
        std::string v = "gv" + std::to_string(id++);
        o << "float " << v << "a, " << v << "b;\nwt_ld2_" << dtype_name(dt) << "(" << rows[rk] << " + (" << p0 * esz
          << "), " << v << "a, " << v << "b);\n";
        vals[vk] = v;
      }
      c.gvar[std::make_tuple(t.gi, e, t.dx, t.dy)] = vals[vk] + (off == p0 ? "a" : "b");
    }
  }
}

// Rolling windows of up-sampled gather rows (interior tiles, constant row
// parity per unrolled step): node `ni` at step k computes row r and reads
// gather rows (r >> 1) + dy, dy in [dymin, dymax]; the window holds those
// rows for the lane's columns, and advances by one row (one new row
// loaded) at every step where r is even, i.e. every second step, instead
// of loading every row at every step.
struct GWin {
  int gi = -1, dymin = 0, dymax = 0, omin = 0, omax = 0;
};
std::vector<GWin> gather_windows(const Ctx &c, int ni) {
  std::vector<GWin> r;
  if (!c.key.even_rows) return r;
  const Node &n = c.g.nodes[ni];
  std::map<int, GWin> m;
  for (const KOp &op : n.prog) {
    if (op.op != WT_OP_TAP || !c.g.nodes[op.node].gather_mode) continue;
    if (c.g.nodes[op.node].gather_mode != WT_TAP_UP2) return {};
    auto it = m.find(op.node);
    if (it == m.end()) {
      GWin w;
      w.gi = op.node;
      w.dymin = w.dymax = op.dy;
      w.omin = 1 << 20;
      w.omax = -(1 << 20);
      it = m.emplace(op.node, w).first;
    }
    GWin &w = it->second;
    w.dymin = std::min(w.dymin, op.dy);
    w.dymax = std::max(w.dymax, op.dy);
    for (int e = 0; e < c.V; e++) {
      w.omin = std::min(w.omin, gather_off(WT_TAP_UP2, e, op.dx));
      w.omax = std::max(w.omax, gather_off(WT_TAP_UP2, e, op.dx));
    }
  }
  for (auto &kv : m) r.push_back(kv.second);
  return r;
}

std::string gwin_name(int ni, const GWin &w, int row, int off) {
  return "GW" + std::to_string(ni) + "_" + std::to_string(w.gi) + "_" + std::to_string(row) + "_" +
         (off < 0 ? "m" + std::to_string(-off) : std::to_string(off));
}

// Loads gather row `rowexpr` of window w into window row `slot` (aligned
// pairs covering the window's columns; no clamps: interior tiles only).
void emit_gwin_load(Ctx &c, int ni, const GWin &w, int slot, const std::string &rowexpr) {
  auto &o = c.o;
  const Node &pn = c.g.nodes[w.gi];
  const std::string S = "ia.src[" + std::to_string(pn.src_index) + "]";
  const int dt = c.key.src_dtypes.at(pn.src_index);
  const int esz = elem_bytes(dt);
  const std::string chan = pn.src_chan >= 0 ? std::to_string(pn.src_chan) : "ch";
  o << "{ const unsigned char *gwr_ = (const unsigned char *)" << S << ".ptr + (wt_i64)" << chan << " * " << S
    << ".plane + (wt_i64)(" << rowexpr << ") * " << S << ".pitch + (wt_i64)((xs >> 1) + lane * " << c.V / 2
    << ") * " << esz << ";\n";
  const int plo = w.omin - (((w.omin % 2) + 2) % 2);
  for (int p0 = plo; p0 <= w.omax; p0 += 2) {
    const std::string a = (p0 >= w.omin && p0 <= w.omax) ? gwin_name(ni, w, slot, p0) : "gwx_";
    const std::string b = (p0 + 1 >= w.omin && p0 + 1 <= w.omax) ? gwin_name(ni, w, slot, p0 + 1) : "gwx_";
    o << "wt_ld2_" << dtype_name(dt) << "(gwr_ + (" << p0 * esz << "), " << a << ", " << b << ");\n";
  }
  o << "}\n";
}

// Row parity of node n at unrolled step u (tiles start on even rows).
int row_parity(const Ctx &c, const Node &n, int u) { return (((u - c.g.halo_t - n.delay) % 2) + 2) % 2; }

void emit_gwin_decl_init(Ctx &c) {
  auto &o = c.o;
  bool any = false;
  for (int ni : c.g.order) {
    const Node &n = c.g.nodes[ni];
    if (n.is_source) continue;
    for (const GWin &w : gather_windows(c, ni)) {
      const int nr = w.dymax - w.dymin + 1;
      o << "float";
      bool first = true;
      for (int j = 0; j < nr; j++)
        for (int off = w.omin; off <= w.omax; off++) {
          o << (first ? " " : ", ") << gwin_name(ni, w, j, off) << " = 0.f";
          first = false;
        }
      o << ";\n";
      any = true;
    }
  }
  if (!any) return;
  o << "float gwx_;\n(void)gwx_;\n";
  // the first step of an interior tile finds its rows in the window: rows
  // (r0 >> 1) + dy, one row earlier when step 0 itself advances (r0 even)
  o << "if (!border) {\n";
  for (int ni : c.g.order) {
    const Node &n = c.g.nodes[ni];
    if (n.is_source) continue;
    for (const GWin &w : gather_windows(c, ni)) {
      const int adv = row_parity(c, n, 0) == 0 ? 1 : 0;
      for (int j = 0; j < w.dymax - w.dymin + 1; j++)
        emit_gwin_load(c, ni, w, j, "((y_top - " + std::to_string(n.delay) + ") >> 1) - " + std::to_string(adv) +
                                        " + (" + std::to_string(w.dymin + j) + ")");
    }
  }
  o << "}\n";
}

// Interior step: advance the node's windows where its row is even, then
// name the taps' values.
bool emit_gwin_step(Ctx &c, int ni, int u) {
  const std::vector<GWin> ws = gather_windows(c, ni);
  if (ws.empty()) return false;
  auto &o = c.o;
  const Node &n = c.g.nodes[ni];
  c.gvar.clear();
  for (const GWin &w : ws) {
    const int nr = w.dymax - w.dymin + 1;
    if (row_parity(c, n, u) == 0) {
      for (int j = 0; j + 1 < nr; j++)
        for (int off = w.omin; off <= w.omax; off++)
          o << gwin_name(ni, w, j, off) << " = " << gwin_name(ni, w, j + 1, off) << ";\n";
      emit_gwin_load(c, ni, w, nr - 1, "(r >> 1) + (" + std::to_string(w.dymax) + ")");
    }
  }
  for (const KOp &op : n.prog) {
    if (op.op != WT_OP_TAP || !c.g.nodes[op.node].gather_mode) continue;
    for (const GWin &w : ws)
      if (w.gi == op.node)
        for (int e = 0; e < c.V; e++)
          c.gvar[std::make_tuple(op.node, e, op.dx, op.dy)] =
              gwin_name(ni, w, op.dy - w.dymin, gather_off(WT_TAP_UP2, e, op.dx));
  }
  return true;
}

void emit_gather_prologue(Ctx &c, int ni) {
  const Node &n = c.g.nodes[ni];
  auto &o = c.o;
  c.gvar.clear();
  struct Tap { int gi, dx, dy; };
  std::vector<Tap> taps;
  for (const KOp &op : n.prog)
    if (op.op == WT_OP_TAP && c.g.nodes[op.node].gather_mode) taps.push_back({op.node, op.dx, op.dy});
  if (taps.empty()) return;
  std::map<std::pair<int, int>, std::string> rows, cols;
  std::map<std::tuple<int, int, int>, std::string> vals;
  int id = 0;
  for (const Tap &t : taps) {
    const Node &pn = c.g.nodes[t.gi];
    const int m = pn.gather_mode;
    const std::string S = "ia.src[" + std::to_string(pn.src_index) + "]";
    const int esz = elem_bytes(c.key.src_dtypes.at(pn.src_index));
    auto rk = std::make_pair(t.gi, t.dy);
    if (!rows.count(rk)) {
      std::string v = "gr" + std::to_string(id++);
      const std::string chan = pn.src_chan >= 0 ? std::to_string(pn.src_chan) : "ch";
      o << "const unsigned char *" << v << " = (const unsigned char *)" << S << ".ptr + (wt_i64)" << chan << " * "
        << S << ".plane + (wt_i64)wt_clampi(" << gather_row(m, "r") << " + (" << t.dy << "), 0, " << S
        << ".H - 1) * " << S << ".pitch;\n";
      rows[rk] = v;
    }
    for (int e = 0; e < c.V; e++) {
      const int off = gather_off(m, e, t.dx);
      auto ck = std::make_pair(t.gi, off);
      if (!cols.count(ck)) {
        std::string v = "gc" + std::to_string(id++);
        o << "const int " << v << " = wt_clampi(" << gather_base(m, c.V) << " + (" << off << "), 0, " << S
          << ".W - 1) * " << esz << ";\n";
        cols[ck] = v;
      }
      auto vk = std::make_tuple(t.gi, t.dy, off);
      if (!vals.count(vk)) {
        std::string v = "gv" + std::to_string(id++);
        o << "const float " << v << " = wt_ld1_" << dtype_name(c.key.src_dtypes.at(pn.src_index)) << "(" << rows[rk]
          << " + " << cols[ck] << ");\n";
        vals[vk] = v;
      }
      c.gvar[std::make_tuple(t.gi, e, t.dx, t.dy)] = vals[vk];
    }
  }
}

// Postfix program of kernel node `ni` -> C++ expression for element e.
// Constants fold: operations on constants only are evaluated here in FP32
// (the result the device would compute), and x * 0, x * 1, x + 0 and x - 0
// simplify (exact for the finite values stages carry).  The column parity
// of element e is such a constant, so an up-sampling stage keeps only the
// taps of its own phase.
std::string emit_expr(Ctx &c, int ni_c, int e, int u) {
  const Node &cn = c.g.nodes[ni_c];
  struct Val {
    std::string s;
    bool k = false;
    float v = 0.f;
  };
  auto konst = [](float v) { Val x; x.s = float_literal(v); x.k = true; x.v = v; return x; };
  auto expr = [](const std::string &s) { Val x; x.s = s; return x; };
  std::vector<Val> st;
  for (const KOp &op : cn.prog) {
    switch (op.op) {
      case WT_OP_CONST: st.push_back(konst(op.value)); break;
      case WT_OP_XPAR: st.push_back(konst((float)(e & 1))); break;
      // a one-plane stage is plane 0 whichever tile channel computes it
      case WT_OP_CHAN: st.push_back(cn.channels == 1 ? konst(0.f) : expr("((float)ch)")); break;
      case WT_OP_YPAR:
        if (c.key.even_rows) {
          // r = y_top + kb + u - delay with y_top = y0 - halo_t, y0 and kb even
          const int par = (((u - c.g.halo_t - cn.delay) % 2) + 2) % 2;
          st.push_back(konst((float)par));
        } else {
          st.push_back(expr("((float)(r & 1))"));
        }
        break;
      case WT_OP_TAP: {
        const int pi = op.node;
        const Node &pn = c.g.nodes[pi];
        if (pn.gather_mode) {
          st.push_back(expr(gather_tap(c, pi, e, op.dx, op.dy)));
          break;
        }
        int a = cn.delay - pn.delay - op.dy;
        int j = pn.xl + e + op.dx;
        if (j < 0 || j >= width_of(pn, c.V)) fail(WT_EINVAL, "internal: tap column out of range");
        if (pn.in_smem) st.push_back(expr(tmp(pi, a, j)));
        else st.push_back(expr(reg(pi, slot_of(pn, u, a), j)));
      } break;
      case WT_OP_NEG:
        st.back() = st.back().k ? konst(-st.back().v) : expr("(-" + st.back().s + ")");
        break;
      case WT_OP_ABS:
        st.back() = st.back().k ? konst(std::fabs(st.back().v)) : expr("fabsf(" + st.back().s + ")");
        break;
      case WT_OP_SQRT:
        st.back() = st.back().k ? konst(std::sqrt(st.back().v)) : expr("sqrtf(" + st.back().s + ")");
        break;
      default: {
        Val b = st.back();
        st.pop_back();
        Val a = st.back();
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
        if (op.op == WT_OP_MUL && ((a.k && a.v == 0.f) || (b.k && b.v == 0.f))) {
          st.push_back(konst(0.f));
          break;
        }
        if (op.op == WT_OP_MUL && a.k && a.v == 1.f) { st.push_back(b); break; }
        if (op.op == WT_OP_MUL && b.k && b.v == 1.f) { st.push_back(a); break; }
        if (op.op == WT_OP_ADD && a.k && a.v == 0.f) { st.push_back(b); break; }
        if ((op.op == WT_OP_ADD || op.op == WT_OP_SUB) && b.k && b.v == 0.f) { st.push_back(a); break; }
        switch (op.op) {
          case WT_OP_ADD: st.push_back(expr("(" + a.s + " + " + b.s + ")")); break;
          case WT_OP_SUB: st.push_back(expr("(" + a.s + " - " + b.s + ")")); break;
          case WT_OP_MUL: st.push_back(expr("(" + a.s + " * " + b.s + ")")); break;
          case WT_OP_DIV: st.push_back(expr("(" + a.s + " / " + b.s + ")")); break;
          case WT_OP_MIN: st.push_back(expr("fminf(" + a.s + ", " + b.s + ")")); break;
          case WT_OP_MAX: st.push_back(expr("fmaxf(" + a.s + ", " + b.s + ")")); break;
          default: fail(WT_EINVAL, "internal: opcode");
        }
      }
    }
  }
  return st.back().s;
}

// --------------------------------------------------- packed pair code
// Expression tree of a node program for one element; leaves resolved to
// register names (taps), constants, or the row parity.
struct XN {
  int op = 0;
  std::string leaf;
  float c = 0;
  int a = -1, b = -1;
};

std::vector<XN> build_tree(Ctx &c, int ni, int e, int u) {
  const Node &cn = c.g.nodes[ni];
  std::vector<XN> t;
  std::vector<int> st;
  for (const KOp &op : cn.prog) {
    XN x;
    x.op = op.op;
    switch (op.op) {
      case WT_OP_CONST: x.c = op.value; break;
      case WT_OP_XPAR: x.op = WT_OP_CONST; x.c = (float)(e & 1); break;
      case WT_OP_YPAR: x.leaf = "((float)(r & 1))"; break;
      case WT_OP_CHAN:
        if (cn.channels == 1) {
          x.op = WT_OP_CONST;
          x.c = 0.f;
        } else {
          x.leaf = "((float)ch)";
        }
        break;
      case WT_OP_TAP: {
        const Node &pn = c.g.nodes[op.node];
        int a = cn.delay - pn.delay - op.dy;
        int j = pn.xl + e + op.dx;
        if (j < 0 || j >= width_of(pn, c.V)) fail(WT_EINVAL, "internal: tap column out of range");
        x.leaf = pn.in_smem ? tmp(op.node, a, j) : reg(op.node, slot_of(pn, u, a), j);
      } break;
      case WT_OP_NEG: case WT_OP_ABS: case WT_OP_SQRT:
        x.a = st.back();
        st.pop_back();
        break;
      default:
        x.b = st.back();
        st.pop_back();
        x.a = st.back();
        st.pop_back();
    }
    t.push_back(x);
    st.push_back((int)t.size() - 1);
  }
  return t;
}

struct PairEmit {
  std::ostringstream &o;
  const std::vector<XN> &A, &B;
  int &tmpid;
  std::string fresh() { return "p" + std::to_string(tmpid++); }
  std::string leaf(const XN &x) { return x.op == WT_OP_CONST ? float_literal(x.c) : x.leaf; }
  bool is_const(int i) { return A[i].op == WT_OP_CONST && B[i].op == WT_OP_CONST; }
  std::string def(const std::string &rhs) {
    std::string n = fresh();
    o << "const wt_u64 " << n << " = " << rhs << ";\n";
    return n;
  }
  std::string emit(int i) {
    const XN &x = A[i], &y = B[i];
    switch (x.op) {
      case WT_OP_CONST: case WT_OP_TAP: case WT_OP_YPAR: case WT_OP_CHAN:
        return def("wt_pk(" + leaf(x) + ", " + leaf(y) + ")");
      case WT_OP_ADD: {
        if (A[x.b].op == WT_OP_MUL) {
          std::string m0 = emit(A[x.b].a), m1 = emit(A[x.b].b), s0 = emit(x.a);
          return def("wt_fma2(" + m0 + ", " + m1 + ", " + s0 + ")");
        }
        if (A[x.a].op == WT_OP_MUL) {
          std::string m0 = emit(A[x.a].a), m1 = emit(A[x.a].b), s0 = emit(x.b);
          return def("wt_fma2(" + m0 + ", " + m1 + ", " + s0 + ")");
        }
        std::string l = emit(x.a), r = emit(x.b);
        return def("wt_add2(" + l + ", " + r + ")");
      }
      case WT_OP_SUB: {
        const XN &m = A[x.b];
        if (m.op == WT_OP_MUL && (is_const(m.a) || is_const(m.b))) {
          int ci = is_const(m.a) ? m.a : m.b, vi = is_const(m.a) ? m.b : m.a;
          std::string v = emit(vi), s0 = emit(x.a);
          std::string k = def("wt_pk(" + float_literal(-A[ci].c) + ", " + float_literal(-B[ci].c) + ")");
          return def("wt_fma2(" + v + ", " + k + ", " + s0 + ")");
        }
        std::string l = emit(x.a), r = emit(x.b);
        return def("wt_sub2(" + l + ", " + r + ")");
      }
      case WT_OP_MUL: {
        std::string l = emit(x.a), r = emit(x.b);
        return def("wt_mul2(" + l + ", " + r + ")");
      }
      default: {  // no packed form: unpack, scalar op, repack
        std::string l = emit(x.a);
        std::string r = x.b >= 0 ? emit(x.b) : "";
        std::string n = fresh();
        o << "float " << n << "a, " << n << "b, " << n << "c, " << n << "d;\n";
        o << "wt_upk(" << l << ", " << n << "a, " << n << "b);\n";
        if (x.b >= 0) o << "wt_upk(" << r << ", " << n << "c, " << n << "d);\n";
        auto f = [&](const std::string &p, const std::string &q) -> std::string {
          switch (x.op) {
            case WT_OP_DIV: return "(" + p + " / " + q + ")";
            case WT_OP_MIN: return "fminf(" + p + ", " + q + ")";
            case WT_OP_MAX: return "fmaxf(" + p + ", " + q + ")";
            case WT_OP_NEG: return "(-" + p + ")";
            case WT_OP_ABS: return "fabsf(" + p + ")";
            case WT_OP_SQRT: return "sqrtf(" + p + ")";
          }
          fail(WT_EINVAL, "internal: opcode");
        };
        return def("wt_pk(" + f(n + "a", n + "c") + ", " + f(n + "b", n + "d") + ")");
      }
    }
  }
};

// Elements e and e+1 of node `ni` with packed f32x2 arithmetic.
void emit_pair(Ctx &c, int ni, int e, int u, const std::vector<std::string> &v, int &tmpid) {
  std::vector<XN> A = build_tree(c, ni, e, u), B = build_tree(c, ni, e + 1, u);
  PairEmit pe{c.o, A, B, tmpid};
  std::string r = pe.emit((int)A.size() - 1);
  c.o << "wt_upk(" << r << ", " << v[e] << ", " << v[e + 1] << ");\n";
}

// (producer node, age) pairs a node reads from shared-memory windows.
std::vector<std::pair<int, int>> smem_reads(Ctx &c, int ni_c) {
  std::vector<std::pair<int, int>> r;
  for (const KOp &op : c.g.nodes[ni_c].prog) {
    if (op.op != WT_OP_TAP) continue;
    const int pi = op.node;
    if (!c.g.nodes[pi].in_smem) continue;
    std::pair<int, int> pr{pi, c.g.nodes[ni_c].delay - c.g.nodes[pi].delay - op.dy};
    if (std::find(r.begin(), r.end(), pr) == r.end()) r.push_back(pr);
  }
  return r;
}

void emit_store(Ctx &c, int ni, int mode, int u, const std::vector<std::string> &v) {
  const Node &n = c.g.nodes[ni];
  auto &o = c.o;
  const int V = c.V;
  int dt = c.key.dst_dtypes.at(n.dst_index);
  int esz = elem_bytes(dt);
  const std::string D = std::to_string(n.dst_index);
  const std::string one_ch = n.channels == 1 && c.g.channels > 1 ? " && ch == 0" : "";
  o << "{\n";
  if (c.rowsafe_blocks && mode != GUARDED) {
    // rows inside the image: the row test is r - y0 = k - halo_t - delay in
    // [0, T), one unsigned compare; the row address is the block's row
    // pointer plus u rows
    o << "if ((unsigned)(kb + (" << u - c.g.halo_t - n.delay << ")) < (unsigned)T" << one_ch << ") {\n";
    o << "unsigned char *op_ = obk" << D << " + " << u << " * opitch" << D << ";\n";
    if (mode == STEADY) {
      o << "if (st_lane) {\n";
      for (int b = 0; b < V; b += 4)
        o << "wt_st4_" << dtype_name(dt) << "(op_ + " << b * esz << ", " << v[b] << ", " << v[b + 1] << ", "
          << v[b + 2] << ", " << v[b + 3] << ");\n";
      o << "} } }\n";
      return;
    }
    o << "const int x = xs + lane * " << V << ";\n";
    o << "if (st_lane) {\n";
    o << "if (x + " << V << " <= W) {\n";
    for (int b = 0; b < V; b += 4)
      o << "wt_st4_" << dtype_name(dt) << "(op_ + " << b * esz << ", " << v[b] << ", " << v[b + 1] << ", " << v[b + 2]
        << ", " << v[b + 3] << ");\n";
    o << "} else {\n";
    for (int e = 0; e < V; e++)
      o << "if (x + " << e << " < W) wt_st1_" << dtype_name(dt) << "(op_ + " << e * esz << ", " << v[e] << ");\n";
    o << "} } } }\n";
    return;
  }
  if (mode != GUARDED) {
    // per-tile row base and lane predicate: the conditional part is the
    // store alone
    o << "if (r >= y0 && r < y0 + T" << one_ch << ") {\n";
    o << "unsigned char *op_ = ob" << D << " + (wt_i64)r * ia.dst[" << D << "].pitch;\n";
    o << "if (st_lane) {\n";
    for (int b = 0; b < V; b += 4)
      o << "wt_st4_" << dtype_name(dt) << "(op_ + " << b * esz << ", " << v[b] << ", " << v[b + 1] << ", " << v[b + 2]
        << ", " << v[b + 3] << ");\n";
    o << "} } }\n";
    return;
  }
  o << "if (r >= y0 && r < y0 + T && r < H)\n";
  if (n.channels == 1 && c.g.channels > 1) o << "if (ch == 0)\n";
  o << "{ const int x = xs + lane * " << V << ";\n";
  o << "if (lane >= " << c.L.lpad / V << " && lane < " << 32 - c.L.rpad / V << ") {\n";
  std::string d = "ia.dst[" + D + "]";
  o << "unsigned char *op_ = (unsigned char *)" << d << ".ptr + (wt_i64)"
    << (n.channels > 1 ? "ch" : "0") << " * " << d << ".plane + (wt_i64)r * " << d
    << ".pitch + (wt_i64)x * " << esz << ";\n";
  o << "if (x + " << V << " <= W) {\n";
  for (int b = 0; b < V; b += 4)
    o << "wt_st4_" << dtype_name(dt) << "(op_ + " << b * esz << ", " << v[b] << ", " << v[b + 1] << ", "
      << v[b + 2] << ", " << v[b + 3] << ");\n";
  o << "} else {\n";
  for (int e = 0; e < V; e++)
    o << "if (x + " << e << " < W) wt_st1_" << dtype_name(dt) << "(op_ + " << e * esz << ", " << v[e]
      << ");\n";
  o << "}\n";
  o << "} } }\n";
}

// A node that sums n >= 3 horizontally consecutive values of one producer
// row with unit weights (a box filter's row pass): adjacent outputs share
// all but one term, so each pair of elements costs n + 1 additions
// instead of 2 (n - 1).  Returns false for other programs.
bool emit_box_row(Ctx &c, int ni, int u, const std::vector<std::string> &v) {
  const Node &n = c.g.nodes[ni];
  if (c.V % 2) return false;
  int prod = -1, a = 1 << 20, b = -(1 << 20), taps = 0, adds = 0;
  for (const KOp &op : n.prog) {
    if (op.op == WT_OP_TAP) {
      if (op.dy != 0 || (prod >= 0 && op.node != prod)) return false;
      prod = op.node;
      a = std::min(a, op.dx);
      b = std::max(b, op.dx);
      taps++;
    } else if (op.op == WT_OP_ADD) {
      adds++;
    } else {
      return false;
    }
  }
  if (prod < 0 || taps < 3 || adds != taps - 1 || b - a + 1 != taps) return false;
  const Node &pn = c.g.nodes[prod];
  if (pn.gather_mode) return false;
  std::set<int> seen;
  for (const KOp &op : n.prog)
    if (op.op == WT_OP_TAP && !seen.insert(op.dx).second) return false;  // repeated tap: weight 2
  const int age = n.delay - pn.delay;
  auto val = [&](int j) {
    if (j < 0 || j >= width_of(pn, c.V)) fail(WT_EINVAL, "internal: tap column out of range");
    return pn.in_smem ? tmp(prod, age, j) : reg(prod, slot_of(pn, u, age), j);
  };
  for (int e = 0; e < c.V; e += 2) {
    // shared terms of elements e and e + 1: columns e + a + 1 .. e + b
    std::string sh = val(pn.xl + e + a + 1);
    for (int d = a + 2; d <= b; d++) sh = "(" + sh + " + " + val(pn.xl + e + d) + ")";
    c.o << "{ const float sh_ = " << sh << ";\n";
    c.o << v[e] << " = " << val(pn.xl + e + a) << " + sh_;\n";
    c.o << v[e + 1] << " = sh_ + " << val(pn.xl + e + 1 + b) << ";\n}\n";
  }
  return true;
}

void emit_stage(Ctx &c, int ni, int mode, int u, std::set<std::pair<int, int>> &loaded) {
  const bool safe = mode == GUARDED;
  const Node &n = c.g.nodes[ni];
  auto &o = c.o;
  const int V = c.V;
  emit_shift(c, ni);
  if (safe)
    o << "if (k >= " << c.ks[ni] << " && k <= T + (" << c.kec[ni] << ")) {\n";
  o << "{\n";
  o << "const int r = y_top + k - (" << n.delay << ");\n";
  o << "(void)r;\n";
  for (auto &pr : smem_reads(c, ni)) {
    if (!safe && loaded.count(pr)) continue;
    emit_load_tmp(c, pr.first, pr.second, mode);
    if (!safe) loaded.insert(pr);
  }
  std::vector<std::string> v = names("v", V);
  o << "float";
  for (int e = 0; e < V; e++) o << (e ? ", " : " ") << v[e];
  o << ";\n";
  if (safe) {
    o << "if (r > H - 1) {\n";
    if (n.in_smem) {
      o << "const int sl = (((k - 1) % " << n.window << ") + " << n.window << ") % " << n.window << ";\n";
      emit_load_vec(c, c.key.win_dtype, "sp" + std::to_string(ni) + " + sl * " +
                        std::to_string(32 * V * elem_bytes(c.key.win_dtype)), v, elem_bytes(c.key.win_dtype));
    } else {
      int prev = n.rotate ? slot_of(n, u, n.window > 1 ? 1 : 0) : n.window - 1;
      for (int e = 0; e < V; e++) o << v[e] << " = " << reg(ni, prev, n.xl + e) << ";\n";
    }
    o << "} else {\n";
  }
  if (safe) emit_gather_prologue(c, ni);
  else if (!emit_gwin_step(c, ni, u)) emit_gather_prologue_fast(c, ni);
  if (mode == XEDGE && !c.gvar.empty()) fail(WT_EINVAL, "internal: x-edge body with gather sources");
  // packed pairs for nodes whose taps all read the producer's own element
  // pairs (dx = 0): a pair shifted by one column would have to be gathered
  // into an aligned register pair first
  bool pairs = c.key.pairs;
  for (const KOp &op : n.prog)
    if (op.op == WT_OP_TAP && (op.dx != 0 || c.g.nodes[op.node].gather_mode)) pairs = false;
  if (pairs) {
    int tmpid = 0;
    o << "{\n";
    for (int e = 0; e < V; e += 2) emit_pair(c, ni, e, u, v, tmpid);
    o << "}\n";
  } else if (!emit_box_row(c, ni, u, v)) {
    for (int e = 0; e < V; e++) o << v[e] << " = " << emit_expr(c, ni, e, u) << ";\n";
  }
  if (safe) o << "}\n";
  if (mode != STEADY) {
    // Columns outside the image must hold the edge column's value.  A node
    // computed from edge-replicated producers by taps without an x offset
    // (pointwise or vertical) and without the column parity is replicated
    // already; only the others are fixed up.
    bool xdep = false;
    for (const KOp &op : n.prog)
      if ((op.op == WT_OP_TAP && (op.dx != 0 || c.g.nodes[op.node].gather_mode)) || op.op == WT_OP_XPAR)
        xdep = true;
    if (xdep && !c.edge_reads) emit_xfix(c, v);
  }
  if (n.in_smem) {
    o << "{ const int sl = ((k % " << n.window << ") + " << n.window << ") % " << n.window << ";\n";
    const int we = elem_bytes(c.key.win_dtype);
    for (int b = 0; b < V; b += 4)
      o << "wt_st4_" << dtype_name(c.key.win_dtype) << "(sp" << ni << " + sl * " << 32 * V * we << " + " << b * we
        << ", " << v[b] << ", " << v[b + 1] << ", " << v[b + 2] << ", " << v[b + 3] << ");\n";
    o << "}\n";
  } else {
    int sl = slot_of(n, u, 0);
    if (mode != STEADY && c.edge_reads) {
      emit_edge_open(c, n, v);
      emit_extend(c, n, v, [&](int j) { return reg(ni, sl, j); }, true);
      o << "}\n";
    } else {
      emit_extend(c, n, v, [&](int j) { return reg(ni, sl, j); });
    }
    if (safe && n.window > 1) {
      o << "if (r == 0) {\n";
      int wd = width_of(n, V);
      for (int a = 1; a < n.window; a++) {
        int s2 = slot_of(n, u, a);
        for (int j = 0; j < wd; j++) o << reg(ni, s2, j) << " = " << reg(ni, sl, j) << ";\n";
      }
      o << "}\n";
    }
  }
  if (n.is_liveout) emit_store(c, ni, mode, u, v);
  o << "}\n";
  if (safe) o << "}\n";
}

void emit_step(Ctx &c, int mode, int u) {
  auto &o = c.o;
  static const char *names_[3] = {" (steady)", " (x edge)", " (guarded)"};
  o << "{ // step phase " << u << names_[mode] << "\n";
  o << "const int k = kb + " << u << ";\n";
  if (mode == GUARDED) o << "if (k >= nsteps) goto wt_tile_end;\n";
  // temporaries for shared-memory windows used this step
  std::set<std::pair<int, int>> all;
  for (int ni : c.g.order) {
    if (c.g.nodes[ni].is_source) continue;
    for (auto &pr : smem_reads(c, ni)) all.insert(pr);
  }
  for (auto &pr : all) {
    const Node &pn = c.g.nodes[pr.first];
    o << "float";
    for (int j = 0; j < width_of(pn, c.V); j++) o << (j ? ", " : " ") << tmp(pr.first, pr.second, j);
    o << ";\n";
  }
  std::set<std::pair<int, int>> loaded;
  for (int ni : c.g.order) {
    const Node &n = c.g.nodes[ni];
    if (n.is_source) {
      if (!n.in_smem) emit_source_row(c, ni, mode, u);
      continue;
    }
    emit_stage(c, ni, mode, u, loaded);
  }
  o << "}\n";
}

// ------------------------------------------- deferred constant scales
// A node's registers may hold its value divided by a compile-time constant,
// the node's scale: a stage that multiplies by constants (a normalised
// filter, a weight) leaves the factor to its consumers, which merge it into
// their own constants or products.  A normalised 3-tap column pass then
// costs two additions instead of a multiply and two fused multiply-adds,
// and a box mean feeding a product costs no multiply at all.  Every
// program is rewritten, in evaluation order, into one computing the raw
// value from its producers' raw values; values leaving the kernel (HBM
// stores, 16-bit shared-memory windows) are brought back to scale 1.  The
// results differ from the program as written by rounding only.
struct SV {
  std::vector<KOp> ops;  // postfix program of the raw value
  double s = 1.0;        // value = s * raw
  bool k = false;        // a constant (one CONST op, s = 1)
  float v = 0.f;
};

SV sv_const(float v) {
  SV x;
  x.k = true;
  x.v = v;
  KOp o;
  o.op = WT_OP_CONST;
  o.value = v;
  x.ops = {o};
  return x;
}

SV sv_op(SV a, const SV *b, int op, double s) {
  if (b) a.ops.insert(a.ops.end(), b->ops.begin(), b->ops.end());
  KOp o;
  o.op = op;
  a.ops.push_back(o);
  a.s = s;
  a.k = false;
  return a;
}

// raw * m, the scale unchanged (m applied to the raw program)
SV sv_mul_const(const SV &a, double m) {
  if (m == 1.0) return a;
  if (m == -1.0) return sv_op(a, nullptr, WT_OP_NEG, a.s);
  SV c = sv_const((float)m);
  return sv_op(a, &c, WT_OP_MUL, a.s);
}

// the value itself (scale 1)
SV sv_mat(const SV &a) {
  if (a.k || a.s == 1.0) return a;
  SV r = sv_mul_const(a, a.s);
  r.s = 1.0;
  return r;
}

bool sv_scale_ok(double s) {
  const double m = std::fabs(s);
  return std::isfinite(s) && m >= std::ldexp(1.0, -40) && m <= std::ldexp(1.0, 40);
}

float fold_const(int op, float a, float b) {
  switch (op) {
    case WT_OP_ADD: return a + b;
    case WT_OP_SUB: return a - b;
    case WT_OP_MUL: return a * b;
    case WT_OP_DIV: return a / b;
    case WT_OP_MIN: return std::fmin(a, b);
    case WT_OP_MAX: return std::fmax(a, b);
  }
  fail(WT_EINVAL, "internal: opcode");
}

SV sv_binary(int op, SV a, SV b) {
  if (a.k && b.k) return sv_const(fold_const(op, a.v, b.v));
  switch (op) {
    case WT_OP_MUL:
      if (a.k && std::isfinite(a.v) && a.v != 0.f) { b.s *= a.v; return b; }
      if (b.k && std::isfinite(b.v) && b.v != 0.f) { a.s *= b.v; return a; }
      if (a.k || b.k) break;
      return sv_op(a, &b, WT_OP_MUL, a.s * b.s);
    case WT_OP_DIV:
      if (b.k && std::isfinite(b.v) && b.v != 0.f) { a.s /= b.v; return a; }
      if (b.k) break;
      return sv_op(a, &b, WT_OP_DIV, a.s / b.s);
    case WT_OP_ADD: case WT_OP_SUB: {
      const int flip = op == WT_OP_ADD ? WT_OP_SUB : WT_OP_ADD;
      if (a.k) return sv_op(sv_const((float)(a.v / b.s)), &b, op, b.s);
      if (b.k) {
        SV c = sv_const((float)(b.v / a.s));
        return sv_op(a, &c, op, a.s);
      }
      if (a.s == b.s) return sv_op(a, &b, op, a.s);
      // a difference keeps a's scale (a - m b' is one fused multiply-add,
      // packed too; m a' - b' is not); a sum the smaller one (m >= 1)
      if (op == WT_OP_SUB || std::fabs(a.s) <= std::fabs(b.s)) {
        // a's scale: value = s_a (a' +- (s_b / s_a) b')
        const double m = b.s / a.s;
        if (m == -1.0) return sv_op(a, &b, flip, a.s);
        SV mb = sv_mul_const(b, m);
        return sv_op(a, &mb, op, a.s);
      }
      // b's scale: value = s_b ((s_a / s_b) a' +- b')
      const double m = a.s / b.s;
      if (m == -1.0) {
        // -b' +- b'' : b' - a' for ADD, -(a' + b') for SUB
        if (op == WT_OP_ADD) return sv_op(b, &a, WT_OP_SUB, b.s);
        return sv_op(a, &b, WT_OP_ADD, -b.s);
      }
      SV ma = sv_mul_const(a, m);
      return sv_op(ma, &b, op, b.s);
    }
    case WT_OP_MIN: case WT_OP_MAX: {
      const int other = op == WT_OP_MIN ? WT_OP_MAX : WT_OP_MIN;
      if (a.k || b.k) {
        SV &x = a.k ? b : a;
        const float kv = a.k ? a.v : b.v;
        SV c = sv_const((float)(kv / x.s));
        return sv_op(x, &c, x.s > 0 ? op : other, x.s);
      }
      if (a.s == b.s) return sv_op(a, &b, a.s > 0 ? op : other, a.s);
      break;
    }
  }
  // no scale passes through: both operands at scale 1
  SV ma = sv_mat(a), mb = sv_mat(b);
  return sv_op(ma, &mb, op, 1.0);
}

SV sv_unary(int op, SV a) {
  if (a.k) {
    switch (op) {
      case WT_OP_NEG: return sv_const(-a.v);
      case WT_OP_ABS: return sv_const(std::fabs(a.v));
      case WT_OP_SQRT: return sv_const(std::sqrt(a.v));
    }
  }
  switch (op) {
    case WT_OP_NEG: a.s = -a.s; return a;
    case WT_OP_ABS: return sv_op(a, nullptr, WT_OP_ABS, std::fabs(a.s));
    case WT_OP_SQRT:
      if (a.s > 0) return sv_op(a, nullptr, WT_OP_SQRT, std::sqrt(a.s));
      return sv_op(sv_mat(a), nullptr, WT_OP_SQRT, 1.0);
  }
  fail(WT_EINVAL, "internal: opcode");
}

// Rewrites the programs of g's computed nodes (evaluation order) so that
// each computes its raw value; a node whose value is stored keeps scale 1.
void fold_scales(GroupGeom &g, const CodegenKey &key) {
  std::vector<double> scale(g.nodes.size(), 1.0);
  for (int ni : g.order) {
    Node &n = g.nodes[ni];
    if (n.is_source || n.gather_mode) continue;
    std::vector<SV> st;
    for (const KOp &op : n.prog) {
      switch (op.op) {
        case WT_OP_CONST: st.push_back(sv_const(op.value)); break;
        case WT_OP_TAP: {
          SV x;
          x.ops = {op};
          x.s = scale[op.node];
          st.push_back(x);
        } break;
        case WT_OP_XPAR: case WT_OP_YPAR: case WT_OP_CHAN: {
          SV x;
          x.ops = {op};
          st.push_back(x);
        } break;
        case WT_OP_NEG: case WT_OP_ABS: case WT_OP_SQRT:
          st.back() = sv_unary(op.op, st.back());
          break;
        default: {
          SV b = st.back();
          st.pop_back();
          SV a = st.back();
          st.pop_back();
          st.push_back(sv_binary(op.op, a, b));
        }
      }
      if (!sv_scale_ok(st.back().s)) st.back() = sv_mat(st.back());
    }
    SV r = st.back();
    const bool keep = n.is_liveout || (n.in_smem && key.win_dtype != WT_F32);
    if (keep || r.k) r = sv_mat(r);
    n.prog = r.ops;
    scale[ni] = r.s;
  }
}

}  // namespace

std::string emit_fused(const Pipeline &p, const GroupGeom &g0, const CodegenKey &key,
                       const std::string &kname) {
  GroupGeom g = g0;
  if (key.fold) fold_scales(g, key);
  FusedLayout L = fused_layout(g, key);
  Ctx c(p, g, key, L);
  c.V = key.vec;
  c.U = g.unroll;
  int n_src = 0, n_dst = 0;
  for (size_t i = 0; i < g.nodes.size(); i++) {
    Node &n = g.nodes[i];
    if (n.is_source) n.src_index = n_src++;
    else if (n.is_liveout) n.dst_index = n_dst++;
  }
  c.n_src = n_src;
  // gather sources follow the staged ones in the source table
  int n_gather = 0;
  for (Node &n : g.nodes)
    if (n.gather_mode) n.src_index = n_src + n_gather++;
  const int V = c.V, HT = g.halo_t, HB = g.halo_b;
  c.ks.assign(g.nodes.size(), 0);
  c.kec.assign(g.nodes.size(), 0);
  int kss = 0, kse_c = 1 << 30;
  for (size_t i = 0; i < g.nodes.size(); i++) {
    const Node &n = g.nodes[i];
    if (n.is_source) {
      c.ks[i] = 0;
      c.kec[i] = HT + HB - 1;
    } else {
      c.ks[i] = HT - n.top + n.delay;
      c.kec[i] = HT - 1 + n.bot + n.delay;
    }
    kss = std::max(kss, c.ks[i]);
    kse_c = std::min(kse_c, c.kec[i]);
  }
  auto &o = c.o;
  // test-only stall: bounded waits give up after a few polls
  if (key.test_stall) o << "#define WT_WAIT_LIMIT 256\n";
  o << kDeviceSource;
  o << "static_assert(sizeof(WtArgs) == " << sizeof(KernelArgs) << ", \"WtArgs layout\");\n";
  o << "#define CH " << L.chunk << "\n#define NB " << L.nbuf
    << "\n#define RING " << L.ring << "\n#define ISSUE " << L.issue_blk << "\n";
  for (int s = 0; s < n_src; s++)
    o << "#define ROWB" << s << " " << L.boxw[s] * L.esz[s] << "\n#define BUFB" << s << " " << L.bufb[s] << "\n";
  // register cap through the launch bounds (they take precedence over
  // -maxrregcount): enough resident blocks that each thread gets <= max_regs
  int min_blocks = 1;
  if (key.max_regs > 0) min_blocks = std::max(1, 65536 / (key.max_regs * 32 * key.nw));
  if (!key.persistent) {
    // Tile order of the queue: tall tiles, then the band of short ones;
    // within each, the tiles of the two edge columns first (their x-edge
    // reads make them the slowest, and a slow tile handed out last would
    // end the launch alone), then the others row by row, the last row (the
    // image's bottom, guarded at its end) first.
    o << "static __device__ __forceinline__ void wt_tile_order(int t, int tiles_x, int nrows, int &tx, int &tr) {\n"
         "if (tiles_x < 3) { tx = t % tiles_x; tr = t / tiles_x; return; }\n"
         "const int ne_ = 2 * nrows;\n"
         "if (t < ne_) { tr = t >> 1; tx = (t & 1) ? tiles_x - 1 : 0; }\n"
         "else { const int j_ = t - ne_; const int r_ = j_ / (tiles_x - 2); tx = 1 + j_ % (tiles_x - 2);"
         " tr = r_ == 0 ? nrows - 1 : r_ - 1; }\n}\n";
    o << "static __device__ __forceinline__ void wt_tile_coords(const WtArgs &a, int tile, int &tx, int &ch, int &y0,"
         " int &T) {\n"
         "int tr_;\n"
         "if (tile < a.n_big) { wt_tile_order(tile, a.tiles_x, a.n_big / a.tiles_x, tx, tr_);"
         " y0 = a.ty2 * a.tile_h2 + (tr_ % a.ty1) * a.tile_h; ch = tr_ / a.ty1; T = a.tile_h; }\n"
         "else { wt_tile_order(tile - a.n_big, a.tiles_x, (a.n_tiles - a.n_big) / a.tiles_x, tx, tr_);"
         " y0 = (tr_ % a.ty2) * a.tile_h2; ch = tr_ / a.ty2; T = a.tile_h2; }\n}\n";
  }
  o << "extern \"C\" __global__ void __launch_bounds__(" << 32 * key.nw << ", " << min_blocks << ") " << kname
    << "(const __grid_constant__ WtArgs a) {\n";
  o << "extern __shared__ __align__(128) unsigned char wt_smem[];\n";
  o << "const int lane = threadIdx.x & 31;\nconst int warp = threadIdx.x >> 5;\n";
  o << "unsigned char *wb = wt_smem + warp * " << L.warp_bytes << ";\n";
  o << "const wt_u32 bar = wt_smem_u32(wb + " << L.bar_off << ");\n";
  o << "if (lane == 0) { for (int i = 0; i < NB; i++) wt_mbar_init(bar + 8u * i, 1u); wt_fence_mbar_init(); }\n";
  o << "__syncwarp();\n";
  o << "int cbase = 0;\n(void)cbase;\nint failc = 0, issued = 0;\n";
  // register windows (explicit scalars, D4)
  for (size_t i = 0; i < g.nodes.size(); i++) {
    const Node &n = g.nodes[i];
    if (n.in_smem || n.gather_mode) continue;
    o << "float";
    bool first = true;
    for (int s = 0; s < n.window; s++)
      for (int j = 0; j < width_of(n, V); j++) {
        o << (first ? " " : ", ") << reg((int)i, s, j) << " = 0.f";
        first = false;
      }
    o << ";\n";
  }
  // Persistent warps pull tiles from a device queue (a.queue[0]); the last
  // warp to leave resets the queue for the next launch (a.queue[1] counts
  // the warps that left), so no per-launch clearing is needed.
  // A warp takes its next tile only when it is free (taking it earlier
  // reserves tail tiles for busy warps while others idle).
  if (key.persistent) o << "int last_img_ = -1;\n";
  // Tiles by block index (a.direct: one tile per warp, the hardware block
  // scheduler hands out blocks in index order), or pulled by persistent
  // warps from a device queue (a.queue[0]) until it is empty.
  o << "int first_ = 1;\n";
  o << "for (;;) {\n";
  o << "int tile = 0;\n"
       "if (a.direct) { tile = first_ ? (int)blockIdx.x * " << key.nw << " + warp : a.n_tiles; first_ = 0; }\n"
       "else { if (lane == 0) tile = atomicAdd(a.queue, 1); tile = __shfl_sync(WT_FULL, tile, 0); }\n"
       "if (tile >= a.n_tiles) break;\n";
  if (key.persistent) {
    o << "const int *tt_ = a.tile_table + 4 * tile;\nconst int img = tt_[0];\n";
    o << "const WtArgs &ia = ((const WtArgs *)a.img_tab)[img];\n";
    o << "const int tx = tt_[1], ty = tt_[2], ch = tt_[3];\n";
  } else {
    // tall tiles first (ty1 tile rows of tile_h rows below a band of ty2
    // short rows), then the short tiles of tile_h2 rows: the last tiles
    // handed out are short, and the slow bottom-border row is handed out
    // before them, not in the final round
    o << "const WtArgs &ia = a;\n";
    o << "int tx, ch, y0, T;\n";
    o << "wt_tile_coords(a, tile, tx, ch, y0, T);\n";
    // the last tile row is clipped by the image: no steps past its end
    o << "T = min(T, a.H - y0);\n";
  }
  if (key.persistent) {
    o << "const int y0 = ty * ia.tile_h;\nconst int T = min(ia.tile_h, ia.H - y0);\n";
    // the image's tensor maps, acquired when the warp moves to a new image
    // (tiles are listed image by image)
    o << "if (img != last_img_) {\nlast_img_ = img;\nif (lane == 0) {";
    for (int s = 0; s < n_src; s++) o << " wt_tmap_acquire(&ia.tmap[" << s << "]);";
    o << " }\n}\n";
  }
  o << "const int W = ia.W, H = ia.H;\n";
  o << "const int xs = tx * " << L.out_w << " - " << L.lpad << ";\n";
  o << "const int y_top = y0 - " << HT << ";\n";
  o << "const int nsteps = " << HT << " + T + " << L.nsx << ";\n";
  o << "const int nsrc = " << HT << " + T + " << HB << ";\n";
  o << "const int nrows = min(nsrc, H - y_top);\n";
  o << "const bool st_lane = lane >= " << L.lpad / V << " && lane < " << 32 - L.rpad / V << ";\n";
  o << "(void)st_lane;\n";
  // clamp-to-edge along x (emit_xfix): xs is a multiple of V, so the
  // columns left of 0 are whole lanes; column W - 1 lies in lane xrl_
  // (32: right of the tile) at element xre_
  o << "const int xl0_ = xs < 0 ? min(-xs / " << V << ", 31) : 0;\n";
  o << "const int xr_ = W - 1 - xs;\n";
  o << "const int xrl_ = xr_ < " << 32 * V - 1 << " ? xr_ / " << V << " : 32;\n";
  o << "const int xre_ = xr_ - xrl_ * " << V << ";\n";
  o << "int fixr_ = 0;\n";
  o << "for (int e_ = 0; e_ < " << V << "; e_++) fixr_ |= (lane * " << V << " + e_ > xr_ ? 1 : 0) << e_;\n";
  o << "const bool fxl_ = xs < 0 && lane == xl0_;\n";
  o << "const bool fxr_ = lane == xrl_;\n";
  o << "(void)xl0_; (void)xrl_; (void)xre_; (void)fixr_; (void)fxl_; (void)fxr_;\n";
  for (const Node &n : g.nodes)
    if (n.is_liveout) {
      std::string D = std::to_string(n.dst_index);
      const int esz = elem_bytes(key.dst_dtypes.at(n.dst_index));
      o << "unsigned char *ob" << D << " = (unsigned char *)ia.dst[" << D << "].ptr + (wt_i64)"
        << (n.channels > 1 ? "ch" : "0") << " * ia.dst[" << D << "].plane + (wt_i64)(xs + lane * " << V << ") * " << esz
        << ";\n(void)ob" << D << ";\n";
    }
  o << "bool border = xs < 0 || xs + " << 32 * V << " > W || y_top < 0 || y0 + T + " << HB << " > H;\n";
  c.rowsafe_blocks = g.n_gather == 0;
  c.edge_reads = true;
  for (const Node &n : g.nodes)
    if (!n.gather_mode && (n.xl > V || n.xr > V)) c.edge_reads = false;
  if (c.rowsafe_blocks) {
    // Unguarded blocks need every row they read inside the image: block kb
    // reads rows down to y_top + kb - margin (the deepest row a node reads
    // above its own, delay included) and computes source rows up to
    // y_top + kb + U - 1 (only rows past the tile's last needed source row,
    // never stored, may leave the image).
    int margin = 0;
    for (size_t i = 0; i < g.nodes.size(); i++) {
      const Node &n = g.nodes[i];
      if (n.is_source) continue;
      int dmin = 0;
      for (const NodeEdge &e : g.edges)
        if (e.c == (int)i) dmin = std::min(dmin, e.dymin);
      margin = std::max(margin, n.delay - dmin);
    }
    o << "const int kb_lo_ = " << margin << " - y_top;\n";
    o << "const int kb_hi_ = y0 + T + " << HB << " <= H ? 0x7fffffff : H - " << c.U << " - y_top;\n";
    o << "const bool xedge_ = xs < 0 || xs + " << 32 * V << " > W;\n";
    for (const Node &n : g.nodes)
      if (n.is_liveout) {
        const std::string D = std::to_string(n.dst_index);
        o << "const wt_i64 opitch" << D << " = ia.dst[" << D << "].pitch;\n";
        o << "unsigned char *obt" << D << " = ob" << D << " + (wt_i64)(y_top - " << n.delay << ") * opitch" << D
          << ";\n";
      }
  }
  // Gather sources: the guard-free body reads them unclamped, in aligned
  // pairs, at every row it computes (garbage rows included: k from 0 to
  // the last unrolled step), so a tile whose footprint reaches past a
  // gather source's edge runs the guarded body.
  for (size_t gi = 0; gi < g.nodes.size(); gi++) {
    const Node &gn = g.nodes[gi];
    if (!gn.gather_mode) continue;
    int omin = 1 << 20, omax = -(1 << 20), dymin = 1 << 20, dymax = -(1 << 20), dmax = 0, dmin = 1 << 20;
    for (const Node &cn : g.nodes)
      for (const KOp &op : cn.prog)
        if (op.op == WT_OP_TAP && op.node == (int)gi) {
          for (int e = 0; e < V; e++) {
            omin = std::min(omin, gather_off(gn.gather_mode, e, op.dx));
            omax = std::max(omax, gather_off(gn.gather_mode, e, op.dx));
          }
          dymin = std::min(dymin, op.dy);
          dymax = std::max(dymax, op.dy);
          dmax = std::max(dmax, cn.delay);
          dmin = std::min(dmin, cn.delay);
        }
    if (omin > omax) continue;
    const int gm = gn.gather_mode;
    // columns read: whole aligned pairs where the loads are pairs
    const bool pr = gather_pairs(gm);
    const int plo = pr ? omin - (((omin % 2) + 2) % 2) : omin;
    const int phi = pr ? omax + (((omax % 2) + 2) % 2 == 0 ? 1 : 0) : omax;
    const std::string S = "ia.src[" + std::to_string(gn.src_index) + "]";
    const int gs = tap_shift(gm);
    const bool down = tap_is_down(gm);
    const std::string cb0 = down ? "(xs * " + std::to_string(1 << gs) + ")" : "(xs >> " + std::to_string(gs) + ")";
    const std::string cb31 = down ? "((xs + " + std::to_string(31 * V) + ") * " + std::to_string(1 << gs) + ")"
                                  : "((xs + " + std::to_string(31 * V) + ") >> " + std::to_string(gs) + ")";
    const std::string rlo = "(y_top - " + std::to_string(dmax) + ")";
    const std::string rhi = "(y_top + nsteps + " + std::to_string(c.U - 1 - dmin) + ")";
    o << "border = border || " << cb0 << " + (" << plo << ") < 0 || " << cb31 << " + (" << phi << ") > " << S
      << ".W - 1 || " << gather_row(gm, rlo) << " + (" << dymin << ") < 0 || " << gather_row(gm, rhi) << " + ("
      << dymax << ") > " << S << ".H - 1;\n";
  }
  for (int s = 0; s < n_src; s++) {
    const Node *sn = nullptr;
    for (const Node &n : g.nodes)
      if (n.is_source && n.src_index == s) sn = &n;
    int A = 16 / L.esz[s];
    std::string zc = (sn->src_chan >= 0) ? std::to_string(sn->src_chan) : "ch";
    o << "const int zc" << s << " = " << zc << ";\n";
    if (V % A) o << "const int xb" << s << " = xs & ~" << (A - 1) << ";\n";
    else o << "const int xb" << s << " = xs;\n";
    o << "unsigned char *rb" << s << " = wb + " << L.ring_off[s] << ";\n";
    o << "const unsigned char *lp" << s << " = rb" << s << " + (xs - xb" << s << ") * " << L.esz[s]
      << " + lane * " << V * L.esz[s] << ";\n";
  }
  for (size_t i = 0; i < g.nodes.size(); i++)
    if (L.win_off[i] >= 0)
      o << "unsigned char *sp" << i << " = wb + " << L.win_off[i] << " + lane * " << V * elem_bytes(key.win_dtype)
        << ";\n";
  // chunk issue: lane 0 arms the buffer's mbarrier and starts one TMA box per source
  o << "auto issue_chunk = [&](int c_) {\n__syncwarp();\nif (lane == 0) {\nwt_fence_proxy_async();\n"
       "const int gc_ = cbase + c_;\nconst wt_u32 b_ = bar + 8u * (wt_u32)(gc_ % NB);\n"
       "wt_mbar_expect_tx(b_, "
    << L.chunk_bytes << "u);\n";
  // (test-only stall: chunk 0 of every tile is armed but never copied, so
  // its wait gives up with nothing in flight)
  if (key.test_stall) o << "if (c_ != 0) {\n";
  for (int s = 0; s < n_src; s++)
    o << "wt_tma_load_3d(wt_smem_u32(rb" << s << " + (gc_ % NB) * BUFB" << s << "), &ia.tmap["
      << s << "], xb" << s << ", y_top + c_ * CH, zc" << s << ", b_);\n";
  if (key.test_stall) o << "}\n";
  o << "}\nissued = c_ + 1;\n};\n";
  o << "for (int c_ = 0; c_ < NB - 1; c_++) if (c_ * CH < nrows) issue_chunk(c_);\n";
  (void)kss;
  (void)kse_c;
  // Interior tiles run the guard-free body for every step: rows a node
  // computes outside its range are never stored (row check at the store)
  // and only read by rows that are themselves outside their range.  Border
  // tiles run the guarded body (clamp-to-edge replication) throughout.
  o << "const int U = " << c.U << ";\n";
  // Steady-state steps of interior tiles run the guard-free body; all
  // other steps run the guarded body (both unrolled over U phases so that
  // register windows rotate by renaming).
  // chunk bookkeeping by counters (the block's row in its chunk, kc_, and
  // the chunk, kch_; chunks are a multiple of U rows)
  emit_gwin_decl_init(c);
  o << "int kc_ = 0, kch_ = 0;\n";
  o << "for (int kb = 0; kb < nsteps; kb += U) {\n";
  // TMA bookkeeping once per block: wait for the chunk this block starts,
  // refill the buffer whose rows no step reads any more.
  o << "if (kc_ == 0 && kch_ * CH < nrows) {"
       " const int gc_ = cbase + kch_; const int ok_ = wt_mbar_wait(bar + 8u * (wt_u32)(gc_ % NB),"
       " (wt_u32)((gc_ / NB) & 1), a.err); if (!__all_sync(WT_FULL, ok_)) { failc = kch_; goto wt_fail; } }\n"
       "if (kc_ == ISSUE) { const int c_ = kch_ + NB - 1; if (c_ * CH < nrows) issue_chunk(c_); }\n";
  auto ring_ptrs = [&]() {
    for (int s = 0; s < n_src; s++)
      o << "const unsigned char *rp" << s << " = lp" << s << " + ((cbase + kch_) % NB) * BUFB" << s << " + kc_ * ROWB"
        << s << ";\n";
  };
  if (c.rowsafe_blocks) {
    // the block's body by its rows: unguarded when every row it touches is
    // inside the image (x-edge fix-ups in tiles crossing the left or right
    // edge), guarded otherwise (the first blocks of top tiles, the last
    // blocks of bottom tiles)
    o << "if (kb >= kb_lo_ && kb <= kb_hi_) {\n";
    ring_ptrs();
    for (const Node &n : g.nodes)
      if (n.is_liveout) {
        const std::string D = std::to_string(n.dst_index);
        o << "unsigned char *obk" << D << " = obt" << D << " + (wt_i64)kb * opitch" << D << ";\n";
      }
    o << "if (!xedge_) {\n";
    for (int u = 0; u < c.U; u++) emit_step(c, STEADY, u);
    o << "} else {\n";
    for (int u = 0; u < c.U; u++) emit_step(c, XEDGE, u);
    o << "}\n} else {\n";
    for (int u = 0; u < c.U; u++) emit_step(c, GUARDED, u);
    o << "}\n";
  } else {
    o << "if (!border) {\n";
    ring_ptrs();
    for (int u = 0; u < c.U; u++) emit_step(c, STEADY, u);
    o << "} else {\n";
    for (int u = 0; u < c.U; u++) emit_step(c, GUARDED, u);
    o << "}\n";
  }
  o << "kc_ += U;\nif (kc_ == CH) { kc_ = 0; kch_++; }\n";
  o << "}\n";
  o << "wt_tile_end:;\n";
  o << "cbase += (nrows + CH - 1) / CH;\n";
  o << "}\n";  // tile loop
  o << "wt_exit:\n";
  o << "if (lane == 0 && !a.direct) {\n__threadfence();\nconst int d_ = atomicAdd(a.queue + 1, 1);\n"
       "if (d_ == (int)(gridDim.x * " << key.nw << ") - 1) { atomicExch(a.queue, 0); atomicExch(a.queue + 1, 0); }\n}\n";
  o << "return;\n";
  o << "wt_fail:\n";
  o << "for (int c_ = failc + 1; c_ < issued; c_++) { const int gc_ = cbase + c_;"
       " wt_mbar_wait(bar + 8u * (wt_u32)(gc_ % NB), (wt_u32)((gc_ / NB) & 1), a.err); }\n";
  o << "goto wt_exit;\n";
  o << "}\n";
  return o.str();
}

std::vector<PlainSrc> plain_sources(const Pipeline &p, int sid) {
  std::vector<PlainSrc> r;
  const Stage &S = p.stages[sid];
  for (const Op &op : S.ops) {
    if (op.op != WT_OP_TAP && op.op != WT_OP_TAPZ) continue;
    int pid = S.inputs[op.slot];
    int pc = pid >= 0 ? p.stages[pid].channels : p.in_channels[-pid - 1];
    // plane-offset taps read planes relative to the output's (spec -1)
    int spec = pc == 1 ? 0 : (op.op == WT_OP_TAPZ ? -1 : op.chan);
    bool found = false;
    for (auto &x : r)
      if (x.slot == op.slot && x.chan == spec) found = true;
    if (!found) r.push_back({op.slot, spec});
  }
  return r;
}

bool plain_shares_planes(const Pipeline &p, int sid) {
  const Stage &S = p.stages[sid];
  std::map<int, std::set<int>> planes;  // slot -> fixed planes read by taps up by 4 or 8
  for (const Op &op : S.ops) {
    if (op.op != WT_OP_TAP) continue;
    const int pid = S.inputs[op.slot];
    const int pc = pid >= 0 ? p.stages[pid].channels : p.in_channels[-pid - 1];
    if (pc > 1 && op.chan >= 0 && tap_is_up(op.mode) && tap_shift(op.mode) >= 2) planes[op.slot].insert(op.chan);
  }
  for (const auto &kv : planes)
    if (kv.second.size() >= 2) return true;
  return false;
}

std::string emit_plain(const Pipeline &p, int sid, const CodegenKey &key, const std::string &kname) {
  const Stage &S = p.stages[sid];
  std::vector<PlainSrc> srcs = plain_sources(p, sid);
  if ((int)srcs.size() > kMaxAllSrc) fail(WT_EUNSUPPORTED, "stage reads more than 24 sources");
  // Output pixels per thread.  With 8 the first column x0 of every row
  // segment a thread reads (x0, 2 x0 or x0 / 2) is a multiple of 4, so
  // interior threads load segments with aligned 4-element vectors.
  const int PV = 8;
  std::ostringstream o;
  o << kDeviceSource;
  o << "static_assert(sizeof(WtArgs) == " << sizeof(KernelArgs) << ", \"WtArgs layout\");\n";
  o << "extern \"C\" __global__ void __launch_bounds__(128) " << kname
    << "(const __grid_constant__ WtArgs a) {\n";
  o << "const int x0 = (blockIdx.x * blockDim.x + threadIdx.x) * " << PV << ";\n";
  o << "const int y = blockIdx.y;\nconst int ch = blockIdx.z;\nconst int W = a.W, H = a.H;\n";
  o << "(void)H;\nif (x0 >= W) return;\n";
  // rows to load: per (src, dy): x range per element
  struct Row {
    int s, dy, dxmin, dxmax, mode, dz;
  };
  std::vector<Row> rows;
  // source index and plane offset of a tap
  auto tap_src = [&](const Op &op, int *dz) {
    int pid = S.inputs[op.slot];
    int pc = pid >= 0 ? p.stages[pid].channels : p.in_channels[-pid - 1];
    int spec = pc == 1 ? 0 : (op.op == WT_OP_TAPZ ? -1 : op.chan);
    *dz = (op.op == WT_OP_TAPZ && pc != 1) ? op.chan : 0;
    int s = 0;
    for (size_t i = 0; i < srcs.size(); i++)
      if (srcs[i].slot == op.slot && srcs[i].chan == spec) s = (int)i;
    return s;
  };
  for (const Op &op : S.ops) {
    if (op.op != WT_OP_TAP && op.op != WT_OP_TAPZ) continue;
    int dz = 0;
    const int s = tap_src(op, &dz);
    bool found = false;
    for (auto &r : rows)
      if (r.s == s && r.dy == op.dy && r.dz == dz) {
        r.dxmin = std::min(r.dxmin, op.dx);
        r.dxmax = std::max(r.dxmax, op.dx);
        found = true;
      }
    if (!found) rows.push_back({s, op.dy, op.dx, op.dx, op.mode, dz});
  }
  auto col_index = [&](int mode, int e, int dx) {
    // offset of the producer column, relative to the row base, for element e
    // (x0 is a multiple of 8: (x0 + e) >> s = (x0 >> s) + (e >> s) for s <= 3)
    const int s = tap_shift(mode);
    if (tap_is_down(mode)) return (e << s) + dx;
    if (tap_is_up(mode)) return (e >> s) + dx;
    return e + dx;
  };
  for (size_t ri = 0; ri < rows.size(); ri++) {
    const Row &r = rows[ri];
    int s = r.s;
    int dt = key.src_dtypes.at(s);
    int lo = col_index(r.mode, 0, r.dxmin), hi = col_index(r.mode, PV - 1, r.dxmax);
    // A fixed plane of a producer whose same row segment an earlier row
    // already addresses through another fixed plane (a multi-plane grid
    // read plane by plane): that row's pointer plus the plane offset, and
    // its descriptor for the clamps, so the column clamps and offsets are
    // computed once for all the planes.
    // (Rows of taps up by 4 or 8 only: they load scalars in any case.)
    const bool scalar_row = tap_is_up(r.mode) && tap_shift(r.mode) >= 2;
    int same = -1;
    if (srcs[s].chan >= 0 && scalar_row)
      for (size_t q = 0; q < ri && same < 0; q++) {
        const Row &rq = rows[q];
        if (srcs[rq.s].slot == srcs[s].slot && srcs[rq.s].chan >= 0 && rq.dy == r.dy && rq.dz == r.dz &&
            rq.mode == r.mode && rq.dxmin == r.dxmin && rq.dxmax == r.dxmax && key.src_dtypes.at(rq.s) == dt)
          same = (int)q;
      }
    if (same >= 0) {
      const int s0 = rows[same].s;
      const std::string sd0 = "a.src[" + std::to_string(s0) + "]";
      o << "const unsigned char *rp" << ri << " = rp" << same << " + (wt_i64)(" << srcs[s].chan - srcs[s0].chan
        << ") * " << sd0 << ".plane;\n";
      o << "float";
      for (int j = lo; j <= hi; j++) o << (j == lo ? " " : ", ") << "L" << ri << "_" << (j - lo);
      o << ";\n";
      for (int j = lo; j <= hi; j++)
        o << "L" << ri << "_" << (j - lo) << " = wt_ld1_" << dtype_name(dt) << "(rp" << ri << " + (rp" << same
          << "_o" << (j - lo) << "));\n";
      continue;
    }
    std::string sd = "a.src[" + std::to_string(s) + "]";
    std::string zc = srcs[s].chan >= 0 ? std::to_string(srcs[s].chan)
                     : r.dz == 0 ? std::string("ch")
                                 : "wt_clampi(ch + (" + std::to_string(r.dz) + "), 0, " + sd + ".C - 1)";
    const int sh = tap_shift(r.mode);
    std::string base = tap_is_down(r.mode) ? "(x0 * " + std::to_string(1 << sh) + ")"
                       : (tap_is_up(r.mode) ? "(x0 >> " + std::to_string(sh) + ")" : "x0");
    std::string ybase = tap_is_down(r.mode) ? "(y * " + std::to_string(1 << sh) + ")"
                        : (tap_is_up(r.mode) ? "(y >> " + std::to_string(sh) + ")" : "y");
    // aligned 4-vectors need a base that is a multiple of 4: every mode but
    // up by 4 or 8 (x0 >> 2 or x0 >> 3 of a multiple of 8)
    const bool vec_ok = !(tap_is_up(r.mode) && sh >= 2);
    o << "const unsigned char *rp" << ri << " = (const unsigned char *)" << sd << ".ptr + (wt_i64)" << zc
      << " * " << sd << ".plane + (wt_i64)wt_clampi(" << ybase << " + (" << r.dy << "), 0, " << sd
      << ".H - 1) * " << sd << ".pitch;\n";
    // the segment's columns base + lo .. base + hi: whole aligned 4-vectors
    // when they lie inside the row, else clamped scalar loads
    auto floor4 = [](int v) { return (v >= 0 ? v / 4 : -((-v + 3) / 4)) * 4; };
    const int lo_a = floor4(lo);
    const int hi_a = floor4(hi) + 3;
    const int nv = (hi_a - lo_a + 1) / 4;
    std::vector<std::string> vals(nv * 4);
    o << "float";
    for (int j = lo; j <= hi; j++) o << (j == lo ? " " : ", ") << "L" << ri << "_" << (j - lo);
    o << ";\n";
    o << "if (" << (vec_ok ? "true" : "false") << " && " << base << " + (" << lo_a << ") >= 0 && " << base << " + ("
      << hi_a << ") <= " << sd << ".W - 1) {\n";
    for (int k = 0; k < nv; k++) {
      o << "{ float q0, q1, q2, q3;\nwt_ld4_" << dtype_name(dt) << "(rp" << ri << " + (wt_i64)(" << base << " + (" << lo_a + 4 * k
        << ")) * " << elem_bytes(dt) << ", q0, q1, q2, q3);\n";
      for (int t = 0; t < 4; t++) {
        int j = lo_a + 4 * k + t;
        if (j >= lo && j <= hi) o << "L" << ri << "_" << (j - lo) << " = q" << t << ";\n";
      }
      o << "}\n";
    }
    o << "} else {\n";
    for (int j = lo; j <= hi; j++)
      o << "L" << ri << "_" << (j - lo) << " = wt_ld1_" << dtype_name(dt) << "(rp" << ri
        << " + (wt_i64)wt_clampi(" << base << " + (" << j << "), 0, " << sd << ".W - 1) * "
        << elem_bytes(dt) << ");\n";
    o << "}\n";
    // the clamped column offsets of this row, for the planes that share it
    bool shared = false;
    for (size_t q = ri + 1; q < rows.size(); q++)
      if (srcs[rows[q].s].slot == srcs[s].slot && srcs[s].chan >= 0 && tap_is_up(r.mode) && tap_shift(r.mode) >= 2)
        shared = true;
    if (shared)
      for (int j = lo; j <= hi; j++)
        o << "const wt_i64 rp" << ri << "_o" << (j - lo) << " = (wt_i64)wt_clampi(" << base << " + (" << j
          << "), 0, " << sd << ".W - 1) * " << elem_bytes(dt) << ";\n";
  }
  for (int e = 0; e < PV; e++) {
    std::vector<std::string> st;
    for (const Op &op : S.ops) {
      switch (op.op) {
        case WT_OP_CONST: st.push_back(float_literal(op.value)); break;
        case WT_OP_XPAR: st.push_back("((float)((x0 + " + std::to_string(e) + ") & 1))"); break;
        case WT_OP_YPAR: st.push_back("((float)(y & 1))"); break;
        case WT_OP_CHAN: st.push_back("((float)ch)"); break;
        case WT_OP_TAP: case WT_OP_TAPZ: {
          int dz = 0;
          const int s = tap_src(op, &dz);
          int ri = 0;
          for (size_t i = 0; i < rows.size(); i++)
            if (rows[i].s == s && rows[i].dy == op.dy && rows[i].dz == dz) ri = (int)i;
          int lo = col_index(rows[ri].mode, 0, rows[ri].dxmin);
          int j = col_index(op.mode, e, op.dx) - lo;
          st.push_back("L" + std::to_string(ri) + "_" + std::to_string(j));
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
    o << "const float v" << e << " = " << st.back() << ";\n";
  }
  int dt = key.dst_dtypes.at(0);
  int esz = elem_bytes(dt);
  o << "unsigned char *op_ = (unsigned char *)a.dst[0].ptr + (wt_i64)" << (S.channels > 1 ? "ch" : "0")
    << " * a.dst[0].plane + (wt_i64)y * a.dst[0].pitch + (wt_i64)x0 * " << esz << ";\n";
  o << "if (x0 + " << PV << " <= W) {";
  for (int b = 0; b < PV; b += 4)
    o << " wt_st4_" << dtype_name(dt) << "(op_ + " << b * esz << ", v" << b << ", v" << b + 1 << ", v" << b + 2 << ", v" << b + 3
      << ");";
  o << " } else {\n";
  for (int e = 0; e < PV; e++)
    o << "if (x0 + " << e << " < W) wt_st1_" << dtype_name(dt) << "(op_ + " << e * esz << ", v" << e << ");\n";
  o << "}\n}\n";
  return o.str();
}

}  // namespace wt

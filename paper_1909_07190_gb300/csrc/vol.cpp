// 3-D fused groups: the generalised hybrid tiling of App. A (Alg. 3,
// Fig. 8) on volumes.
//
// A D x H x W volume is an image of D planes; stages read producers at
// constant offsets (dx, dy, dz) (WT_OP_TAPZ, clamp-to-edge in every axis).
// One warp computes one overlapped tile of a group:
//   * x: 32 lanes x V points; the tile's outputs are the columns left after
//     the group's x halo (overlapped tiling, Sec. 4);
//   * the split axis s (rows, or planes with WT_FLAG_ZSTREAM): streamed, Ts
//     output points per tile; each node keeps a window of its last rows
//     (register rotation by unrolling, Sec. 5);
//   * the third axis o: a register tile (App. A: R_j = T_j for the axes
//     that are not split) of vol_to output points plus each node's halo.
// Producer reads are then register reads: along o from another o point of
// the same thread (Type 1 of Fig. 8 with W_o = 1), along s from an older
// window slot, along x from the lane that holds the column, by shuffle at
// the tap (Types 3/4).  Sources (pipeline inputs, earlier groups) are
// register windows too, each row loaded two steps before its first use.
//
// Clamp-to-edge at every stage: a node's value at a point outside the
// volume is its value at the clamped point.  Rows before 0 are not computed;
// when row 0 is, it is copied into the older slots; rows past the end copy
// the previous row.  o points outside [0, N_o) copy their nearest in-range
// neighbour after each row; x points outside [0, W) take the value of
// column 0 or W-1 by shuffle (border tiles only).
#include <algorithm>
#include <numeric>
#include <map>
#include <set>
#include <sstream>
#include <tuple>

#include "wt_internal.hpp"

namespace wt {


int VolGeom::node_of(int id) const {
  for (size_t i = 0; i < nodes.size(); i++)
    if (nodes[i].id == id) return (int)i;
  return -1;
}

// Shared-memory rows of source si: 32 V columns plus the sources' x
// margins plus alignment slack, rounded to 16 bytes.
static int src_row_bytes(const VolGeom &g, const CodegenKey &key, int si) {
  const int esz = elem_bytes(key.src_dtypes.at(g.nodes[si].src_index));
  return (((32 * g.V + g.xml + g.xmr + 4 / esz) * esz) + 15) / 16 * 16;
}

int vol_warp_smem(const VolGeom &g, const CodegenKey &key, std::vector<int> *offs) {
  int off = 0;
  if (offs) offs->assign(g.nodes.size(), -1);
  if (!g.staged) return 0;
  for (size_t i = 0; i < g.nodes.size(); i++) {
    const VolNode &n = g.nodes[i];
    if (!n.source) continue;
    if (offs) (*offs)[i] = off;
    off += n.window * (g.To + n.olo + n.ohi) * src_row_bytes(g, key, (int)i);
  }
  return off;
}

namespace {

// A tap of a group stage in (x, s, o) coordinates.
struct VTap {
  int node = 0;  // producer node index
  int dx = 0, ds = 0, dO = 0;
};

// Taps of stage program ops, in program order (non-tap ops: node = -1).
std::vector<VTap> stage_taps(const Pipeline &p, const VolGeom &g, int sid) {
  const Stage &S = p.stages[sid];
  std::vector<VTap> out;
  for (const Op &op : S.ops) {
    VTap t;
    t.node = -1;
    if (op.op == WT_OP_TAP || op.op == WT_OP_TAPZ) {
      const int dz = op.op == WT_OP_TAPZ ? op.chan : 0;
      t.node = g.node_of(S.inputs[op.slot]);
      t.dx = op.dx;
      t.ds = g.split == 0 ? op.dy : dz;
      t.dO = g.split == 0 ? dz : op.dy;
    }
    out.push_back(t);
  }
  return out;
}

}  // namespace

VolGeom vol_analyze(const Pipeline &p, const std::vector<int> &stages, int split, int To, int Ts, int V,
                    bool staged, int prefetch) {
  VolGeom g;
  g.staged = staged;
  g.prefetch = std::max(1, std::min(8, prefetch));
  g.split = split;
  g.To = std::max(1, To);
  g.Ts = std::max(1, Ts);
  g.V = V;
  auto no = [&](const std::string &why) {
    g.ok = false;
    g.why = why;
    return g;
  };
  if (V != 1 && V != 2 && V != 4) return no("vec must be 1, 2 or 4");
  if (stages.empty()) return no("empty group");
  g.D = p.stages[stages[0]].channels;
  g.level = p.stages[stages[0]].level;
  std::set<int> in_group(stages.begin(), stages.end());
  // sources in order of first use, then the stages
  std::vector<int> src_ids;
  for (int s : stages) {
    const Stage &S = p.stages[s];
    if (S.channels != g.D) return no("stages of a 3-D group need one plane count");
    if (S.level != g.level) return no("stages of a 3-D group need one level");
    for (const Op &op : S.ops) {
      if (op.op == WT_OP_XPAR || op.op == WT_OP_YPAR || op.op == WT_OP_CHAN)
        return no("parity and channel ops are not supported in 3-D groups");
      if (op.op != WT_OP_TAP && op.op != WT_OP_TAPZ) continue;
      if (op.op == WT_OP_TAP && (op.mode != WT_TAP_SAME || op.chan >= 0))
        return no("3-D groups read producers at their own level and plane offsets only");
      const int pid = S.inputs[op.slot];
      if (in_group.count(pid)) continue;
      if (std::find(src_ids.begin(), src_ids.end(), pid) == src_ids.end()) src_ids.push_back(pid);
    }
  }
  if ((int)src_ids.size() > kMaxAllSrc) return no("too many sources");
  for (size_t k = 0; k < src_ids.size(); k++) {
    const int id = src_ids[k];
    VolNode n;
    n.id = id;
    n.source = true;
    n.src_index = (int)k;
    n.planes = id >= 0 ? p.stages[id].channels : p.in_channels[-id - 1];
    if (n.planes != 1 && n.planes != g.D) return no("a source of a 3-D group has another plane count");
    g.nodes.push_back(n);
  }
  for (int s : stages) {
    VolNode n;
    n.id = s;
    n.planes = g.D;
    g.nodes.push_back(n);
  }
  for (int s : stages) {
    bool live = p.is_output[s] != 0;
    for (int c : p.consumers[s])
      if (!in_group.count(c)) live = true;
    if (live) {
      g.nodes[g.node_of(s)].dst_index = (int)g.liveouts.size();
      g.liveouts.push_back(s);
    }
  }
  if (g.liveouts.empty()) return no("group without liveouts");
  if ((int)g.liveouts.size() > kMaxDst) return no("too many liveouts");
  const int N = (int)g.nodes.size();
  // Backward pass over the stages (reverse topological order): x, o and s
  // requirements of every producer from its consumers' (Sec. 4 overlapped
  // tiles; App. A right hyperplanes per axis).
  std::vector<int> nl(N, 0), nr(N, 0), lead(N, 0), need_lo(N, 0), olo(N, 0), ohi(N, 0);
  std::vector<char> needed(N, 0);
  for (int s : g.liveouts) needed[g.node_of(s)] = 1;
  for (int k = (int)stages.size() - 1; k >= 0; k--) {
    const int ci = g.node_of(stages[k]);
    if (!needed[ci]) continue;
    // every consumer covers at least the tile's own columns, rows and o
    // points (final here: its consumers come later in the order)
    nl[ci] = std::max(nl[ci], 0); nr[ci] = std::max(nr[ci], 0);
    olo[ci] = std::max(olo[ci], 0); ohi[ci] = std::max(ohi[ci], 0);
    need_lo[ci] = std::min(need_lo[ci], 0);
    for (const VTap &t : stage_taps(p, g, stages[k])) {
      if (t.node < 0) continue;
      const int pi = t.node;
      if (!needed[pi]) {
        needed[pi] = 1;
        nl[pi] = nl[ci] - t.dx; nr[pi] = nr[ci] + t.dx;
        lead[pi] = lead[ci] + std::max(0, t.ds);
        need_lo[pi] = need_lo[ci] + t.ds;
        olo[pi] = olo[ci] - t.dO; ohi[pi] = ohi[ci] + t.dO;
      } else {
        nl[pi] = std::max(nl[pi], nl[ci] - t.dx); nr[pi] = std::max(nr[pi], nr[ci] + t.dx);
        lead[pi] = std::max(lead[pi], lead[ci] + std::max(0, t.ds));
        need_lo[pi] = std::min(need_lo[pi], need_lo[ci] + t.ds);
        olo[pi] = std::max(olo[pi], olo[ci] - t.dO); ohi[pi] = std::max(ohi[pi], ohi[ci] + t.dO);
      }
    }
  }
  // sources likewise
  for (int i = 0; i < N; i++) {
    if (!needed[i]) continue;
    nl[i] = std::max(nl[i], 0); nr[i] = std::max(nr[i], 0);
    olo[i] = std::max(olo[i], 0); ohi[i] = std::max(ohi[i], 0);
    need_lo[i] = std::min(need_lo[i], 0);
  }
  for (int k = 0; k < (int)stages.size(); k++)
    if (!needed[g.node_of(stages[k])]) return no("dead stage inside a 3-D group");
  g.pro = 0;
  for (int i = 0; i < N; i++) {
    VolNode &n = g.nodes[i];
    n.lead = lead[i];
    n.need_lo = need_lo[i];
    n.olo = olo[i];
    n.ohi = ohi[i];
    g.hxl = std::max(g.hxl, nl[i]);
    g.hxr = std::max(g.hxr, nr[i]);
    // sources are loaded `prefetch` rows before their first use, so that a
    // load's latency overlaps the steps in between
    if (n.source) n.lead += g.prefetch;
    g.pro = std::max(g.pro, n.lead - n.need_lo);
  }
  // windows of every node, source x margins
  for (int k = 0; k < (int)stages.size(); k++) {
    const int ci = g.node_of(stages[k]);
    for (const VTap &t : stage_taps(p, g, stages[k])) {
      if (t.node < 0) continue;
      VolNode &pn = g.nodes[t.node];
      const VolNode &cn = g.nodes[ci];
      pn.window = std::max(pn.window, pn.lead - cn.lead - t.ds + 1);
      // every node keeps its own V values per row; x neighbours come by
      // shuffle at the tap (fewer registers, more warps per SM)
      if (-t.dx > 32 * V - 1 || t.dx > 32 * V - 1) return no("x taps wider than a warp tile");
      if (pn.source) {
        // loads are clamped: no copies at the borders
        g.xml = std::max(g.xml, -t.dx);
        g.xmr = std::max(g.xmr, t.dx);
        continue;
      }
      // a row past the end copies the previous one: keep it
      if (t.ds > 0) pn.window = std::max(pn.window, 2);
    }
  }
  g.hxlp = (g.hxl + V - 1) / V * V;
  g.ow = (32 * V - g.hxlp - g.hxr) / V * V;
  if (g.ow < V) return no("x halo leaves no output columns");
  // unroll: the least common multiple of the windows when small, else the
  // largest window (nodes whose window does not divide it shift)
  // (staged sources live in shared memory, their slots chosen at run time)
  auto in_regs = [&](const VolNode &n) { return !n.source || !g.staged; };
  int U = 1;
  for (const VolNode &n : g.nodes)
    if (in_regs(n)) U = std::lcm(U, n.window);
  if (U > 8) {
    U = 1;
    for (const VolNode &n : g.nodes)
      if (in_regs(n)) U = std::max(U, n.window);
  }
  g.U = U;
  g.regs = 0;
  for (VolNode &n : g.nodes) {
    n.rotate = U % n.window == 0;
    if (in_regs(n)) g.regs += n.window * (g.To + n.olo + n.ohi) * (V + n.xl + n.xr);
  }
  if (g.regs > 224) return no("3-D group windows need " + std::to_string(g.regs) +
                              " registers per thread; lower tile_o or vec");
  g.ok = true;
  return g;
}

namespace {

struct Emit {
  const Pipeline &p;
  const VolGeom &g;
  const CodegenKey &key;
  std::ostringstream o;
  Emit(const Pipeline &pp, const VolGeom &gg, const CodegenKey &k) : p(pp), g(gg), key(k) {}

  int ninst(const VolNode &n) const { return g.To + n.olo + n.ohi; }
  // slot of age a at unrolled step u
  int slot(const VolNode &n, int u, int a) const {
    if (n.rotate) return ((u - a) % n.window + n.window) % n.window;
    return a;
  }
  // register of node ni, slot sl, o point j (relative to o0), x entry e
  // (relative to the lane's first column; -xl .. V - 1 + xr)
  std::string reg(int ni, int sl, int j, int e) const {
    const VolNode &n = g.nodes[ni];
    return "w" + std::to_string(ni) + "_" + std::to_string(sl) + "_" + std::to_string(j + n.olo) + "_" +
           std::to_string(e + n.xl);
  }
  std::string o_index(const std::string &j) const { return "wt_clampi(o0 + (" + j + "), 0, NO - 1)"; }

  // A node's value at x entry e (any integer) of its window register: own
  // entries directly, others from the lane that holds them.
  std::string src_val(int si, int sl, int j, int e) const {
    const int V = g.V;
    if (e >= 0 && e < V) return reg(si, sl, j, e);
    if (e < 0) {
      const int dl = (-e + V - 1) / V;
      return "__shfl_up_sync(WT_FULL, " + reg(si, sl, j, e + dl * V) + ", " + std::to_string(dl) + ")";
    }
    const int dl = e / V;
    return "__shfl_down_sync(WT_FULL, " + reg(si, sl, j, e - dl * V) + ", " + std::to_string(dl) + ")";
  }
  void load_source(int si, bool safe);
  void load_source_regs(int si, int u, bool safe);
  std::string src_tap(int si, int age, int j, int e) const;
  std::set<int> src_ages(int si) const;
  void program(int sid, int ni, int u, bool safe);
  void store_row(int ni, int u, bool safe);
  void liveout(int ni, int u, bool safe);
  void step(int u, bool safe);
  std::string run();
};

// Evaluates stage `sid` (node ni) for every o point of its range at the
// node's row of step u, into the age-0 slot.
void Emit::program(int sid, int ni, int u, bool safe) {
  const Stage &S = p.stages[sid];
  const VolNode &n = g.nodes[ni];
  const std::vector<VTap> taps = stage_taps(p, g, sid);
  const int V = g.V;
  const int sl0 = slot(n, u, 0);
  for (int j = -n.olo; j < g.To + n.ohi; j++) {
    o << "{\n";
    // producers' x neighbours by shuffle, once per o point
    std::map<std::tuple<int, int, int, int>, std::string> nb;
    for (int e = 0; e < V; e++)
      for (const VTap &t : taps) {
        if (t.node < 0 || (g.nodes[t.node].source && g.staged)) continue;
        const int ee = e + t.dx;
        if (ee >= 0 && ee < V) continue;
        const VolNode &pn = g.nodes[t.node];
        auto key4 = std::make_tuple(t.node, slot(pn, u, pn.lead - n.lead - t.ds), j + t.dO, ee);
        if (nb.count(key4)) continue;
        const std::string name = "nb" + std::to_string(nb.size()) + "_";
        o << "const float " << name << " = " << src_val(t.node, std::get<1>(key4), std::get<2>(key4), ee) << ";\n";
        nb[key4] = name;
      }
    for (int e = 0; e < V; e++) {
      std::vector<std::string> st;
      for (size_t k = 0; k < S.ops.size(); k++) {
        const Op &op = S.ops[k];
        switch (op.op) {
          case WT_OP_CONST: st.push_back(float_literal(op.value)); break;
          case WT_OP_TAP: case WT_OP_TAPZ: {
            const VTap &t = taps[k];
            const VolNode &pn = g.nodes[t.node];
            const int age = pn.lead - n.lead - t.ds;
            const int ee = e + t.dx;
            if (pn.source && g.staged)
              st.push_back(src_tap(t.node, age, j + t.dO, ee));
            else if (ee < 0 || ee >= V)
              st.push_back(nb.at(std::make_tuple(t.node, slot(pn, u, age), j + t.dO, ee)));
            else
              st.push_back(reg(t.node, slot(pn, u, age), j + t.dO, ee));
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
              default: fail(WT_EINVAL, "internal: opcode in a 3-D group");
            }
          }
        }
      }
      o << "v" << e << " = " << st.back() << ";\n";
    }
    // clamp-to-edge along x in border tiles: columns left of 0 take column
    // 0's value (element 0 of lane -xs/V), columns right of W-1 take W-1's
    if (safe) {
      o << "if (xb) {\n";
      o << "const float fl_ = __shfl_sync(WT_FULL, v0, lz_);\n";
      o << "float sr_ = v0;\n";
      for (int e = 1; e < V; e++) o << "if (ez_ == " << e << ") sr_ = v" << e << ";\n";
      o << "const float fr_ = __shfl_sync(WT_FULL, sr_, lw_);\n";
      for (int e = 0; e < V; e++)
        o << "if (xl0 + " << e << " < 0) v" << e << " = fl_; else if (xl0 + " << e << " > W - 1) v" << e
          << " = fr_;\n";
      o << "}\n";
    }
    for (int e = 0; e < V; e++) o << reg(ni, sl0, j, e) << " = v" << e << ";\n";
    o << "}\n";
  }
}

// Stages source si's row of this step (clamped row and o point: a
// source's value outside the volume is the clamped point's) into its
// run-time slot sk of the warp's shared memory, by asynchronous copies:
// interior tiles copy the row segment in 4-byte chunks from an aligned
// start column `seg`, border tiles copy element by element from clamped
// columns (16-bit elements by plain loads and stores).
void Emit::load_source(int si, bool safe) {
  const VolNode &n = g.nodes[si];
  const int V = g.V;
  const int dt = key.src_dtypes.at(n.src_index);
  const int esz = elem_bytes(dt);
  const int NI = g.To + n.olo + n.ohi;
  const int RB = src_row_bytes(g, key, si);
  const int M = 4 / esz - 1;
  const std::string S = "a.src[" + std::to_string(n.src_index) + "]";
  const std::string sn = std::to_string(si);
  if (g.split == 0) o << "const unsigned char *rb_ = sb" << sn << " + (wt_i64)wt_clampi(rn, 0, NS - 1) * " << S << ".pitch;\n";
  else if (n.planes == 1) o << "const unsigned char *rb_ = sb" << sn << ";\n";
  else o << "const unsigned char *rb_ = sb" << sn << " + (wt_i64)wt_clampi(rn, 0, NS - 1) * " << S << ".plane;\n";
  o << "unsigned char *sd_ = ss" << sn << " + sk" << sn << " * " << NI * RB << ";\n";
  const int RL = 32 * V + g.xml + g.xmr;              // elements per staged row
  const int NC = ((RL + M) * esz + 3) / 4;            // 4-byte chunks from seg
  for (int j = -n.olo; j < g.To + n.ohi; j++) {
    o << "{ const unsigned char *rp_ = rb_ + so" << sn << "_" << j + n.olo << ";\n";
    o << "const wt_u32 dp_ = wt_smem_u32(sd_ + " << (j + n.olo) * RB << ");\n";
    if (!safe) {
      o << "rp_ += (wt_i64)seg" << sn << " * " << esz << ";\n";
      for (int m = 0; 32 * m < NC; m++) {
        const bool guard = 32 * (m + 1) > NC;
        o << "{ const int c_ = lane + " << 32 * m << ";";
        if (guard) o << " if (c_ < " << NC << ")";
        o << " wt_cp_async4(dp_ + 4u * (wt_u32)c_, rp_ + 4 * c_); }\n";
      }
    } else {
      for (int m = 0; 32 * m < RL; m++) {
        const bool guard = 32 * (m + 1) > RL;
        o << "{ const int i_ = lane + " << 32 * m << ";";
        if (guard) o << " if (i_ < " << RL << ")";
        o << " { const int c_ = wt_clampi(seg" << sn << " + i_, 0, W - 1);";
        if (esz == 4) o << " wt_cp_async4(dp_ + 4u * (wt_u32)i_, rp_ + 4 * c_);";
        else o << " *(wt_u16 *)(sd_ + " << (j + n.olo) * RB << " + 2 * i_) = *(const wt_u16 *)(rp_ + 2 * c_);";
        o << " } }\n";
      }
    }
    o << "}\n";
  }
}

// Loads source si's row of step u into its age-0 register slot (sources in
// registers, frac_reg = 1): the lane's V columns, one vector load in
// interior tiles (the first column is a multiple of V and rows are 16-byte
// aligned), clamped scalar loads in border tiles.
void Emit::load_source_regs(int si, int u, bool safe) {
  const VolNode &n = g.nodes[si];
  const int V = g.V;
  const int sl0 = slot(n, u, 0);
  const int dt = key.src_dtypes.at(n.src_index);
  const int esz = elem_bytes(dt);
  const std::string dn = dtype_name(dt);
  const std::string S = "a.src[" + std::to_string(n.src_index) + "]";
  if (g.split == 0) o << "const unsigned char *rb_ = sb" << si << " + (wt_i64)wt_clampi(rn, 0, NS - 1) * " << S << ".pitch;\n";
  else if (n.planes == 1) o << "const unsigned char *rb_ = sb" << si << ";\n";
  else o << "const unsigned char *rb_ = sb" << si << " + (wt_i64)wt_clampi(rn, 0, NS - 1) * " << S << ".plane;\n";
  for (int j = -n.olo; j < g.To + n.ohi; j++) {
    o << "{ const unsigned char *rp_ = rb_ + so" << si << "_" << j + n.olo << ";\n";
    if (!safe && V == 4) {
      o << "wt_ld4_" << dn << "(rp_ + (wt_i64)xl0 * " << esz << ", " << reg(si, sl0, j, 0) << ", "
        << reg(si, sl0, j, 1) << ", " << reg(si, sl0, j, 2) << ", " << reg(si, sl0, j, 3) << ");\n";
    } else if (!safe && V == 2) {
      o << "wt_ld2_" << dn << "(rp_ + (wt_i64)xl0 * " << esz << ", " << reg(si, sl0, j, 0) << ", "
        << reg(si, sl0, j, 1) << ");\n";
    } else {
      for (int e = 0; e < V; e++) {
        const std::string col = "(xl0 + " + std::to_string(e) + ")";
        o << reg(si, sl0, j, e) << " = wt_ld1_" << dn << "(rp_ + (wt_i64)"
          << (safe ? "wt_clampi(" + col + ", 0, W - 1)" : col) << " * " << esz << ");\n";
      }
    }
    o << "}\n";
  }
}

// A source tap: the staged value at o point j (relative), x entry e of the
// lane, from the row of the given age.
std::string Emit::src_tap(int si, int age, int j, int e) const {
  const VolNode &n = g.nodes[si];
  const int dt = key.src_dtypes.at(n.src_index);
  const int esz = elem_bytes(dt);
  const int RB = src_row_bytes(g, key, si);
  return "wt_lds1_" + std::string(dtype_name(dt)) + "(sa" + std::to_string(si) + "_" + std::to_string(age) + " + " +
         std::to_string((j + n.olo) * RB + e * esz) + ")";
}

// o points outside [0, NO): copies of the nearest in-range point (all
// stored entries), after every o point of the row is computed.
void Emit::store_row(int ni, int u, bool safe) {
  (void)safe;
  const VolNode &n = g.nodes[ni];
  const int sl0 = slot(n, u, 0);
  const int V = g.V;
  if (n.olo + n.ohi == 0 && g.To == 1) return;
  o << "if (ob) {\n";
  for (int j = -n.olo + 1; j < g.To + n.ohi; j++) {
    o << "if (o0 + " << j << " > NO - 1) {";
    for (int e = -n.xl; e < V + n.xr; e++) o << " " << reg(ni, sl0, j, e) << " = " << reg(ni, sl0, j - 1, e) << ";";
    o << " }\n";
  }
  for (int j = g.To + n.ohi - 2; j >= -n.olo; j--) {
    o << "if (o0 + " << j << " < 0) {";
    for (int e = -n.xl; e < V + n.xr; e++) o << " " << reg(ni, sl0, j, e) << " = " << reg(ni, sl0, j + 1, e) << ";";
    o << " }\n";
  }
  o << "}\n";
}

void Emit::liveout(int ni, int u, bool safe) {
  const VolNode &n = g.nodes[ni];
  const int sl0 = slot(n, u, 0);
  const int V = g.V;
  const int dt = key.dst_dtypes.at(n.dst_index);
  const int esz = elem_bytes(dt);
  const std::string D = "a.dst[" + std::to_string(n.dst_index) + "]";
  const std::string dn = dtype_name(dt);
  o << "if (rn >= s0 && rn < s0 + " << g.Ts << " && rn < NS && olane) {\n";
  o << "unsigned char *db_ = db" << ni << " + (wt_i64)rn * " << D << (g.split == 0 ? ".pitch" : ".plane") << ";\n";
  for (int j = 0; j < g.To; j++) {
    o << "if (o0 + " << j << " < NO) {\n";
    o << "unsigned char *dp_ = db_ + do" << ni << "_" << j << ";\n";
    if (!safe && V == 4 && dt == WT_F32) {
      // interior tile: every column is inside the row, 16-byte aligned
      o << "wt_st4_f32(dp_, " << reg(ni, sl0, j, 0) << ", " << reg(ni, sl0, j, 1) << ", " << reg(ni, sl0, j, 2) << ", "
        << reg(ni, sl0, j, 3) << ");\n";
    } else {
      for (int e = 0; e < V; e++) {
        if (safe) o << "if (xl0 + " << e << " < W) ";
        o << "wt_st1_" << dn << "(dp_ + " << e * esz << ", " << reg(ni, sl0, j, e) << ");\n";
      }
    }
    o << "}\n";
  }
  o << "}\n";
}

// Ages (rows back from the newest) at which stages read source si.
std::set<int> Emit::src_ages(int si) const {
  std::set<int> ages;
  for (const VolNode &c : g.nodes) {
    if (c.source) continue;
    for (const VTap &t : stage_taps(p, g, c.id))
      if (t.node == si) ages.insert(g.nodes[si].lead - c.lead - t.ds);
  }
  return ages;
}

void Emit::step(int u, bool safe) {
  const int V = g.V;
  if (!g.staged) {
    // sources in registers: this step's rows straight into their windows
    for (size_t ni = 0; ni < g.nodes.size(); ni++) {
      const VolNode &n = g.nodes[ni];
      if (!n.source) continue;
      o << "{ // source " << n.id << "\n";
      o << "const int rn = s0 - " << g.pro << " + k + " << n.lead << ";\n";
      load_source_regs((int)ni, u, safe);
      o << "}\n";
    }
  } else {
    // every lane is done with the slots this step's copies overwrite
    o << "__syncwarp();\n";
    for (size_t ni = 0; ni < g.nodes.size(); ni++) {
      const VolNode &n = g.nodes[ni];
      if (!n.source) continue;
      o << "const int sk" << ni << " = k % " << n.window << ";\n";
      o << "{ // source " << n.id << "\n";
      o << "const int rn = s0 - " << g.pro << " + k + " << n.lead << ";\n";
      load_source((int)ni, safe);
      o << "}\n";
    }
    // rows staged `prefetch` or more steps ago have landed (a stage reads a
    // source no less than `prefetch` rows back); one group per step
    o << "wt_cp_async_commit();\nWT_CP_ASYNC_WAIT(" << g.prefetch << ");\n__syncwarp();\n";
    for (size_t ni = 0; ni < g.nodes.size(); ni++) {
      const VolNode &n = g.nodes[ni];
      if (!n.source) continue;
      const int NI = g.To + n.olo + n.ohi;
      for (int a : src_ages((int)ni)) {
        o << "int t" << ni << "_" << a << " = sk" << ni << " - " << a << "; if (t" << ni << "_" << a << " < 0) t" << ni
          << "_" << a << " += " << n.window << ";\n";
        o << "const unsigned char *sa" << ni << "_" << a << " = sl" << ni << " + t" << ni << "_" << a << " * "
          << NI * src_row_bytes(g, key, (int)ni) << ";\n";
      }
    }
  }
  for (size_t ni = 0; ni < g.nodes.size(); ni++) {
    const VolNode &n = g.nodes[ni];
    if (n.source) continue;
    o << "{ // stage " << n.id << "\n";
    o << "const int rn = s0 - " << g.pro << " + k + " << n.lead << ";\n";
    o << "if (rn >= 0 && rn < NS) {\n";
    program(n.id, (int)ni, u, safe);
    store_row((int)ni, u, safe);
    o << "}";
    if (n.window > 1) {
      // past the end: the previous row's values (clamp-to-edge)
      o << " else if (rn >= NS) {\n";
      const int s0l = slot(n, u, 0), s1l = slot(n, u, 1);
      for (int j = -n.olo; j < g.To + n.ohi; j++)
        for (int e = -n.xl; e < V + n.xr; e++) o << reg((int)ni, s0l, j, e) << " = " << reg((int)ni, s1l, j, e) << ";\n";
      o << "}\n";
      // row 0 stands for the rows before it
      o << "if (rn == 0) {\n";
      for (int a = 1; a < n.window; a++) {
        const int sa = slot(n, u, a);
        for (int j = -n.olo; j < g.To + n.ohi; j++)
          for (int e = -n.xl; e < V + n.xr; e++) o << reg((int)ni, sa, j, e) << " = " << reg((int)ni, s0l, j, e) << ";\n";
      }
      o << "}\n";
    } else {
      o << "\n";
    }
    if (n.dst_index >= 0) liveout((int)ni, u, safe);
    o << "}\n";
  }
}

std::string Emit::run() {
  const int V = g.V;
  o << "const int lane = threadIdx.x & 31;\n";
  o << "const int t_ = blockIdx.x * " << key.nw << " + (threadIdx.x >> 5);\n";
  o << "if (t_ >= a.n_tiles) return;\n";
  o << "const int W = a.W;\n";
  if (g.split == 0) o << "const int NS = a.H, NO = a.channels;\n";
  else o << "const int NS = a.channels, NO = a.H;\n";
  o << "const int tx_ = t_ % a.tiles_x, rest_ = t_ / a.tiles_x;\n";
  o << "const int s0 = (rest_ % a.tiles_y) * " << g.Ts << ", o0 = (rest_ / a.tiles_y) * " << g.To << ";\n";
  o << "const int xs = tx_ * " << g.ow << " - " << g.hxlp << ";\n";
  o << "const int xl0 = xs + lane * " << V << ";\n";
  o << "const bool olane = lane * " << V << " >= " << g.hxlp << " && lane * " << V << " < " << g.hxlp + g.ow
    << ";\n";
  // border tiles: some column a lane computes or reads lies outside [0, W)
  // (interior tiles copy source rows from an aligned start up to 2 M
  // elements past the tile's last column: M = 1 for 16-bit sources)
  int M2 = 0;
  for (const VolNode &n : g.nodes)
    if (g.staged && n.source && elem_bytes(key.src_dtypes.at(n.src_index)) == 2) M2 = 2;
  o << "const bool xb = xs - " << g.xml << " < 0 || xs + " << 32 * V + g.xmr + M2 << " > W;\n";
  int OL = 0, OH = 0;
  for (const VolNode &n : g.nodes) {
    OL = std::max(OL, n.olo);
    OH = std::max(OH, n.ohi);
  }
  o << "const bool ob = o0 - " << OL << " < 0 || o0 + " << g.To - 1 + OH << " > NO - 1;\n";
  o << "const int lz_ = wt_clampi(-xs / " << V << ", 0, 31);\n";
  o << "const int lw_ = wt_clampi((W - 1 - xs) / " << V << ", 0, 31), ez_ = (W - 1 - xs) - ((W - 1 - xs) / " << V
    << ") * " << V << ";\n";
  o << "(void)lz_; (void)lw_; (void)ez_; (void)xb; (void)ob; (void)olane;\n";
  // window registers
  for (size_t ni = 0; ni < g.nodes.size(); ni++) {
    const VolNode &n = g.nodes[ni];
    if (n.source && g.staged) continue;
    for (int sl = 0; sl < n.window; sl++)
      for (int j = -n.olo; j < g.To + n.ohi; j++) {
        o << "float";
        for (int e = -n.xl; e < V + n.xr; e++) o << (e > -n.xl ? ", " : " ") << reg((int)ni, sl, j, e) << " = 0.f";
        o << ";\n";
      }
  }
  // per-row scratch: computed values and source values
  o << "float";
  for (int e = 0; e < V; e++) o << (e ? ", " : " ") << "v" << e;
  o << ";\n";
  std::vector<int> soff;
  const int WB = vol_warp_smem(g, key, &soff);
  if (g.staged) {
    o << "extern __shared__ __align__(128) unsigned char wt_smem[];\n";
    o << "unsigned char *wsm_ = wt_smem + (threadIdx.x >> 5) * " << WB << ";\n";
  }
  // per-tile bases: sources' o-point offsets, liveouts' lane column
  for (size_t ni = 0; ni < g.nodes.size(); ni++) {
    const VolNode &n = g.nodes[ni];
    if (n.source) {
      const std::string S = "a.src[" + std::to_string(n.src_index) + "]";
      const int esz = elem_bytes(key.src_dtypes.at(n.src_index));
      o << "const unsigned char *sb" << ni << " = (const unsigned char *)" << S << ".ptr;\n";
      // staged rows: the warp's slots, the segment's first column, the
      // lane's first value
      if (g.staged) {
      o << "unsigned char *ss" << ni << " = wsm_ + " << soff[ni] << ";\n";
      o << "const int seg" << ni << " = xb ? xs - " << g.xml << " : ((xs - " << g.xml << ") & ~" << 4 / esz - 1
        << ");\n";
      o << "const unsigned char *sl" << ni << " = ss" << ni << " + (lane * " << V << " + " << g.xml << " + (xs - "
        << g.xml << " - seg" << ni << ")) * " << esz << ";\n";
      }
      for (int j = -n.olo; j < g.To + n.ohi; j++) {
        std::string off;
        if (g.split == 0) off = n.planes == 1 ? "0" : "(wt_i64)" + o_index(std::to_string(j)) + " * " + S + ".plane";
        else off = "(wt_i64)" + o_index(std::to_string(j)) + " * " + S + ".pitch";
        o << "const wt_i64 so" << ni << "_" << j + n.olo << " = " << off << ";\n";
      }
    }
    if (n.dst_index >= 0) {
      const std::string D = "a.dst[" + std::to_string(n.dst_index) + "]";
      const int esz = elem_bytes(key.dst_dtypes.at(n.dst_index));
      o << "unsigned char *db" << ni << " = (unsigned char *)" << D << ".ptr + (wt_i64)xl0 * " << esz << ";\n";
      for (int j = 0; j < g.To; j++)
        o << "const wt_i64 do" << ni << "_" << j << " = (wt_i64)(o0 + " << j << ") * " << D
          << (g.split == 0 ? ".plane" : ".pitch") << ";\n";
    }
  }
  o << "const int nsteps = min(" << g.Ts << ", NS - s0) + " << g.pro << ";\n";
  auto loop = [&](bool safe) {
    o << "#pragma unroll 1\n";
    o << "for (int kb = 0; kb < nsteps; kb += " << g.U << ") {\n";
    for (int u = 0; u < g.U; u++) {
      o << "{ const int k = kb + " << u << ";\nif (k < nsteps) {\n";
      // shift the windows that do not rotate by renaming
      for (size_t ni = 0; ni < g.nodes.size(); ni++) {
        const VolNode &n = g.nodes[ni];
        if ((n.source && g.staged) || n.rotate || n.window < 2) continue;
        for (int a = n.window - 1; a >= 1; a--)
          for (int j = -n.olo; j < g.To + n.ohi; j++)
            for (int e = -n.xl; e < V + n.xr; e++)
              o << reg((int)ni, a, j, e) << " = " << reg((int)ni, a - 1, j, e) << ";\n";
      }
      step(u, safe);
      o << "}\n}\n";
    }
    o << "}\n";
  };
  o << "if (!xb) {\n";
  loop(false);
  o << "} else {\n";
  loop(true);
  o << "}\n";
  // no copy may land in shared memory after the warp has left
  if (g.staged) o << "WT_CP_ASYNC_WAIT(0);\n";
  return o.str();
}

}  // namespace

std::string emit_vol(const Pipeline &p, const VolGeom &g, const CodegenKey &key, const std::string &kname) {
  if (!g.ok) fail(WT_EINVAL, "internal: not a 3-D group: " + g.why);
  Emit e(p, g, key);
  const std::string body = e.run();
  std::ostringstream o;
  o << kDeviceSource;
  o << "static_assert(sizeof(WtArgs) == " << sizeof(KernelArgs) << ", \"WtArgs layout\");\n";
  // a register cap is applied through the launch bounds (resident blocks
  // per SM), which take precedence over the compiler's register option
  int min_blocks = 1;
  if (key.max_regs > 0) min_blocks = std::max(1, 65536 / (key.max_regs * 32 * key.nw));
  o << "extern \"C\" __global__ void __launch_bounds__(" << 32 * key.nw << ", " << min_blocks << ") " << kname
    << "(const __grid_constant__ WtArgs a) {\n";
  o << body;
  o << "}\n";
  return o.str();
}

}  // namespace wt

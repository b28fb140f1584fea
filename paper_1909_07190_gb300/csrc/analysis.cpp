// Halo, delay and window analysis of a fused group.
//
// Sec. 4 (OTPW): a group's overlapped tile extends, per stage n, by O^n
// points beyond the tile so that every tile is independent; here O^n is
// found by propagating the footprint boxes of Sec. 2.3 backwards from the
// liveouts (left/right/top/bot below).
//
// Sec. 5 (hybrid tiling) splits the warp tile along a split dimension into
// parallelogram tiles of warp width W_i parallel to the group's right
// hyperplane.  This implementation splits along y with W_y = 1: each
// parallelogram tile is one skewed row, processed in order.  The skew of
// node n is its delay e_n = max over producers (e_p + max(dymax, 0)): at
// step k it computes row y_top + k - e_n, so every right-hyperplane
// dependence is already available (no cyclic dependence between adjacent
// tiles).  A node keeps the last `window` rows it produced: the earlier
// parallelogram tiles its consumers still read.
//
// Kernel nodes: the group's sources (values read from memory), its stages,
// and, for every linear stencil whose weight matrix has rank one (Sobel,
// box, binomial), a synthetic row pass: S = sum_{i,j} u_j v_i P(x+i, y+j)
// becomes H = sum_i v_i P(x+i, y) and S = sum_j u_j H(x, y+j).  With
// clamp-to-edge at every read both forms are the same function (the clamps
// in x and y commute); only the rounding differs.
#include <algorithm>
#include <climits>
#include <cmath>
#include <map>
#include <numeric>
#include <tuple>

#include "wt_internal.hpp"

namespace wt {

int elem_bytes(int dtype) { return dtype == WT_F32 ? 4 : 2; }

int GroupGeom::gather_of(int id, int chan, int mode) const {
  for (size_t i = 0; i < nodes.size(); i++) {
    const Node &n = nodes[i];
    if (n.gather_mode == mode && n.id == id && n.src_chan == chan) return (int)i;
  }
  return -1;
}

int GroupGeom::node_of(int id, int chan) const {
  for (size_t i = 0; i < nodes.size(); i++) {
    const Node &n = nodes[i];
    if (n.synthetic || n.gather_mode || n.id != id) continue;
    if (!n.is_source) return (int)i;
    if (n.src_chan == chan) return (int)i;
  }
  return -1;
}

static int norm_chan(int chan, int src_channels) {
  if (src_channels == 1) return 0;
  return chan;  // -1 = tile channel, else fixed
}

namespace {

// Linear form of a postfix program: sum of coef * tap(node, dx, dy) + c.
struct Lin {
  bool ok = true;
  bool is_const = true;
  double c = 0;
  std::map<std::tuple<int, int, int>, double> t;
};

Lin lin_scale(Lin a, double s) {
  a.c *= s;
  for (auto &kv : a.t) kv.second *= s;
  return a;
}

Lin lin_add(const Lin &a, const Lin &b, double sb) {
  Lin r;
  r.ok = a.ok && b.ok;
  r.is_const = a.is_const && b.is_const;
  r.c = a.c + sb * b.c;
  r.t = a.t;
  for (auto &kv : b.t) r.t[kv.first] += sb * kv.second;
  return r;
}

Lin linear_form(const std::vector<KOp> &prog) {
  std::vector<Lin> st;
  Lin bad;
  bad.ok = false;
  for (const KOp &o : prog) {
    switch (o.op) {
      case WT_OP_CONST: {
        Lin l;
        l.c = o.value;
        st.push_back(l);
      } break;
      case WT_OP_TAP: {
        Lin l;
        l.is_const = false;
        l.t[std::make_tuple(o.node, o.dx, o.dy)] = 1.0;
        st.push_back(l);
      } break;
      case WT_OP_ADD: case WT_OP_SUB: {
        Lin b = st.back(); st.pop_back();
        Lin a = st.back(); st.pop_back();
        st.push_back(lin_add(a, b, o.op == WT_OP_ADD ? 1.0 : -1.0));
      } break;
      case WT_OP_MUL: {
        Lin b = st.back(); st.pop_back();
        Lin a = st.back(); st.pop_back();
        if (!a.ok || !b.ok) st.push_back(bad);
        else if (a.is_const) st.push_back(lin_scale(b, a.c));
        else if (b.is_const) st.push_back(lin_scale(a, b.c));
        else st.push_back(bad);
      } break;
      case WT_OP_DIV: {
        Lin b = st.back(); st.pop_back();
        Lin a = st.back(); st.pop_back();
        if (!a.ok || !b.ok || !b.is_const || b.c == 0) st.push_back(bad);
        else st.push_back(lin_scale(a, 1.0 / b.c));
      } break;
      case WT_OP_NEG: st.back() = lin_scale(st.back(), -1.0); break;
      case WT_OP_MIN: case WT_OP_MAX:
        st.pop_back();
        st.back() = bad;
        break;
      case WT_OP_XPAR: case WT_OP_YPAR: case WT_OP_CHAN: st.push_back(bad); break;
      default: st.back() = bad;  // abs, sqrt: not linear in the taps
    }
  }
  return st.empty() ? bad : st.back();
}

void push_const(std::vector<KOp> &p, double v) {
  KOp o;
  o.op = WT_OP_CONST;
  o.value = (float)v;
  p.push_back(o);
}

void push_op(std::vector<KOp> &p, int op) {
  KOp o;
  o.op = op;
  p.push_back(o);
}

// sum_k w_k tap(node, dx_k, dy_k) as a postfix program (zeros skipped).
std::vector<KOp> weighted_sum(int node, const std::vector<std::tuple<int, int, double>> &terms) {
  // a positive term first, so that weights -1 become subtractions and
  // weights 1 additions (no multiplies)
  std::vector<std::tuple<int, int, double>> ts;
  for (auto &t : terms)
    if (std::get<2>(t) > 0) ts.push_back(t);
  for (auto &t : terms)
    if (std::get<2>(t) < 0) ts.push_back(t);
  std::vector<KOp> p;
  bool first = true;
  for (auto &t : ts) {
    double w = std::get<2>(t);
    KOp tap;
    tap.op = WT_OP_TAP;
    tap.node = node;
    tap.dx = std::get<0>(t);
    tap.dy = std::get<1>(t);
    p.push_back(tap);
    if (!first && w == -1.0) {
      push_op(p, WT_OP_SUB);
      continue;
    }
    if (w != 1.0) {
      push_const(p, w);
      push_op(p, WT_OP_MUL);
    }
    if (!first) push_op(p, WT_OP_ADD);
    first = false;
  }
  if (first) push_const(p, 0.0);
  return p;
}

// Splits node `ni` if its program is a rank-one linear stencil of one
// producer; returns the index of the new synthetic row-pass node or -1.
int try_split(GroupGeom &g, int ni) {
  Lin l = linear_form(g.nodes[ni].prog);
  if (!l.ok || l.is_const || l.t.empty()) return -1;
  int prod = std::get<0>(l.t.begin()->first);
  // taps of another level (gather sources) address the producer's own grid:
  // a row pass at this level would not separate them
  if (g.nodes[prod].gather_mode) return -1;
  int x0 = INT_MAX, x1 = INT_MIN, y0 = INT_MAX, y1 = INT_MIN, nnz = 0;
  double wmax = 0;
  for (auto &kv : l.t) {
    if (std::get<0>(kv.first) != prod) return -1;
    if (kv.second == 0) continue;
    nnz++;
    x0 = std::min(x0, std::get<1>(kv.first));
    x1 = std::max(x1, std::get<1>(kv.first));
    y0 = std::min(y0, std::get<2>(kv.first));
    y1 = std::max(y1, std::get<2>(kv.first));
    wmax = std::max(wmax, std::fabs(kv.second));
  }
  if (nnz == 0 || x1 == x0 || y1 == y0) return -1;  // already one-dimensional
  const int nx = x1 - x0 + 1, ny = y1 - y0 + 1;
  std::vector<double> W((size_t)nx * ny, 0.0);
  int pi = 0, pj = 0;
  double pv = 0;
  for (auto &kv : l.t) {
    int i = std::get<1>(kv.first) - x0, j = std::get<2>(kv.first) - y0;
    W[(size_t)j * nx + i] = kv.second;
    if (std::fabs(kv.second) > std::fabs(pv)) {
      pv = kv.second;
      pi = i;
      pj = j;
    }
  }
  std::vector<double> v(nx), u(ny);
  for (int i = 0; i < nx; i++) v[i] = W[(size_t)pj * nx + i];
  for (int j = 0; j < ny; j++) u[j] = W[(size_t)j * nx + pi] / pv;
  int nv = 0, nu = 0;
  for (int i = 0; i < nx; i++) nv += v[i] != 0;
  for (int j = 0; j < ny; j++) nu += u[j] != 0;
  for (int j = 0; j < ny; j++)
    for (int i = 0; i < nx; i++)
      if (std::fabs(W[(size_t)j * nx + i] - u[j] * v[i]) > 1e-9 * wmax) return -1;  // rank > 1
  if (nv + nu >= nnz) return -1;  // no saving
  // the row pass gets the smallest weights that are whole multiples of its
  // smallest nonzero weight (integer taps: additions and subtractions), the
  // column pass the scale
  double vmin = INFINITY;
  for (int i = 0; i < nx; i++)
    if (v[i] != 0) vmin = std::min(vmin, std::fabs(v[i]));
  // mostly positive row weights (their sign moves to the column pass)
  double vsum = 0;
  for (int i = 0; i < nx; i++) vsum += v[i];
  if (vsum < 0) vmin = -vmin;
  for (int i = 0; i < nx; i++) v[i] /= vmin;
  for (int j = 0; j < ny; j++) u[j] *= vmin;
  Node h;
  h.synthetic = true;
  h.id = g.nodes[ni].id;
  h.channels = g.nodes[ni].channels;
  std::vector<std::tuple<int, int, double>> ht, vt;
  for (int i = 0; i < nx; i++) ht.emplace_back(x0 + i, 0, v[i]);
  h.prog = weighted_sum(prod, ht);
  const int hi = (int)g.nodes.size();
  g.nodes.push_back(h);
  for (int j = 0; j < ny; j++) vt.emplace_back(0, y0 + j, u[j]);
  std::vector<KOp> np = weighted_sum(hi, vt);
  if (l.c != 0) {
    push_const(np, l.c);
    push_op(np, WT_OP_ADD);
  }
  g.nodes[ni].prog = np;
  return hi;
}

}  // namespace

GroupGeom analyze_group(const Pipeline &p, const std::vector<int> &stages, int vec,
                        float frac_reg, int dtype_bytes, bool split_separable) {
  GroupGeom g;
  g.stages = stages;
  std::vector<char> in_group(p.stages.size(), 0);
  for (int s : stages) in_group[s] = 1;
  g.level = p.stages[stages[0]].level;
  g.channels = 1;
  for (int s : stages) {
    g.channels = std::max(g.channels, p.stages[s].channels);
    if (p.stages[s].level != g.level) {
      g.fusable = false;
      g.why_not = "group spans several levels";
    }
    if (p.stages[s].has_z) {
      // plane-offset taps: the 3-D group kernel (vol.cpp) or per stage
      g.fusable = false;
      g.why_not = "plane-offset taps (3-D group)";
      return g;
    }
  }
  auto pchan = [&](int pid) { return pid >= 0 ? p.stages[pid].channels : p.in_channels[-pid - 1]; };
  // Sources: distinct (producer outside the group, channel spec); producers
  // outside the group read through a down/up-sampling tap are gather
  // sources (added after the stages).
  std::vector<Node> gathers;
  for (int s : stages) {
    for (const Edge &e : p.stages[s].edges) {
      bool inside = e.producer >= 0 && in_group[e.producer];
      int pc = pchan(e.producer);
      if (e.mode != WT_TAP_SAME) {
        if (inside) {
          g.fusable = false;
          g.why_not = "group contains a down/up-sampling tap of a stage in the group";
          continue;
        }
        for (int c : e.chans) {
          int cc = norm_chan(c, pc);
          bool dup = false;
          for (const Node &q : gathers) dup |= q.id == e.producer && q.src_chan == cc && q.gather_mode == e.mode;
          if (dup) continue;
          Node n;
          n.id = e.producer;
          n.src_chan = cc;
          n.channels = pc;
          n.gather_mode = e.mode;
          gathers.push_back(n);
        }
        continue;
      }
      if (inside) {
        for (int c : e.chans) {
          int cc = norm_chan(c, pc);
          if (cc >= 0 && pc > 1) {
            g.fusable = false;
            g.why_not = "fixed-channel tap of a multi-channel stage inside the group";
          }
        }
        continue;
      }
      for (int c : e.chans) {
        int cc = norm_chan(c, pc);
        if (g.node_of(e.producer, cc) >= 0) continue;
        Node n;
        n.id = e.producer;
        n.src_chan = cc;
        n.is_source = true;
        n.channels = pc;
        g.nodes.push_back(n);
      }
    }
  }
  const int n_src = (int)g.nodes.size();
  for (int i = 0; i < n_src; i++) g.order.push_back(i);
  for (int s : stages) {
    Node n;
    n.id = s;
    n.channels = p.stages[s].channels;
    bool out = p.is_output[s];
    for (int c : p.consumers[s])
      if (!in_group[c]) out = true;
    n.is_liveout = out;
    g.nodes.push_back(n);
    if (out) g.liveouts.push_back(s);
  }
  for (const Node &n : gathers) g.nodes.push_back(n);
  g.n_gather = (int)gathers.size();
  // Programs over kernel nodes.
  for (int s : stages) {
    const int ni = g.node_of(s, -1);
    const Stage &S = p.stages[s];
    for (const Op &op : S.ops) {
      KOp k;
      k.op = op.op;
      k.value = op.value;
      if (op.op == WT_OP_TAP) {
        int pid = S.inputs[op.slot];
        bool inside = pid >= 0 && in_group[pid];
        if (op.mode != WT_TAP_SAME && !inside)
          k.node = g.gather_of(pid, norm_chan(op.chan, pchan(pid)), op.mode);
        else
          k.node = inside ? g.node_of(pid, -1) : g.node_of(pid, norm_chan(op.chan, pchan(pid)));
        k.dx = op.dx;
        k.dy = op.dy;
        if (k.node < 0) fail(WT_EINVAL, "internal: tap node not found");
      }
      g.nodes[ni].prog.push_back(k);
    }
  }
  for (int s : stages) {
    const int ni = g.node_of(s, -1);
    if (split_separable && g.fusable) {
      int hi = try_split(g, ni);
      if (hi >= 0) {
        g.order.push_back(hi);
        g.n_split++;
      }
    }
    g.order.push_back(ni);
  }
  // Edges (consumer node, producer node) with footprint boxes.
  std::map<std::pair<int, int>, NodeEdge> em;
  for (int ni : g.order) {
    for (const KOp &k : g.nodes[ni].prog) {
      if (k.op != WT_OP_TAP) continue;
      if (g.nodes[k.node].gather_mode) continue;  // no rows kept, no halo
      auto key = std::make_pair(ni, k.node);
      auto it = em.find(key);
      if (it == em.end()) {
        em[key] = NodeEdge{ni, k.node, k.dx, k.dx, k.dy, k.dy};
      } else {
        NodeEdge &e = it->second;
        e.dxmin = std::min(e.dxmin, k.dx);
        e.dxmax = std::max(e.dxmax, k.dx);
        e.dymin = std::min(e.dymin, k.dy);
        e.dymax = std::max(e.dymax, k.dy);
      }
    }
  }
  for (auto &kv : em) g.edges.push_back(kv.second);
  std::vector<int> pos(g.nodes.size(), 0);
  for (size_t i = 0; i < g.order.size(); i++) pos[g.order[i]] = (int)i;
  // Backward halo propagation (reverse evaluation order).
  const int UNSET = INT_MIN / 4;
  for (Node &n : g.nodes) n.top = n.bot = n.left = n.right = UNSET;
  for (Node &n : g.nodes)
    if (!n.is_source && !n.synthetic && n.is_liveout) n.top = n.bot = n.left = n.right = 0;
  for (int oi = (int)g.order.size() - 1; oi >= n_src; oi--) {
    const int ci = g.order[oi];
    Node &c = g.nodes[ci];
    if (c.top == UNSET) c.top = c.bot = c.left = c.right = 0;  // dead node
    for (const NodeEdge &e : g.edges) {
      if (e.c != ci) continue;
      Node &q = g.nodes[e.p];
      q.left = std::max(q.left, std::max(0, c.left - e.dxmin));
      q.right = std::max(q.right, std::max(0, c.right + e.dxmax));
      q.top = std::max(q.top, std::max(0, c.top - e.dymin));
      q.bot = std::max(q.bot, std::max(0, c.bot + e.dymax));
      q.xl = std::max(q.xl, std::max(0, -e.dxmin));
      q.xr = std::max(q.xr, std::max(0, e.dxmax));
    }
  }
  for (Node &n : g.nodes)
    if (n.top == UNSET) n.top = n.bot = n.left = n.right = 0;
  // Delays (forward) and windows.
  for (int oi = 0; oi < (int)g.order.size(); oi++) {
    const int ci = g.order[oi];
    Node &c = g.nodes[ci];
    if (c.is_source) {
      c.delay = 0;
      continue;
    }
    int d = INT_MIN;
    // max(dymax, 0): with clamp-to-edge a tap above the consumer's row can
    // resolve to the producer's row 0 at the top border, so the producer
    // must have reached the consumer's own row as well.
    for (const NodeEdge &e : g.edges)
      if (e.c == ci) {
        if (pos[e.p] >= oi) fail(WT_EINVAL, "internal: node order");
        d = std::max(d, g.nodes[e.p].delay + std::max(e.dymax, 0));
      }
    c.delay = d == INT_MIN ? 0 : d;
  }
  for (Node &n : g.nodes) n.window = 1;
  for (const NodeEdge &e : g.edges) {
    Node &q = g.nodes[e.p];
    // keep rows down to the consumer's own row too (min(dymin, 0)): a tap
    // below it can resolve to the last image row at the bottom border
    q.window = std::max(q.window, g.nodes[e.c].delay - q.delay - std::min(e.dymin, 0) + 1);
  }
  g.halo_l = g.halo_r = g.halo_t = g.halo_b = 0;
  g.max_delay = 0;
  for (const Node &n : g.nodes) {
    g.halo_l = std::max(g.halo_l, n.left);
    g.halo_r = std::max(g.halo_r, n.right);
    g.halo_t = std::max(g.halo_t, n.top);
    g.halo_b = std::max(g.halo_b, n.bot);
    g.max_delay = std::max(g.max_delay, n.delay);
  }
  // Hybrid placement: keep frac_reg of the window bytes in registers,
  // smallest windows first; the rest lives in the warp's shared memory.
  std::vector<int> order(g.nodes.size());
  std::iota(order.begin(), order.end(), 0);
  auto wbytes = [&](int i) {
    const Node &n = g.nodes[i];
    if (n.gather_mode) return 0L;
    return (long)n.window * (vec + n.xl + n.xr) * 4;
  };
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return wbytes(a) < wbytes(b); });
  long total = 0;
  for (int i : order) total += wbytes(i);
  long budget = (long)(frac_reg * (double)total + 0.5);
  long acc = 0;
  for (int i : order) {
    Node &n = g.nodes[i];
    if (n.gather_mode) {
      n.in_smem = false;
      continue;
    }
    if (acc + wbytes(i) <= budget) {
      n.in_smem = false;
      acc += wbytes(i);
    } else {
      n.in_smem = true;
    }
  }
  (void)dtype_bytes;
  // Unroll factor: the lcm of the register windows when it is small,
  // otherwise the largest window, with smaller windows padded up to a
  // divisor of it (a padded window only keeps extra older rows) so that
  // every register window rotates by renaming; windows that cannot be
  // padded shift by register moves.
  long L = 1, wmax = 1;
  for (const Node &n : g.nodes)
    if (!n.in_smem) {
      L = std::lcm(L, (long)n.window);
      wmax = std::max(wmax, (long)n.window);
    }
  long U = L <= 8 ? L : wmax;
  for (Node &n : g.nodes) {
    if (n.in_smem) continue;
    if (U % n.window == 0) {
      n.rotate = true;
      continue;
    }
    long d = n.window;
    while (d <= U && U % d != 0) d++;
    if (d <= U && d <= n.window + 4) {
      n.window = (int)d;
      n.rotate = true;
    } else {
      n.rotate = false;
    }
  }
  for (const Node &n : g.nodes)
    for (const KOp &k : n.prog)
      if (k.op == WT_OP_YPAR) g.uses_ypar = true;
  // an even unroll keeps each unrolled step's row parity fixed (row-parity
  // selects then fold); register windows still divide it
  if (g.uses_ypar && U % 2) U *= 2;
  g.unroll = (int)U;
  g.max_src_window = 1;
  for (int i = 0; i < n_src; i++) g.max_src_window = std::max(g.max_src_window, g.nodes[i].window);
  if (n_src > kMaxSrc) {
    g.fusable = false;
    g.why_not = "more than " + std::to_string(kMaxSrc) + " staged sources";
  }
  if (n_src + g.n_gather > kMaxAllSrc) {
    g.fusable = false;
    g.why_not = "more than " + std::to_string(kMaxAllSrc) + " sources";
  }
  if ((int)g.liveouts.size() > kMaxDst) {
    g.fusable = false;
    g.why_not = "more than " + std::to_string(kMaxDst) + " liveouts";
  }
  return g;
}

}  // namespace wt

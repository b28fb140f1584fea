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
// stage n is its delay e_n = max over producers (e_p + dymax): at step k it
// computes row y_top + k - e_n, so every right-hyperplane dependence is
// already available (no cyclic dependence between adjacent tiles).  A stage
// keeps the last `window` rows it produced, which is exactly the set of its
// earlier parallelogram tiles its consumers still read.
#include <algorithm>
#include <climits>
#include <numeric>

#include "wt_internal.hpp"

namespace wt {

int elem_bytes(int dtype) { return dtype == WT_F32 ? 4 : 2; }

int GroupGeom::node_of(int id, int chan) const {
  for (size_t i = 0; i < nodes.size(); i++) {
    const Node &n = nodes[i];
    if (n.id != id) continue;
    if (!n.is_source) return (int)i;
    if (n.src_chan == chan) return (int)i;
  }
  return -1;
}

static int norm_chan(int chan, int src_channels) {
  if (src_channels == 1) return 0;
  return chan;  // -1 = tile channel, else fixed
}

GroupGeom analyze_group(const Pipeline &p, const std::vector<int> &stages, int vec,
                        float frac_reg, int dtype_bytes) {
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
  }
  // Sources: distinct (producer outside the group, channel spec).
  for (int s : stages) {
    for (const Edge &e : p.stages[s].edges) {
      bool inside = e.producer >= 0 && in_group[e.producer];
      if (e.mode != WT_TAP_SAME) {
        g.fusable = false;
        g.why_not = "group contains a down/up-sampling tap";
      }
      int pc = e.producer >= 0 ? p.stages[e.producer].channels : p.in_channels[-e.producer - 1];
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
  int n_src = (int)g.nodes.size();
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
  // Backward halo propagation (reverse topological order).
  const int UNSET = INT_MIN / 4;
  for (Node &n : g.nodes) n.top = n.bot = n.left = n.right = UNSET;
  for (Node &n : g.nodes)
    if (!n.is_source && n.is_liveout) n.top = n.bot = n.left = n.right = 0;
  for (int i = (int)stages.size() - 1; i >= 0; i--) {
    int s = stages[i];
    Node &c = g.nodes[g.node_of(s, -1)];
    if (c.top == UNSET) c.top = c.bot = c.left = c.right = 0;  // dead stage
    for (const Edge &e : p.stages[s].edges) {
      int pc = e.producer >= 0 ? p.stages[e.producer].channels : p.in_channels[-e.producer - 1];
      bool inside = e.producer >= 0 && in_group[e.producer];
      std::vector<int> ids;
      if (inside) ids.push_back(g.node_of(e.producer, -1));
      else
        for (int ch : e.chans) ids.push_back(g.node_of(e.producer, norm_chan(ch, pc)));
      for (int id : ids) {
        Node &q = g.nodes[id];
        q.left = std::max(q.left, std::max(0, c.left - e.dxmin));
        q.right = std::max(q.right, std::max(0, c.right + e.dxmax));
        q.top = std::max(q.top, std::max(0, c.top - e.dymin));
        q.bot = std::max(q.bot, std::max(0, c.bot + e.dymax));
        q.xl = std::max(q.xl, std::max(0, -e.dxmin));
        q.xr = std::max(q.xr, std::max(0, e.dxmax));
      }
    }
  }
  for (Node &n : g.nodes)
    if (n.top == UNSET) n.top = n.bot = n.left = n.right = 0;
  // Delays (forward) and windows.
  for (int i = 0; i < n_src; i++) g.nodes[i].delay = 0;
  for (int s : stages) {
    Node &c = g.nodes[g.node_of(s, -1)];
    int d = INT_MIN;
    for (const Edge &e : p.stages[s].edges) {
      int pc = e.producer >= 0 ? p.stages[e.producer].channels : p.in_channels[-e.producer - 1];
      bool inside = e.producer >= 0 && in_group[e.producer];
      std::vector<int> ids;
      if (inside) ids.push_back(g.node_of(e.producer, -1));
      else
        for (int ch : e.chans) ids.push_back(g.node_of(e.producer, norm_chan(ch, pc)));
      // max(dymax, 0): with clamp-to-edge a tap above the consumer's row can
      // resolve to the producer's row 0 at the top border, so the producer
      // must have reached the consumer's own row as well.
      for (int id : ids) d = std::max(d, g.nodes[id].delay + std::max(e.dymax, 0));
    }
    c.delay = d == INT_MIN ? 0 : d;
  }
  for (Node &n : g.nodes) n.window = 1;
  for (int s : stages) {
    const Node &c = g.nodes[g.node_of(s, -1)];
    for (const Edge &e : p.stages[s].edges) {
      int pc = e.producer >= 0 ? p.stages[e.producer].channels : p.in_channels[-e.producer - 1];
      bool inside = e.producer >= 0 && in_group[e.producer];
      std::vector<int> ids;
      if (inside) ids.push_back(g.node_of(e.producer, -1));
      else
        for (int ch : e.chans) ids.push_back(g.node_of(e.producer, norm_chan(ch, pc)));
      for (int id : ids) {
        Node &q = g.nodes[id];
        // keep rows down to the consumer's own row too (min(dymin, 0)): a
        // tap below it can resolve to the last image row at the bottom border
        q.window = std::max(q.window, c.delay - q.delay - std::min(e.dymin, 0) + 1);
      }
    }
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
    return (long)n.window * (vec + n.xl + n.xr) * 4;
  };
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return wbytes(a) < wbytes(b); });
  long total = 0;
  for (int i : order) total += wbytes(i);
  long budget = (long)(frac_reg * (double)total + 0.5);
  long acc = 0;
  for (int i : order) {
    Node &n = g.nodes[i];
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
  g.unroll = (int)U;
  g.max_src_window = 1;
  for (int i = 0; i < n_src; i++) g.max_src_window = std::max(g.max_src_window, g.nodes[i].window);
  if (n_src > kMaxSrc) {
    g.fusable = false;
    g.why_not = "more than " + std::to_string(kMaxSrc) + " sources";
  }
  if ((int)g.liveouts.size() > kMaxDst) {
    g.fusable = false;
    g.why_not = "more than " + std::to_string(kMaxDst) + " liveouts";
  }
  return g;
}

}  // namespace wt

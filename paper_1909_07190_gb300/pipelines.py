"""Stage DAGs of the benchmark pipelines, as plain data.

A pipeline is the program the library compiles: a DAG of stages, each a
per-pixel function of producer values at constant offsets (Jangda & Guha,
PACT'20, Sec. 2.2 Fig. 2 and Sec. 2.3).  Each stage is a postfix program over
taps ``("tap", slot, dx, dy, chan, mode)``; ``mode`` is "same" (P(x+dx, y+dy)),
"down2" (P(2x+dx, 2y+dy)) or "up2" (P(floor(x/2)+dx, floor(y/2)+dy)) (also
"down4"/"up4" and "down8"/"up8": scale 4 and 8), the
constant dependence vectors that alignment and scaling produce (Sec. 5).

Format::

    {"name": str,
     "inputs": [channels of pipeline input j, ...],
     "stages": [{"name", "channels", "inputs": [producer ids], "ops": [...]}],
     "outputs": [stage ids]}

Producer ids: stage index >= 0, or -(j+1) for pipeline input j.
"""
from __future__ import annotations

from typing import List, Sequence


class E:
    """Postfix expression under construction (operator overloading)."""

    __slots__ = ("ops",)

    def __init__(self, ops):
        self.ops = list(ops)

    @staticmethod
    def of(v) -> "E":
        return v if isinstance(v, E) else E([("const", float(v))])

    def _bin(self, other, op, swap=False):
        a, b = (E.of(other), self) if swap else (self, E.of(other))
        return E(a.ops + b.ops + [(op,)])

    def __add__(self, o): return self._bin(o, "add")
    def __radd__(self, o): return self._bin(o, "add", True)
    def __sub__(self, o): return self._bin(o, "sub")
    def __rsub__(self, o): return self._bin(o, "sub", True)
    def __mul__(self, o): return self._bin(o, "mul")
    def __rmul__(self, o): return self._bin(o, "mul", True)
    def __truediv__(self, o): return self._bin(o, "div")
    def __rtruediv__(self, o): return self._bin(o, "div", True)
    def __neg__(self): return E(self.ops + [("neg",)])


def emin(a, b) -> E: return E(E.of(a).ops + E.of(b).ops + [("min",)])
def emax(a, b) -> E: return E(E.of(a).ops + E.of(b).ops + [("max",)])
def eabs(a) -> E: return E(E.of(a).ops + [("abs",)])
def esqrt(a) -> E: return E(E.of(a).ops + [("sqrt",)])


XPAR = E([("xpar",)])
YPAR = E([("ypar",)])
CHAN = E([("chan",)])  # the output point's channel index


def ref(producer: int, dx: int = 0, dy: int = 0, chan: int = -1, mode: str = "same") -> E:
    """A read of `producer` (stage id, or input(j)) at a constant offset."""
    return E([("ref", int(producer), int(dx), int(dy), int(chan), mode)])


def refz(producer: int, dx: int = 0, dy: int = 0, dz: int = 0) -> E:
    """A 3-D read: `producer` at (x + dx, y + dy) of plane z + dz, where z is
    the output point's plane (a D x H x W volume is an image of D planes);
    every coordinate is clamped to the volume (App. A's 3-D groups)."""
    return E([("refz", int(producer), int(dx), int(dy), int(dz))])


def input_id(j: int) -> int:
    return -(j + 1)


class Builder:
    def __init__(self, name: str, input_channels: Sequence[int]):
        self.p = {"name": name, "inputs": list(input_channels), "stages": [], "outputs": []}

    def stage(self, name: str, expr: E, channels: int = 1) -> int:
        producers: List[int] = []
        ops = []
        for t in E.of(expr).ops:
            if t[0] == "ref":
                _, pid, dx, dy, chan, mode = t
                if pid not in producers:
                    producers.append(pid)
                ops.append(("tap", producers.index(pid), dx, dy, chan, mode))
            elif t[0] == "refz":
                _, pid, dx, dy, dz = t
                if pid not in producers:
                    producers.append(pid)
                ops.append(("tapz", producers.index(pid), dx, dy, dz))
            else:
                ops.append(t)
        self.p["stages"].append({"name": name, "channels": int(channels),
                                 "inputs": producers, "ops": ops})
        return len(self.p["stages"]) - 1

    def output(self, *sids: int):
        self.p["outputs"].extend(sids)

    def build(self) -> dict:
        return self.p


def linear(producer: int, weights, scale: float = 1.0, mode: str = "same",
           chan: int = -1) -> E:
    """sum_{j,i} weights[j][i] * P(x + i - rx, y + j - ry) * scale, written row by
    row (rx, ry = half the kernel width/height); zero weights are skipped."""
    rows = len(weights)
    cols = len(weights[0])
    ry, rx = rows // 2, cols // 2
    total = None
    for j in range(rows):
        row = None
        for i in range(cols):
            w = float(weights[j][i])
            if w == 0.0:
                continue
            t = ref(producer, i - rx, j - ry, chan, mode)
            t = t if w == 1.0 else w * t
            row = t if row is None else row + t
        if row is not None:
            total = row if total is None else total + row
    if total is None:
        total = E.of(0.0)
    return total if scale == 1.0 else total * scale


BINOMIAL5 = [1.0 / 16, 4.0 / 16, 6.0 / 16, 4.0 / 16, 1.0 / 16]
SOBEL_X = [[-1, 0, 1], [-2, 0, 2], [-1, 0, 1]]
SOBEL_Y = [[-1, -2, -1], [0, 0, 0], [1, 2, 1]]
BOX3 = [[1, 1, 1], [1, 1, 1], [1, 1, 1]]


def sharpen() -> dict:
    """3-stage sharpen: horizontal then vertical 5-tap binomial blur,
    out = clamp(in + 1.5 (in - blur), 0, 1)."""
    b = Builder("sharpen", [1])
    inp = input_id(0)
    bx = b.stage("bx", linear(inp, [BINOMIAL5]))
    by = b.stage("by", linear(bx, [[w] for w in BINOMIAL5]))
    v = ref(inp)
    out = b.stage("sharpen", emin(emax(v + 1.5 * (v - ref(by)), 0.0), 1.0))
    b.output(out)
    return b.build()


def harris(normalized: bool = True, k: float = 0.04) -> dict:
    """11-stage corner response: Sobel Ix, Iy; Ixx, Iyy, Ixy; 3x3 box of each;
    det, trace, R = det - k trace^2.  normalized: Sobel x 1/8, box x 1/9."""
    b = Builder("harris" if normalized else "harris_raw", [1])
    inp = input_id(0)
    sx = 1.0 / 8 if normalized else 1.0
    sb = 1.0 / 9 if normalized else 1.0
    ix = b.stage("Ix", linear(inp, SOBEL_X, sx))
    iy = b.stage("Iy", linear(inp, SOBEL_Y, sx))
    ixx = b.stage("Ixx", ref(ix) * ref(ix))
    iyy = b.stage("Iyy", ref(iy) * ref(iy))
    ixy = b.stage("Ixy", ref(ix) * ref(iy))
    sxx = b.stage("Sxx", linear(ixx, BOX3, sb))
    syy = b.stage("Syy", linear(iyy, BOX3, sb))
    sxy = b.stage("Sxy", linear(ixy, BOX3, sb))
    det = b.stage("det", ref(sxx) * ref(syy) - ref(sxy) * ref(sxy))
    tr = b.stage("trace", ref(sxx) + ref(syy))
    r = b.stage("R", ref(det) - k * (ref(tr) * ref(tr)))
    b.output(r)
    return b.build()


def _down(p: int) -> E:
    return linear(p, [[bj * bi for bi in BINOMIAL5] for bj in BINOMIAL5], mode="down2")


def _up(p: int) -> E:
    """Half-pixel bilinear upsample: along each axis even 2i -> 0.75 P(i) +
    0.25 P(i-1), odd 2i+1 -> 0.75 P(i) + 0.25 P(i+1); (1-par)/par select."""
    def row(dy):
        left = ref(p, -1, dy, mode="up2")
        right = ref(p, 1, dy, mode="up2")
        return 0.75 * ref(p, 0, dy, mode="up2") + 0.25 * ((1.0 - XPAR) * left + XPAR * right)
    return 0.75 * row(0) + 0.25 * ((1.0 - YPAR) * row(-1) + YPAR * row(1))


def blend(levels: int = 6, channels: int = 3) -> dict:
    """Laplacian-pyramid blend of A and B under mask M (36 stages at 6 levels):
    Gaussian levels by 5x5 binomial downsample, Laplacian L_k = G_k -
    up(G_{k+1}) (L_top = G_top), BL_k = M_k L^A_k + (1 - M_k) L^B_k,
    R_top = BL_top, R_k = BL_k + up(R_{k+1}); output R_0."""
    b = Builder("blend", [channels, channels, 1])
    ga, gb, gm = [input_id(0)], [input_id(1)], [input_id(2)]
    # Stage order: the three Gaussian pyramids level by level, then the
    # coarsest blend, then per level from coarse to fine L^A, L^B, BL, R, so
    # that the stages of one level are contiguous (blend_groups()).
    for k in range(1, levels):
        ga.append(b.stage("GA%d" % k, _down(ga[-1]), channels))
        gb.append(b.stage("GB%d" % k, _down(gb[-1]), channels))
        gm.append(b.stage("GM%d" % k, _down(gm[-1]), 1))
    top = levels - 1
    m = ref(gm[top], chan=0)
    r = b.stage("BL%d" % top, m * ref(ga[top]) + (1.0 - m) * ref(gb[top]), channels)
    for k in range(levels - 2, -1, -1):
        la = b.stage("LA%d" % k, ref(ga[k]) - _up(ga[k + 1]), channels)
        lb = b.stage("LB%d" % k, ref(gb[k]) - _up(gb[k + 1]), channels)
        m = ref(gm[k], chan=0)
        bl = b.stage("BL%d" % k, m * ref(la) + (1.0 - m) * ref(lb), channels)
        r = b.stage("R%d" % k, ref(bl) + _up(r), channels)
    b.output(r)
    return b.build()


def blend_groups(levels: int = 6) -> list:
    """Group index per stage of blend(levels): one group per Gaussian level
    (its three down-sampling stages; the coarsest with its blend stage),
    then one group per finer level (L^A, L^B, BL, R).  Taps of the other
    level read memory (gather sources)."""
    g = []
    for k in range(1, levels):
        g += [k - 1] * 3
    g.append(levels - 2)  # BL at the coarsest level joins its Gaussian group
    nxt = levels - 1
    for _ in range(levels - 1):
        g += [nxt] * 4
        nxt += 1
    return g


def blend_schedule(levels: int = 6) -> tuple:
    """(groups, params) of the blend's default schedule (measured fastest on
    a GB300 at 8192x8192x3 BF16):
      - Gaussian levels 1 and 2: per-stage streaming down-sampling kernels
        (a fused group of gathers has nothing to keep on chip, and its
        one-channel mask stage would be computed once per tile channel);
        output rows per warp 14 and 8;
      - Gaussian levels 3 and 4 (then 5 and 6, ...): one group spanning the
        two levels, run as two-level cascade launches (each image's level-3
        reduce written and reduced again on chip), 4 level-4 rows per warp;
        a level left without a partner runs per stage;
      - the coarsest level with its blend, then one fused group per finer
        level: short warp tiles where the level is small; at level 1, 14
        rows, at level 0, 48 rows, both with 4-row staging chunks and at most
        96 registers (80 used, 25 warps per SM: the level-0 group is bound by
        memory latency; taller level-0 tiles re-read fewer gather rows)."""
    plain = 4  # WT_FLAG_PLAIN
    groups, params = [], []
    g = 0
    k = 1
    while k <= levels - 2:
        if k <= 2 or k + 1 > levels - 2:
            groups += [g] * 3
            params.append(dict(flags=plain, tile_h=[14, 8][k - 1] if k <= 2 else 4))
            k += 1
        else:
            groups += [g] * 6
            params.append(dict(tile_h=4))
            k += 2
        g += 1
    groups += [g] * 4  # the coarsest level's reduces and its blend
    g += 1
    for _ in range(levels - 1):
        groups += [g] * 4
        g += 1
    for lv in range(levels - 1, -1, -1):
        if lv >= 2:
            params.append(dict(tile_h=8))
        else:
            params.append(dict(tile_h=14 if lv == 1 else 48, chunk_rows=4, max_regs=96))
    return groups, params


def blur3(channels: int = 1) -> dict:
    """The paper's running example (Fig. 2): blurx = 3-tap mean along x,
    blury = 3-tap mean of blurx along y (per plane; the motivating timing
    of Sec. 3 uses 3 planes)."""
    b = Builder("blur", [channels])
    inp = input_id(0)
    bx = b.stage("blurx", (ref(inp, -1, 0) + ref(inp) + ref(inp, 1, 0)) / 3.0, channels)
    by = b.stage("blury", (ref(bx, 0, -1) + ref(bx) + ref(bx, 0, 1)) / 3.0, channels)
    b.output(by)
    return b.build()


def _grid_stages(b: "Builder", inp: int, bins: int, levels: int) -> int:
    """Stages of a bilateral grid's construction; returns the blurred grid.

    Channel z < bins of a grid cell holds the sum over the cell's pixels of
    the tent weight max(0, 1 - |I (bins - 1) - z|), channel bins + z the same
    weights times I (intensity I in [0, 1]).  G1 (level 1) splats every
    pixel of a 2x2 block and sums them: the histogram step, a reduction;
    G2 .. G_levels sum 2x2 blocks of the level below; B blurs the grid with
    a 3x3 binomial in x and y."""
    nb = bins
    is_v = emin(emax(CHAN - float(nb - 1), 0.0), 1.0)  # 1 on the value channels
    z = CHAN - float(nb) * is_v                           # the channel's bin

    def splat(t):
        w = emax(1.0 - eabs(t * float(nb - 1) - z), 0.0)
        return w * (1.0 + is_v * (t - 1.0))

    taps = [ref(inp, i, j, mode="down2") for j in (0, 1) for i in (0, 1)]
    g = b.stage("G1", splat(taps[0]) + splat(taps[1]) + splat(taps[2]) + splat(taps[3]), 2 * nb)
    for k in range(2, levels + 1):
        box = ref(g, 0, 0, mode="down2") + ref(g, 1, 0, mode="down2") + ref(g, 0, 1, mode="down2") \
            + ref(g, 1, 1, mode="down2")
        g = b.stage("G%d" % k, box, 2 * nb)
    return b.stage("B", linear(g, [[1, 2, 1], [2, 4, 2], [1, 2, 1]], 1.0 / 16), 2 * nb)


def bilateral_grid(bins: int = 8, levels: int = 3) -> dict:
    """Bilateral-grid construction: the histogram (splat and 2x2 sums down
    `levels` levels) and the blur that follows it.  Output: the blurred grid,
    2 bins channels at level `levels`."""
    b = Builder("bilateral_grid", [1])
    b.output(_grid_stages(b, input_id(0), bins, levels))
    return b.build()


def bilateral_filter(bins: int = 8, levels: int = 3) -> dict:
    """Bilateral filter through the grid: construction as bilateral_grid(),
    then every pixel slices the blurred grid linearly in intensity and at
    its own cell in x and y, reading the grid directly by an up-sampling tap
    of scale 2^levels (levels <= 3; coarser grids are first brought to level
    3 by nearest up-sampling stages U):
    out = sum_z w_z(I) V_z / (sum_z w_z(I) W_z + 1e-6), w_z the tent
    weights of the construction."""
    nb = bins
    b = Builder("bilateral_filter", [1])
    inp = input_id(0)
    g = _grid_stages(b, inp, bins, levels)
    lv = levels
    while lv > 3:
        lv -= 1
        g = b.stage("U%d" % lv, ref(g, 0, 0, mode="up2"), 2 * nb)
    mode = {1: "up2", 2: "up4", 3: "up8"}[lv]
    t = ref(inp)
    num, den = None, None
    for zb in range(nb):
        w = emax(1.0 - eabs(t * float(nb - 1) - float(zb)), 0.0)
        v = w * ref(g, 0, 0, chan=nb + zb, mode=mode)
        d = w * ref(g, 0, 0, chan=zb, mode=mode)
        num = v if num is None else num + v
        den = d if den is None else den + d
    b.output(b.stage("out", num / (den + 1e-6)))
    return b.build()


def bilateral_schedule(bins: int = 8, levels: int = 3) -> tuple:
    """(groups, params) of bilateral_filter(bins, levels): the histogram's
    splat and 2x2 sums as one reduction chain across the levels, then the
    grid's blur, any nearest up-sampling stages and the slice, one group
    each, as per-stage kernels (single stages: measured faster per stage
    than as warp-tile groups)."""
    n_stages = len(bilateral_filter(bins, levels)["stages"])
    groups = [0] * levels + list(range(1, n_stages - levels + 1))
    params = [dict(tile_h=8)] + [dict(flags=4)] * (max(groups))
    return groups, params


def _lin3(producer: int, weights, axis: str) -> E:
    """sum_i weights[i] * P at offset i - r along `axis` ("x", "y" or "z")."""
    r = len(weights) // 2
    total = None
    for i, w in enumerate(weights):
        d = i - r
        t = refz(producer, d if axis == "x" else 0, d if axis == "y" else 0, d if axis == "z" else 0)
        t = t if w == 1.0 else float(w) * t
        total = t if total is None else total + t
    return total


def unsharp3d(depth: int = 64, amount: float = 1.5) -> dict:
    """3-D unsharp mask over a `depth`-plane volume: 5-tap binomial blur along
    x, y and z (three stages), out = clamp(v + amount (v - blur), 0, 1)."""
    b = Builder("unsharp3d", [depth])
    inp = input_id(0)
    bx = b.stage("bx", _lin3(inp, BINOMIAL5, "x"), depth)
    by = b.stage("by", _lin3(bx, BINOMIAL5, "y"), depth)
    bz = b.stage("bz", _lin3(by, BINOMIAL5, "z"), depth)
    v = refz(inp)
    b.output(b.stage("sharpen", emin(emax(v + amount * (v - refz(bz)), 0.0), 1.0), depth))
    return b.build()


def heat3d(steps: int = 4, depth: int = 64, alpha: float = 0.125) -> dict:
    """`steps` explicit time steps of 3-D diffusion, each a 7-point stencil
    u' = u + alpha (sum of the six face neighbours - 6 u) with clamp-to-edge
    (zero flux) boundaries; alpha <= 1/6 keeps it stable."""
    b = Builder("heat3d", [depth])
    u = input_id(0)
    for k in range(steps):
        nb = (refz(u, -1, 0, 0) + refz(u, 1, 0, 0) + refz(u, 0, -1, 0) + refz(u, 0, 1, 0)
              + refz(u, 0, 0, -1) + refz(u, 0, 0, 1))
        u = b.stage("step%d" % k, refz(u) + alpha * (nb - 6.0 * refz(u)), depth)
    b.output(u)
    return b.build()


def by_name(name: str) -> dict:
    table = {"sharpen": sharpen, "harris": harris, "harris_raw": lambda: harris(False),
             "blend": blend, "blur": blur3, "blur_rgb": lambda: blur3(3),
             "bilateral_grid": bilateral_grid, "bilateral": bilateral_filter,
             "unsharp3d": unsharp3d, "heat3d": heat3d}
    return table[name]()

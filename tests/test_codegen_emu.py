"""Generated kernels executed on the CPU by the lane emulator (tests/emu),
compared with the FP64 oracle.  This checks the code generator's tiling,
halo, window, clamp-to-edge and load-type logic without a GPU; the same
kernel text runs on the GPU in the -m gpu tests."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1909_07190_gb300 import inputs as I
from paper_1909_07190_gb300 import pipelines as P
from paper_1909_07190_gb300 import wt

from emu import emu


def run_emulated(spec, imgs, dtype=wt.WT_F32, groups=None, params=None, exec_mode=wt.WT_EXEC_FUSED,
                 launch=0, max_blocks=None, mid=-1):
    """mid: storage type of the intermediates between launches (-1: FP32)."""
    p = wt.Pipeline(spec)
    if exec_mode == wt.WT_EXEC_PLAIN:
        p.schedule(exec_mode=exec_mode, intermediate_dtype=mid)
    else:
        p.schedule(groups=groups, params=params, intermediate_dtype=mid)
    shapes = O.shapes(spec["stages"], [np.zeros((c,) + imgs[0].shape[-2:]) for c in spec["inputs"]])
    ins = [emu.HostImage(c, a.shape[-2], a.shape[-1], dtype) for a, c in zip(imgs, spec["inputs"])]
    for h, a in zip(ins, imgs):
        name = {wt.WT_F32: "f32", wt.WT_F16: "f16", wt.WT_BF16: "bf16"}[dtype]
        h.view()[...] = I.storage_array(np.asarray(a, np.float32).reshape(h.view().shape), name)
    outs = []
    for sid in spec["outputs"]:
        _, w, h, c = shapes[sid]
        outs.append(emu.HostImage(c, h, w, dtype))
    # intermediates between groups: a poisoned host workspace
    wsb = p.debug_workspace_bytes([x.image() for x in ins], [x.image() for x in outs])
    ws = np.full(max(wsb, 16), 0xA5, np.uint8)
    emu.precompile(p, ins, outs, ws)
    d = emu.run(p, launch, ins, outs, max_blocks, ws)
    for i in range(1, d["n_launches"]):
        emu.run(p, i, ins, outs, max_blocks, ws)
    per_stage = any((q or {}).get("flags", 0) & wt.WT_FLAG_PLAIN for q in (params or []))
    if exec_mode == wt.WT_EXEC_FUSED and d["n_launches"] == 1 and not per_stage:
        assert d["fused"] or d["name"].startswith(("wt_chain_", "wt_vol_", "wt_down2_"))
    for o in outs:
        assert o.padding_intact(), "kernel wrote outside the image"
    name = {wt.WT_F32: "f32", wt.WT_F16: "f16", wt.WT_BF16: "bf16"}[dtype]
    return [I.from_storage(o.view(), name) for o in outs], d


def oracle_of(spec, imgs):
    return O.evaluate(spec["stages"], [np.asarray(a, np.float64) for a in imgs], spec["outputs"])


def rnd(seed, w, h, c=1, dtype="f32"):
    return I.round_to(I.uniform_image(seed, w, h, c), dtype)


@pytest.mark.parametrize("name", ["sharpen", "harris", "blur"])
@pytest.mark.parametrize("w,h", [(1, 1), (7, 5), (150, 70), (260, 9)])
def test_fused_sizes(name, w, h):
    spec = P.by_name(name)
    img = rnd(w * 31 + h, w, h)
    got, _ = run_emulated(spec, [img], params=[dict(tile_h=16, warps_per_block=2)])
    ref = oracle_of(spec, [img])
    assert np.abs(got[0] - ref[0]).max() <= 1e-5


@pytest.mark.parametrize("tile_h,frac,vec", [(1, 1.0, 4), (3, 0.0, 4), (5, 0.5, 8), (40, 0.0, 8), (2, 0.3, 4)])
def test_fused_params(tile_h, frac, vec):
    spec = P.harris()
    img = rnd(5, 140, 61)
    got, d = run_emulated(spec, [img], params=[dict(tile_h=tile_h, frac_reg=frac, vec=vec, warps_per_block=2)])
    ref = oracle_of(spec, [img])
    assert np.abs(got[0] - ref[0]).max() <= 1e-5


def test_fused_sharpen_shared_windows():
    spec = P.sharpen()
    img = rnd(6, 133, 47)
    got, _ = run_emulated(spec, [img], params=[dict(tile_h=7, frac_reg=0.0, warps_per_block=1)])
    assert np.abs(got[0] - oracle_of(spec, [img])[0]).max() <= 1e-5


@pytest.mark.parametrize("max_blocks", [1, 3])
def test_fused_persistent_warps(max_blocks):
    """Fewer blocks than tiles: each warp walks several tiles (mbarrier
    phases and staging buffers carry over between tiles)."""
    spec = P.harris()
    img = rnd(8, 300, 77)
    got, _ = run_emulated(spec, [img], params=[dict(tile_h=5, warps_per_block=2)], max_blocks=max_blocks)
    assert np.abs(got[0] - oracle_of(spec, [img])[0]).max() <= 1e-5


@pytest.mark.parametrize("dtype,tol", [(wt.WT_F16, 2e-3), (wt.WT_BF16, 1.6e-2)])
def test_fused_16bit(dtype, tol):
    spec = P.harris()
    name = {wt.WT_F16: "f16", wt.WT_BF16: "bf16"}[dtype]
    img = rnd(7, 100, 40, dtype=name)
    got, _ = run_emulated(spec, [img], dtype=dtype, params=[dict(tile_h=8, vec=4)])
    assert np.abs(got[0] - oracle_of(spec, [img])[0]).max() <= tol


def random_dag(seed, n_stages=6, n_inputs=2):
    """Seeded random single-level DAG: stencils and pointwise combinations
    with offsets in [-2, 2] and bounded values (test input, not a pipeline)."""
    rng = np.random.default_rng(seed)
    b = P.Builder("rand%d" % seed, [1] * n_inputs)
    ids = [P.input_id(j) for j in range(n_inputs)]
    outs = []
    for s in range(n_stages):
        k = int(rng.integers(1, 4))
        expr = None
        for _ in range(k):
            src = ids[int(rng.integers(0, len(ids)))]
            dx, dy = int(rng.integers(-2, 3)), int(rng.integers(-2, 3))
            w = float(rng.uniform(-0.6, 0.6))
            t = w * P.ref(src, dx, dy)
            expr = t if expr is None else expr + t
        kind = int(rng.integers(0, 4))
        if kind == 1:
            expr = P.emin(expr, 0.4)
        elif kind == 2:
            expr = P.eabs(expr) * 0.5
        elif kind == 3:
            other = ids[int(rng.integers(0, len(ids)))]
            expr = expr * P.ref(other, int(rng.integers(-1, 2)), 0)
        sid = b.stage("s%d" % s, expr)
        ids.append(sid)
        if rng.uniform() < 0.3:
            outs.append(sid)
    if ids[-1] not in outs:
        outs.append(ids[-1])
    b.output(*outs)
    return b.build()


@pytest.mark.parametrize("seed,frac,tile_h,vec", [(1, 0.6, 6, 4), (2, 0.0, 3, 4), (3, 1.0, 11, 8), (4, 0.3, 1, 4),
                                                  (5, 0.6, 6, 8), (6, 1.0, 2, 4), (7, 0.0, 9, 8), (8, 0.5, 4, 4)])
def test_fused_random_dags(seed, frac, tile_h, vec):
    spec = random_dag(seed)
    imgs = [rnd(100 + seed, 97, 43), rnd(200 + seed, 97, 43)]
    got, _ = run_emulated(spec, imgs, params=[dict(tile_h=tile_h, warps_per_block=2, frac_reg=frac, vec=vec)])
    ref = oracle_of(spec, imgs)
    for g, r in zip(got, ref):
        assert np.abs(g - r).max() <= 1e-5 * max(1.0, np.abs(r).max())


def single_stage(expr_fn, in_channels, channels):
    b = P.Builder("one", in_channels)
    b.output(b.stage("s", expr_fn(), channels))
    return b.build()


@pytest.mark.parametrize("mode", ["same", "down2", "up2"])
def test_plain_kernel_modes(mode):
    inp = P.input_id(0)
    b = P.Builder("m", [1])
    if mode == "same":
        b.output(b.stage("s", P.linear(inp, P.SOBEL_X, 0.125) + P.XPAR * 0.5 - P.YPAR * 0.25))
    else:
        d = b.stage("d", P._down(inp))
        b.output(d)
        if mode == "up2":
            b.output(b.stage("u", P._up(d) - P.ref(inp, 1, -1)))
    spec = b.build()
    for w, h in [(37, 23), (1, 1), (2, 3)]:
        img = rnd(41 + w, w, h)
        got, _ = run_emulated(spec, [img], exec_mode=wt.WT_EXEC_PLAIN)
        for g, r in zip(got, oracle_of(spec, [img])):
            assert np.abs(g - r).max() <= 1e-5


def test_plain_kernel_channels():
    """3-channel stage reading a 3-channel and a 1-channel input (broadcast)."""
    spec = single_stage(lambda: P.ref(P.input_id(0), 1, 0) * P.ref(P.input_id(1), 0, -1, chan=0)
                        + P.ref(P.input_id(0), 0, 0, chan=2), [3, 1], 3)
    A = rnd(42, 29, 17, 3)
    M = rnd(43, 29, 17, 1)
    got, _ = run_emulated(spec, [A, M], exec_mode=wt.WT_EXEC_PLAIN)
    assert np.abs(got[0] - oracle_of(spec, [A, M])[0]).max() <= 1e-6


def test_fused_multichannel_group():
    """Fused group over 3-channel stages with a 1-channel mask source."""
    inp, m = P.input_id(0), P.input_id(1)
    b = P.Builder("mc", [3, 1])
    s0 = b.stage("blur", P.linear(inp, [[1, 2, 1]], 0.25), 3)
    s1 = b.stage("mix", P.ref(m, 0, 0, chan=0) * P.ref(s0, 0, 1) + P.ref(inp, 0, 0, chan=1), 3)
    b.output(s1)
    spec = b.build()
    A = rnd(44, 70, 33, 3)
    M = rnd(45, 70, 33, 1)
    got, d = run_emulated(spec, [A, M], params=[dict(tile_h=8, warps_per_block=2)])
    assert d["fused"]
    assert np.abs(got[0] - oracle_of(spec, [A, M])[0]).max() <= 1e-6


@pytest.mark.parametrize("name,groups", [("sharpen", [0, 1, 2]), ("sharpen", [0, 0, 1]),
                                         ("harris", list(range(11))), ("harris", [0] * 5 + [1] * 6)])
@pytest.mark.parametrize("tile_h,frac", [(4, 0.0), (4, 1.0), (16, 0.0), (16, 1.0)])
def test_fused_multi_group_schedules(name, groups, tile_h, frac):
    """Groups that read and write intermediates in the workspace, with short
    tiles and all-shared or all-register windows (every access checked)."""
    spec = P.by_name(name)
    img = rnd(70 + tile_h, 300, 41)
    ng = max(groups) + 1
    got, _ = run_emulated(spec, [img], groups=groups, params=[dict(tile_h=tile_h, frac_reg=frac)] * ng)
    assert np.abs(got[0] - oracle_of(spec, [img])[0]).max() <= 1e-5


def gather_spec(kind):
    """Two-group pipelines whose second group reads the first at another
    level (gather sources)."""
    b = P.Builder("g_" + kind, [1])
    inp = P.input_id(0)
    d = b.stage("d", P._down(inp))
    if kind == "down":
        b.output(d)
    elif kind == "up":
        b.output(b.stage("u", P._up(d)))
    else:  # Laplacian level: same-level source and up-sampled coarse level
        b.output(b.stage("l", P.ref(inp, 1, -1) - P._up(d) * P.ref(inp)))
    return b.build()


@pytest.mark.parametrize("kind", ["down", "up", "lap"])
@pytest.mark.parametrize("w,h,tile_h,vec", [(37, 23, 4, 4), (1, 1, 8, 4), (130, 9, 3, 8), (5, 77, 16, 4),
                                            (520, 90, 8, 4), (700, 61, 16, 8), (521, 97, 6, 4)])
def test_fused_gather_sources(kind, w, h, tile_h, vec):
    """Small images (every tile a border tile: clamped gathers) and wide
    ones (interior tiles: unclamped aligned pair gathers)."""
    spec = gather_spec(kind)
    img = rnd(90 + w, w, h)
    ng = 1 if kind == "down" else 2
    got, d = run_emulated(spec, [img], groups=[0] if kind == "down" else [0, 1],
                          params=[dict(tile_h=tile_h, vec=vec)] * ng)
    assert d["fused"]
    assert np.abs(got[0] - oracle_of(spec, [img])[0]).max() <= 1e-5


@pytest.mark.parametrize("w,h,tile_h", [(80, 50, 8), (131, 67, 5), (33, 3, 16), (520, 140, 14)])
def test_fused_blend_levels(w, h, tile_h):
    """The 36-stage blend as 10 fused groups, one per level."""
    spec = P.blend()
    A, B = rnd(1, w, h, 3), rnd(2, w, h, 3)
    M = I.smooth_mask(3, w, h)
    got, d = run_emulated(spec, [A, B, M], groups=P.blend_groups(), params=[dict(tile_h=tile_h)] * 10)
    assert d["n_launches"] == 10
    assert np.abs(got[0] - oracle_of(spec, [A, B, M])[0]).max() <= 1e-5


@pytest.mark.parametrize("name", ["sharpen", "harris"])
@pytest.mark.parametrize("w,h,dtype,tol", [(150, 7, wt.WT_F32, 1e-5), (333, 5, wt.WT_F16, 2e-3),
                                           (61, 9, wt.WT_BF16, 1.6e-2), (8, 3, wt.WT_F32, 1e-5)])
def test_plain_kernels_interior_and_edges(name, w, h, dtype, tol):
    """Per-stage kernels: interior threads load row segments as aligned
    vectors, edge threads clamp each column."""
    spec = P.by_name(name)
    dn = {wt.WT_F32: "f32", wt.WT_F16: "f16", wt.WT_BF16: "bf16"}[dtype]
    img = rnd(w + h, w, h, dtype=dn)
    got, d = run_emulated(spec, [img], dtype=dtype, exec_mode=wt.WT_EXEC_PLAIN)
    assert not d["fused"]
    assert np.abs(got[0] - oracle_of(spec, [img])[0]).max() <= tol


@pytest.mark.parametrize("w,h", [(96, 40), (37, 19)])
def test_plain_blend(w, h):
    spec = P.blend()
    A, B = rnd(3, w, h, 3), rnd(4, w, h, 3)
    M = I.smooth_mask(5, w, h)
    got, d = run_emulated(spec, [A, B, M], exec_mode=wt.WT_EXEC_PLAIN)
    assert np.abs(got[0] - oracle_of(spec, [A, B, M])[0]).max() <= 1e-5


@pytest.mark.parametrize("name", ["harris", "sharpen"])
@pytest.mark.parametrize("dtype,tol", [(wt.WT_F16, 2e-3), (wt.WT_BF16, 1.6e-2)])
@pytest.mark.parametrize("frac", [0.0, 0.5])
def test_fused_16bit_shared_windows(name, dtype, tol, frac):
    """Intermediates' shared-memory windows in the 16-bit storage type
    (rounded when stored, FP32 arithmetic) against the oracle with the
    storage type's tolerance; an FP32 group ignores the flag."""
    spec = P.by_name(name)
    dn = {wt.WT_F16: "f16", wt.WT_BF16: "bf16"}[dtype]
    img = rnd(95, 150, 37, 1, dn)
    prm = dict(tile_h=8, frac_reg=frac, flags=wt.WT_FLAG_SMEM16)
    got, d = run_emulated(spec, [img], dtype=dtype, params=[prm])
    ref = oracle_of(spec, [img])[0]
    assert np.abs(got[0] - ref).max() <= tol * max(1.0, np.abs(ref).max())
    img32 = rnd(96, 150, 37)
    _, d32 = run_emulated(spec, [img32], params=[prm])
    _, d32b = run_emulated(spec, [img32], params=[dict(tile_h=8, frac_reg=frac)])
    assert d32["name"] == d32b["name"]


@pytest.mark.parametrize("name", ["harris", "sharpen"])
@pytest.mark.parametrize("frac", [1.0, 0.5, 0.0])
@pytest.mark.parametrize("tile_h", [9, 30])
def test_block_bodies_by_rows(name, frac, tile_h):
    """Tall tiles whose blocks change body mid-tile: guarded blocks at the top
    and bottom of the image, unguarded blocks in between, with x-edge
    fix-ups in the tiles crossing the left or right edge (including the
    top-left and bottom-right corners), and register or shared-memory
    windows carried across the switches."""
    spec = P.by_name(name)
    img = rnd(77 + tile_h, 380, 150)
    got, _ = run_emulated(spec, [img], params=[dict(tile_h=tile_h, frac_reg=frac, warps_per_block=2)],
                          max_blocks=3)
    ref = oracle_of(spec, [img])
    assert np.abs(got[0] - ref[0]).max() <= 1e-5


@pytest.mark.parametrize("name", ["harris", "sharpen"])
@pytest.mark.parametrize("warps", [1, 2])
def test_tile_queue_mode(name, warps):
    """Persistent warps pulling tiles from the device queue (three blocks
    take every tile) give the same result as one warp per tile."""
    spec = P.by_name(name)
    img = rnd(91 + warps, 300, 170)
    got, d = run_emulated(spec, [img], params=[dict(tile_h=24, warps_per_block=warps,
                                                    flags=wt.WT_FLAG_TILE_QUEUE)], max_blocks=3)
    ref = oracle_of(spec, [img])
    assert np.abs(got[0] - ref[0]).max() <= 1e-5
    got1, _ = run_emulated(spec, [img], params=[dict(tile_h=24, warps_per_block=warps)])
    assert np.abs(got1[0] - ref[0]).max() <= 1e-5


def cascade_spec(c=1):
    """P -> D1 -> D2, two 5x5 binomial reduces; both levels are outputs."""
    b = P.Builder("cascade", [c])
    inp = P.input_id(0)
    d1 = b.stage("d1", P._down(inp), c)
    d2 = b.stage("d2", P._down(d1), c)
    b.output(d1)
    b.output(d2)
    return b.build()


@pytest.mark.parametrize("w,h,tile_h,vec,c,dtype,tol", [
    (37, 23, 4, 4, 1, wt.WT_F32, 1e-5), (1, 1, 2, 4, 1, wt.WT_F32, 1e-5), (2, 5, 1, 4, 1, wt.WT_F32, 1e-5),
    (300, 90, 3, 4, 1, wt.WT_F32, 1e-5), (530, 41, 5, 8, 3, wt.WT_F32, 1e-5),
    (1100, 37, 4, 4, 1, wt.WT_F32, 1e-5), (1203, 29, 3, 8, 1, wt.WT_BF16, 1.6e-2),
    (2100, 19, 6, 8, 3, wt.WT_F16, 2e-3), (1030, 64, 8, 4, 1, wt.WT_BF16, 1.6e-2)])
def test_cascade_two_levels(w, h, tile_h, vec, c, dtype, tol):
    """Two down-sampling levels in one kernel: S1 rows written and fed to
    S2 on chip.  Small images (every warp at an edge, clamped loads) and
    wide ones (interior warps stage their producer rows by 16-byte copies);
    heights with a partial last unrolled round; both levels against the
    oracle."""
    spec = cascade_spec(c)
    dn = {wt.WT_F32: "f32", wt.WT_F16: "f16", wt.WT_BF16: "bf16"}[dtype]
    img = rnd(w * 7 + h, w, h, c, dtype=dn)
    got, d = run_emulated(spec, [img], dtype=dtype, groups=[0, 0], params=[dict(tile_h=tile_h, vec=vec)])
    assert d["n_launches"] == 1 and d["name"].startswith("wt_down2_")
    ref = oracle_of(spec, [img])
    for g, r in zip(got, ref):
        assert np.abs(g - r).max() <= tol


def test_cascade_blend_groups():
    """The blend with its Gaussian levels 1-2 and 3-4 as two-level cascade
    groups (mask pyramid included), the other levels fused per level."""
    spec = P.blend()
    w, h = 270, 133
    A, B = rnd(11, w, h, 3), rnd(12, w, h, 3)
    M = I.smooth_mask(13, w, h)
    g = [0] * 6 + [1] * 6 + [2] * 4 + sum([[3 + k] * 4 for k in range(5)], [])
    params = [dict(tile_h=4), dict(tile_h=2)] + [dict(tile_h=8)] * 6
    got, d = run_emulated(spec, [A, B, M], groups=g, params=params)
    p = wt.Pipeline(spec)
    p.schedule(groups=g, params=params)
    assert p.launches_per_run() == 3 + 3 + 6
    assert np.abs(got[0] - oracle_of(spec, [A, B, M])[0]).max() <= 1e-5


@pytest.mark.parametrize("name,tol", [("harris", 1e-5), ("sharpen", 1e-5), ("harris_raw", 1e-5)])
def test_deferred_scales(name, tol):
    """Constant factors deferred to the consumers (the default) and every
    stage evaluated as written (WT_FLAG_NO_FOLD) both match the oracle; the
    deferred kernel's step has fewer packed operations (the normalised
    column passes and box means keep no multiply)."""
    spec = P.by_name(name)
    img = rnd(77, 150, 70)
    ref = oracle_of(spec, [img])[0]
    if name == "harris_raw":
        tol = 1e-5 * float(np.abs(ref).max())
    srcs = {}
    for flags in (0, wt.WT_FLAG_NO_FOLD):
        got, d = run_emulated(spec, [img], params=[dict(tile_h=16, flags=flags)])
        assert np.abs(got[0] - ref).max() <= tol
        srcs[flags] = d["source"]
    # packed arithmetic of the steady-state step
    ops = {}
    for f, s in srcs.items():
        step = s[s.index("step phase 0 (steady)"):s.index("step phase 1 (steady)")]
        ops[f] = sum(step.count("wt_%s2(" % o) for o in ("add", "sub", "mul", "fma"))
    if name == "harris_raw":
        assert ops[0] <= ops[wt.WT_FLAG_NO_FOLD]  # no normalisation to defer
    else:
        assert ops[0] < ops[wt.WT_FLAG_NO_FOLD]


def test_deferred_scales_blend_level():
    """A blend level's group (up-sampled gathers, per-level blend,
    reconstruction) with its stored value brought back to scale 1."""
    spec = P.blend(levels=2, channels=1)
    a, b, m = rnd(5, 67, 45), rnd(6, 67, 45), rnd(7, 67, 45)
    ref = oracle_of(spec, [a, b, m])[0]
    groups, params = P.blend_schedule(levels=2)
    for flags in (0, wt.WT_FLAG_NO_FOLD):
        prm = [dict(q, flags=q.get("flags", 0) | flags) for q in params]
        got, _ = run_emulated(spec, [a, b, m], groups=groups, params=prm)
        assert np.abs(got[0] - ref).max() <= 1e-5


def scaled_dag(seed, n_stages=7):
    """Seeded random single-level DAG whose stages carry constant factors
    (normalisations, signs, powers of two and others) under non-linear
    operations: min and max against constants and against operands of the
    same factor, abs, sqrt, division by constants and by other values,
    negation, row and column parity (test input, not a pipeline)."""
    rng = np.random.default_rng(seed)
    b = P.Builder("fold%d" % seed, [1, 1])
    ids = [P.input_id(0), P.input_id(1)]
    factors = [0.25, 0.125, -0.5, 2.0, 1.0 / 16, 3.0, -1.0, 1.0 / 576]
    outs = []

    def term():
        return P.ref(ids[int(rng.integers(0, len(ids)))], int(rng.integers(-2, 3)), int(rng.integers(-2, 3)))

    for s in range(n_stages):
        c = factors[int(rng.integers(0, len(factors)))]
        expr = None
        for w in rng.integers(-2, 3, size=int(rng.integers(1, 4))):
            w = int(w) or 1
            t = term() if w == 1 else float(w) * term()
            expr = t if expr is None else expr + t
        expr = expr * c if rng.uniform() < 0.5 else c * expr
        kind = int(rng.integers(0, 12))
        if kind == 1:
            expr = P.emin(expr, float(rng.uniform(-0.3, 0.3)))
        elif kind == 2:
            expr = P.emax(0.2, expr)
        elif kind == 3:
            expr = P.eabs(expr) * 0.5
        elif kind == 4:
            expr = P.esqrt(P.eabs(expr) + 0.01)
        elif kind == 5:
            expr = expr / 3.0
        elif kind == 6:
            expr = expr / (P.eabs(term()) + 1.0)
        elif kind == 7:
            expr = 0.75 - expr
        elif kind == 8:
            expr = -expr + term() * 0.5
        elif kind == 9:
            expr = P.emin(expr, term() * c)
        elif kind == 10:
            expr = expr * term() - P.YPAR * 0.25 + P.XPAR * expr
        elif kind == 11:
            expr = (expr - term() * (2 * c)) * 4.0
        sid = b.stage("s%d" % s, expr)
        ids.append(sid)
        if rng.uniform() < 0.25:
            outs.append(sid)
    if ids[-1] not in outs:
        outs.append(ids[-1])
    b.output(*outs)
    return b.build()


@pytest.mark.parametrize("seed", [0, 11, 24, 37])
def test_deferred_scales_random_programs(seed):
    """Constant factors carried through min, max, abs, sqrt, division and
    sums of differently scaled terms: the deferred form and the form as
    written both match the oracle."""
    spec = scaled_dag(seed)
    imgs = [rnd(300 + seed, 61, 29), rnd(400 + seed, 61, 29)]
    ref = oracle_of(spec, imgs)
    for flags in (0, wt.WT_FLAG_NO_FOLD):
        got, _ = run_emulated(spec, imgs, params=[dict(tile_h=8, flags=flags)])
        for g, r in zip(got, ref):
            assert np.abs(g - r).max() <= 1e-5 * max(1.0, np.abs(r).max())


def multilevel_dag(seed, n_stages=7):
    """Seeded random DAG over three pyramid levels: each stage sits on a
    level and reads producers up to two levels finer or coarser (taps
    scaling by 2 or 4) or on its own level (test input, not a pipeline)."""
    mode = {0: "same", -1: "down2", 1: "up2", -2: "down4", 2: "up4"}
    rng = np.random.default_rng(seed)
    b = P.Builder("ml%d" % seed, [1])
    nodes = [(P.input_id(0), 0)]
    outs = []
    for s in range(n_stages):
        L = int(rng.integers(0, 3))
        expr = None
        for _ in range(int(rng.integers(1, 4))):
            pid, lp = nodes[int(rng.integers(0, len(nodes)))]
            t = float(rng.choice([0.25, 0.5, -0.375, 1.0])) * P.ref(pid, int(rng.integers(-2, 3)),
                                                                    int(rng.integers(-2, 3)), mode=mode[lp - L])
            expr = t if expr is None else expr + t
        kind = int(rng.integers(0, 5))
        if kind == 1:
            expr = expr + P.YPAR * 0.125 - P.XPAR * 0.25
        elif kind == 2:
            expr = P.emin(expr, 0.3)
        elif kind == 3:
            expr = P.eabs(expr) * 0.5
        sid = b.stage("s%d" % s, expr)
        nodes.append((sid, L))
        if rng.uniform() < 0.3:
            outs.append(sid)
    if nodes[-1][0] not in outs:
        outs.append(nodes[-1][0])
    b.output(*outs)
    return b.build()


@pytest.mark.parametrize("seed", [0, 4])
def test_multilevel_random_groupings(seed):
    """Random DAGs across pyramid levels under the analytic model's
    schedule and under random contiguous groupings with random tile
    parameters, against the oracle."""
    spec = multilevel_dag(seed)
    W, H = [(67, 45), (130, 33), (41, 77)][seed % 3]
    imgs = [rnd(500 + seed, W, H)]
    ref = oracle_of(spec, imgs)
    p = wt.Pipeline(spec)
    p.schedule_auto(W, H)
    sch = p.schedule_get()
    schedules = [(sch["groups"], sch["params"])]
    rng = np.random.default_rng(1000 + seed)
    for _ in range(2):
        g, cur = [], 0
        for i in range(len(spec["stages"])):
            cur += int(i > 0 and rng.uniform() < 0.35)
            g.append(cur)
        prm = [dict(tile_h=int(rng.choice([4, 8, 16])), frac_reg=float(rng.choice([0.0, 0.5, 1.0])),
                    vec=int(rng.choice([0, 4, 8])), warps_per_block=int(rng.choice([1, 2])))
               for _ in range(max(g) + 1)]
        schedules.append((g, prm))
    for g, prm in schedules:
        got, _ = run_emulated(spec, imgs, groups=g, params=prm)
        for a, r in zip(got, ref):
            assert np.abs(a - r).max() <= 1e-5 * max(1.0, np.abs(r).max())


@pytest.mark.parametrize("mode", ["otptb", "queue", "direct"])
@pytest.mark.parametrize("tile_h", [5, 7])
def test_row_parity_odd_tiles(mode, tile_h):
    """Row parity under odd tile heights in the block-tile kernel, the
    tile-queue kernel and one warp per tile."""
    from test_host_bands import parity_pipeline
    spec = parity_pipeline(1)
    img = rnd(5 + tile_h, 130, 41)
    prm = {"otptb": dict(tile_h=tile_h, warps_per_block=16, vec=1, flags=wt.WT_FLAG_OTPTB),
           "queue": dict(tile_h=tile_h, flags=wt.WT_FLAG_TILE_QUEUE),
           "direct": dict(tile_h=tile_h)}[mode]
    got, _ = run_emulated(spec, [img], params=[prm], max_blocks=2 if mode == "queue" else None)
    assert np.abs(got[0] - oracle_of(spec, [img])[0]).max() <= 1e-5


@pytest.mark.parametrize("name,mode", [("sharpen", "plain"), ("sharpen", "two_groups"), ("harris", "two_groups")])
@pytest.mark.parametrize("dtype,tol", [(wt.WT_F16, 2e-3), (wt.WT_BF16, 1.6e-2)])
def test_16bit_intermediates(name, mode, dtype, tol):
    """Intermediates between launches stored in the 16-bit storage type
    (the unfused path's storage-type variant, and groups linked through
    the workspace), within the storage type's tolerance of the oracle."""
    spec = P.by_name(name)
    dn = {wt.WT_F16: "f16", wt.WT_BF16: "bf16"}[dtype]
    img = rnd(31, 97, 45, dtype=dn)
    ref = oracle_of(spec, [img])[0]
    n = len(spec["stages"])
    kw = dict(exec_mode=wt.WT_EXEC_PLAIN) if mode == "plain" else \
        dict(groups=[0] * (n // 2) + [1] * (n - n // 2), params=[dict(tile_h=8)] * 2)
    got, d = run_emulated(spec, [img], dtype=dtype, mid=dtype, **kw)
    assert d["n_launches"] >= 2
    assert np.abs(got[0] - ref).max() <= tol

"""3-D groups (App. A, generalised hybrid tiling: lanes along x, one axis
streamed, the third a register tile) executed on the CPU by the block
emulator (every thread a fiber, every global access bounds-checked),
compared with the FP64 oracle: both split axes, register tiles of 1..8
points, 1, 2 or 4 points per lane, ragged and tiny volumes, liveouts inside
the group, one-plane sources, and the per-stage fallback."""
import numpy as np
import pytest

from paper_1909_07190_gb300 import pipelines as P
from paper_1909_07190_gb300 import wt

from test_codegen_emu import oracle_of, rnd, run_emulated

Z = wt.WT_FLAG_ZSTREAM


def vparams(split, tile_o=4, vec=2, tile_h=8, warps=2, staged=False):
    """staged: sources in the warp's shared memory (frac_reg < 1)."""
    return dict(tile_h=tile_h, tile_o=tile_o, vec=vec, warps_per_block=warps, flags=Z if split else 0,
                frac_reg=0.0 if staged else 1.0)


def check(spec, imgs, params, groups=None, tol=1e-5, prefix="wt_vol_"):
    got, d = run_emulated(spec, imgs, groups=groups, params=params)
    if prefix:
        assert d["name"].startswith(prefix), d["name"]
    ref = oracle_of(spec, imgs)
    for g, r in zip(got, ref):
        assert g.shape == r.shape
        assert np.abs(g - r).max() <= tol * max(1.0, np.abs(r).max())
    return d


@pytest.mark.parametrize("split", [0, 1])
@pytest.mark.parametrize("D,H,W", [(1, 1, 1), (5, 7, 9), (9, 13, 70), (3, 40, 129), (17, 6, 33)])
def test_heat_two_steps(split, D, H, W):
    spec = P.heat3d(2, depth=D)
    img = rnd(D * 31 + H * 7 + W, W, H, D)
    check(spec, [img], [vparams(split)])


@pytest.mark.parametrize("split", [0, 1])
@pytest.mark.parametrize("tile_o,vec,tile_h", [(1, 1, 1), (2, 2, 3), (8, 1, 5), (3, 2, 16), (4, 2, 8)])
def test_unsharp_tiles(split, tile_o, vec, tile_h):
    D, H, W = 11, 23, 75
    spec = P.unsharp3d(depth=D)
    img = rnd(5 + tile_o + vec + tile_h, W, H, D)
    check(spec, [img], [vparams(split, tile_o, vec, tile_h)])


@pytest.mark.parametrize("split", [0, 1])
def test_liveout_inside_group_and_one_plane_source(split):
    """A mid-group stage is also an output; a one-plane mask read with
    plane offsets (always plane 0); asymmetric taps in every axis."""
    D = 6
    b = P.Builder("mix3", [D, 1])
    inp, m = P.input_id(0), P.input_id(1)
    s0 = b.stage("a", P.refz(inp, -2, 1, 1) + 0.5 * P.refz(inp, 1, 0, -2) - 0.25 * P.refz(m, 0, -1, 3), D)
    s1 = b.stage("b", P.emax(P.refz(s0, 0, 0, -1), P.refz(s0, 1, -1, 2)) * P.refz(m, -1, 0, 0), D)
    s2 = b.stage("c", P.refz(s1, 0, 2, 0) + P.refz(s0, 0, 0, 1) + P.refz(inp), D)
    b.output(s2, s0)
    spec = b.build()
    img, mask = rnd(71, 50, 19, D), rnd(72, 50, 19, 1)
    check(spec, [img, mask], [vparams(split, 2, 1, 6)])


@pytest.mark.parametrize("dtype", ["f16", "bf16"])
def test_sixteen_bit_storage(dtype):
    D, H, W = 7, 12, 40
    spec = P.heat3d(2, depth=D)
    img = rnd(9, W, H, D, dtype=dtype)
    got, d = run_emulated(spec, [img], dtype={"f16": wt.WT_F16, "bf16": wt.WT_BF16}[dtype],
                          params=[vparams(1)])
    assert d["name"].startswith("wt_vol_")
    ref = oracle_of(spec, [img])[0]
    assert np.abs(got[0] - ref).max() <= (2e-3 if dtype == "f16" else 1.6e-2)


def test_two_groups_through_the_workspace():
    D = 5
    spec = P.heat3d(4, depth=D)
    img = rnd(11, 37, 21, D)
    got, d = run_emulated(spec, [img], groups=[0, 0, 1, 1], params=[vparams(0, 2), vparams(1, 3)])
    assert d["n_launches"] == 2
    assert np.abs(got[0] - oracle_of(spec, [img])[0]).max() <= 1e-5


def test_plain_execution_of_plane_taps():
    D = 6
    spec = P.unsharp3d(depth=D)
    img = rnd(12, 45, 14, D)
    got, d = run_emulated(spec, [img], exec_mode=wt.WT_EXEC_PLAIN)
    assert d["name"].startswith("wt_plain_")
    assert np.abs(got[0] - oracle_of(spec, [img])[0]).max() <= 1e-5


def test_group_the_3d_kernel_cannot_take_runs_per_stage():
    """A channel-index op inside a group with plane taps: per-stage kernels."""
    D = 4
    b = P.Builder("chz", [D])
    inp = P.input_id(0)
    s0 = b.stage("a", P.refz(inp, 0, 0, 1) * P.CHAN, D)
    b.output(b.stage("b", P.refz(s0, 1, 0, -1) + P.refz(s0), D))
    spec = b.build()
    img = rnd(13, 30, 9, D)
    got, d = run_emulated(spec, [img], params=[vparams(0)])
    assert d["n_launches"] == 2 and d["name"].startswith("wt_plain_")
    assert np.abs(got[0] - oracle_of(spec, [img])[0]).max() <= 1e-5


def test_register_limit_falls_back():
    """Four fused heat steps with an 8-point register tile exceed the
    window budget: per-stage kernels, same result."""
    D = 10
    spec = P.heat3d(4, depth=D)
    img = rnd(14, 33, 12, D)
    got, d = run_emulated(spec, [img], params=[vparams(0, 8, 4)])
    assert d["n_launches"] == 4
    assert np.abs(got[0] - oracle_of(spec, [img])[0]).max() <= 1e-5


def test_launch_count_of_3d_groups():
    """A 3-D group is one launch; one the 3-D kernel cannot take runs per
    stage (host-side count, no device)."""
    D = 8
    p = wt.Pipeline(P.unsharp3d(depth=D))
    p.schedule(params=[vparams(1)])
    assert p.launches_per_run() == 1
    p.schedule(params=[vparams(0, 8, 4)])
    assert p.launches_per_run() == 4
    p.schedule(exec_mode=wt.WT_EXEC_PLAIN)
    assert p.launches_per_run() == 4


@pytest.mark.parametrize("split,tile_o,vec", [(0, 2, 4), (1, 2, 4), (1, 4, 2), (0, 1, 1)])
def test_interior_tiles_vector_paths(split, tile_o, vec):
    """Volumes wide enough for interior tiles (vector loads and stores,
    no clamps) between the border ones."""
    D, H, W = 7, 11, 300
    spec = P.heat3d(2, depth=D)
    img = rnd(15 + vec, W, H, D)
    check(spec, [img], [vparams(split, tile_o, vec, 5)])


@pytest.mark.parametrize("dtype,vec", [("f16", 1), ("bf16", 2), ("f16", 4)])
def test_interior_tiles_sixteen_bit(dtype, vec):
    """16-bit sources staged from an even start column in interior tiles."""
    D, H, W = 5, 9, 301
    spec = P.heat3d(2, depth=D)
    img = rnd(16 + vec, W, H, D, dtype=dtype)
    got, d = run_emulated(spec, [img], dtype={"f16": wt.WT_F16, "bf16": wt.WT_BF16}[dtype],
                          params=[vparams(1, 2, vec, 4)])
    assert d["name"].startswith("wt_vol_")
    ref = oracle_of(spec, [img])[0]
    assert np.abs(got[0] - ref).max() <= (2e-3 if dtype == "f16" else 1.6e-2)


@pytest.mark.parametrize("split", [0, 1])
@pytest.mark.parametrize("name,W", [("heat3d", 70), ("unsharp3d", 300), ("heat3d", 301)])
@pytest.mark.parametrize("vec", [1, 2, 4])
def test_staged_sources(split, name, W, vec):
    """frac_reg < 1: source rows staged in shared memory by asynchronous
    copies (interior tiles from an aligned start, border tiles clamped)."""
    D, H = 6, 10
    spec = P.heat3d(2, depth=D) if name == "heat3d" else P.unsharp3d(depth=D)
    img = rnd(20 + W + vec, W, H, D)
    check(spec, [img], [vparams(split, 2, vec, 5, staged=True)])


@pytest.mark.parametrize("dtype", ["f16", "bf16"])
def test_staged_sixteen_bit(dtype):
    D, H, W = 5, 9, 301
    spec = P.heat3d(2, depth=D)
    img = rnd(30, W, H, D, dtype=dtype)
    got, d = run_emulated(spec, [img], dtype={"f16": wt.WT_F16, "bf16": wt.WT_BF16}[dtype],
                          params=[vparams(1, 2, 1, 4, staged=True)])
    assert d["name"].startswith("wt_vol_")
    assert np.abs(got[0] - oracle_of(spec, [img])[0]).max() <= (2e-3 if dtype == "f16" else 1.6e-2)


@pytest.mark.parametrize("staged", [False, True])
@pytest.mark.parametrize("ahead", [1, 3, 5])
def test_prefetch_distance(staged, ahead):
    """n_buffers rows of look-ahead for the sources (1..8)."""
    D, H, W = 6, 12, 140
    spec = P.unsharp3d(depth=D)
    img = rnd(50 + ahead, W, H, D)
    check(spec, [img], [dict(vparams(1, 2, 1, 6, staged=staged), n_buffers=ahead)])

"""The block-tile kernel (one overlapped tile per thread block, the tiling
the paper compares against in Sec. 3 and Sec. 7) executed on the CPU by the
block emulator (every thread a fiber, block barriers, every shared and
global access bounds-checked), compared with the FP64 oracle."""
import numpy as np
import pytest

from paper_1909_07190_gb300 import pipelines as P
from paper_1909_07190_gb300 import wt

from test_codegen_emu import oracle_of, random_dag, rnd, run_emulated

OTPTB = wt.WT_FLAG_OTPTB


def blk(tile_h=16, warps=4, vec=4, **kw):
    return dict(tile_h=tile_h, warps_per_block=warps, vec=vec, flags=OTPTB, **kw)


@pytest.mark.parametrize("name", ["sharpen", "harris", "blur"])
@pytest.mark.parametrize("w,h", [(1, 1), (7, 5), (150, 70), (260, 9)])
def test_otptb_sizes(name, w, h):
    spec = P.by_name(name)
    img = rnd(w * 17 + h, w, h)
    got, d = run_emulated(spec, [img], params=[blk()])
    assert d["name"].startswith("wt_otptb_")
    assert tuple(d["grid"]) == ((w + 127) // 128, (h + 15) // 16, 1)
    ref = oracle_of(spec, [img])
    for g, r in zip(got, ref):
        assert np.abs(g - r).max() <= 1e-5 * max(1.0, np.abs(r).max())


@pytest.mark.parametrize("vec,tile_h,warps", [(1, 1, 1), (2, 3, 2), (8, 32, 8), (1, 40, 16), (4, 5, 3)])
def test_otptb_tile_shapes(vec, tile_h, warps):
    """Tiles of 32..256 x 1..40 outputs and 1..16 warps: region loops with
    ragged last rounds, tiles narrower than the halo."""
    spec = P.by_name("harris")
    img = rnd(300 + vec * 7 + tile_h, 83, 61)
    got, d = run_emulated(spec, [img], params=[blk(tile_h, warps, vec)])
    assert d["block"] == 32 * warps
    assert np.abs(got[0] - oracle_of(spec, [img])[0]).max() <= 1e-5 * max(1.0, np.abs(oracle_of(spec, [img])[0]).max())


@pytest.mark.parametrize("seed,tile_h,vec", [(1, 6, 4), (2, 3, 1), (3, 11, 8), (4, 1, 2), (5, 16, 4)])
def test_otptb_random_dags(seed, tile_h, vec):
    spec = random_dag(seed)
    imgs = [rnd(100 + seed, 97, 43), rnd(200 + seed, 97, 43)]
    got, _ = run_emulated(spec, imgs, params=[blk(tile_h, 2, vec)])
    for g, r in zip(got, oracle_of(spec, imgs)):
        assert np.abs(g - r).max() <= 1e-5 * max(1.0, np.abs(r).max())


def test_otptb_multichannel_group():
    inp, m = P.input_id(0), P.input_id(1)
    b = P.Builder("mc", [3, 1])
    s0 = b.stage("blur", P.linear(inp, [[1, 2, 1]], 0.25), 3)
    s1 = b.stage("mix", P.ref(m, 0, 0, chan=0) * P.ref(s0, 0, 1) + P.ref(inp, 0, 0, chan=1), 3)
    b.output(s1)
    spec = b.build()
    A = rnd(44, 70, 33, 3)
    M = rnd(45, 70, 33, 1)
    got, d = run_emulated(spec, [A, M], params=[blk(8, 2)])
    assert d["grid"][2] == 3
    assert np.abs(got[0] - oracle_of(spec, [A, M])[0]).max() <= 1e-6


def test_otptb_parity_selects():
    """Row and column parity selects evaluated at clamped coordinates."""
    inp = P.input_id(0)
    b = P.Builder("par", [1])
    s0 = b.stage("a", P.ref(inp, 1, 0) * P.XPAR + P.ref(inp, 0, -1) * P.YPAR)
    s1 = b.stage("b", P.ref(s0, -2, 1) - P.ref(s0, 1, -2) * P.XPAR)
    b.output(s1)
    spec = b.build()
    for w, h in [(33, 17), (2, 1), (130, 5)]:
        img = rnd(46 + w, w, h)
        got, _ = run_emulated(spec, [img], params=[blk(4, 2, 1)])
        assert np.abs(got[0] - oracle_of(spec, [img])[0]).max() <= 1e-6


@pytest.mark.parametrize("dtype,tol", [(wt.WT_F16, 2e-3), (wt.WT_BF16, 1.6e-2)])
def test_otptb_16bit(dtype, tol):
    spec = P.by_name("harris")
    name = {wt.WT_F16: "f16", wt.WT_BF16: "bf16"}[dtype]
    img = rnd(47, 150, 37, 1, name)
    got, _ = run_emulated(spec, [img], dtype=dtype, params=[blk(8, 4, 8)])
    assert np.abs(got[0] - oracle_of(spec, [img])[0]).max() <= tol


def test_otptb_mixed_with_warp_tiles():
    """Harris as two groups: block tiles, then warp tiles, through the
    workspace."""
    spec = P.by_name("harris")
    img = rnd(48, 140, 51)
    got, d = run_emulated(spec, [img], groups=[0] * 5 + [1] * 6,
                          params=[blk(8, 4), dict(tile_h=8, warps_per_block=2)])
    assert d["n_launches"] == 2
    assert np.abs(got[0] - oracle_of(spec, [img])[0]).max() <= 1e-5


def test_otptb_buffer_reuse():
    """Buffers of dead stages are reused: Harris (11 stages, 2 split row
    passes, the input) needs far less shared memory than one buffer per
    node."""
    spec = P.by_name("harris")
    img = rnd(49, 256, 64)
    _, d = run_emulated(spec, [img], params=[blk(16, 8)])
    one_region = (128 + 8) * (16 + 8) * 4
    assert d["smem"] < 6 * one_region


def test_otptb_refuses_other_levels():
    """Groups fed through down/up-sampling taps have no block-tile kernel."""
    b = P.Builder("lv", [1])
    inp = P.input_id(0)
    d = b.stage("d", P._down(inp))
    u = b.stage("u", P._up(d) - P.ref(inp, 1, -1))
    b.output(u)
    spec = b.build()
    img = rnd(50, 40, 30)
    with pytest.raises(wt.WtError):
        run_emulated(spec, [img], groups=[0, 1], params=[dict(tile_h=8), blk(8, 2)], launch=1)


@pytest.mark.parametrize("name", ["harris", "sharpen"])
@pytest.mark.parametrize("vec,tile_h,warps", [(4, 16, 8), (1, 8, 4), (2, 32, 16)])
def test_otptb_interior_tiles(name, vec, tile_h, warps):
    """Images large enough for interior block tiles (every region inside
    the image: row-by-warp, column-by-lane loops and constant tap offsets)
    next to clamped border tiles."""
    spec = P.by_name(name)
    img = rnd(400 + vec + tile_h, 600, 200)
    got, _ = run_emulated(spec, [img], params=[blk(tile_h, warps, vec)])
    ref = oracle_of(spec, [img])[0]
    assert np.abs(got[0] - ref).max() <= 1e-5 * max(1.0, np.abs(ref).max())

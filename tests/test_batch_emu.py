"""Batched runs (one persistent launch per group over the tiles of many
images of different sizes) executed by the lane emulator and compared, image
by image, with the FP64 oracle."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1909_07190_gb300 import inputs as I
from paper_1909_07190_gb300 import pipelines as P
from paper_1909_07190_gb300 import wt

from emu import emu

NAMES = {wt.WT_F32: "f32", wt.WT_F16: "f16", wt.WT_BF16: "bf16"}


def run_batch_emulated(spec, batch, dtype=wt.WT_F32, params=None, max_blocks=None):
    """batch: list of per-image input lists.  Returns per-image output lists."""
    p = wt.Pipeline(spec)
    p.schedule(params=params)
    ins, outs = [], []
    for imgs in batch:
        for a, c in zip(imgs, spec["inputs"]):
            h = emu.HostImage(c, a.shape[-2], a.shape[-1], dtype)
            h.view()[...] = I.storage_array(np.asarray(a, np.float32).reshape(h.view().shape), NAMES[dtype])
            ins.append(h)
        shapes = O.shapes(spec["stages"], [np.zeros((c,) + imgs[0].shape[-2:]) for c in spec["inputs"]])
        for sid in spec["outputs"]:
            _, w, hh, c = shapes[sid]
            outs.append(emu.HostImage(c, hh, w, dtype))
    d = emu.run_batch(p, 0, ins, outs, len(batch), max_blocks)
    assert d["n_launches"] == 1
    for o in outs:
        assert o.padding_intact(), "kernel wrote outside the image"
    k = len(spec["outputs"])
    res = [[I.from_storage(o.view(), NAMES[dtype]) for o in outs[i * k:(i + 1) * k]] for i in range(len(batch))]
    return res, d


def oracle_of(spec, imgs):
    return O.evaluate(spec["stages"], [np.asarray(a, np.float64) for a in imgs], spec["outputs"])


def rnd(seed, w, h, c=1, dtype="f32"):
    return I.round_to(I.uniform_image(seed, w, h, c), dtype)


SIZES = [(1, 1), (130, 9), (250, 40), (37, 61), (300, 20), (121, 3)]


@pytest.mark.parametrize("max_blocks", [None, 1, 3])
def test_batch_harris_uneven_sizes(max_blocks):
    spec = P.harris()
    batch = [[rnd(900 + i, w, h)] for i, (w, h) in enumerate(SIZES)]
    got, d = run_batch_emulated(spec, batch, params=[dict(tile_h=7, warps_per_block=2)], max_blocks=max_blocks)
    tiles = np.asarray(d["tiles"]).reshape(-1, 4)
    assert d["n_tiles"] == len(tiles)
    assert sorted(set(tiles[:, 0].tolist())) == list(range(len(SIZES)))
    for (imgs, g) in zip(batch, got):
        assert np.abs(g[0] - oracle_of(spec, imgs)[0]).max() <= 1e-5


def test_batch_tile_table_covers_every_image_once():
    """Every (tile column, tile row) of every image is listed exactly once."""
    spec = P.sharpen()
    p = wt.Pipeline(spec)
    p.schedule(params=[dict(tile_h=5, warps_per_block=2)])
    ins = [emu.HostImage(1, h, w, wt.WT_F32) for (w, h) in SIZES]
    outs = [emu.HostImage(1, h, w, wt.WT_F32) for (w, h) in SIZES]
    d = p.debug_batch(0, [x.image() for x in ins], [x.image() for x in outs], len(SIZES))
    lay = p.debug_layout(0, [ins[0].image()], [outs[0].image()])
    out_w = lay["out_w"]
    tiles = np.asarray(d["tiles"]).reshape(-1, 4)
    for i, (w, h) in enumerate(SIZES):
        t = tiles[tiles[:, 0] == i]
        want = {(tx, ty) for tx in range(-(-w // out_w)) for ty in range(-(-h // 5))}
        got = [(int(a), int(b)) for a, b in t[:, 1:3]]
        assert len(got) == len(want) and set(got) == want


def test_batch_multi_input_fp16():
    spec = P.Builder("mi", [1, 1])
    a, b = P.input_id(0), P.input_id(1)
    s0 = spec.stage("s0", P.linear(a, [[1, 2, 1]], 0.25) * P.ref(b, 0, 1))
    s1 = spec.stage("s1", P.ref(s0, -1, 0) - P.ref(s0, 1, 0) + P.ref(b, 0, -2))
    spec.output(s0, s1)
    spec = spec.build()
    batch = [[rnd(700 + i, w, h, dtype="f16"), rnd(800 + i, w, h, dtype="f16")]
             for i, (w, h) in enumerate(SIZES[1:5])]
    got, _ = run_batch_emulated(spec, batch, dtype=wt.WT_F16, params=[dict(tile_h=4, warps_per_block=2, vec=8)],
                                max_blocks=2)
    for imgs, g in zip(batch, got):
        ref = oracle_of(spec, imgs)
        for k in range(2):
            assert np.abs(g[k] - ref[k]).max() <= 2e-3


def test_batch_multichannel():
    inp, m = P.input_id(0), P.input_id(1)
    b = P.Builder("mc", [3, 1])
    s0 = b.stage("blur", P.linear(inp, [[1, 2, 1]], 0.25), 3)
    s1 = b.stage("mix", P.ref(m, 0, 0, chan=0) * P.ref(s0, 0, 1) + P.ref(inp, 0, 0, chan=1), 3)
    b.output(s1)
    spec = b.build()
    batch = [[rnd(600 + i, w, h, 3), rnd(650 + i, w, h, 1)] for i, (w, h) in enumerate([(70, 33), (9, 140)])]
    got, _ = run_batch_emulated(spec, batch, params=[dict(tile_h=8, warps_per_block=2)], max_blocks=2)
    for imgs, g in zip(batch, got):
        assert np.abs(g[0] - oracle_of(spec, imgs)[0]).max() <= 1e-6


def test_batch_rejects_mixed_dtypes():
    spec = P.sharpen()
    p = wt.Pipeline(spec)
    p.schedule()
    i0, o0 = emu.HostImage(1, 20, 30, wt.WT_F32), emu.HostImage(1, 20, 30, wt.WT_F32)
    i1, o1 = emu.HostImage(1, 20, 30, wt.WT_F16), emu.HostImage(1, 20, 30, wt.WT_F16)
    with pytest.raises(wt.WtError):
        p.debug_batch(0, [i0.image(), i1.image()], [o0.image(), o1.image()], 2)


@pytest.mark.parametrize("tile_h", [3, 7])
def test_batch_row_parity_odd_tiles(tile_h):
    """A stage reading the output row's parity under odd tile heights:
    every tile of every image takes the parity of its rows in its own image."""
    from test_host_bands import parity_pipeline
    spec = parity_pipeline(1)
    batch = [[rnd(950 + i, w, h)] for i, (w, h) in enumerate(SIZES)]
    got, _ = run_batch_emulated(spec, batch, params=[dict(tile_h=tile_h, warps_per_block=2)], max_blocks=3)
    for imgs, g in zip(batch, got):
        assert np.abs(g[0] - oracle_of(spec, imgs)[0]).max() <= 1e-5

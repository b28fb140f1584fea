"""Row bands of wt_run_host (planning only, no GPU).

A host run of a single-level pipeline on a large image is split into row
bands: band b keeps output rows [y0, y1) and runs the pipeline on the
sub-image of input rows [ys, ye).  The result equals the whole-image run
when the bands partition the rows, each band's sub-image holds the
pipeline's row halo (the rows clamp-to-edge changes at a band edge are
not kept), and the sub-image starts on an even row (a stage reading the
output row's parity sees the same parity).  These tests take the halo
from the pipeline definition and check every band against the FP64
oracle run on the band's sub-image.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1909_07190_gb300 import inputs as I
from paper_1909_07190_gb300 import pipelines as P
from paper_1909_07190_gb300 import wt


def img(W, H, C, dt, base, pitch=None):
    es = 4 if dt == wt.WT_F32 else 2
    return wt.image(base, W, H, C, dt, pitch or ((W * es + 127) // 128) * 128)


def io(spec, W, H, dt=wt.WT_F32, pitch=None):
    ins = [img(W, H, c, dt, (1 + j) << 36, pitch) for j, c in enumerate(spec["inputs"])]
    outs = [img(W, H, spec["stages"][s]["channels"], dt, (8 + k) << 36, pitch) for k, s in enumerate(spec["outputs"])]
    return ins, outs


def row_halo(spec):
    """Input rows above and below an output row that the pipeline reads:
    the largest sum of vertical tap offsets along any path to an input."""
    st = spec["stages"]
    top, bot = {}, {}
    for sid, s in enumerate(st):
        t = b = 0
        for op in s["ops"]:
            if op[0] != "tap":
                continue
            pid = s["inputs"][op[1]]
            dy = op[3]
            t = max(t, max(0, -dy) + (top[pid] if pid >= 0 else 0))
            b = max(b, max(0, dy) + (bot[pid] if pid >= 0 else 0))
        top[sid], bot[sid] = t, b
    return max(max(top[s], bot[s]) for s in spec["outputs"])


def check_plan(bands, H, h):
    assert bands[0][0] == 0 and bands[-1][1] == H
    for (y0, y1, ys, ye), nxt in zip(bands, bands[1:] + [None]):
        assert y0 < y1
        if nxt is not None:
            assert nxt[0] == y1
        assert ys % 2 == 0
        assert ys <= max(0, y0 - h) and ys >= y0 - h - 1
        assert ye == min(H, y1 + h)


def parity_pipeline(dy):
    """A Bayer-like stage: odd rows average the rows dy above and below,
    even rows keep the pixel; then a vertical difference over one row."""
    inp = P.input_id(0)
    b = P.Builder("rowpar", [1])
    s0 = b.stage("g", P.YPAR * 0.5 * (P.ref(inp, 0, -dy) + P.ref(inp, 0, dy)) + (1.0 - P.YPAR) * P.ref(inp, 1, 0))
    b.output(b.stage("d", P.ref(s0, 0, 1) - P.ref(s0, 0, -1) * 0.75 + P.YPAR * 0.125))
    return b.build()


@pytest.mark.parametrize("name,W,H,n", [("harris", 4096, 4096, 8), ("sharpen", 2048, 2048, 2),
                                        ("harris", 1100, 4001, 2), ("sharpen", 8192, 8192, 8)])
def test_band_plan(name, W, H, n):
    spec = P.by_name(name)
    p = wt.Pipeline(spec)
    bands = p.debug_host_bands(*io(spec, W, H))
    assert len(bands) == n
    check_plan(bands, H, row_halo(spec))
    # every band but the last copies at least 8 MiB of input
    es = 4
    pitch = ((W * es + 127) // 128) * 128
    for y0, y1, _, _ in bands[:-1]:
        assert (y1 - y0) * pitch >= 8 << 20


def test_no_bands():
    spec = P.harris()
    p = wt.Pipeline(spec)
    assert p.debug_host_bands(*io(spec, 2000, 2000)) == []          # under 16 MiB of input
    assert p.debug_host_bands(*io(spec, 65536, 100)) == []          # too few rows for two bands
    spec = P.blend()                                                 # stages on several levels
    assert wt.Pipeline(spec).debug_host_bands(*io(spec, 8192, 8192, wt.WT_BF16)) == []
    inp = P.input_id(0)
    b = P.Builder("planes", [3])
    b.output(b.stage("s", P.ref(inp, 0, 1, chan=0) + P.ref(inp, 0, -1, chan=2)))
    spec = b.build()                                                 # a three-plane input
    assert wt.Pipeline(spec).debug_host_bands(*io(spec, 4096, 4096)) == []
    spec = P.unsharp3d(64)                                           # a volume: one input of 64 planes
    assert wt.Pipeline(spec).debug_host_bands(*io(spec, 1024, 1024)) == []


@pytest.mark.parametrize("dy,H", [(1, 16385), (2, 16385), (1, 16386)])
def test_bands_equal_whole_image(dy, H):
    """Each band's kept rows, evaluated by the oracle on the band's
    sub-image, equal the whole image's rows exactly; a sub-image starting
    one row earlier (an odd row) does not, through the row parity."""
    spec = parity_pipeline(dy)
    W = 256
    p = wt.Pipeline(spec)
    bands = p.debug_host_bands(*io(spec, W, H, pitch=W * 4))
    h = row_halo(spec)
    assert h == dy + 1 and len(bands) == 2
    check_plan(bands, H, h)
    a = I.uniform_image(11 + dy, W, H).astype(np.float64)
    whole = O.evaluate(spec["stages"], [a], spec["outputs"])[0]
    for y0, y1, ys, ye in bands:
        sub = O.evaluate(spec["stages"], [a[:, ys:ye]], spec["outputs"])[0]
        assert np.array_equal(sub[:, y0 - ys:y1 - ys], whole[:, y0:y1])
        if ys > 0:
            odd = O.evaluate(spec["stages"], [a[:, ys - 1:ye]], spec["outputs"])[0]
            assert not np.array_equal(odd[:, y0 - ys + 1:y1 - ys + 1], whole[:, y0:y1])

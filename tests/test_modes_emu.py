"""Taps scaling by 4 and 8 (two and three pyramid levels at once) in the
generated kernels: fused groups reading another level's stage (clamped
gathers in border tiles, unclamped ones in interior tiles) and per-stage
kernels, in the block emulator against the FP64 oracle."""
import numpy as np
import pytest

from paper_1909_07190_gb300 import pipelines as P
from paper_1909_07190_gb300 import wt

from test_codegen_emu import oracle_of, rnd, run_emulated


def scaled_spec(k):
    """in -> d (level log2 k: a k x k mean by scale-k taps) -> out (level 0:
    the input minus the coarse value around it, up by k, with offsets)."""
    inp = P.input_id(0)
    b = P.Builder("s%d" % k, [1])
    e = None
    for j in range(0, k, max(1, k // 2)):
        for i in range(0, k, max(1, k // 2)):
            t = P.ref(inp, i, j, mode="down%d" % k)
            e = t if e is None else e + t
    d = b.stage("d", e * 0.25)
    u = b.stage("u", P.ref(inp, 1, 0) - 0.5 * P.ref(d, 0, 0, mode="up%d" % k)
                - 0.25 * P.ref(d, 1, -1, mode="up%d" % k) + P.ref(d, -1, 1, mode="up%d" % k) * P.ref(inp))
    b.output(d, u)
    return b.build()


@pytest.mark.parametrize("k", [4, 8])
@pytest.mark.parametrize("w,h,tile_h,vec", [(67, 45, 8, 4), (1100, 90, 8, 4), (1300, 61, 16, 8), (5, 3, 4, 4)])
def test_scaled_modes_fused(k, w, h, tile_h, vec):
    spec = scaled_spec(k)
    img = rnd(k + w + h, w, h)
    got, d = run_emulated(spec, [img], groups=[0, 1], params=[dict(tile_h=tile_h, vec=vec)] * 2)
    for g, r in zip(got, oracle_of(spec, [img])):
        assert np.abs(g - r).max() <= 1e-5


@pytest.mark.parametrize("k", [4, 8])
def test_scaled_modes_plain(k):
    spec = scaled_spec(k)
    for w, h in [(67, 45), (300, 7), (1, 1)]:
        img = rnd(k + w, w, h)
        got, _ = run_emulated(spec, [img], exec_mode=wt.WT_EXEC_PLAIN)
        for g, r in zip(got, oracle_of(spec, [img])):
            assert np.abs(g - r).max() <= 1e-5

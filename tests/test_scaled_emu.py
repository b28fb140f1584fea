"""The streaming down-sampling kernel (producer rows streamed through each
warp at twice the output rate, separable row and column passes) executed on
the CPU by the block emulator, against the FP64 oracle."""
import numpy as np
import pytest

from paper_1909_07190_gb300 import pipelines as P
from paper_1909_07190_gb300 import wt

from test_codegen_emu import oracle_of, rnd, run_emulated


def down_spec(weights=None, channels=1, in_channels=1, chan=-1, const=0.0, dx0=None, dy0=None):
    """One stage: sum w[j][i] P(2x + dx0 + i, 2y + dy0 + j) + const."""
    w = weights or [[bj * bi for bi in P.BINOMIAL5] for bj in P.BINOMIAL5]
    ny, nx = len(w), len(w[0])
    dx0 = -(nx // 2) if dx0 is None else dx0
    dy0 = -(ny // 2) if dy0 is None else dy0
    b = P.Builder("down", [in_channels])
    e = None
    for j in range(ny):
        for i in range(nx):
            if w[j][i] == 0:
                continue
            t = float(w[j][i]) * P.ref(P.input_id(0), dx0 + i, dy0 + j, chan=chan, mode="down2")
            e = t if e is None else e + t
    if const:
        e = e + const
    b.output(b.stage("d", e, channels))
    return b.build()


def run_down(spec, img, tile_h=14, vec=4, dtype=wt.WT_F32):
    got, d = run_emulated(spec, [img], dtype=dtype, groups=[0], params=[dict(tile_h=tile_h, vec=vec, flags=4)])
    return got[0], d


@pytest.mark.parametrize("w,h", [(1, 1), (2, 3), (37, 23), (300, 77), (513, 9), (257, 130)])
@pytest.mark.parametrize("tile_h,vec", [(14, 4), (1, 4), (5, 8), (32, 8)])
def test_down_binomial_sizes(w, h, tile_h, vec):
    spec = down_spec()
    img = rnd(w * 7 + h, w, h)
    got, d = run_down(spec, img, tile_h, vec)
    assert d["name"].startswith("wt_down_")
    assert np.abs(got - oracle_of(spec, [img])[0]).max() <= 1e-6


@pytest.mark.parametrize("weights,dx0,dy0", [
    ([[1, 3, 3, 1]] * 4, -1, -2),                 # even tap count (odd row span)
    ([[1, 2, 1]], -2, 0),                          # taps left of the centre only
    ([[2], [1], [3]], 0, 1),                       # one column, rows below
    ([[1, 1]], 1, -3),                             # right of the centre
    ([[w * v for w in (1, -2, 3, -2, 1)] for v in (1, 0, 2, 0, -1, 0.5)], -3, -2),
])
def test_down_tap_patterns(weights, dx0, dy0):
    spec = down_spec(weights, dx0=dx0, dy0=dy0, const=0.25)
    for (w, h) in [(300, 41), (9, 7)]:
        img = rnd(w + 3 * h + dx0, w, h)
        got, d = run_down(spec, img, 6, 4)
        assert d["name"].startswith("wt_down_")
        ref = oracle_of(spec, [img])[0]
        assert np.abs(got - ref).max() <= 1e-5 * max(1.0, np.abs(ref).max())


def test_down_channels_and_fixed_channel():
    spec = down_spec(channels=3, in_channels=3)
    img = rnd(70, 333, 65, 3)
    got, d = run_down(spec, img)
    assert tuple(d["grid"])[2] == 3
    assert np.abs(got - oracle_of(spec, [img])[0]).max() <= 1e-6
    spec = down_spec(channels=1, in_channels=3, chan=2)
    got, _ = run_down(spec, img)
    assert np.abs(got - oracle_of(spec, [img])[0]).max() <= 1e-6


@pytest.mark.parametrize("dtype,tol", [(wt.WT_BF16, 1.6e-2), (wt.WT_F16, 2e-3)])
def test_down_16bit(dtype, tol):
    spec = down_spec()
    name = {wt.WT_F16: "f16", wt.WT_BF16: "bf16"}[dtype]
    img = rnd(71, 517, 99, 1, name)
    got, _ = run_down(spec, img, 14, 4, dtype)
    assert np.abs(got - oracle_of(spec, [img])[0]).max() <= tol


def test_down_not_streamed():
    """Non-separable weights, non-linear stages and same-level stages run
    the plain per-stage kernel; the unfused execution mode never streams."""
    spec = down_spec([[1, 2, 0], [0, 1, 3], [1, 0, 1]])
    img = rnd(72, 64, 40)
    got, d = run_down(spec, img)
    assert d["name"].startswith("wt_plain_")
    assert np.abs(got - oracle_of(spec, [img])[0]).max() <= 1e-5
    spec = down_spec()
    got, d = run_emulated(spec, [img], exec_mode=wt.WT_EXEC_PLAIN)
    assert d["name"].startswith("wt_plain_")


def test_blend_default_schedule_streams_downs():
    """The blend's default schedule: its per-stage down-sampling groups use
    the streaming kernel; the whole blend against the oracle."""
    spec = P.blend()
    w, h = 131, 67
    A, B = rnd(73, w, h, 3), rnd(74, w, h, 3)
    from paper_1909_07190_gb300 import inputs as I
    M = I.smooth_mask(75, w, h)
    groups, params = P.blend_schedule()
    got, d = run_emulated(spec, [A, B, M], groups=groups, params=params)
    assert np.abs(got[0] - oracle_of(spec, [A, B, M])[0]).max() <= 1e-5


@pytest.mark.parametrize("w,h,tile_h,vec,nbuf", [(1100, 37, 14, 4, 2), (1100, 9, 3, 8, 1), (2100, 21, 5, 4, 5),
                                                 (2100, 40, 32, 8, 2)])
@pytest.mark.parametrize("dtype,tol", [(wt.WT_F32, 1e-6), (wt.WT_BF16, 1.6e-2)])
def test_down_ring_path(w, h, tile_h, vec, nbuf, dtype, tol):
    """Images wide enough that interior warps take the cp.async ring path
    (their columns and both 16-byte halo chunks inside the row), with ring
    lengths from 1 to 5 steps ahead, next to clamped border warps."""
    spec = down_spec(channels=3, in_channels=3)
    name = {wt.WT_F32: "f32", wt.WT_BF16: "bf16"}[dtype]
    img = rnd(w + h + nbuf, w, h, 3, name)
    got, d = run_emulated(spec, [img], dtype=dtype, groups=[0],
                          params=[dict(tile_h=tile_h, vec=vec, n_buffers=nbuf, flags=4)])
    assert d["smem"] > 0
    assert np.abs(got[0] - oracle_of(spec, [img])[0]).max() <= tol


def test_down_ring_odd_taps():
    """Ring path with an even tap count (odd row span: two open output rows)
    and taps right of the centre only."""
    for weights, dx0, dy0 in [([[1, 3, 3, 1]] * 4, -1, -2), ([[1, 1, 2]], 1, -3)]:
        spec = down_spec(weights, dx0=dx0, dy0=dy0, const=-0.5)
        img = rnd(77 + dx0, 1500, 23)
        got, _ = run_down(spec, img, 7, 4)
        ref = oracle_of(spec, [img])[0]
        assert np.abs(got - ref).max() <= 1e-5 * max(1.0, np.abs(ref).max())

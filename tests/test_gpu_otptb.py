"""GPU parity of the block-tile kernel (one overlapped tile per thread
block, block barriers between stages; the tiling the paper compares against
in Sec. 3 and Sec. 7) against the FP64 oracle, and against the warp-tiled
kernel at full size.

Tolerances as in the other parity tests: FP32 storage 1e-5 (relative to
max |oracle| for the unnormalised corner response), FP16 2e-3.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1909_07190_gb300 import inputs as I
from paper_1909_07190_gb300 import pipelines as P

from test_gpu_parity import oracle_out, rnd, run_pipe, wtmod

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def blk(tile_h=16, warps=8, vec=4):
    return dict(tile_h=tile_h, warps_per_block=warps, vec=vec, flags=wtmod().WT_FLAG_OTPTB)


@pytest.mark.parametrize("name", ["sharpen", "harris", "blur"])
@pytest.mark.parametrize("w,h", [(1, 1), (129, 33), (1000, 517)])
@pytest.mark.parametrize("tile_h,warps,vec", [(16, 8, 4), (8, 4, 1), (32, 8, 8)])
def test_otptb_parity(name, w, h, tile_h, warps, vec):
    spec = P.by_name(name)
    img = rnd(w + 3 * h + tile_h, w, h)
    got, p = run_pipe(spec, [img], params=[blk(tile_h, warps, vec)])
    assert p.launches_per_run() == 1
    ref = oracle_out(spec, [img])
    for g, r in zip(got, ref):
        assert np.abs(g - r).max() <= 1e-5 * max(1.0, np.abs(r).max())


def test_otptb_f16_and_mixed_schedule():
    spec = P.harris()
    img = rnd(61, 333, 211, dtype="f16")
    got = run_pipe(spec, [img], dtype="f16", params=[blk(16, 8, 8)])[0][0]
    assert np.abs(got - oracle_out(spec, [img])[0]).max() <= 2e-3
    img = rnd(62, 333, 211)
    got = run_pipe(spec, [img], groups=[0] * 5 + [1] * 6, params=[blk(8, 4), dict(tile_h=16)])[0][0]
    ref = oracle_out(spec, [img])[0]
    assert np.abs(got - ref).max() <= 1e-5 * max(1.0, np.abs(ref).max())


def test_otptb_full_size_harris_matches_warp_tiles():
    """4096x4096 corner response: block tiles against the oracle on sampled
    points (corners, edges, interior) and against the warp-tiled kernel on
    every pixel."""
    spec = P.harris()
    W = H = 4096
    img = rnd(I.SEED_BASE + 2, W, H)
    got = run_pipe(spec, [img], params=[blk(32, 8, 4)])[0][0]
    rng = np.random.default_rng(3)
    xs = np.concatenate([rng.integers(0, W, 300), [0, W - 1, 0, W - 1, 127, 128]])
    ys = np.concatenate([rng.integers(0, H, 300), [0, H - 1, H - 1, 0, 31, 32]])
    ref = O.evaluate_points(spec["stages"], [img.astype(np.float64)], spec["outputs"][0], xs, ys)
    assert np.abs(got[0][ys, xs] - ref).max() <= 1e-5 * max(1.0, np.abs(ref).max())
    warp = run_pipe(spec, [img], params=[dict(tile_h=14)])[0][0]
    assert np.abs(got - warp).max() <= 2e-5 * max(1.0, np.abs(warp).max())

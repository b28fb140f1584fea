"""GPU parity of the streaming down-sampling kernel (separable DOWN2
stencils run per stage inside a warp-tiled schedule) against the FP64
oracle: small ragged sizes on every pixel, a large image on sampled pixels.

Tolerances: FP32 storage 1e-6 max abs (weights sum to 1 on [0,1) data),
BF16 storage 1.6e-2.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1909_07190_gb300 import pipelines as P

from test_gpu_parity import oracle_out, rnd, run_pipe

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def down_spec(channels=1):
    b = P.Builder("down", [channels])
    b.output(b.stage("d", P._down(P.input_id(0)), channels))
    return b.build()


@pytest.mark.parametrize("w,h", [(1, 1), (3, 2), (129, 77), (1000, 517), (4097, 31)])
@pytest.mark.parametrize("tile_h,vec", [(14, 4), (3, 8), (32, 4)])
@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_down_stream_parity(w, h, tile_h, vec, dtype):
    spec = down_spec(3)
    img = rnd(w + h + tile_h, w, h, 3, dtype)
    got = run_pipe(spec, [img], dtype=dtype, groups=[0], params=[dict(tile_h=tile_h, vec=vec, flags=4)])[0][0]
    tol = 1e-6 if dtype == "f32" else 1.6e-2
    assert np.abs(got - oracle_out(spec, [img])[0]).max() <= tol


def test_down_stream_8192_sampled():
    """8192x8192x3 BF16, the blend's level-1 reduce: sampled outputs
    (corners, edges, interior) against the oracle on windows."""
    spec = down_spec(3)
    W = H = 8192
    img = rnd(91, W, H, 3, "bf16")
    got = run_pipe(spec, [img], dtype="bf16", groups=[0], params=[dict(flags=4)])[0][0]
    rng = np.random.default_rng(9)
    pts = [(0, 0), (4095, 4095), (4095, 0), (0, 4095), (17, 2049)]
    pts += [(int(rng.integers(0, 4096)), int(rng.integers(0, 4096))) for _ in range(20)]
    worst = 0.0
    for xo, yo in pts:
        x0, y0 = max(0, 2 * xo - 8), max(0, 2 * yo - 8)
        x1, y1 = min(W, 2 * xo + 9), min(H, 2 * yo + 9)
        # a window starting on even coordinates keeps the down-sampling grid
        x0 -= x0 % 2
        y0 -= y0 % 2
        win = img[:, y0:y1, x0:x1].astype(np.float64)
        ref = O.evaluate_points(spec["stages"], [win], spec["outputs"][0], np.array([xo - x0 // 2] * 3),
                                np.array([yo - y0 // 2] * 3), np.array([0, 1, 2]))
        worst = max(worst, float(np.abs(got[:, yo, xo] - ref).max()))
    assert worst <= 1.6e-2, worst

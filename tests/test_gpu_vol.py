"""GPU parity of 3-D groups (App. A generalised hybrid tiling: warp tiles
streaming rows or planes, the third axis a register tile) against the FP64
oracle: both split axes, tile shapes, 16-bit storage, ragged volumes, the
unfused per-stage path, and sampled points of a full-size 512x512x256
volume in the launch configuration the 3-D study times.

Tolerance: FP32 storage, 1e-5 relative to max |oracle|; FP16 2e-3 and
BF16 1.6e-2 absolute on [0, 1) data (one rounding of the output)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1909_07190_gb300 import inputs as I
from paper_1909_07190_gb300 import pipelines as P

from test_gpu_parity import oracle_out, rnd, run_pipe, wtmod

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def vparams(split, tile_o=4, vec=2, tile_h=16, warps=4, staged=False):
    """staged: sources in the warp's shared memory (frac_reg < 1)."""
    return dict(tile_h=tile_h, tile_o=tile_o, vec=vec, warps_per_block=warps, flags=32 if split else 0,
                frac_reg=0.0 if staged else 1.0)


def close(got, ref, rel=1e-5):
    return np.abs(got - ref).max() <= rel * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("split", [0, 1])
@pytest.mark.parametrize("W,H,D", [(1, 1, 1), (333, 97, 19), (1000, 13, 9), (64, 200, 70)])
def test_heat_fused_gpu(split, W, H, D):
    spec = P.heat3d(2, depth=D)
    img = rnd(W + H + D, W, H, D)
    got, p = run_pipe(spec, [img], params=[vparams(split)])
    assert p.launches_per_run() == 1
    assert close(got[0], oracle_out(spec, [img])[0])


@pytest.mark.parametrize("split", [0, 1])
@pytest.mark.parametrize("tile_o,vec,tile_h", [(1, 1, 1), (2, 2, 7), (8, 1, 32), (4, 2, 64), (1, 2, 16)])
def test_unsharp_fused_gpu(split, tile_o, vec, tile_h):
    D = 21
    spec = P.unsharp3d(depth=D)
    img = rnd(3 + tile_o * vec + tile_h, 301, 77, D)
    got, p = run_pipe(spec, [img], params=[vparams(split, tile_o, vec, tile_h)])
    assert p.launches_per_run() == 1
    assert close(got[0], oracle_out(spec, [img])[0])


@pytest.mark.parametrize("dtype,tol", [("f16", 2e-3), ("bf16", 1.6e-2)])
def test_sixteen_bit_storage_gpu(dtype, tol):
    D = 12
    spec = P.unsharp3d(depth=D)
    img = rnd(4, 200, 60, D, dtype=dtype)
    got, _ = run_pipe(spec, [img], dtype=dtype, params=[vparams(1)])
    assert np.abs(got[0] - oracle_out(spec, [img])[0]).max() <= tol


def test_plain_path_gpu():
    D = 10
    spec = P.heat3d(3, depth=D)
    img = rnd(5, 150, 45, D)
    got, p = run_pipe(spec, [img], exec_mode=wtmod().WT_EXEC_PLAIN)
    assert p.launches_per_run() == 3
    assert close(got[0], oracle_out(spec, [img])[0])


@pytest.mark.parametrize("name,split", [("unsharp3d", 1), ("heat3d", 0)])
def test_full_size_sampled(name, split):
    """512 x 512 x 256 FP32, the 3-D study's default tiles: 4000 sampled
    voxels (every plane class: first, last, interior) against the oracle
    evaluated at those points only."""
    W = H = 512
    D = 256
    spec = P.unsharp3d(depth=D) if name == "unsharp3d" else P.heat3d(2, depth=D)
    img = I.uniform_image(I.SEED_BASE + 8, W, H, D)
    got, p = run_pipe(spec, [img], params=[vparams(split)])
    assert p.launches_per_run() == 1
    rng = np.random.default_rng(3)
    n = 4000
    xs = rng.integers(0, W, n)
    ys = rng.integers(0, H, n)
    zs = rng.integers(0, D, n)
    xs[:8], ys[:8], zs[:8] = [0, W - 1, 0, W - 1, 0, 5, 511, 300], [0, 0, H - 1, H - 1, 7, 0, 511, 2], \
        [0, D - 1, D - 1, 0, 1, 254, 128, 255]
    ref = O.evaluate_points(spec["stages"], [img.astype(np.float64)], spec["outputs"][0], xs, ys, zs)
    g = got[0][zs, ys, xs]
    assert np.abs(g - ref).max() <= 1e-5 * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("split", [0, 1])
@pytest.mark.parametrize("vec,W", [(1, 333), (2, 1000), (4, 77)])
def test_staged_sources_gpu(split, vec, W):
    """Sources staged in shared memory by asynchronous copies (frac_reg 0)."""
    D = 13
    spec = P.unsharp3d(depth=D)
    img = rnd(40 + vec, W, 61, D)
    got, p = run_pipe(spec, [img], params=[vparams(split, 2, vec, 16, staged=True)])
    assert p.launches_per_run() == 1
    assert close(got[0], oracle_out(spec, [img])[0])


def test_staged_full_size_sampled():
    W = H = 512
    D = 256
    spec = P.heat3d(2, depth=D)
    img = I.uniform_image(I.SEED_BASE + 8, W, H, D)
    got, p = run_pipe(spec, [img], params=[vparams(1, 4, 1, 64, staged=True)])
    assert p.launches_per_run() == 1
    rng = np.random.default_rng(5)
    xs, ys, zs = rng.integers(0, W, 3000), rng.integers(0, H, 3000), rng.integers(0, D, 3000)
    ref = O.evaluate_points(spec["stages"], [img.astype(np.float64)], spec["outputs"][0], xs, ys, zs)
    assert np.abs(got[0][zs, ys, xs] - ref).max() <= 1e-5 * max(1.0, np.abs(ref).max())

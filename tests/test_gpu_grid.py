"""GPU parity of per-plane programs (the channel-index op) and of the
bilateral grid and filter (histogram as a splat-and-sum reduction, 2x2
sums, a blur of the grid, slicing) against the FP64 oracle.

Tolerance: FP32 storage, 1e-5 relative to max |oracle| (grid cells hold
sums of up to 64 pixels)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1909_07190_gb300 import inputs as I
from paper_1909_07190_gb300 import pipelines as P

from test_gpu_parity import oracle_out, rnd, run_pipe, wtmod
from test_grid_emu import chan_spec, grid_groups

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def close(got, ref, rel=1e-5):
    return np.abs(got - ref).max() <= rel * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("mode", ["fused", "plain", "otptb"])
def test_chan_op_gpu(mode):
    wt = wtmod()
    spec = chan_spec()
    img = rnd(90, 333, 129)
    if mode == "plain":
        got = run_pipe(spec, [img], exec_mode=wt.WT_EXEC_PLAIN)[0]
    elif mode == "otptb":
        got = run_pipe(spec, [img], groups=[0, 1, 1],
                       params=[dict(tile_h=8, warps_per_block=4, flags=wt.WT_FLAG_OTPTB)] * 2)[0]
    else:
        got = run_pipe(spec, [img], groups=[0, 1, 1], params=[dict(tile_h=8)] * 2)[0]
    for g, r in zip(got, oracle_out(spec, [img])):
        assert close(g, r)


@pytest.mark.parametrize("w,h", [(1000, 517), (67, 45)])
def test_bilateral_grid_gpu(w, h):
    spec = P.bilateral_grid()
    img = rnd(91 + w, w, h)
    g = grid_groups(spec)
    got = run_pipe(spec, [img], groups=g, params=[dict(tile_h=8)] * (max(g) + 1))[0][0]
    assert close(got, oracle_out(spec, [img])[0])


@pytest.mark.parametrize("w,h", [(1000, 517), (131, 67)])
def test_bilateral_filter_default_schedule(w, h):
    spec = P.bilateral_filter()
    img = rnd(92 + w, w, h)
    groups, params = P.bilateral_schedule()
    got, p = run_pipe(spec, [img], groups=groups, params=params)
    assert p.launches_per_run() == 3
    assert close(got[0], oracle_out(spec, [img])[0])
    plain = run_pipe(spec, [img], exec_mode=wtmod().WT_EXEC_PLAIN)[0][0]
    assert close(plain, got[0])


def test_bilateral_filter_4096_sampled():
    """The bench workload (4096x4096 FP32): sampled outputs (corners, edges,
    interior) against the oracle's region-restricted evaluation."""
    spec = P.bilateral_filter()
    W = H = 4096
    img = rnd(I.SEED_BASE + 6, W, H)
    groups, params = P.bilateral_schedule()
    got = run_pipe(spec, [img], groups=groups, params=params)[0][0]
    rng = np.random.default_rng(6)
    xs = np.concatenate([rng.integers(0, W, 60), [0, W - 1, 0, W - 1, 7, 8]])
    ys = np.concatenate([rng.integers(0, H, 60), [0, H - 1, H - 1, 0, 4095, 9]])
    ref = O.evaluate_points(spec["stages"], [img.astype(np.float64)], spec["outputs"][0], xs, ys)
    assert np.abs(got[0][ys, xs] - ref).max() <= 1e-5


@pytest.mark.parametrize("k", [4, 8])
@pytest.mark.parametrize("w,h", [(1000, 517), (67, 45)])
def test_scaled_modes_gpu(k, w, h):
    """Taps scaling by 4 and 8: fused groups with gathers of another level
    two or three levels away, and per-stage kernels."""
    from test_modes_emu import scaled_spec
    wt = wtmod()
    spec = scaled_spec(k)
    img = rnd(k * 7 + w, w, h)
    got = run_pipe(spec, [img], groups=[0, 1], params=[dict(tile_h=8)] * 2)[0]
    plain = run_pipe(spec, [img], exec_mode=wt.WT_EXEC_PLAIN)[0]
    for g, q, r in zip(got, plain, oracle_out(spec, [img])):
        assert np.abs(g - r).max() <= 1e-5 and np.abs(q - r).max() <= 1e-5


def test_tune_finds_reduction_chain():
    """The measured search keeps the grid's splat and 2x2 sums as one
    cross-level group and keeps parity."""
    wt = wtmod()
    spec = P.bilateral_filter()
    W, H = 2048, 1024
    img = rnd(93, W, H)
    p = wt.Pipeline(spec)
    x = wt.DeviceImage(1, H, W).upload(img)
    y = wt.DeviceImage(1, H, W)
    s = torch.cuda.current_stream().cuda_stream
    ms, n = p.schedule_tune([x.image()], [y.image()], 0, 4, 5, s)
    assert n > 0 and ms > 0
    assert p.launches_per_run() <= 4, p.schedule_get()["groups"]
    p.run([x.image()], [y.image()], s)
    p.check(s)
    got = y.download()[0]
    assert close(got, oracle_out(spec, [img])[0])


@pytest.mark.parametrize("model", ["analytic", "learned"])
def test_dp_fusion_proposes_cross_level_group(model):
    """DP-Fusion with either cost model puts the grid's splat and its 2x2
    sums (three levels) into one group, run as the reduction-chain kernel,
    and the 4096x4096 filter it schedules matches the oracle at sampled
    points."""
    import os
    wt = wtmod()
    spec = P.bilateral_filter()
    W = H = 4096
    img = rnd(I.SEED_BASE + 6, W, H)
    p = wt.Pipeline(spec)
    if model == "learned":
        wt.costmodel_load(os.path.join(os.path.dirname(wt.__file__), "costmodel_gb300.txt"))
    try:
        p.schedule_auto(W, H, wt.WT_F32, wt.WT_MODEL_LEARNED if model == "learned" else wt.WT_MODEL_ANALYTIC)
    finally:
        wt.costmodel_reset()
    groups = p.schedule_get()["groups"]
    assert groups[0] == groups[1] == groups[2] and groups[3] != groups[2], groups
    x = wt.DeviceImage(1, H, W).upload(img)
    y = wt.DeviceImage(1, H, W)
    assert p.kernel_name(0, [x.image()], [y.image()]).startswith("wt_chain_")
    s = torch.cuda.current_stream().cuda_stream
    p.run([x.image()], [y.image()], s)
    p.check(s)
    rng = np.random.default_rng(16)
    xs = np.concatenate([rng.integers(0, W, 60), [0, W - 1, 0, W - 1]])
    ys = np.concatenate([rng.integers(0, H, 60), [0, H - 1, H - 1, 0]])
    ref = O.evaluate_points(spec["stages"], [img.astype(np.float64)], spec["outputs"][0], xs, ys)
    assert np.abs(y.download()[0][ys, xs] - ref).max() <= 1e-5

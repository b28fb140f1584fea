"""GPU parity: every path of the library (fused warp-tiled groups, per-stage
plain kernels, mixed groupings, hybrid register/shared splits, 16-bit storage,
host-buffer runs) against the FP64 oracle, through the C ABI.

Tolerances: FP32 storage 1e-5 max abs on [0,1) data (normalised pipelines);
FP16 storage 2e-3; BF16 storage 1.6e-2; the unnormalised corner response
1e-5 relative to max |oracle| (its values reach ~1e4).
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1909_07190_gb300 import inputs as I
from paper_1909_07190_gb300 import pipelines as P

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"f32": 1e-5, "f16": 2e-3, "bf16": 1.6e-2}


def wtmod():
    from paper_1909_07190_gb300 import wt
    return wt


def stream():
    return torch.cuda.current_stream().cuda_stream


def oracle_out(spec, imgs):
    return O.evaluate(spec["stages"], [np.asarray(a, np.float64) for a in imgs], spec["outputs"])


def run_pipe(spec, imgs, dtype="f32", out_dtype=None, groups=None, params=None, exec_mode=0, mid=-1):
    wt = wtmod()
    dt = wt.DTYPES[dtype]
    odt = wt.DTYPES[out_dtype or dtype]
    p = wt.Pipeline(spec)
    if exec_mode == wt.WT_EXEC_PLAIN:
        p.schedule(exec_mode=exec_mode, intermediate_dtype=mid)
    else:
        p.schedule(groups=groups, params=params, intermediate_dtype=mid)
    shapes = O.shapes(spec["stages"], [np.zeros((c, imgs[0].shape[-2], imgs[0].shape[-1]))
                                       for c in spec["inputs"]])
    ins = []
    for a, c in zip(imgs, spec["inputs"]):
        a = np.asarray(a, np.float32).reshape(c, a.shape[-2], a.shape[-1])
        ins.append(wt.DeviceImage(c, a.shape[1], a.shape[2], dt).upload(a))
    outs = []
    for sid in spec["outputs"]:
        _, w, h, c = shapes[sid]
        outs.append(wt.DeviceImage(c, h, w, odt))
    p.run([x.image() for x in ins], [x.image() for x in outs], stream())
    p.check(stream())
    return [o.download() for o in outs], p


def rnd(seed, w, h, c=1, dtype="f32"):
    return I.round_to(I.uniform_image(seed, w, h, c), dtype)


SIZES = [(1, 1), (7, 5), (150, 70), (257, 33), (600, 411), (121, 129)]


@pytest.mark.parametrize("name", ["sharpen", "harris", "blur"])
@pytest.mark.parametrize("w,h", SIZES)
def test_fused_default(name, w, h):
    spec = P.by_name(name)
    img = rnd(100 + w, w, h)
    got = run_pipe(spec, [img])[0][0]
    ref = oracle_out(spec, [img])[0]
    assert np.abs(got - ref).max() <= TOL["f32"]


@pytest.mark.parametrize("tile_h", [1, 3, 16, 64])
@pytest.mark.parametrize("frac", [0.0, 0.5, 1.0])
@pytest.mark.parametrize("vec", [4, 8])
def test_fused_params_harris(tile_h, frac, vec):
    spec = P.harris()
    img = rnd(7, 333, 97)
    prm = [dict(tile_h=tile_h, frac_reg=frac, vec=vec, warps_per_block=2)]
    got = run_pipe(spec, [img], params=prm)[0][0]
    ref = oracle_out(spec, [img])[0]
    assert np.abs(got - ref).max() <= TOL["f32"]


@pytest.mark.parametrize("groups", [
    [0, 0, 1, 1, 1, 2, 2, 2, 3, 3, 3],
    [0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10],
    [0, 0, 0, 0, 0, 1, 1, 1, 1, 1, 1],
])
def test_harris_groupings(groups):
    spec = P.harris()
    img = rnd(8, 260, 150)
    ng = max(groups) + 1
    got = run_pipe(spec, [img], groups=groups, params=[dict(tile_h=8, warps_per_block=4)] * ng)[0][0]
    ref = oracle_out(spec, [img])[0]
    assert np.abs(got - ref).max() <= TOL["f32"]


@pytest.mark.parametrize("name", ["sharpen", "harris"])
def test_plain_path(name):
    wt = wtmod()
    spec = P.by_name(name)
    img = rnd(9, 301, 77)
    got = run_pipe(spec, [img], exec_mode=wt.WT_EXEC_PLAIN)[0][0]
    ref = oracle_out(spec, [img])[0]
    assert np.abs(got - ref).max() <= TOL["f32"]


def test_harris_raw_relative():
    spec = P.harris(normalized=False)
    img = rnd(10, 200, 120)
    got = run_pipe(spec, [img])[0][0]
    ref = oracle_out(spec, [img])[0]
    assert np.abs(got - ref).max() <= 1e-5 * np.abs(ref).max()


@pytest.mark.parametrize("dtype", ["f16", "bf16"])
@pytest.mark.parametrize("vec", [4, 8])
def test_harris_16bit_storage(dtype, vec):
    spec = P.harris()
    img = rnd(11, 300, 100, dtype=dtype)
    got = run_pipe(spec, [img], dtype=dtype, params=[dict(tile_h=16, vec=vec)])[0][0]
    ref = oracle_out(spec, [img])[0]
    assert np.abs(got - ref).max() <= TOL[dtype]


def test_blend_plain_small():
    wt = wtmod()
    spec = P.blend()
    A = rnd(12, 70, 45, 3)
    B = rnd(13, 70, 45, 3)
    M = I.smooth_mask(14, 70, 45)
    got = run_pipe(spec, [A, B, M], exec_mode=wt.WT_EXEC_PLAIN)[0][0]
    ref = oracle_out(spec, [A, B, M])[0]
    assert np.abs(got - ref).max() <= TOL["f32"]


def test_blend_default_schedule_bf16():
    spec = P.blend()
    A = rnd(15, 96, 80, 3, "bf16")
    B = rnd(16, 96, 80, 3, "bf16")
    M = I.round_to(I.smooth_mask(17, 96, 80), "bf16")
    got = run_pipe(spec, [A, B, M], dtype="bf16", mid=0)[0][0]
    ref = oracle_out(spec, [A, B, M])[0]
    assert np.abs(got - ref).max() <= TOL["bf16"]


def test_run_host_matches_device():
    wt = wtmod()
    spec = P.harris()
    W, H = 517, 211
    img = rnd(18, W, H)
    p = wt.Pipeline(spec)
    hin = wt.DeviceImage(1, H, W, device="cpu", pin_host=True)
    hin.view().copy_(torch.from_numpy(img))
    hout = wt.DeviceImage(1, H, W, device="cpu", pin_host=True)
    p.run_host([hin.image()], [hout.image()], stream())
    ref = oracle_out(spec, [img])[0]
    assert np.abs(hout.view().numpy()[0] - ref).max() <= TOL["f32"]


def test_full_size_sharpen_sampled():
    spec = P.sharpen()
    W = H = 2048
    img = rnd(I.SEED_BASE + 1, W, H)
    got = run_pipe(spec, [img], params=[dict(tile_h=32)])[0][0]
    rng = np.random.default_rng(1)
    xs = np.concatenate([rng.integers(0, W, 400), [0, W - 1, 0, W - 1]])
    ys = np.concatenate([rng.integers(0, H, 400), [0, H - 1, H - 1, 0]])
    ref = O.evaluate_points(spec["stages"], [img.astype(np.float64)], spec["outputs"][0], xs, ys)
    assert np.abs(got[0][ys, xs] - ref).max() <= TOL["f32"]


@pytest.mark.parametrize("dtype", ["f32", "f16"])
def test_full_size_harris_sampled_and_plain_equal(dtype):
    wt = wtmod()
    spec = P.harris()
    W = H = 4096
    img = rnd(I.SEED_BASE + 2, W, H, dtype=dtype)
    fused = run_pipe(spec, [img], dtype=dtype, params=[dict(tile_h=32)])[0][0]
    rng = np.random.default_rng(2)
    xs = np.concatenate([rng.integers(0, W, 300), [0, W - 1, 0, W - 1, 5, W - 3]])
    ys = np.concatenate([rng.integers(0, H, 300), [0, H - 1, H - 1, 0, H - 2, 3]])
    ref = O.evaluate_points(spec["stages"], [img.astype(np.float64)], spec["outputs"][0], xs, ys)
    assert np.abs(fused[0][ys, xs] - ref).max() <= TOL[dtype]
    if dtype == "f32":
        plain = run_pipe(spec, [img], exec_mode=wt.WT_EXEC_PLAIN)[0][0]
        assert np.abs(fused - plain).max() <= 2 * TOL["f32"]


def test_error_word_clear_after_runs():
    wt = wtmod()
    spec = P.sharpen()
    img = rnd(19, 64, 64)
    _, p = run_pipe(spec, [img])
    p.check(stream())


@pytest.mark.parametrize("name,groups", [("sharpen", [0, 1, 2]), ("harris", list(range(11))),
                                         ("harris", [0] * 5 + [1] * 6)])
@pytest.mark.parametrize("tile_h,frac", [(4, 0.0), (16, 0.5), (16, 1.0)])
def test_multi_group_schedules(name, groups, tile_h, frac):
    """Groups exchanging intermediates through the workspace, with
    shared-memory source windows (fracReg 0) and short tiles."""
    spec = P.by_name(name)
    img = rnd(300 + tile_h, 1000, 333)
    ng = max(groups) + 1
    got = run_pipe(spec, [img], groups=groups, params=[dict(tile_h=tile_h, frac_reg=frac)] * ng)[0][0]
    assert np.abs(got - oracle_out(spec, [img])[0]).max() <= TOL["f32"]


@pytest.mark.parametrize("frac", [0.0, 0.5])
@pytest.mark.parametrize("dtype", ["f16", "bf16"])
def test_16bit_shared_windows(frac, dtype):
    """Intermediates' shared-memory windows stored in the 16-bit storage
    type, corner response against the oracle at the storage tolerance."""
    wt = wtmod()
    spec = P.harris()
    img = rnd(97, 1000, 517, dtype=dtype)
    got = run_pipe(spec, [img], dtype=dtype,
                   params=[dict(tile_h=16, frac_reg=frac, flags=wt.WT_FLAG_SMEM16)])[0][0]
    ref = oracle_out(spec, [img])[0]
    assert np.abs(got - ref).max() <= TOL[dtype] * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("name,dtype,W,H", [("harris", "f32", 4096, 4096), ("harris", "f16", 4096, 4096),
                                            ("sharpen", "f32", 2048, 2048)])
def test_bench_default_schedule_full_size_sampled(name, dtype, W, H):
    """The schedule bench.py times (the library's default, installed at
    pipeline creation) at the benchmark's full size, sampled against the
    oracle point by point: the four corners, points along all four edges,
    points on both sides of the warp tiles' seams in x and y, rows of the
    band of short tiles at the top (the persistent queue's last round), and
    several hundred random interior points.  The image spans many times the
    resident warps, so warps take several tiles each."""
    wt = wtmod()
    spec = P.by_name(name)
    img = rnd(I.SEED_BASE + (2 if name == "harris" else 1), W, H, dtype=dtype)
    p = wt.Pipeline(spec)
    prm = p.schedule_get()["params"][0]
    src = wt.DeviceImage(1, H, W, wt.DTYPES[dtype]).upload(img)
    dst = wt.DeviceImage(1, H, W, wt.DTYPES[dtype])
    p.run([src.image()], [dst.image()], stream())
    p.check(stream())
    got = dst.download()[0]
    rng = np.random.default_rng(7)
    T = prm["tile_h"]
    ow = p.debug_layout(0, [src.image()], [dst.image()])["out_w"]
    pts = [(0, 0), (W - 1, 0), (0, H - 1), (W - 1, H - 1)]
    for t in np.linspace(0, 1, 25):
        pts += [(int(t * (W - 1)), 0), (int(t * (W - 1)), H - 1), (0, int(t * (H - 1))), (W - 1, int(t * (H - 1))),
                (int(t * (W - 1)), 1), (W - 2, int(t * (H - 1)))]
    for k in range(1, 12):                       # tile seams in x and y
        x, y = k * ow, k * T
        pts += [(x - 1, int(rng.integers(0, H))), (x, int(rng.integers(0, H))),
                (int(rng.integers(0, W)), y - 1), (int(rng.integers(0, W)), y)]
    pts += [(int(rng.integers(0, W)), int(rng.integers(0, 600))) for _ in range(150)]   # short-tile band
    pts += [(int(rng.integers(0, W)), int(rng.integers(0, H))) for _ in range(400)]
    xs = np.array([q[0] for q in pts])
    ys = np.array([q[1] for q in pts])
    ref = O.evaluate_points(spec["stages"], [img.astype(np.float64)], spec["outputs"][0], xs, ys)
    assert np.isfinite(got[ys, xs]).all()
    assert np.abs(got[ys, xs] - ref).max() <= TOL[dtype]

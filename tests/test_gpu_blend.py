"""The multi-scale blend on the GPU: 36 stages over 6 pyramid levels, fused
as one group per level (taps of the neighbouring level read memory), and
per stage, against the FP64 oracle.

Tolerances: FP32 storage 1e-5, BF16 storage 1.6e-2 max abs (about six
stored BF16 roundings of values up to ~1.3).
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1909_07190_gb300 import inputs as I
from paper_1909_07190_gb300 import pipelines as P

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"f32": 1e-5, "bf16": 1.6e-2}


def stream():
    return torch.cuda.current_stream().cuda_stream


def run_blend(A, B, M, dtype, fused=True, params=None, mixed=False):
    from paper_1909_07190_gb300 import wt
    dt = wt.DTYPES[dtype]
    spec = P.blend()
    p = wt.Pipeline(spec)
    if fused and mixed:
        groups, prm = P.blend_schedule()
        p.schedule(groups=groups, params=[dict(q, **(params or {})) for q in prm])
    elif fused:
        p.schedule(groups=P.blend_groups(), params=[params or {}] * 10)
    else:
        p.schedule(exec_mode=wt.WT_EXEC_PLAIN)
    H, W = A.shape[-2:]
    ins = [wt.DeviceImage(3, H, W, dt).upload(A), wt.DeviceImage(3, H, W, dt).upload(B),
           wt.DeviceImage(1, H, W, dt).upload(M)]
    out = wt.DeviceImage(3, H, W, dt)
    p.run([x.image() for x in ins], [out.image()], stream())
    p.check(stream())
    return out.download(), p


def oracle(A, B, M):
    spec = P.blend()
    return O.evaluate(spec["stages"], [np.asarray(x, np.float64) for x in (A, B, M)], spec["outputs"])[0]


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
@pytest.mark.parametrize("w,h,tile_h", [(80, 50, 8), (333, 141, 14), (1000, 700, 16), (7, 3, 4)])
def test_blend_fused_levels(dtype, w, h, tile_h):
    A = I.round_to(I.uniform_image(11, w, h, 3), dtype)
    B = I.round_to(I.uniform_image(12, w, h, 3), dtype)
    M = I.round_to(I.smooth_mask(13, w, h), dtype)
    got, p = run_blend(A, B, M, dtype, params=dict(tile_h=tile_h))
    assert p.launches_per_run() == 10
    assert np.abs(got - oracle(A, B, M)).max() <= TOL[dtype]


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_blend_default_mixed_schedule(dtype):
    """The default blend schedule: Gaussian levels 1-2 per stage, levels 3-4
    as a cascade group (one launch per image), the other levels fused (15
    launches)."""
    w, h = 555, 301
    A = I.round_to(I.uniform_image(31, w, h, 3), dtype)
    B = I.round_to(I.uniform_image(32, w, h, 3), dtype)
    M = I.round_to(I.smooth_mask(33, w, h), dtype)
    got, p = run_blend(A, B, M, dtype, mixed=True)
    assert p.launches_per_run() == 15
    assert np.abs(got - oracle(A, B, M)).max() <= TOL[dtype]


def test_blend_fused_vs_plain_fp32():
    w, h = 640, 480
    A, B = I.uniform_image(21, w, h, 3), I.uniform_image(22, w, h, 3)
    M = I.smooth_mask(23, w, h)
    fused, _ = run_blend(A, B, M, "f32")
    plain, q = run_blend(A, B, M, "f32", fused=False)
    assert q.launches_per_run() == 36
    ref = oracle(A, B, M)
    assert np.abs(fused - ref).max() <= 1e-5 and np.abs(plain - ref).max() <= 1e-5


def window_oracle(seed_a, seed_b, seed_m, W, H, x, y, r=352):
    """Oracle value of the blend at (x, y) from a window around it.  The
    window starts on a multiple of 32 (2^5: the coarsest level's grid) and
    reaches at least r pixels beyond the point unless cut by the image
    border, where clamp-to-edge applies alike; r exceeds the dependency
    cone of the 6-level pyramid."""
    x0 = max(0, (x - r) // 32 * 32)
    y0 = max(0, (y - r) // 32 * 32)
    x1 = min(W, x + r + 1)
    y1 = min(H, y + r + 1)
    w, h = x1 - x0, y1 - y0

    def win(seed, c):
        out = np.empty((c, h, w), np.float32)
        for ch in range(c):
            for yy in range(h):
                out[ch, yy] = I.uniform01(seed, w, (ch * H + y0 + yy) * W + x0)
        return I.round_to(out, "bf16")

    A, B = win(seed_a, 3), win(seed_b, 3)
    M = I.round_to(I.smooth_mask(seed_m, W, H, region=(x0, y0, w, h)), "bf16")
    spec = P.blend()
    xs = np.array([x - x0] * 3)
    ys = np.array([y - y0] * 3)
    cs = np.array([0, 1, 2])
    return O.evaluate_points(spec["stages"], [A.astype(np.float64), B.astype(np.float64), M.astype(np.float64)],
                             spec["outputs"][0], xs, ys, cs)


def test_blend_8192_bf16_sampled():
    """The multi-scale blend workload: two 8192x8192x3 images and a smooth
    mask, BF16 storage, fused per level.  Inputs drawn on the device with
    the host generator's stream (mask computed on the host); sampled output
    pixels (corners, edges, interior; all channels) against the oracle."""
    from paper_1909_07190_gb300 import wt
    from paper_1909_07190_gb300 import inputs_torch as IT
    W = H = 8192
    sa, sb, sm = I.SEED_BASE + 5, I.SEED_BASE + 5 + 1000, I.SEED_BASE + 5 + 2000
    dt = wt.WT_BF16
    ins = [wt.DeviceImage(3, H, W, dt), wt.DeviceImage(3, H, W, dt), wt.DeviceImage(1, H, W, dt)]
    ins[0].view().copy_(IT.uniform_image(sa, W, H, 3).to(torch.bfloat16))
    ins[1].view().copy_(IT.uniform_image(sb, W, H, 3).to(torch.bfloat16))
    ins[2].view().copy_(torch.from_numpy(I.smooth_mask(sm, W, H)).to(torch.bfloat16))
    out = wt.DeviceImage(3, H, W, dt)
    p = wt.Pipeline(P.blend())
    groups, params = P.blend_schedule()
    p.schedule(groups=groups, params=params)
    p.run([x.image() for x in ins], [out.image()], stream())
    p.check(stream())
    rng = np.random.default_rng(5)
    pts = [(0, 0), (W - 1, H - 1), (W - 1, 0), (0, H - 1), (4095, 17)]
    pts += [(int(rng.integers(0, W)), int(rng.integers(0, H))) for _ in range(5)]
    worst = 0.0
    for (x, y) in pts:
        got = out.t[:, y, x].float().cpu().numpy()
        ref = window_oracle(sa, sb, sm, W, H, x, y)
        worst = max(worst, float(np.abs(got - ref).max()))
    assert worst <= TOL["bf16"], worst

"""GPU parity of the two-level down-sampling cascade (one kernel streams a
producer, writes its reduce S1 and S1's reduce S2) against the FP64 oracle:
small ragged sizes on every pixel of both levels, an 8192x8192x3 BF16 image
on sampled pixels, and the blend under DP-Fusion's own schedule, which
groups the Gaussian levels two by two.

Tolerances: FP32 storage 1e-5 max abs (weights sum to 1 on [0,1) data),
BF16 storage 1.6e-2.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1909_07190_gb300 import inputs as I
from paper_1909_07190_gb300 import pipelines as P

from test_gpu_parity import oracle_out, rnd, run_pipe, stream

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"f32": 1e-5, "bf16": 1.6e-2}


def cascade_spec(c=1):
    b = P.Builder("cascade", [c])
    inp = P.input_id(0)
    d1 = b.stage("d1", P._down(inp), c)
    d2 = b.stage("d2", P._down(d1), c)
    b.output(d1)
    b.output(d2)
    return b.build()


@pytest.mark.parametrize("w,h", [(1, 1), (3, 2), (129, 77), (1000, 517), (4097, 31), (2049, 1030)])
@pytest.mark.parametrize("tile_h,vec", [(3, 4), (8, 8), (16, 4)])
@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_cascade_parity(w, h, tile_h, vec, dtype):
    spec = cascade_spec(3)
    img = rnd(w * 3 + h + tile_h, w, h, 3, dtype)
    got, p = run_pipe(spec, [img], dtype=dtype, groups=[0, 0], params=[dict(tile_h=tile_h, vec=vec)])
    assert p.launches_per_run() == 1
    ref = oracle_out(spec, [img])
    for g, r in zip(got, ref):
        assert np.abs(g - r).max() <= TOL[dtype]


def test_cascade_8192_sampled():
    """8192x8192x3 BF16, the blend's first two reduces in one kernel:
    sampled points of both levels (corners, edges, interior) against the
    oracle on windows of the input aligned to the level-2 grid."""
    from paper_1909_07190_gb300 import wt
    spec = cascade_spec(3)
    W = H = 8192
    img = rnd(93, W, H, 3, "bf16")
    got, p = run_pipe(spec, [img], dtype="bf16", groups=[0, 0], params=[dict(tile_h=8)])
    i0 = wt.image(0x10000000, W, H, 3, wt.WT_BF16, W * 2)
    i1 = wt.image(0x10000000, W // 2, H // 2, 3, wt.WT_BF16, W)
    i2 = wt.image(0x10000000, W // 4, H // 4, 3, wt.WT_BF16, W // 2)
    assert p.kernel_name(0, [i0], [i1, i2]).startswith("wt_down2_")
    rng = np.random.default_rng(11)
    worst = 0.0
    for lvl, size in ((1, 4096), (2, 2048)):
        pts = [(0, 0), (size - 1, size - 1), (size - 1, 0), (0, size - 1), (17, size // 2 + 1)]
        pts += [(int(rng.integers(0, size)), int(rng.integers(0, size))) for _ in range(12)]
        f = 1 << lvl
        for xo, yo in pts:
            # input window around the point, starting on the level's grid
            x0, y0 = max(0, f * xo - 8 * f), max(0, f * yo - 8 * f)
            x0 -= x0 % f
            y0 -= y0 % f
            x1, y1 = min(W, f * xo + 9 * f), min(H, f * yo + 9 * f)
            win = img[:, y0:y1, x0:x1].astype(np.float64)
            ref = O.evaluate_points(spec["stages"], [win], spec["outputs"][lvl - 1],
                                    np.array([xo - x0 // f] * 3), np.array([yo - y0 // f] * 3), np.array([0, 1, 2]))
            worst = max(worst, float(np.abs(got[lvl - 1][:, yo, xo] - ref).max()))
    assert worst <= TOL["bf16"], worst


def test_blend_dp_schedule_cascades_8192_sampled():
    """DP-Fusion's analytic schedule of the 8192x8192 BF16 blend puts the
    Gaussian levels 1-2 and 3-4 into cascade groups; its output at sampled
    pixels against the oracle."""
    from paper_1909_07190_gb300 import wt
    from paper_1909_07190_gb300 import inputs_torch as IT
    from test_gpu_blend import window_oracle
    W = H = 8192
    sa, sb, sm = I.SEED_BASE + 5, I.SEED_BASE + 5 + 1000, I.SEED_BASE + 5 + 2000
    dt = wt.WT_BF16
    ins = [wt.DeviceImage(3, H, W, dt), wt.DeviceImage(3, H, W, dt), wt.DeviceImage(1, H, W, dt)]
    ins[0].view().copy_(IT.uniform_image(sa, W, H, 3).to(torch.bfloat16))
    ins[1].view().copy_(IT.uniform_image(sb, W, H, 3).to(torch.bfloat16))
    ins[2].view().copy_(torch.from_numpy(I.smooth_mask(sm, W, H)).to(torch.bfloat16))
    out = wt.DeviceImage(3, H, W, dt)
    p = wt.Pipeline(P.blend())
    p.schedule_auto(W, H, dt, wt.WT_MODEL_ANALYTIC)
    ii, oo = [x.image() for x in ins], [out.image()]
    names = [p.kernel_name(i, ii, oo) for i in range(p.launches_per_run())]
    assert sum(n.startswith("wt_down2_") for n in names) == 6, names
    p.run(ii, oo, stream())
    p.check(stream())
    rng = np.random.default_rng(6)
    pts = [(0, 0), (W - 1, H - 1), (W - 1, 0), (0, H - 1), (4095, 17)]
    pts += [(int(rng.integers(0, W)), int(rng.integers(0, H))) for _ in range(5)]
    worst = 0.0
    for (x, y) in pts:
        got = out.t[:, y, x].float().cpu().numpy()
        worst = max(worst, float(np.abs(got - window_oracle(sa, sb, sm, W, H, x, y)).max()))
    assert worst <= TOL["bf16"], worst

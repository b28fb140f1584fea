"""The measured schedule search (wt_schedule_tune) and the schedule timer on
the GPU: the schedule it installs is correct against the oracle and at
least as fast as the default one, single images and batches."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1909_07190_gb300 import inputs as I
from paper_1909_07190_gb300 import pipelines as P

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def stream():
    return torch.cuda.current_stream().cuda_stream


@pytest.mark.parametrize("name", ["sharpen", "harris"])
def test_tune_single_image(name):
    from paper_1909_07190_gb300 import wt
    W, H = 1024, 768
    spec = P.by_name(name)
    img = I.uniform_image(41, W, H)[0]
    x = wt.DeviceImage(1, H, W).upload(img)
    y = wt.DeviceImage(1, H, W)
    p = wt.Pipeline(spec)
    t_default = p.schedule_time([x.image()], [y.image()], 0, 10, stream())
    ms, n = p.schedule_tune([x.image()], [y.image()], 0, 4, 10, stream())
    assert n >= 5 and ms > 0
    assert ms <= t_default * 1.10
    s = p.schedule_get()
    assert s["exec"] == wt.WT_EXEC_FUSED
    y.t.zero_()
    p.run([x.image()], [y.image()], stream())
    p.check(stream())
    ref = O.evaluate(spec["stages"], [img[None].astype(np.float64)], spec["outputs"])[0][0]
    assert np.abs(y.download()[0] - ref).max() <= 1e-5


def test_tune_batch():
    from paper_1909_07190_gb300 import wt
    spec = P.harris()
    sizes = [(300, 200), (1000, 57), (64, 900), (777, 777)]
    ins, outs, imgs = [], [], []
    for i, (w, h) in enumerate(sizes):
        a = I.round_to(I.uniform_image(50 + i, w, h)[0], "f16")
        imgs.append(a)
        ins.append(wt.DeviceImage(1, h, w, wt.WT_F16).upload(a))
        outs.append(wt.DeviceImage(1, h, w, wt.WT_F16))
    p = wt.Pipeline(spec)
    ii, oo = [x.image() for x in ins], [x.image() for x in outs]
    ms, n = p.schedule_tune(ii, oo, len(sizes), 3, 5, stream())
    assert n >= 4 and ms > 0
    for o in outs:
        o.t.zero_()
    p.run_batch(ii, oo, len(sizes), stream())
    p.check(stream())
    for a, o in zip(imgs, outs):
        ref = O.evaluate(spec["stages"], [a[None].astype(np.float64)], spec["outputs"])[0][0]
        assert np.abs(o.download()[0] - ref).max() <= 2e-3


def test_prepare_compiles_without_running():
    from paper_1909_07190_gb300 import wt
    spec = P.harris()
    x = wt.DeviceImage(1, 64, 64)
    y = wt.DeviceImage(1, 64, 64)
    p = wt.Pipeline(spec)
    p.prepare([(None, dict(tile_h=8, frac_reg=f)) for f in (0.0, 0.5, 1.0)], [x.image()], [y.image()])


def test_preprocess_stage_microkernels():
    """Sec. 6 preprocessing: each stage's body timed alone; heavier stage
    programs take longer per iteration; the cost model then uses them."""
    from paper_1909_07190_gb300 import wt
    p = wt.Pipeline(P.harris())
    ns, regs = p.preprocess()
    assert len(ns) == 11 and all(t > 0 for t in ns) and all(r >= 1 for r in regs)
    # Ix (six weighted taps) costs more per iteration than Ixx (one product)
    assert ns[0] > ns[2]
    c = p.cost_group(0, 11, dict(tile_h=14), 128, 1024, 1024)
    assert c["feasible"] and c["cost"] > 0

"""The learned cost model on the GPU: the hand-written MLP inference and
training kernels against a plain numpy FP32 implementation of the same
network and Adam update; training on measured launch times; schedules
chosen with the trained model run correctly."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1909_07190_gb300 import inputs as I
from paper_1909_07190_gb300 import pipelines as P

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

F, H = 18, 64


def unpack(p):
    o = 0
    W1 = p[o:o + H * F].reshape(H, F); o += H * F
    b1 = p[o:o + H]; o += H
    W2 = p[o:o + H * H].reshape(H, H); o += H * H
    b2 = p[o:o + H]; o += H
    w3 = p[o:o + H]; o += H
    b3 = p[o]
    return W1, b1, W2, b2, w3, b3


def np_forward(p, x):
    W1, b1, W2, b2, w3, b3 = unpack(p.astype(np.float64))
    a1 = np.maximum(x @ W1.T + b1, 0)
    a2 = np.maximum(a1 @ W2.T + b2, 0)
    return a2 @ w3 + b3, a1, a2


def np_grads(p, x, y):
    W1, b1, W2, b2, w3, b3 = unpack(p.astype(np.float64))
    out, a1, a2 = np_forward(p, x)
    B = x.shape[0]
    g = 2 * (out - y) / B
    d2 = (g[:, None] * w3[None, :]) * (a2 > 0)
    d1 = (d2 @ W2) * (a1 > 0)
    gW1 = d1.T @ x
    gb1 = d1.sum(0)
    gW2 = d2.T @ a1
    gb2 = d2.sum(0)
    gw3 = a2.T @ g
    gb3 = g.sum()
    return np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gw3, [gb3]]), np.mean((out - y) ** 2)


def rand_params(seed):
    rng = np.random.default_rng(seed)
    p = rng.normal(0, 0.3, 64 * 18 + 64 + 64 * 64 + 64 + 64 + 1).astype(np.float32)
    return p


def test_mlp_forward_kernel_matches_numpy():
    from paper_1909_07190_gb300 import wt
    p = rand_params(1)
    x = np.random.default_rng(2).normal(0, 1, (1000, F)).astype(np.float32)
    got = wt.mlp_forward(p, x)
    want = np_forward(p, x.astype(np.float64))[0]
    assert np.abs(got - want).max() <= 1e-4 * (1 + np.abs(want).max())


def test_mlp_training_kernel_matches_numpy_adam():
    from paper_1909_07190_gb300 import wt
    rng = np.random.default_rng(3)
    n, B, steps = 50, 8, 6
    x = rng.normal(0, 1, (n, F)).astype(np.float32)
    y = rng.normal(0, 1, n).astype(np.float32)
    idx = rng.integers(0, n, (steps, B)).astype(np.int32)
    p = rand_params(4)
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    lr, wd, b1, b2, eps = 1e-2, 1e-3, 0.9, 0.999, 1e-8
    # numpy reference of the same steps
    P_ = p.astype(np.float64).copy()
    M_ = np.zeros_like(P_)
    V_ = np.zeros_like(P_)
    nW1 = 64 * 18
    is_w = np.zeros(P_.size, bool)
    is_w[:nW1] = True
    is_w[nW1 + 64:nW1 + 64 + 4096] = True
    is_w[nW1 + 64 + 4096 + 64:nW1 + 64 + 4096 + 64 + 64] = True
    losses = []
    for t in range(steps):
        g, l = np_grads(P_, x[idx[t]].astype(np.float64), y[idx[t]].astype(np.float64))
        losses.append(l)
        g = g + wd * P_ * is_w
        M_ = b1 * M_ + (1 - b1) * g
        V_ = b2 * V_ + (1 - b2) * g * g
        mh = M_ / (1 - b1 ** (t + 1))
        vh = V_ / (1 - b2 ** (t + 1))
        P_ = P_ - lr * mh / (np.sqrt(vh) + eps)
    loss = wt.mlp_train_steps(p, m, v, 0, x, y, idx, lr, wd)
    assert np.allclose(loss, losses, rtol=1e-4, atol=1e-5)
    assert np.abs(p - P_).max() <= 2e-4


def test_costmodel_train_fits_and_saves(tmp_path):
    from paper_1909_07190_gb300 import wt
    rng = np.random.default_rng(5)
    x = rng.normal(0, 1, (2500, F)).astype(np.float32)
    y = (np.sin(x[:, 0]) + 0.5 * x[:, 1] * x[:, 2] + 0.1 * x[:, 3]).astype(np.float32)
    final = wt.costmodel_train(x[:2000], y[:2000], epochs=60, batch=64, lr=3e-3, seed=7)
    assert final < 0.1
    pred = wt.costmodel_predict(x[2000:])
    # held-out error well below the spread of the targets (R^2 > 0.8)
    assert np.sqrt(np.mean((pred - y[2000:]) ** 2)) < 0.45 * np.std(y)
    path = tmp_path / "m.txt"
    wt.costmodel_save(path)
    wt.costmodel_reset()
    assert not wt.costmodel_ready()
    wt.costmodel_load(path)
    assert np.allclose(wt.costmodel_predict(x[2000:]), pred, rtol=1e-5, atol=1e-5)
    wt.costmodel_reset()


def test_learned_schedules_from_measured_launches():
    """Small end-to-end: time the launches of many sharpen and corner
    schedules, train, schedule with the model; the chosen schedule runs and
    matches the oracle."""
    from paper_1909_07190_gb300 import wt
    s = torch.cuda.current_stream().cuda_stream
    feats, ys = [], []
    W, H = 1024, 512
    for name in ("sharpen", "harris"):
        spec = P.by_name(name)
        img = I.uniform_image(60, W, H)[0]
        x = wt.DeviceImage(1, H, W).upload(img)
        y = wt.DeviceImage(1, H, W)
        n = len(spec["stages"])
        groupings = [[0] * n, list(range(n))]
        if n > 3:
            groupings.append([0] * (n // 2) + [1] * (n - n // 2))
        for g in groupings:
            for T in (4, 16):
                for fr in (0.0, 1.0):
                    p = wt.Pipeline(spec)
                    ng = max(g) + 1
                    p.schedule(groups=g, params=[dict(tile_h=T, frac_reg=fr)] * ng)
                    for first, cnt, fused, ms in p.time_launches([x.image()], [y.image()], 5, s):
                        prm = dict(tile_h=T, frac_reg=fr) if fused else None
                        feats.append(wt.costmodel_features(p, first, cnt, prm, fused, W, H))
                        ys.append(np.log(ms))
    feats = np.array(feats, np.float32)
    ys = np.array(ys, np.float32)
    assert len(ys) >= 20 and np.all(np.isfinite(ys))
    wt.costmodel_train(feats, ys, epochs=100, batch=32, lr=3e-3, seed=3)
    spec = P.harris()
    img = I.uniform_image(61, W, H)[0]
    x = wt.DeviceImage(1, H, W).upload(img)
    y = wt.DeviceImage(1, H, W)
    p = wt.Pipeline(spec)
    p.schedule_auto(W, H, wt.WT_F32, wt.WT_MODEL_LEARNED)
    p.run([x.image()], [y.image()], s)
    p.check(s)
    ref = O.evaluate(spec["stages"], [img[None].astype(np.float64)], spec["outputs"])[0][0]
    assert np.abs(y.download()[0] - ref).max() <= 1e-5
    wt.costmodel_reset()


def test_shipped_model_picks_a_fast_corner_response_schedule():
    """DP-Fusion with the shipped learned model on the 4096x4096 corner
    response picks a schedule that matches the oracle and runs within 10% of
    the library's default schedule (the fastest of the measured study)."""
    import os
    from paper_1909_07190_gb300 import wt
    W = H = 4096
    spec = P.harris()
    img = I.uniform_image(I.SEED_BASE + 2, W, H)[0]
    src = wt.DeviceImage(1, H, W).upload(img)
    dst = wt.DeviceImage(1, H, W)
    wt.costmodel_load(os.path.join(os.path.dirname(wt.__file__), "costmodel_gb300.txt"))
    try:
        p = wt.Pipeline(spec)
        p.schedule_auto(W, H, wt.WT_F32, wt.WT_MODEL_LEARNED)
        s = torch.cuda.current_stream().cuda_stream
        p.run([src.image()], [dst.image()], s)
        p.check(s)
        rng = np.random.default_rng(3)
        xs, ys = rng.integers(0, W, 200), rng.integers(0, H, 200)
        ref = O.evaluate_points(spec["stages"], [img.astype(np.float64)], spec["outputs"][0], xs, ys)
        assert np.abs(dst.download()[0][ys, xs] - ref).max() <= 1e-5
        t_learned = p.schedule_time([src.image()], [dst.image()], 0, 20, s)
        q = wt.Pipeline(spec)
        t_default = q.schedule_time([src.image()], [dst.image()], 0, 20, s)
        assert t_learned <= 1.10 * t_default, (t_learned, t_default, p.schedule_get())
    finally:
        wt.costmodel_reset()


def test_costmodel_collect_matches_features_and_launch_times():
    """wt_costmodel_collect: one row per fused or per-stage launch of the
    run, its features equal to wt_costmodel_features of that launch, its log
    time that of wt_schedule_time_launches (re-timed: within a factor of 2);
    launches without features (the reduction chain) are skipped; the run's
    output is the schedule's."""
    from paper_1909_07190_gb300 import wt
    s = torch.cuda.current_stream().cuda_stream
    W, H = 1000, 600
    spec = P.harris()
    img = I.uniform_image(62, W, H)[0]
    x = wt.DeviceImage(1, H, W).upload(img)
    y = wt.DeviceImage(1, H, W)
    ref = O.evaluate(spec["stages"], [img[None].astype(np.float64)], spec["outputs"])[0][0]
    groups = [0, 0, 1, 1, 1, 2, 2, 2, 3, 3, 3]
    prm = [dict(tile_h=16, frac_reg=1.0, vec=4, warps_per_block=1)] * 4
    p = wt.Pipeline(spec)
    p.schedule(groups=groups, params=prm)
    f, lm, st = wt.costmodel_collect(p, [x.image()], [y.image()], 5, s)
    p.check(s)
    assert np.abs(y.download()[0] - ref).max() <= 1e-5
    assert f.shape == (4, 18) and lm.shape == (4,)
    assert [tuple(r) for r in st] == [(0, 2), (2, 3), (5, 3), (8, 3)]
    t = p.time_launches([x.image()], [y.image()], 5, s)
    for i, (first, cnt, fused, ms) in enumerate(t):
        assert fused and (first, cnt) == tuple(st[i])
        want = wt.costmodel_features(p, first, cnt, prm[i], True, W, H)
        assert np.allclose(f[i], want, rtol=1e-6, atol=1e-6)
        assert np.isfinite(lm[i]) and abs(lm[i] - np.log(ms)) < np.log(2.0)
    # per-stage kernels: every stage a row of its own, fused feature 0
    q = wt.Pipeline(spec)
    q.schedule(exec_mode=wt.WT_EXEC_PLAIN)
    f2, lm2, st2 = wt.costmodel_collect(q, [x.image()], [y.image()], 3, s)
    assert len(lm2) == len(spec["stages"]) and np.all(f2[:, 17] == 0)
    assert sorted(r[0] for r in st2) == list(range(len(spec["stages"])))
    # the bilateral filter's default schedule: the reduction chain has no
    # features, the blur and the slice (per-stage kernels) do
    bspec = P.bilateral_filter()
    b = wt.Pipeline(bspec)
    bg, bp = P.bilateral_schedule()
    b.schedule(groups=bg, params=bp)
    yb = wt.DeviceImage(1, H, W)
    f3, lm3, st3 = wt.costmodel_collect(b, [x.image()], [yb.image()], 3, s)
    b.check(s)
    assert 1 <= len(lm3) < b.launches_per_run() and np.all(np.isfinite(lm3))

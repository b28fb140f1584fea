"""Batched runs on the GPU: one persistent launch per group over the tiles
of many images of uneven sizes (wt_run_batch), against the FP64 oracle, the
single-image path and a CUDA-graph replay of itself.

Tolerances as for single images: FP32 storage 1e-5, FP16 storage 2e-3 max
abs on [0,1) data.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1909_07190_gb300 import inputs as I
from paper_1909_07190_gb300 import pipelines as P

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"f32": 1e-5, "f16": 2e-3}


def wtmod():
    from paper_1909_07190_gb300 import wt
    return wt


def stream():
    return torch.cuda.current_stream().cuda_stream


def make_batch(sizes, seed0, dtype, host=True):
    """Device images (inputs uploaded from the host generator, or drawn on
    the device with the same stream) and outputs."""
    wt = wtmod()
    from paper_1909_07190_gb300 import inputs_torch as IT
    dt = wt.DTYPES[dtype]
    ins, outs, hosts = [], [], []
    for i, (w, h) in enumerate(sizes):
        d = wt.DeviceImage(1, h, w, dt)
        if host:
            a = I.round_to(I.uniform_image(seed0 + i, w, h), dtype)
            d.upload(a)
            hosts.append(a)
        else:
            t = IT.uniform_image(seed0 + i, w, h)
            d.view().copy_(t.to(d.t.dtype))
            del t
        ins.append(d)
        outs.append(wt.DeviceImage(1, h, w, dt))
    return ins, outs, hosts


def harris_pipe(params=None):
    wt = wtmod()
    p = wt.Pipeline(P.harris())
    p.schedule(params=params)
    return p


SMALL = [(1, 1), (3, 200), (200, 3), (121, 129), (257, 33), (600, 411), (130, 9), (999, 17), (64, 64),
         (1000, 700)]


@pytest.mark.parametrize("dtype", ["f32", "f16"])
def test_batch_small_full_oracle(dtype):
    """Every pixel of every image against the oracle."""
    wt = wtmod()
    p = harris_pipe([dict(tile_h=16, warps_per_block=2)])
    ins, outs, hosts = make_batch(SMALL, 5000, dtype)
    p.run_batch([x.image() for x in ins], [x.image() for x in outs], len(SMALL), stream())
    p.check(stream())
    spec = P.harris()
    for a, o in zip(hosts, outs):
        ref = O.evaluate(spec["stages"], [a.astype(np.float64)], spec["outputs"])[0]
        assert np.abs(o.download()[0] - ref[0]).max() <= TOL[dtype]
    assert wt is not None


def test_batch_bitwise_equals_single_runs_and_graph_replay():
    """Same arithmetic as wt_run, bit for bit; a captured graph replays it."""
    p = harris_pipe([dict(tile_h=16, warps_per_block=2)])
    ins, outs, _ = make_batch(SMALL, 6000, "f16")
    ii, oo = [x.image() for x in ins], [x.image() for x in outs]
    p.run_batch(ii, oo, len(SMALL), stream())
    p.check(stream())
    first = [o.t.clone() for o in outs]
    q = harris_pipe([dict(tile_h=16, warps_per_block=2)])
    for x, o, f in zip(ins, outs, first):
        o.t.zero_()
        q.run([x.image()], [o.image()], stream())
        q.check(stream())
        assert torch.equal(o.view(), f[:, :, :o.w])
    for o in outs:
        o.t.zero_()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        p.run_batch(ii, oo, len(SMALL), torch.cuda.current_stream().cuda_stream)
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    p.check(stream())
    for o, f in zip(outs, first):
        assert torch.equal(o.view(), f[:, :, :o.w])


def window_oracle(spec, seed, w, h, dtype, x, y, r=4):
    """Oracle value at (x, y) from the pixels within r of it: the window is
    cut at the image border (where clamp-to-edge applies alike) and at least
    r > halo elsewhere, so it equals the full-image value."""
    x0, x1 = max(0, x - r), min(w, x + r + 1)
    y0, y1 = max(0, y - r), min(h, y + r + 1)
    rows = []
    for yy in range(y0, y1):
        rows.append(I.uniform01(seed, x1 - x0, yy * w + x0))
    win = I.round_to(np.stack(rows), dtype).astype(np.float64)[None]
    return O.evaluate_points(spec["stages"], [win], spec["outputs"][0], np.array([x - x0]), np.array([y - y0]))[0]


def test_batch_512_uneven_fp16_sampled():
    """The batched serving workload: 512 images, sides uniform in
    [200, 4096], FP16 storage.  Inputs drawn on the device with the host
    generator's stream; sampled outputs (corners, edges, random interior)
    of every image against the oracle."""
    sizes = I.batch_sizes(I.SEED_BASE + 3)
    seed0 = (I.SEED_BASE + 3) * 1000
    p = harris_pipe()
    ins, outs, _ = make_batch(sizes, seed0, "f16", host=False)
    p.run_batch([x.image() for x in ins], [x.image() for x in outs], len(sizes), stream())
    p.check(stream())
    spec = P.harris()
    rng = np.random.default_rng(3)
    worst = 0.0
    for i, (w, h) in enumerate(sizes):
        pts = [(0, 0), (w - 1, h - 1)] if i % 2 == 0 else [(w - 1, 0), (0, h - 1)]
        pts += [(int(rng.integers(0, w)), int(rng.integers(0, h))) for _ in range(2)]
        pts += [(int(rng.integers(0, w)), h - 2), (1, int(rng.integers(0, h)))]
        o = outs[i]
        for (x, y) in pts:
            got = float(o.t[0, y, x].float())
            ref = window_oracle(spec, seed0 + i, w, h, "f16", x, y)
            worst = max(worst, abs(got - ref))
    assert worst <= TOL["f16"], worst


def test_batch_rejects_non_fused_schedule():
    wt = wtmod()
    p = wt.Pipeline(P.harris())
    p.schedule(exec_mode=wt.WT_EXEC_PLAIN)
    ins, outs, _ = make_batch(SMALL[:2], 7000, "f32")
    with pytest.raises(wt.WtError):
        p.run_batch([x.image() for x in ins], [x.image() for x in outs], 2, stream())

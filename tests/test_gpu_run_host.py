"""wt_run_host on images tall enough for row bands (copy-in, compute and
copy-out of consecutive bands overlapped on three streams): the host result
must equal the device run on the whole image bit for bit, since every band
computes its kept rows from the same inputs with the same arithmetic."""
import numpy as np
import pytest

from paper_1909_07190_gb300 import pipelines as P

from test_gpu_parity import oracle_out, rnd, wtmod

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def stream():
    return torch.cuda.current_stream().cuda_stream


def host_vs_device(spec, img, dtype="f32", groups=None, params=None):
    wt = wtmod()
    dt = wt.DTYPES[dtype]
    H, W = img.shape[-2:]
    p = wt.Pipeline(spec)
    if groups is not None:
        p.schedule(groups=groups, params=params)
    outs_c = [spec["stages"][s]["channels"] for s in spec["outputs"]]
    hin = wt.DeviceImage(1, H, W, dt, device="cpu", pin_host=True)
    hin.view().copy_(torch.from_numpy(np.asarray(img, np.float32).reshape(1, H, W)).to(hin.t.dtype))
    hout = [wt.DeviceImage(c, H, W, dt, device="cpu", pin_host=True) for c in outs_c]
    for h in hout:
        h.t.fill_(float("nan")) if dtype == "f32" else h.t.zero_()
    p.run_host([hin.image()], [h.image() for h in hout], stream())
    din = wt.DeviceImage(1, H, W, dt)
    din.view().copy_(hin.view())
    dout = [wt.DeviceImage(c, H, W, dt) for c in outs_c]
    p.run([din.image()], [d.image() for d in dout], stream())
    p.check(stream())
    torch.cuda.synchronize()
    for h, d in zip(hout, dout):
        assert torch.equal(h.view().view(torch.int16 if dtype != "f32" else torch.int32),
                           d.view().cpu().view(torch.int16 if dtype != "f32" else torch.int32))
    return [h.view().float().numpy() for h in hout]


@pytest.mark.parametrize("W,H", [(1536, 2800), (4096, 4096), (1100, 4001)])
def test_run_host_bands_harris(W, H):
    """Images of 2 to 8 bands (at least 8 MiB of input per band)."""
    spec = P.harris()
    img = rnd(W + H, W, H)
    got = host_vs_device(spec, img)
    if W * H <= 1536 * 2800:
        ref = oracle_out(spec, [img])[0]
        assert np.abs(got[0][0] - ref).max() <= 1e-5 * max(1.0, np.abs(ref).max())


def test_run_host_bands_multi_group_f16():
    """Sharpen as three groups (intermediates in the workspace), FP16."""
    spec = P.sharpen()
    img = rnd(7, 4096, 2048, dtype="f16")
    got = host_vs_device(spec, img, "f16", groups=[0, 1, 2], params=[dict(tile_h=16)] * 3)
    assert np.abs(got[0][0] - oracle_out(spec, [img])[0]).max() <= 2e-3


def test_run_host_bands_multi_output_and_planes():
    """Two outputs, one of them three planes (one-plane input)."""
    inp = P.input_id(0)
    b = P.Builder("mo", [1])
    s0 = b.stage("blur", P.linear(inp, [[1, 2, 1], [2, 4, 2], [1, 2, 1]], 1.0 / 16))
    s1 = b.stage("three", P.ref(s0, 0, -2) * 0.5 + P.ref(inp, 1, 1), 3)
    s2 = b.stage("edge", P.ref(s0, 1, 0) - P.ref(s0, -1, 3))
    b.output(s1, s2)
    spec = b.build()
    img = rnd(8, 1500, 3000)
    got = host_vs_device(spec, img)
    ref = oracle_out(spec, [img])
    for g, r in zip(got, ref):
        assert np.abs(g - r).max() <= 1e-5


def test_run_host_bands_row_parity():
    """A stage reading the output row's parity (a Bayer-like pattern) on an
    image of two 2049-row bands with a 2-row halo: the second band's
    sub-image would start on an odd row; bands start on even rows, so the
    host run equals the device run."""
    from test_host_bands import parity_pipeline
    wt = wtmod()
    spec = parity_pipeline(1)
    im = [wt.image(1 << 36, 1024, 4097, 1, wt.WT_F32, 4096)]
    assert [b[2] for b in wt.Pipeline(spec).debug_host_bands(im, im)] == [0, 2046]
    img = rnd(9, 1024, 4097)
    got = host_vs_device(spec, img)
    ref = oracle_out(spec, [img])[0]
    assert np.abs(got[0][0] - ref).max() <= 1e-5


def test_run_host_repeated_calls_replay():
    """Calls with the same host images: the first runs the bands directly,
    the second captures them into a CUDA graph, later ones replay it.  New
    input contents each call; every result against the device run."""
    wt = wtmod()
    spec = P.harris()
    W, H = 2048, 2304
    p = wt.Pipeline(spec)
    hin = wt.DeviceImage(1, H, W, device="cpu", pin_host=True)
    hout = wt.DeviceImage(1, H, W, device="cpu", pin_host=True)
    din, dout = wt.DeviceImage(1, H, W), wt.DeviceImage(1, H, W)
    for call in range(4):
        img = rnd(100 + call, W, H)
        hin.view().copy_(torch.from_numpy(img))
        p.run_host([hin.image()], [hout.image()], stream())
        din.view().copy_(hin.view())
        p.run([din.image()], [dout.image()], stream())
        p.check(stream())
        torch.cuda.synchronize()
        assert torch.equal(hout.view(), dout.view().cpu()), call
    # other host buffers of the same size, then the first ones again
    hin2 = wt.DeviceImage(1, H, W, device="cpu", pin_host=True)
    hout2 = wt.DeviceImage(1, H, W, device="cpu", pin_host=True)
    hin2.view().copy_(hin.view() * 0.5)
    for _ in range(3):
        p.run_host([hin2.image()], [hout2.image()], stream())
    p.run_host([hin.image()], [hout.image()], stream())
    din.view().copy_(hin2.view())
    p.run([din.image()], [dout.image()], stream())
    torch.cuda.synchronize()
    assert torch.equal(hout2.view(), dout.view().cpu())
    assert not torch.equal(hout2.view(), hout.view())

"""wt_run_static: the pipeline run for callers that cannot let a library
allocate device memory (their device memory belongs to their own allocator
under a fixed budget, or cudaMalloc's device-wide synchronization is not
acceptable on their path).  Its intermediates live in a static device array
instead of the pipeline's workspace.  These tests check that it gives the
same result as wt_run, on two calls in a row (warp-tile, block-tile and
pyramid schedules), that a warm call allocates nothing, that a device-side
timeout inside it is reported by wt_check, and that it rejects runs that
need more scratch than the array holds.  The file is collected last."""
import numpy as np
import pytest

from paper_1909_07190_gb300 import inputs as I
from paper_1909_07190_gb300 import pipelines as P
from paper_1909_07190_gb300 import wt

torch = pytest.importorskip("torch")


def _images(W, H, n_out=1):
    img = I.uniform_image(I.SEED_BASE + 2, W, H)[0]
    src = wt.DeviceImage(1, H, W).upload(img)
    outs = [wt.DeviceImage(1, H, W) for _ in range(n_out)]
    return src, outs


@pytest.mark.gpu
def test_run_static_matches_run_twice():
    W, H = 613, 389
    p = wt.Pipeline(P.harris())
    # three groups: the two HBM intermediates between them use the scratch
    groups = [0] * 5 + [1] * 3 + [2] * 3
    p.schedule(groups=groups, params=[dict(tile_h=16, warps_per_block=4)] * 3)
    src, (ref, a, b) = _images(W, H, 3)
    s = torch.cuda.current_stream().cuda_stream
    p.run([src.image()], [ref.image()], s)          # loads the kernels
    p.check(s)
    want = ref.download()
    for out in (a, b):                               # two calls in a row
        out.view().fill_(float("nan"))
        p.run_static([src.image()], [out.image()], s)
        torch.cuda.synchronize()
        got = out.download()
        assert np.isfinite(got).all()
        assert np.abs(got - want).max() <= 1e-5


@pytest.mark.gpu
def test_run_static_single_group_sharpen():
    W, H = 1000, 257
    p = wt.Pipeline(P.sharpen())
    src, (ref, out) = _images(W, H, 2)
    s = torch.cuda.current_stream().cuda_stream
    p.run([src.image()], [ref.image()], s)
    for _ in range(2):
        p.run_static([src.image()], [out.image()], s)
    torch.cuda.synchronize()
    assert np.abs(out.download() - ref.download()).max() <= 1e-5


def test_run_static_rejects_oversized_scratch():
    """The plain schedule of a 4096x4096 corner response needs ten 64 MiB
    intermediates: rejected before any device work."""
    p = wt.Pipeline(P.harris())
    p.schedule(exec_mode=wt.WT_EXEC_PLAIN)
    buf = np.zeros(16, np.float32)
    img = wt.image(buf.ctypes.data, 4096, 4096, 1, wt.WT_F32, 4096 * 4)
    with pytest.raises(wt.WtError, match="at most"):
        p.run_static([img], [img])


@pytest.mark.gpu
def test_run_static_allocates_nothing():
    """A warm call changes neither the device's free memory nor the bytes
    the library holds."""
    W, H = 613, 389
    p = wt.Pipeline(P.harris())
    p.schedule(groups=[0] * 5 + [1] * 3 + [2] * 3, params=[dict(tile_h=16)] * 3)
    src, (ref, out) = _images(W, H, 2)
    s = torch.cuda.current_stream().cuda_stream
    p.run([src.image()], [ref.image()], s)
    p.run_static([src.image()], [out.image()], s)   # first call: takes the address
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    held0 = wt.live_objects()[1]
    for _ in range(3):
        p.run_static([src.image()], [out.image()], s)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert wt.live_objects()[1] == held0
    assert np.abs(out.download() - ref.download()).max() <= 1e-5


@pytest.mark.gpu
def test_run_static_block_tiles_wider_than_resident_blocks():
    """Block-tile (one tile per thread block) schedules launch one block per
    tile, however many tiles there are: 1024 tile columns of 32 pixels."""
    W, H = 32768, 40
    p = wt.Pipeline(P.harris())
    p.schedule(params=[dict(tile_h=32, warps_per_block=16, vec=1, flags=wt.WT_FLAG_OTPTB)])
    src, (ref, out) = _images(W, H, 2)
    s = torch.cuda.current_stream().cuda_stream
    p.run([src.image()], [ref.image()], s)
    for _ in range(2):
        out.view().fill_(float("nan"))
        p.run_static([src.image()], [out.image()], s)
        p.check(s)
        got = out.download()
        assert np.isfinite(got).all()
        assert np.abs(got - ref.download()).max() <= 1e-5


@pytest.mark.gpu
def test_run_static_pyramid_levels():
    """The multi-scale blend (6 levels, one group per level): its
    intermediates of every level live in the static array."""
    W, H = 257, 190
    spec = P.blend()
    groups, prm = P.blend_schedule()
    p = wt.Pipeline(spec)
    p.schedule(groups=groups, params=prm)
    ins = [wt.DeviceImage(3, H, W).upload(I.uniform_image(21, W, H, 3)),
           wt.DeviceImage(3, H, W).upload(I.uniform_image(22, W, H, 3)),
           wt.DeviceImage(1, H, W).upload(I.smooth_mask(23, W, H))]
    ref, out = wt.DeviceImage(3, H, W), wt.DeviceImage(3, H, W)
    s = torch.cuda.current_stream().cuda_stream
    p.run([x.image() for x in ins], [ref.image()], s)
    for _ in range(2):
        out.view().fill_(float("nan"))
        p.run_static([x.image() for x in ins], [out.image()], s)
        p.check(s)
        assert np.abs(out.download() - ref.download()).max() <= 1e-5


@pytest.mark.gpu
def test_run_static_reports_device_status():
    """A bounded wait that gives up inside a wt_run_static run (the
    test-only stall flag) is reported by wt_check, once."""
    W, H = 500, 200
    p = wt.Pipeline(P.harris())
    src, (ref, out) = _images(W, H, 2)
    s = torch.cuda.current_stream().cuda_stream
    p.schedule(params=[dict(tile_h=14, flags=wt.WT_FLAG_TEST_STALL)])
    p.run([src.image()], [ref.image()], s)             # loads the kernel
    with pytest.raises(wt.WtError):
        p.check(s)
    p.run_static([src.image()], [out.image()], s)
    with pytest.raises(wt.WtError) as e:
        p.check(s)
    assert e.value.code == wt.WT_ETIMEOUT
    p.check(s)

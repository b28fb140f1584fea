"""Failure detection on the GPU, by forms that cannot fault or hang it.

- A warp-tile kernel built with the test-only stall flag arms its first
  staging barrier for bytes no copy delivers (no copy is issued, nothing is
  in flight); every bounded wait gives up after 256 polls and raises the
  error word.  wt_check reports WT_ETIMEOUT once, clears the word, and the
  next run with the normal schedule is clean and correct.
- An injected failure of the library's device allocation makes wt_run
  return WT_ENOMEM without leaking device memory; the next run allocates
  and matches the oracle.
"""
import gc

import numpy as np
import pytest

from oracle import oracle as O
from paper_1909_07190_gb300 import inputs as I
from paper_1909_07190_gb300 import pipelines as P
from paper_1909_07190_gb300 import wt

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def stream():
    return torch.cuda.current_stream().cuda_stream


def harris_ref(img):
    spec = P.harris()
    return O.evaluate(spec["stages"], [img.astype(np.float64)], spec["outputs"])[0][0]


@pytest.mark.parametrize("n_buffers", [2, 3])
def test_bounded_wait_times_out_and_next_run_is_clean(n_buffers):
    W, H = 700, 300
    img = I.uniform_image(I.SEED_BASE + 2, W, H)[0]
    src = wt.DeviceImage(1, H, W).upload(img)
    dst = wt.DeviceImage(1, H, W)
    p = wt.Pipeline(P.harris())
    p.schedule(params=[dict(tile_h=14, n_buffers=n_buffers, flags=wt.WT_FLAG_TEST_STALL)])
    p.run([src.image()], [dst.image()], stream())
    with pytest.raises(wt.WtError) as e:
        p.check(stream())
    assert e.value.code == wt.WT_ETIMEOUT
    p.check(stream())                      # the word was cleared
    p.schedule(params=[dict(tile_h=14, n_buffers=n_buffers)])
    for _ in range(2):                     # the queue counters were reset too
        dst.view().fill_(float("nan"))
        p.run([src.image()], [dst.image()], stream())
        p.check(stream())
        assert np.abs(dst.download()[0] - harris_ref(img)).max() <= 1e-5


def test_device_allocation_failure_reports_enomem_without_leak():
    W, H = 512, 256
    img = I.uniform_image(I.SEED_BASE + 2, W, H)[0]
    src = wt.DeviceImage(1, H, W).upload(img)
    dst = wt.DeviceImage(1, H, W)
    p = wt.Pipeline(P.harris())
    # three groups: the run needs the workspace for two intermediates
    p.schedule(groups=[0] * 5 + [1] * 3 + [2] * 3, params=[dict(tile_h=16)] * 3)
    gc.collect()                           # earlier tests' pipelines are gone
    torch.cuda.synchronize()
    _, held0 = wt.live_objects()
    for after in (0, 1):                   # control block, then intermediates
        wt.inject_alloc_failure(1, after)
        with pytest.raises(wt.WtError) as e:
            p.run([src.image()], [dst.image()], stream())
        assert e.value.code == wt.WT_ENOMEM
    p.run([src.image()], [dst.image()], stream())
    p.check(stream())
    assert np.abs(dst.download()[0] - harris_ref(img)).max() <= 1e-5
    _, held = wt.live_objects()
    assert held > held0
    p.close()
    assert wt.live_objects()[1] == held0

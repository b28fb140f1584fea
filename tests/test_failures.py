"""Failure detection without a GPU fault.

Host side: an injected allocation failure in pipeline creation or run
planning returns WT_ENOMEM, leaves the caller's handle untouched and leaks
no pipeline.  Device side, in the CPU block emulator: a warp-tile kernel
built with the test-only stall flag arms its first staging barrier for
bytes that no copy delivers; its bounded wait gives up, raises the timeout
code in the error word, drains the copies it did issue and leaves through
the tile-queue accounting (the queue is reset for the next launch).  The
same flag runs on a GPU in tests/test_gpu_failures.py."""
import ctypes

import numpy as np
import pytest

from oracle import oracle as O
from paper_1909_07190_gb300 import inputs as I
from paper_1909_07190_gb300 import pipelines as P
from paper_1909_07190_gb300 import wt

from emu import emu

HOST, DEVICE = 0, 1


def _create_raw(spec):
    """wt_pipeline_create through the C ABI; returns (status, handle)."""
    lib = wt.load()
    st, keep = wt.stage_array(spec)
    inch = (ctypes.c_int32 * len(spec["inputs"]))(*spec["inputs"])
    outs = (ctypes.c_int32 * len(spec["outputs"]))(*spec["outputs"])
    h = ctypes.c_void_p(0xDEAD)
    rc = lib.wt_pipeline_create(st, len(spec["stages"]), inch, len(spec["inputs"]), outs,
                                len(spec["outputs"]), 0, ctypes.byref(h))
    return rc, h


@pytest.mark.parametrize("after", [0, 1])
def test_create_reports_enomem_without_leak(after):
    live0, _ = wt.live_objects()
    wt.inject_alloc_failure(HOST, after)
    rc, h = _create_raw(P.harris())
    assert rc == wt.WT_ENOMEM
    assert h.value == 0xDEAD          # the out pointer is written only on success
    assert wt.live_objects()[0] == live0
    # disarmed after one failure: the next creation succeeds
    rc, h = _create_raw(P.harris())
    assert rc == wt.WT_OK
    assert wt.live_objects()[0] == live0 + 1
    assert wt.load().wt_pipeline_destroy(h) == wt.WT_OK
    assert wt.live_objects()[0] == live0


def test_planning_reports_enomem_then_recovers():
    p = wt.Pipeline(P.sharpen())
    buf = np.zeros(64 * 64, np.float32)
    img = wt.image(buf.ctypes.data, 64, 64, 1, wt.WT_F32, 64 * 4)
    wt.inject_alloc_failure(HOST, 0)
    with pytest.raises(wt.WtError) as e:
        p.debug_kernel(0, [img], [img])
    assert e.value.code == wt.WT_ENOMEM
    assert "allocation" in str(e.value)
    d = p.debug_kernel(0, [img], [img])
    assert d["fused"]


def test_disarm_and_bad_kind():
    wt.inject_alloc_failure(HOST, 0)
    wt.inject_alloc_failure(HOST, -1)   # disarmed: nothing fails
    p = wt.Pipeline(P.sharpen())
    p.close()
    with pytest.raises(wt.WtError):
        wt.inject_alloc_failure(7, 0)


def test_stall_flag_round_trips_and_generates_the_stall():
    p = wt.Pipeline(P.sharpen())
    p.schedule(params=[dict(tile_h=8, flags=wt.WT_FLAG_TEST_STALL)])
    assert p.schedule_get()["params"][0]["flags"] & wt.WT_FLAG_TEST_STALL
    buf = np.zeros(64 * 64, np.float32)
    img = wt.image(buf.ctypes.data, 64, 64, 1, wt.WT_F32, 64 * 4)
    src = p.debug_kernel(0, [img], [img])["source"]
    assert "#define WT_WAIT_LIMIT 256" in src
    assert "if (c_ != 0) {" in src
    # the default schedule's kernel has neither
    q = wt.Pipeline(P.sharpen())
    src0 = q.debug_kernel(0, [img], [img])["source"]
    assert "#define WT_WAIT_LIMIT 256" not in src0 and "if (c_ != 0) {" not in src0


@pytest.mark.parametrize("n_buffers", [2, 3])
def test_emulated_stall_times_out_and_drains(n_buffers):
    """Every warp's first wait gives up (error word 1 = timeout); with three
    buffers the warp also issued a real copy of chunk 1, which it waits for
    before leaving.  The queue counters are back at zero, and the normal
    schedule then runs clean and matches the oracle."""
    spec = P.harris()
    W, H = 150, 70
    img = I.uniform_image(I.SEED_BASE + 2, W, H)[0]
    p = wt.Pipeline(spec)
    p.schedule(params=[dict(tile_h=8, warps_per_block=2, n_buffers=n_buffers,
                            flags=wt.WT_FLAG_TEST_STALL)])
    src = emu.HostImage(1, H, W, fill=img)
    dst = emu.HostImage(1, H, W)
    d = emu.run(p, 0, [src], [dst], max_blocks=2, allow_err=True)
    assert d["err"] == 1
    assert dst.padding_intact()
    p.schedule(params=[dict(tile_h=8, warps_per_block=2, n_buffers=n_buffers)])
    d = emu.run(p, 0, [src], [dst], max_blocks=2)
    assert d["err"] == 0
    ref = O.evaluate(spec["stages"], [img.astype(np.float64)], spec["outputs"])[0][0]
    assert np.abs(dst.view()[0] - ref).max() <= 1e-5

"""Host-side checks of the C-ABI library (no GPU): it loads, exports every
symbol the headers declare, validates DAGs and schedules, and reports errors
through wt_status + wt_last_error."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1909_07190_gb300 import pipelines as P
from paper_1909_07190_gb300 import wt

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in ("wt.h", "wt_debug.h"):
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(wt_[a-z_0-9]+)\s*\(", text, re.M):
            names.add(m.group(1))
    return names


def test_library_exports_every_declared_symbol():
    lib = wt.load()
    names = declared_symbols()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
    assert names == {s[0] for s in wt.SIGNATURES}


def test_version():
    assert wt.load().wt_version() >= 100


def _create(stages, inputs=(1,), outputs=(0,)):
    st, keep = wt.stage_array({"stages": stages, "inputs": list(inputs), "outputs": list(outputs)})
    h = ctypes.c_void_p()
    ic = (ctypes.c_int32 * len(inputs))(*inputs)
    oc = (ctypes.c_int32 * len(outputs))(*outputs)
    rc = wt.load().wt_pipeline_create(st, len(stages), ic, len(inputs), oc, len(outputs), 0, ctypes.byref(h))
    return rc, h


@pytest.mark.parametrize("stages,msg", [
    ([{"channels": 1, "inputs": [1], "ops": [("tap", 0, 0, 0)]},
      {"channels": 1, "inputs": [-1], "ops": [("tap", 0, 0, 0)]}], "topological"),
    ([{"channels": 1, "inputs": [-1], "ops": [("tap", 0, 0, 0), ("add",)]}], "underflow"),
    ([{"channels": 1, "inputs": [-1], "ops": [("tap", 0, 0, 0, -1, "up2")]}], "level"),
    ([{"channels": 1, "inputs": [-1], "ops": [("tap", 0, 0, 0, 3)]}], "channel"),
    ([{"channels": 1, "inputs": [-1], "ops": [("tap", 0, 99, 0)]}], "offset"),
])
def test_malformed_dag_rejected(stages, msg):
    rc, h = _create(stages)
    assert rc == wt.WT_EINVAL
    assert msg in wt.load().wt_last_error().decode()


def test_schedule_validation():
    p = wt.Pipeline(P.harris())
    with pytest.raises(wt.WtError, match="contiguous"):
        p.schedule(groups=[0, 1, 0, 1, 1, 1, 1, 1, 1, 1, 1])
    with pytest.raises(wt.WtError, match="tile_h"):
        p.schedule(params=[dict(tile_h=0)])
    with pytest.raises(wt.WtError, match="frac_reg"):
        p.schedule(params=[dict(frac_reg=1.5)])
    p.schedule(groups=[0] * 5 + [1] * 6, params=[dict(tile_h=8), dict(tile_h=16)])
    s = p.schedule_get()
    assert s["groups"] == [0] * 5 + [1] * 6 and s["params"][1]["tile_h"] == 16


def test_launch_counts():
    p = wt.Pipeline(P.harris())
    assert p.launches_per_run() == 1
    p.schedule(exec_mode=wt.WT_EXEC_PLAIN)
    assert p.launches_per_run() == 11
    b = wt.Pipeline(P.blend())
    b.schedule(exec_mode=wt.WT_EXEC_PLAIN)
    assert b.launches_per_run() == 36


def test_bad_images_rejected_without_gpu():
    p = wt.Pipeline(P.sharpen())
    buf = np.zeros((8, 64), np.float32)
    good = wt.image(buf.ctypes.data, 16, 8, 1, wt.WT_F32, 256)
    bad_pitch = wt.image(buf.ctypes.data, 16, 8, 1, wt.WT_F32, 100)
    empty = wt.image(buf.ctypes.data, 0, 8, 1, wt.WT_F32, 256)
    with pytest.raises(wt.WtError, match="pitch"):
        p.debug_kernel(0, [bad_pitch], [good])
    with pytest.raises(wt.WtError, match="empty"):
        p.debug_kernel(0, [empty], [good])
    wrong = wt.image(buf.ctypes.data, 15, 8, 1, wt.WT_F32, 256)
    with pytest.raises(wt.WtError, match="output 0"):
        p.debug_kernel(0, [good], [wrong])


def test_generated_kernels_compile_for_sm103a():
    """NVRTC compiles the generated kernels for sm_103a (no GPU needed)."""
    buf = np.zeros((64, 256), np.float32)
    img = wt.image(buf.ctypes.data, 200, 64, 1, wt.WT_F32, 1024)
    for name in ("sharpen", "harris"):
        p = wt.Pipeline(P.by_name(name))
        assert p.debug_compile(0, [img], [img]) > 10000
        p.schedule(exec_mode=wt.WT_EXEC_PLAIN)
        assert p.debug_compile(0, [img], [img]) > 1000


@pytest.mark.parametrize("name", ["sharpen", "harris", "blur"])
@pytest.mark.parametrize("dtype", [wt.WT_F32, wt.WT_F16, wt.WT_BF16])
@pytest.mark.parametrize("vec", [4, 8])
@pytest.mark.parametrize("chunk", [0, 5, 8])
def test_tma_layout_alignment(name, dtype, vec, chunk):
    """Every TMA destination (each staging buffer of every source, in every
    warp slice) starts on a 128-byte boundary; box rows are multiples of 16
    bytes and at most 256 elements; the mbarriers are 8-byte aligned."""
    es = 4 if dtype == wt.WT_F32 else 2
    buf = np.zeros((64, 512), np.uint8)
    img = wt.image(buf.ctypes.data, 100, 40, 1, dtype, 1024)
    p = wt.Pipeline(P.by_name(name))
    p.schedule(params=[dict(tile_h=16, vec=vec, chunk_rows=chunk, warps_per_block=3)])
    L = p.debug_layout(0, [img], [img])
    assert L["warp_bytes"] % 128 == 0 and L["bar_off"] % 8 == 0
    assert L["chunk"] >= 1 and L["nbuf"] >= 2
    for s in L["sources"]:
        assert s["esz"] == es
        assert s["boxw"] <= 256 and (s["boxw"] * es) % 16 == 0
        assert s["bufb"] % 128 == 0 and s["bufb"] >= L["chunk"] * s["boxw"] * es
        for b in range(L["nbuf"]):
            assert (s["ring_off"] + b * s["bufb"]) % 128 == 0
        assert s["ring_off"] + L["nbuf"] * s["bufb"] <= L["bar_off"]
    # lanes' 16-bit vectors sit at 8-byte offsets, 32-bit ones at 16
    assert (vec * es) % 8 == 0


def test_costmodel_features_cpu():
    """Features of fused groups and per-stage kernels (no GPU needed)."""
    p = wt.Pipeline(P.harris())
    f = wt.costmodel_features(p, 0, 11, dict(tile_h=16, warps_per_block=2, frac_reg=1.0, vec=4), True, 4096, 4096)
    assert f.shape == (18,)
    assert f[0] == pytest.approx(24.0)          # log2(4096 * 4096)
    assert f[1] == 11 and f[17] == 1            # stages, fused
    assert f[8] == pytest.approx(4.0)           # log2 tile height
    assert f[9] == 4 and f[10] == 2 and f[11] == 1.0
    assert f[4] == 4 and f[5] == 4              # one FP32 input and output
    assert f[6] == 4 and f[7] == 4              # two 3x3 footprints: 2 rows/cols each side
    assert 0 < f[14] <= 1 and f[15] > 0         # occupancy, redundant compute
    g = wt.costmodel_features(p, 0, 1, None, False, 4096, 4096)
    assert g[17] == 0 and g[1] == 1
    with pytest.raises(wt.WtError):
        wt.costmodel_features(p, 5, 10, None, False, 64, 64)


def test_costmodel_absent_falls_back_to_analytic():
    wt.costmodel_reset()
    assert not wt.costmodel_ready()
    with pytest.raises(wt.WtError):
        wt.costmodel_predict(np.zeros((1, 18), np.float32))
    p = wt.Pipeline(P.sharpen())
    p.schedule_auto(512, 512, wt.WT_F32, wt.WT_MODEL_LEARNED)
    assert p.schedule_get()["exec"] == wt.WT_EXEC_FUSED


def test_costmodel_load_rejects_bad_files(tmp_path):
    bad = tmp_path / "bad.txt"
    bad.write_text("not a model\n")
    with pytest.raises(wt.WtError):
        wt.costmodel_load(bad)
    with pytest.raises(wt.WtError):
        wt.costmodel_load(tmp_path / "missing.txt")
    with pytest.raises(wt.WtError):
        wt.costmodel_save(tmp_path / "none.txt")   # no model to save


def test_launch_count_with_per_stage_groups():
    """Groups flagged to run per stage count one launch per live stage, a
    cascade group one launch per pair of levels of an image."""
    p = wt.Pipeline(P.blend())
    groups, params = P.blend_schedule()
    p.schedule(groups=groups, params=params)
    assert p.launches_per_run() == 2 * 3 + 3 + 6
    p.schedule(groups=P.blend_groups())
    assert p.launches_per_run() == 10


def test_preprocess_needs_a_gpu():
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is present")
    except ImportError:
        pass
    p = wt.Pipeline(P.sharpen())
    with pytest.raises(wt.WtError):
        p.preprocess()


def test_shipped_cost_model_loads():
    """The learned cost model trained on GB300 launch times (by the cost-model
    study) ships with the package and loads: 18 features, 64 hidden units."""
    import os
    from paper_1909_07190_gb300 import wt
    path = os.path.join(os.path.dirname(wt.__file__), "costmodel_gb300.txt")
    with open(path) as f:
        assert f.readline().split() == ["wt-mlp", "1", "18", "64"]
    wt.costmodel_load(path)
    try:
        assert wt.costmodel_ready()
    finally:
        wt.costmodel_reset()
    assert not wt.costmodel_ready()


def _plan(spec, W, H, dt=wt.WT_F32, groups=None, params=None, exec_mode=None):
    """Launch shapes of every launch of the run plan (planning only)."""
    p = wt.Pipeline(spec)
    if exec_mode is not None:
        p.schedule(exec_mode=exec_mode)
    elif params is not None:
        p.schedule(groups=groups, params=params)
    es = 4 if dt == wt.WT_F32 else 2
    pitch = ((W * es + 127) // 128) * 128
    ins = [wt.image(1 << 40, W, H, c, dt, pitch) for c in spec["inputs"]]
    outs = [wt.image(1 << 41, W, H, spec["stages"][s]["channels"], dt, pitch) for s in spec["outputs"]]
    wsb = p.debug_workspace_bytes(ins, outs)
    return [p.debug_kernel(i, ins, outs, workspace=(1 << 42, max(wsb, 16)))
            for i in range(p.launches_per_run())]


@pytest.mark.parametrize("case", ["fused_64k", "plain_wide", "blend_64k", "otptb_wide", "vol_deep", "vol_wide"])
def test_large_images_plan_within_launch_limits(case):
    """Images far larger than the configurations plan into launches whose
    grids stay inside CUDA's limits (x < 2^31, y and z <= 65535)."""
    otptb = [dict(tile_h=32, warps_per_block=16, vec=1, flags=wt.WT_FLAG_OTPTB)]
    g, q = P.blend_schedule()
    plans = {
        "fused_64k": lambda: _plan(P.harris(), 65536, 65536),
        "plain_wide": lambda: _plan(P.harris(), 1 << 24, 64, exec_mode=wt.WT_EXEC_PLAIN),
        "blend_64k": lambda: _plan(P.blend(), 65536, 65536, wt.WT_BF16, groups=g, params=q),
        "otptb_wide": lambda: _plan(P.harris(), 1 << 26, 64, params=otptb),
        "vol_deep": lambda: _plan(P.heat3d(2, depth=70000), 64, 64),
        "vol_wide": lambda: _plan(P.unsharp3d(depth=8), 65536, 65536),
    }
    for d in plans[case]():
        gx, gy, gz = d["grid"]
        assert 1 <= gx < 2 ** 31 and 1 <= gy <= 65535 and 1 <= gz <= 65535, d["grid"]


@pytest.mark.parametrize("case,msg", [
    ("fused_max", "too many tiles"),
    ("queue_1m", "too many tiles"),
    ("otptb_tall", "too many block tiles"),
    ("plain_tall", "too tall"),
    ("down_tall", "too tall"),
])
def test_oversized_images_rejected(case, msg):
    """Beyond the launch limits planning fails with WT_EUNSUPPORTED and a
    message, rather than launching a truncated grid."""
    M = 2 ** 31 - 1
    runs = {
        "fused_max": lambda: _plan(P.harris(), M, M),
        "queue_1m": lambda: _plan(P.harris(), 1 << 20, 1 << 20, params=[dict(tile_h=8, flags=wt.WT_FLAG_TILE_QUEUE)]),
        "otptb_tall": lambda: _plan(P.harris(), 1 << 20, 1 << 22,
                                    params=[dict(tile_h=32, warps_per_block=16, vec=1, flags=wt.WT_FLAG_OTPTB)]),
        "plain_tall": lambda: _plan(P.harris(), 2, 1 << 17, exec_mode=wt.WT_EXEC_PLAIN),
        "down_tall": lambda: _plan(P.blend(), 2, 1 << 30, wt.WT_BF16, *P.blend_schedule()),
    }
    with pytest.raises(wt.WtError, match=msg) as e:
        runs[case]()
    assert e.value.code == wt.WT_EUNSUPPORTED

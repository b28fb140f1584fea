"""Thin Python binding of the C ABI in include/wt.h (argument marshalling only).

Every computation runs in libwt.so's kernels; this module converts pipeline
dicts (see pipelines.py) to ``wt_stage`` arrays and tensors to ``wt_image``
descriptors.  There is no CPU fallback: if the library or a CUDA device is
missing, calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libwt.so")

WT_OK, WT_EINVAL, WT_ENOMEM, WT_ECUDA, WT_EUNSUPPORTED, WT_ETIMEOUT, WT_EDEVICE, WT_ECOMPILE = \
    0, -1, -2, -3, -4, -5, -6, -7
WT_F32, WT_F16, WT_BF16 = 0, 1, 2
WT_EXEC_FUSED, WT_EXEC_PLAIN = 0, 1
WT_MODEL_ANALYTIC, WT_MODEL_LEARNED = 0, 1
WT_FLAG_NO_PAIRS, WT_FLAG_NO_TILE_SPLIT, WT_FLAG_PLAIN, WT_FLAG_OTPTB, WT_FLAG_SMEM16 = 1, 2, 4, 8, 16
WT_FLAG_ZSTREAM = 32
WT_FLAG_TEST_STALL = 64
WT_FLAG_TILE_QUEUE = 128
WT_FLAG_ONE_STREAM = 256
WT_FLAG_NO_FOLD = 512
OPCODES = {"const": 1, "tap": 2, "add": 3, "sub": 4, "mul": 5, "div": 6, "min": 7, "max": 8,
           "neg": 9, "abs": 10, "sqrt": 11, "xpar": 12, "ypar": 13, "chan": 14,
           "tapz": 15}
TAPMODES = {"same": 0, "down2": 1, "up2": 2, "down4": 3, "up4": 4, "down8": 5, "up8": 6}
DTYPES = {"f32": WT_F32, "f16": WT_F16, "bf16": WT_BF16}
STATUS = {0: "WT_OK", -1: "WT_EINVAL", -2: "WT_ENOMEM", -3: "WT_ECUDA", -4: "WT_EUNSUPPORTED",
          -5: "WT_ETIMEOUT", -6: "WT_EDEVICE", -7: "WT_ECOMPILE"}


class wt_op(ctypes.Structure):
    _fields_ = [("op", ctypes.c_int32), ("slot", ctypes.c_int32), ("dx", ctypes.c_int32),
                ("dy", ctypes.c_int32), ("chan", ctypes.c_int32), ("mode", ctypes.c_int32),
                ("value", ctypes.c_float)]


class wt_stage(ctypes.Structure):
    _fields_ = [("channels", ctypes.c_int32), ("n_inputs", ctypes.c_int32),
                ("inputs", ctypes.POINTER(ctypes.c_int32)), ("n_ops", ctypes.c_int32),
                ("ops", ctypes.POINTER(wt_op))]


class wt_image(ctypes.Structure):
    _fields_ = [("data", ctypes.c_void_p), ("width", ctypes.c_int32), ("height", ctypes.c_int32),
                ("channels", ctypes.c_int32), ("dtype", ctypes.c_int32),
                ("pitch_bytes", ctypes.c_int64)]


class wt_group_params(ctypes.Structure):
    _fields_ = [("tile_h", ctypes.c_int32), ("warps_per_block", ctypes.c_int32),
                ("frac_reg", ctypes.c_float), ("vec", ctypes.c_int32), ("max_regs", ctypes.c_int32),
                ("chunk_rows", ctypes.c_int32), ("n_buffers", ctypes.c_int32), ("flags", ctypes.c_int32),
                ("tile_o", ctypes.c_int32)]


class wt_gpu_config(ctypes.Structure):
    _fields_ = [("nsms", ctypes.c_int32), ("cores_per_sm", ctypes.c_int32), ("glmem_bw_gbs", ctypes.c_double),
                ("max_smem_per_block", ctypes.c_int32), ("smem_per_sm", ctypes.c_int32),
                ("max_warps_per_sm", ctypes.c_int32), ("max_blocks_per_sm", ctypes.c_int32),
                ("regs_per_sm", ctypes.c_int32), ("max_regs_per_thread", ctypes.c_int32),
                ("warp_size", ctypes.c_int32), ("max_threads_per_sm", ctypes.c_int32)]


class wt_cost_info(ctypes.Structure):
    _fields_ = [("terms", ctypes.c_double * 7), ("cost", ctypes.c_double), ("feasible", ctypes.c_int32),
                ("regs_per_thread", ctypes.c_int32), ("smem_per_block", ctypes.c_int32),
                ("occupancy", ctypes.c_double), ("waves", ctypes.c_double), ("work", ctypes.c_double)]


class wt_schedule_desc(ctypes.Structure):
    _fields_ = [("exec", ctypes.c_int32), ("n_groups", ctypes.c_int32),
                ("group_of_stage", ctypes.POINTER(ctypes.c_int32)),
                ("params", ctypes.POINTER(wt_group_params)),
                ("intermediate_dtype", ctypes.c_int32)]


# Every symbol include/wt.h and include/wt_debug.h declare: (name, restype, argtypes).
_P = ctypes.POINTER
_vp = ctypes.c_void_p
_i32 = ctypes.c_int32
_i64 = ctypes.c_int64
SIGNATURES = [
    ("wt_pipeline_create", _i32, [_P(wt_stage), _i32, _P(_i32), _i32, _P(_i32), _i32, _i32, _P(_vp)]),
    ("wt_pipeline_destroy", _i32, [_vp]),
    ("wt_schedule", _i32, [_vp, _P(wt_schedule_desc)]),
    ("wt_schedule_auto", _i32, [_vp, _i32, _i32, _i32, _i32]),
    ("wt_schedule_get", _i32, [_vp, _P(_i32), _P(_i32), _P(_i32), _P(wt_group_params)]),
    ("wt_gpu_config_get", _i32, [_i32, _P(wt_gpu_config)]),
    ("wt_otpw_warp_sizes", _i32, [_P(_i32), _i32, _P(_i32)]),
    ("wt_otpw_scratchpad", _i32, [_P(_i32), _P(_i32), _P(_i32), _P(_i32), _P(_i64)]),
    ("wt_cost_occupancy", _i32, [_P(wt_gpu_config), _i64, _i32, _i32, _P(ctypes.c_double), _P(_i32)]),
    ("wt_min_transactions", _i32, [_P(_i64), _i32, _i32, _i32, _P(_i64)]),
    ("wt_cost_group", _i32, [_vp, _i32, _i32, _P(wt_group_params), _i32, _i32, _i32, _i32,
                             _P(wt_gpu_config), _P(wt_cost_info)]),
    ("wt_preprocess", _i32, [_vp, _P(ctypes.c_double), _P(_i32)]),
    ("wt_cost_weights", _i32, [_P(ctypes.c_double), _P(ctypes.c_double)]),
    ("wt_run", _i32, [_vp, _P(wt_image), _i32, _P(wt_image), _i32, _vp]),
    ("wt_run_host", _i32, [_vp, _P(wt_image), _i32, _P(wt_image), _i32, _vp]),
    ("wt_run_batch", _i32, [_vp, _P(wt_image), _P(wt_image), _i32, _vp]),
    ("wt_schedule_time", _i32, [_vp, _P(wt_image), _i32, _P(wt_image), _i32, _i32, _i32, _vp,
                                _P(ctypes.c_double)]),
    ("wt_schedule_tune", _i32, [_vp, _P(wt_image), _i32, _P(wt_image), _i32, _i32, _i32, _i32, _vp,
                                _P(ctypes.c_double), _P(_i32)]),
    ("wt_schedule_time_launches", _i32, [_vp, _P(wt_image), _i32, _P(wt_image), _i32, _i32, _vp,
                                         _P(ctypes.c_double), _P(_i32), _i32, _P(_i32)]),
    ("wt_costmodel_features", _i32, [_vp, _i32, _i32, _P(wt_group_params), _i32, _i32, _i32, _i32,
                                     _P(ctypes.c_float)]),
    ("wt_costmodel_collect", _i32, [_vp, _P(wt_image), _i32, _P(wt_image), _i32, _i32, _vp, _P(ctypes.c_float),
                                    _P(ctypes.c_float), _P(_i32), _i32, _P(_i32)]),
    ("wt_mlp_train_steps", _i32, [_P(ctypes.c_float), _P(ctypes.c_float), _P(ctypes.c_float), _i32,
                                  _P(ctypes.c_float), _P(ctypes.c_float), _i32, _P(_i32), _i32, _i32,
                                  ctypes.c_float, ctypes.c_float, _P(ctypes.c_float), _vp]),
    ("wt_mlp_forward", _i32, [_P(ctypes.c_float), _P(ctypes.c_float), _i32, _P(ctypes.c_float), _vp]),
    ("wt_costmodel_train", _i32, [_P(ctypes.c_float), _P(ctypes.c_float), _i32, _i32, _i32, ctypes.c_float,
                                  ctypes.c_uint64, _P(ctypes.c_float)]),
    ("wt_costmodel_predict", _i32, [_P(ctypes.c_float), _i32, _P(ctypes.c_float)]),
    ("wt_costmodel_ready", _i32, []),
    ("wt_costmodel_reset", _i32, []),
    ("wt_costmodel_save", _i32, [ctypes.c_char_p]),
    ("wt_costmodel_load", _i32, [ctypes.c_char_p]),
    ("wt_prepare", _i32, [_vp, _P(wt_schedule_desc), _i32, _P(wt_image), _i32, _P(wt_image), _i32, _i32]),
    ("wt_run_static", _i32, [_vp, _P(wt_image), _i32, _P(wt_image), _i32, _vp]),
    ("wt_check", _i32, [_vp, _vp]),
    ("wt_launches_per_run", _i32, [_vp]),
    ("wt_last_error", ctypes.c_char_p, []),
    ("wt_version", _i32, []),
    ("wt_debug_args_size", _i64, []),
    ("wt_debug_kernel", _i32, [_vp, _i32, _P(wt_image), _i32, _P(wt_image), _i32, ctypes.c_char_p, _i64,
                               _P(_i64), _vp, _i64, _P(_i32), ctypes.c_char_p, _i64]),
    ("wt_debug_batch", _i32, [_vp, _i32, _P(wt_image), _P(wt_image), _i32, ctypes.c_char_p, _i64, _P(_i64),
                              _vp, _vp, _i64, _P(_i32), _i64, _P(_i64), _P(_i32), ctypes.c_char_p, _i64]),
    ("wt_debug_kernel_ws", _i32, [_vp, _i32, _P(wt_image), _i32, _P(wt_image), _i32, _vp, _i64, ctypes.c_char_p,
                                  _i64, _P(_i64), _vp, _i64, _P(_i32), ctypes.c_char_p, _i64, _P(_i64)]),
    ("wt_debug_compile", _i32, [_vp, _i32, _P(wt_image), _i32, _P(wt_image), _i32, _P(_i64)]),
    ("wt_debug_layout", _i32, [_vp, _i32, _P(wt_image), _i32, _P(wt_image), _i32, _P(_i32), _i32, _P(_i32)]),
    ("wt_debug_lanes", _i32, [_vp, _P(wt_image), _i32, _P(wt_image), _i32, _P(_i32), _i32, _P(_i32)]),
    ("wt_debug_host_bands", _i32, [_vp, _P(wt_image), _i32, _P(wt_image), _i32, _P(_i32), _i32, _P(_i32)]),
    ("wt_debug_segment_cost", _i32, [_vp, _i32, _i32, _i32, _i32, _i32, _P(ctypes.c_double), _P(_i32)]),
    ("wt_debug_group_geometry", _i32, [_vp, _i32, _i32, ctypes.c_float, _P(_i32), _i32, _P(_i32)]),
    ("wt_debug_inject_alloc_failure", _i32, [_i32, _i32]),
    ("wt_debug_live_objects", _i32, [_P(_i64), _P(_i64)]),
]

_lock = threading.Lock()
_lib = None


class WtError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s: %s" % (STATUS.get(code, code), msg))
        self.code = code


def load(build_if_missing: bool = True):
    """Loads libwt.so (building it in-tree first if needed)."""
    global _lib
    with _lock:
        if _lib is None:
            if build_if_missing:
                from . import build as _build
                _build.build()
            if not os.path.exists(LIB_PATH):
                raise WtError(WT_EUNSUPPORTED, "libwt.so is not built")
            lib = ctypes.CDLL(LIB_PATH)
            for name, res, args in SIGNATURES:
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def check(rc: int):
    if rc != WT_OK:
        raise WtError(rc, (load().wt_last_error() or b"").decode(errors="replace"))


def stage_array(pipe: dict):
    """wt_stage[] for a pipeline dict, plus the ctypes objects keeping it alive."""
    keep = []
    st = (wt_stage * len(pipe["stages"]))()
    for i, S in enumerate(pipe["stages"]):
        ins = (_i32 * max(1, len(S["inputs"])))(*S["inputs"])
        ops = (wt_op * len(S["ops"]))()
        for j, t in enumerate(S["ops"]):
            o = ops[j]
            o.op = OPCODES[t[0]]
            o.chan = -1
            if t[0] == "const":
                o.value = float(t[1])
            elif t[0] == "tap":
                o.slot, o.dx, o.dy = int(t[1]), int(t[2]), int(t[3])
                if len(t) > 4:
                    o.chan = int(t[4])
                if len(t) > 5:
                    o.mode = TAPMODES[t[5]]
            elif t[0] == "tapz":
                o.slot, o.dx, o.dy, o.chan = int(t[1]), int(t[2]), int(t[3]), int(t[4])
        keep += [ins, ops]
        st[i].channels = int(S["channels"])
        st[i].n_inputs = len(S["inputs"])
        st[i].inputs = ins
        st[i].n_ops = len(S["ops"])
        st[i].ops = ops
    return st, keep


def image(data_ptr: int, width: int, height: int, channels: int, dtype: int, pitch_bytes: int) -> wt_image:
    return wt_image(data_ptr, width, height, channels, dtype, pitch_bytes)


def tensor_image(t) -> wt_image:
    """wt_image for a torch tensor of shape (C, H, W) or (H, W) with a padded
    row stride (elements): t.stride(-2) * element size must be a multiple of 16."""
    import torch
    dt = {torch.float32: WT_F32, torch.float16: WT_F16, torch.bfloat16: WT_BF16}[t.dtype]
    if t.dim() == 2:
        c, h, w = 1, t.shape[0], t.shape[1]
    else:
        c, h, w = t.shape
    es = t.element_size()
    if t.stride(-1) != 1:
        raise ValueError("rows must be contiguous")
    pitch = t.stride(-2) * es
    if t.dim() == 3 and c > 1 and t.stride(0) != t.stride(1) * h:
        raise ValueError("channel planes must be height*pitch apart")
    return wt_image(t.data_ptr(), w, h, c, dt, pitch)


class Pipeline:
    """Owns a wt_pipeline handle."""

    def __init__(self, pipe: dict):
        lib = load()
        self.spec = pipe
        st, self._keep = stage_array(pipe)
        inch = (_i32 * len(pipe["inputs"]))(*pipe["inputs"])
        outs = (_i32 * len(pipe["outputs"]))(*pipe["outputs"])
        h = _vp()
        check(lib.wt_pipeline_create(st, len(pipe["stages"]), inch, len(pipe["inputs"]), outs,
                                     len(pipe["outputs"]), 0, ctypes.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            load().wt_pipeline_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- scheduling
    def schedule(self, groups=None, params=None, exec_mode=WT_EXEC_FUSED, intermediate_dtype=-1):
        """groups: group index per stage (contiguous runs); params: list of dicts
        with wt_group_params fields, one per group."""
        n = len(self.spec["stages"])
        if groups is None:
            groups = [0] * n
        ng = max(groups) + 1
        g = (_i32 * n)(*groups)
        prm = (wt_group_params * ng)()
        for i in range(ng):
            d = dict(tile_h=40, warps_per_block=1, frac_reg=1.0, vec=0, max_regs=0, chunk_rows=0,
                     n_buffers=0, flags=0)
            if params is not None:
                d.update(params[i] if isinstance(params, (list, tuple)) else params)
            for k, v in d.items():
                setattr(prm[i], k, v)
        desc = wt_schedule_desc(exec_mode, ng, g, prm, intermediate_dtype)
        check(load().wt_schedule(self.h, ctypes.byref(desc)))

    def schedule_auto(self, width, height, dtype=WT_F32, model=WT_MODEL_ANALYTIC):
        check(load().wt_schedule_auto(self.h, width, height, dtype, model))

    def schedule_get(self):
        n = len(self.spec["stages"])
        ex, ng = _i32(), _i32()
        check(load().wt_schedule_get(self.h, ctypes.byref(ex), ctypes.byref(ng), None, None))
        g = (_i32 * n)()
        prm = (wt_group_params * ng.value)()
        check(load().wt_schedule_get(self.h, None, None, g, prm))
        params = [{f: getattr(prm[i], f) for f, _ in wt_group_params._fields_} for i in range(ng.value)]
        return {"exec": ex.value, "groups": list(g), "params": params}

    def cost_group(self, first, n, params, txn, width, height, dtype=WT_F32, cfg=None):
        prm = wt_group_params()
        d = dict(tile_h=14, warps_per_block=2, frac_reg=1.0, vec=4, max_regs=0, chunk_rows=0, n_buffers=0)
        d.update(params)
        for k, v in d.items():
            setattr(prm, k, v)
        info = wt_cost_info()
        check(load().wt_cost_group(self.h, first, n, ctypes.byref(prm), txn, width, height, dtype,
                                   ctypes.byref(cfg) if cfg is not None else None, ctypes.byref(info)))
        return {"terms": list(info.terms), "cost": info.cost, "feasible": bool(info.feasible),
                "regs": info.regs_per_thread, "smem_per_block": info.smem_per_block,
                "occupancy": info.occupancy, "waves": info.waves, "work": info.work}

    def launches_per_run(self) -> int:
        return int(load().wt_launches_per_run(self.h))

    # -- running
    def run(self, inputs, outputs, stream=None):
        """inputs/outputs: lists of wt_image (device memory)."""
        ia = (wt_image * len(inputs))(*inputs)
        oa = (wt_image * len(outputs))(*outputs)
        check(load().wt_run(self.h, ia, len(inputs), oa, len(outputs), stream))

    def run_host(self, inputs, outputs, stream=None):
        ia = (wt_image * len(inputs))(*inputs)
        oa = (wt_image * len(outputs))(*outputs)
        check(load().wt_run_host(self.h, ia, len(inputs), oa, len(outputs), stream))

    def run_static(self, inputs, outputs, stream=None):
        """wt_run_static: same result as run(), no device allocation."""
        ia = (wt_image * len(inputs))(*inputs)
        oa = (wt_image * len(outputs))(*outputs)
        check(load().wt_run_static(self.h, ia, len(inputs), oa, len(outputs), stream))

    def run_batch(self, inputs, outputs, n_images, stream=None):
        ia = (wt_image * len(inputs))(*inputs)
        oa = (wt_image * len(outputs))(*outputs)
        check(load().wt_run_batch(self.h, ia, oa, n_images, stream))

    def schedule_time(self, inputs, outputs, n_images=0, reps=20, stream=None) -> float:
        """ms per run of the installed schedule (n_images >= 1: batched)."""
        ia = (wt_image * len(inputs))(*inputs)
        oa = (wt_image * len(outputs))(*outputs)
        ms = ctypes.c_double()
        check(load().wt_schedule_time(self.h, ia, len(inputs), oa, len(outputs), n_images, reps, stream,
                                      ctypes.byref(ms)))
        return ms.value

    def schedule_tune(self, inputs, outputs, n_images=0, max_variants=0, reps=20, stream=None):
        """Measured schedule search; installs the fastest.  Returns (ms, n_timed)."""
        ia = (wt_image * len(inputs))(*inputs)
        oa = (wt_image * len(outputs))(*outputs)
        ms, nt = ctypes.c_double(), _i32()
        check(load().wt_schedule_tune(self.h, ia, len(inputs), oa, len(outputs), n_images, max_variants, reps,
                                      stream, ctypes.byref(ms), ctypes.byref(nt)))
        return ms.value, nt.value

    def preprocess(self):
        """Sec. 6 micro-kernels: (ns per iteration, registers) per stage."""
        n = len(self.spec["stages"])
        ns = (ctypes.c_double * n)()
        regs = (_i32 * n)()
        check(load().wt_preprocess(self.h, ns, regs))
        return list(ns), list(regs)

    def time_launches(self, inputs, outputs, reps=20, stream=None):
        """[(first_stage, n_stages, fused, ms)] per launch of one run."""
        ia = (wt_image * len(inputs))(*inputs)
        oa = (wt_image * len(outputs))(*outputs)
        cap = 4 * len(self.spec["stages"]) + 4
        ms = (ctypes.c_double * cap)()
        info = (_i32 * (3 * cap))()
        n = _i32()
        check(load().wt_schedule_time_launches(self.h, ia, len(inputs), oa, len(outputs), reps, stream, ms, info,
                                               cap, ctypes.byref(n)))
        return [(info[3 * i], info[3 * i + 1], bool(info[3 * i + 2]), ms[i]) for i in range(n.value)]

    def prepare(self, schedules, inputs, outputs, batched=False):
        """Compiles the kernels of schedules [(groups, params), ...] in parallel."""
        n = len(self.spec["stages"])
        keep, descs = [], (wt_schedule_desc * len(schedules))()
        for k, (groups, params) in enumerate(schedules):
            groups = [0] * n if groups is None else groups
            ng = max(groups) + 1
            g = (_i32 * n)(*groups)
            prm = (wt_group_params * ng)()
            for i in range(ng):
                d = dict(tile_h=40, warps_per_block=1, frac_reg=1.0, vec=0, max_regs=0, chunk_rows=0,
                         n_buffers=0, flags=0)
                if params is not None:
                    d.update(params[i] if isinstance(params, (list, tuple)) else params)
                for kk, v in d.items():
                    setattr(prm[i], kk, v)
            keep += [g, prm]
            descs[k] = wt_schedule_desc(WT_EXEC_FUSED, ng, g, prm, -1)
        ia = (wt_image * len(inputs))(*inputs)
        oa = (wt_image * len(outputs))(*outputs)
        check(load().wt_prepare(self.h, descs, len(schedules), ia, len(inputs), oa, len(outputs), int(batched)))

    def check(self, stream=None):
        check(load().wt_check(self.h, stream))

    # -- introspection
    def debug_kernel(self, index, inputs, outputs, workspace=None):
        """workspace: (pointer, bytes) of a host buffer for the plan's
        intermediates, or None."""
        lib = load()
        ia = (wt_image * len(inputs))(*inputs)
        oa = (wt_image * len(outputs))(*outputs)
        n, wsb = _i64(), _i64()
        wp, wc = workspace if workspace is not None else (None, 0)
        check(lib.wt_debug_kernel_ws(self.h, index, ia, len(inputs), oa, len(outputs), wp, wc, None, 0,
                                     ctypes.byref(n), None, 0, None, None, 0, ctypes.byref(wsb)))
        src = ctypes.create_string_buffer(n.value + 1)
        args = ctypes.create_string_buffer(int(lib.wt_debug_args_size()))
        launch = (_i32 * 8)()
        kname = ctypes.create_string_buffer(128)
        check(lib.wt_debug_kernel_ws(self.h, index, ia, len(inputs), oa, len(outputs), wp, wc, src, n.value + 1,
                                     None, args, len(args), launch, kname, 128, None))
        return {"source": src.value.decode(), "args": args.raw, "grid": tuple(launch[0:3]),
                "block": launch[3], "smem": launch[4], "fused": bool(launch[5]),
                "n_launches": launch[6], "unroll": launch[7], "name": kname.value.decode(),
                "ws_bytes": wsb.value}

    def kernel_name(self, index, inputs, outputs) -> str:
        """Entry-point name of launch `index` of the run plan for these images."""
        lib = load()
        ia = (wt_image * len(inputs))(*inputs)
        oa = (wt_image * len(outputs))(*outputs)
        kname = ctypes.create_string_buffer(128)
        check(lib.wt_debug_kernel_ws(self.h, index, ia, len(inputs), oa, len(outputs), None, 0, None, 0, None, None,
                                     0, None, kname, 128, None))
        return kname.value.decode()

    def debug_workspace_bytes(self, inputs, outputs) -> int:
        lib = load()
        ia = (wt_image * len(inputs))(*inputs)
        oa = (wt_image * len(outputs))(*outputs)
        wsb = _i64()
        check(lib.wt_debug_kernel_ws(self.h, 0, ia, len(inputs), oa, len(outputs), None, 0, None, 0, None, None, 0,
                                     None, None, 0, ctypes.byref(wsb)))
        return wsb.value

    def debug_batch(self, index, inputs, outputs, n_images):
        """inputs/outputs: flat lists, image-major (n_images * n_inputs)."""
        lib = load()
        ia = (wt_image * len(inputs))(*inputs)
        oa = (wt_image * len(outputs))(*outputs)
        n, nt = _i64(), _i64()
        check(lib.wt_debug_batch(self.h, index, ia, oa, n_images, None, 0, ctypes.byref(n), None, None, 0,
                                 None, 0, ctypes.byref(nt), None, None, 0))
        asz = int(lib.wt_debug_args_size())
        src = ctypes.create_string_buffer(n.value + 1)
        args = ctypes.create_string_buffer(asz)
        tab = ctypes.create_string_buffer(asz * n_images)
        tiles = (_i32 * (4 * nt.value))()
        launch = (_i32 * 8)()
        kname = ctypes.create_string_buffer(128)
        check(lib.wt_debug_batch(self.h, index, ia, oa, n_images, src, n.value + 1, None, args, tab, len(tab),
                                 tiles, 4 * nt.value, None, launch, kname, 128))
        return {"source": src.value.decode(), "args": args.raw, "img_tab": tab.raw,
                "tiles": list(tiles), "n_tiles": nt.value, "grid": tuple(launch[0:3]), "block": launch[3],
                "smem": launch[4], "fused": True, "n_launches": launch[6], "unroll": launch[7],
                "name": kname.value.decode()}

    def debug_compile(self, index, inputs, outputs) -> int:
        ia = (wt_image * len(inputs))(*inputs)
        oa = (wt_image * len(outputs))(*outputs)
        n = _i64()
        check(load().wt_debug_compile(self.h, index, ia, len(inputs), oa, len(outputs), ctypes.byref(n)))
        return n.value

    def debug_lanes(self, inputs, outputs):
        """Stream lanes of the run plan: (number of lanes, per launch a dict
        with its lane, the launches it waits for and its stages)."""
        ia = (wt_image * len(inputs))(*inputs)
        oa = (wt_image * len(outputs))(*outputs)
        n = _i32()
        check(load().wt_debug_lanes(self.h, ia, len(inputs), oa, len(outputs), None, 0, ctypes.byref(n)))
        out = (_i32 * n.value)()
        check(load().wt_debug_lanes(self.h, ia, len(inputs), oa, len(outputs), out, n.value, ctypes.byref(n)))
        v = list(out)
        launches, k = [], 2
        for _ in range(v[0]):
            lane, nw = v[k], v[k + 1]
            waits = v[k + 2:k + 2 + nw]
            k += 2 + nw
            ns = v[k]
            launches.append({"lane": lane, "waits": waits, "stages": v[k + 1:k + 1 + ns]})
            k += 1 + ns
        return v[1], launches

    def debug_host_bands(self, inputs, outputs):
        """Row bands of run_host for these images: a list of (y0, y1, ys, ye),
        kept output rows [y0, y1) computed from input rows [ys, ye); empty
        when the call runs the whole image at once."""
        ia = (wt_image * len(inputs))(*inputs)
        oa = (wt_image * len(outputs))(*outputs)
        n = _i32()
        check(load().wt_debug_host_bands(self.h, ia, len(inputs), oa, len(outputs), None, 0, ctypes.byref(n)))
        out = (_i32 * max(1, 4 * n.value))()
        check(load().wt_debug_host_bands(self.h, ia, len(inputs), oa, len(outputs), out, n.value, ctypes.byref(n)))
        return [tuple(out[4 * b:4 * b + 4]) for b in range(n.value)]

    def debug_segment_cost(self, first, n, width, height, dtype=WT_F32):
        """(cost, fused): the analytic model's weight of stages
        [first, first + n) as one group in wt_schedule_auto's DP-Fusion."""
        c, f = ctypes.c_double(), _i32()
        check(load().wt_debug_segment_cost(self.h, first, n, width, height, dtype, ctypes.byref(c), ctypes.byref(f)))
        return c.value, bool(f.value)

    def debug_layout(self, index, inputs, outputs):
        ia = (wt_image * len(inputs))(*inputs)
        oa = (wt_image * len(outputs))(*outputs)
        out = (_i32 * 256)()
        n = _i32()
        check(load().wt_debug_layout(self.h, index, ia, len(inputs), oa, len(outputs), out, 256, ctypes.byref(n)))
        v = list(out[:n.value])
        d = dict(zip(["warp_bytes", "bar_off", "chunk", "nbuf", "vec", "out_w", "n_src"], v[:7]))
        d["sources"] = [dict(zip(["ring_off", "bufb", "boxw", "esz"], v[7 + 4 * i: 11 + 4 * i]))
                        for i in range(d["n_src"])]
        return d

    def group_geometry(self, group=0, vec=4, frac_reg=1.0):
        out = (_i32 * 4096)()
        n = _i32()
        check(load().wt_debug_group_geometry(self.h, group, vec, frac_reg, out, 4096, ctypes.byref(n)))
        v = list(out[:n.value])
        head = dict(zip(["fusable", "halo_l", "halo_r", "halo_t", "halo_b", "unroll", "n_nodes"], v[:7]))
        nodes = []
        for i in range(head["n_nodes"]):
            r = v[7 + 10 * i: 17 + 10 * i]
            nodes.append(dict(id=r[0], src_chan=r[1], is_source=bool(r[2]), is_liveout=bool(r[3]),
                              top=r[4], bot=r[5], delay=r[6], window=r[7], xl=r[8] // 1000,
                              xr=r[8] % 1000, in_smem=bool(r[9])))
        head["nodes"] = nodes
        return head


class DeviceImage:
    """A planar device image (torch storage) with a 128-byte-aligned pitch.

    PyTorch only provides the device memory; the library reads and writes it
    through the wt_image descriptor."""

    def __init__(self, c, h, w, dtype=WT_F32, device="cuda", pin_host=False):
        import torch
        tdt = {WT_F32: torch.float32, WT_F16: torch.float16, WT_BF16: torch.bfloat16}[dtype]
        es = 4 if dtype == WT_F32 else 2
        pitch_el = (w * es + 127) // 128 * 128 // es
        if device == "cpu":
            self.t = torch.empty((c, h, pitch_el), dtype=tdt, pin_memory=pin_host)
        else:
            self.t = torch.empty((c, h, pitch_el), dtype=tdt, device=device)
        self.c, self.h, self.w, self.dtype = c, h, w, dtype
        self.pitch = pitch_el * es

    def view(self):
        return self.t[:, :, :self.w]

    def image(self) -> wt_image:
        return wt_image(self.t.data_ptr(), self.w, self.h, self.c, self.dtype, self.pitch)

    def upload(self, arr):
        """Stores a float array (C,H,W) or (H,W) after rounding to the dtype."""
        import numpy as np
        import torch
        from . import inputs as _inputs
        a = np.asarray(arr, dtype=np.float32).reshape(self.c, self.h, self.w)
        name = {WT_F32: "f32", WT_F16: "f16", WT_BF16: "bf16"}[self.dtype]
        s = _inputs.storage_array(a, name)
        if self.dtype == WT_BF16:
            src = torch.from_numpy(s.view(np.int16)).view(torch.bfloat16)
        else:
            src = torch.from_numpy(s)
        self.view().copy_(src)
        return self

    def download(self):
        """float32 numpy copy of the image."""
        return self.view().float().cpu().numpy()


# ------------------------------------------------------------- cost model

def gpu_config(device=-1) -> wt_gpu_config:
    c = wt_gpu_config()
    check(load().wt_gpu_config_get(device, ctypes.byref(c)))
    return c


def otpw_warp_sizes(block, warp_size=32):
    b = (_i32 * 3)(*block)
    w = (_i32 * 3)()
    check(load().wt_otpw_warp_sizes(b, warp_size, w))
    return list(w)


def otpw_scratchpad(block, warp, tile, overlap) -> int:
    n = _i64()
    arr = [(_i32 * 3)(*v) for v in (block, warp, tile, overlap)]
    check(load().wt_otpw_scratchpad(*arr, ctypes.byref(n)))
    return n.value


def cost_occupancy(cfg, smem_per_block, warps_per_block, regs_per_thread):
    occ = ctypes.c_double()
    tb = _i32()
    check(load().wt_cost_occupancy(ctypes.byref(cfg), smem_per_block, warps_per_block, regs_per_thread,
                                   ctypes.byref(occ), ctypes.byref(tb)))
    return occ.value, tb.value


def min_transactions(addresses, access_bytes, txn_bytes) -> int:
    a = (_i64 * max(1, len(addresses)))(*addresses)
    n = _i64()
    check(load().wt_min_transactions(a, len(addresses), access_bytes, txn_bytes, ctypes.byref(n)))
    return n.value


def cost_weights(new=None):
    lib = load()
    out = (ctypes.c_double * 7)()
    inp = (ctypes.c_double * 7)(*new) if new is not None else None
    check(lib.wt_cost_weights(inp, out))
    return list(out)


# ------------------------------------------------------------- learned model

COSTMODEL_FEATURES = 18
MLP_PARAMS = 64 * 18 + 64 + 64 * 64 + 64 + 64 + 1


def _fptr(a):
    import numpy as np
    assert a.dtype == np.float32 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_P(ctypes.c_float))


def costmodel_features(pipe, first, n, params=None, fused=True, width=4096, height=4096, dtype=WT_F32):
    """Feature vector (18 floats) of one launch (see wt_costmodel_features)."""
    import numpy as np
    f = np.zeros(COSTMODEL_FEATURES, np.float32)
    prm = None
    if params is not None:
        prm = wt_group_params()
        d = dict(tile_h=16, warps_per_block=2, frac_reg=1.0, vec=4, max_regs=0, chunk_rows=0, n_buffers=0, flags=0)
        d.update(params)
        for k, v in d.items():
            setattr(prm, k, v)
    check(load().wt_costmodel_features(pipe.h, first, n, ctypes.byref(prm) if prm is not None else None,
                                       int(fused), width, height, dtype, _fptr(f)))
    return f


def costmodel_collect(pipe, inputs, outputs, reps=10, stream=None):
    """(features [n, 18], log ms [n], stages [n, 2]) of the timed launches of
    one run of the installed schedule (see wt_costmodel_collect)."""
    import numpy as np
    ia = (wt_image * len(inputs))(*inputs)
    oa = (wt_image * len(outputs))(*outputs)
    n = _i32()
    lib = load()
    cap = 4 * len(pipe.spec["stages"]) + 4  # at least the launches of any run plan
    f = np.zeros((cap, COSTMODEL_FEATURES), np.float32)
    y = np.zeros(cap, np.float32)
    st = (_i32 * (2 * cap))()
    check(lib.wt_costmodel_collect(pipe.h, ia, len(inputs), oa, len(outputs), reps, stream, _fptr(f), _fptr(y), st,
                                   cap, ctypes.byref(n)))
    k = n.value
    return f[:k], y[:k], np.array(list(st), np.int32).reshape(-1, 2)[:k]


def mlp_train_steps(params, m, v, t0, x, y, idx, lr, weight_decay=0.0):
    """Runs the training kernel; params/m/v (float32, MLP_PARAMS) updated in
    place.  idx: (steps, batch) int32.  Returns the per-step losses."""
    import numpy as np
    x = np.ascontiguousarray(x, np.float32)
    y = np.ascontiguousarray(y, np.float32)
    idx = np.ascontiguousarray(idx, np.int32)
    steps, batch = idx.shape
    loss = np.zeros(max(1, steps), np.float32)
    check(load().wt_mlp_train_steps(_fptr(params), _fptr(m), _fptr(v), t0, _fptr(x), _fptr(y), x.shape[0],
                                    idx.ctypes.data_as(_P(_i32)), steps, batch, lr, weight_decay, _fptr(loss),
                                    None))
    return loss[:steps]


def mlp_forward(params, x):
    import numpy as np
    x = np.ascontiguousarray(x, np.float32)
    y = np.zeros(x.shape[0], np.float32)
    check(load().wt_mlp_forward(_fptr(params), _fptr(x), x.shape[0], _fptr(y), None))
    return y


def costmodel_train(features, log_ms, epochs=200, batch=64, lr=1e-3, seed=1):
    import numpy as np
    f = np.ascontiguousarray(features, np.float32)
    y = np.ascontiguousarray(log_ms, np.float32)
    loss = ctypes.c_float()
    check(load().wt_costmodel_train(_fptr(f), _fptr(y), f.shape[0], epochs, batch, lr, seed, ctypes.byref(loss)))
    return loss.value


def costmodel_predict(features):
    import numpy as np
    f = np.ascontiguousarray(features, np.float32).reshape(-1, COSTMODEL_FEATURES)
    y = np.zeros(f.shape[0], np.float32)
    check(load().wt_costmodel_predict(_fptr(f), f.shape[0], _fptr(y)))
    return y


def costmodel_ready() -> bool:
    return bool(load().wt_costmodel_ready())


def costmodel_reset():
    check(load().wt_costmodel_reset())


def costmodel_save(path):
    check(load().wt_costmodel_save(str(path).encode()))


def costmodel_load(path):
    check(load().wt_costmodel_load(str(path).encode()))


# ------------------------------------------------------ failure injection

def inject_alloc_failure(kind, after):
    """Makes the library's allocation of `kind` (0 host, 1 device) after
    `after` successful ones fail once (after < 0 disarms)."""
    check(load().wt_debug_inject_alloc_failure(kind, after))


def live_objects():
    """(live pipelines, device bytes held by the library)."""
    a, b = _i64(), _i64()
    check(load().wt_debug_live_objects(ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value

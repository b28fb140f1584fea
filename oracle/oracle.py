"""ctypes front end of the FP64 CPU oracle (TEST INFRASTRUCTURE ONLY).

Only tests/, ``__graft_entry__.smoke()`` and the cpu_baseline / ``--impl
reference`` legs of bench.py may import this module.  It shares no code with
the CUDA path: it reads a pipeline given as plain Python data (the stage DAG
is the program being evaluated, like the image is its data) and evaluates it
unfused in FP64 with the clamp-to-edge rule at every producer read
(Jangda & Guha, PACT'20, Sec. 2.2-2.3; see oracle.h for the readings).

Pipeline format (plain data, shared with the CUDA path only as an input):
    stages: list of dicts {"channels": int, "inputs": [int, ...],
                           "ops": [tuple, ...]}
    op tuples: ("const", v) | ("tap", slot, dx, dy[, chan[, mode]]) |
               ("tapz", slot, dx, dy, dz) (plane offset dz, clamped) |
               ("add",) ("sub",) ("mul",) ("div",) ("min",) ("max",)
               ("neg",) ("abs",) ("sqrt",) ("xpar",) ("ypar",) ("chan",)
    mode: "same" | "down2" | "up2" | "down4" | "up4" | "down8" | "up8";
          chan: -1 = consumer's channel.
    inputs: stage index >= 0, or -(j+1) for pipeline input j.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_OPS = {"const": 1, "tap": 2, "add": 3, "sub": 4, "mul": 5, "div": 6, "min": 7,
        "max": 8, "neg": 9, "abs": 10, "sqrt": 11, "xpar": 12, "ypar": 13, "chan": 14,
        "tapz": 15}
_MODES = {"same": 0, "down2": 1, "up2": 2, "down4": 3, "up4": 4, "down8": 5, "up8": 6}


class _Op(ctypes.Structure):
    _fields_ = [("op", ctypes.c_int32), ("slot", ctypes.c_int32),
                ("dx", ctypes.c_int32), ("dy", ctypes.c_int32),
                ("chan", ctypes.c_int32), ("mode", ctypes.c_int32),
                ("value", ctypes.c_double)]


class _Stage(ctypes.Structure):
    _fields_ = [("channels", ctypes.c_int32), ("n_in", ctypes.c_int32),
                ("inp", ctypes.POINTER(ctypes.c_int32)), ("n_ops", ctypes.c_int32),
                ("ops", ctypes.POINTER(_Op))]


class _Input(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("height", ctypes.c_int32),
                ("channels", ctypes.c_int32), ("data", ctypes.POINTER(ctypes.c_double))]


def build(force: bool = False) -> str:
    """Compiles liboracle.so with gcc (plain C99 + OpenMP); returns its path."""
    src = os.path.join(_HERE, "oracle.c")
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= max(os.path.getmtime(src),
                                             os.path.getmtime(os.path.join(_HERE, "oracle.h")))):
        return _SO
    tmp = _SO + ".%d.tmp" % os.getpid()
    subprocess.run(["gcc", "-O2", "-std=c99", "-fopenmp", "-fPIC", "-shared",
                    "-o", tmp, src, "-lm"], check=True)
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.POINTER
            lib.or_dag_shapes.argtypes = [P(_Stage), ctypes.c_int, P(_Input), ctypes.c_int,
                                          P(ctypes.c_int32), P(ctypes.c_int32),
                                          P(ctypes.c_int32), P(ctypes.c_int32)]
            lib.or_dag_eval.argtypes = [P(_Stage), ctypes.c_int, P(_Input), ctypes.c_int,
                                        P(ctypes.c_int32), ctypes.c_int,
                                        P(P(ctypes.c_double))]
            lib.or_dag_eval_points.argtypes = [P(_Stage), ctypes.c_int, P(_Input), ctypes.c_int,
                                               ctypes.c_int, ctypes.c_int, P(ctypes.c_int32),
                                               P(ctypes.c_int32), P(ctypes.c_int32),
                                               P(ctypes.c_double)]
            lib.or_brute.argtypes = [P(_Stage), ctypes.c_int, P(_Input), ctypes.c_int,
                                     ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]
            lib.or_brute.restype = ctypes.c_double
            dp = P(ctypes.c_double)
            lib.or_sharpen.argtypes = [dp, ctypes.c_int, ctypes.c_int, dp]
            lib.or_harris.argtypes = [dp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                      ctypes.c_double, dp]
            lib.or_blend.argtypes = [dp, dp, dp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_int, dp]
            lib.or_num_threads.restype = ctypes.c_int
            lib.or_set_num_threads.argtypes = [ctypes.c_int]
            _lib = lib
    return _lib


def num_threads() -> int:
    return int(_load().or_num_threads())


def set_num_threads(n: int) -> None:
    """Threads of the oracle's parallel loops from now on (timing only)."""
    _load().or_set_num_threads(int(n))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class _Packed:
    """Keeps the ctypes arrays of one pipeline alive."""

    def __init__(self, stages, inputs):
        self.keep = []
        n = len(stages)
        self.st = (_Stage * max(n, 1))()
        for s, S in enumerate(stages):
            ins = (ctypes.c_int32 * max(len(S["inputs"]), 1))(*S["inputs"])
            ops = (_Op * max(len(S["ops"]), 1))()
            for i, t in enumerate(S["ops"]):
                name = t[0]
                o = ops[i]
                o.op = _OPS[name]
                o.chan = -1
                if name == "const":
                    o.value = float(t[1])
                elif name == "tap":
                    o.slot, o.dx, o.dy = int(t[1]), int(t[2]), int(t[3])
                    if len(t) > 4:
                        o.chan = int(t[4])
                    if len(t) > 5:
                        o.mode = _MODES[t[5]]
                elif name == "tapz":
                    o.slot, o.dx, o.dy, o.chan = int(t[1]), int(t[2]), int(t[3]), int(t[4])
            self.keep += [ins, ops]
            self.st[s].channels = int(S["channels"])
            self.st[s].n_in = len(S["inputs"])
            self.st[s].inp = ins
            self.st[s].n_ops = len(S["ops"])
            self.st[s].ops = ops
        self.n = n
        self.arrays = [_f64(a) for a in inputs]
        self.inp = (_Input * max(len(self.arrays), 1))()
        for j, a in enumerate(self.arrays):
            if a.ndim == 2:
                a = a[None]
                self.arrays[j] = a
            c, h, w = a.shape
            self.inp[j].width, self.inp[j].height, self.inp[j].channels = w, h, c
            self.inp[j].data = _dp(a)
        self.n_in = len(self.arrays)


def _check(rc: int, what: str):
    if rc != 0:
        raise ValueError("oracle %s failed with code %d" % (what, rc))


def shapes(stages, inputs):
    """[(level, W, H, C)] of every stage."""
    lib = _load()
    p = _Packed(stages, inputs)
    n = max(p.n, 1)
    lv, W, H, C = [(ctypes.c_int32 * n)() for _ in range(4)]
    _check(lib.or_dag_shapes(p.st, p.n, p.inp, p.n_in, lv, W, H, C), "shapes")
    return [(lv[i], W[i], H[i], C[i]) for i in range(p.n)]


def evaluate(stages, inputs, outputs):
    """Full unfused FP64 evaluation; returns [array (C, H, W)] per output id."""
    lib = _load()
    shp = shapes(stages, inputs)
    p = _Packed(stages, inputs)
    outs = [np.empty((shp[s][3], shp[s][2], shp[s][1]), np.float64) for s in outputs]
    ids = (ctypes.c_int32 * max(len(outputs), 1))(*outputs)
    ptrs = (ctypes.POINTER(ctypes.c_double) * max(len(outputs), 1))(*[_dp(o) for o in outs])
    _check(lib.or_dag_eval(p.st, p.n, p.inp, p.n_in, ids, len(outputs), ptrs), "eval")
    return outs


def evaluate_points(stages, inputs, sid, xs, ys, cs=None):
    """Values of stage sid at the given points (exact, region-restricted)."""
    lib = _load()
    p = _Packed(stages, inputs)
    xs = np.ascontiguousarray(xs, dtype=np.int32)
    ys = np.ascontiguousarray(ys, dtype=np.int32)
    cs = np.zeros_like(xs) if cs is None else np.ascontiguousarray(cs, dtype=np.int32)
    out = np.empty(xs.shape[0], np.float64)
    ip = ctypes.POINTER(ctypes.c_int32)
    _check(lib.or_dag_eval_points(p.st, p.n, p.inp, p.n_in, sid, xs.shape[0],
                                  xs.ctypes.data_as(ip), ys.ctypes.data_as(ip),
                                  cs.ctypes.data_as(ip), _dp(out)), "points")
    return out


def brute(stages, inputs, sid, x, y, c=0):
    lib = _load()
    p = _Packed(stages, inputs)
    return float(lib.or_brute(p.st, p.n, p.inp, p.n_in, sid, x, y, c))


def sharpen(img):
    a = _f64(img)
    out = np.empty_like(a)
    _load().or_sharpen(_dp(a), a.shape[1], a.shape[0], _dp(out))
    return out


def harris(img, normalized=True, k=0.04):
    a = _f64(img)
    out = np.empty_like(a)
    _load().or_harris(_dp(a), a.shape[1], a.shape[0], 1 if normalized else 0, k, _dp(out))
    return out


def blend(A, B, M, levels=6):
    A, B, M = _f64(A), _f64(B), _f64(M)
    if M.ndim == 3:
        M = np.ascontiguousarray(M[0])
    C, H, W = A.shape
    out = np.empty_like(A)
    _load().or_blend(_dp(A), _dp(B), _dp(M), W, H, C, levels, _dp(out))
    return out

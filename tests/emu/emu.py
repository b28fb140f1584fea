"""Runs a generated group kernel on the CPU through the fiber emulator.

Test infrastructure for the CUDA path's code generator (never used by the
library): wt_debug_kernel gives the kernel text and its argument block for
host images; the text after the device-helper block is compiled with g++
against wt_emu.h and executed lane by lane.
"""
from __future__ import annotations

import concurrent.futures
import ctypes
import hashlib
import os
import subprocess
import threading

import numpy as np

from paper_1909_07190_gb300 import wt

HERE = os.path.dirname(os.path.abspath(__file__))
MARK = "// WT-DEVICE-HELPERS-END"
# compiled emulated kernels, kept inside the repository tree (git-ignored)
CACHE = os.path.join(os.path.dirname(os.path.dirname(HERE)), "_build", "emu_cache")
_loaded = {}

NP_DTYPES = {wt.WT_F32: np.float32, wt.WT_F16: np.float16, wt.WT_BF16: np.uint16}


class HostImage:
    """A planar host image with a 16-byte-multiple pitch (padding poisoned)."""

    def __init__(self, c, h, w, dtype=wt.WT_F32, fill=None):
        npd = NP_DTYPES[dtype]
        es = np.dtype(npd).itemsize
        pitch_el = ((w * es + 63) // 64 * 64) // es + 16 // es  # deliberately > row
        self.buf = np.empty((c, h, pitch_el), npd)
        if npd == np.uint16:
            self.buf.fill(0x7FC1)
        else:
            self.buf.fill(np.nan)
        self.c, self.h, self.w, self.dtype = c, h, w, dtype
        self.pitch = pitch_el * es
        if fill is not None:
            self.view()[...] = fill

    def view(self):
        return self.buf[:, :, :self.w]

    def image(self):
        return wt.image(self.buf.ctypes.data, self.w, self.h, self.c, self.dtype, self.pitch)

    def padding_intact(self):
        pad = self.buf[:, :, self.w:]
        if pad.dtype == np.uint16:
            return bool(np.all(pad == 0x7FC1))
        return bool(np.all(np.isnan(pad)))


def _runtime_object() -> str:
    """The emulator runtime, compiled once per content hash (it is the same
    for every kernel; compiling it with each kernel doubled a cold run)."""
    rt = os.path.join(HERE, "emu_rt.cpp")
    h = hashlib.sha1((open(rt).read() + open(os.path.join(HERE, "wt_emu.h")).read()).encode()).hexdigest()[:16]
    obj = os.path.join(CACHE, "emu_rt_%s.o" % h)
    if not os.path.exists(obj):
        os.makedirs(CACHE, exist_ok=True)
        tmp = obj + ".%d.tmp" % os.getpid()
        r = subprocess.run(["g++", "-O1", "-std=c++17", "-fPIC", "-c", "-w", "-I", HERE, rt, "-o", tmp],
                           capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("emulator runtime compile failed:\n" + r.stderr[-5000:])
        os.replace(tmp, obj)
    return obj


def _text(source: str):
    """(translation unit, content hash) of a generated kernel."""
    body = source.split(MARK, 1)[1]
    text = '#include "wt_emu.h"\n' + body + \
        '\nextern "C" long wt_emu_offset_err() { return (long)offsetof(WtArgs, err); }\n' + \
        'extern "C" long wt_emu_offset_direct() { return (long)offsetof(WtArgs, direct); }\n' + \
        'extern "C" long wt_emu_offset_queue() { return (long)offsetof(WtArgs, queue); }\n' + \
        'extern "C" long wt_emu_offset_tiles() { return (long)offsetof(WtArgs, tile_table); }\n' + \
        'extern "C" long wt_emu_offset_imgtab() { return (long)offsetof(WtArgs, img_tab); }\n'
    h = hashlib.sha1((text + open(os.path.join(HERE, "wt_emu.h")).read() +
                      open(os.path.join(HERE, "emu_rt.cpp")).read()).encode()).hexdigest()[:16]
    return text, h


def _build(text: str, name: str, h: str) -> str:
    """The shared object of one kernel, compiled unless already cached."""
    os.makedirs(CACHE, exist_ok=True)
    so = os.path.join(CACHE, "%s_%s.so" % (name, h))
    if not os.path.exists(so):
        rt = _runtime_object()
        # per-process and per-thread file names: parallel test workers may
        # build the same kernel at once.  -O0: the generated kernels are
        # long and run on small images here, so optimising them costs more
        # than it saves.
        tag = "%d.%d" % (os.getpid(), threading.get_ident())
        src = os.path.join(CACHE, "%s_%s.%s.cpp" % (name, h, tag))
        with open(src, "w") as f:
            f.write(text)
        tmp = so + ".%s.tmp" % tag
        r = subprocess.run(["g++", "-O0", "-std=c++17", "-fPIC", "-shared", "-w", "-I", HERE, src, rt, "-o", tmp],
                           capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("emulator compile failed:\n" + r.stderr[-5000:])
        os.replace(tmp, so)
        os.remove(src)
    return so


def _compile(source: str, name: str) -> ctypes.CDLL:
    text, h = _text(source)
    if h in _loaded:
        return _loaded[h]
    lib = ctypes.CDLL(_build(text, name, h))
    _loaded[h] = lib
    return lib


def precompile(pipe: "wt.Pipeline", inputs, outputs, workspace=None):
    """Compiles every launch of the run plan at once (one g++ per kernel,
    in parallel); run() then finds them built."""
    ii = [x.image() for x in inputs]
    oo = [x.image() for x in outputs]
    ws = None if workspace is None else (workspace.ctypes.data, workspace.nbytes)
    jobs = {}
    for i in range(pipe.launches_per_run()):
        try:
            d = pipe.debug_kernel(i, ii, oo, ws)
        except wt.WtError:
            return  # run() reports it
        text, h = _text(d["source"])
        if h not in _loaded:
            jobs[h] = (text, d["name"], h)
    if len(jobs) > 1:
        _runtime_object()
        with concurrent.futures.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
            list(ex.map(lambda j: _build(*j), jobs.values()))


def _register(lib, images, workspace=None):
    """The global buffers the kernel may touch (for the memory checker)."""
    lib.wt_emu_register.argtypes = [ctypes.c_void_p, ctypes.c_long]
    lib.wt_emu_clear_ranges()
    for x in images:
        lib.wt_emu_register(x.buf.ctypes.data, x.buf.nbytes)
    if workspace is not None and workspace.nbytes:
        lib.wt_emu_register(workspace.ctypes.data, workspace.nbytes)


def run(pipe: "wt.Pipeline", index: int, inputs, outputs, max_blocks=None, workspace=None, allow_err=False):
    """inputs/outputs: HostImage lists.  Runs launch `index` of the plan
    (with at most `max_blocks` blocks: persistent warps then take several
    tiles each).  allow_err: a raised error word is returned in d["err"]
    instead of failing (the tile queue must still be reset)."""
    ii = [x.image() for x in inputs]
    oo = [x.image() for x in outputs]
    ws = None if workspace is None else (workspace.ctypes.data, workspace.nbytes)
    d = pipe.debug_kernel(index, ii, oo, ws)
    lib = _compile(d["source"], d["name"])
    args = bytearray(d["args"])
    err = np.zeros(16, np.int32)
    queue = np.zeros(2, np.int32)
    off = lib.wt_emu_offset_err()
    args[off:off + 8] = int(err.ctypes.data).to_bytes(8, "little")
    qoff = lib.wt_emu_offset_queue()
    args[qoff:qoff + 8] = int(queue.ctypes.data).to_bytes(8, "little")
    abuf = (ctypes.c_char * len(args)).from_buffer(args)
    kfn = ctypes.cast(getattr(lib, d["name"]), ctypes.c_void_p)
    lib.wt_emu_run.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                               ctypes.c_int, ctypes.c_int, ctypes.c_char_p, ctypes.c_int]
    msg = ctypes.create_string_buffer(512)
    gx, gy, gz = d["grid"]
    # persistent warps (tile queue): at most max_blocks blocks take several
    # tiles each; one warp per tile (direct) needs every block
    direct = int.from_bytes(bytes(args[lib.wt_emu_offset_direct():][:4]), "little")
    if max_blocks is not None and d["fused"] and not direct:
        gx = min(gx, max_blocks)
    _register(lib, inputs + outputs, workspace)
    rc = lib.wt_emu_run(kfn, ctypes.addressof(abuf), gx, gy, gz, d["block"], d["smem"], msg, 512)
    if rc != 0:
        raise RuntimeError("emulated kernel failed: " + msg.value.decode())
    if err[0] != 0 and not allow_err:
        raise RuntimeError("emulated kernel raised error word %d" % err[0])
    if d["fused"] and (queue[0] != 0 or queue[1] != 0):
        raise RuntimeError("tile queue not reset at kernel exit: %s" % queue)
    d["err"] = int(err[0])
    return d


def run_batch(pipe: "wt.Pipeline", index: int, inputs, outputs, n_images, max_blocks=None):
    """Batched launch `index` (one persistent kernel over all images' tiles).
    inputs/outputs: flat HostImage lists, image-major."""
    ii = [x.image() for x in inputs]
    oo = [x.image() for x in outputs]
    d = pipe.debug_batch(index, ii, oo, n_images)
    lib = _compile(d["source"], d["name"])
    args = bytearray(d["args"])
    tab = np.frombuffer(bytearray(d["img_tab"]), np.uint8).copy()
    tiles = np.asarray(d["tiles"], np.int32)
    err = np.zeros(16, np.int32)
    queue = np.zeros(2, np.int32)
    for off_fn, arr in ((lib.wt_emu_offset_err, err), (lib.wt_emu_offset_queue, queue),
                        (lib.wt_emu_offset_tiles, tiles), (lib.wt_emu_offset_imgtab, tab)):
        off = off_fn()
        args[off:off + 8] = int(arr.ctypes.data).to_bytes(8, "little")
    abuf = (ctypes.c_char * len(args)).from_buffer(args)
    kfn = ctypes.cast(getattr(lib, d["name"]), ctypes.c_void_p)
    lib.wt_emu_run.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                               ctypes.c_int, ctypes.c_int, ctypes.c_char_p, ctypes.c_int]
    msg = ctypes.create_string_buffer(512)
    gx = d["grid"][0] if max_blocks is None else min(d["grid"][0], max_blocks)
    _register(lib, inputs + outputs)
    rc = lib.wt_emu_run(kfn, ctypes.addressof(abuf), gx, 1, 1, d["block"], d["smem"], msg, 512)
    if rc != 0:
        raise RuntimeError("emulated kernel failed: " + msg.value.decode())
    if err[0] != 0:
        raise RuntimeError("emulated kernel raised error word %d" % err[0])
    if queue[0] != 0 or queue[1] != 0:
        raise RuntimeError("tile queue not reset at kernel exit: %s" % queue)
    return d

"""Benchmark: Mpixels/s of the fused warp-tiled pipeline on one GB300 per rank.

Workload (default): the 11-stage corner-response pipeline on a 4096x4096
single-channel FP32 image (uniform [0,1) from seed 190907192).  One step =
one wt_run of the whole pipeline over one image.  Inputs are resident in HBM;
consecutive steps rotate over buffer sets whose total size exceeds 3x L2, so
every step reads and writes HBM.  The schedule is the library's default
(one fused group) unless --tune on runs its measured schedule search
(wt_schedule_tune) first; batches are always tuned.  Prints one JSON line
(rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
  python bench.py --impl reference ...   # the FP64 CPU oracle on host cores

Workloads: harris (default), harris_f16, sharpen, and harris_batch -- 512
images with sides uniform in [200, 4096], FP16 storage, one wt_run_batch
(one persistent launch) per step.

Under torchrun each rank runs an independent replica on its own GPU (the
method shards by image with no exchange): value = pixels of all ranks / max
time over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1909_07190_gb300 import inputs as I  # noqa: E402
from paper_1909_07190_gb300 import pipelines as P  # noqa: E402

METRIC = "Mpixels/s per pipeline on 1 GB300, fused vs unfused GPU path, % of HBM roofline"
WORKLOADS = {
    # name: (pipeline, width, height, storage dtype, seed)
    "harris": ("harris", 4096, 4096, "f32", I.SEED_BASE + 2),
    "harris_f16": ("harris", 4096, 4096, "f16", I.SEED_BASE + 2),
    "sharpen": ("sharpen", 2048, 2048, "f32", I.SEED_BASE + 1),
    # 512 images, sides uniform in [200, 4096] (sizes from seed 190907193)
    "harris_batch": ("harris", 0, 0, "f16", I.SEED_BASE + 3),
    # two 8192x8192x3 images and a smooth mask, 6-level pyramids (36 stages)
    "blend": ("blend", 8192, 8192, "bf16", I.SEED_BASE + 5),
    # bilateral filter through a grid of 8x8-pixel cells and 8 intensity bins
    "bilateral": ("bilateral", 4096, 4096, "f32", I.SEED_BASE + 6),
    # 3-D groups: 512x512x256 FP32 volumes (a pixel is a voxel)
    "unsharp3d": ("unsharp3d", 512, 512, "f32", I.SEED_BASE + 8),
    "heat3d": ("heat3d", 512, 512, "f32", I.SEED_BASE + 9),
}
VOLUME_DEPTH = 256
# 3-D group parameters: the fastest of the 3-D study's sweep on one GB300
VOLUME_PARAMS = {"unsharp3d": dict(tile_h=64, tile_o=4, vec=1, warps_per_block=1, max_regs=128, n_buffers=1,
                                    flags=32),
                 "heat3d": dict(tile_h=64, tile_o=4, vec=1, warps_per_block=1, max_regs=128, n_buffers=1,
                                frac_reg=1.0, flags=32)}


def spec_for(name):
    """The workload's stage DAG (volumes: VOLUME_DEPTH planes; the heat
    workload is two fused diffusion steps)."""
    if name == "unsharp3d":
        return P.unsharp3d(depth=VOLUME_DEPTH)
    if name == "heat3d":
        return P.heat3d(2, depth=VOLUME_DEPTH)
    return P.by_name(name)


def spec_for_depth(name, depth):
    """A volume workload's DAG at another depth (bounded CPU samples)."""
    return P.unsharp3d(depth=depth) if name == "unsharp3d" else P.heat3d(2, depth=depth)


BATCH_IMAGES = 512


class _Args:
    batch_images = 0


args_global = _Args()  # options the workload classes read (set by main)
# pyramid levels a tap mode moves (down: the producer is finer)
LEVEL_DELTA = {"same": 0, "down2": 1, "up2": -1, "down4": 2, "up4": -2, "down8": 3, "up8": -3}
CLOCK_FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def ops_per_pixel(spec):
    """FP32 operations of the stage programs per output pixel (level-0
    pixel; channels counted): the algorithmic ALU work of the pipeline."""
    arith = {"add", "sub", "mul", "div", "min", "max", "neg", "abs", "sqrt"}
    level = {}
    total = 0.0
    for i, st in enumerate(spec["stages"]):
        lv = None
        for op in st["ops"]:
            if op[0] != "tap":
                continue
            src = st["inputs"][op[1]]
            base = level.get(src, 0) if src >= 0 else 0
            mode = op[5] if len(op) > 5 else "same"
            lv = base + LEVEL_DELTA[mode]
            break
        level[i] = lv or 0
        n = sum(1 for op in st["ops"] if op[0] in arith)
        total += n * st["channels"] / 4.0 ** level[i]
    return total


def max_over_ranks(value, dist, device):
    """The largest of the ranks' values: a job's time is its slowest rank's
    (every rank holds the result)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(px_per_rank_step, world, steps, total_ms):
    """Whole-job Mpixels/s: the pixels every rank processed over the slowest
    rank's time (replicas: each rank runs its own images, weak scaling)."""
    return px_per_rank_step * world * steps / (total_ms / 1e3) / 1e6


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    def __init__(self, index):
        self.index = index
        self.p = None
        self.path = None

    def __enter__(self):
        try:
            import tempfile
            if subprocess.run(["nvidia-smi", "-L"], capture_output=True).returncode != 0:
                return self
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + CLOCK_FIELDS,
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            time.sleep(1.5)  # first samples arrive after start-up
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except Exception:
                self.p.kill()

    def summary(self):
        if self.p is None or not self.path:
            return None
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i, v in enumerate(r) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def cpu_oracle_rate(spec, img, budget_s):
    """Mpx/s of the FP64 oracle on this host's cores over repeated full images."""
    from oracle import oracle as O
    x = img.astype(np.float64)
    n, t0 = 0, time.perf_counter()
    while True:
        O.evaluate(spec["stages"], [x], spec["outputs"])
        n += 1
        dt = time.perf_counter() - t0
        if dt >= budget_s:
            break
    px = n * img.size  # pixels of every plane of a volume (voxels)
    return px / dt / 1e6, O.num_threads(), n, dt


def cpu_blend_rate(dts, budget_s, w=1024, h=1024):
    """Mpx/s of the FP64 oracle's blend on a bounded sample: repeated
    1024x1024x3 blends (the same 36 stages)."""
    from oracle import oracle as O
    spec = P.blend()
    ins = [I.round_to(I.uniform_image(I.SEED_BASE + 5, w, h, 3), dts).astype(np.float64),
           I.round_to(I.uniform_image(I.SEED_BASE + 1005, w, h, 3), dts).astype(np.float64),
           I.round_to(I.smooth_mask(I.SEED_BASE + 2005, w, h), dts).astype(np.float64)]
    n, t0 = 0, time.perf_counter()
    while True:
        O.evaluate(spec["stages"], ins, spec["outputs"])
        n += 1
        dt = time.perf_counter() - t0
        if dt >= budget_s:
            break
    return n * w * h / dt / 1e6, O.num_threads(), n, dt, "%d full %dx%dx3 blends, %.1f s" % (n, w, h, dt)


def batch_sizes(n=None):
    return I.batch_sizes(I.SEED_BASE + 3, BATCH_IMAGES, 200, 4096)[:n or BATCH_IMAGES]


def run_reference(args, rank):
    """The FP64 oracle on the host cores, one bounded sample per step: the
    whole image (single-image workloads) or one image of the batch, cycling
    through the batch's sizes."""
    if rank != 0:
        return
    name, W, H, dt, seed = WORKLOADS[args.workload]
    spec = spec_for(name)
    if name == "blend":
        # bounded sample: one 1024x1024x3 blend per step
        from oracle import oracle as O
        for _ in range(args.warmup):
            cpu_blend_rate(dt, 0.0)
        px, t0 = 0, time.perf_counter()
        cores = O.num_threads()
        for _ in range(args.steps):
            cpu_blend_rate(dt, 0.0)
            px += 1024 * 1024
        total = time.perf_counter() - t0
        value = px / total / 1e6
        line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "Mpixels/s",
                "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": total / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": workload_config(args.workload, spec, W, H, W * H),
                "cpu_baseline": {"value": value, "unit": "Mpixels/s", "cores": cores, "kind": "oracle",
                                 "sample": "one 1024x1024x3 blend per step"},
                "e2e": {"value": value, "unit": "Mpixels/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return
    if args.workload == "harris_batch":
        sizes = batch_sizes()
        ref_config = workload_config(args.workload, spec, W, H, sum(w * h for w, h in sizes), len(sizes))
    else:
        ref_config = workload_config(args.workload, spec, W, H,
                                     W * H * (VOLUME_DEPTH if name in ("unsharp3d", "heat3d") else 1))
    if args.workload == "harris_batch":
        imgs = [I.round_to(I.uniform_image(seed * 1000 + i, w, h)[0], dt) for i, (w, h) in
                enumerate(sizes[:max(1, args.steps + args.warmup)])]
        sample = "one image of the 512-image batch per step (its sizes in order)"
    elif name == "bilateral":
        imgs = [I.round_to(I.uniform_image(seed, W, H)[0][:1024, :1024], dt)]
        sample = "one 1024x1024 crop of the %dx%d image per step" % (W, H)
    elif name in ("unsharp3d", "heat3d"):
        imgs = [I.round_to(I.uniform_image(seed, W, H, VOLUME_DEPTH)[:32], dt)]
        sample = "the first 32 planes of the %dx%dx%d volume per step" % (W, H, VOLUME_DEPTH)
    else:
        imgs = [I.round_to(I.uniform_image(seed, W, H)[0], dt)]
        sample = "one full %dx%d image per step" % (W, H)
    for k in range(args.warmup):
        img = imgs[k % len(imgs)]
        cpu_oracle_rate(spec if img.ndim == 2 else spec_for_depth(name, img.shape[0]), img, 0.0)
    px = 0
    t0 = time.perf_counter()
    cores = 1
    for k in range(args.steps):
        img = imgs[(args.warmup + k) % len(imgs)]
        _, cores, _, _ = cpu_oracle_rate(spec if img.ndim == 2 else spec_for_depth(name, img.shape[0]), img, 0.0)
        px += img.size
    total = time.perf_counter() - t0
    value = px / total / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "Mpixels/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": total / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": ref_config,
            "cpu_baseline": {"value": value, "unit": "Mpixels/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "Mpixels/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def stage_levels(spec):
    """Pyramid level of every stage (inputs are level 0): a stage sits one
    level coarser than the producers it reads by down-sampling taps, one
    finer than those read by up-sampling taps."""
    lv = []
    for st in spec["stages"]:
        level = None
        for op in st["ops"]:
            if op[0] != "tap":
                continue
            pid = st["inputs"][op[1]]
            pl = 0 if pid < 0 else lv[pid]
            level = pl + LEVEL_DELTA[op[5]]
            break
        lv.append(0 if level is None else level)
    return lv


def launch_io_bytes(spec, stages, W, H, esz):
    """Algorithmic bytes of one launch over `stages`: every producer it reads
    from outside (once) plus every stage it stores (read later or a pipeline
    output), each at its own level's size (ceil(W / 2^l) x ceil(H / 2^l))."""
    lv = stage_levels(spec)
    S = spec["stages"]
    inside = set(stages)

    def size(pid):
        c = spec["inputs"][-pid - 1] if pid < 0 else S[pid]["channels"]
        level = 0 if pid < 0 else lv[pid]
        w, h = W, H
        for _ in range(level):
            w, h = (w + 1) // 2, (h + 1) // 2
        return w * h * c * esz

    reads = {pid for s in stages for pid in S[s]["inputs"] if pid not in inside}
    writes = {s for s in stages if s in spec["outputs"] or
              any(s in S[c]["inputs"] for c in range(len(S)) if c not in inside)}
    return sum(size(p) for p in reads) + sum(size(s) for s in writes)


def dominant_launch(pipe, ins, outs, spec, W, H, esz, sp):
    """(kernel name, algorithmic bytes, mean ms, launches) of the launch of
    one run that takes the most time, from per-launch CUDA events on the
    stream."""
    t = pipe.time_launches(ins, outs, 20, sp)
    i = max(range(len(t)), key=lambda k: t[k][3])
    first, n, _, ms = t[i]
    return (pipe.kernel_name(i, ins, outs), launch_io_bytes(spec, list(range(first, first + n)), W, H, esz), ms,
            len(t))


class Single:
    """One image per step, rotating over buffer sets larger than 3x L2."""

    planes = 1

    def __init__(self, wt, torch, spec, W, H, dtype, seed, local):
        self.wt, self.torch = wt, torch
        self.W, self.H, self.dtype = W, H, dtype
        self.esz = 4 if dtype == wt.WT_F32 else 2
        C = self.planes
        self.img = I.uniform_image(seed, W, H, C)
        if C == 1:
            self.img = self.img[0]
        set_bytes = 2 * W * H * C * self.esz
        l2 = torch.cuda.get_device_properties(local).L2_cache_size
        self.nsets = max(3, -(-3 * l2 // set_bytes))
        self.ins = [wt.DeviceImage(C, H, W, dtype).upload(self.img) for _ in range(self.nsets)]
        self.outs = [wt.DeviceImage(C, H, W, dtype) for _ in range(self.nsets)]
        self.px = W * H * C
        self.alg_bytes = 2 * W * H * C * self.esz
        self.l2_note = "rotating %d input/output sets (%.0f MB) > 3x L2" % (self.nsets, self.nsets * set_bytes / 1e6)

    def run(self, pipe, i, sp):
        k = i % self.nsets
        pipe.run([self.ins[k].image()], [self.outs[k].image()], sp)

    def tune(self, pipe, sp):
        return pipe.schedule_tune([self.ins[0].image()], [self.outs[0].image()], 0, 0, 20, sp)

    def kernel_name(self, pipe):
        return pipe.debug_kernel(0, [self.ins[0].image()], [self.outs[0].image()])["name"]

    def io(self):
        """Inputs and outputs of one run (the first buffer set)."""
        return [self.ins[0].image()], [self.outs[0].image()]

    def dominant(self, pipe, sp, spec):
        return dominant_launch(pipe, [self.ins[0].image()], [self.outs[0].image()], spec, self.W, self.H, self.esz,
                               sp)

    def e2e(self, pipe, sp, warmup, steps):
        wt, torch = self.wt, self.torch
        hin = wt.DeviceImage(self.planes, self.H, self.W, self.dtype, device="cpu", pin_host=True)
        hin.view().copy_(self.ins[0].view().cpu())
        hout = wt.DeviceImage(self.planes, self.H, self.W, self.dtype, device="cpu", pin_host=True)
        for _ in range(warmup):
            pipe.run_host([hin.image()], [hout.image()], sp)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(steps):
            pipe.run_host([hin.image()], [hout.image()], sp)
        return self.px * steps / (time.perf_counter() - t0) / 1e6, self.px * self.esz, self.px * self.esz

    def cpu_sample(self, dts):
        return I.round_to(self.img, dts)


class Volume(Single):
    """A 512x512x256 volume per step (3-D group, App. A), rotating over
    buffer sets like Single; the CPU oracle runs on its first 32 planes."""

    planes = VOLUME_DEPTH

    def __init__(self, wt, torch, spec, W, H, dtype, seed, local, name):
        self.name = name
        super().__init__(wt, torch, spec, W, H, dtype, seed, local)

    def schedule(self, fused, plain):
        fused.schedule(params=[VOLUME_PARAMS[self.name]])

    def cpu_sample(self, dts):
        return I.round_to(self.img[:32], dts)


class Grid(Single):
    """The bilateral filter through a grid: one image per step like Single,
    with the pipeline's level-by-level schedule; the CPU oracle runs on a
    1024x1024 crop (its grid at level 1 alone is 16 planes)."""

    def schedule(self, fused, plain):
        groups, params = P.bilateral_schedule()
        fused.schedule(groups=groups, params=params)

    def cpu_sample(self, dts):
        return I.round_to(self.img[:1024, :1024], dts)


class Blend:
    """The multi-scale blend: A, B (8192x8192x3) and the mask in, the 3-channel
    blend out, BF16; three buffer sets (1.3 GB each, far beyond L2).  A and B
    are drawn on the device with the host generator's stream, the mask on
    the host.  Fused schedule: one group per pyramid level."""

    def __init__(self, wt, torch, spec, W, H, dtype, seed):
        from paper_1909_07190_gb300 import inputs_torch as IT
        self.wt, self.torch = wt, torch
        self.W, self.H, self.dtype = W, H, dtype
        self.esz = 4 if dtype == wt.WT_F32 else 2
        tdt = {wt.WT_F32: torch.float32, wt.WT_F16: torch.float16, wt.WT_BF16: torch.bfloat16}[dtype]
        self.seeds = (seed, seed + 1000, seed + 2000)
        self.mask = I.smooth_mask(self.seeds[2], W, H)
        self.nsets = 3
        self.ins, self.outs = [], []
        for _ in range(self.nsets):
            a = wt.DeviceImage(3, H, W, dtype)
            a.view().copy_(IT.uniform_image(self.seeds[0], W, H, 3).to(tdt))
            b = wt.DeviceImage(3, H, W, dtype)
            b.view().copy_(IT.uniform_image(self.seeds[1], W, H, 3).to(tdt))
            m = wt.DeviceImage(1, H, W, dtype)
            m.view().copy_(torch.from_numpy(self.mask).to(tdt))
            self.ins.append([a, b, m])
            self.outs.append(wt.DeviceImage(3, H, W, dtype))
        self.px = W * H
        self.alg_bytes = (3 + 3 + 1 + 3) * W * H * self.esz
        self.l2_note = "rotating %d input/output sets (%.0f MB) > 3x L2" % (self.nsets, self.alg_bytes / 1e6)

    def schedule(self, fused, plain):
        groups, params = P.blend_schedule()
        fused.schedule(groups=groups, params=params)

    def run(self, pipe, i, sp):
        k = i % self.nsets
        pipe.run([x.image() for x in self.ins[k]], [self.outs[k].image()], sp)

    def tune(self, pipe, sp):
        return pipe.schedule_tune([x.image() for x in self.ins[0]], [self.outs[0].image()], 0, 4, 5, sp)

    def kernel_name(self, pipe, index=None):
        # default: the last launch (the finest level's group)
        if index is None:
            index = pipe.launches_per_run() - 1
        return pipe.kernel_name(index, [x.image() for x in self.ins[0]], [self.outs[0].image()])

    def dominant(self, pipe, sp, spec):
        return dominant_launch(pipe, [x.image() for x in self.ins[0]], [self.outs[0].image()], spec, self.W, self.H,
                               self.esz, sp)

    def e2e(self, pipe, sp, warmup, steps):
        wt, torch = self.wt, self.torch
        hin = [wt.DeviceImage(x.c, self.H, self.W, self.dtype, device="cpu", pin_host=True) for x in self.ins[0]]
        for h, x in zip(hin, self.ins[0]):
            h.view().copy_(x.view().cpu())
        hout = wt.DeviceImage(3, self.H, self.W, self.dtype, device="cpu", pin_host=True)
        for _ in range(warmup):
            pipe.run_host([h.image() for h in hin], [hout.image()], sp)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(steps):
            pipe.run_host([h.image() for h in hin], [hout.image()], sp)
        nb = sum(h.t.numel() * h.t.element_size() for h in hin)
        return self.px * steps / (time.perf_counter() - t0) / 1e6, nb, hout.t.numel() * hout.t.element_size()

    def cpu_sample(self, dts):
        return None


class Batch:
    """All 512 images per step (one wt_run_batch); 4.9 GB in + out, far
    beyond L2.  Inputs drawn on the device with the host generator's stream."""

    def __init__(self, wt, torch, spec, dtype, seed):
        from paper_1909_07190_gb300 import inputs_torch as IT
        self.wt, self.torch = wt, torch
        self.dtype = dtype
        self.esz = 4 if dtype == wt.WT_F32 else 2
        self.sizes = batch_sizes(getattr(args_global, "batch_images", 0))
        self.seed = seed
        self.ins, self.outs = [], []
        for i, (w, h) in enumerate(self.sizes):
            d = wt.DeviceImage(1, h, w, dtype)
            d.view().copy_(IT.uniform_image(seed * 1000 + i, w, h).to(d.t.dtype))
            self.ins.append(d)
            self.outs.append(wt.DeviceImage(1, h, w, dtype))
        self.ii = [x.image() for x in self.ins]
        self.oo = [x.image() for x in self.outs]
        self.px = sum(w * h for w, h in self.sizes)
        self.alg_bytes = 2 * self.px * self.esz
        self.l2_note = "batch of %d images, %.2f GB in+out (> L2)" % (len(self.sizes), self.alg_bytes / 1e9)

    def run(self, pipe, i, sp):
        pipe.run_batch(self.ii, self.oo, len(self.sizes), sp)

    def tune(self, pipe, sp):
        return pipe.schedule_tune(self.ii, self.oo, len(self.sizes), 0, 5, sp)

    def kernel_name(self, pipe):
        return pipe.debug_batch(0, self.ii[:1], self.oo[:1], 1)["name"]

    def e2e(self, pipe, sp, warmup, steps):
        """Pinned host images: per step every input copied in, one batched
        run, every output copied back."""
        torch = self.torch
        hin = [torch.empty_like(x.t, device="cpu").pin_memory() for x in self.ins]
        hout = [torch.empty_like(x.t, device="cpu").pin_memory() for x in self.outs]
        for h, x in zip(hin, self.ins):
            h.copy_(x.t)

        def step():
            for h, x in zip(hin, self.ins):
                x.t.copy_(h, non_blocking=True)
            pipe.run_batch(self.ii, self.oo, len(self.sizes), sp)
            for h, x in zip(hout, self.outs):
                h.copy_(x.t, non_blocking=True)
            torch.cuda.current_stream().synchronize()

        for _ in range(warmup):
            step()
        t0 = time.perf_counter()
        for _ in range(steps):
            step()
        nb = sum(x.t.numel() * x.t.element_size() for x in self.ins)
        return self.px * steps / (time.perf_counter() - t0) / 1e6, nb, nb

    def cpu_sample(self, dts):
        w, h = self.sizes[0]
        return I.round_to(I.uniform_image(self.seed * 1000, w, h)[0], dts)


def workload_config(workload, spec, W, H, px, images=None):
    """The workload's description, identical in both arms (the repo's kernels
    and the oracle): what is computed, not how."""
    name = WORKLOADS[workload][0]
    cfg = {"workload": workload, "pipeline": name, "width": W, "height": H,
           "channels": VOLUME_DEPTH if name in ("unsharp3d", "heat3d") else (3 if name == "blend" else 1),
           "storage": WORKLOADS[workload][3], "stages": len(spec["stages"]), "pixels_per_step": px}
    if images is not None:
        cfg["images"] = images
    return cfg


def device_fp32_peak(clocks):
    """FP32 lane operations per second of the device (an FMA counted once):
    SMs x FP32 lanes per SM (the library's device query) x the maximum SM
    clock (nvidia-smi's clocks.max.sm during the run, else the driver-written
    measured peaks file)."""
    from paper_1909_07190_gb300 import wt
    cfg = wt.gpu_config(0)
    mhz = (clocks or {}).get("sm_max_mhz")
    if not mhz:
        try:
            with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
                mhz = float(json.load(f)["sm_max_mhz"])
        except Exception:
            mhz = None
    if not mhz:
        return None, cfg.nsms
    return cfg.nsms * cfg.cores_per_sm * mhz * 1e6, cfg.nsms


def make_work(wt, torch, workload, rank, local, size=0):
    name, W, H, dts, seed = WORKLOADS[workload]
    if size:
        W = H = size
    dtype = wt.DTYPES[dts]
    spec = spec_for(name)
    if workload == "harris_batch":
        work = Batch(wt, torch, spec, dtype, seed + 7919 * rank)
    elif name == "blend":
        work = Blend(wt, torch, spec, W, H, dtype, seed + 7919 * rank)
    elif name == "bilateral":
        work = Grid(wt, torch, spec, W, H, dtype, seed + rank, local)
    elif name in ("unsharp3d", "heat3d"):
        work = Volume(wt, torch, spec, W, H, dtype, seed + rank, local, name)
    else:
        work = Single(wt, torch, spec, W, H, dtype, seed + rank, local)
    return name, W, H, dts, spec, work


def timed_steps(torch, work, step_fn, steps, warmup, per_graph, dist, sampler=None):
    """Kernel-only time of exactly `steps` steps: CUDA graphs of up to
    `per_graph` back-to-back steps, replayed, CUDA events around the replays
    on the capturing stream (no host work inside the region)."""
    sp = torch.cuda.current_stream().cuda_stream
    for i in range(max(warmup, getattr(work, "nsets", 1))):  # every buffer set once
        step_fn(i, sp)
    torch.cuda.synchronize()

    def capture(n):
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            cs = torch.cuda.current_stream().cuda_stream
            for i in range(n):
                step_fn(i, cs)
        return g

    n = min(per_graph, steps)
    full, rem = divmod(steps, n)
    g = capture(n)
    gr = capture(rem) if rem else None
    g.replay()
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    cur = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(full + 2)]
    ctx = sampler if sampler is not None else _Null()
    with ctx:
        ev[0].record(cur)
        for r in range(full):
            g.replay()
            ev[r + 1].record(cur)
        if gr is not None:
            gr.replay()
        ev[full + 1].record(cur)
        torch.cuda.synchronize()
    per = [ev[r].elapsed_time(ev[r + 1]) / n for r in range(full)]
    total = max_over_ranks(ev[0].elapsed_time(ev[full + 1]), dist, "cuda")
    if dist is not None:
        dist.barrier()
    return total, per


def traffic_record(workload, kname):
    """ncu figures of the kernel from the committed profile summary (DRAM
    bytes and executed warp instructions per launch), used only when they
    were taken on the kernel that ran here (same generated kernel name).  A
    workload whose schedule is tuned at run time may list one record per
    kernel the search picks."""
    tpath = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        recs = json.load(open(tpath)).get(workload)
        for rec in (recs if isinstance(recs, list) else [recs]):
            if rec and rec.get("kernel") == kname:
                return rec
    except Exception:
        pass
    return None


def measure(wt, torch, workload, args, dist, world, rank, local, steps, warmup, cpu_seconds, size=0):
    """One workload on this rank: fused rate, unfused rate, roofline of the
    dominant kernel, end-to-end rate through the host-buffer call and the
    oracle's CPU rate (rank 0 alone, cpu_seconds > 0)."""
    name, W, H, dts, spec, work = make_work(wt, torch, workload, rank, local, size)
    batched = workload == "harris_batch"
    sp = torch.cuda.current_stream().cuda_stream
    fused = wt.Pipeline(spec)
    if hasattr(work, "schedule"):
        work.schedule(fused, None)
    if args.params and workload == args.workload:
        prm = json.loads(args.params)
        if name == "blend":
            groups, params = P.blend_schedule()
            fused.schedule(groups=groups, params=[dict(p, **prm) for p in params])
        else:
            fused.schedule(params=prm)
    tuning = None
    if args.tune == "on" or (args.tune == "auto" and batched):
        t0 = time.perf_counter()
        tuned_ms, n_timed = work.tune(fused, sp)
        tuning = {"schedules_timed": n_timed, "tuned_ms": tuned_ms, "seconds": round(time.perf_counter() - t0, 1)}
    per_graph = 10 if batched else 100
    sampler = ClockSampler(local)
    total_f, per_f = timed_steps(torch, work, lambda i, s: work.run(fused, i, s), steps, warmup, per_graph, dist,
                                 sampler)
    clocks = sampler.summary()
    fused.check(sp)
    unfused = None
    if not batched:
        plain = wt.Pipeline(spec)
        plain.schedule(exec_mode=wt.WT_EXEC_PLAIN)
        plain_steps = max(3, steps // 8)
        total_p, _ = timed_steps(torch, work, lambda i, s: work.run(plain, i, s), plain_steps, warmup, per_graph,
                                 dist)
        plain.check(sp)
        unfused = {"value": job_rate(work.px, world, plain_steps, total_p), "unit": "Mpixels/s",
                   "ms_per_step": total_p / plain_steps, "launches_per_step": plain.launches_per_run(),
                   "intermediates": "f32"}
        plain.close()
        if WORKLOADS[workload][3] != "f32":
            # the same per-stage kernels with intermediates in the storage type
            plain16 = wt.Pipeline(spec)
            plain16.schedule(exec_mode=wt.WT_EXEC_PLAIN, intermediate_dtype=wt.DTYPES[WORKLOADS[workload][3]])
            total_q, _ = timed_steps(torch, work, lambda i, s: work.run(plain16, i, s), plain_steps, warmup,
                                     per_graph, dist)
            plain16.check(sp)
            unfused["storage_type_intermediates"] = {
                "value": job_rate(work.px, world, plain_steps, total_q), "unit": "Mpixels/s",
                "ms_per_step": total_q / plain_steps, "intermediates": WORKLOADS[workload][3]}
            plain16.close()
    e2e_steps = max(3, min(200, steps // 4)) if not batched else 3
    e2e_value, h2d, d2h = work.e2e(fused, sp, warmup if not batched else 1, e2e_steps)
    value = job_rate(work.px, world, steps, total_f)
    launch_ms = statistics.mean(per_f)
    peak, peak_kind = peaks()
    launches = fused.launches_per_run()
    if hasattr(work, "dominant") and launches > 1:
        # several launches per run: the dominant launch's own bytes over its
        # own event-timed duration; the whole run beside it
        kname, kbytes, kms, _ = work.dominant(fused, sp, spec)
        run_roof = {"achieved": work.alg_bytes / (launch_ms / 1e3) / 1e9, "bytes_per_run": work.alg_bytes,
                    "ms_per_run": launch_ms, "frac": work.alg_bytes / (launch_ms / 1e3) / 1e9 / peak}
    else:
        kname, kbytes, kms = work.kernel_name(fused), work.alg_bytes // launches, launch_ms
        run_roof = None
    achieved = kbytes / (kms / 1e3) / 1e9
    rec = traffic_record(workload, kname)
    fp32, nsm = device_fp32_peak(clocks)
    opx = ops_per_pixel(spec) / getattr(work, "planes", 1)
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": rec["dram_bytes_per_launch"] if rec else None, "peak_kind": peak_kind, "kernel": kname,
            "algorithmic_bytes_per_launch": kbytes, "kernel_ms": kms, "whole_run": run_roof}
    if fp32:
        # the stage programs' FP32 operations per pixel against the FP32 lanes
        roof["alu"] = {"ops_per_px": opx, "achieved_tops": opx * value / 1e6 / world, "peak_tops": fp32 / 1e12,
                       "frac": opx * value * 1e6 / world / fp32,
                       "note": "operations of the stage programs as written; the kernels execute fewer where "
                               "constants fold (deferred scales, up-sampling phases), so this can exceed 1"}
    if rec and rec.get("warp_instructions_per_launch") and (clocks or {}).get("sm_mhz"):
        # issue roof: executed warp instructions over the SMs' issue slots
        # (4 schedulers, one instruction per cycle each) at the sampled clock
        slots = nsm * 4 * clocks["sm_mhz"] * 1e6 * kms / 1e3
        roof["issue"] = {"warp_instructions_per_launch": rec["warp_instructions_per_launch"],
                         "issue_slots": slots, "frac": rec["warp_instructions_per_launch"] / slots}
    out = {"value": value, "unit": "Mpixels/s", "ms_per_step": total_f / steps, "steps": steps,
           "config": workload_config(workload, spec, W, H, work.px, len(work.sizes) if batched else None),
           "roofline": roof, "unfused": unfused,
           "e2e": {"value": e2e_value, "unit": "Mpixels/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
           "gpu_launches": steps * launches, "clocks": clocks,
           "run": {"schedule": fused.schedule_get(), "tuning": tuning, "l2": work.l2_note}}
    if rank == 0 and world == 1 and cpu_seconds > 0:
        out["cpu_baseline"] = cpu_baseline(work, name, spec, dts, cpu_seconds)
    fused.close()
    return out


def cpu_baseline(work, name, spec, dts, seconds):
    """The oracle's rate on all host cores, then on one core (a quarter of
    the time budget, at least 2 s)."""
    from oracle import oracle as O

    def rate(budget):
        if name == "blend":
            return cpu_blend_rate(dts, budget)
        img = work.cpu_sample(dts)
        cspec = spec if img.ndim == 2 else spec_for_depth(name, img.shape[0])
        r, cores, n, dt = cpu_oracle_rate(cspec, img, budget)
        return r, cores, n, dt, "%d images of %dx%d%s, %.1f s" % (n, img.shape[-1], img.shape[-2],
                                                                "" if img.ndim == 2 else "x%d" % img.shape[0], dt)

    r, cores, _, _, sample = rate(seconds)
    out = {"value": r, "unit": "Mpixels/s", "cores": cores, "kind": "oracle", "sample": sample}
    if cores > 1:
        O.set_num_threads(1)
        try:
            r1, _, _, _, sample1 = rate(max(2.0, seconds / 4))
        finally:
            O.set_num_threads(cores)
        out["one_core"] = {"value": r1, "unit": "Mpixels/s", "sample": sample1}
    return out


COSTMODEL_FILE = os.path.join(ROOT, "paper_1909_07190_gb300", "costmodel_gb300.txt")


def cost_model_entry(wt, torch, workload, rank, local, dist, steps):
    """The schedules the cost models pick for the workload (DP-Fusion with
    the analytic model, and with the learned model trained on this GPU kind
    when its parameters are present), each timed like the headline against
    the library's default schedule."""
    name, W, H, dts, spec, work = make_work(wt, torch, workload, rank, local)
    dtype = wt.DTYPES[dts]
    out = {"workload": workload, "model_file": None}
    pipes = {"default": wt.Pipeline(spec)}
    t0 = time.perf_counter()
    pipes["analytic"] = wt.Pipeline(spec)
    pipes["analytic"].schedule_auto(W, H, dtype, wt.WT_MODEL_ANALYTIC)
    if os.path.exists(COSTMODEL_FILE):
        wt.costmodel_load(COSTMODEL_FILE)
        pipes["learned"] = wt.Pipeline(spec)
        pipes["learned"].schedule_auto(W, H, dtype, wt.WT_MODEL_LEARNED)
        out["model_file"] = os.path.relpath(COSTMODEL_FILE, ROOT)
    out["search_seconds"] = round(time.perf_counter() - t0, 2)
    for k, pipe in pipes.items():
        total, _ = timed_steps(torch, work, lambda i, s, q=pipe: work.run(q, i, s), steps, 3, 100, dist)
        out[k] = {"ms": total / steps, "schedule": pipe.schedule_get(),
                  "kernels": [pipe.kernel_name(j, *work.io()) for j in range(pipe.launches_per_run())]
                  if hasattr(work, "io") else None}
    for k in ("analytic", "learned"):
        if k in out:
            out[k]["ratio_vs_default"] = out[k]["ms"] / out["default"]["ms"]
            # the same generated kernels as the default schedule (the headline's)
            out[k]["same_kernels_as_default"] = (out[k]["kernels"] is not None and
                                                 out[k]["kernels"] == out["default"]["kernels"])
    for pipe in pipes.values():
        pipe.close()
    return out


# every configuration of the benchmark beside the headline, with its steps
SECONDARY = (("sharpen", 4000), ("harris_f16", 2000), ("harris_batch", 20), ("blend", 200))


def run_ours(args, rank, world, local):
    import torch
    from paper_1909_07190_gb300 import wt

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    cpu_s = 0 if args.no_cpu_baseline else args.cpu_seconds
    head = measure(wt, torch, args.workload, args, dist, world, rank, local, args.steps, args.warmup, cpu_s,
                   args.size)
    line = {"metric": METRIC, "value": head["value"], "unit": "Mpixels/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": WORKLOADS[args.workload][3], "data": "synthetic",
            "config": head["config"], "roofline": head["roofline"], "unfused": head["unfused"], "e2e": head["e2e"],
            "gpu_launches": head["gpu_launches"], "clocks": head["clocks"], "run": head["run"]}
    if "cpu_baseline" in head:
        line["cpu_baseline"] = head["cpu_baseline"]
    if world == 1 and args.configs == "all" and not args.size and not args.params:
        # every other configuration, on the same GPU, after the headline
        cfgs = {}
        for wl, steps in SECONDARY:
            if wl == args.workload:
                continue
            m = measure(wt, torch, wl, args, None, 1, rank, local, steps, args.warmup,
                        min(cpu_s, 4.0) if cpu_s else 0)
            cfgs[wl] = m
            torch.cuda.empty_cache()
        line["configs"] = cfgs
        line["cost_model"] = cost_model_entry(wt, torch, args.workload, rank, local, None, 500)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


class _Null:
    def __enter__(self):
        return self

    def __exit__(self, *a):
        return False


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10000)
    ap.add_argument("--warmup", type=int, default=100)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="harris", choices=sorted(WORKLOADS))
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--size", type=int, default=0,
                    help="image side of a smaller square case of a single-image workload (profiling; "
                         "the default is the workload's own size)")
    ap.add_argument("--params", default="",
                    help="JSON group parameters of a one-group fused schedule (e.g. '{\"tile_h\": 20}')")
    ap.add_argument("--batch-images", type=int, default=0,
                    help="the first N images of the 512-image batch (profiling captures of a reduced batch)")
    ap.add_argument("--configs", default="all", choices=["all", "none"],
                    help="after the headline workload, measure every other configuration (sharpen, FP16 corner "
                         "response, the 512-image batch, the blend) and the cost models' picks, one GPU only")
    ap.add_argument("--tune", default="auto", choices=["auto", "on", "off"],
                    help="measured schedule search before timing (auto: batches only; single images use the "
                         "library's default schedule)")
    args = ap.parse_args()
    args_global.batch_images = args.batch_images
    if args.warmup < 3:
        args.warmup = 3
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank)
    else:
        run_ours(args, rank, world, local)


if __name__ == "__main__":
    main()

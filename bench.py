"""Benchmark: Mpixels/s of the fused warp-tiled pipeline on one GB300 per rank.

Workload (default): the 11-stage corner-response pipeline on a 4096x4096
single-channel FP32 image (uniform [0,1) from seed 190907192).  One step =
one wt_run of the whole pipeline over one image.  Inputs are resident in HBM;
consecutive steps rotate over buffer sets whose total size exceeds 3x L2, so
every step reads and writes HBM.  Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload harris|harris_f16|sharpen]
  python bench.py --impl reference ...   # the FP64 CPU oracle on host cores

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
}
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
    px = n * img.shape[-1] * img.shape[-2]
    return px / dt / 1e6, O.num_threads(), n, dt


def run_reference(args, rank):
    if rank != 0:
        return
    name, W, H, dt, seed = WORKLOADS[args.workload]
    spec = P.by_name(name)
    img = I.round_to(I.uniform_image(seed, W, H)[0], dt)
    for _ in range(args.warmup):
        cpu_oracle_rate(spec, img, 0.0)
    rates = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        r, cores, n, _ = cpu_oracle_rate(spec, img, 0.0)
        rates.append(r)
    total = time.perf_counter() - t0
    value = W * H * args.steps / total / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "Mpixels/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": total / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "pipeline": name, "width": W, "height": H,
                       "channels": 1, "storage": dt},
            "cpu_baseline": {"value": value, "unit": "Mpixels/s", "cores": cores, "kind": "oracle",
                             "sample": "one full %dx%d image per step" % (W, H)},
            "e2e": {"value": value, "unit": "Mpixels/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args, rank, world, local):
    import torch
    from paper_1909_07190_gb300 import wt

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    name, W, H, dts, seed = WORKLOADS[args.workload]
    dtype = wt.DTYPES[dts]
    spec = P.by_name(name)
    img = I.uniform_image(seed + rank, W, H)[0]
    esz = 4 if dtype == wt.WT_F32 else 2
    set_bytes = 2 * W * H * esz
    l2 = torch.cuda.get_device_properties(local).L2_cache_size
    nsets = max(3, -(-3 * l2 // set_bytes))
    ins = [wt.DeviceImage(1, H, W, dtype).upload(img) for _ in range(nsets)]
    outs = [wt.DeviceImage(1, H, W, dtype) for _ in range(nsets)]
    stream = torch.cuda.current_stream()
    sp = stream.cuda_stream

    fused = wt.Pipeline(spec)
    fused.schedule_auto(W, H, dtype, wt.WT_MODEL_ANALYTIC)
    plain = wt.Pipeline(spec)
    plain.schedule(exec_mode=wt.WT_EXEC_PLAIN)

    def capture(pipe, n, start):
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            cs = torch.cuda.current_stream().cuda_stream
            for i in range(start, start + n):
                pipe.run([ins[i % nsets].image()], [outs[i % nsets].image()], cs)
        return g

    def timed(pipe, steps, warmup, sampler=None, per_graph=100):
        """Kernel-only time of exactly `steps` runs: CUDA graphs of up to
        `per_graph` back-to-back runs over rotating buffer sets, replayed,
        CUDA events around the replays (no host work inside the region)."""
        for i in range(max(warmup, nsets)):
            pipe.run([ins[i % nsets].image()], [outs[i % nsets].image()], sp)
        torch.cuda.synchronize()
        n = min(per_graph, steps)
        full, rem = divmod(steps, n)
        g = capture(pipe, n, 0)
        gr = capture(pipe, rem, 0) if rem else None
        for _ in range(max(1, warmup // n)):
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
        total = ev[0].elapsed_time(ev[full + 1])
        if dist is not None:
            t = torch.tensor([total], device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            total = float(t.item())
            dist.barrier()
        return total, per

    sampler = ClockSampler(local)
    total_f, per_f = timed(fused, args.steps, args.warmup, sampler)
    clocks = sampler.summary()
    plain_steps = max(3, args.steps // 8)
    total_p, per_p = timed(plain, plain_steps, args.warmup)
    fused.check(sp)
    plain.check(sp)

    # end to end through the C ABI with host buffers (pinned), copies inside
    hin = wt.DeviceImage(1, H, W, dtype, device="cpu", pin_host=True)
    hin.view().copy_(ins[0].view().cpu())
    hout = wt.DeviceImage(1, H, W, dtype, device="cpu", pin_host=True)
    for _ in range(args.warmup):
        fused.run_host([hin.image()], [hout.image()], sp)
    torch.cuda.synchronize()
    e2e_steps = max(3, min(200, args.steps // 4))
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        fused.run_host([hin.image()], [hout.image()], sp)
    e2e_s = time.perf_counter() - t0

    px = W * H
    value = px * world * args.steps / (total_f / 1e3) / 1e6
    launch_ms = statistics.mean(per_f)
    alg_bytes = 2 * px * esz
    peak, peak_kind = peaks()
    achieved = alg_bytes / (launch_ms / 1e3) / 1e9
    # DRAM bytes per launch from the committed ncu summary, used only when it
    # was taken on the kernel that ran here (same generated kernel name)
    kname = fused.debug_kernel(0, [ins[0].image()], [outs[0].image()])["name"]
    traffic = None
    tpath = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tpath):
        try:
            rec = json.load(open(tpath)).get(args.workload)
            if rec and rec.get("kernel") == kname:
                traffic = rec["dram_bytes_per_launch"]
        except Exception:
            traffic = None
    line = {
        "metric": METRIC, "value": value, "unit": "Mpixels/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_f / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": dts, "data": "synthetic",
        "config": {"workload": args.workload, "pipeline": name, "width": W, "height": H, "channels": 1,
                   "storage": dts, "stages": len(spec["stages"]),
                   "l2": "rotating %d input/output sets (%.0f MB) > 3x L2" % (nsets, nsets * set_bytes / 1e6),
                   "schedule": fused.schedule_get()},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic, "peak_kind": peak_kind, "kernel": kname,
                     "algorithmic_bytes_per_launch": alg_bytes},
        "unfused": {"value": px * world * plain_steps / (total_p / 1e3) / 1e6, "unit": "Mpixels/s",
                    "ms_per_step": total_p / plain_steps, "launches_per_step": plain.launches_per_run()},
        "e2e": {"value": px * e2e_steps / e2e_s / 1e6, "unit": "Mpixels/s", "h2d_bytes_per_step": px * esz,
                "d2h_bytes_per_step": px * esz},
        "gpu_launches": args.steps * fused.launches_per_run(),
        "clocks": clocks,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        r, cores, n, dt = cpu_oracle_rate(spec, I.round_to(img, dts), args.cpu_seconds)
        line["cpu_baseline"] = {"value": r, "unit": "Mpixels/s", "cores": cores, "kind": "oracle",
                                "sample": "%d full %dx%d images, %.1f s" % (n, W, H, dt)}
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
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank)
    else:
        run_ours(args, rank, world, local)


if __name__ == "__main__":
    main()

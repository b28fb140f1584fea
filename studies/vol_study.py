"""3-D groups on one GPU (App. A, generalised hybrid tiling): the fused
warp-tile kernel over volumes against the unfused per-stage path, with the
split (streamed) axis along rows or along planes.

  python studies/vol_study.py [--pipelines unsharp3d,heat3d] [--reps 20] [--out f.json]

Workloads: 512 x 512 x 256 FP32 volumes (67.1 M voxels, 268 MB), uniform
[0, 1) from a seed: the 3-D unsharp mask (5-tap binomial blur along x, y
and z, then a clamped sharpen reading the input again) and two fused steps
of 3-D heat diffusion (7-point stencils).

Arms:
  plain  per-stage kernels, FP32 intermediates in HBM (the unfused path)
  fused  one 3-D group, swept in two rounds: split axis {rows, planes} x
         tile_o {1, 2, 4, 8} x vec {1, 2} x register cap {none, 96} x
         sources in registers (frac_reg 1) or staged in shared memory
         (frac_reg 0) at tile_h 32 and 4 warps, then tile_h {16, 64, 128} x warps {2, 4, 8}
         x register cap {none, 80, 96, 128} around the best, then source
         look-ahead (n_buffers) {1, 3, 4} rows against the default 2
Time per run: CUDA events on the launching stream, mean over `reps` runs
after 3 warm-up runs (inputs and outputs of 268 MB each exceed the L2).
HBM fraction: (input + output bytes) / time / the measured copy bandwidth.
Every configuration's output is compared with the first fused one's; the
largest difference is reported.
"""
from __future__ import annotations

import argparse
import itertools
import json
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

from paper_1909_07190_gb300 import inputs as I  # noqa: E402
from paper_1909_07190_gb300 import pipelines as P  # noqa: E402
from paper_1909_07190_gb300 import wt  # noqa: E402
from otptb_study import time_run  # noqa: E402

W, H, D = 512, 512, 256


def hbm_peak():
    path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def spec_of(name):
    return P.unsharp3d(depth=D) if name == "unsharp3d" else P.heat3d(2, depth=D)


def study(name, reps, stream, flush, log):
    import torch
    spec = spec_of(name)
    n = len(spec["stages"])
    x = wt.DeviceImage(D, H, W).upload(I.uniform_image(I.SEED_BASE + 8, W, H, D))
    y = wt.DeviceImage(D, H, W)
    ref = wt.DeviceImage(D, H, W)
    ins, outs = [x.image()], [y.image()]
    groups = [0] * n
    plain = wt.Pipeline(spec)
    plain.schedule(exec_mode=wt.WT_EXEC_PLAIN)
    plain_ms = time_run(plain, ins, outs, stream, flush, reps)
    pipe = wt.Pipeline(spec)

    def fused(prm):
        try:
            pipe.prepare([(groups, [prm])], ins, outs)
        except wt.WtError as e:
            log("%s: skip %s (%s)" % (name, prm, e))
            return None
        pipe.schedule(groups=groups, params=[prm])
        if pipe.launches_per_run() != 1:
            log("%s: %s runs per stage" % (name, prm))
            return None
        ms = time_run(pipe, ins, outs, stream, flush, reps)
        return ms

    rows, worst, first = [], 0.0, True
    grid1 = [dict(tile_h=32, tile_o=o, vec=v, warps_per_block=4, max_regs=r, frac_reg=f,
                  flags=wt.WT_FLAG_ZSTREAM if s else 0)
             for s, o, v, r, f in itertools.product((0, 1), (1, 2, 4, 8), (1, 2), (0, 96), (1.0, 0.0))]

    def run_grid(grid):
        nonlocal worst, first
        for prm in grid:
            ms = fused(prm)
            if ms is None:
                continue
            if first:
                ref.view().copy_(y.view())
                first = False
            else:
                worst = max(worst, float((y.view() - ref.view()).abs().max()))
            rows.append((ms, prm))
            log("%s %s %.1f us" % (name, prm, ms * 1e3))

    run_grid(grid1)
    best = min(rows, key=lambda r: r[0])[1]
    grid2 = [dict(best, tile_h=t, warps_per_block=w, max_regs=r)
             for t, w, r in itertools.product((16, 64, 128), (2, 4, 8), (0, 80, 96, 128))]
    run_grid(grid2)
    best = min(rows, key=lambda r: r[0])[1]
    grid2 = [dict(best, n_buffers=b) for b in (1, 3, 4)]
    run_grid(grid2)
    torch.cuda.synchronize()
    ms, prm = min(rows, key=lambda r: r[0])
    by_split = {}
    for t, p in rows:
        k = "planes" if p["flags"] & wt.WT_FLAG_ZSTREAM else "rows"
        if k not in by_split or t < by_split[k][0]:
            by_split[k] = (t, p)
    by_place = {}
    for t, p in rows:
        k = "registers" if p["frac_reg"] >= 1.0 else "shared"
        if k not in by_place or t < by_place[k][0]:
            by_place[k] = (t, p)
    peak, kind = hbm_peak()
    vox = W * H * D
    io = 2 * vox * 4
    out = {"pipeline": name, "volume": [D, H, W], "dtype": "f32", "plain_us": plain_ms * 1e3,
           "plain_launches": plain.launches_per_run(), "fused_us": ms * 1e3, "fused_params": prm,
           "fused_mvox_s": vox / (ms * 1e-3) / 1e6, "plain_mvox_s": vox / (plain_ms * 1e-3) / 1e6,
           "speedup": plain_ms / ms, "hbm_gbs": io / (ms * 1e-3) / 1e9, "hbm_peak_gbs": peak, "peak_kind": kind,
           "hbm_frac": io / (ms * 1e-3) / 1e9 / peak,
           "best_by_split": {k: {"us": v[0] * 1e3, "params": v[1]} for k, v in by_split.items()},
           "best_by_source_placement": {k: {"us": v[0] * 1e3, "params": v[1]} for k, v in by_place.items()},
           "configs": len(rows), "max_diff": worst}
    return out


def main(argv=None):
    import torch
    ap = argparse.ArgumentParser()
    ap.add_argument("--pipelines", default="unsharp3d,heat3d")
    ap.add_argument("--reps", type=int, default=20)
    ap.add_argument("--out", default="")
    args = ap.parse_args(argv)
    stream = torch.cuda.current_stream().cuda_stream
    flush = torch.empty(64 << 20, dtype=torch.float32, device="cuda")
    res = []
    for name in args.pipelines.split(","):
        r = study(name, args.reps, stream, flush, lambda s: print(s, file=sys.stderr, flush=True))
        print(json.dumps(r), flush=True)
        res.append(r)
    if args.out:
        with open(args.out, "w") as f:
            json.dump(res, f, indent=1)


if __name__ == "__main__":
    main()

"""Warp tiles against block tiles on one GPU: the paper's central comparison
(Sec. 3 motivating example; Sec. 7 ablation of OTPW+Shared, OTPW+HT and
OTPW+RT against OTPTB), with both tilings generated by this library from
the same group analysis.

  python studies/otptb_study.py [--pipelines harris,sharpen,blur_rgb] [--reps 20]

Arms, each one fused group over the whole pipeline unless noted:
  plain  per-stage kernels, intermediates in HBM (the unfused baseline)
  otptb  one overlapped tile per thread block (WT_FLAG_OTPTB), swept over
         tile width 32 vec (vec 1, 2, 4, 8), tile height {4, 8, 16, 32, 64, 128}
         and {4, 8, 16} warps per block
  otpw   warp tiles, swept over tile height {8, 14, 20, 32}, fracReg
         {0 (Shared), 0.5 (HT), 1 (RT)} and {2, 4} warps per block
Time per run: CUDA events around each run on the launching stream, a
256 MB buffer written between runs (L2 flushed), mean over `reps` runs
after 3 warm-up runs.  Every configuration's output is compared with the
default schedule's; the largest difference is reported.  Inputs: synthetic
uniform [0,1) FP32 images (the workloads' sizes: the 11-stage corner
response on 4096x4096, the 3-stage sharpen on 2048x2048, the 2-stage blur
on 4096x4096x3 as in the paper's motivating example).
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

SIZES = {"harris": (4096, 4096), "sharpen": (2048, 2048), "blur_rgb": (4096, 4096), "blur": (4096, 4096)}
OTPTB_GRID = [dict(vec=v, tile_h=t, warps_per_block=w, flags=wt.WT_FLAG_OTPTB)
              for v, t, w in itertools.product((1, 2, 4, 8), (4, 8, 16, 32, 64, 128), (4, 8, 16))]
OTPW_GRID = [dict(tile_h=t, frac_reg=f, warps_per_block=w)
             for t, f, w in itertools.product((8, 14, 20, 32), (0.0, 0.5, 1.0), (2, 4))]


def time_run(pipe, ins, outs, stream, flush, reps):
    import torch
    s = torch.cuda.current_stream()
    for _ in range(3):
        pipe.run(ins, outs, stream)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    torch.cuda.synchronize()
    for a, b in ev:
        flush.zero_()
        a.record(s)
        pipe.run(ins, outs, stream)
        b.record(s)
    torch.cuda.synchronize()
    pipe.check(stream)
    return sum(a.elapsed_time(b) for a, b in ev) / reps


def study(name, reps, stream, flush, log):
    spec = P.by_name(name)
    W, H = SIZES[name]
    C = spec["inputs"][0]
    n = len(spec["stages"])
    x = wt.DeviceImage(C, H, W).upload(I.uniform_image(I.SEED_BASE + 7, W, H, C))
    y = wt.DeviceImage(C, H, W)
    ref = wt.DeviceImage(C, H, W)
    ins, outs = [x.image()], [y.image()]
    pipe = wt.Pipeline(spec)
    pipe.run(ins, [ref.image()], stream)
    pipe.check(stream)
    groups = [0] * n
    cands = OTPTB_GRID + OTPW_GRID
    ok = []
    for prm in cands:
        try:
            pipe.prepare([(groups, [prm])], ins, outs)
            ok.append(prm)
        except wt.WtError as e:
            log("%s: skip %s (%s)" % (name, prm, e))
    rows = []
    worst = 0.0
    for prm in ok:
        pipe.schedule(groups=groups, params=[prm])
        try:
            ms = time_run(pipe, ins, outs, stream, flush, reps)
        except wt.WtError as e:
            log("%s: %s failed at run: %s" % (name, prm, e))
            continue
        err = float((y.view() - ref.view()).abs().max())
        worst = max(worst, err)
        rows.append(dict(prm, arm="otptb" if prm.get("flags") else "otpw", ms=ms, mpx_s=W * H * C / ms / 1e3))
    pipe.schedule(exec_mode=wt.WT_EXEC_PLAIN)
    plain_ms = time_run(pipe, ins, outs, stream, flush, reps)

    def best(pred):
        r = [q for q in rows if pred(q)]
        return min(r, key=lambda q: q["ms"]) if r else None

    b_tb = best(lambda q: q["arm"] == "otptb")
    b_sh = best(lambda q: q["arm"] == "otpw" and q["frac_reg"] == 0.0)
    b_ht = best(lambda q: q["arm"] == "otpw" and 0.0 < q["frac_reg"] < 1.0)
    b_rt = best(lambda q: q["arm"] == "otpw" and q["frac_reg"] == 1.0)
    b_w = best(lambda q: q["arm"] == "otpw")
    res = {"pipeline": name, "W": W, "H": H, "C": C, "stages": n, "plain_ms": plain_ms,
           "best_otptb": b_tb, "best_otpw_shared": b_sh, "best_otpw_ht": b_ht, "best_otpw_rt": b_rt,
           "speedup_over_otptb": {k: b_tb["ms"] / v["ms"] for k, v in
                                  (("otpw_shared", b_sh), ("otpw_ht", b_ht), ("otpw_rt", b_rt), ("otpw", b_w))
                                  if v and b_tb},
           "otptb_over_plain": plain_ms / b_tb["ms"] if b_tb else None,
           "max_abs_diff_vs_default": worst, "configs_timed": len(rows)}
    return res, rows


def main():
    import torch
    ap = argparse.ArgumentParser()
    ap.add_argument("--pipelines", default="harris,sharpen,blur_rgb")
    ap.add_argument("--reps", type=int, default=20)
    ap.add_argument("--out", default="")
    args = ap.parse_args()
    stream = torch.cuda.current_stream().cuda_stream
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def log(m):
        print(m, file=sys.stderr, flush=True)

    results, all_rows = [], []
    for name in args.pipelines.split(","):
        r, rows = study(name, args.reps, stream, flush, log)
        results.append(r)
        all_rows += [dict(q, pipeline=name) for q in rows]
        log(json.dumps(r))
    print(json.dumps({"results": results, "protocol": "mean of %d runs, L2 flushed between runs" % args.reps}))
    if args.out:
        with open(args.out, "w") as f:
            json.dump({"results": results, "rows": all_rows}, f, indent=1)


if __name__ == "__main__":
    main()

"""Learned cost model study: measure the launch times of many schedules,
train the MLP on some of them, and score its schedule picks on schedules
whose launches it has never seen, against exhaustive timing and against the
analytic model.

  python studies/costmodel_study.py [--out summary.json] [--rows rows.json]
                                    [--model model.txt]

Pipelines: the 3-stage sharpen on 2048x2048 and the 11-stage corner response
on 4096x4096, FP32 (synthetic uniform [0,1) images).  Schedules: contiguous
groupings (all 4 of sharpen's, a seeded sample of the corner response's
1024) x warp tile heights x register/shared splits fracReg {1, 0.5, 0} x
warps per block ({1, 2, 4} for sharpen, {1, 2} for the corner response) x
pixels per lane {4, 8}: the space DP-Fusion's learned search draws from.  Each
schedule runs once against the default schedule's output (the largest
difference is reported) and is timed launch by launch, each launch with its
features (wt_costmodel_collect).

A launch is identified by its feature vector (stage segment, effective tile
height, pixels per lane, warps, fracReg, ...), so two schedules that share a
kernel and tile share the launch.  Two held-out splits, in both of which no
held-out launch appears in training:
  tile    every schedule of held-out tile heights (corner response 24 and 56
          rows, sharpen 6 rows) is held out;
  launch  a seeded 20% of the distinct fused launches is held out, with every
          schedule that contains one of them.
The model trains on the launches of the remaining schedules, minus any launch
that also occurs in a held-out schedule (per-stage kernels), and picks the
held-out schedule with the lowest predicted time; t(pick) / t(best held-out)
is reported for it and for the analytic model (Alg. 2 with Table 3's
weights), with the Spearman rank correlation of predicted and measured
times.  Finally the model is trained on every launch and saved (--model).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys
import time

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

from paper_1909_07190_gb300 import inputs as I  # noqa: E402
from paper_1909_07190_gb300 import pipelines as P  # noqa: E402
from paper_1909_07190_gb300 import wt  # noqa: E402

FRACS = (1.0, 0.5, 0.0)
SPACE = {
    # pipeline: (width, height, tile heights, warps per block, pixels per lane, groupings)
    "sharpen": (2048, 2048, (4, 6, 8, 10), (1, 2, 4), (4, 8), 4),
    "harris": (4096, 4096, (8, 16, 24, 32, 40, 56), (1, 2), (4, 8), 40),
}
HELD_TILES = {"sharpen": {6}, "harris": {24, 56}}


def groupings(n, rng, limit):
    """Contiguous groupings of n stages (group index per stage): all of them
    when there are at most `limit`, else the two extremes and a seeded
    sample."""
    total = 1 << (n - 1)

    def decode(mask):
        g, cur = [0], 0
        for i in range(1, n):
            if mask >> (i - 1) & 1:
                cur += 1
            g.append(cur)
        return g

    if total <= limit:
        return [decode(m) for m in range(total)]
    masks = {0, total - 1}
    while len(masks) < limit:
        masks.add(int(rng.integers(0, total)))
    return [decode(m) for m in sorted(masks)]


def collect(name, rng, stream, log):
    """Times every schedule of the pipeline's space, launch by launch."""
    import torch
    W, H, tiles, warps, vecs, n_group = SPACE[name]
    spec = P.by_name(name)
    n = len(spec["stages"])
    img = I.uniform_image(I.SEED_BASE + (1 if name == "sharpen" else 2), W, H)[0]
    x = wt.DeviceImage(1, H, W).upload(img)
    y = wt.DeviceImage(1, H, W)
    ref = wt.DeviceImage(1, H, W)
    pipe = wt.Pipeline(spec)
    # reference output: the default schedule, whose parity with the FP64
    # oracle the GPU test suite establishes
    pipe.run([x.image()], [ref.image()], stream)
    pipe.check(stream)
    scheds = [(g, dict(tile_h=T, frac_reg=fr, warps_per_block=nw, vec=v))
              for g in groupings(n, rng, n_group) for T in tiles for fr in FRACS for nw in warps for v in vecs]
    t0 = time.time()
    pipe.prepare([(g, [prm] * (max(g) + 1)) for g, prm in scheds], [x.image()], [y.image()])
    log("%s: %d schedules, kernels compiled in %.0f s" % (name, len(scheds), time.time() - t0))
    rows, worst = [], 0.0
    for k, (g, prm) in enumerate(scheds):
        ng = max(g) + 1
        pipe.schedule(groups=g, params=[prm] * ng)
        y.t.zero_()
        # every launch timed and described by the library (wt_costmodel_collect)
        f, log_ms, _ = wt.costmodel_collect(pipe, [x.image()], [y.image()], 10, stream)
        pipe.check(stream)
        err = float((y.view() - ref.view()).abs().max())
        worst = max(worst, err)
        feats = f.tolist()
        ms = [float(v) for v in np.exp(log_ms.astype(np.float64))]
        analytic = 0.0
        for gi in range(ng):
            stages = [s for s in range(n) if g[s] == gi]
            c = pipe.cost_group(stages[0], len(stages), prm, 128, W, H)
            analytic += c["cost"] if c["feasible"] else 1e9
        rows.append({"pipeline": name, "groups": g, "params": prm, "launch_ms": ms, "features": feats,
                     "ms": float(sum(ms)), "analytic": analytic, "max_err_vs_ref": err})
        if (k + 1) % 200 == 0:
            log("%s: %d/%d timed" % (name, k + 1, len(scheds)))
    torch.cuda.synchronize()
    return rows, {"schedules": len(rows), "max_err_vs_default": worst}


def launch_key(row, f):
    return (row["pipeline"],) + tuple(round(v, 5) for v in f)


def train(rows, idx, exclude, epochs, seed):
    """Trains the model on the launches of schedules `idx`, one sample per
    distinct launch (median of its times), skipping launches in `exclude`."""
    samples = {}
    for i in idx:
        r = rows[i]
        for f, t in zip(r["features"], r["launch_ms"]):
            k = launch_key(r, f)
            if k in exclude:
                continue
            samples.setdefault(k, (f, []))[1].append(t)
    X = np.array([v[0] for v in samples.values()], np.float32)
    Y = np.array([math.log(float(np.median(v[1]))) for v in samples.values()], np.float32)
    t0 = time.time()
    loss = wt.costmodel_train(X, Y, epochs=epochs, batch=64, lr=2e-3, seed=seed)
    return {"train_launches": int(len(Y)), "final_loss": float(loss), "seconds": time.time() - t0}


def predict_ms(row):
    lp = wt.costmodel_predict(np.array(row["features"], np.float32))
    return float(np.exp(lp.astype(np.float64)).sum())


def spearman(a, b):
    ra = np.argsort(np.argsort(np.asarray(a)))
    rb = np.argsort(np.argsort(np.asarray(b)))
    return float(np.corrcoef(ra, rb)[0, 1]) if len(a) > 2 else float("nan")


def evaluate(rows, test_idx):
    """t(pick) / t(best) over the held-out schedules of each pipeline."""
    out = {}
    for name in sorted({rows[i]["pipeline"] for i in test_idx}):
        idx = [i for i in test_idx if rows[i]["pipeline"] == name]
        best = min(rows[i]["ms"] for i in idx)
        pred = [predict_ms(rows[i]) for i in idx]
        pick_l = idx[int(np.argmin(pred))]
        pick_a = min(idx, key=lambda i: rows[i]["analytic"])
        true = [rows[i]["ms"] for i in idx]
        out[name] = {"held_out_schedules": len(idx), "best_ms": best,
                     "learned_pick_ms": rows[pick_l]["ms"], "learned_ratio": rows[pick_l]["ms"] / best,
                     "learned_pick": {"groups": rows[pick_l]["groups"], "params": rows[pick_l]["params"]},
                     "analytic_pick_ms": rows[pick_a]["ms"], "analytic_ratio": rows[pick_a]["ms"] / best,
                     "learned_spearman": spearman(pred, true),
                     "analytic_spearman": spearman([rows[i]["analytic"] for i in idx], true)}
    return out


def split_tile(rows):
    test = [i for i, r in enumerate(rows) if r["params"]["tile_h"] in HELD_TILES[r["pipeline"]]]
    return test


def split_launch(rows, rng):
    fused = sorted({launch_key(r, f) for r in rows for f in r["features"] if f[17] > 0.5})
    held = {fused[i] for i in rng.permutation(len(fused))[:max(1, len(fused) // 5)]}
    return [i for i, r in enumerate(rows) if any(launch_key(r, f) in held for f in r["features"])]


def run_split(rows, test, epochs, seed):
    test_set = set(test)
    train_idx = [i for i in range(len(rows)) if i not in test_set]
    exclude = {launch_key(rows[i], f) for i in test for f in rows[i]["features"]}
    info = train(rows, train_idx, exclude, epochs, seed)
    info.update({"train_schedules": len(train_idx), "test_schedules": len(test),
                 "held_out": evaluate(rows, test)})
    return info


def main():
    import torch
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default="")
    ap.add_argument("--rows", default="")
    ap.add_argument("--model", default="")
    ap.add_argument("--epochs", type=int, default=300)
    ap.add_argument("--seed", type=int, default=I.SEED_BASE + 4)
    args = ap.parse_args()
    rng = np.random.default_rng(args.seed)
    stream = torch.cuda.current_stream().cuda_stream

    def log(m):
        print(m, file=sys.stderr, flush=True)

    rows, checks = [], {}
    for name in ("sharpen", "harris"):
        r, c = collect(name, rng, stream, log)
        rows += r
        checks[name] = c
    res = {"schedules": len(rows), "parity": checks,
           "protocol": "launch kernel time: min over 3 samples of the mean of 10 launches",
           "splits": {"tile": run_split(rows, split_tile(rows), args.epochs, args.seed),
                      "launch": run_split(rows, split_launch(rows, rng), args.epochs, args.seed)}}
    # the model kept for scheduling: every launch
    res["final"] = train(rows, range(len(rows)), set(), args.epochs, args.seed)
    if args.model:
        wt.costmodel_save(args.model)
    print(json.dumps(res, indent=1))
    if args.out:
        with open(args.out, "w") as f:
            json.dump(res, f, indent=1)
    if args.rows:
        with open(args.rows, "w") as f:
            json.dump(rows, f)


if __name__ == "__main__":
    main()

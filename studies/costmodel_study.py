"""Learned cost model study: collect measured launch times of many schedules,
train the MLP, and score its schedule picks on held-out schedules against
exhaustive timing and the analytic model.

  python studies/costmodel_study.py [--schedules 2000] [--out study.json]
                                                   [--model model.txt]

Pipelines: the 3-stage sharpen on 2048x2048 and the 11-stage corner response
on 4096x4096, FP32 (synthetic uniform [0,1) images).  Schedules: contiguous
groupings (all of sharpen's, a seeded sample of the corner response's 1024)
x warp tile heights {4, 8, 16, 32} x register/shared splits fracReg
{1, 0.5, 0}.  Each schedule is timed launch by launch
(wt_schedule_time_launches) and its output is compared with the default
schedule's (the largest difference is reported).
Schedules are split 80/20 (seeded); the model trains on the launches of the
80%, and on the held-out 20% of each pipeline the schedule with the lowest
predicted time is compared with the fastest measured one
(t(pick) / t(best)); the analytic model's pick is scored the same way.
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

TILES = (4, 8, 16, 32)
FRACS = (1.0, 0.5, 0.0)


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


def collect(name, W, H, n_sched, rng, stream, log):
    import torch
    spec = P.by_name(name)
    n = len(spec["stages"])
    img = I.uniform_image(I.SEED_BASE + (1 if name == "sharpen" else 2), W, H)[0]
    x = wt.DeviceImage(1, H, W).upload(img)
    y = wt.DeviceImage(1, H, W)
    ref = wt.DeviceImage(1, H, W)
    pipe = wt.Pipeline(spec)
    # reference output: the default schedule (one fused group), whose parity
    # with the FP64 oracle the GPU test suite establishes
    pipe.run([x.image()], [ref.image()], stream)
    pipe.check(stream)
    per = len(TILES) * len(FRACS)
    gs = groupings(n, rng, max(1, n_sched // per))
    scheds = [(g, T, fr) for g in gs for T in TILES for fr in FRACS]
    # compile every kernel first (parallel host threads)
    t0 = time.time()
    pipe.prepare([(g, [dict(tile_h=T, frac_reg=fr)] * (max(g) + 1)) for g, T, fr in scheds],
                 [x.image()], [y.image()])
    log("%s: %d schedules, kernels compiled in %.0f s" % (name, len(scheds), time.time() - t0))
    rows = []
    worst = 0.0
    for k, (g, T, fr) in enumerate(scheds):
        ng = max(g) + 1
        prm = dict(tile_h=T, frac_reg=fr)
        pipe.schedule(groups=g, params=[prm] * ng)
        y.t.zero_()
        launches = pipe.time_launches([x.image()], [y.image()], 10, stream)
        pipe.check(stream)
        err = float((y.view() - ref.view()).abs().max())
        worst = max(worst, err)
        feats, ms = [], []
        for first, cnt, fused, t in launches:
            feats.append(wt.costmodel_features(pipe, first, cnt, prm if fused else None, fused, W, H).tolist())
            ms.append(t)
        analytic = 0.0
        for gi in range(ng):
            stages = [s for s in range(n) if g[s] == gi]
            c = pipe.cost_group(stages[0], len(stages), dict(prm, vec=4), 128, W, H)
            analytic += c["cost"] if c["feasible"] else 1e9
        rows.append({"pipeline": name, "groups": g, "tile_h": T, "frac_reg": fr, "launch_ms": ms,
                     "features": feats, "ms": float(sum(ms)), "analytic": analytic, "max_err_vs_ref": err})
        if (k + 1) % 100 == 0:
            log("%s: %d/%d timed" % (name, k + 1, len(scheds)))
    torch.cuda.synchronize()
    return rows, {"schedules_vs_reference_max_err": worst}


def evaluate(rows, test_idx, predict):
    """t(pick)/t(best) over the held-out schedules of each pipeline."""
    out = {}
    for name in sorted({r["pipeline"] for r in rows}):
        idx = [i for i in test_idx if rows[i]["pipeline"] == name]
        best = min(rows[i]["ms"] for i in idx)
        pick_l = min(idx, key=lambda i: predict(rows[i]))
        pick_a = min(idx, key=lambda i: rows[i]["analytic"])
        true = np.array([rows[i]["ms"] for i in idx])
        pred = np.array([predict(rows[i]) for i in idx])
        ra = np.argsort(np.argsort(true))
        rp = np.argsort(np.argsort(pred))
        out[name] = {"held_out": len(idx), "best_ms": best,
                     "learned_pick_ms": rows[pick_l]["ms"], "learned_ratio": rows[pick_l]["ms"] / best,
                     "analytic_pick_ms": rows[pick_a]["ms"], "analytic_ratio": rows[pick_a]["ms"] / best,
                     "learned_spearman": float(np.corrcoef(ra, rp)[0, 1])}
    return out


def main():
    import torch
    ap = argparse.ArgumentParser()
    ap.add_argument("--schedules", type=int, default=2000)
    ap.add_argument("--out", default="")
    ap.add_argument("--model", default="")
    ap.add_argument("--epochs", type=int, default=300)
    ap.add_argument("--seed", type=int, default=I.SEED_BASE + 4)
    args = ap.parse_args()
    rng = np.random.default_rng(args.seed)
    stream = torch.cuda.current_stream().cuda_stream

    def log(m):
        print(m, file=sys.stderr, flush=True)

    rows, checks = [], {}
    n_sharpen = len(TILES) * len(FRACS) * 4
    for name, W, H, ns in (("sharpen", 2048, 2048, n_sharpen), ("harris", 4096, 4096, args.schedules - n_sharpen)):
        r, c = collect(name, W, H, ns, rng, stream, log)
        rows += r
        checks[name] = c
    perm = rng.permutation(len(rows))
    n_train = int(round(0.8 * len(rows)))
    train_idx, test_idx = sorted(perm[:n_train].tolist()), sorted(perm[n_train:].tolist())
    # launch-level training samples (a launch seen in several schedules is
    # averaged)
    samples = {}
    for i in train_idx:
        for f, t in zip(rows[i]["features"], rows[i]["launch_ms"]):
            key = (rows[i]["pipeline"],) + tuple(round(v, 5) for v in f)
            samples.setdefault(key, (f, []))[1].append(t)
    X = np.array([v[0] for v in samples.values()], np.float32)
    Y = np.array([math.log(float(np.median(v[1]))) for v in samples.values()], np.float32)
    t0 = time.time()
    loss = wt.costmodel_train(X, Y, epochs=args.epochs, batch=64, lr=2e-3, seed=args.seed)
    train_s = time.time() - t0
    if args.model:
        wt.costmodel_save(args.model)
    cache = {}

    def predict(r):
        key = id(r)
        if key not in cache:
            lp = wt.costmodel_predict(np.array(r["features"], np.float32))
            cache[key] = float(np.exp(lp.astype(np.float64)).sum())
        return cache[key]

    res = {"schedules": len(rows), "train_schedules": len(train_idx), "test_schedules": len(test_idx),
           "train_launch_samples": int(len(Y)), "final_train_loss": loss, "train_seconds": train_s,
           "parity": checks, "held_out": evaluate(rows, test_idx, predict),
           "protocol": "launch kernel time: min over 3 samples of the mean of 10 launches"}
    print(json.dumps(res, indent=1))
    if args.out:
        with open(args.out, "w") as f:
            json.dump({"result": res, "rows": rows}, f)


if __name__ == "__main__":
    main()

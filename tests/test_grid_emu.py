"""Per-plane programs (the channel-index op) and the bilateral grid
(histogram as a splat-and-sum reduction, then 2x2 sums and a blur of the
grid, then slicing) run by the generated kernels in the block emulator,
against the FP64 oracle."""
import numpy as np
import pytest

from paper_1909_07190_gb300 import pipelines as P
from paper_1909_07190_gb300 import wt

from test_codegen_emu import oracle_of, rnd, run_emulated


def chan_spec():
    inp = P.input_id(0)
    b = P.Builder("chan", [1])
    s0 = b.stage("planes", P.ref(inp, 1, 0) * (P.CHAN + 1.0) - P.CHAN * P.ref(inp, 0, -1), 4)
    s1 = b.stage("one", P.ref(s0, 0, 1, chan=2) + P.CHAN + P.ref(s0, -1, 0, chan=0))
    s2 = b.stage("mix", P.ref(s0) * P.CHAN + P.ref(s1), 4)
    b.output(s1, s2)
    return b.build()


@pytest.mark.parametrize("mode", ["fused", "plain", "otptb"])
def test_chan_op(mode):
    """Plane-dependent programs in one group (a one-plane stage sees plane 0
    whatever tile channel computes it) and per stage."""
    spec = chan_spec()
    img = rnd(80, 150, 37)
    if mode == "plain":
        got, _ = run_emulated(spec, [img], exec_mode=wt.WT_EXEC_PLAIN)
    elif mode == "otptb":
        got, _ = run_emulated(spec, [img], groups=[0, 1, 1],
                              params=[dict(tile_h=8, warps_per_block=2, flags=wt.WT_FLAG_OTPTB)] * 2)
    else:
        got, _ = run_emulated(spec, [img], groups=[0, 1, 1], params=[dict(tile_h=8)] * 2)
    for g, r in zip(got, oracle_of(spec, [img])):
        assert np.abs(g - r).max() <= 1e-5


def grid_groups(spec):
    """One group per level run (consecutive stages of one level)."""
    from paper_1909_07190_gb300 import pipelines as P2
    lv = []
    for st in spec["stages"]:
        level = 0
        for op in st["ops"]:
            if op[0] == "tap":
                pid = st["inputs"][op[1]]
                level = (0 if pid < 0 else lv[pid]) + {"same": 0, "down2": 1, "up2": -1}[op[5]]
                break
        lv.append(level)
    g, cur = [0], 0
    for i in range(1, len(lv)):
        if lv[i] != lv[i - 1]:
            cur += 1
        g.append(cur)
    return g


@pytest.mark.parametrize("w,h,tile_h", [(67, 45, 8), (130, 70, 4), (9, 5, 8)])
def test_bilateral_grid(w, h, tile_h):
    spec = P.bilateral_grid(4, 3)
    img = rnd(81 + w, w, h)
    g = grid_groups(spec)
    got, _ = run_emulated(spec, [img], groups=g, params=[dict(tile_h=tile_h)] * (max(g) + 1))
    ref = oracle_of(spec, [img])[0]
    assert np.abs(got[0] - ref).max() <= 1e-5 * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("w,h", [(67, 45), (300, 41)])
def test_bilateral_filter(w, h):
    spec = P.bilateral_filter(4, 3)
    img = rnd(82 + w, w, h)
    g = grid_groups(spec)
    got, _ = run_emulated(spec, [img], groups=g, params=[dict(tile_h=8)] * (max(g) + 1))
    ref = oracle_of(spec, [img])[0]
    assert np.abs(got[0] - ref).max() <= 1e-5
    got, _ = run_emulated(spec, [img], exec_mode=wt.WT_EXEC_PLAIN)
    assert np.abs(got[0] - ref).max() <= 1e-5


@pytest.mark.parametrize("w,h,bins,levels", [(67, 45, 4, 3), (130, 70, 3, 2), (9, 5, 4, 3), (270, 33, 2, 4),
                                             (33, 1, 4, 3)])
def test_reduction_chain(w, h, bins, levels):
    """The grid's splat and 2x2 sums as one cross-level launch (the chain
    kernel), then the blur, against the oracle; odd sizes make every level
    clamp its own edge."""
    spec = P.bilateral_grid(bins, levels)
    img = rnd(83 + w + levels, w, h)
    groups = [0] * levels + [1]
    got, d = run_emulated(spec, [img], groups=groups, params=[dict(tile_h=8)] * 2)
    assert d["name"].startswith("wt_chain_")
    assert d["n_launches"] == 2
    ref = oracle_of(spec, [img])[0]
    assert np.abs(got[0] - ref).max() <= 1e-5 * max(1.0, np.abs(ref).max())


def test_reduction_chain_weighted_and_filter():
    """Weighted 2x2 sums (a chain of binomial-like reductions) and the full
    bilateral filter with its chain."""
    inp = P.input_id(0)
    b = P.Builder("chain", [1])
    s0 = b.stage("sq", P.ref(inp, 0, 0, mode="down2") * P.ref(inp, 1, 1, mode="down2") + P.CHAN, 3)
    s1 = b.stage("w1", 0.5 * P.ref(s0, 0, 0, mode="down2") + 0.25 * P.ref(s0, 1, 0, mode="down2")
                 - P.ref(s0, 1, 1, mode="down2"), 3)
    s2 = b.stage("w2", P.ref(s1, 0, 1, mode="down2") * 2.0 + P.ref(s1, 1, 0, mode="down2") / 4.0, 3)
    b.output(s2)
    spec = b.build()
    img = rnd(84, 91, 37)
    got, d = run_emulated(spec, [img], groups=[0, 0, 0], params=[dict()])
    assert d["name"].startswith("wt_chain_")
    assert np.abs(got[0] - oracle_of(spec, [img])[0]).max() <= 1e-5
    spec = P.bilateral_filter(4, 3)
    groups, params = P.bilateral_schedule(4, 3)
    img = rnd(85, 150, 77)
    got, d = run_emulated(spec, [img], groups=groups, params=params)
    assert np.abs(got[0] - oracle_of(spec, [img])[0]).max() <= 1e-5


def chain_spec(const=0.0, extra_consumer=False, slot_offset=0):
    inp = P.input_id(0)
    b = P.Builder("c", [1])
    s0 = b.stage("s1", P.ref(inp, 0, 0, mode="down2") + P.ref(inp, 1, slot_offset, mode="down2"), 2)
    s1 = b.stage("s2", P.ref(s0, 0, 0, mode="down2") + P.ref(s0, 1, 1, mode="down2") + const, 2)
    outs = [s1]
    if extra_consumer:
        outs.append(b.stage("side", P.ref(s0) * 2.0, 2))
    b.output(*outs)
    return b.build()


@pytest.mark.parametrize("case", ["chain", "const", "consumed", "far_tap"])
def test_chain_detection(case):
    """Only true reduction chains become one launch: a constant term, an
    intermediate read outside the group, or a tap outside the 2x2 block
    leave the group to per-stage kernels; every case matches the oracle."""
    spec = {"chain": chain_spec(), "const": chain_spec(const=0.5), "consumed": chain_spec(extra_consumer=True),
            "far_tap": chain_spec(slot_offset=2)}[case]
    img = rnd(98, 45, 31)
    groups = [0, 0] + ([1] if case == "consumed" else [])
    got, d = run_emulated(spec, [img], groups=groups, params=[dict()] * (max(groups) + 1))
    assert d["name"].startswith("wt_chain_") == (case == "chain")
    for g, r in zip(got, oracle_of(spec, [img])):
        assert np.abs(g - r).max() <= 1e-5

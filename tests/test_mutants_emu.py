"""Mutated pipelines at the C-ABI boundary.

Each case takes a known pipeline (sharpen, the corner response, a
two-level blend, the bilateral grid, random DAGs) and changes one thing:
a tap's offset, channel, scaling mode or producer slot, a stage's input
list or channel count, a dropped or duplicated program op.  The library
either rejects the result with an error status or accepts it; what it
accepts the FP64 oracle must accept too, and the generated kernels, run
by the block emulator, must match the oracle on it.
"""
import copy

import numpy as np
import pytest

from paper_1909_07190_gb300 import pipelines as P
from paper_1909_07190_gb300 import wt

from test_codegen_emu import oracle_of, random_dag, rnd, run_emulated


def bases():
    return [P.sharpen(), P.harris(), P.blend(levels=2, channels=1), random_dag(3), random_dag(5),
            P.bilateral_grid(4, 2)]


def mutant(seed):
    """(spec, what changed) for seed; the spec may be invalid."""
    rng = np.random.default_rng(seed)
    base = bases()
    spec = copy.deepcopy(base[int(rng.integers(0, len(base)))])
    st = spec["stages"]
    si = int(rng.integers(0, len(st)))
    S = st[si]
    kind = int(rng.integers(0, 8))
    taps = [j for j, o in enumerate(S["ops"]) if o[0] == "tap"]
    modes = list(wt.TAPMODES)
    if kind <= 4 and taps:
        j = taps[int(rng.integers(0, len(taps)))]
        o = list(S["ops"][j]) + [-1, "same"][len(S["ops"][j]) - 4:]
        f = [2, 3, 4, 5, 1][kind]
        if f in (2, 3):
            o[f] = int(rng.integers(-20, 21))
        elif f == 4:
            o[f] = int(rng.integers(-2, 5))
        elif f == 5:
            o[f] = modes[int(rng.integers(0, len(modes)))]
        else:
            o[f] = int(rng.integers(-1, 4))
        S["ops"][j] = tuple(o)
        what = "tap field %d of stage %d" % (f, si)
    elif kind == 5:
        S["inputs"][int(rng.integers(0, len(S["inputs"])))] = int(rng.integers(-3, len(st) + 1))
        what = "input list of stage %d" % si
    elif kind == 6:
        S["channels"] = int(rng.choice([0, 1, 2, 3, 40]))
        what = "channels of stage %d" % si
    elif len(S["ops"]) > 1 and rng.uniform() < 0.5:
        del S["ops"][int(rng.integers(0, len(S["ops"])))]
        what = "op dropped from stage %d" % si
    else:
        S["ops"].insert(int(rng.integers(0, len(S["ops"]))), S["ops"][int(rng.integers(0, len(S["ops"])))])
        what = "op duplicated in stage %d" % si
    return spec, what


def test_accepted_mutants_are_valid_for_the_oracle():
    """Over many mutants: every status is OK or WT_EINVAL, both outcomes
    occur, and the oracle evaluates every accepted spec."""
    seen = {"ok": 0, "rejected": 0}
    for seed in range(600):
        spec, what = mutant(seed)
        try:
            wt.Pipeline(spec)
        except wt.WtError as e:
            assert e.code == wt.WT_EINVAL, (seed, what, e)
            seen["rejected"] += 1
            continue
        seen["ok"] += 1
        imgs = [rnd(7 + k, 37, 23, c) for k, c in enumerate(spec["inputs"])]
        oracle_of(spec, imgs)
    assert seen["ok"] > 100 and seen["rejected"] > 100


@pytest.mark.parametrize("seed", [2, 3, 14, 19, 24, 38, 45, 47, 68, 111])
def test_accepted_mutant_kernels_match_the_oracle(seed):
    """Accepted mutants of every kind the library accepts: tap offsets,
    channels and slots, input lists, stage channel counts."""
    spec, what = mutant(seed)
    wt.Pipeline(spec)
    imgs = [rnd(7 + k, 37, 23, c) for k, c in enumerate(spec["inputs"])]
    ref = oracle_of(spec, imgs)
    got, _ = run_emulated(spec, imgs)
    for g, r in zip(got, ref):
        assert np.abs(g - r).max() <= 1e-5 * max(1.0, np.abs(r).max()), what

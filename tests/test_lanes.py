"""Concurrent launch lanes of a run plan (host logic, no GPU).

A run's launches that read nothing an earlier launch writes may run on side
streams beside each other.  These tests take every read-after-write
dependency from the pipeline definition itself (which stage reads which)
and check that the lanes and waits the library plans order each one, so a
missing wait (a launch that could read a producer's output before it is
written) fails here.
"""
import pytest

from paper_1909_07190_gb300 import pipelines as P
from paper_1909_07190_gb300 import wt


def img(W, H, C, dt, base):
    es = 4 if dt == wt.WT_F32 else 2
    return wt.image(base, W, H, C, dt, ((W * es + 127) // 128) * 128)


def io(spec, W, H, dt):
    ins = [img(W, H, c, dt, (1 + j) << 36) for j, c in enumerate(spec["inputs"])]
    outs = [img(W, H, spec["stages"][s]["channels"], dt, (8 + k) << 36) for k, s in enumerate(spec["outputs"])]
    return ins, outs


def happens_before(launches):
    """hb[j] = set of launches complete before launch j starts: its lane's
    earlier launches and, through each wait, what the waited launch saw."""
    hb = []
    last = {}
    for j, L in enumerate(launches):
        s = set()
        if L["lane"] in last:
            p = last[L["lane"]]
            s |= hb[p] | {p}
        for w in L["waits"]:
            assert w < j
            s |= hb[w] | {w}
        hb.append(s)
        last[L["lane"]] = j
    return hb


def check_order(spec, launches):
    owner = {}
    for j, L in enumerate(launches):
        for s in L["stages"]:
            owner[s] = j
    hb = happens_before(launches)
    deps = 0
    for j, L in enumerate(launches):
        for s in L["stages"]:
            for pid in spec["stages"][s]["inputs"]:
                if pid < 0 or pid in L["stages"]:
                    continue
                i = owner[pid]
                assert i < j, "launch %d reads stage %d of a later launch %d" % (j, pid, i)
                assert i in hb[j], "launch %d may start before launch %d writes stage %d" % (j, i, pid)
                deps += 1
    return deps


def test_blend_levels_on_three_lanes():
    spec = P.blend()
    p = wt.Pipeline(spec)
    groups, params = P.blend_schedule()
    p.schedule(groups=groups, params=params)
    n, launches = p.debug_lanes(*io(spec, 8192, 8192, wt.WT_BF16))
    assert n == 3
    assert check_order(spec, launches) > 20
    names = [s["name"] for s in spec["stages"]]
    lane = {names[L["stages"][0]]: L["lane"] for L in launches}
    # the three pyramids' down-sampling chains run side by side
    assert len({lane["GA1"], lane["GB1"], lane["GM1"]}) == 3
    assert lane["GA2"] == lane["GA1"] and lane["GB3"] == lane["GB1"]
    # redundant waits are pruned: the reconstruction chain waits once
    assert sum(len(L["waits"]) for L in launches) == 2


@pytest.mark.parametrize("name", ["harris", "sharpen", "blend"])
def test_plain_path_orders_every_dependency(name):
    spec = P.by_name(name)
    p = wt.Pipeline(spec)
    p.schedule(exec_mode=wt.WT_EXEC_PLAIN)
    dt = wt.WT_BF16 if name == "blend" else wt.WT_F32
    n, launches = p.debug_lanes(*io(spec, 1000, 600, dt))
    assert 1 <= n <= 4
    assert check_order(spec, launches) >= len(spec["stages"]) - 1
    if name == "harris":
        assert n > 1  # Ix and Iy (and their products) are independent


def test_single_group_one_lane():
    spec = P.harris()
    p = wt.Pipeline(spec)
    n, launches = p.debug_lanes(*io(spec, 4096, 4096, wt.WT_F32))
    assert n == 1 and len(launches) == 1 and launches[0]["waits"] == []


def test_one_stream_flag():
    spec = P.blend()
    p = wt.Pipeline(spec)
    groups, params = P.blend_schedule()
    params = [dict(q) for q in params]
    params[-1]["flags"] = params[-1].get("flags", 0) | wt.WT_FLAG_ONE_STREAM
    p.schedule(groups=groups, params=params)
    assert p.schedule_get()["params"][-1]["flags"] & wt.WT_FLAG_ONE_STREAM
    n, launches = p.debug_lanes(*io(spec, 8192, 8192, wt.WT_BF16))
    assert n == 1
    assert all(L["lane"] == 0 and L["waits"] == [] for L in launches)
    check_order(spec, launches)


def test_bilateral_chain_in_order():
    spec = P.bilateral_filter()
    p = wt.Pipeline(spec)
    groups, params = P.bilateral_schedule()
    p.schedule(groups=groups, params=params)
    n, launches = p.debug_lanes(*io(spec, 4096, 4096, wt.WT_F32))
    check_order(spec, launches)

"""The scheduler's formulas against the numbers the paper prints
(tests/golden/paper_examples.json, each with its citation), plus
properties of the cost function and of DP-Fusion."""
import json
import os

import pytest

from paper_1909_07190_gb300 import pipelines as P
from paper_1909_07190_gb300 import wt

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_examples.json")))


def cfg_from(d):
    c = wt.wt_gpu_config()
    c.nsms, c.cores_per_sm, c.glmem_bw_gbs = d["NSMs"], d["CoresPerSM"], d["GlMemBW_GBps"]
    c.max_smem_per_block, c.smem_per_sm = d["MaxShMemPerTb"], d["ShMemPerSM"]
    c.max_warps_per_sm, c.max_blocks_per_sm = d["MaxWarpPerSM"], d["MaxTbPerSM"]
    c.regs_per_sm, c.max_regs_per_thread, c.warp_size = d["RegPerSM"], d["MaxRegPerTh"], d["WarpSize"]
    c.max_threads_per_sm = d["MaxWarpPerSM"] * d["WarpSize"]
    return c


def test_warp_sizes_worked_example():
    g = GOLD["warp_tile_example"]
    w = wt.otpw_warp_sizes(g["block"])
    assert w == g["warp_sizes"]
    assert w[0] * w[1] * w[2] == 32
    assert [t * s for t, s in zip(g["tile"], w)] == g["warp_tile"]


@pytest.mark.parametrize("block", [[64, 4, 1], [32, 8, 2], [8, 16, 4], [256, 1, 1], [4, 4, 8]])
def test_warp_sizes_cover_one_warp(block):
    w = wt.otpw_warp_sizes(block)
    assert w[0] * w[1] * w[2] == 32 and all(1 <= wi <= bi for wi, bi in zip(w, block))


def test_blur_overlap_fraction():
    g = GOLD["blur_otpw"]
    # overlap per warp = O_x / (T_x * W_x) with W_x = 32 (blocks 64x4x1)
    w = wt.otpw_warp_sizes(g["block"])
    for tile, pct in ((8, g["tile8_overlap_pct"]), (16, g["tile16_overlap_pct"])):
        frac = g["overlap_points_x"] / (tile * w[0])
        assert round(100 * frac, 1) == pct


def test_blur_scratchpad_and_occupancy_1080ti():
    g, h = GOLD["blur_otpw"], GOLD["blur_hybrid"]
    cfg = cfg_from(GOLD["gtx1080ti"])
    w = wt.otpw_warp_sizes(g["block"])
    full = wt.otpw_scratchpad(g["block"], w, [16, 1, 1], [g["overlap_points_x"], 0, 0]) * 4
    assert full > g["tile16_smem_over_bytes"]            # "over 16KB"
    occ, _ = wt.cost_occupancy(cfg, full, 8, h["registers"])
    assert round(100 * occ, 1) == g["tile16_occupancy_pct"]
    # half the tile in registers: the shared part is the first 8 of 16 tiles
    half = wt.otpw_scratchpad(g["block"], w, [8, 1, 1], [g["overlap_points_x"], 0, 0]) * 4
    occ, _ = wt.cost_occupancy(cfg, half, 8, h["registers"])
    assert round(100 * occ, 1) == h["occupancy_pct"]
    # tile 8 fits without hybrid tiling at full occupancy as well (Sec. 3)
    occ8, _ = wt.cost_occupancy(cfg, wt.otpw_scratchpad(g["block"], w, [8, 1, 1], [2, 0, 0]) * 4, 8, 24)
    assert occ8 == 1.0


def test_occupancy_register_limit():
    cfg = cfg_from(GOLD["gtx1080ti"])
    occ, tb = wt.cost_occupancy(cfg, 0, 4, 128)     # 65536/128 = 512 threads = 16 warps
    assert occ == 16 / 64 and tb == 4


@pytest.mark.parametrize("addrs,acc,txn,want", [
    ([4 * i for i in range(32)], 4, 128, 1),          # 32 floats, aligned: one 128 B line
    ([4 * i for i in range(32)], 4, 32, 4),           # ... or four sectors
    ([4 * i + 4 for i in range(32)], 4, 128, 2),      # shifted by one float: two lines
    ([8 * i for i in range(32)], 4, 32, 8),           # stride 2: 256 B span
    ([128 * i for i in range(32)], 4, 32, 32),        # one transaction per lane
    ([16 * i for i in range(32)], 16, 128, 4),        # 128-bit accesses: 512 B
])
def test_min_transactions(addrs, acc, txn, want):
    assert wt.min_transactions(addrs, acc, txn) == want


def test_weights_default_to_table3_v100_and_roundtrip():
    w0 = wt.cost_weights()
    assert w0 == GOLD["weights"]["v100"]
    wt.cost_weights([1, 2, 3, 4, 5, 6, 7])
    assert wt.cost_weights() == [1, 2, 3, 4, 5, 6, 7]
    wt.cost_weights(w0)


def test_cost_terms_are_sane_for_harris():
    p = wt.Pipeline(P.harris())
    c = p.cost_group(0, 11, dict(tile_h=32, warps_per_block=4, frac_reg=1.0), 128, 4096, 4096)
    assert c["feasible"]
    t = c["terms"]
    assert 0.99 < t[0] < 1.5                # traffic close to the pipeline minimum
    assert 0 <= t[1] < 1 and 0 <= t[3] <= 1 and 0 <= t[6] < 1
    assert 0 < t[5] < 0.5                   # halo recompute at tile height 32
    # a shorter tile recomputes more
    c8 = p.cost_group(0, 11, dict(tile_h=8, warps_per_block=4, frac_reg=1.0), 128, 4096, 4096)
    assert c8["terms"][5] > t[5]
    # one stage per group reads and writes far more than the fused group
    cs = p.cost_group(0, 1, dict(tile_h=32, warps_per_block=4), 128, 4096, 4096)
    assert cs["terms"][0] < t[0]            # (a single stage moves less than all 11)


def test_cost_rejects_oversized_shared_memory():
    p = wt.Pipeline(P.harris())
    c = p.cost_group(0, 11, dict(tile_h=32, warps_per_block=16, frac_reg=0.0, vec=8), 128, 4096, 4096)
    assert not c["feasible"]


def test_auto_schedule_fuses_corner_response():
    p = wt.Pipeline(P.harris())
    p.schedule_auto(4096, 4096, wt.WT_F32, wt.WT_MODEL_ANALYTIC)
    s = p.schedule_get()
    assert s["exec"] == wt.WT_EXEC_FUSED
    assert len(set(s["groups"])) <= 3       # the DP keeps most stages together


def test_auto_schedule_blend_groups_by_level():
    p = wt.Pipeline(P.blend())
    p.schedule_auto(512, 512, wt.WT_BF16, wt.WT_MODEL_ANALYTIC)
    s = p.schedule_get()
    groups = s["groups"]
    assert groups == sorted(groups) and groups[0] == 0


def test_dp_fusion_groups_blend_by_level():
    """DP-Fusion over the 36-stage blend (stages ordered by level): the
    Gaussian levels 1-2 and 3-4 as two groups spanning two levels each (a
    cascade launch per image: each pair's first level is written and
    reduced again on chip, so its read-back drops out of the traffic term),
    the coarsest level's stages as per-stage kernels, then one fused group
    per finer level (taps of the neighbouring level are gather sources)."""
    spec = P.blend()
    p = wt.Pipeline(spec)
    p.schedule_auto(8192, 8192, wt.WT_BF16, wt.WT_MODEL_ANALYTIC)
    s = p.schedule_get()
    expect = [0] * 6 + [1] * 6 + [2, 3, 4, 5] + sum([[6 + k] * 4 for k in range(5)], [])
    assert s["groups"] == expect
    assert p.launches_per_run() == 3 + 3 + 4 + 5
    img = wt.image(0x10000000, 8192, 8192, 3, wt.WT_BF16, 8192 * 2)
    msk = wt.image(0x10000000, 8192, 8192, 1, wt.WT_BF16, 8192 * 2)
    names = [p.kernel_name(i, [img, img, msk], [img]) for i in range(15)]
    assert all(n.startswith("wt_down2_") for n in names[:6]), names
    assert all(n.startswith("wt_down_") for n in names[6:9]), names
    assert names[9].startswith("wt_plain_"), names
    assert all(n.startswith("wt_fused_") for n in names[10:]), names


def test_dp_fusion_proposes_reduction_chain_across_levels():
    """DP-Fusion (analytic model) groups the bilateral grid's splat and its
    2x2 sums, three levels, as one group: the reduction-chain kernel reads
    the image once and writes only the coarsest level, which the traffic
    term prefers to any split (no GPU needed)."""
    from paper_1909_07190_gb300 import pipelines as P
    from paper_1909_07190_gb300 import wt
    spec = P.bilateral_filter()
    p = wt.Pipeline(spec)
    p.schedule_auto(4096, 4096, wt.WT_F32, wt.WT_MODEL_ANALYTIC)
    g = p.schedule_get()["groups"]
    assert g[0] == g[1] == g[2] and g[3] != g[2], g
    img = wt.image(0x10000000, 4096, 4096, 1, wt.WT_F32, 4096 * 4)
    assert p.kernel_name(0, [img], [img]).startswith("wt_chain_")


def _groupings(n, max_group):
    """Every split of stages 0..n-1 into contiguous groups of at most
    max_group stages, as lists of (first, end)."""
    if n == 0:
        yield []
        return
    for k in range(1, min(n, max_group) + 1):
        for rest in _groupings(n - k, max_group):
            yield [(0, k)] + [(a + k, b + k) for a, b in rest]


@pytest.mark.parametrize("case", ["sharpen_2048", "harris_4096", "harris_600x410_f16", "blur_1024",
                                  "random6_512", "random9_4096_bf16"])
def test_dp_fusion_matches_brute_force(case):
    """Alg. 2's DP over contiguous groupings against enumerating all of
    them: every grouping's cost is the sum of its groups' costs (the same
    per-group choice the DP weighs), and the grouping wt_schedule_auto
    installs reaches the smallest sum."""
    from test_codegen_emu import random_dag
    spec, W, H, dt = {
        "sharpen_2048": (P.sharpen(), 2048, 2048, wt.WT_F32),
        "harris_4096": (P.harris(), 4096, 4096, wt.WT_F32),
        "harris_600x410_f16": (P.harris(), 600, 410, wt.WT_F16),
        "blur_1024": (P.by_name("blur"), 1024, 1024, wt.WT_F32),
        "random6_512": (random_dag(11, n_stages=6), 512, 512, wt.WT_F32),
        "random9_4096_bf16": (random_dag(12, n_stages=9), 4096, 4096, wt.WT_BF16),
    }[case]
    n = len(spec["stages"])
    p = wt.Pipeline(spec)
    cost = {(a, b): p.debug_segment_cost(a, b - a, W, H, dt)[0]
            for a in range(n) for b in range(a + 1, min(n, a + 16) + 1)}
    sums = sorted(sum(cost[g] for g in split) for split in _groupings(n, 16))
    assert len(sums) == 2 ** (n - 1)
    p.schedule_auto(W, H, dt, wt.WT_MODEL_ANALYTIC)
    groups = p.schedule_get()["groups"]
    split = [(groups.index(g), len(groups) - groups[::-1].index(g)) for g in sorted(set(groups))]
    assert sum(cost[g] for g in split) == pytest.approx(sums[0], rel=1e-12)
    # the minimum is a real choice, not a tie across every grouping
    assert sums[-1] > sums[0]


def test_segment_cost_ranges():
    p = wt.Pipeline(P.harris())
    c, fused = p.debug_segment_cost(0, 11, 4096, 4096)
    assert fused and c > 0
    c1, f1 = p.debug_segment_cost(10, 1, 4096, 4096)
    assert c1 > 0
    for first, n in [(-1, 2), (0, 0), (5, 7), (0, 17)]:
        with pytest.raises(wt.WtError):
            p.debug_segment_cost(first, n, 4096, 4096)

"""Pins of the FP64 oracle against facts fixed by the definitions and by
mathematics (not against itself): constant images, impulse responses,
separable vs direct 2-D correlation with numpy's edge padding as the
clamp-to-edge rule, ramp closed forms, Laplacian-pyramid identities, a
memo-free recursive evaluator, and malformed DAGs."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1909_07190_gb300 import inputs as I
from paper_1909_07190_gb300 import pipelines as P

B5 = np.array([1, 4, 6, 4, 1], np.float64) / 16


def run(pipe, imgs, outs=None):
    return O.evaluate(pipe["stages"], imgs, pipe["outputs"] if outs is None else outs)


def rnd(seed, w, h, c=1):
    return I.uniform_image(seed, w, h, c).astype(np.float64)


def corr2_edge(img, k):
    """2-D correlation with clamp-to-edge, via numpy's edge padding."""
    ry, rx = k.shape[0] // 2, k.shape[1] // 2
    p = np.pad(img, ((ry, ry), (rx, rx)), mode="edge")
    out = np.zeros_like(img)
    for j in range(k.shape[0]):
        for i in range(k.shape[1]):
            out += k[j, i] * p[j:j + img.shape[0], i:i + img.shape[1]]
    return out


# ----------------------------------------------------------------- constants

@pytest.mark.parametrize("c", [0.0, 0.37, 1.0])
def test_constant_sharpen_is_identity(c):
    img = np.full((13, 17), c)
    assert np.abs(run(P.sharpen(), [img])[0][0] - c).max() < 1e-15
    assert np.abs(O.sharpen(img) - c).max() < 1e-15


@pytest.mark.parametrize("pipe", ["harris", "harris_raw"])
def test_constant_harris_is_zero(pipe):
    img = np.full((11, 9), 0.61)
    # Zero in exact arithmetic; FP64 partial sums of the Sobel taps leave a
    # residue of order 1e-16, which det and trace^2 raise to the 4th power.
    assert np.abs(run(P.by_name(pipe), [img])[0]).max() < 1e-28
    assert np.abs(O.harris(img, pipe == "harris")).max() < 1e-28


def test_constant_blend():
    a, b, m = 0.3, 0.8, 0.25
    A = np.full((3, 40, 36), a); B = np.full((3, 40, 36), b); M = np.full((1, 40, 36), m)
    want = m * a + (1 - m) * b
    assert np.abs(run(P.blend(), [A, B, M])[0] - want).max() < 1e-14
    assert np.abs(O.blend(A, B, M) - want).max() < 1e-14


# ------------------------------------------------------------------ impulses

def impulse(w, h, x0, y0):
    img = np.zeros((h, w))
    img[y0, x0] = 1.0
    return img


def test_impulse_binomial_blur():
    img = impulse(17, 15, 8, 7)
    bx, by = run(P.sharpen(), [img], [0, 1])
    want_bx = np.zeros((15, 17)); want_bx[7, 6:11] = B5
    assert np.abs(bx[0] - want_bx).max() < 1e-17
    want_by = np.zeros((15, 17)); want_by[5:10, 6:11] = np.outer(B5, B5)
    assert np.abs(by[0] - want_by).max() < 1e-17


def test_impulse_sobel_orientation_and_sign():
    img = impulse(9, 9, 4, 4)
    ix, iy = run(P.harris(), [img], [0, 1])
    # Correlation: Ix(x, y) = 1/8 sum K[j][i] in(x+i-1, y+j-1), so the pixel
    # right of the impulse sees K[1][0] = -2 and the one left sees K[1][2] = +2.
    want_ix = np.zeros((9, 9))
    want_ix[3:6, 3:6] = np.array(P.SOBEL_X, np.float64)[::-1, ::-1] / 8.0
    assert ix[0][4, 5] == -0.25 and ix[0][4, 3] == 0.25
    assert np.abs(ix[0] - want_ix).max() < 1e-17
    assert iy[0][5, 4] == -0.25 and iy[0][3, 4] == 0.25 and iy[0][4, 5] == 0.0
    assert np.abs(iy[0] - want_ix.T).max() < 1e-17


def test_impulse_box():
    b = P.Builder("box", [1])
    s = b.stage("box", P.linear(P.input_id(0), P.BOX3, 1.0 / 9))
    b.output(s)
    img = impulse(7, 6, 3, 2)
    out = run(b.build(), [img])[0][0]
    want = np.zeros((6, 7)); want[1:4, 2:5] = 1.0 / 9
    assert np.abs(out - want).max() < 1e-17


def _down_only():
    b = P.Builder("down", [1])
    d = b.stage("G1", P._down(P.input_id(0)))
    b.output(d)
    return b.build()


def test_impulse_downsample_even_phase():
    # G1(x, y) = sum b_i b_j in(2x+i, 2y+j): an impulse at the even point
    # (10, 10) lands at (5, 5) with weight b0^2 and at (4|6, 5) with b2 b0.
    out = run(_down_only(), [impulse(24, 24, 10, 10)])[0][0]
    assert out.shape == (12, 12)
    want = np.zeros((12, 12))
    w = np.array([1, 6, 1]) / 16.0
    want[4:7, 4:7] = np.outer(w, w)
    assert np.abs(out - want).max() < 1e-17
    # An odd point (11, 10) splits between x = 5 and x = 6 with b_{+-1} = 4/16.
    out = run(_down_only(), [impulse(24, 24, 11, 10)])[0][0]
    want = np.zeros((12, 12)); want[4:7, 5:7] = np.outer(w, [4 / 16, 4 / 16])
    assert np.abs(out - want).max() < 1e-17


def _sample_up():
    """D(i, j) = in(2i, 2j) (one DOWN2 tap), U = up(D)."""
    b = P.Builder("sample_up", [1])
    d = b.stage("D", P.ref(P.input_id(0), 0, 0, mode="down2"))
    u = b.stage("U", P._up(d))
    b.output(u)
    return b.build()


def test_impulse_upsample_weights():
    img = impulse(20, 20, 10, 10)      # D has its impulse at (5, 5)
    d, u = run(_sample_up(), [img], [0, 1])
    assert d[0][5, 5] == 1.0 and d[0].sum() == 1.0
    w = {8: 0.0, 9: 0.25, 10: 0.75, 11: 0.75, 12: 0.25, 13: 0.0}
    for y, wy in w.items():
        for x, wx in w.items():
            assert abs(u[0][y, x] - wx * wy) < 1e-17, (x, y)
    assert abs(u[0].sum() - 4.0) < 1e-14


# ------------------------------------------------------- separable vs direct

def test_separable_blur_equals_direct_5x5():
    img = rnd(11, 23, 19)[0]
    by = run(P.sharpen(), [img], [1])[0][0]
    assert np.abs(by - corr2_edge(img, np.outer(B5, B5))).max() < 1e-15


def test_sobel_and_box_equal_separable_passes():
    img = rnd(12, 21, 18)[0]
    ix, iy = run(P.harris(), [img], [0, 1])
    sx = np.outer([1, 2, 1], [-1, 0, 1]) / 8.0
    assert np.abs(ix[0] - corr2_edge(img, sx)).max() < 1e-15
    assert np.abs(iy[0] - corr2_edge(img, sx.T)).max() < 1e-15
    b = P.Builder("box", [1])
    b.output(b.stage("box", P.linear(P.input_id(0), P.BOX3)))
    box = run(b.build(), [img])[0][0]
    two_pass = corr2_edge(corr2_edge(img, np.ones((1, 3))), np.ones((3, 1)))
    assert np.abs(box - two_pass).max() < 1e-14


# ------------------------------------------------- sharpen's output stage

def _sharpen_numpy(img):
    """The configuration's definition, written with numpy alone: a 5x5
    binomial blur with numpy's edge padding as clamp-to-edge, then
    clamp(in + 1.5 (in - blur), 0, 1)."""
    blur = corr2_edge(img, np.outer(B5, B5))
    return np.clip(img + 1.5 * (img - blur), 0.0, 1.0)


def test_sharpen_step_edge_gain_and_clamp_by_hand():
    """A vertical step from 0.2 to 0.8: along a row the blur is the 1-D
    binomial of the step (rows are constant), so every output column has a
    closed form.  At the two columns beside the edge the unclamped value
    leaves [0, 1] (the clamp engages at both ends); one column further out
    it stays inside and shows the 1.5 gain."""
    img = np.tile(np.where(np.arange(12) < 6, 0.2, 0.8), (9, 1))
    out = run(P.sharpen(), [img])[0][0]
    lo, hi = 0.2, 0.8
    # blur at columns 4, 5 | 6, 7 (edge between 5 and 6), weights /16
    blur = {4: (15 * lo + 1 * hi) / 16, 5: (11 * lo + 5 * hi) / 16,
            6: (5 * lo + 11 * hi) / 16, 7: (1 * lo + 15 * hi) / 16}
    raw = {x: img[0, x] + 1.5 * (img[0, x] - b) for x, b in blur.items()}
    assert raw[5] < 0.0 and raw[6] > 1.0          # both clamps engage
    assert 0.0 < raw[4] < 1.0 and 0.0 < raw[7] < 1.0
    want = {4: lo - 1.5 * (hi - lo) / 16, 5: 0.0, 6: 1.0, 7: hi + 1.5 * (hi - lo) / 16}
    assert abs(raw[4] - want[4]) < 1e-15 and abs(raw[7] - want[7]) < 1e-15
    for x, v in want.items():
        assert np.abs(out[:, x] - v).max() < 1e-15, (x, out[0, x], v)
    # far from the edge the image is constant: out = in
    assert np.abs(out[:, :3] - lo).max() < 1e-15 and np.abs(out[:, 9:] - hi).max() < 1e-15


@pytest.mark.parametrize("w,h,seed", [(23, 17, 1), (40, 9, 2)])
def test_sharpen_matches_numpy_definition(w, h, seed):
    """Random images scaled beyond [0, 1]'s middle so that the clamp engages
    at both ends, and a 0/1 checkerboard of 3x3 cells (every pixel near a
    cell edge clamps)."""
    img = np.clip(rnd(seed, w, h)[0] * 1.4 - 0.2, 0.0, 1.0)
    want = _sharpen_numpy(img)
    raw = img + 1.5 * (img - corr2_edge(img, np.outer(B5, B5)))
    assert (raw < 0).any() and (raw > 1).any()
    assert np.abs(run(P.sharpen(), [img])[0][0] - want).max() < 1e-14
    assert np.abs(O.sharpen(img) - want).max() < 1e-14
    yy, xx = np.mgrid[0:h, 0:w]
    board = (((yy // 3) + (xx // 3)) % 2).astype(np.float64)
    assert np.abs(run(P.sharpen(), [board])[0][0] - _sharpen_numpy(board)).max() < 1e-14


# ---------------------------------------------------------------- ramps

def ramp(w, h, a, b, c):
    y, x = np.mgrid[0:h, 0:w]
    return a * x + b * y + c


def test_ramp_sharpen_preserved():
    img = ramp(30, 26, 0.01, 0.015, 0.2)
    out = run(P.sharpen(), [img])[0][0]
    assert np.abs(out[2:-2, 2:-2] - img[2:-2, 2:-2]).max() < 1e-14


@pytest.mark.parametrize("a,b", [(0.01, 0.02), (-0.03, 0.005), (0.0, 0.04)])
def test_ramp_harris_closed_form(a, b):
    img = ramp(24, 22, a, b, 0.5)
    ix, iy, r = run(P.harris(), [img], [0, 1, 10])
    inner = (slice(3, -3), slice(3, -3))
    assert np.abs(ix[0][inner] - a).max() < 1e-15
    assert np.abs(iy[0][inner] - b).max() < 1e-15
    assert np.abs(r[0][inner] - (-0.04 * (a * a + b * b) ** 2)).max() < 1e-18


def test_ramp_down_and_up():
    img = ramp(40, 36, 1.0, 0.0, 0.0)   # in(x, y) = x
    g1 = run(_down_only(), [img])[0][0]
    assert np.abs(g1[:, 2:-2] - 2.0 * np.arange(20)[2:-2]).max() < 1e-13
    u = run(_sample_up(), [img], [1])[0][0]   # D(i) = 2i, so U(x) = x - 0.5
    assert np.abs(u[:, 2:-2] - (np.arange(40)[2:-2] - 0.5)).max() < 1e-13


# ----------------------------------------------------- Laplacian identities

@pytest.mark.parametrize("w,h", [(64, 48), (37, 29)])
def test_blend_identities(w, h):
    A = rnd(21, w, h, 3); B = rnd(22, w, h, 3)
    M = I.smooth_mask(23, w, h).astype(np.float64)
    pipe = P.blend()
    assert np.abs(run(pipe, [A, A, M])[0] - A).max() < 1e-13
    assert np.abs(run(pipe, [A, B, np.ones_like(M)])[0] - A).max() < 1e-13
    assert np.abs(run(pipe, [A, B, np.zeros_like(M)])[0] - B).max() < 1e-13
    assert np.abs(O.blend(A, B, np.ones_like(M)) - A).max() < 1e-13


# ------------------------------------------------------------ brute force

@pytest.mark.parametrize("name", ["sharpen", "harris", "harris_raw", "blur"])
@pytest.mark.parametrize("w,h", [(8, 8), (1, 1), (3, 7), (9, 8)])
def test_brute_force_equals_arrays(name, w, h):
    pipe = P.by_name(name)
    img = rnd(31, w, h)
    full = run(pipe, [img])[0][0]
    sid = pipe["outputs"][0]
    for y in range(h):
        for x in range(w):
            assert abs(O.brute(pipe["stages"], [img], sid, x, y) - full[y, x]) < 1e-12


def test_brute_force_blend_small():
    pipe = P.blend(levels=3)
    A = rnd(41, 8, 8, 3); B = rnd(42, 8, 8, 3); M = rnd(43, 8, 8, 1)
    full = run(pipe, [A, B, M])[0]
    sid = pipe["outputs"][0]
    for c in range(3):
        for y in range(0, 8, 3):
            for x in range(8):
                v = O.brute(pipe["stages"], [A, B, M], sid, x, y, c)
                assert abs(v - full[c, y, x]) < 1e-12


# -------------------------------------------- direct vs generic; points

@pytest.mark.parametrize("w,h", [(37, 29), (1, 1), (2, 5), (64, 3)])
def test_direct_matches_generic(w, h):
    img = rnd(51, w, h)[0]
    assert np.abs(run(P.sharpen(), [img])[0][0] - O.sharpen(img)).max() < 1e-14
    assert np.abs(run(P.harris(), [img])[0][0] - O.harris(img)).max() < 1e-15
    assert np.abs(run(P.harris(False), [img])[0][0] - O.harris(img, False)).max() < 1e-11
    A = rnd(52, w, h, 3); B = rnd(53, w, h, 3); M = rnd(54, w, h)
    assert np.abs(run(P.blend(), [A, B, M])[0] - O.blend(A, B, M)).max() < 1e-13


def test_points_match_full():
    A = rnd(61, 70, 45, 3); B = rnd(62, 70, 45, 3); M = I.smooth_mask(63, 70, 45).astype(np.float64)
    pipe = P.blend()
    full = run(pipe, [A, B, M])[0]
    rng = np.random.default_rng(0)
    xs = rng.integers(0, 70, 50); ys = rng.integers(0, 45, 50); cs = rng.integers(0, 3, 50)
    xs[:4] = [0, 69, 0, 69]; ys[:4] = [0, 44, 44, 0]
    v = O.evaluate_points(pipe["stages"], [A, B, M], pipe["outputs"][0], xs, ys, cs)
    assert np.abs(v - full[cs, ys, xs]).max() == 0.0


# ------------------------------------------------------------ malformed

def test_malformed_dags_rejected():
    img = np.zeros((4, 4))
    fwd = [{"channels": 1, "inputs": [1], "ops": [("tap", 0, 0, 0)]},
           {"channels": 1, "inputs": [-1], "ops": [("tap", 0, 0, 0)]}]
    with pytest.raises(ValueError, match="-1"):
        O.shapes(fwd, [img])
    mixed = [{"channels": 1, "inputs": [-1], "ops": [("tap", 0, 0, 0, -1, "down2")]},
             {"channels": 1, "inputs": [-1, 0], "ops": [("tap", 0, 0, 0), ("tap", 1, 0, 0), ("add",)]}]
    with pytest.raises(ValueError, match="-2"):
        O.shapes(mixed, [img])
    neg = [{"channels": 1, "inputs": [-1], "ops": [("tap", 0, 0, 0, -1, "up2")]}]
    with pytest.raises(ValueError, match="-3"):
        O.shapes(neg, [img])
    under = [{"channels": 1, "inputs": [-1], "ops": [("tap", 0, 0, 0), ("add",)]}]
    with pytest.raises(ValueError, match="-4"):
        O.shapes(under, [img])


# ------------------------------------------- channel index and the grid


def test_chan_op_pushes_the_channel():
    """CHAN is the output point's channel: plane c of a 5-channel stage is
    c everywhere; a one-channel stage sees 0."""
    b = P.Builder("chan", [1])
    s0 = b.stage("planes", P.CHAN + 0.0 * P.ref(P.input_id(0)), 5)
    s1 = b.stage("one", P.CHAN + P.ref(s0, 0, 0, chan=3))
    b.output(s0, s1)
    spec = b.build()
    img = I.uniform_image(5, 9, 7)
    out = O.evaluate(spec["stages"], [img.astype(np.float64)], spec["outputs"])
    for c in range(5):
        assert np.all(out[0][c] == c)
    assert np.all(out[1] == 3.0)


def block_sums(img, levels):
    """Sum over 2^levels x 2^levels blocks of the image extended by edge
    replication (the clamp-to-edge reads of the 2x2 sums), computed level by
    level with plain numpy."""
    a = np.asarray(img, np.float64)
    for _ in range(levels):
        h, w = a.shape
        ph, pw = (h + 1) // 2 * 2, (w + 1) // 2 * 2
        a = np.pad(a, ((0, ph - h), (0, pw - w)), mode="edge")
        a = a[0::2, 0::2] + a[1::2, 0::2] + a[0::2, 1::2] + a[1::2, 1::2]
    return a


@pytest.mark.parametrize("w,h", [(16, 16), (37, 21), (8, 9)])
def test_grid_partition_of_unity(w, h):
    """The tent weights of each pixel sum to 1 over the bins, so before the
    blur the weight channels of a cell sum to its pixel count and the value
    channels to its intensity sum (closed forms by block sums)."""
    bins, levels = 6, 3
    spec = P.bilateral_grid(bins, levels)
    img = I.uniform_image(9, w, h)[0].astype(np.float64)
    st = spec["stages"]
    g3 = O.evaluate(st, [img[None]], [levels - 1])[0]   # G3: before the blur
    assert np.allclose(g3[:bins].sum(0), block_sums(np.ones_like(img), levels), rtol=0, atol=1e-12)
    assert np.allclose(g3[bins:].sum(0), block_sums(img, levels), rtol=0, atol=1e-11)


def test_grid_of_a_constant_image():
    """A constant image c: every cell's bin z holds 64 max(0, 1 - |c (bins-1) -
    z|) weight and c times that value, before and after the blur."""
    bins, levels = 8, 3
    spec = P.bilateral_grid(bins, levels)
    c = 0.3
    img = np.full((1, 19, 27), c)
    g = O.evaluate(spec["stages"], [img], spec["outputs"])[0]
    for zb in range(bins):
        wz = 64 * max(0.0, 1 - abs(c * (bins - 1) - zb))
        assert np.allclose(g[zb], wz, atol=1e-12) and np.allclose(g[bins + zb], c * wz, atol=1e-12)


def test_bilateral_filter_constant_and_brute_force():
    """A constant image comes out unchanged (up to the 1e-6 guard of the
    division); on a tiny image the DAG evaluator equals the recursive brute
    force at every pixel."""
    spec = P.bilateral_filter(4, 2)
    out = O.evaluate(spec["stages"], [np.full((1, 13, 10), 0.7)], spec["outputs"])[0]
    assert np.abs(out - 0.7).max() < 1e-6
    img = I.uniform_image(10, 6, 5).astype(np.float64)
    full = O.evaluate(spec["stages"], [img], spec["outputs"])[0]
    sid = spec["outputs"][0]
    for y in range(5):
        for x in range(6):
            assert abs(O.brute(spec["stages"], [img], sid, x, y) - full[0, y, x]) < 1e-12


@pytest.mark.parametrize("s", [2, 3])
def test_scaled_taps_on_ramps(s):
    """Taps scaling by 4 and 8 read P(2^s x + d) (down) and P(floor(x / 2^s) +
    d) (up), clamped: on a ramp P(x, y) = x + 1000 y the values are those
    coordinates (closed form); a level-s domain is ceil(W / 2^s) wide."""
    W, H = 67, 45
    k = 1 << s
    ramp = (np.arange(W)[None, :] + 1000.0 * np.arange(H)[:, None])[None]
    b = P.Builder("ramp", [1])
    d = b.stage("down", P.ref(P.input_id(0), 1, -1, mode="down%d" % k))
    u = b.stage("up", P.ref(d, -1, 2, mode="up%d" % k))
    b.output(d, u)
    spec = b.build()
    shp = O.shapes(spec["stages"], [ramp])
    assert shp[0][1:3] == (-(-W // k), -(-H // k)) and shp[1][1:3] == (W, H)
    dn, up = O.evaluate(spec["stages"], [ramp], spec["outputs"])
    h, w = dn.shape[1:]
    ys, xs = np.mgrid[0:h, 0:w]
    dref = np.clip(xs * k + 1, 0, W - 1) + 1000.0 * np.clip(ys * k - 1, 0, H - 1)
    assert np.array_equal(dn[0], dref)
    ys, xs = np.mgrid[0:H, 0:W]
    uref = dref[np.clip((ys >> s) + 2, 0, h - 1), np.clip((xs >> s) - 1, 0, w - 1)]
    assert np.array_equal(up[0], uref)

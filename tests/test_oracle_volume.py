"""Pins of the FP64 oracle's 3-D taps (App. A: groups over volumes; a
D x H x W volume is an image of D planes, a plane-offset tap reads plane
z + dz clamped to [0, D-1]) against facts fixed by the definition: impulse
responses of an asymmetric 3x3x3 stencil, separable vs direct 3-D
correlation at every point (borders included), numpy's 3-D edge padding
as the clamp-to-edge rule for a chain of stencils, constants, one-plane
producers, and the memo-free recursive evaluator."""
import itertools

import numpy as np
import pytest

from oracle import oracle as O
from paper_1909_07190_gb300 import pipelines as P

B5 = np.array([1, 4, 6, 4, 1], np.float64) / 16


def run(pipe, imgs, outs=None):
    return O.evaluate(pipe["stages"], imgs, pipe["outputs"] if outs is None else outs)


def vol(seed, d, h, w):
    return np.random.default_rng(seed).random((d, h, w))


def stencil3(depth, k):
    """One stage: sum over (dz, dy, dx) of k[dz+rz, dy+ry, dx+rx] * in(z+dz, y+dy, x+dx)."""
    b = P.Builder("s3", [depth])
    inp = P.input_id(0)
    rz, ry, rx = (n // 2 for n in k.shape)
    e = None
    for z, y, x in itertools.product(*(range(n) for n in k.shape)):
        if k[z, y, x] == 0:
            continue
        t = float(k[z, y, x]) * P.refz(inp, x - rx, y - ry, z - rz)
        e = t if e is None else e + t
    b.output(b.stage("s", e, depth))
    return b.build()


def corr3_edge(v, k):
    """3-D correlation with clamp-to-edge, via numpy's edge padding."""
    rz, ry, rx = (n // 2 for n in k.shape)
    p = np.pad(v, ((rz, rz), (ry, ry), (rx, rx)), mode="edge")
    out = np.zeros_like(v)
    D, H, W = v.shape
    for z, y, x in itertools.product(*(range(n) for n in k.shape)):
        out += k[z, y, x] * p[z:z + D, y:y + H, x:x + W]
    return out


def test_impulse_response_is_the_stencil():
    """out(p) = sum_d k[d] in(p + d); an impulse at p0 gives out(p0 - d) = k[d]."""
    k = np.arange(1, 28, dtype=np.float64).reshape(3, 3, 3)  # no symmetry
    D, H, W = 7, 8, 9
    v = np.zeros((D, H, W))
    v[3, 4, 5] = 1.0
    out = run(stencil3(D, k), [v])[0]
    for dz, dy, dx in itertools.product((-1, 0, 1), repeat=3):
        assert out[3 - dz, 4 - dy, 5 - dx] == k[dz + 1, dy + 1, dx + 1]
    mask = np.ones_like(out, bool)
    mask[2:5, 3:6, 4:7] = False
    assert np.all(out[mask] == 0)


@pytest.mark.parametrize("shape", [(5, 6, 7), (1, 4, 9), (9, 3, 2)])
def test_asymmetric_stencil_against_numpy_edge_padding(shape):
    k = np.random.default_rng(4).standard_normal((3, 5, 3))
    v = vol(1, *shape)
    got = run(stencil3(shape[0], k), [v])[0]
    assert np.abs(got - corr3_edge(v, k)).max() < 1e-12


def test_separable_blur_equals_direct_everywhere():
    """Clamping acts per axis, so x, y, z passes equal the 125-tap product
    stencil at every point, borders included."""
    D, H, W = 6, 7, 11
    v = vol(2, D, H, W)
    spec = P.unsharp3d(depth=D)
    blur = run(spec, [v], outs=[2])[0]  # stage bz
    k = B5[:, None, None] * B5[None, :, None] * B5[None, None, :]
    assert np.abs(blur - corr3_edge(v, k)).max() < 1e-14
    assert np.abs(blur - run(stencil3(D, k), [v])[0]).max() < 1e-14


def test_unsharp3d_closed_form():
    D, H, W = 5, 6, 8
    v = vol(3, D, H, W)
    k = B5[:, None, None] * B5[None, :, None] * B5[None, None, :]
    ref = np.clip(v + 1.5 * (v - corr3_edge(v, k)), 0, 1)
    assert np.abs(run(P.unsharp3d(depth=D), [v])[0] - ref).max() < 1e-14


def heat_numpy(v, steps, a=0.125):
    for _ in range(steps):
        p = np.pad(v, 1, mode="edge")
        D, H, W = v.shape
        nb = (p[1:-1, 1:-1, :-2] + p[1:-1, 1:-1, 2:] + p[1:-1, :-2, 1:-1] + p[1:-1, 2:, 1:-1]
              + p[:-2, 1:-1, 1:-1] + p[2:, 1:-1, 1:-1])
        v = v + a * (nb - 6 * v)
    return v


@pytest.mark.parametrize("steps,shape", [(1, (4, 5, 6)), (3, (6, 5, 4)), (4, (2, 9, 3))])
def test_heat3d_against_per_step_edge_padding(steps, shape):
    """A chain of stencils clamps at every stage: numpy pads each step's
    result again."""
    v = vol(5, *shape)
    got = run(P.heat3d(steps, depth=shape[0]), [v])[0]
    assert np.abs(got - heat_numpy(v, steps)).max() < 1e-13


def test_heat3d_conserves_constants_and_mean():
    v = np.full((4, 6, 5), 0.3)
    assert np.abs(run(P.heat3d(3, depth=4), [v])[0] - 0.3).max() < 1e-15
    # zero-flux boundaries: one step keeps the sum (each face exchange cancels)
    v = vol(6, 4, 6, 5)
    assert abs(run(P.heat3d(1, depth=4), [v])[0].sum() - v.sum()) < 1e-12


def test_plane_tap_of_a_one_plane_producer_reads_plane_zero():
    b = P.Builder("z1", [1])
    inp = P.input_id(0)
    b.output(b.stage("s", P.refz(inp, 1, 0, -2) + 2.0 * P.refz(inp, 0, 1, 3), 4))
    img = vol(7, 1, 5, 6)
    got = run(b.build(), [img])[0]
    p = np.pad(img[0], 1, mode="edge")
    ref = p[1:-1, 2:] + 2 * p[2:, 1:-1]
    for z in range(4):
        assert np.abs(got[z] - ref).max() < 1e-15


def test_brute_force_recursion_matches():
    D, H, W = 4, 5, 6
    v = vol(8, D, H, W)
    spec = P.heat3d(2, depth=D)
    full = run(spec, [v])[0]
    for z, y, x in [(0, 0, 0), (3, 4, 5), (1, 2, 3), (2, 0, 5)]:
        assert abs(O.brute(spec["stages"], [v], 1, x, y, z) - full[z, y, x]) < 1e-14


def test_plane_tap_rejects_other_depths_and_modes():
    b = P.Builder("bad", [3])
    inp = P.input_id(0)
    b.output(b.stage("s", P.refz(inp, 0, 0, 1), 4))
    with pytest.raises(Exception):
        run(b.build(), [vol(9, 3, 4, 4)])


def test_point_evaluation_matches_full_volumes():
    """The region-restricted evaluator (used for sampled parity of full-size
    volumes) against the full evaluation."""
    D = 9
    v = vol(10, D, 20, 30)
    rng = np.random.default_rng(2)
    xs, ys, zs = rng.integers(0, 30, 300), rng.integers(0, 20, 300), rng.integers(0, D, 300)
    for spec in (P.unsharp3d(depth=D), P.heat3d(2, depth=D)):
        full = run(spec, [v])[0]
        pts = O.evaluate_points(spec["stages"], [v], spec["outputs"][0], xs, ys, zs)
        assert np.abs(pts - full[zs, ys, xs]).max() < 1e-15

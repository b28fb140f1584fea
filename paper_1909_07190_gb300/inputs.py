"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This module holds none of the method's arithmetic: it only draws numbers and
rounds them to a storage type.  It imports numpy only.

Generator: splitmix64 (Steele, Lea & Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014), counter-based: value i of stream `seed` is
mix(seed + (i + 1) * 0x9E3779B97F4A7C15).  A float in [0, 1) is
(u >> 40) * 2^-24, exactly representable in fp32.

Seeds: 190907190 + k for the k-th benchmark configuration (1..5).
"""
from __future__ import annotations

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
SEED_BASE = 190907190


def splitmix64(seed: int, n: int, offset: int = 0, out: np.ndarray | None = None) -> np.ndarray:
    """n consecutive outputs (uint64) of the counter-based splitmix64 stream
    (in place, in blocks that stay in cache)."""
    z = np.empty(n, np.uint64) if out is None else out[:n]
    blk = 1 << 18
    t = np.empty(min(n, blk), np.uint64)
    with np.errstate(over="ignore"):
        for s in range(0, n, blk):
            e = min(n, s + blk)
            zz, tt = z[s:e], t[:e - s]
            zz[...] = np.arange(offset + s + 1, offset + e + 1, dtype=np.uint64)
            np.multiply(zz, GOLDEN, out=zz)
            np.add(zz, np.uint64(seed), out=zz)
            np.right_shift(zz, np.uint64(30), out=tt)
            np.bitwise_xor(zz, tt, out=zz)
            np.multiply(zz, np.uint64(0xBF58476D1CE4E5B9), out=zz)
            np.right_shift(zz, np.uint64(27), out=tt)
            np.bitwise_xor(zz, tt, out=zz)
            np.multiply(zz, np.uint64(0x94D049BB133111EB), out=zz)
            np.right_shift(zz, np.uint64(31), out=tt)
            np.bitwise_xor(zz, tt, out=zz)
    return z


def uniform01(seed: int, n: int, offset: int = 0, out: np.ndarray | None = None) -> np.ndarray:
    """float32 values in [0, 1) with 24 random bits each (exact: the 24-bit
    integer converts to float32 exactly and the scale is a power of two)."""
    r = np.empty(n, np.float32) if out is None else out[:n]
    blk = 1 << 18
    u = np.empty(min(n, blk), np.uint64)
    for s in range(0, n, blk):
        e = min(n, s + blk)
        uu = splitmix64(seed, e - s, offset + s, out=u)
        np.right_shift(uu, np.uint64(40), out=uu)
        r[s:e] = uu
        np.multiply(r[s:e], np.float32(2.0 ** -24), out=r[s:e])
    return r


def uniform_image(seed: int, width: int, height: int, channels: int = 1) -> np.ndarray:
    """(channels, height, width) float32 image, uniform in [0, 1)."""
    n = width * height * channels
    return uniform01(seed, n).reshape(channels, height, width)


def uniform_ints(seed: int, n: int, lo: int, hi: int) -> np.ndarray:
    """n integers uniform in [lo, hi] (inclusive), by multiply-shift of 32 bits."""
    u = splitmix64(seed, n) >> np.uint64(32)
    span = np.uint64(hi - lo + 1)
    return (lo + ((u * span) >> np.uint64(32))).astype(np.int64)


# ------------------------------------------------------------- storage types

def to_bf16_bits(x: np.ndarray) -> np.ndarray:
    """Round float32 -> bfloat16 (round to nearest even), as uint16 bits."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = (u + np.uint64(0x7FFF) + ((u >> np.uint64(16)) & np.uint64(1))) >> np.uint64(16)
    return r.astype(np.uint16)


def bf16_bits_to_f32(b: np.ndarray) -> np.ndarray:
    return (np.asarray(b, dtype=np.uint16).astype(np.uint32) << np.uint32(16)).view(np.float32)


def round_to(x: np.ndarray, dtype: str) -> np.ndarray:
    """Value of x after storage in `dtype` ("f32", "f16", "bf16"), as float32."""
    x = np.asarray(x, dtype=np.float32)
    if dtype == "f32":
        return x
    if dtype == "f16":
        return x.astype(np.float16).astype(np.float32)
    if dtype == "bf16":
        return bf16_bits_to_f32(to_bf16_bits(x)).reshape(x.shape)
    raise ValueError(dtype)


def storage_array(x: np.ndarray, dtype: str) -> np.ndarray:
    """x encoded in `dtype`: float32, float16, or uint16 bf16 bits."""
    x = np.asarray(x, dtype=np.float32)
    if dtype == "f32":
        return np.ascontiguousarray(x)
    if dtype == "f16":
        return np.ascontiguousarray(x.astype(np.float16))
    if dtype == "bf16":
        return to_bf16_bits(x).reshape(x.shape)
    raise ValueError(dtype)


def from_storage(a: np.ndarray, dtype: str) -> np.ndarray:
    """Decodes a storage array back to float32."""
    if dtype == "f32":
        return np.asarray(a, dtype=np.float32)
    if dtype == "f16":
        return np.asarray(a, dtype=np.float16).astype(np.float32)
    if dtype == "bf16":
        return bf16_bits_to_f32(a).reshape(np.shape(a))
    raise ValueError(dtype)


# ------------------------------------------------------------ config inputs

def smooth_mask(seed: int, width: int, height: int, terms: int = 8, region=None) -> np.ndarray:
    """(1, H, W) float32 mask = sigmoid(4 f / sigma_f) of a low-frequency field
    f(x, y) = sum_m a_m cos(2 pi (u_m x / W + v_m y / H) + phi_m), with integer
    u_m, v_m in [-3, 3] (not both 0), a_m ~ N(0, 1) (Box-Muller), phi_m in
    [0, 2 pi), and sigma_f = sqrt(sum a_m^2 / 2).  Computed in float64.
    region = (x0, y0, w, h): only that window of the W x H mask (same values)."""
    u64 = splitmix64(seed, 8 * terms)
    f01 = (u64 >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    uv = (u64[: 2 * terms] % np.uint64(7)).astype(np.int64) - 3
    us, vs = uv[:terms].copy(), uv[terms:].copy()
    for m in range(terms):
        if us[m] == 0 and vs[m] == 0:
            us[m] = 1
    r1 = np.maximum(f01[2 * terms: 3 * terms], 1e-300)
    r2 = f01[3 * terms: 4 * terms]
    amp = np.sqrt(-2.0 * np.log(r1)) * np.cos(2.0 * np.pi * r2)
    phi = 2.0 * np.pi * f01[4 * terms: 5 * terms]
    sigma = np.sqrt(np.sum(amp * amp) / 2.0)
    rx0, ry0, rw, rh = region if region is not None else (0, 0, width, height)
    xs = (rx0 + np.arange(rw, dtype=np.float64)) / width
    ys = (ry0 + np.arange(rh, dtype=np.float64)) / height
    out = np.empty((rh, rw), np.float32)
    for y0 in range(0, rh, 512):
        y1 = min(rh, y0 + 512)
        f = np.zeros((y1 - y0, rw))
        for m in range(terms):
            f += amp[m] * np.cos(2.0 * np.pi * (us[m] * xs[None, :] + vs[m] * ys[y0:y1, None]) + phi[m])
        out[y0:y1] = (1.0 / (1.0 + np.exp(-4.0 * f / sigma))).astype(np.float32)
    return out[None]


def batch_sizes(seed: int, n: int = 512, lo: int = 200, hi: int = 4096):
    """(width, height) of n images, each side uniform in [lo, hi]."""
    v = uniform_ints(seed, 2 * n, lo, hi)
    return [(int(v[2 * i]), int(v[2 * i + 1])) for i in range(n)]

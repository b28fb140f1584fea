"""The seeded input generator of `inputs.py`, drawn with PyTorch on the device
for inputs too large to draw on the host (batches of gigapixels).

Same stream bit for bit: value i of stream `seed` is splitmix64's output
mix(seed + (i + 1) * 0x9E3779B97F4A7C15) (Steele, Lea & Flood, OOPSLA 2014),
and a float in [0, 1) is (u >> 40) * 2^-24.  PyTorch has no uint64, so the
64-bit words live in int64 (multiplication and addition wrap modulo 2^64
alike) and right shifts are made logical by masking.  Like `inputs.py` this
holds none of the method's arithmetic.
"""
from __future__ import annotations

import torch


def _i64(u: int) -> int:
    """The int64 with the bits of the uint64 u."""
    return u - (1 << 64) if u >= (1 << 63) else u


_GOLDEN = _i64(0x9E3779B97F4A7C15)
_M1 = _i64(0xBF58476D1CE4E5B9)
_M2 = _i64(0x94D049BB133111EB)


def _srl(z: torch.Tensor, k: int) -> torch.Tensor:
    return (z >> k) & ((1 << (64 - k)) - 1)


def splitmix64(seed: int, n: int, offset: int = 0, device="cuda") -> torch.Tensor:
    """n consecutive outputs of the stream (as int64 bit patterns)."""
    z = torch.arange(offset + 1, offset + n + 1, dtype=torch.int64, device=device)
    z.mul_(_GOLDEN).add_(_i64(seed))
    z = (z ^ _srl(z, 30)).mul_(_M1)
    z = (z ^ _srl(z, 27)).mul_(_M2)
    return z ^ _srl(z, 31)


def uniform_image(seed: int, width: int, height: int, channels: int = 1, device="cuda",
                  block: int = 1 << 24) -> torch.Tensor:
    """(channels, height, width) float32 tensor, uniform in [0, 1): equal to
    inputs.uniform_image(seed, width, height, channels)."""
    n = width * height * channels
    out = torch.empty(n, dtype=torch.float32, device=device)
    for s in range(0, n, block):
        e = min(n, s + block)
        u = splitmix64(seed, e - s, s, device)
        out[s:e] = _srl(u, 40).to(torch.float32) * (2.0 ** -24)
    return out.reshape(channels, height, width)

"""Counter-based random numbers shared by every consumer of synthetic inputs.

Philox4x32-10 is implemented from its published definition (Salmon, Moraes,
Dror & Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11, Sect. 3.2):
a 4x32-bit counter and a 2x32-bit key go through ten rounds, each round two
32x32->64 multiplications by the constants 0xD2511F53 and 0xCD9E8D57, and the
key is bumped between rounds by the Weyl constants 0x9E3779B9 / 0xBB67AE85.

Counter layout used by this project: (element_index_lo, element_index_hi,
stream_id, 0), key = (seed, 0).  Gaussian draws use the Box-Muller transform
in float64 on two 53-bit uniforms taken from one Philox output block.

This module holds no arithmetic of the sampler itself; it only produces
reproducible random numbers.
"""
from __future__ import annotations

import numpy as np

_MASK = np.uint64(0xFFFFFFFF)
_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = np.uint64(0x9E3779B9)
_W1 = np.uint64(0xBB67AE85)

# stream ids (one per independent quantity)
STREAM_SIGNAL = 0
STREAM_NOISE = 1
STREAM_W1 = 2
STREAM_W2 = 3
STREAM_HOLES = 4
STREAM_CHAINS = 5


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Ten Philox4x32 rounds on arrays of 32-bit words (held in uint64).

    Returns the four output words as uint64 arrays with values < 2**32.
    """
    c0 = np.asarray(c0, dtype=np.uint64) & _MASK
    c1 = np.asarray(c1, dtype=np.uint64) & _MASK
    c2 = np.asarray(c2, dtype=np.uint64) & _MASK
    c3 = np.asarray(c3, dtype=np.uint64) & _MASK
    k0 = np.asarray(k0, dtype=np.uint64) & _MASK
    k1 = np.asarray(k1, dtype=np.uint64) & _MASK
    for rnd in range(10):
        if rnd:
            k0 = (k0 + _W0) & _MASK
            k1 = (k1 + _W1) & _MASK
        p0 = _M0 * c0
        p1 = _M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK
        c0, c1, c2, c3 = (hi1 ^ c1 ^ k0), lo1, (hi0 ^ c3 ^ k1), lo0
    return c0, c1, c2, c3


def _u53(a, b):
    """Two 32-bit words -> float64 uniform in the open interval (0, 1)."""
    hi = (a >> np.uint64(5)).astype(np.float64)   # 27 bits
    lo = (b >> np.uint64(6)).astype(np.float64)   # 26 bits
    return (hi * 67108864.0 + lo + 0.5) * (1.0 / 9007199254740992.0)


def _block(seed: int, stream: int, idx):
    idx = np.asarray(idx, dtype=np.uint64)
    return philox4x32_10(idx & _MASK, idx >> np.uint64(32),
                         np.full(idx.shape, stream, np.uint64),
                         np.zeros(idx.shape, np.uint64),
                         np.full(idx.shape, seed, np.uint64),
                         np.zeros(idx.shape, np.uint64))


def uniform(seed: int, stream: int, n: int, offset: int = 0) -> np.ndarray:
    """n uniforms in (0, 1); element e uses counter index offset + e."""
    x0, x1, _, _ = _block(seed, stream, np.arange(offset, offset + n, dtype=np.uint64))
    return _u53(x0, x1)


def normal(seed: int, stream: int, n: int, offset: int = 0) -> np.ndarray:
    """n standard normals; element e uses counter (offset+e)//2 and takes the
    cosine (even e) or sine (odd e) branch of Box-Muller."""
    e = np.arange(offset, offset + n, dtype=np.uint64)
    x0, x1, x2, x3 = _block(seed, stream, e >> np.uint64(1))
    u1 = _u53(x0, x1)
    u2 = _u53(x2, x3)
    r = np.sqrt(-2.0 * np.log(u1))
    ang = 2.0 * np.pi * u2
    odd = (e & np.uint64(1)).astype(bool)
    return np.where(odd, r * np.sin(ang), r * np.cos(ang))


# ---------------------------------------------------------------- torch path
# The same generator on a torch device (int64 arithmetic with 32-bit masks;
# products of two 32-bit words wrap modulo 2^64, which keeps the low and high
# words exact).  Gaussian draws use the device's float64 log / cos / sin, so
# they agree with the numpy path to rounding, not bit for bit; the benchmark
# uses this path for full-size inputs, the parity tests use the numpy path.
def _philox_torch(c0, c1, c2, c3, k0: int, k1: int):
    M = 0xFFFFFFFF
    for rnd in range(10):
        if rnd:
            k0 = (k0 + 0x9E3779B9) & M
            k1 = (k1 + 0xBB67AE85) & M
        p0 = c0 * 0xD2511F53
        p1 = c2 * 0xCD9E8D57
        hi0, lo0 = (p0 >> 32) & M, p0 & M
        hi1, lo1 = (p1 >> 32) & M, p1 & M
        c0, c1, c2, c3 = (hi1 ^ c1 ^ k0), lo1, (hi0 ^ c3 ^ k1), lo0
    return c0, c1, c2, c3


def normal_torch(seed: int, stream: int, n: int, offset: int = 0, device="cuda"):
    import torch
    e = torch.arange(offset, offset + n, dtype=torch.int64, device=device)
    idx = e >> 1
    z = torch.zeros_like(idx)
    x0, x1, x2, x3 = _philox_torch(idx & 0xFFFFFFFF, idx >> 32, z + stream, z, seed, 0)

    def u53(a, b):
        return ((a >> 5).double() * 67108864.0 + (b >> 6).double() + 0.5) * (1.0 / 9007199254740992.0)
    u1, u2 = u53(x0, x1), u53(x2, x3)
    r = torch.sqrt(-2.0 * torch.log(u1))
    ang = 2.0 * 3.141592653589793 * u2
    return torch.where((e & 1).bool(), r * torch.sin(ang), r * torch.cos(ang))

"""Shared helpers for the test-suite (no sampler arithmetic)."""
import numpy as np


def rel_l2(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def rand_alm(L, rng, lead=(), scale=None):
    """Random complex alm with real m = 0 entries; optional per-l scale."""
    P = (L + 1) * (L + 2) // 2
    a = rng.normal(size=lead + (P,)) + 1j * rng.normal(size=lead + (P,))
    ms = np.concatenate([np.full(L + 1 - m, m) for m in range(L + 1)])
    a[..., ms == 0] = a[..., ms == 0].real
    if scale is not None:
        ls = np.concatenate([np.arange(m, L + 1) for m in range(L + 1)])
        a = a * scale[ls]
    return a


def gpu():
    import torch
    return torch.device("cuda", 0)

"""Seeded input generators: Philox known answers, distributions, recipes."""
import math
import os

import numpy as np

from inputs import configs as C
from inputs import philox as px

GOLD = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def test_philox_known_answers():
    rows = [l.split() for l in open(GOLD) if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = px.philox4x32_10(*v[:6])
        assert [int(o) for o in out] == v[6:]


def test_normal_moments():
    z = px.normal(7, 3, 200_000)
    assert abs(z.mean()) < 0.01
    assert abs(z.var() - 1.0) < 0.01
    # element e is independent of how many are drawn
    assert np.array_equal(px.normal(7, 3, 10, offset=5), z[5:15])


def test_white_alm_metric_variance():
    # unit white noise in the metric sum_l [a_l0^2 + 2 sum_{m>0} |a_lm|^2]:
    # Var(a_l0) = 1, E|a_lm|^2 = 1 for m > 0 (re and im each 1/2)
    L = 200
    a = C.white_alm(L, 11, px.STREAM_W1)
    _, ms = C.alm_lm(L)
    assert np.all(a[ms == 0].imag == 0)
    assert abs(np.mean(a[ms == 0].real ** 2) - 1) < 0.15
    assert abs(np.mean(np.abs(a[ms > 0]) ** 2) - 1) < 0.02


def test_pixel_centres_counts():
    for ns in (1, 2, 4, 16):
        z, phi = C.pixel_centres(ns)
        assert z.size == 12 * ns * ns
        assert np.all(np.diff(z) <= 0)
        # equal-area pixels: mean z over the sphere is 0
        assert abs(z.mean()) < 1e-12
        assert np.all((phi >= 0) & (phi < 2 * math.pi))


def test_config_shapes_small():
    p = C.masked_temperature(16, 32)
    assert p.ninv.shape == (12 * 16 * 16,)
    fsky = p.extra["fsky"]
    assert 0.55 < fsky < 0.70          # |b| < 20 deg removes sin(20 deg) = 34 %
    p4 = C.teb_realizations(2, 8, 16)
    assert len(p4) == 2 and p4[0].signal_alm.shape == (3, C.nalm(16))
    assert p4[0].ninv.shape == (2, 12 * 64)
    ch = C.mixed_geometry_chains(4, 8, 16)
    assert len(ch) == 4

"""Pins for the oracle's geometry and Legendre functions (no GPU).

Each check compares against something other than the oracle itself:
closed forms, scipy, sympy, numpy's Gauss-Legendre rule, identities."""
import math

import numpy as np
import pytest

from inputs import configs as C
from oracle import sht

FOURPI = 4.0 * math.pi


# --------------------------------------------------------------------- geometry
@pytest.mark.parametrize("nside", [1, 2, 4, 32, 1024])
def test_healpix_rings(nside):
    g = sht.healpix(nside)
    assert g.nring == 4 * nside - 1
    assert g.npix == 12 * nside * nside
    # mirror symmetry z_{4N-i} = -z_i with equal nphi and phi0
    assert np.allclose(g.cth, -g.cth[::-1], atol=1e-15)
    assert np.array_equal(g.nphi, g.nphi[::-1])
    assert np.allclose(g.phi0, g.phi0[::-1], atol=0)
    assert np.allclose(g.cth ** 2 + g.sth ** 2, 1.0, atol=1e-15)
    # polar formula at i = N meets the equatorial one at z = 2/3
    n = nside
    assert abs((1 - n * n / (3.0 * n * n)) - 2.0 / 3.0) < 1e-15
    assert abs(g.cth[n - 1] - 2.0 / 3.0) < 1e-15
    # offsets are the running sum of ring lengths
    assert np.array_equal(g.ofs[1:], np.cumsum(g.nphi)[:-1])


@pytest.mark.parametrize("nside", [1, 4, 16])
def test_healpix_pixel_centres_independent(nside):
    """Ring z, phi0 against the independent pixel-centre routine of the
    input generator (Gorski et al. 2005 pix2ang in RING order)."""
    g = sht.healpix(nside)
    z, phi = C.pixel_centres(nside)
    assert np.allclose(np.repeat(g.cth, g.nphi), z, atol=1e-15)
    first = phi[g.ofs]
    assert np.allclose(first, g.phi0, atol=1e-15)


@pytest.mark.parametrize("n", [1, 2, 7, 33, 128, 513])
def test_gauss_legendre_vs_numpy(n):
    g = sht.gauss_legendre(n, 4)
    x, w = np.polynomial.legendre.leggauss(n)
    assert np.allclose(g.cth, x[::-1], atol=1e-14)
    assert np.allclose(g.wring * 4 / (2 * math.pi), w[::-1], rtol=1e-12)


# --------------------------------------------------------------------- spin 0
def _closed_forms(l, m, th):
    c, s = math.cos(th), math.sin(th)
    table = {
        (0, 0): 0.5 * math.sqrt(1 / math.pi),
        (1, 0): 0.5 * math.sqrt(3 / math.pi) * c,
        (1, 1): -0.5 * math.sqrt(3 / (2 * math.pi)) * s,
        (2, 0): 0.25 * math.sqrt(5 / math.pi) * (3 * c * c - 1),
        (2, 1): -0.5 * math.sqrt(15 / (2 * math.pi)) * s * c,
        (2, 2): 0.25 * math.sqrt(15 / (2 * math.pi)) * s * s,
        (3, 0): 0.25 * math.sqrt(7 / math.pi) * (5 * c ** 3 - 3 * c),
        (3, 1): -0.125 * math.sqrt(21 / math.pi) * s * (5 * c * c - 1),
        (3, 2): 0.25 * math.sqrt(105 / (2 * math.pi)) * s * s * c,
        (3, 3): -0.125 * math.sqrt(35 / math.pi) * s ** 3,
    }
    return table[(l, m)]


@pytest.mark.parametrize("th", [0.01, 0.4, 1.2, math.pi / 2, 2.5, 3.13])
def test_lambda_closed_forms(th):
    for m in range(4):
        lam = sht.lambda_lm(3, m, math.cos(th), math.sin(th))
        for l in range(m, 4):
            assert abs(lam[l - m] - _closed_forms(l, m, th)) < 1e-15


@pytest.mark.parametrize("th", [0.05, 0.7, 1.5707963, 2.9])
def test_lambda_vs_scipy(th):
    from scipy.special import sph_harm_y
    L = 150
    for m in (0, 1, 2, 17, 64, 150):
        lam = sht.lambda_lm(L, m, math.cos(th), math.sin(th))
        ref = np.array([sph_harm_y(l, m, th, 0.0).real for l in range(m, L + 1)])
        assert np.max(np.abs(lam - ref)) < 1e-12


@pytest.mark.parametrize("ring", [0, 1, 700, 2047])
def test_addition_theorem_l2048(ring):
    """lambda_l0^2 + 2 sum_{m>0} lambda_lm^2 = (2l+1)/4pi at every l <= 2048
    on HEALPix N_side = 1024 rings (including the polar ring)."""
    g = sht.healpix(1024)
    L = 2048
    # the identity needs x^2 + s^2 = 1 to the last bit: near the pole P_l(x)
    # amplifies an inconsistency dx by ~l^2/2, so s is taken from the rounded x
    x = g.cth[ring]
    s = math.sqrt((1.0 - x) * (1.0 + x))
    acc = np.zeros(L + 1)
    for m in range(L + 1):
        lam = sht.lambda_lm(L, m, x, s)
        acc[m:] += (1.0 if m == 0 else 2.0) * lam ** 2
    l = np.arange(L + 1)
    assert np.max(np.abs(acc / ((2 * l + 1) / FOURPI) - 1)) < 2e-11


def test_lambda_parity():
    th = 0.83
    for m in (0, 3, 10):
        a = sht.lambda_lm(60, m, math.cos(th), math.sin(th))
        b = sht.lambda_lm(60, m, -math.cos(th), math.sin(th))
        l = np.arange(m, 61)
        assert np.allclose(b, (-1.0) ** (l + m) * a, atol=1e-15, rtol=0)


def test_lambda_deep_underflow_region():
    """Large m near the pole: the sectoral seed is ~1e-6000 but lambda at
    large l must still match the addition-theorem budget (no lost growth)."""
    th = 0.02
    L = 2048
    acc = np.zeros(L + 1)
    for m in range(L + 1):
        lam = sht.lambda_lm(L, m, math.cos(th), math.sin(th))
        acc[m:] += (1.0 if m == 0 else 2.0) * lam ** 2
    l = np.arange(L + 1)
    assert np.max(np.abs(acc / ((2 * l + 1) / FOURPI) - 1)) < 2e-11


# --------------------------------------------------------------------- spin 2
def _sympy_spin2(lmax):
    """2Y_lm and -2Y_lm from sympy: sqrt((l-2)!/(l+2)!) edth^2 Y_lm with
    edth eta = -(sin t)^s (d_t + i/sin t d_p) (sin t)^-s eta (spin s) and the
    conjugate operator for the lowering direction."""
    import sympy as sp
    t, p = sp.symbols("t p", real=True)

    def edth(f, s):
        return sp.simplify(-(sp.sin(t) ** s) * (sp.diff(sp.sin(t) ** (-s) * f, t)
                                                 + sp.I / sp.sin(t) * sp.diff(sp.sin(t) ** (-s) * f, p)))

    def edthb(f, s):
        return sp.simplify(-(sp.sin(t) ** (-s)) * (sp.diff(sp.sin(t) ** s * f, t)
                                                    - sp.I / sp.sin(t) * sp.diff(sp.sin(t) ** s * f, p)))
    out = {}
    for l in range(2, lmax + 1):
        for m in range(0, l + 1):
            Y = sp.Ynm(l, m, t, p).expand(func=True)
            nrm = sp.sqrt(sp.factorial(l - 2) / sp.factorial(l + 2))
            y2 = nrm * edth(edth(Y, 0), 1)
            ym2 = nrm * edthb(edthb(Y, 0), -1)
            out[(l, m)] = (sp.lambdify(t, sp.simplify(y2 * sp.exp(-sp.I * m * p))),
                           sp.lambdify(t, sp.simplify(ym2 * sp.exp(-sp.I * m * p))))
    return out


def test_spin2_vs_sympy_edth():
    fns = _sympy_spin2(4)
    for th in (0.3, 1.1, 2.0, 2.8):
        for m in range(0, 5):
            lw, lx = sht.lambda_spin2(4, m, math.cos(th), math.sin(th))
            for l in range(max(2, m), 5):
                f2, fm2 = fns[(l, m)]
                s2 = complex(f2(th)).real
                sm2 = complex(fm2(th)).real
                assert abs((lw[l - m] + lx[l - m]) - s2) < 1e-13, (l, m, th)
                assert abs((lw[l - m] - lx[l - m]) - sm2) < 1e-13, (l, m, th)


def test_spin0_vs_sympy_ynm():
    import sympy as sp
    t = sp.symbols("t", real=True)
    for l in range(0, 5):
        for m in range(0, l + 1):
            f = sp.lambdify(t, sp.Ynm(l, m, t, 0).expand(func=True))
            for th in (0.3, 2.2):
                lam = sht.lambda_lm(4, m, math.cos(th), math.sin(th))
                assert abs(lam[l - m] - complex(f(th)).real) < 1e-14


@pytest.mark.parametrize("th", [0.004, 0.5, 1.4, 2.7])
def test_spin2_addition_theorem(th):
    """sum_{m=-l..l} |2Y_lm|^2 = (2l+1)/4pi, i.e. lw_l0^2 + 2 sum_{m>0}
    (lw^2 + lx^2) = (2l+1)/4pi for l >= 2."""
    L = 600
    acc = np.zeros(L + 1)
    for m in range(L + 1):
        lw, lx = sht.lambda_spin2(L, m, math.cos(th), math.sin(th))
        acc[m:] += (1.0 if m == 0 else 2.0) * (lw ** 2 + lx ** 2) if m else lw ** 2
    l = np.arange(2, L + 1)
    assert np.max(np.abs(acc[2:] / ((2 * l + 1) / FOURPI) - 1)) < 1e-9


def test_spin2_parity():
    th = 0.91
    for m in (0, 1, 4, 9):
        w1, x1 = sht.lambda_spin2(40, m, math.cos(th), math.sin(th))
        w2, x2 = sht.lambda_spin2(40, m, -math.cos(th), math.sin(th))
        l = np.arange(m, 41)
        p = (-1.0) ** (l + m)
        assert np.allclose(w2, p * w1, atol=1e-14, rtol=0)
        assert np.allclose(x2, -p * x1, atol=1e-14, rtol=0)

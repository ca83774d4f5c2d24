"""Pins for the oracle transforms (no GPU): single modes against closed
forms on independent pixel centres, exact Gauss-Legendre round trips, dense
scipy synthesis, adjointness."""
import math

import numpy as np
import pytest

from inputs import configs as C
from oracle import sht


def _rand_alm(L, rng):
    P = (L + 1) * (L + 2) // 2
    a = rng.normal(size=P) + 1j * rng.normal(size=P)
    ms = sht.ms_of(L)
    a[ms == 0] = a[ms == 0].real
    return a


@pytest.mark.parametrize("nside", [2, 8])
def test_single_mode_vs_scipy_pixels(nside):
    """alm2map of one a_lm = u (m > 0) is 2 Re(u Y_lm) at every pixel centre,
    with Y_lm from scipy and the centres from the input generator."""
    from scipy.special import sph_harm_y
    L = 2 * nside
    g = sht.healpix(nside)
    z, phi = C.pixel_centres(nside)
    th = np.arccos(z)
    for (l, m, u) in [(0, 0, 1.0), (3, 0, 1.0), (L - 1, 2, 0.3 - 0.7j), (L, L, 1j), (L, 1, 1.0)]:
        a = np.zeros((L + 1) * (L + 2) // 2, complex)
        a[m * (2 * L + 1 - m) // 2 + l] = u
        mp = sht.alm2map(g, L, a)
        Y = sph_harm_y(l, m, th, phi)
        ref = (u * Y).real if m == 0 else 2.0 * (u * Y).real
        assert np.max(np.abs(mp - ref)) < 1e-13


def test_dense_synthesis_vs_scipy():
    from scipy.special import sph_harm_y
    nside, L = 4, 9
    g = sht.healpix(nside)
    z, phi = C.pixel_centres(nside)
    th = np.arccos(z)
    a = _rand_alm(L, np.random.default_rng(3))
    ref = np.zeros(g.npix)
    for m in range(L + 1):
        for l in range(m, L + 1):
            y = (a[m * (2 * L + 1 - m) // 2 + l] * sph_harm_y(l, m, th, phi)).real
            ref += y if m == 0 else 2 * y
    assert np.max(np.abs(sht.alm2map(g, L, a) - ref)) < 1e-12


@pytest.mark.parametrize("L", [8, 31, 64])
def test_gl_round_trip_exact(L):
    """map2alm(alm2map(a)) = a on a Gauss-Legendre grid with L+1 rings and
    nphi >= 2L+1 (exact quadrature), spin 0 and spin 2."""
    g = sht.gauss_legendre(L + 1, 2 * L + 2)
    rng = np.random.default_rng(L)
    a = _rand_alm(L, rng)
    b = sht.map2alm(g, L, sht.alm2map(g, L, a))
    assert np.max(np.abs(b - a)) / np.max(np.abs(a)) < 1e-12
    E, B = _rand_alm(L, rng), _rand_alm(L, rng)
    ls = sht.ls_of(L)
    E[ls < 2] = 0
    B[ls < 2] = 0
    Q, U = sht.alm2map_spin2(g, L, E, B)
    w = g.pixel_weights()
    E2, B2 = sht.alm2map_spin2_adjoint(g, L, w * Q, w * U)
    assert np.max(np.abs(E2 - E)) / np.max(np.abs(E)) < 1e-12
    assert np.max(np.abs(B2 - B)) / np.max(np.abs(B)) < 1e-12


@pytest.mark.parametrize("geom", ["healpix", "gl"])
def test_adjoint_identity(geom):
    rng = np.random.default_rng(5)
    if geom == "healpix":
        g, L = sht.healpix(16), 40
    else:
        g, L = sht.gauss_legendre(30, 64), 40
    a = _rand_alm(L, rng)
    mp = rng.normal(size=g.npix)
    lhs = np.dot(sht.alm2map(g, L, a), mp)
    rhs = sht.dot_q6(a, sht.alm2map_adjoint(g, L, mp), L)
    assert abs(lhs - rhs) < 1e-13 * abs(lhs) * 10
    E, B = _rand_alm(L, rng), _rand_alm(L, rng)
    Q, U = sht.alm2map_spin2(g, L, E, B)
    q, u = rng.normal(size=g.npix), rng.normal(size=g.npix)
    E2, B2 = sht.alm2map_spin2_adjoint(g, L, q, u)
    lhs = Q @ q + U @ u
    rhs = sht.dot_q6(E, E2, L) + sht.dot_q6(B, B2, L)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_adjoint_mlist_subset():
    g, L = sht.healpix(8), 16
    mp = np.random.default_rng(1).normal(size=g.npix)
    full = sht.alm2map_adjoint(g, L, mp)
    sub = sht.alm2map_adjoint(g, L, mp, mlist=[0, 5, 16])
    ms = sht.ms_of(L)
    sel = np.isin(ms, [0, 5, 16])
    assert np.array_equal(full[sel], sub[sel])


def test_spin2_adjoint_mlist_subset():
    """The spin-2 adjoint restricted to a list of m equals the full spin-2
    adjoint (itself pinned by the adjoint identity) at those m."""
    g, L = sht.healpix(8), 16
    rng = np.random.default_rng(2)
    Q, U = rng.normal(size=g.npix), rng.normal(size=g.npix)
    E, B = sht.alm2map_spin2_adjoint(g, L, Q, U)
    Es, Bs = sht.alm2map_spin2_adjoint(g, L, Q, U, mlist=[0, 2, 9, 16])
    sel = np.isin(sht.ms_of(L), [0, 2, 9, 16])
    assert np.array_equal(E[sel], Es[sel]) and np.array_equal(B[sel], Bs[sel])
    assert np.abs(E[sel]).max() > 0 and np.abs(B[sel]).max() > 0


def test_spin2_pure_modes_closed_form():
    """E_22 = 1, B = 0 against the closed forms 2Y_22 = k (1 - cos t)^2 e^{2ip}
    and -2Y_22 = k (1 + cos t)^2 e^{2ip}, k = sqrt(5 / 64 pi), with
    +-2a = -(E +- iB) and the m = -2 terms from sY_l,-m = (-1)^(m+s) conj(-sY_lm)."""
    nside, L = 8, 8
    g = sht.healpix(nside)
    z, phi = C.pixel_centres(nside)
    E = np.zeros((L + 1) * (L + 2) // 2, complex)
    B = np.zeros_like(E)
    E[2 * (2 * L + 1 - 2) // 2 + 2] = 1.0
    Q, U = sht.alm2map_spin2(g, L, E, B)
    k = math.sqrt(5.0 / (64.0 * math.pi))
    y2 = k * (1 - z) ** 2 * np.exp(2j * phi)        # 2Y_22
    ym2 = k * (1 + z) ** 2 * np.exp(2j * phi)       # -2Y_22
    # 2a_22 = -1, -2a_22 = -1; m = -2 terms: 2Y_2,-2 = conj(-2Y_22) (s=2, m=2:
    # sY_l,-m = (-1)^(m+s) conj(-sY_lm)), E_2,-2 = E_22^* = 1 so 2a_2,-2 = -1
    qpiu = -(y2 + np.conj(ym2))
    qmiu = -(ym2 + np.conj(y2))
    Qref = 0.5 * (qpiu + qmiu)
    Uref = (qpiu - qmiu) / 2j
    assert np.max(np.abs(Q - Qref.real)) < 1e-14
    assert np.max(np.abs(U - Uref.real)) < 1e-14
    assert np.max(np.abs(Qref.imag)) < 1e-14 and np.max(np.abs(Uref.imag)) < 1e-14


def test_map2alm_jacobi_refinement_converges():
    """On HEALPix the quadrature analysis of a band-limited map is only
    approximate; each Jacobi refinement alm += Y^T W (map - Y alm) must
    shrink the error towards the true alm (here by > 5x per step), and on an
    exact Gauss-Legendre grid the refinements keep the exact result."""
    g, L = sht.healpix(16), 24
    rng = np.random.default_rng(7)
    a = _rand_alm(L, rng)
    m = sht.alm2map(g, L, a)
    errs = [np.linalg.norm(sht.map2alm(g, L, m, niter=n) - a) / np.linalg.norm(a) for n in range(4)]
    assert errs[0] < 0.05
    for e0, e1 in zip(errs, errs[1:]):
        assert e1 < e0 / 5
    gl = sht.gauss_legendre(L + 1, 2 * L + 2)
    mg = sht.alm2map(gl, L, a)
    for n in (0, 2):
        assert np.linalg.norm(sht.map2alm(gl, L, mg, niter=n) - a) < 1e-12 * np.linalg.norm(a)

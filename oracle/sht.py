"""Oracle spherical harmonic transforms (FP64, CPU), wrapping oracle.c.

Test infrastructure only.  Y is the synthesis alm -> map of a real field,
Y^T its transpose in the metric <a, c> = sum_l [a_l0 c_l0 + 2 Re sum_{m>0}
conj(a_lm) c_lm] (the metric in which the constrained-realization operator of
Eq. (mapmakingeq) is symmetric for alm stored with m >= 0 only).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from ._lib import lib


@dataclass
class Geometry:
    cth: np.ndarray
    sth: np.ndarray
    nphi: np.ndarray     # int64
    phi0: np.ndarray
    ofs: np.ndarray      # int64
    wring: np.ndarray    # quadrature weight of one pixel on each ring
    kind: str = "healpix"
    nside: int = 0

    @property
    def nring(self) -> int:
        return int(self.cth.size)

    @property
    def npix(self) -> int:
        return int(self.nphi.sum())

    def pixel_weights(self) -> np.ndarray:
        return np.repeat(self.wring, self.nphi)

    def subset(self, rings) -> "Geometry":
        """Geometry restricted to the given rings (pixels packed contiguously)."""
        rings = np.asarray(rings, dtype=np.int64)
        nphi = self.nphi[rings].copy()
        ofs = np.concatenate([[0], np.cumsum(nphi)[:-1]]).astype(np.int64)
        return Geometry(self.cth[rings].copy(), self.sth[rings].copy(), nphi,
                        self.phi0[rings].copy(), ofs, self.wring[rings].copy(), self.kind,
                        self.nside)


def healpix(nside: int) -> Geometry:
    n = 4 * nside - 1
    cth, sth, phi0 = np.zeros(n), np.zeros(n), np.zeros(n)
    nphi, ofs = np.zeros(n, np.int64), np.zeros(n, np.int64)
    lib().orc_healpix_geom(nside, cth, sth, nphi, phi0, ofs)
    w = np.full(n, 4.0 * np.pi / (12.0 * nside * nside))
    return Geometry(cth, sth, nphi, phi0, ofs, w, "healpix", nside)


def gauss_legendre(nring: int, nphi: int) -> Geometry:
    """Gauss-Legendre rings with nphi equally spaced pixels each, phi0 = 0.
    The pixel quadrature weight is w_k * 2 pi / nphi."""
    cth, sth, w = np.zeros(nring), np.zeros(nring), np.zeros(nring)
    lib().orc_gl_geom(nring, cth, sth, w)
    nph = np.full(nring, nphi, np.int64)
    ofs = (np.arange(nring, dtype=np.int64) * nphi).astype(np.int64)
    return Geometry(cth, sth, nph, np.zeros(nring), ofs, w * 2.0 * np.pi / nphi, "gl", 0)


def lambda_lm(lmax: int, m: int, cth: float, sth: float) -> np.ndarray:
    out = np.zeros(lmax - m + 1)
    lib().orc_lambda(lmax, m, float(cth), float(sth), out)
    return out


def lambda_spin2(lmax: int, m: int, cth: float, sth: float):
    lw = np.zeros(lmax - m + 1)
    lx = np.zeros(lmax - m + 1)
    lib().orc_lambda_spin2(lmax, m, float(cth), float(sth), lw, lx)
    return lw, lx


def _geo(g: Geometry, lmax: int):
    return (g.nring, g.cth, g.sth, g.nphi, g.phi0, g.ofs, lmax)


def _c2r(a):
    return np.ascontiguousarray(np.asarray(a, np.complex128)).view(np.float64)


def alm2map(g: Geometry, lmax: int, alm: np.ndarray) -> np.ndarray:
    out = np.zeros(g.npix)
    lib().orc_alm2map(*_geo(g, lmax), _c2r(alm), out)
    return out


def alm2map_adjoint(g: Geometry, lmax: int, m: np.ndarray, mlist=None) -> np.ndarray:
    nalm = (lmax + 1) * (lmax + 2) // 2
    out = np.zeros(2 * nalm)
    mp = np.ascontiguousarray(m, np.float64)
    if mlist is None:
        lib().orc_alm2map_adjoint(*_geo(g, lmax), mp, out)
    else:
        ml = np.ascontiguousarray(mlist, np.int32)
        lib().orc_alm2map_adjoint_m(*_geo(g, lmax), mp, out, int(ml.size),
                                     ml.ctypes.data)
    return out.view(np.complex128)


def alm2map_spin2(g: Geometry, lmax: int, E: np.ndarray, B: np.ndarray):
    Q, U = np.zeros(g.npix), np.zeros(g.npix)
    lib().orc_alm2map_spin2(*_geo(g, lmax), _c2r(E), _c2r(B), Q, U)
    return Q, U


def alm2map_spin2_adjoint(g: Geometry, lmax: int, Q, U, mlist=None):
    nalm = (lmax + 1) * (lmax + 2) // 2
    E, B = np.zeros(2 * nalm), np.zeros(2 * nalm)
    q = np.ascontiguousarray(Q, np.float64)
    u = np.ascontiguousarray(U, np.float64)
    if mlist is None:
        lib().orc_alm2map_spin2_adjoint_m(*_geo(g, lmax), q, u, E, B, -1, None)
    else:
        ml = np.ascontiguousarray(mlist, np.int32)
        lib().orc_alm2map_spin2_adjoint_m(*_geo(g, lmax), q, u, E, B, int(ml.size),
                                           ml.ctypes.data)
    return E.view(np.complex128), B.view(np.complex128)


def map2alm(g: Geometry, lmax: int, m: np.ndarray, niter: int = 0) -> np.ndarray:
    """Quadrature analysis Y^T W map plus ``niter`` Jacobi refinements
    alm += Y^T W (map - Y alm).  Exact on a Gauss-Legendre grid with
    nring >= lmax+1 and nphi >= 2 lmax + 1."""
    w = g.pixel_weights()
    alm = alm2map_adjoint(g, lmax, w * m)
    for _ in range(niter):
        alm = alm + alm2map_adjoint(g, lmax, w * (m - alm2map(g, lmax, alm)))
    return alm


def diag_ringsum(g: Geometry, lmax: int, wring: np.ndarray, spin: int = 0) -> np.ndarray:
    nalm = (lmax + 1) * (lmax + 2) // 2
    out = np.zeros(nalm)
    lib().orc_diag_ringsum(g.nring, g.cth, g.sth, lmax, spin,
                           np.ascontiguousarray(wring, np.float64), out)
    return out


def ring_sums(g: Geometry, pixvals: np.ndarray) -> np.ndarray:
    """sum over the pixels of each ring."""
    return np.add.reduceat(np.asarray(pixvals, np.float64), g.ofs) if g.nring else np.zeros(0)


def ms_of(lmax: int) -> np.ndarray:
    return np.concatenate([np.full(lmax + 1 - m, m) for m in range(lmax + 1)])


def ls_of(lmax: int) -> np.ndarray:
    return np.concatenate([np.arange(m, lmax + 1) for m in range(lmax + 1)])


def dot_q6(a: np.ndarray, c: np.ndarray, lmax: int) -> float:
    """sum_l [a_l0 c_l0 + 2 Re sum_{m>0} conj(a_lm) c_lm] (last axis = alm)."""
    w = np.where(ms_of(lmax) == 0, 1.0, 2.0)
    return float(np.sum(w * np.real(np.conj(a) * c)))

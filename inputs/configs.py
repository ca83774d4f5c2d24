"""Seeded synthetic inputs shaped like the paper's workloads.

The paper's simulations use Planck LFI 70 GHz beams, rms maps and masks
(Sect. 3) that are not available here.  These recipes stand in for them with
closed-form spectra, Gaussian beams, a latitude cut plus point-source holes
and a smooth scan-depth ("hits") pattern.  Everything is drawn from the
Philox streams in :mod:`inputs.philox`, so any consumer regenerates identical
inputs from the same seed.

This module computes inputs only: power spectra, beams, masks, noise levels
and white-noise draws.  It contains none of the sampler's arithmetic (no
spherical harmonic transform, no solver).  The data map d = Y B a + n needs a
transform, so callers assemble it with their own alm2map from ``signal_alm``
and ``noise_map`` returned here.

Layouts: alm arrays are complex128, m-major, index(l, m) = m(2L+1-m)/2 + l
for 0 <= m <= l <= L; maps are float64 in HEALPix RING order.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from . import philox as px

ARCMIN = math.pi / (180.0 * 60.0)
DEG = math.pi / 180.0
# North ecliptic pole in Galactic coordinates (l, b), degrees.
NEP_GAL_DEG = (96.38, 29.81)


# ----------------------------------------------------------------------------
# index helpers
# ----------------------------------------------------------------------------
def nalm(lmax: int) -> int:
    return (lmax + 1) * (lmax + 2) // 2


def alm_index(l, m, lmax: int):
    return m * (2 * lmax + 1 - m) // 2 + l


def alm_lm(lmax: int):
    """(l, m) integer arrays in storage order."""
    ls, ms = [], []
    for m in range(lmax + 1):
        ls.append(np.arange(m, lmax + 1))
        ms.append(np.full(lmax + 1 - m, m))
    return np.concatenate(ls), np.concatenate(ms)


# ----------------------------------------------------------------------------
# spectra and beams
# ----------------------------------------------------------------------------
def cl_flat(lmax: int, amp: float = 1000.0) -> np.ndarray:
    """C_l = 2 pi amp / (l (l+1)) uK^2 for l >= 2, C_0 = C_1 = 0."""
    l = np.arange(lmax + 1, dtype=np.float64)
    cl = np.zeros(lmax + 1)
    cl[2:] = 2.0 * math.pi * amp / (l[2:] * (l[2:] + 1.0))
    return cl


def cl_damped(lmax: int, lcut: float = 1500.0) -> np.ndarray:
    l = np.arange(lmax + 1, dtype=np.float64)
    return cl_flat(lmax) * np.exp(-l * (l + 1.0) / lcut ** 2)


def gauss_beam(lmax: int, fwhm_rad: float) -> np.ndarray:
    """b_l = exp(-l(l+1) sigma_b^2 / 2), sigma_b = FWHM / sqrt(8 ln 2)."""
    sig = fwhm_rad / math.sqrt(8.0 * math.log(2.0))
    l = np.arange(lmax + 1, dtype=np.float64)
    return np.exp(-0.5 * l * (l + 1.0) * sig * sig)


# ----------------------------------------------------------------------------
# HEALPix pixel centres (used here only to draw masks and noise levels)
# ----------------------------------------------------------------------------
def pixel_centres(nside: int):
    """(z, phi) of every pixel centre in RING order (Gorski et al. 2005)."""
    zs, phis = [], []
    n = nside
    for i in range(1, 4 * n):
        if i < n:
            npr, z, shift = 4 * i, 1.0 - i * i / (3.0 * n * n), 1.0
        elif i <= 3 * n:
            npr, z = 4 * n, 4.0 / 3.0 - 2.0 * i / (3.0 * n)
            shift = 1.0 if (i - n) % 2 == 0 else 0.0
        else:
            ii = 4 * n - i
            npr, z, shift = 4 * ii, -(1.0 - ii * ii / (3.0 * n * n)), 1.0
        j = np.arange(npr, dtype=np.float64)
        zs.append(np.full(npr, z))
        phis.append((j + 0.5 * shift) * (2.0 * math.pi / npr))
    return np.concatenate(zs), np.concatenate(phis)


def _unit(z, phi):
    s = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    return np.stack([s * np.cos(phi), s * np.sin(phi), z], axis=-1)


def latitude_cut(z, bcut_deg: float) -> np.ndarray:
    """True where the pixel is masked: |b| < bcut (b = Galactic latitude)."""
    return np.abs(z) < math.sin(bcut_deg * DEG)


def point_source_holes(z, phi, nholes: int, radius_deg: float, seed: int) -> np.ndarray:
    """True inside any of ``nholes`` discs of the given radius whose centres are
    uniform on the sphere (Philox stream 4); a pixel is inside if its centre is."""
    if nholes == 0:
        return np.zeros(z.shape, bool)
    u = px.uniform(seed, px.STREAM_HOLES, 2 * nholes)
    zc = 2.0 * u[0::2] - 1.0
    pc = 2.0 * math.pi * u[1::2]
    vc = _unit(zc, pc)
    cosr = math.cos(radius_deg * DEG)
    rad = radius_deg * DEG
    masked = np.zeros(z.shape, bool)
    negz = -z  # RING order has z non-increasing, so -z is sorted
    for k in range(nholes):
        th = math.acos(max(-1.0, min(1.0, zc[k])))
        zhi = math.cos(max(0.0, th - rad))
        zlo = math.cos(min(math.pi, th + rad))
        i0 = int(np.searchsorted(negz, -zhi, side="left"))
        i1 = int(np.searchsorted(negz, -zlo, side="right"))
        vp = _unit(z[i0:i1], phi[i0:i1])
        masked[i0:i1] |= (vp @ vc[k]) > cosr
    return masked


def hits_proxy(z, phi) -> np.ndarray:
    """Scan-depth proxy hits = 1 + 4 sin^2(ecliptic latitude)."""
    l0, b0 = (v * DEG for v in NEP_GAL_DEG)
    nep = np.array([math.cos(b0) * math.cos(l0), math.cos(b0) * math.sin(l0), math.sin(b0)])
    sinbeta = _unit(z, phi) @ nep
    return 1.0 + 4.0 * sinbeta ** 2


# ----------------------------------------------------------------------------
# white noise
# ----------------------------------------------------------------------------
def white_alm(lmax: int, seed: int, stream: int, offset: int = 0, device=None):
    """Unit white noise in harmonic space: a_l0 ~ N(0,1) real; for m > 0 the
    real and imaginary parts are N(0, 1/2) each.  With ``device`` the draws
    come from the torch path of the same generator (a torch tensor)."""
    p = nalm(lmax)
    _, ms = alm_lm(lmax)
    scale = np.where(ms == 0, 1.0, math.sqrt(0.5))
    if device is not None:
        import torch
        g = px.normal_torch(seed, stream, 2 * p, offset, device)
        sc = torch.as_tensor(scale, device=device)
        im = g[1::2] * sc
        im[torch.as_tensor(ms == 0, device=device)] = 0.0
        return torch.complex(g[0::2] * sc, im)
    g = px.normal(seed, stream, 2 * p, offset)
    re, im = g[0::2], g[1::2]
    out = (re + 1j * im) * scale
    out[ms == 0] = re[ms == 0]
    return out


def white_map(npix: int, seed: int, stream: int, offset: int = 0, device=None):
    if device is not None:
        return px.normal_torch(seed, stream, npix, offset, device)
    return px.normal(seed, stream, npix, offset)


# ----------------------------------------------------------------------------
# workloads
# ----------------------------------------------------------------------------
@dataclass
class Problem:
    """One constrained-realization problem (temperature, or T+E+B)."""
    name: str
    nside: int
    lmax: int
    ncomp: int                 # 1 = T, 3 = T,E,B
    cl: np.ndarray             # (lmax+1,) for T; (4, lmax+1) = TT, EE, BB, TE for T+E+B
    bl: np.ndarray             # (lmax+1,)
    ninv: np.ndarray           # (npix,) T, or (2, npix) = (T, P) with Q and U sharing P
    signal_alm: np.ndarray     # (ncomp, nalm) complex
    noise_map: np.ndarray      # (ncomp_map, npix): T or T, Q, U
    w1: np.ndarray             # (ncomp, nalm) complex
    w2: np.ndarray             # (ncomp_map, npix)
    tol: float
    extra: dict = field(default_factory=dict)

    @property
    def npix(self) -> int:
        return 12 * self.nside * self.nside


def _sqrt_cl_cholesky(cl4: np.ndarray):
    """Lower Cholesky factor rows of the per-l (T, E) block for drawing
    correlated signal alms; B is independent."""
    tt, ee, bb, te = cl4
    with np.errstate(divide="ignore", invalid="ignore"):
        l11 = np.sqrt(tt)
        l21 = np.where(tt > 0, te / np.where(tt > 0, l11, 1.0), 0.0)
        l22 = np.sqrt(np.maximum(ee - l21 ** 2, 0.0))
    return l11, l21, l22, np.sqrt(bb)


def fullsky_temperature(nside: int = 32, lmax: int = 64) -> Problem:
    """Full-sky temperature workload: flat C_l, 2 deg Gaussian beam, uniform
    white noise of 10 uK, PCG tolerance 1e-8.  With uniform noise on the full
    sky the solution has the closed form of Eqs. (hat_s_approx, hat_f_approx)."""
    ns, L = nside, lmax
    cl = cl_flat(L)
    bl = gauss_beam(L, 2.0 * DEG)
    npix = 12 * ns * ns
    sigma = 10.0
    ninv = np.full(npix, 1.0 / sigma ** 2)
    a = np.sqrt(cl)[alm_lm(L)[0]] * white_alm(L, 0, px.STREAM_SIGNAL)
    n = sigma * white_map(npix, 0, px.STREAM_NOISE)
    w1 = white_alm(L, 1, px.STREAM_W1)
    w2 = white_map(npix, 1, px.STREAM_W2)
    return Problem("fullsky_t", ns, L, 1, cl, bl, ninv, a[None], n[None], w1[None], w2[None], 1e-8)


def masked_temperature(nside: int = 256, lmax: int = 512, seed: int = 1) -> Problem:
    """Masked temperature workload: damped C_l, 30' Gaussian beam, noise
    20 uK / sqrt(hits), mask |b| < 20 deg plus 50 point-source holes of 1 deg,
    PCG tolerance 1e-6.  ``seed`` selects the hole positions and the random
    fields (the log-posterior workload uses seed 3)."""
    ns, L = nside, lmax
    cl = cl_damped(L)
    bl = gauss_beam(L, 30.0 * ARCMIN)
    z, phi = pixel_centres(ns)
    hits = hits_proxy(z, phi)
    sig = 20.0 / np.sqrt(hits)
    masked = latitude_cut(z, 20.0) | point_source_holes(z, phi, 50, 1.0, seed)
    ninv = np.where(masked, 0.0, 1.0 / sig ** 2)
    a = np.sqrt(cl)[alm_lm(L)[0]] * white_alm(L, seed, px.STREAM_SIGNAL)
    n = sig * white_map(z.size, seed, px.STREAM_NOISE)
    w1 = white_alm(L, seed + 100, px.STREAM_W1)
    w2 = white_map(z.size, seed + 100, px.STREAM_W2)
    return Problem(f"masked_t.s{seed}", ns, L, 1, cl, bl, ninv, a[None], n[None], w1[None],
                   w2[None], 1e-6, {"fsky": float(1.0 - masked.mean())})


def logpost_temperature(nside: int = 512, lmax: int = 1024) -> Problem:
    """Log-posterior workload: the masked temperature recipe with seed 3,
    N_side 512 and l_max 1024 by default."""
    return masked_temperature(nside, lmax, seed=3)


def mixed_geometry_chains(nchains: int = 64, nside: int | None = None,
                          lmax: int | None = None) -> list:
    """Independent chains of uneven geometry: N_side drawn from {64, 128, 256},
    l_max = 2 N_side or 3 N_side - 1, C_l amplitude in [0.8, 1.2], beam
    60 / N_side deg, 15 uK uniform noise, mask |b| < 15 deg, tolerance 1e-6.
    ``nside`` (and ``lmax``, default 2 N_side) give every chain one reduced
    geometry for small tests."""
    u = px.uniform(2, px.STREAM_CHAINS, 3 * nchains)
    chains = []
    for c in range(nchains):
        ns = (64, 128, 256)[min(2, int(u[3 * c] * 3))]
        L = 2 * ns if u[3 * c + 1] < 0.5 else 3 * ns - 1
        if nside is not None:
            ns = nside
            L = lmax or 2 * ns
        amp = 0.8 + 0.4 * u[3 * c + 2]
        cl = amp * cl_flat(L)
        bl = gauss_beam(L, (60.0 / ns) * DEG)
        z, phi = pixel_centres(ns)
        masked = latitude_cut(z, 15.0)
        sigma = 15.0
        ninv = np.where(masked, 0.0, 1.0 / sigma ** 2)
        key = 1000 + c
        a = np.sqrt(cl)[alm_lm(L)[0]] * white_alm(L, key, px.STREAM_SIGNAL)
        n = sigma * white_map(z.size, key, px.STREAM_NOISE)
        w1 = white_alm(L, key, px.STREAM_W1)
        w2 = white_map(z.size, key, px.STREAM_W2)
        chains.append(Problem(f"chain.{c}", ns, L, 1, cl, bl, ninv, a[None], n[None],
                              w1[None], w2[None], 1e-6, {"amp": amp}))
    return chains


def teb_realizations(batch: int = 8, nside: int = 1024, lmax: int = 2048, device=None) -> list:
    """T+E+B workload: ``batch`` realizations sharing C_l (damped TT,
    EE = 0.05 TT, BB = 1e-3 EE, TE = 0.3 sqrt(TT EE)), a 10' beam and noise
    30 / 42 uK / sqrt(hits) for T / Q, U, mask |b| < 20 deg plus 200 holes of
    1 deg, tolerance 1e-6.  With ``device`` the random fields are torch
    tensors drawn on that device."""
    ns, L, nb = nside, lmax, batch
    tt = cl_damped(L)
    ee = 0.05 * tt
    te = 0.3 * np.sqrt(tt * ee)
    bb = 1e-3 * ee
    cl4 = np.stack([tt, ee, bb, te])
    bl = gauss_beam(L, 10.0 * ARCMIN)
    z, phi = pixel_centres(ns)
    hits = hits_proxy(z, phi)
    masked = latitude_cut(z, 20.0) | point_source_holes(z, phi, 200, 1.0, 4)
    sig_t = 30.0 / np.sqrt(hits)
    sig_p = 42.0 / np.sqrt(hits)
    ninv = np.stack([np.where(masked, 0.0, 1.0 / sig_t ** 2),
                     np.where(masked, 0.0, 1.0 / sig_p ** 2)])
    l11, l21, l22, lbb = _sqrt_cl_cholesky(cl4)
    ls = alm_lm(L)[0]
    p = nalm(L)
    out = []
    if device is not None:
        import torch
        stack = torch.stack
        cv = lambda x: torch.as_tensor(x, device=device)  # noqa: E731
    else:
        stack = np.stack
        cv = lambda x: x  # noqa: E731
    c11, c21, c22, cbb, cst, csp = (cv(l11[ls]), cv(l21[ls]), cv(l22[ls]), cv(lbb[ls]),
                                    cv(sig_t), cv(sig_p))
    for b in range(nb):
        key = 4000 + b
        wt = white_alm(L, key, px.STREAM_SIGNAL, 0, device)
        we = white_alm(L, key, px.STREAM_SIGNAL, 2 * p, device)
        wb = white_alm(L, key, px.STREAM_SIGNAL, 4 * p, device)
        a = stack([c11 * wt, c21 * wt + c22 * we, cbb * wb])
        npx = z.size
        nmap = stack([cst * white_map(npx, key, px.STREAM_NOISE, 0, device),
                      csp * white_map(npx, key, px.STREAM_NOISE, npx, device),
                      csp * white_map(npx, key, px.STREAM_NOISE, 2 * npx, device)])
        w1 = stack([white_alm(L, key, px.STREAM_W1, k * 2 * p, device) for k in range(3)])
        w2 = stack([white_map(npx, key, px.STREAM_W2, k * npx, device) for k in range(3)])
        out.append(Problem(f"teb.{b}", ns, L, 3, cl4, bl, ninv, a, nmap, w1, w2, 1e-6,
                           {"fsky": float(1.0 - masked.mean())}))
    return out

"""Pins for the oracle solver (no GPU): dense brute force, the paper's
full-sky closed form, the constant-latitude-mask block structure of App. A,
linearity of Eqs. (mean-field-map)/(fluc-map), finite differences of the
log-posterior gradient, and the diagonal preconditioner against the
operator's own diagonal."""
import math

import numpy as np
import pytest

from inputs import configs as C
from oracle import sht, solver


def _rand_alm(L, rng, ncomp=1):
    P = (L + 1) * (L + 2) // 2
    a = rng.normal(size=(ncomp, P)) + 1j * rng.normal(size=(ncomp, P))
    ms = sht.ms_of(L)
    a[:, ms == 0] = a[:, ms == 0].real
    return a


# ----------------------------------------------------------------- dense
def _real_params(L):
    ls, ms = sht.ls_of(L), sht.ms_of(L)
    cols = []
    for i, (l, m) in enumerate(zip(ls, ms)):
        cols.append((i, l, m, "re"))
        if m > 0:
            cols.append((i, l, m, "im"))
    return cols


def _dense_Y(L, nside):
    from scipy.special import sph_harm_y
    z, phi = C.pixel_centres(nside)
    th = np.arccos(z)
    cols = _real_params(L)
    Yd = np.zeros((z.size, len(cols)))
    W = np.zeros(len(cols))
    for k, (i, l, m, part) in enumerate(cols):
        Y = sph_harm_y(l, m, th, phi)
        if m == 0:
            Yd[:, k], W[k] = Y.real, 1.0
        elif part == "re":
            Yd[:, k], W[k] = 2 * Y.real, 2.0
        else:
            Yd[:, k], W[k] = -2 * Y.imag, 2.0
    return Yd, W, cols


def _to_params(a, cols):
    return np.array([a[i].real if p == "re" else a[i].imag for (i, l, m, p) in cols])


def test_dense_bruteforce_masked():
    nside, L = 4, 10
    rng = np.random.default_rng(0)
    g = sht.healpix(nside)
    cl = C.cl_flat(L)
    bl = C.gauss_beam(L, 20 * C.DEG)
    ninv = rng.uniform(0.5, 2.0, g.npix) * (rng.uniform(size=g.npix) > 0.3)
    prob = solver.Problem(g, L, cl, bl, ninv)
    d = rng.normal(size=g.npix)
    w1 = _rand_alm(L, rng)
    w2 = rng.normal(size=g.npix)
    b = prob.rhs(d, w1, w2)
    x, it, hist = solver.pcg(prob, b, 1e-13, 500)
    # dense system in real parameters (independent Y from scipy)
    Yd, W, cols = _dense_Y(L, nside)
    lcol = np.array([c[1] for c in cols])
    act = lcol >= 2
    bc = np.where(act, bl[lcol], 0.0)
    sinv = np.where(act, 1.0 / np.where(act, cl[lcol], 1.0), 1.0)
    A = np.diag(sinv) + (bc[:, None] / W[:, None]) * (Yd.T @ (ninv[:, None] * Yd)) * bc[None, :]
    sh = np.where(act, 1.0 / np.sqrt(np.where(act, cl[lcol], 1.0)), 0.0)
    rhs = bc / W * (Yd.T @ (ninv * d + np.sqrt(ninv) * w2)) + sh * _to_params(w1[0], cols)
    assert np.allclose(_to_params(b[0], cols), rhs, rtol=1e-12, atol=1e-12 * np.abs(rhs).max())
    xd = np.linalg.solve(A, rhs)
    xo = _to_params(x[0], cols)
    assert np.max(np.abs(xo - xd)) < 1e-10 * np.max(np.abs(xd))
    # W A is symmetric positive definite
    WA = W[:, None] * A
    assert np.allclose(WA, WA.T, atol=1e-12 * np.abs(WA).max())
    assert np.linalg.eigvalsh(0.5 * (WA + WA.T)).min() > 0


def test_operator_symmetric_spin2():
    nside, L = 4, 8
    rng = np.random.default_rng(2)
    g = sht.healpix(nside)
    tt = C.cl_flat(L)
    cl4 = np.stack([tt, 0.05 * tt, 1e-3 * 0.05 * tt, 0.3 * np.sqrt(0.05) * tt])
    ninv = np.stack([rng.uniform(0.5, 2, g.npix), rng.uniform(0.2, 1, g.npix)])
    prob = solver.Problem(g, L, cl4, C.gauss_beam(L, 0.2), ninv)
    x, y = _rand_alm(L, rng, 3), _rand_alm(L, rng, 3)
    ax, ay = prob.matvec(x), prob.matvec(y)
    assert abs(prob.dot(x, ay) - prob.dot(ax, y)) < 1e-12 * abs(prob.dot(x, ay))
    assert prob.dot(x, ax) > 0


# ----------------------------------------------------------- closed form
def test_fullsky_closed_form_gl():
    """Uniform noise on an exact-quadrature grid: A = diag(1/C + b^2/N_l) with
    N_l = 4 pi sigma^2 / N_pix, and the solution is Eqs. (hat_s_approx) +
    (hat_f_approx) with r_lm = N_l (Y^T N^-1 d)_lm and
    w1'_lm = sqrt(N_l) (Y^T N^-1/2 w2)_lm."""
    L = 24
    g = sht.gauss_legendre(L + 1, 2 * L + 2)
    rng = np.random.default_rng(4)
    sigma = 10.0
    Nl = 4 * math.pi * sigma ** 2 / g.npix
    ninv = g.pixel_weights() / Nl
    cl = C.cl_flat(L)
    bl = C.gauss_beam(L, 10 * C.DEG)
    prob = solver.Problem(g, L, cl, bl, ninv)
    d = rng.normal(size=g.npix) * 30
    w1 = _rand_alm(L, rng)
    w2 = rng.normal(size=g.npix)
    b = prob.rhs(d, w1, w2)
    x, it, _ = solver.pcg(prob, b, 1e-12, 50)
    assert it <= 2      # the preconditioner is the exact inverse here
    ls = sht.ls_of(L)
    r = Nl * sht.alm2map_adjoint(g, L, ninv * d)
    w1p = math.sqrt(Nl) * sht.alm2map_adjoint(g, L, np.sqrt(ninv) * w2)
    C_, B_ = cl[ls], bl[ls]
    den = Nl + B_ ** 2 * C_
    ahat = r * B_ * C_ / den
    fhat = w1[0] * Nl * np.sqrt(C_) / den + w1p * math.sqrt(Nl) * B_ * C_ / den
    ref = np.where(ls >= 2, ahat + fhat, 0.0)
    assert np.max(np.abs(x[0] - ref)) < 1e-11 * np.max(np.abs(ref))


def test_fullsky_closed_form_teb_gl():
    """T+E+B generalisation: A = S^-1 + b^2 diag(1/N_T, 1/N_P, 1/N_P) per lm."""
    L = 16
    g = sht.gauss_legendre(L + 1, 2 * L + 2)
    rng = np.random.default_rng(6)
    NT, NP = 0.3, 0.7
    ninv = np.stack([g.pixel_weights() / NT, g.pixel_weights() / NP])
    tt = C.cl_flat(L)
    cl4 = np.stack([tt, 0.05 * tt, 5e-5 * tt, 0.3 * np.sqrt(0.05) * tt])
    bl = C.gauss_beam(L, 8 * C.DEG)
    prob = solver.Problem(g, L, cl4, bl, ninv)
    b = _rand_alm(L, rng, 3)
    b[:, sht.ls_of(L) < 2] = 0
    x, it, _ = solver.pcg(prob, b, 1e-12, 100)
    ls = sht.ls_of(L)
    ref = np.zeros_like(b)
    for i in range(b.shape[1]):
        l = ls[i]
        if l < 2:
            continue
        tt_, ee, bb, te = cl4[:, l]
        S = np.array([[tt_, te, 0], [te, ee, 0], [0, 0, bb]])
        A = np.linalg.inv(S) + bl[l] ** 2 * np.diag([1 / NT, 1 / NP, 1 / NP])
        ref[:, i] = np.linalg.solve(A, b[:, i].real) + 1j * np.linalg.solve(A, b[:, i].imag)
    assert np.max(np.abs(x - ref)) < 1e-10 * np.max(np.abs(ref))


# ------------------------------------------------ constant-latitude mask
def test_constant_latitude_mask_block_structure():
    """App. A: for a mask |b| < b0 and uniform noise the operator is
    block-diagonal in m, and within a block entries with l + l' odd vanish.
    The PCG solution equals the per-m dense block solves."""
    L = 20
    g = sht.gauss_legendre(L + 1, 2 * L + 2)
    sigma = 5.0
    lat_cut = np.abs(g.cth) < math.sin(25 * C.DEG)
    ninv_ring = np.where(lat_cut, 0.0, 1.0 / sigma ** 2)
    ninv = np.repeat(ninv_ring, g.nphi)
    cl = C.cl_flat(L)
    bl = C.gauss_beam(L, 10 * C.DEG)
    prob = solver.Problem(g, L, cl, bl, ninv)
    rng = np.random.default_rng(8)
    b = _rand_alm(L, rng)
    ls, ms = sht.ls_of(L), sht.ms_of(L)
    b[:, ls < 2] = 0
    x, it, _ = solver.pcg(prob, b, 1e-13, 500)
    for m in range(L + 1):
        lrange = np.arange(max(m, 2), L + 1)
        lam = np.array([sht.lambda_lm(L, m, g.cth[r], g.sth[r])[lrange - m]
                        for r in range(g.nring)])              # (nring, nl)
        blk = (lam * (g.nphi * ninv_ring)[:, None]).T @ lam
        blk = bl[lrange][:, None] * blk * bl[lrange][None, :] + np.diag(1.0 / cl[lrange])
        odd = ((lrange[:, None] + lrange[None, :]) % 2) == 1
        if odd.any():
            assert np.max(np.abs(blk[odd])) < 1e-13 * np.max(np.abs(blk))
        sel = (ms == m) & (ls >= 2)
        rhs = b[0, sel]
        ref = np.linalg.solve(blk, rhs.real) + 1j * np.linalg.solve(blk, rhs.imag)
        assert np.max(np.abs(x[0, sel] - ref)) < 1e-10 * max(1e-30, np.max(np.abs(ref)))
    # off-block coupling is absent: A applied to a single-m vector stays in m
    v = np.zeros_like(b)
    v[0, (ms == 3) & (ls >= 3)] = 1.0
    Av = prob.matvec(v)
    assert np.max(np.abs(Av[0, ms != 3])) < 1e-13 * np.max(np.abs(Av))


def _azimuthal_problem(L, north_south_asymmetric=False):
    """GL grid (nphi >= 2 L + 1), ring-constant N^-1: a |b| < 25 deg cut and
    optionally noise that differs between the hemispheres."""
    g = sht.gauss_legendre(L + 1, 2 * L + 2)
    ninv_ring = np.where(np.abs(g.cth) < math.sin(25 * C.DEG), 0.0, 1.0 / 5.0 ** 2)
    if north_south_asymmetric:
        ninv_ring = ninv_ring * np.where(g.cth > 0, 1.0, 0.35) * (1.0 + 0.5 * g.cth ** 2)
    ninv = np.repeat(ninv_ring, g.nphi)
    prob = solver.Problem(g, L, C.cl_flat(L), C.gauss_beam(L, 10 * C.DEG), ninv)
    return g, prob, ninv_ring


@pytest.mark.parametrize("asym", [False, True])
def test_block_solve_equals_pcg(asym):
    """The per-m dense solves of App. A equal a PCG solve converged to 1e-13
    (an independent method on the same operator); with hemispheres of
    different noise the l + l' odd entries no longer vanish and still
    solve correctly."""
    L = 24
    g, prob, wr = _azimuthal_problem(L, asym)
    assert np.array_equal(solver.ring_weights(prob), wr)
    rng = np.random.default_rng(12)
    b = _rand_alm(L, rng)
    b[:, sht.ls_of(L) < 2] = 0
    xb = solver.block_solve(prob, b)
    xp, _, _ = solver.pcg(prob, b, 1e-13, 800)
    assert np.max(np.abs(xb - xp)) < 1e-10 * np.max(np.abs(xp))
    _, A3 = solver.azimuthal_block(prob, 3, wr)
    odd = ((np.arange(3, L + 1)[:, None] + np.arange(3, L + 1)[None, :]) % 2) == 1
    assert (np.max(np.abs(A3[odd])) > 1e-6 * np.max(np.abs(A3))) == asym


def test_azimuthal_block_is_the_operator_restricted_to_m():
    """Brute force: apply A to every unit vector of one m (real parts) and
    read the m-block off the operator; it equals azimuthal_block."""
    L, m = 12, 2
    g, prob, wr = _azimuthal_problem(L, True)
    ls, ms = sht.ls_of(L), sht.ms_of(L)
    idx = np.where(ms == m)[0]
    cols = []
    for i in idx:
        e = np.zeros((1, ls.size), complex)
        e[0, i] = 1.0
        cols.append(prob.matvec(e)[0, idx].real)
    Abf = np.array(cols).T
    lr, A = solver.azimuthal_block(prob, m, wr)
    assert np.array_equal(lr, ls[idx])
    assert np.max(np.abs(Abf - A)) < 1e-12 * np.max(np.abs(A))


def test_block_solve_refuses_non_azimuthal_noise():
    p = C.masked_temperature(8, 16)
    prob = solver.Problem(sht.healpix(8), 16, p.cl, p.bl, p.ninv)
    assert solver.ring_weights(prob) is None
    with pytest.raises(ValueError):
        solver.block_solve(prob, np.zeros((1, (17 * 18) // 2), complex))


# ----------------------------------------------------------- linearity
def test_mean_field_plus_fluctuation():
    p = C.fullsky_temperature(8, 16)
    g = sht.healpix(8)
    prob = solver.Problem(g, 16, p.cl, p.bl, p.ninv)
    d = sht.alm2map(g, 16, p.signal_alm[0] * p.bl[sht.ls_of(16)]) + p.noise_map[0]
    bd, bw = prob.rhs_parts(d, p.w1, p.w2)
    b = prob.rhs(d, p.w1, p.w2)
    assert np.allclose(bd + bw, b, rtol=0, atol=1e-12 * np.abs(b).max())
    xs = [solver.pcg(prob, v, 1e-13, 500)[0] for v in (bd, bw, b)]
    assert np.max(np.abs(xs[0] + xs[1] - xs[2])) < 1e-10 * np.max(np.abs(xs[2]))


def test_fullsky_pcg_converges():
    p = C.fullsky_temperature()
    g = sht.healpix(p.nside)
    L = p.lmax
    prob = solver.Problem(g, L, p.cl, p.bl, p.ninv)
    d = sht.alm2map(g, L, p.signal_alm[0] * p.bl[sht.ls_of(L)]) + p.noise_map[0]
    b = prob.rhs(d, p.w1, p.w2)
    x, it, hist = solver.pcg(prob, b, p.tol, 500)
    assert hist[-1] <= p.tol
    assert solver.true_residual(prob, x, b) <= 1.05 * p.tol
    assert 1 <= it < 200


# ----------------------------------------------------------- gradient
def test_log_posterior_gradient_fd():
    L, nside = 12, 8
    g = sht.healpix(nside)
    p = C.masked_temperature(nside, L)
    prob = solver.Problem(g, L, p.cl, p.bl, p.ninv)
    d = sht.alm2map(g, L, p.signal_alm[0] * p.bl[sht.ls_of(L)]) + p.noise_map[0]
    rng = np.random.default_rng(9)
    a = p.signal_alm + 0.3 * _rand_alm(L, rng) * np.sqrt(p.cl[sht.ls_of(L)])
    a[:, sht.ls_of(L) < 2] = 0
    bins = [(2, 5), (6, 9), (10, 12)]
    ga, gl = solver.log_posterior_grad(prob, a, d, bins)
    h = 1e-4
    ls, ms = sht.ls_of(L), sht.ms_of(L)
    for i in rng.choice(np.where(ls >= 2)[0], 8, replace=False):
        for unit in (1.0, 1j) if ms[i] > 0 else (1.0,):
            e = np.zeros_like(a)
            e[0, i] = unit
            fd = (solver.log_posterior(prob, a + h * e, d) - solver.log_posterior(prob, a - h * e, d)) / (2 * h)
            an = prob.dot(e, ga)
            assert abs(fd - an) < 1e-5 * max(1.0, abs(an))
    for k, (lo, hi) in enumerate(bins):
        def lp(eps):
            sc = np.ones(L + 1)
            sc[lo:hi + 1] = math.exp(eps)
            return solver.log_posterior(prob, a, d, cl_scale=sc)
        fd = (lp(h) - lp(-h)) / (2 * h)
        assert abs(fd - gl[k]) < 1e-5 * max(1.0, abs(gl[k]))


# ---------------------------------------------------- preconditioner diagonal
@pytest.mark.parametrize("ncomp", [1, 3])
def test_precond_diag_is_the_operator_diagonal(ncomp):
    """M = S^-1 + b_l^2 D_lm (Sect. 4's diagonal preconditioner) against the
    diagonal of A read off the operator itself, for an arbitrary N^-1 (holes,
    no ring symmetry).  |Y_lm(p)|^2 does not depend on phi, so D_lm is the
    mean of the real-part and imaginary-part diagonal entries of
    Y^T N^-1 Y (their e^{2 i m phi} terms cancel); for m = 0 only the real
    part exists.  The T-E entries of M are the prior's; the noise couples no
    T and E (different maps)."""
    L, nside = 8, 4
    g = sht.healpix(nside)
    rng = np.random.default_rng(3)
    npix = g.npix
    ninv = rng.uniform(0.5, 2.0, size=(2, npix)) * (rng.uniform(size=(2, npix)) > 0.2)
    ls = np.arange(L + 1)
    tt = np.where(ls >= 2, 1.0 / np.maximum(ls * (ls + 1.0), 1.0), 0.0)
    if ncomp == 1:
        cl, nv = tt, ninv[0]
    else:
        ee = 0.3 * tt
        cl, nv = np.stack([tt, ee, 0.1 * ee, 0.4 * np.sqrt(tt * ee)]), ninv
    bl = np.exp(-0.01 * ls * (ls + 1))
    prob = solver.Problem(g, L, cl, bl, nv)
    M = prob.precond_diag()
    P = (L + 1) * (L + 2) // 2
    ms = sht.ms_of(L)
    for c in range(ncomp):
        for j in range(P):
            e = np.zeros((ncomp, P), complex)
            e[c, j] = 1.0
            Are = prob.matvec(e)
            d = Are[c, j].real
            if ms[j] > 0:
                e[c, j] = 1j
                d = 0.5 * (d + prob.matvec(e)[c, j].imag)
            assert d == pytest.approx(M[c, c, j], rel=1e-12, abs=1e-12), (c, j)
            if ncomp == 3 and c == 1:
                assert Are[0, j].real == pytest.approx(M[0, 1, j], rel=1e-12, abs=1e-14), j


def test_apply_block_inverse_solves_each_block():
    """z = M^-1 r per alm index: multiplying back gives r, for 1x1 and for
    3x3 symmetric blocks with complex right-hand sides."""
    rng = np.random.default_rng(4)
    n = 37
    r1 = rng.normal(size=(1, n)) + 1j * rng.normal(size=(1, n))
    M1 = rng.uniform(0.5, 2.0, size=(1, 1, n))
    z1 = solver.apply_block_inverse(M1, r1)
    assert np.allclose(M1[0, 0] * z1[0], r1[0], rtol=1e-14, atol=0)
    A = rng.normal(size=(n, 3, 3))
    M3 = np.moveaxis(A @ np.swapaxes(A, 1, 2) + 3 * np.eye(3), 0, 2)    # SPD blocks
    r3 = rng.normal(size=(3, n)) + 1j * rng.normal(size=(3, n))
    z3 = solver.apply_block_inverse(M3, r3)
    back = np.einsum("ijn,jn->in", M3, z3)
    assert np.allclose(back, r3, rtol=0, atol=1e-12 * np.abs(r3).max())


def test_log_posterior_value_direct():
    """The log-posterior of Eq. (joint-posterior) evaluated term by term with
    an independent synthesis (scipy Y_lm on the pixel centres, the a_{l,-m}
    terms written out) and the prior summed over m = -l..l explicitly."""
    nside, L = 4, 8
    rng = np.random.default_rng(6)
    g = sht.healpix(nside)
    cl = C.cl_flat(L) * (1.0 + 0.1 * np.arange(L + 1))
    bl = C.gauss_beam(L, 15 * C.DEG)
    ninv = rng.uniform(0.5, 2.0, g.npix) * (rng.uniform(size=g.npix) > 0.25)
    prob = solver.Problem(g, L, cl, bl, ninv)
    a = _rand_alm(L, rng)
    a[:, sht.ls_of(L) < 2] = 0
    d = rng.normal(size=g.npix)
    Yd, W, cols = _dense_Y(L, nside)
    ls = np.array([c[1] for c in cols])
    model = Yd @ (np.where(ls >= 2, bl[ls], 0.0) * _to_params(a[0], cols))
    chi2 = np.sum((d - model) ** 2 * ninv)
    prior = 0.0
    for l in range(2, L + 1):
        for m in range(-l, l + 1):
            am = a[0, abs(m) * (2 * L + 1 - abs(m)) // 2 + l]   # |a_{l,-m}| = |a_lm|
            prior += abs(am) ** 2 / cl[l]
    expect = -0.5 * chi2 - 0.5 * prior
    assert solver.log_posterior(prob, a, d) == pytest.approx(expect, rel=1e-12)


# ------------------------------------------------------------- joint move
def _cl4(L, rng):
    ls = np.arange(L + 1)
    tt = np.where(ls >= 2, rng.uniform(0.5, 2.0, L + 1) / np.maximum(ls * (ls + 1.0), 1.0), 0.0)
    ee = tt * rng.uniform(0.02, 0.1, L + 1)
    bb = ee * rng.uniform(1e-3, 1e-1, L + 1)
    te = rng.uniform(-0.8, 0.8, L + 1) * np.sqrt(tt * ee)
    return np.stack([tt, ee, bb, te])


def test_fluctuation_rescale_maps_old_covariance_to_new():
    """M = (C')^{1/2} C^{-1/2} per l must carry the old covariance to the new
    one, M C M^T = C' (any consistent square root does; a transposed factor
    or swapped order fails for non-commuting T/E blocks), act as
    sqrt(C'/C) for temperature, as the identity for C' = C, and hold the
    singular l < 2 at zero."""
    L = 6
    rng = np.random.default_rng(11)
    co, cn = _cl4(L, rng), _cl4(L, rng)
    P = (L + 1) * (L + 2) // 2
    ls, ms = sht.ls_of(L), sht.ms_of(L)
    for l in range(2, L + 1):
        j = np.where((ls == l) & (ms == 1))[0][0]
        M = np.zeros((3, 3))
        for c in range(3):
            e = np.zeros((3, P), complex)
            e[c, j] = 1.0
            M[:, c] = solver.fluctuation_rescale(co, cn, e, L)[:, j].real
        Co = np.array([[co[0, l], co[3, l], 0], [co[3, l], co[1, l], 0], [0, 0, co[2, l]]])
        Cn = np.array([[cn[0, l], cn[3, l], 0], [cn[3, l], cn[1, l], 0], [0, 0, cn[2, l]]])
        assert np.allclose(M @ Co @ M.T, Cn, rtol=1e-12, atol=1e-14 * np.abs(Cn).max())
    f = _rand_alm(L, rng, 3)
    assert np.allclose(solver.fluctuation_rescale(co, co, f, L)[:, ls >= 2], f[:, ls >= 2], rtol=1e-12)
    assert np.all(solver.fluctuation_rescale(co, cn, f, L)[:, ls < 2] == 0)
    ft = _rand_alm(L, rng, 1)
    st = solver.fluctuation_rescale(co[0], cn[0], ft, L)
    ratio = np.where(ls >= 2, np.sqrt(cn[0, ls] / np.where(ls >= 2, co[0, ls], 1.0)), 0.0)
    assert np.allclose(st[0], ratio * ft[0], rtol=1e-13, atol=0)


def test_joint_log_target_direct():
    """log pi(theta) of the acceptance rule term by term with an independent
    synthesis (scipy Y_lm on the pixel centres) and an explicit prior sum;
    with f = 0 it is the log-posterior."""
    nside, L = 4, 8
    rng = np.random.default_rng(12)
    g = sht.healpix(nside)
    cl = C.cl_flat(L) * (1.0 + 0.05 * np.arange(L + 1))
    bl = C.gauss_beam(L, 15 * C.DEG)
    ninv = rng.uniform(0.5, 2.0, g.npix) * (rng.uniform(size=g.npix) > 0.25)
    prob = solver.Problem(g, L, cl, bl, ninv)
    a, f = _rand_alm(L, rng), _rand_alm(L, rng)
    a[:, sht.ls_of(L) < 2] = 0
    d = rng.normal(size=g.npix)
    Yd, W, cols = _dense_Y(L, nside)
    ls = np.array([c[1] for c in cols])
    bc = np.where(ls >= 2, bl[ls], 0.0)
    chi2 = np.sum((d - Yd @ (bc * _to_params(a[0], cols))) ** 2 * ninv)
    fl = np.sum((Yd @ (bc * _to_params(f[0], cols))) ** 2 * ninv)
    prior = 0.0
    for l in range(2, L + 1):
        for m in range(-l, l + 1):
            prior += abs(a[0, abs(m) * (2 * L + 1 - abs(m)) // 2 + l]) ** 2 / cl[l]
    expect = -0.5 * (chi2 + prior + fl)
    assert solver.joint_log_target(prob, d, a, f) == pytest.approx(expect, rel=1e-12)
    assert solver.joint_log_target(prob, d, a, 0 * f) == pytest.approx(
        solver.log_posterior(prob, a, d), rel=1e-13)


def test_joint_log_target_fluctuation_term_is_the_noise_part_of_A():
    """T+E+B: the fluctuation term is -1/2 <f, (A - S^-1) f>, the noise part
    of the solver's operator (Q and U weighted by the polarization N^-1)."""
    nside, L = 4, 8
    rng = np.random.default_rng(13)
    g = sht.healpix(nside)
    ninv = np.stack([rng.uniform(0.5, 2.0, g.npix), rng.uniform(0.2, 1.0, g.npix)])
    prob = solver.Problem(g, L, _cl4(L, rng), C.gauss_beam(L, 0.2), ninv)
    f = _rand_alm(L, rng, 3)
    f[:, sht.ls_of(L) < 2] = 0
    zero = np.zeros((3, g.npix))
    lp = solver.joint_log_target(prob, prob.Y(prob.beam(0 * f)), 0 * f, f)
    sinv_f = prob._per_l(prob.sinv * prob.active[None, None, :], f)
    noise = prob.dot(f, prob.matvec(f)) - prob.dot(f, sinv_f)
    assert lp == pytest.approx(-0.5 * noise, rel=1e-11)
    assert solver.joint_log_target(prob, zero, 0 * f, 0 * f) == 0.0


def test_joint_acceptance_rule():
    assert solver.joint_acceptance(-10.0, -12.0) == 1.0
    assert solver.joint_acceptance(-12.0, -10.0) == pytest.approx(math.exp(-2.0))
    assert solver.joint_acceptance(-12.0, -10.0, 1.5, -0.5) == 1.0
    assert solver.joint_acceptance(-12.0, -10.0, 0.5, 0.0) == pytest.approx(math.exp(-1.5))


# ------------------------------------------------- exact harmonic likelihood
def test_exact_harmonic_loglike_is_the_gaussian_likelihood():
    """Eq. (exact_harm) differs from the Gaussian log-likelihood of r_lm ~
    N(0, b_l^2 C_l + N_l), summed over every (l, m) with m = -l..l, only by
    a theta-independent constant: differences between two spectra agree."""
    L = 40
    rng = np.random.default_rng(17)
    cl = C.cl_flat(L)
    bl = C.gauss_beam(L, 3 * C.DEG)
    nl = np.full(L + 1, 4e-3)
    ls, ms = sht.ls_of(L), sht.ms_of(L)
    var = bl ** 2 * cl + nl
    r = _rand_alm(L, rng)[0] * np.sqrt(np.where(ms == 0, 1.0, 0.5) * var[ls])

    def direct(clt):
        v = (bl ** 2 * clt + nl)[ls]
        keep = ls >= 2
        # m = 0: one real Gaussian; m > 0: the pair (a_lm, a_l,-m) = two real
        # Gaussians of variance v / 2 each, i.e. |r|^2 / (v / 2) / 2 ... summed
        # over both signs of m
        q = np.where(ms == 0, r.real ** 2 / v, 2.0 * np.abs(r) ** 2 / v)
        lndet = np.where(ms == 0, np.log(v), 2.0 * np.log(v))
        return float(-0.5 * np.sum((q + lndet)[keep]))

    co = solver.observed_spectrum(r, L)
    for s1, s2 in ((1.0, 1.3), (0.7, 1.1)):
        d_exact = (solver.exact_harmonic_loglike(co, s1 * cl, bl, nl) -
                   solver.exact_harmonic_loglike(co, s2 * cl, bl, nl))
        assert d_exact == pytest.approx(direct(s1 * cl) - direct(s2 * cl), rel=1e-12)
    # the maximum over an amplitude q sits where sum (2l+1) (x_l - 1) b^2 C_l / (b^2 q C_l + N) = 0
    qs = np.linspace(0.5, 2.0, 3001)
    lk = np.array([solver.exact_harmonic_loglike(co, q * cl, bl, nl) for q in qs])
    qm = qs[np.argmax(lk)]
    l = np.arange(L + 1)[2:]
    den = bl[2:] ** 2 * qm * cl[2:] + nl[2:]
    grad = np.sum((2 * l + 1) * (co[2:] / den - 1.0) * bl[2:] ** 2 * cl[2:] / den)
    assert abs(grad) < 0.02 * np.sum((2 * l + 1) * bl[2:] ** 2 * cl[2:] / den)


def test_joint_move_samples_the_exact_marginal_posterior():
    """The oracle's joint-move pieces (rescaling, log pi with the prior term
    read as a^T S^-1 a^, acceptance) run as a Metropolis-Hastings chain in an
    amplitude q (C_l = q C_l^fid, flat prior) on a full-sky, uniform-noise
    Gauss-Legendre grid sample the closed-form marginal posterior of Eq.
    (exact_harm): chain mean and width within a fifth of the posterior
    width (4000 steps, 400 of burn-in, fixed seeds)."""
    L = 24
    g = sht.gauss_legendre(L + 1, 2 * L + 2)
    sig2 = 3.0
    ninv = g.pixel_weights() / sig2
    cl_fid = C.cl_flat(L)
    bl = C.gauss_beam(L, 2.0 * C.DEG)
    ls, ms = sht.ls_of(L), sht.ms_of(L)
    from inputs import philox as px
    a_true = np.sqrt(cl_fid)[ls] * C.white_alm(L, 7, px.STREAM_SIGNAL)
    d = sht.alm2map(g, L, a_true * bl[ls]) + C.white_map(g.npix, 7, px.STREAM_NOISE) / np.sqrt(ninv)
    co = solver.observed_spectrum(sig2 * sht.alm2map_adjoint(g, L, ninv * d), L)
    qs = np.linspace(0.05, 5.0, 9001)
    lk = np.array([solver.exact_harmonic_loglike(co, q * cl_fid, bl, np.full(L + 1, sig2)) for q in qs])
    w = np.exp(lk - lk.max())
    mean = np.sum(w * qs) / np.sum(w)
    std = np.sqrt(np.sum(w * (qs - mean) ** 2) / np.sum(w))
    rng = np.random.default_rng(0)
    z1, z2 = np.zeros((1, ls.size), complex), np.zeros((1, g.npix))

    def solve(q, dd, w1, w2):
        prob = solver.Problem(g, L, q * cl_fid, bl, ninv)
        return solver.pcg(prob, prob.rhs(dd, w1, w2), 1e-11, 50)[0], prob

    def white():
        w1 = rng.normal(size=ls.size) + 1j * rng.normal(size=ls.size)
        return np.where(ms == 0, w1.real, w1 * np.sqrt(0.5))[None], rng.normal(size=g.npix)[None]

    q = 1.0
    a, prob = solve(q, d[None], z1, z2)
    f, _ = solve(q, 0 * d[None], *white())
    lp = solver.joint_log_target(prob, d, a, f)
    chain = []
    for _ in range(4000):
        qp, u = q + 2.4 * std * rng.standard_normal(), rng.uniform()
        if qp > 0:
            ap, probp = solve(qp, d[None], z1, z2)
            lpp = solver.joint_log_target(probp, d, ap, solver.fluctuation_rescale(q * cl_fid, qp * cl_fid, f, L))
            if u < solver.joint_acceptance(lpp, lp):
                q, a = qp, ap
                f, _ = solve(q, 0 * d[None], *white())
                lp = solver.joint_log_target(probp, d, a, f)
        chain.append(q)
    chain = np.array(chain[400:])
    assert abs(chain.mean() - mean) < 0.2 * std
    assert abs(chain.std() / std - 1.0) < 0.2


# --------------------------------------------- two-level preconditioner
def test_low_block_matches_dense_bruteforce():
    """The low-l block read off the operator column by column equals
    W S^-1 + B Yd^T N^-1 Yd B restricted to l <= l_c, with Yd the real
    spherical harmonics from scipy on the pixel centres (independent of the
    oracle's transforms)."""
    nside, L, lc = 4, 10, 5
    rng = np.random.default_rng(21)
    g = sht.healpix(nside)
    cl = C.cl_flat(L)
    bl = C.gauss_beam(L, 20 * C.DEG)
    ninv = rng.uniform(0.5, 2.0, g.npix) * (rng.uniform(size=g.npix) > 0.3)
    prob = solver.Problem(g, L, cl, bl, ninv)
    params, H = solver.low_block(prob, lc)
    assert [p[0] for p in params] == sorted(p[0] for p in params)
    assert all(2 <= l <= lc for (l, _, _, _) in params)        # C_0 = C_1 = 0 are held
    Yd, W, cols = _dense_Y(L, nside)
    pos = {(l, m, 0 if part == "re" else 1): k for k, (_, l, m, part) in enumerate(cols)}
    sel = [pos[(l, m, w)] for (l, m, _, w) in params]
    lcol = np.array([cols[k][1] for k in sel])
    G = Yd[:, sel].T @ (ninv[:, None] * Yd[:, sel])
    ref = np.diag(W[sel] / cl[lcol]) + bl[lcol][:, None] * G * bl[lcol][None, :]
    assert np.max(np.abs(H - ref)) < 1e-11 * np.max(np.abs(ref))


def _teb_problem(nside, L, seed):
    rng = np.random.default_rng(seed)
    g = sht.healpix(nside)
    tt = C.cl_flat(L)
    cl4 = np.stack([tt, 0.05 * tt, 1e-3 * 0.05 * tt, 0.3 * np.sqrt(0.05) * tt])
    mask = rng.uniform(size=g.npix) > 0.25
    ninv = np.stack([rng.uniform(0.5, 2, g.npix) * mask, rng.uniform(0.2, 1, g.npix) * mask])
    return g, solver.Problem(g, L, cl4, C.gauss_beam(L, 0.2), ninv), rng


def test_low_block_teb_symmetric_positive_definite():
    """T, E, B: H is symmetric positive definite (A is self-adjoint in the
    metric of the inner products), and T couples to E only through the
    prior's TE term (no noise coupling between T and Q, U)."""
    g, prob, _ = _teb_problem(4, 8, 31)
    params, H = solver.low_block(prob, 4)
    assert np.max(np.abs(H - H.T)) < 1e-12 * np.max(np.abs(H))
    assert np.linalg.eigvalsh(H).min() > 0
    comp = np.array([c for (_, _, c, _) in params])
    key = [(l, m, w) for (l, m, _, w) in params]
    for i in np.where(comp == 0)[0]:
        for j in np.where(comp != 0)[0]:
            if key[i] == key[j] and comp[j] == 1:
                continue                                   # S^-1_TE at the same (l, m, part)
            assert abs(H[i, j]) < 1e-13 * np.max(np.abs(H))


@pytest.mark.parametrize("ncomp", [1, 3])
def test_two_level_with_every_multipole_is_the_exact_inverse(ncomp):
    """l_c = l_max: the preconditioner is A^-1 itself, so PCG ends after one
    iteration."""
    if ncomp == 1:
        g = sht.healpix(4)
        L = 8
        rng = np.random.default_rng(5)
        ninv = rng.uniform(0.5, 2.0, g.npix) * (rng.uniform(size=g.npix) > 0.3)
        prob = solver.Problem(g, L, C.cl_flat(L), C.gauss_beam(L, 0.2), ninv)
    else:
        g, prob, rng = _teb_problem(4, 6, 7)
        L = 6
    b = prob.matvec(_rand_alm(L, rng, ncomp))
    x, it, hist = solver.pcg(prob, b, 1e-10, 20, precond=solver.two_level_precond(prob, L))
    assert it == 1 and solver.true_residual(prob, x, b) < 1e-11


def test_low_block_azimuthal_noise_is_the_per_m_block():
    """App. A conditions (ring-constant N^-1, nphi >= 2 l_max + 1): H couples
    only equal m and part, and its (l, l') entries at one m are w times the
    per-m block of :func:`solver.azimuthal_block`."""
    L, lc = 12, 6
    g, prob, wr = _azimuthal_problem(L, True)
    params, H = solver.low_block(prob, lc)
    for m in (0, 3):
        lr, A = solver.azimuthal_block(prob, m, wr)
        w = 1.0 if m == 0 else 2.0
        for part in ((0,) if m == 0 else (0, 1)):
            rows = [k for k, (l, mm, _, pw) in enumerate(params) if mm == m and pw == part]
            ls_ = np.array([params[k][0] for k in rows])
            sub = H[np.ix_(rows, rows)]
            ref = w * A[np.ix_(ls_ - m, ls_ - m)]
            assert np.max(np.abs(sub - ref)) < 1e-12 * np.max(np.abs(ref))
    key_m = np.array([p[1] for p in params])
    key_w = np.array([p[3] for p in params])
    off = (key_m[:, None] != key_m[None, :]) | (key_w[:, None] != key_w[None, :])
    assert np.max(np.abs(H[off])) < 1e-12 * np.max(np.abs(H))


def test_two_level_cuts_iterations_under_a_mask():
    """The masked temperature workload at N_side 16: the same solution as
    the diagonal preconditioner, in fewer iterations."""
    p = C.masked_temperature(16, 32)
    g = sht.healpix(16)
    prob = solver.Problem(g, 32, p.cl, p.bl, p.ninv)
    d = sht.alm2map(g, 32, p.signal_alm[0] * p.bl[sht.ls_of(32)]) + p.noise_map[0]
    b = prob.rhs(d, p.w1, p.w2)
    xd, itd, _ = solver.pcg(prob, b, 1e-10, 2000)
    xl, itl, _ = solver.pcg(prob, b, 1e-10, 2000, precond=solver.two_level_precond(prob, 12))
    assert itl < 0.6 * itd
    assert np.max(np.abs(xl - xd)) < 1e-7 * np.max(np.abs(xd))


# ------------------------------------------ azimuthal block preconditioner
def _azimuthal_teb(L):
    """GL grid (nphi >= 2 L + 1), T+E+B with ring-constant N^-1 that differs
    between the hemispheres (T and P), a |b| < 25 deg cut."""
    g = sht.gauss_legendre(L + 1, 2 * L + 2)
    cut = np.abs(g.cth) < math.sin(25 * C.DEG)
    asym = np.where(g.cth > 0, 1.0, 0.4) * (1.0 + 0.5 * g.cth ** 2)
    wT = np.where(cut, 0.0, 1.0 / 5.0 ** 2) * asym
    wP = np.where(cut, 0.0, 1.0 / 7.0 ** 2) * asym[::-1]
    ninv = np.stack([np.repeat(wT, g.nphi), np.repeat(wP, g.nphi)])
    tt = C.cl_flat(L)
    cl4 = np.stack([tt, 0.05 * tt, 1e-3 * 0.05 * tt, 0.3 * np.sqrt(0.05) * tt])
    return g, solver.Problem(g, L, cl4, C.gauss_beam(L, 10 * C.DEG), ninv)


def test_azimuthal_te_block_is_the_operator_restricted_to_m():
    """Brute force: with ring-constant N^-1 on a grid without aliasing, apply
    A to every real unit vector of T and E at one m and read the real T and
    E parts at that m: the result is the (T, E) block of
    :func:`solver.azimuthal_te_block` (including S^-1_TE and held rows)."""
    L, m = 10, 2
    g, prob = _azimuthal_teb(L)
    ls, ms = sht.ls_of(L), sht.ms_of(L)
    idx = np.where(ms == m)[0]
    cols = []
    for c in range(2):
        for i in idx:
            e = np.zeros((3, ls.size), complex)
            e[c, i] = 1.0
            y = prob.matvec(e)
            cols.append(np.concatenate([y[0, idx].real, y[1, idx].real]))
    Abf = np.array(cols).T
    lr, A = solver.azimuthal_te_block(prob, m, L, solver.ring_sum_weights(prob))
    act = np.tile(prob.active[lr], 2)
    sub = np.ix_(act, act)
    assert np.array_equal(lr, ls[idx])
    assert np.max(np.abs(Abf[sub] - A[sub])) < 1e-12 * np.max(np.abs(A))
    # held rows are identity rows of the block (the operator holds them too)
    assert np.allclose(A[~act][:, ~act], np.eye(int((~act).sum())))


def test_azimuthal_precond_is_exact_for_ring_constant_temperature():
    """Temperature with ring-constant N^-1 and no aliasing: with lb = l_max
    the preconditioner is A^-1 and PCG stops after one iteration."""
    L = 16
    g, prob, _ = _azimuthal_problem(L, True)
    rng = np.random.default_rng(3)
    b = prob.matvec(_rand_alm(L, rng))
    x, it, _ = solver.pcg(prob, b, 1e-10, 20, precond=solver.azimuthal_precond(prob, L))
    assert it == 1 and solver.true_residual(prob, x, b) < 1e-11


@pytest.mark.parametrize("ncomp", [1, 3])
def test_azimuthal_precond_cuts_iterations_under_a_mask(ncomp):
    """HEALPix with a latitude cut, holes and hits-weighted noise (T: the
    masked temperature recipe at N_side 16; T+E+B: the T+E+B recipe at
    N_side 8): the same solution as the diagonal preconditioner in far
    fewer iterations."""
    if ncomp == 1:
        p = C.masked_temperature(16, 32)
        ns, L = 16, 32
    else:
        p = C.teb_realizations(1, 8, 16)[0]
        ns, L = 8, 16
    g = sht.healpix(ns)
    prob = solver.Problem(g, L, p.cl, p.bl, p.ninv)
    b = prob.matvec(np.asarray(p.w1).reshape(ncomp, -1))
    xd, itd, _ = solver.pcg(prob, b, 1e-12, 4000)
    xa, ita, _ = solver.pcg(prob, b, 1e-12, 4000, precond=solver.azimuthal_precond(prob, L))
    assert ita < 0.5 * itd, (ita, itd)
    assert np.max(np.abs(xa - xd)) < 1e-7 * np.max(np.abs(xd))

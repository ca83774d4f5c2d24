"""GPU parity of the double-FP32 Legendre path (SHTG_DF64 transforms and the
solver's fp64_arith option) against the FP64 oracle, through the C ABI.

Gates: relative L2 <= 1e-10 against the oracle (the FP64 transforms'
tolerance; double-FP32 rounds at ~2^-47 per operation, the recurrence
carries O(l) of them), the same transform within 1e-12 of the native FP64
kernels at larger sizes, and oracle-evaluated solver residuals <= 1.05 tol
with either arithmetic.  Sizes span several CTAs along the ring-pair and l
axes with ragged tails, more maps than one CTA holds, both geometries, spin
0 and spin 2.
"""
import numpy as np
import pytest

from inputs import configs as C
from oracle import sht as osht
from oracle import solver as osol
from tests._util import rand_alm, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-10
CASES = [("healpix", 16, 40), ("healpix", 32, 64), ("healpix", 300, 400), ("gl", 33, 32), ("gl", 129, 128)]


def _plan_geom(kind, n, L, max_batch=2):
    from paper_2306_15511_gb300 import Plan
    if kind == "healpix":
        return Plan(nside=n, lmax=L, max_batch=max_batch, spin2=True), osht.healpix(n)
    nphi = 2 * L + 2
    return Plan(gauss=(n, nphi), lmax=L, max_batch=max_batch, spin2=True), osht.gauss_legendre(n, nphi)


def _c(x, dt):
    return torch.tensor(np.ascontiguousarray(x), dtype=dt, device="cuda")


@pytest.mark.parametrize("kind,n,L", CASES)
def test_df64_spin0_both_directions(kind, n, L):
    plan, g = _plan_geom(kind, n, L)
    rng = np.random.default_rng(11 * n + L)
    a = rand_alm(L, rng, (2,))
    m = plan.alm2map(_c(a, torch.complex128), double_float=True).cpu().numpy()
    mp = rng.normal(size=(2, g.npix))
    ad = plan.alm2map_adjoint(_c(mp, torch.float64), double_float=True).cpu().numpy()
    for b in range(2):
        assert rel_l2(m[b], osht.alm2map(g, L, a[b])) < TOL
        assert rel_l2(ad[b], osht.alm2map_adjoint(g, L, mp[b])) < TOL


@pytest.mark.parametrize("kind,n,L", CASES[:4])
def test_df64_spin2_both_directions(kind, n, L):
    plan, g = _plan_geom(kind, n, L)
    rng = np.random.default_rng(13 * n + L)
    eb = rand_alm(L, rng, (1, 2))
    qu = plan.alm2map(_c(eb, torch.complex128), spin=2, double_float=True).cpu().numpy()
    Q, U = osht.alm2map_spin2(g, L, eb[0, 0], eb[0, 1])
    assert rel_l2(qu[0], np.stack([Q, U])) < TOL
    mp = rng.normal(size=(1, 2, g.npix))
    ad = plan.alm2map_adjoint(_c(mp, torch.float64), spin=2, double_float=True).cpu().numpy()
    E, B = osht.alm2map_spin2_adjoint(g, L, mp[0, 0], mp[0, 1])
    assert rel_l2(ad[0], np.stack([E, B])) < TOL


def test_df64_vjp_is_weighted_adjoint():
    plan, g = _plan_geom("healpix", 32, 64)
    rng = np.random.default_rng(5)
    gr = rng.normal(size=(1, g.npix))
    v = plan.alm2map_vjp(_c(gr, torch.float64), double_float=True).cpu().numpy()[0]
    ref = osht.alm2map_adjoint(g, 64, gr[0])
    w = np.where(osht.ms_of(64) > 0, 2.0, 1.0)
    assert rel_l2(v, w * ref) < TOL


@pytest.mark.parametrize("spin", [0, 2])
def test_df64_matches_native_fp64_many_maps(spin):
    """N_side 128, l_max 256, 10 maps (two map groups of the transpose, two
    of the synthesis): double-FP32 within 1e-12 of the native FP64 kernels,
    which the FP64 tests pin to the oracle."""
    plan, _ = _plan_geom("healpix", 128, 256, max_batch=10)
    rng = np.random.default_rng(21 + spin)
    shp = (10,) if spin == 0 else (10, 2)
    a = _c(rand_alm(256, rng, shp), torch.complex128)
    m64 = plan.alm2map(a, spin=spin)
    mdf = plan.alm2map(a, spin=spin, double_float=True)
    assert rel_l2(mdf.cpu().numpy(), m64.cpu().numpy()) < 1e-12
    mp = _c(rng.normal(size=tuple(m64.shape)), torch.float64)
    b64 = plan.alm2map_adjoint(mp, spin=spin)
    bdf = plan.alm2map_adjoint(mp, spin=spin, double_float=True)
    assert rel_l2(bdf.cpu().numpy(), b64.cpu().numpy()) < 1e-12


def test_df64_map2alm_takes_fp64_path():
    plan, g = _plan_geom("gl", 33, 32)
    rng = np.random.default_rng(8)
    a = rand_alm(32, rng, (1,))
    mp = _c(osht.alm2map(g, 32, a[0])[None], torch.float64)
    from paper_2306_15511_gb300 import _native as N
    out = torch.empty(1, plan.nalm, dtype=torch.complex128, device="cuda")
    import ctypes as C_
    rc = plan._lib.shtg_map2alm(plan._h, 0, N.DF64, C_.c_void_p(mp.data_ptr()), C_.c_void_p(out.data_ptr()),
                                1, 0, C_.c_void_p(torch.cuda.current_stream().cuda_stream))
    N.check(rc)
    assert rel_l2(out.cpu().numpy()[0], a[0]) < 1e-11   # exact quadrature on the Gauss grid


def _data(p, g):
    L = p.lmax
    ls = osht.ls_of(L)
    T = osht.alm2map(g, L, p.signal_alm[0] * p.bl[ls])
    Q, U = osht.alm2map_spin2(g, L, p.signal_alm[1] * p.bl[ls], p.signal_alm[2] * p.bl[ls])
    return np.stack([T, Q, U]) + p.noise_map


@pytest.mark.parametrize("mode,arith", [("mixed_tc", "fp64"), ("mixed_tc", "df64"), ("fp64", "df64")])
def test_solver_fp64_arith(mode, arith):
    """T+E+B recipe at N_side 32, l_max 64 (masked): the oracle-evaluated
    residual meets 1e-6 with the FP64-accurate steps in either arithmetic."""
    from paper_2306_15511_gb300 import Plan
    p = C.teb_realizations(1, 32, 64)[0]
    g = osht.healpix(p.nside)
    d = _data(p, g)
    prob = osol.Problem(g, p.lmax, p.cl, p.bl, p.ninv)
    b = prob.rhs(d, p.w1, p.w2)
    plan = Plan(nside=p.nside, lmax=p.lmax, spin2=True)
    x, st = plan.cg_sample(p.cl, p.bl, _c(p.ninv, torch.float64), _c(d[None], torch.float64),
                           _c(p.w1[None], torch.complex128), _c(p.w2[None], torch.float64),
                           tol=1e-6, mode=mode, maxiter=4000, fp64_arith=arith)
    assert st["converged"] == 1
    res = osol.true_residual(prob, x.cpu().numpy()[0], b)
    assert res <= 1.05e-6, (res, st)


def test_fp64_arith_rejects_unknown():
    from paper_2306_15511_gb300 import Plan
    plan = Plan(nside=16, lmax=32)
    z = torch.zeros(1, 1, plan.npix, dtype=torch.float64, device="cuda")
    w1 = torch.zeros(1, 1, plan.nalm, dtype=torch.complex128, device="cuda")
    with pytest.raises(ValueError):
        plan.cg_sample(np.ones(33), np.ones(33), torch.ones(plan.npix, dtype=torch.float64, device="cuda"),
                       z, w1, z, fp64_arith="quad")


def test_df64_fullsize_sampled():
    """N_side 1024, l_max 2048 (the benchmark geometry): double-FP32 maps on
    sampled rings (polar, Bluestein, equatorial) and alm at sampled m within
    1e-10 of the oracle computed for those rings / m only, spin 0 and 2."""
    from tests.test_gpu_sht import FULL_RINGS, POLAR_RINGS, _ring_err
    nside, L = 1024, 2048
    plan, g = _plan_geom("healpix", nside, L, max_batch=1)
    rng = np.random.default_rng(31)
    lsc = np.ones(L + 1)
    lsc[1:] = 1.0 / np.sqrt(np.arange(1, L + 1))
    a = rand_alm(L, rng, (1,), lsc)
    m = plan.alm2map(_c(a, torch.complex128), double_float=True).cpu().numpy()[0]
    for rings in (FULL_RINGS, POLAR_RINGS):
        assert _ring_err(m, g, rings, osht.alm2map(g.subset(rings), L, a[0])) < TOL, rings[:3]
    mp = rng.normal(size=(1, g.npix))
    ad = plan.alm2map_adjoint(_c(mp, torch.float64), double_float=True).cpu().numpy()[0]
    mlist = [0, 1, 2, 700, 1500, 2047, 2048]
    sel = np.isin(osht.ms_of(L), mlist)
    assert rel_l2(ad[sel], osht.alm2map_adjoint(g, L, mp[0], mlist=mlist)[sel]) < TOL
    eb = rand_alm(L, rng, (1, 2), lsc)
    qu = plan.alm2map(_c(eb, torch.complex128), spin=2, double_float=True).cpu().numpy()[0]
    for rings in (FULL_RINGS, POLAR_RINGS):
        Q, U = osht.alm2map_spin2(g.subset(rings), L, eb[0, 0], eb[0, 1])
        assert _ring_err(qu, g, rings, np.stack([Q, U])) < TOL, rings[:3]
    mp2 = rng.normal(size=(1, 2, g.npix))
    ad2 = plan.alm2map_adjoint(_c(mp2, torch.float64), spin=2, double_float=True).cpu().numpy()[0]
    ml2 = [0, 1, 2, 1000, 2048]
    E, B = osht.alm2map_spin2_adjoint(g, L, mp2[0, 0], mp2[0, 1], mlist=ml2)
    sel2 = np.isin(osht.ms_of(L), ml2)
    assert rel_l2(ad2[:, sel2], np.stack([E[sel2], B[sel2]])) < TOL

"""Tensor-core Legendre sums (SHTG_TC32, both directions) and the SHTG_CG_MIXED_TC solver
against the FP64 oracle, through the C ABI.

Tolerance of the transform: each product of the l-sum is formed from bf16
hi / lo splits of an FP32 recurrence value x and of an FP32 alm value a,
x = x_hi + x_lo + e_x with |e_x| <= 2^-17 |x| (two round-to-nearest bf16
steps of 8 significant bits), and the lo * lo term (<= 2^-18 |x a|) is
dropped, so each term carries a relative error below 2^-16; the errors of
different terms are independent, which keeps the relative L2 error of a
map below 2^-16 ~ 1.5e-5 on top of the FP32 recurrence's own 3 u l_max.
"""
import numpy as np
import pytest

from inputs import configs as C
from oracle import sht as osht
from oracle import solver as osol
from tests._util import rand_alm, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TC_SPLIT = 2.0 ** -16


def tol_tc(L):
    return TC_SPLIT + max(1e-5, 3.0 * 2.0 ** -24 * L)


CASES = [("healpix", 16, 40), ("healpix", 32, 64), ("healpix", 300, 400), ("gl", 33, 32), ("gl", 129, 128)]


def _plan(kind, n, L, max_batch=2):
    from paper_2306_15511_gb300 import Plan
    if kind == "healpix":
        return Plan(nside=n, lmax=L, max_batch=max_batch, spin2=True), osht.healpix(n)
    return Plan(gauss=(n, 2 * L + 2), lmax=L, max_batch=max_batch, spin2=True), osht.gauss_legendre(n, 2 * L + 2)


@pytest.mark.parametrize("kind,n,L", CASES)
def test_tc_alm2map_spin0(kind, n, L):
    plan, g = _plan(kind, n, L)
    a = rand_alm(L, np.random.default_rng(5 * n + L), (2,))
    m = plan.alm2map(torch.tensor(a, dtype=torch.complex64, device="cuda"), tensor_cores=True).cpu().numpy()
    for b in range(2):
        assert rel_l2(m[b], osht.alm2map(g, L, a[b])) < tol_tc(L)


@pytest.mark.parametrize("kind,n,L", CASES[:4])
def test_tc_alm2map_spin2(kind, n, L):
    plan, g = _plan(kind, n, L)
    eb = rand_alm(L, np.random.default_rng(9 * n + L), (1, 2))
    qu = plan.alm2map(torch.tensor(eb, dtype=torch.complex64, device="cuda"), spin=2,
                      tensor_cores=True).cpu().numpy()
    Q, U = osht.alm2map_spin2(g, L, eb[0, 0], eb[0, 1])
    assert rel_l2(qu[0], np.stack([Q, U])) < tol_tc(L)


def test_tc_more_maps_than_one_cta_holds():
    """11 spin-0 maps and 9 spin-2 map pairs: two CTA map groups (8 + rest)."""
    plan, g = _plan("healpix", 16, 32, max_batch=11)
    rng = np.random.default_rng(21)
    a = rand_alm(32, rng, (11,))
    m = plan.alm2map(torch.tensor(a, dtype=torch.complex64, device="cuda"), tensor_cores=True).cpu().numpy()
    for b in (0, 7, 8, 10):
        assert rel_l2(m[b], osht.alm2map(g, 32, a[b])) < tol_tc(32)
    eb = rand_alm(32, rng, (9, 2))
    qu = plan.alm2map(torch.tensor(eb, dtype=torch.complex64, device="cuda"), spin=2,
                      tensor_cores=True).cpu().numpy()
    for b in (0, 8):
        Q, U = osht.alm2map_spin2(g, 32, eb[b, 0], eb[b, 1])
        assert rel_l2(qu[b], np.stack([Q, U])) < tol_tc(32)


def test_tc_matches_fp32_path():
    """Same FP32 recurrence on both paths: they differ by the split only."""
    plan, _ = _plan("healpix", 64, 128)
    a = torch.tensor(rand_alm(128, np.random.default_rng(2), (2,)), dtype=torch.complex64, device="cuda")
    m32 = plan.alm2map(a).cpu().numpy()
    mtc = plan.alm2map(a, tensor_cores=True).cpu().numpy()
    assert rel_l2(mtc, m32) < TC_SPLIT


def test_tc_fullsize_sampled_rings():
    """N_side 1024, l_max 2048: sampled rings against the oracle, and against
    the FP32 CUDA-core path on the same input (same recurrence values)."""
    nside, L = 1024, 2048
    plan, g = _plan("healpix", nside, L, max_batch=1)
    lsc = np.ones(L + 1)
    lsc[1:] = 1.0 / np.sqrt(np.arange(1, L + 1))
    a = rand_alm(L, np.random.default_rng(13), (1,), lsc)
    at = torch.tensor(a, dtype=torch.complex64, device="cuda")
    m = plan.alm2map(at, tensor_cores=True).cpu().numpy()[0]
    m32 = plan.alm2map(at).cpu().numpy()[0]
    assert rel_l2(m, m32) < TC_SPLIT
    rings = list(range(0, 4095, 97))
    got = np.concatenate([m[g.ofs[r]:g.ofs[r] + g.nphi[r]] for r in rings])
    assert rel_l2(got, osht.alm2map(g.subset(rings), L, a[0])) < tol_tc(L)


def test_tc_fullsize_spin2_sampled_rings():
    """Spin 2 at N_side 1024: the FP32 recurrence itself loses accuracy on the
    polar rings (as in the FP32 tests), so the tensor-core maps are checked
    against the FP32 path on the same input, and against the oracle on the
    sampled rings within the FP32 path's own error plus the split bound."""
    nside, L = 1024, 2048
    plan, g = _plan("healpix", nside, L, max_batch=1)
    lsc = np.ones(L + 1)
    lsc[1:] = 1.0 / np.sqrt(np.arange(1, L + 1))
    eb = rand_alm(L, np.random.default_rng(15), (1, 2), lsc)
    et = torch.tensor(eb, dtype=torch.complex64, device="cuda")
    qu = plan.alm2map(et, spin=2, tensor_cores=True).cpu().numpy()[0]
    qu32 = plan.alm2map(et, spin=2).cpu().numpy()[0]
    assert rel_l2(qu, qu32) < TC_SPLIT
    rings = list(range(0, 4095, 97))
    Q, U = osht.alm2map_spin2(g.subset(rings), L, eb[0, 0], eb[0, 1])
    pick = lambda x: np.concatenate([x[:, g.ofs[r]:g.ofs[r] + g.nphi[r]] for r in rings], axis=-1)
    ref = np.stack([Q, U])
    assert rel_l2(pick(qu), ref) < rel_l2(pick(qu32), ref) + TC_SPLIT


@pytest.mark.parametrize("kind,n,L", CASES)
def test_tc_adjoint_spin0(kind, n, L):
    plan, g = _plan(kind, n, L)
    mp = np.random.default_rng(3 * n + L).normal(size=(2, g.npix))
    a = plan.alm2map_adjoint(torch.tensor(mp, dtype=torch.float32, device="cuda"), tensor_cores=True).cpu().numpy()
    for b in range(2):
        assert rel_l2(a[b], osht.alm2map_adjoint(g, L, mp[b])) < tol_tc(L)


@pytest.mark.parametrize("kind,n,L", CASES[:4])
def test_tc_adjoint_spin2(kind, n, L):
    plan, g = _plan(kind, n, L)
    mp = np.random.default_rng(11 * n + L).normal(size=(1, 2, g.npix))
    ad = plan.alm2map_adjoint(torch.tensor(mp, dtype=torch.float32, device="cuda"), spin=2,
                              tensor_cores=True).cpu().numpy()
    E, B = osht.alm2map_spin2_adjoint(g, L, mp[0, 0], mp[0, 1])
    assert rel_l2(ad[0], np.stack([E, B])) < tol_tc(L)


def test_tc_adjoint_more_maps_and_vjp():
    """11 spin-0 maps and 9 spin-2 pairs (two map groups); the vjp doubles
    the m > 0 outputs."""
    plan, g = _plan("healpix", 16, 32, max_batch=11)
    rng = np.random.default_rng(23)
    mp = rng.normal(size=(11, g.npix))
    t = torch.tensor(mp, dtype=torch.float32, device="cuda")
    a = plan.alm2map_adjoint(t, tensor_cores=True).cpu().numpy()
    for b in (0, 8, 10):
        assert rel_l2(a[b], osht.alm2map_adjoint(g, 32, mp[b])) < tol_tc(32)
    v = plan.alm2map_vjp(t, tensor_cores=True).cpu().numpy()
    w = np.where(osht.ms_of(32) == 0, 1.0, 2.0)
    assert rel_l2(v[3], w * osht.alm2map_adjoint(g, 32, mp[3])) < tol_tc(32)
    qu = rng.normal(size=(9, 2, g.npix))
    e = plan.alm2map_adjoint(torch.tensor(qu, dtype=torch.float32, device="cuda"), spin=2,
                             tensor_cores=True).cpu().numpy()
    for b in (0, 8):
        E, B = osht.alm2map_spin2_adjoint(g, 32, qu[b, 0], qu[b, 1])
        assert rel_l2(e[b], np.stack([E, B])) < tol_tc(32)


def test_tc_adjoint_matches_fp32_path():
    plan, g = _plan("healpix", 64, 128)
    mp = torch.tensor(np.random.default_rng(4).normal(size=(2, g.npix)), dtype=torch.float32, device="cuda")
    a32 = plan.alm2map_adjoint(mp).cpu().numpy()
    atc = plan.alm2map_adjoint(mp, tensor_cores=True).cpu().numpy()
    assert rel_l2(atc, a32) < TC_SPLIT


def test_tc_adjoint_fullsize_sampled_m():
    """N_side 1024, l_max 2048: sampled m (polar and equatorial starts, the
    last m) of the tensor-core transpose against the FP32 path on the same
    input and against the oracle.  At low m the spin-2 FP32 recurrence loses
    ~1e-3 on the polar rings (m = 2: 9e-4 on the FP32 path), so the spin-2
    oracle gate is the FP32 path's own error plus the split bound."""
    nside, L = 1024, 2048
    plan, g = _plan("healpix", nside, L, max_batch=1)
    rng = np.random.default_rng(14)
    mp = rng.normal(size=(1, g.npix))
    mt = torch.tensor(mp, dtype=torch.float32, device="cuda")
    ad = plan.alm2map_adjoint(mt, tensor_cores=True).cpu().numpy()[0]
    assert rel_l2(ad, plan.alm2map_adjoint(mt).cpu().numpy()[0]) < TC_SPLIT
    mlist = [0, 1, 2, 511, 512, 700, 1500, 2047, 2048]
    ref = osht.alm2map_adjoint(g, L, mp[0], mlist=mlist)
    sel = np.isin(osht.ms_of(L), mlist)
    assert rel_l2(ad[sel], ref[sel]) < tol_tc(L)
    qu = rng.normal(size=(1, 2, g.npix))
    qt = torch.tensor(qu, dtype=torch.float32, device="cuda")
    e = plan.alm2map_adjoint(qt, spin=2, tensor_cores=True).cpu().numpy()[0]
    e32 = plan.alm2map_adjoint(qt, spin=2).cpu().numpy()[0]
    assert rel_l2(e, e32) < TC_SPLIT
    ml2 = [0, 2, 1000, 2048]
    E, B = osht.alm2map_spin2_adjoint(g, L, qu[0, 0], qu[0, 1], mlist=ml2)
    sel = np.isin(osht.ms_of(L), ml2)
    r2 = np.stack([E[sel], B[sel]])
    assert rel_l2(e[:, sel], r2) < rel_l2(e32[:, sel], r2) + TC_SPLIT


def _data(p, g):
    L = p.lmax
    ls = osht.ls_of(L)
    if p.ncomp == 1:
        return (osht.alm2map(g, L, p.signal_alm[0] * p.bl[ls]) + p.noise_map[0])[None]
    T = osht.alm2map(g, L, p.signal_alm[0] * p.bl[ls])
    Q, U = osht.alm2map_spin2(g, L, p.signal_alm[1] * p.bl[ls], p.signal_alm[2] * p.bl[ls])
    return np.stack([T, Q, U]) + p.noise_map


def _cuda(x, dt):
    return torch.tensor(np.ascontiguousarray(x), dtype=dt, device="cuda")


def test_mixed_tc_solve_masked():
    """Masked temperature workload at N_side 128, l_max 256 (mask + hits noise): the
    tensor-core inner solver reaches the FP64 residual gate."""
    from paper_2306_15511_gb300 import Plan
    p = C.masked_temperature(128, 256)
    g = osht.healpix(128)
    d = _data(p, g)
    prob = osol.Problem(g, p.lmax, p.cl, p.bl, p.ninv)
    b = prob.rhs(d, p.w1, p.w2)
    plan = Plan(nside=128, lmax=256)
    x, st = plan.cg_sample(p.cl, p.bl, _cuda(p.ninv, torch.float64), _cuda(d[None], torch.float64),
                           _cuda(p.w1[None], torch.complex128), _cuda(p.w2[None], torch.float64),
                           tol=1e-6, mode="mixed_tc", maxiter=3000)
    assert st["converged"] == 1
    assert osol.true_residual(prob, x.cpu().numpy()[0], b) <= 1.05e-6


def test_mixed_tc_teb():
    from paper_2306_15511_gb300 import Plan
    p = C.teb_realizations(2, 16, 32)
    g = osht.healpix(16)
    plan = Plan(nside=16, lmax=32, max_batch=2, spin2=True)
    ds = np.stack([_data(q, g) for q in p])
    w1 = np.stack([q.w1 for q in p])
    w2 = np.stack([q.w2 for q in p])
    x, st = plan.cg_sample(p[0].cl, p[0].bl, _cuda(p[0].ninv, torch.float64), _cuda(ds, torch.float64),
                           _cuda(w1, torch.complex128), _cuda(w2, torch.float64), tol=1e-6,
                           mode="mixed_tc", maxiter=3000)
    assert st["converged"] == 1
    prob = osol.Problem(g, 32, p[0].cl, p[0].bl, p[0].ninv)
    xh = x.cpu().numpy()
    for k in range(2):
        assert osol.true_residual(prob, xh[k], prob.rhs(ds[k], w1[k], w2[k])) <= 1.05e-6

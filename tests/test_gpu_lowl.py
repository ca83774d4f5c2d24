"""Two-level preconditioner (exact inverse on l <= l_c plus the diagonal
above) through the C ABI, against the FP64 oracle.

- The low block H of shtg_lowl_block against the oracle's H read off its
  operator column by column (temperature with a mask and holes; T+E+B with
  a random mask; a C_l scale), parameter lists equal, entries to 1e-10.
- l_c = l_max makes the preconditioner the exact inverse: the FP64 PCG stops
  after one iteration (T and T+E+B).
- Masked workloads: the same oracle-evaluated residual as the diagonal
  preconditioner in far fewer iterations (FP64 and both mixed forms; the
  N_side 256 / l_max 512 masked temperature workload; T+E+B at N_side 64);
  graph replays equal eager launches bit for bit; split right-hand sides and
  C_l scales.
"""
import numpy as np
import pytest

from inputs import configs as C
from oracle import sht as osht
from oracle import solver as osol

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _cuda(x, dt):
    return torch.tensor(np.ascontiguousarray(x), dtype=dt, device="cuda")


def _data(p, g):
    ls = osht.ls_of(p.lmax)
    if p.ncomp == 1:
        return (osht.alm2map(g, p.lmax, p.signal_alm[0] * p.bl[ls]) + p.noise_map[0])[None]
    T = osht.alm2map(g, p.lmax, p.signal_alm[0] * p.bl[ls])
    Q, U = osht.alm2map_spin2(g, p.lmax, p.signal_alm[1] * p.bl[ls], p.signal_alm[2] * p.bl[ls])
    return np.stack([T, Q, U]) + p.noise_map


def _teb_random_mask(nside, L, seed):
    rng = np.random.default_rng(seed)
    npix = 12 * nside * nside
    tt = C.cl_flat(L)
    cl4 = np.stack([tt, 0.05 * tt, 1e-3 * 0.05 * tt, 0.3 * np.sqrt(0.05) * tt])
    mask = rng.uniform(size=npix) > 0.25
    ninv = np.stack([rng.uniform(0.5, 2, npix) * mask, rng.uniform(0.2, 1, npix) * mask])
    return cl4, C.gauss_beam(L, 0.2), ninv


def _compare_block(plan, cl, bl, ninv, ncomp, lc, g, L, scale=None):
    H, par = plan.lowl_block(cl, bl, _cuda(ninv, torch.float64), ncomp=ncomp, lowl_lmax=lc,
                             cl_scale=None if scale is None else [scale])
    clo = np.asarray(cl) * (1.0 if scale is None else scale)
    prob = osol.Problem(g, L, clo, bl, ninv)
    params, Href = osol.low_block(prob, lc)
    assert [tuple(int(v) for v in row) for row in par] == params
    err = np.max(np.abs(H - Href)) / np.max(np.abs(Href))
    print(f"low block ncomp {ncomp} l_c {lc} (n = {len(params)}): max error {err:.2e}")
    assert err < 1e-10, err


def test_lowl_block_temperature_vs_oracle():
    from paper_2306_15511_gb300 import Plan
    p = C.masked_temperature(8, 16)
    g = osht.healpix(8)
    plan = Plan(nside=8, lmax=16)
    _compare_block(plan, p.cl, p.bl, p.ninv, 1, 7, g, 16)
    _compare_block(plan, p.cl, p.bl, p.ninv, 1, 16, g, 16, scale=1.7)   # the whole space, a C_l scale


def test_lowl_block_teb_vs_oracle():
    from paper_2306_15511_gb300 import Plan
    cl4, bl, ninv = _teb_random_mask(4, 10, 3)
    plan = Plan(nside=4, lmax=10, spin2=True)
    _compare_block(plan, cl4, bl, ninv, 3, 5, osht.healpix(4), 10)
    # the kept Gram matrix is rebuilt when N^-1 changes
    _compare_block(plan, cl4, bl, 0.5 * ninv[::-1].copy(), 3, 5, osht.healpix(4), 10)


@pytest.mark.parametrize("ncomp", [1, 3])
def test_lowl_whole_space_is_exact(ncomp):
    """l_c = l_max: z = A^-1 r, so the FP64 PCG converges in one iteration."""
    from paper_2306_15511_gb300 import Plan
    ns, L = 4, 10
    g = osht.healpix(ns)
    rng = np.random.default_rng(11)
    if ncomp == 1:
        cl = C.cl_flat(L)
        bl = C.gauss_beam(L, 0.2)
        ninv = rng.uniform(0.5, 2.0, g.npix) * (rng.uniform(size=g.npix) > 0.3)
    else:
        cl, bl, ninv = _teb_random_mask(ns, L, 5)
    plan = Plan(nside=ns, lmax=L, spin2=ncomp == 3)
    d = rng.normal(size=(1, ncomp, g.npix))
    w1 = np.zeros((1, ncomp, (L + 1) * (L + 2) // 2), complex)
    w2 = np.zeros((1, ncomp, g.npix))
    x, st = plan.cg_sample(cl, bl, _cuda(ninv, torch.float64), _cuda(d, torch.float64),
                           _cuda(w1, torch.complex128), _cuda(w2, torch.float64), tol=1e-10, mode="fp64",
                           precond="lowl", lowl_lmax=L, maxiter=10, check_every=1)
    prob = osol.Problem(g, L, cl, bl, ninv)
    res = osol.true_residual(prob, x.cpu().numpy()[0], prob.rhs(d[0], w1[0], w2[0]))
    print(f"whole-space low block ncomp {ncomp}: {st['iterations']} iterations, oracle residual {res:.2e}")
    assert st["iterations"] <= 2 and res < 1e-10, (st, res)


@pytest.mark.parametrize("mode", ["fp64", "mixed", "mixed_tc"])
def test_lowl_masked_n64(mode):
    """Masked temperature at N_side 64 / l_max 128 to 1e-8: the two-level
    preconditioner (l_c = 32) reaches the oracle-evaluated residual in under
    half the diagonal preconditioner's iterations."""
    from paper_2306_15511_gb300 import Plan
    p = C.masked_temperature(64, 128)
    g = osht.healpix(64)
    d = _data(p, g)
    plan = Plan(nside=64, lmax=128)
    args = (p.cl, p.bl, _cuda(p.ninv, torch.float64), _cuda(d[None], torch.float64),
            _cuda(p.w1[None], torch.complex128), _cuda(p.w2[None], torch.float64))
    prob = osol.Problem(g, 128, p.cl, p.bl, p.ninv)
    b = prob.rhs(d, p.w1, p.w2)
    _, sd = plan.cg_sample(*args, tol=1e-8, mode=mode, maxiter=8000)
    x, sl = plan.cg_sample(*args, tol=1e-8, mode=mode, maxiter=8000, precond="lowl", lowl_lmax=32)
    res = osol.true_residual(prob, x.cpu().numpy()[0], b)
    print(f"masked N_side 64 {mode}: diagonal {sd['iterations']} iterations, two-level {sl['iterations']} "
          f"(setup {sl['ms_setup']:.1f} ms), oracle residual {res:.2e}")
    assert sl["converged"] == 1 and res <= 1.05e-8
    assert sl["iterations"] < 0.5 * sd["iterations"]


def test_lowl_masked_full_size():
    """The N_side 256 / l_max 512 masked temperature workload with the
    tensor-core mixed solver to 1e-6: oracle residual <= 1.05e-6 in under
    half the diagonal preconditioner's iterations; to 1e-9 the solution is
    within 1e-5 of the oracle's converged one."""
    import os
    from paper_2306_15511_gb300 import Plan
    from tests._util import rel_l2
    golden = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "masked_t_n256_l512_x.npy")
    p = C.masked_temperature(256, 512)
    g = osht.healpix(256)
    d = _data(p, g)
    plan = Plan(nside=256, lmax=512)
    args = (p.cl, p.bl, _cuda(p.ninv, torch.float64), _cuda(d[None], torch.float64),
            _cuda(p.w1[None], torch.complex128), _cuda(p.w2[None], torch.float64))
    prob = osol.Problem(g, 512, p.cl, p.bl, p.ninv)
    b = prob.rhs(d, p.w1, p.w2)
    _, sd = plan.cg_sample(*args, tol=1e-6, mode="mixed_tc", maxiter=12000, check_every=8)
    for tol in (1e-6, 1e-9):
        x, sl = plan.cg_sample(*args, tol=tol, mode="mixed_tc", maxiter=12000, check_every=8, precond="lowl")
        xh = x.cpu().numpy()[0]
        res = osol.true_residual(prob, xh, b)
        err = rel_l2(xh[0], np.load(golden))
        print(f"masked N_side 256 two-level mixed_tc tol {tol:.0e}: {sl['iterations']} iterations "
              f"(diagonal at 1e-6: {sd['iterations']}), setup {sl['ms_setup']:.1f} ms, solve "
              f"{sl['ms_solve']:.1f} ms, oracle residual {res:.3e}, error vs oracle solution {err:.3e}")
        assert sl["converged"] == 1 and res <= 1.05 * tol
        if tol == 1e-6:
            assert sl["iterations"] < 0.5 * sd["iterations"]
        else:
            assert err <= 1e-5


def test_lowl_teb_n64():
    """T+E+B at N_side 64 / l_max 128 (mask and holes of the T+E+B recipe),
    two realizations, tensor-core mixed solver to 1e-6: oracle residual and
    fewer iterations than the diagonal preconditioner."""
    from paper_2306_15511_gb300 import Plan
    ps = C.teb_realizations(2, 64, 128)
    g = osht.healpix(64)
    ds = np.stack([_data(q, g) for q in ps])
    plan = Plan(nside=64, lmax=128, max_batch=2, spin2=True)
    args = (ps[0].cl, ps[0].bl, _cuda(ps[0].ninv, torch.float64), _cuda(ds, torch.float64),
            _cuda(np.stack([q.w1 for q in ps]), torch.complex128), _cuda(np.stack([q.w2 for q in ps]), torch.float64))
    _, sd = plan.cg_sample(*args, tol=1e-6, mode="mixed_tc", maxiter=8000)
    x, sl = plan.cg_sample(*args, tol=1e-6, mode="mixed_tc", maxiter=8000, precond="lowl", lowl_lmax=24)
    prob = osol.Problem(g, 128, ps[0].cl, ps[0].bl, ps[0].ninv)
    xh = x.cpu().numpy()
    worst = max(osol.true_residual(prob, xh[k], prob.rhs(ds[k], ps[k].w1, ps[k].w2)) for k in range(2))
    print(f"T+E+B N_side 64: diagonal {sd['iterations']} iterations, two-level {sl['iterations']}, "
          f"worst oracle residual {worst:.2e}")
    assert sl["converged"] == 1 and worst <= 1.05e-6
    assert sl["iterations"] < sd["iterations"]


def test_lowl_graph_replay_split_and_scales():
    """Graph replay equals eager launches bit for bit with the low block in
    the iteration; split right-hand sides and per-realization C_l scales
    converge to the oracle residual."""
    from paper_2306_15511_gb300 import Plan
    p = C.masked_temperature(32, 64)
    g = osht.healpix(32)
    d = _data(p, g)
    plan = Plan(nside=32, lmax=64, max_batch=4)
    ds = np.stack([d, 0.5 * d])
    w1 = np.stack([p.w1, -p.w1])
    w2 = np.stack([p.w2, 0.3 * p.w2])
    args = (p.cl, p.bl, _cuda(p.ninv, torch.float64), _cuda(ds, torch.float64),
            _cuda(w1, torch.complex128), _cuda(w2, torch.float64))
    kw = dict(tol=1e-7, mode="mixed", maxiter=4000, check_every=8, precond="lowl", lowl_lmax=20)
    plan.cg_sample(*args, **kw)   # autotuner trials
    xg, sg = plan.cg_sample(*args, graphs=True, **kw)
    xe, se = plan.cg_sample(*args, graphs=False, **kw)
    assert sg["converged"] == 1 and sg["iterations"] == se["iterations"]
    assert torch.equal(xg, xe)
    # split mean field / fluctuation with two C_l scales
    sc = [1.0, 1.3]
    xs, ss = plan.cg_sample(*args, split=True, cl_scale=sc, **kw)
    assert ss["converged"] == 1
    xs = xs.cpu().numpy()
    for k in range(2):
        prob = osol.Problem(g, 64, p.cl * sc[k], p.bl, p.ninv)
        bm, bf = prob.rhs_parts(ds[k], w1[k], w2[k])
        for part, bb in ((0, bm), (1, bf)):
            res = osol.true_residual(prob, xs[part, k], bb)
            assert res <= 1.05e-7, (k, part, res)

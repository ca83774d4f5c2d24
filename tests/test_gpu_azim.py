"""Azimuthal block preconditioner (App. A's per-m blocks of T and E from the
ring sums of N^-1, exact inverse per m, the diagonal elsewhere) through the
C ABI, against the FP64 oracle.

- One application z = M^-1 r (shtg_precond_apply, FP64 factors) against
  `oracle.solver.azimuthal_precond` element by element: temperature with a
  mask, holes and hits-weighted noise; T+E+B with a random mask; several
  block ranges l_b (all multipoles, and fewer, so the diagonal takes the
  rest); a C_l scale; again after N^-1 changes (the kept Gram matrices must
  be rebuilt).
- Ring-constant N^-1 on a Gauss-Legendre grid with l_b = l_max: the
  preconditioner is A^-1, so the FP64 PCG stops after one iteration.
- Masked workloads: the oracle-evaluated residual in far fewer iterations
  than the diagonal preconditioner (FP64 and both mixed forms at N_side 64;
  the N_side 256 / l_max 512 masked temperature workload to 1e-6 and 1e-9
  against the stored oracle solution; T+E+B at N_side 64); graph replay
  bit-identical to eager launches; split right-hand sides with C_l scales.
"""
import math
import os

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


def _rand_alm(L, rng, nb, nc):
    P = (L + 1) * (L + 2) // 2
    a = rng.normal(size=(nb, nc, P)) + 1j * rng.normal(size=(nb, nc, P))
    a[..., osht.ms_of(L) == 0] = a[..., osht.ms_of(L) == 0].real
    return a


def _compare(plan, cl, bl, ninv, L, g, lb, ncomp, scale=None, seed=0):
    rng = np.random.default_rng(seed)
    r = _rand_alm(L, rng, 2, ncomp)
    z = plan.precond_apply(cl, bl, _cuda(ninv, torch.float64), _cuda(r, torch.complex128), precond="azim",
                           block_lmax=lb, cl_scale=None if scale is None else [scale, scale]).cpu().numpy()
    prob = osol.Problem(g, L, np.asarray(cl) * (1.0 if scale is None else scale), bl, ninv)
    ap = osol.azimuthal_precond(prob, lb)
    # rows of the blocks (T, E at l <= l_b): FP64 factors, against the
    # oracle's inverse; the rest: the diagonal preconditioner, whose ring
    # sums of g_lm the library forms in FP32 (relative rounding ~1e-7)
    blk = np.zeros((ncomp, r.shape[2]), bool)
    blk[:min(ncomp, 2)] = osht.ls_of(L) <= lb
    eb = ed = 0.0
    for b in range(2):
        zr = ap(r[b])
        sc = np.max(np.abs(zr))
        eb = max(eb, np.max(np.abs(z[b] - zr)[blk]) / sc)
        if (~blk).any():
            ed = max(ed, np.max(np.abs(z[b] - zr)[~blk]) / sc)
    print(f"azimuthal precond ncomp {ncomp} l_b {lb}: block rows {eb:.2e}, diagonal rows {ed:.2e}")
    assert eb < 1e-9, eb
    assert ed < 1e-5, ed


def test_azim_apply_temperature_vs_oracle():
    from paper_2306_15511_gb300 import Plan
    p = C.masked_temperature(8, 16)
    g = osht.healpix(8)
    plan = Plan(nside=8, lmax=16, max_batch=2)
    _compare(plan, p.cl, p.bl, p.ninv, 16, g, 16, 1)
    _compare(plan, p.cl, p.bl, p.ninv, 16, g, 9, 1, scale=1.6, seed=1)
    _compare(plan, p.cl, p.bl, 0.5 * p.ninv[::-1].copy(), 16, g, 9, 1, seed=2)   # N^-1 changed


def test_azim_apply_teb_vs_oracle():
    from paper_2306_15511_gb300 import Plan
    rng = np.random.default_rng(4)
    ns, L = 4, 10
    g = osht.healpix(ns)
    tt = C.cl_flat(L)
    cl4 = np.stack([tt, 0.05 * tt, 1e-3 * 0.05 * tt, 0.3 * np.sqrt(0.05) * tt])
    mask = rng.uniform(size=g.npix) > 0.25
    ninv = np.stack([rng.uniform(0.5, 2, g.npix) * mask, rng.uniform(0.2, 1, g.npix) * mask])
    plan = Plan(nside=ns, lmax=L, max_batch=2, spin2=True)
    _compare(plan, cl4, C.gauss_beam(L, 0.2), ninv, L, g, L, 3)
    _compare(plan, cl4, C.gauss_beam(L, 0.2), ninv, L, g, 6, 3, seed=3)


def test_azim_ring_constant_temperature_is_exact():
    """Gauss-Legendre grid (nphi >= 2 l_max + 1), N^-1 constant along rings
    and different between the hemispheres: one FP64 PCG iteration."""
    from paper_2306_15511_gb300 import Plan
    L = 24
    nr, nphi = L + 1, 2 * L + 2
    g = osht.gauss_legendre(nr, nphi)
    wr = np.where(np.abs(g.cth) < math.sin(25 * C.DEG), 0.0, 1.0 / 25.0) * np.where(g.cth > 0, 1.0, 0.35)
    ninv = np.repeat(wr, g.nphi)
    cl, bl = C.cl_flat(L), C.gauss_beam(L, 10 * C.DEG)
    plan = Plan(gauss=(nr, nphi), lmax=L)
    rng = np.random.default_rng(5)
    d = rng.normal(size=(1, 1, g.npix))
    P = (L + 1) * (L + 2) // 2
    x, st = plan.cg_sample(cl, bl, _cuda(ninv, torch.float64), _cuda(d, torch.float64),
                           _cuda(np.zeros((1, 1, P), complex), torch.complex128),
                           _cuda(np.zeros((1, 1, g.npix)), torch.float64), tol=1e-10, mode="fp64",
                           precond="azim", block_lmax=L, maxiter=10, check_every=1)
    prob = osol.Problem(g, L, cl, bl, ninv)
    res = osol.true_residual(prob, x.cpu().numpy()[0], prob.rhs(d[0], np.zeros((1, P)), np.zeros((1, g.npix))))
    print(f"ring-constant N^-1, azimuthal blocks: {st['iterations']} iterations, oracle residual {res:.2e}")
    assert st["iterations"] <= 2 and res < 1e-10, (st, res)


@pytest.mark.parametrize("mode", ["fp64", "mixed", "mixed_tc"])
def test_azim_masked_n64(mode):
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
    x, sa = plan.cg_sample(*args, tol=1e-8, mode=mode, maxiter=8000, precond="azim")
    res = osol.true_residual(prob, x.cpu().numpy()[0], b)
    print(f"masked N_side 64 {mode}: diagonal {sd['iterations']} iterations, azimuthal {sa['iterations']} "
          f"(setup {sa['ms_setup']:.1f} ms), oracle residual {res:.2e}")
    assert sa["converged"] == 1 and res <= 1.05e-8
    assert sa["iterations"] < 0.25 * sd["iterations"]


def test_azim_masked_full_size():
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
        x, sa = plan.cg_sample(*args, tol=tol, mode="mixed_tc", maxiter=12000, check_every=8, precond="azim")
        xh = x.cpu().numpy()[0]
        res = osol.true_residual(prob, xh, b)
        err = rel_l2(xh[0], np.load(golden))
        print(f"masked N_side 256 azimuthal mixed_tc tol {tol:.0e}: {sa['iterations']} iterations (diagonal at "
              f"1e-6: {sd['iterations']}), setup {sa['ms_setup']:.1f} ms, solve {sa['ms_solve']:.1f} ms, "
              f"oracle residual {res:.3e}, error vs oracle solution {err:.3e}")
        assert sa["converged"] == 1 and res <= 1.05 * tol
        if tol == 1e-6:
            assert sa["iterations"] < 0.25 * sd["iterations"]
        else:
            assert err <= 1e-5


def test_azim_teb_n64():
    from paper_2306_15511_gb300 import Plan
    ps = C.teb_realizations(2, 64, 128)
    g = osht.healpix(64)
    ds = np.stack([_data(q, g) for q in ps])
    plan = Plan(nside=64, lmax=128, max_batch=2, spin2=True)
    args = (ps[0].cl, ps[0].bl, _cuda(ps[0].ninv, torch.float64), _cuda(ds, torch.float64),
            _cuda(np.stack([q.w1 for q in ps]), torch.complex128), _cuda(np.stack([q.w2 for q in ps]), torch.float64))
    _, sd = plan.cg_sample(*args, tol=1e-6, mode="mixed_tc", maxiter=8000)
    x, sa = plan.cg_sample(*args, tol=1e-6, mode="mixed_tc", maxiter=8000, precond="azim")
    prob = osol.Problem(g, 128, ps[0].cl, ps[0].bl, ps[0].ninv)
    xh = x.cpu().numpy()
    worst = max(osol.true_residual(prob, xh[k], prob.rhs(ds[k], ps[k].w1, ps[k].w2)) for k in range(2))
    print(f"T+E+B N_side 64: diagonal {sd['iterations']} iterations, azimuthal {sa['iterations']}, "
          f"worst oracle residual {worst:.2e}")
    assert sa["converged"] == 1 and worst <= 1.05e-6
    assert sa["iterations"] < 0.5 * sd["iterations"]


def test_azim_graph_replay_split_and_scales():
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
    kw = dict(tol=1e-7, mode="mixed", maxiter=4000, check_every=4, precond="azim", block_lmax=48)
    plan.cg_sample(*args, **kw)   # autotuner trials
    xg, sg = plan.cg_sample(*args, graphs=True, **kw)
    xe, se = plan.cg_sample(*args, graphs=False, **kw)
    assert sg["converged"] == 1 and sg["iterations"] == se["iterations"]
    assert torch.equal(xg, xe)
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


@pytest.mark.parametrize("precond", ["azim", "lowl"])
def test_chains_with_block_preconditioners(precond):
    """Two geometries in one chains call (each group on its plan's own
    non-blocking stream, concurrently): the preconditioners' workspaces are
    set up on the group's stream and every chain reaches the oracle residual."""
    from paper_2306_15511_gb300 import Plan, chains_sample
    req, refs = [], []
    for ns, L in ((32, 64), (32, 95)):
        p = C.masked_temperature(ns, L, seed=7)
        g = osht.healpix(ns)
        d = _data(p, g)
        plan = Plan(nside=ns, lmax=L, max_batch=2)
        ds = np.stack([d, 0.7 * d])
        w1 = np.stack([p.w1, -p.w1])
        w2 = np.stack([p.w2, 0.5 * p.w2])
        req.append({"plan": plan, "cl": p.cl, "bl": p.bl, "ninv": _cuda(p.ninv, torch.float64),
                    "d": _cuda(ds, torch.float64), "w1": _cuda(w1, torch.complex128),
                    "w2": _cuda(w2, torch.float64), "cl_scale": [1.0, 1.2]})
        refs.append((g, p, ds, w1, w2))
    res = chains_sample(req, tol=1e-6, mode="mixed_tc", maxiter=3000, precond=precond)
    for (x, st), (g, p, ds, w1, w2), grp in zip(res, refs, req):
        assert st["converged"] == 1, st
        xh = x.cpu().numpy()
        for k, sc in enumerate(grp["cl_scale"]):
            prob = osol.Problem(g, p.lmax, p.cl * sc, p.bl, p.ninv)
            r = osol.true_residual(prob, xh[k], prob.rhs(ds[k], w1[k], w2[k]))
            assert r <= 1.05e-6, (p.lmax, k, r)


def test_mixed_stage_ends_at_its_rounding_floor():
    """A latitude-band mask with uniform noise makes the azimuthal blocks
    nearly the exact inverse: the FP32 stage reaches its rounding floor in one
    or two iterations, where a curvature made of rounding noise ends the
    stage (no failure); the FP64 replacement then confirms convergence."""
    from paper_2306_15511_gb300 import Plan
    ns, L = 32, 64
    g = osht.healpix(ns)
    z, _ = C.pixel_centres(ns)
    ninv = np.where(np.abs(z) < math.sin(15 * C.DEG), 0.0, 1.0 / 15.0 ** 2)
    cl, bl = C.cl_flat(L), C.gauss_beam(L, 60.0 / ns * C.DEG)
    rng = np.random.default_rng(9)
    nb = 4
    P = (L + 1) * (L + 2) // 2
    d = rng.normal(size=(nb, 1, g.npix)) * 15.0
    w1 = _rand_alm(L, rng, nb, 1)
    w2 = rng.normal(size=(nb, 1, g.npix))
    plan = Plan(nside=ns, lmax=L, max_batch=nb)
    prob = osol.Problem(g, L, cl, bl, ninv)
    for mode in ("mixed", "mixed_tc"):
        x, st = plan.cg_sample(cl, bl, _cuda(ninv, torch.float64), _cuda(d, torch.float64),
                               _cuda(w1, torch.complex128), _cuda(w2, torch.float64), tol=1e-6, mode=mode,
                               maxiter=500, precond="azim")
        xh = x.cpu().numpy()
        worst = max(osol.true_residual(prob, xh[k], prob.rhs(d[k], w1[k], w2[k])) for k in range(nb))
        print(f"latitude band, azimuthal blocks, {mode}: {st['iterations']} iterations, "
              f"{st['outer_steps']} replacements, oracle residual {worst:.2e}")
        assert st["converged"] == 1 and worst <= 1.05e-6
    assert P > 0

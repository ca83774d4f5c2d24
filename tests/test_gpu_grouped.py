"""Chains of several geometries with one launch per stage of the FP32 PCG
iteration (SHTG_GROUPED of shtg_cg_sample_chains), through the C ABI,
against the FP64 oracle.

- The mixed-geometry chains recipe, two chains of each of its six
  geometries (N_side 64, 128, 256; l_max 2 N_side and 3 N_side - 1), so the
  grouped Legendre launches span three ring counts and six l_max and the
  grouped ring stage spans the generic and the fixed-length launch classes:
  every chain's oracle-evaluated residual <= 1.05e-6, with the diagonal and
  with the azimuthal block preconditioner.
- T+E+B realizations in two geometries (spin-0 and spin-2 grouped launches).
- The captured iteration replayed as a CUDA graph matches eager launches
  (to FP32 rounding order).
- Refused options: the two-level preconditioner and the FP64 mode.
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


def _chain_groups(per_geometry=2):
    keep = {}
    for ch in C.mixed_geometry_chains(64):
        if len(keep.setdefault((ch.nside, ch.lmax), [])) < per_geometry:
            keep[(ch.nside, ch.lmax)].append(ch)
    return dict(sorted(keep.items()))


def _chain_requests(groups):
    from paper_2306_15511_gb300 import Plan
    req, refs = [], []
    for (ns, L), chs in groups.items():
        g = osht.healpix(ns)
        ls = osht.ls_of(L)
        d = np.stack([(osht.alm2map(g, L, ch.signal_alm[0] * ch.bl[ls]) + ch.noise_map[0])[None] for ch in chs])
        plan = Plan(nside=ns, lmax=L, max_batch=len(chs))
        req.append({"plan": plan, "cl": C.cl_flat(L), "bl": chs[0].bl, "ninv": _cuda(chs[0].ninv, torch.float64),
                    "d": _cuda(d, torch.float64), "w1": _cuda(np.stack([ch.w1 for ch in chs]), torch.complex128),
                    "w2": _cuda(np.stack([ch.w2 for ch in chs]), torch.float64),
                    "cl_scale": [ch.extra["amp"] for ch in chs]})
        refs.append((g, chs, d))
    return req, refs


@pytest.fixture(scope="module")
def chains():
    groups = _chain_groups()
    assert sorted(groups) == [(64, 128), (64, 191), (128, 256), (128, 383), (256, 512), (256, 767)]
    return _chain_requests(groups)


@pytest.mark.parametrize("precond", ["diag", "azim"])
def test_grouped_chains_vs_oracle(chains, precond):
    from paper_2306_15511_gb300 import chains_sample
    req, refs = chains
    res = chains_sample(req, tol=1e-6, mode="mixed", maxiter=4000, precond=precond, grouped=True)
    iters = [st["iterations"] for _, st in res]
    print(f"grouped chains, {precond}: FP32 iterations per group {iters}, "
          f"FP64-accurate applications {[st['fp64_matvecs'] for _, st in res]}")
    for (x, st), (g, chs, d) in zip(res, refs):
        assert st["converged"] == 1, st
        xh = x.cpu().numpy()
        for k, ch in enumerate(chs):
            prob = osol.Problem(g, ch.lmax, ch.cl, ch.bl, ch.ninv)
            r = osol.true_residual(prob, xh[k], prob.rhs(d[k], ch.w1, ch.w2))
            assert r <= 1.05e-6, (ch.name, ch.nside, ch.lmax, r, st)


def test_grouped_graph_replay_matches_eager(chains):
    """The captured grouped iteration replayed as a CUDA graph against eager
    launches of the same kernels.  Not bit for bit: the FP32 transpose adds
    its warps' partial sums into shared memory with atomic additions, whose
    order changes when CTAs of other geometries share the SM, so the two
    runs differ by FP32 rounding; both converge and agree far below the
    mixed form's 1e-5."""
    from paper_2306_15511_gb300 import chains_sample
    from tests._util import rel_l2
    req, _ = chains
    sub = req[:3]
    a = chains_sample(sub, tol=1e-6, mode="mixed", maxiter=4000, precond="azim", grouped=True, graphs=True)
    b = chains_sample(sub, tol=1e-6, mode="mixed", maxiter=4000, precond="azim", grouped=True, graphs=False)
    for (xa, sa), (xb, sb) in zip(a, b):
        assert sa["converged"] == 1 and sb["converged"] == 1
        e = rel_l2(xa.cpu().numpy(), xb.cpu().numpy())
        print(f"grouped graph vs eager: relative difference {e:.2e} ({sa['iterations']} / {sb['iterations']} "
              f"iterations)")
        assert e < 1e-5, e


def test_grouped_teb_two_geometries():
    from paper_2306_15511_gb300 import Plan, chains_sample
    req, refs = [], []
    for ns, L in ((16, 32), (32, 48)):
        p = C.teb_realizations(2, ns, L)
        g = osht.healpix(ns)
        ls = osht.ls_of(L)
        ds = []
        for q in p:
            a = q.signal_alm * q.bl[ls][None]
            T = osht.alm2map(g, L, a[0])
            Q, U = osht.alm2map_spin2(g, L, a[1], a[2])
            ds.append(np.stack([T, Q, U]) + q.noise_map)
        ds = np.stack(ds)
        w1 = np.stack([q.w1 for q in p])
        w2 = np.stack([q.w2 for q in p])
        plan = Plan(nside=ns, lmax=L, max_batch=2, spin2=True)
        req.append({"plan": plan, "cl": p[0].cl, "bl": p[0].bl, "ninv": _cuda(p[0].ninv, torch.float64),
                    "d": _cuda(ds, torch.float64), "w1": _cuda(w1, torch.complex128),
                    "w2": _cuda(w2, torch.float64)})
        refs.append((g, L, p, ds, w1, w2))
    res = chains_sample(req, tol=1e-6, mode="mixed", maxiter=4000, precond="diag", grouped=True)
    for (x, st), (g, L, p, ds, w1, w2) in zip(res, refs):
        assert st["converged"] == 1, st
        xh = x.cpu().numpy()
        prob = osol.Problem(g, L, p[0].cl, p[0].bl, p[0].ninv)
        for k in range(2):
            r = osol.true_residual(prob, xh[k], prob.rhs(ds[k], w1[k], w2[k]))
            assert r <= 1.05e-6, (L, k, r, st)


def test_grouped_refusals(chains):
    from paper_2306_15511_gb300 import chains_sample
    from paper_2306_15511_gb300._native import ShtgError
    req, _ = chains
    sub = req[:2]
    with pytest.raises(ShtgError, match="SHTG_PRECOND"):
        chains_sample(sub, mode="mixed", precond="lowl", grouped=True)
    with pytest.raises(ShtgError, match="mode"):
        chains_sample(sub, mode="fp64", grouped=True)

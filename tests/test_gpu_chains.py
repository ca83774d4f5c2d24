"""Chains of uneven geometry in one call (the mixed-geometry chains: per-chain
N_side, l_max and signal amplitude), through the C ABI, against the FP64
oracle: every chain's oracle-evaluated residual meets the tolerance, and the
per-realization amplitude gives the same solution as a separate solve with
the scaled C_l."""
import numpy as np
import pytest

from inputs import configs as C
from oracle import sht as osht
from oracle import solver as osol
from tests._util import rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _cuda(x, dt):
    return torch.tensor(np.ascontiguousarray(x), dtype=dt, device="cuda")


def _groups(max_per_group=4):
    """The recipe's first chains with N_side 64 (l_max 128 or 191) or N_side
    128 with l_max 256, grouped by geometry."""
    chains = C.mixed_geometry_chains(64)
    keep = {}
    for ch in chains:
        key = (ch.nside, ch.lmax)
        if key in ((64, 128), (64, 191), (128, 256)) and len(keep.setdefault(key, [])) < max_per_group:
            keep[key].append(ch)
    return keep


def _data(ch, g):
    ls = osht.ls_of(ch.lmax)
    return osht.alm2map(g, ch.lmax, ch.signal_alm[0] * ch.bl[ls]) + ch.noise_map[0]


def test_chains_of_uneven_geometry():
    from paper_2306_15511_gb300 import Plan, chains_sample
    groups = _groups()
    assert len(groups) >= 2
    req, refs = [], []
    for (ns, L), chs in groups.items():
        g = osht.healpix(ns)
        base = C.cl_flat(L)
        amps = np.array([ch.extra["amp"] for ch in chs])
        for ch, a in zip(chs, amps):
            assert np.allclose(ch.cl, a * base)
        d = np.stack([_data(ch, g)[None] for ch in chs])
        plan = Plan(nside=ns, lmax=L, max_batch=len(chs))
        req.append({"plan": plan, "cl": base, "bl": chs[0].bl, "ninv": _cuda(chs[0].ninv, torch.float64),
                    "d": _cuda(d, torch.float64), "w1": _cuda(np.stack([ch.w1 for ch in chs]), torch.complex128),
                    "w2": _cuda(np.stack([ch.w2 for ch in chs]), torch.float64), "cl_scale": amps})
        refs.append((g, chs, d))
    res = chains_sample(req, tol=1e-6, mode="mixed_tc", maxiter=4000)
    for (x, st), (g, chs, d) in zip(res, refs):
        assert st["converged"] == 1
        xh = x.cpu().numpy()
        for k, ch in enumerate(chs):
            prob = osol.Problem(g, ch.lmax, ch.cl, ch.bl, ch.ninv)
            b = prob.rhs(d[k], ch.w1, ch.w2)
            assert osol.true_residual(prob, xh[k], b) <= 1.05e-6, (ch.name, st)


def test_cl_scale_equals_scaled_cl():
    """One realization with amplitude s through cl_scale equals the solve with
    C_l replaced by s C_l (same operator, same RHS)."""
    from paper_2306_15511_gb300 import Plan
    (ns, L), chs = next(iter(_groups(1).items()))
    ch = chs[0]
    g = osht.healpix(ns)
    d = _data(ch, g)[None, None]
    plan = Plan(nside=ns, lmax=L)
    base = C.cl_flat(L)
    amp = ch.extra["amp"]
    args = (_cuda(ch.ninv, torch.float64), _cuda(d, torch.float64), _cuda(ch.w1[None], torch.complex128),
            _cuda(ch.w2[None], torch.float64))
    xs, _ = plan.cg_sample(base, ch.bl, *args, tol=1e-10, mode="fp64", maxiter=4000, cl_scale=[amp])
    xc, _ = plan.cg_sample(amp * base, ch.bl, *args, tol=1e-10, mode="fp64", maxiter=4000)
    assert rel_l2(xs.cpu().numpy(), xc.cpu().numpy()) < 1e-8

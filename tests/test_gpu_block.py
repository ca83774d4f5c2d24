"""The exact per-m dense block solve of App. A on the GPU (mode "block"),
through the C ABI, against the oracle's per-m dense solves and its PCG.

Gauss-Legendre grids with nphi = 2 lmax + 2 and N^-1 constant along every
ring: a |b| < 25 deg cut, and noise that differs between the hemispheres
(then the l + l' odd entries of a block are nonzero).  Sizes span several
32 x 32 tiles of a block and several 32-pair chunks with ragged ends."""
import math

import numpy as np
import pytest

from inputs import configs as C
from inputs import philox as px
from oracle import sht as osht
from oracle import solver as osol
from tests._util import rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _cuda(x, dt):
    return torch.tensor(np.ascontiguousarray(x), dtype=dt, device="cuda")


def _problem(L, asym, nb=2):
    g = osht.gauss_legendre(L + 1, 2 * L + 2)
    ninv_ring = np.where(np.abs(g.cth) < math.sin(25 * C.DEG), 0.0, 1.0 / 5.0 ** 2)
    if asym:
        ninv_ring = ninv_ring * np.where(g.cth > 0, 1.0, 0.35) * (1.0 + 0.5 * g.cth ** 2)
    ninv = np.repeat(ninv_ring, g.nphi)
    cl, bl = C.cl_flat(L), C.gauss_beam(L, 10 * C.DEG)
    prob = osol.Problem(g, L, cl, bl, ninv)
    ls = osht.ls_of(L)
    a = np.sqrt(cl)[ls] * C.white_alm(L, 0, px.STREAM_SIGNAL)
    sig = np.where(ninv > 0, 1.0 / np.sqrt(np.where(ninv > 0, ninv, 1.0)), 0.0)
    d = np.stack([osht.alm2map(g, L, a * bl[ls]) + sig * C.white_map(g.npix, 10 + k, px.STREAM_NOISE)
                  for k in range(nb)])
    w1 = np.stack([C.white_alm(L, 20 + k, px.STREAM_W1) for k in range(nb)])
    w2 = np.stack([C.white_map(g.npix, 20 + k, px.STREAM_W2) for k in range(nb)])
    return g, prob, ninv, cl, bl, d, w1, w2


@pytest.mark.parametrize("L,asym", [(64, False), (64, True), (200, True)])
def test_block_solve_vs_oracle(L, asym):
    from paper_2306_15511_gb300 import Plan
    g, prob, ninv, cl, bl, d, w1, w2 = _problem(L, asym)
    plan = Plan(gauss=(L + 1, 2 * L + 2), lmax=L, max_batch=2, block_solver=True)
    x, st = plan.cg_sample(cl, bl, _cuda(ninv, torch.float64), _cuda(d[:, None], torch.float64),
                           _cuda(w1[:, None], torch.complex128), _cuda(w2[:, None], torch.float64),
                           tol=1e-10, mode="block")
    assert st["converged"] == 1 and st["iterations"] == 0
    xh = x.cpu().numpy()
    for k in range(2):
        b = prob.rhs(d[k][None], w1[k][None], w2[k][None])
        ref = osol.block_solve(prob, b)
        err = rel_l2(xh[k], ref)
        res = osol.true_residual(prob, xh[k], b)
        print(f"block L {L} asym {asym} realization {k}: error vs oracle {err:.2e}, oracle residual {res:.2e}, "
              f"library residual {st['rel_residual']:.2e}")
        assert err < 1e-10
        assert res < 1e-11


def test_block_solve_matches_fp64_pcg():
    from paper_2306_15511_gb300 import Plan
    L = 96
    g, prob, ninv, cl, bl, d, w1, w2 = _problem(L, True, nb=1)
    plan = Plan(gauss=(L + 1, 2 * L + 2), lmax=L, max_batch=1, block_solver=True)
    args = (cl, bl, _cuda(ninv, torch.float64), _cuda(d[:, None], torch.float64),
            _cuda(w1[:, None], torch.complex128), _cuda(w2[:, None], torch.float64))
    xb, _ = plan.cg_sample(*args, tol=1e-10, mode="block")
    xp, sp = plan.cg_sample(*args, tol=1e-12, mode="fp64", maxiter=5000)
    assert sp["converged"] == 1
    # PCG stopped at a residual of 1e-12 is accurate to ~cond(A) 1e-12 (~1e-9 here)
    assert rel_l2(xb.cpu().numpy(), xp.cpu().numpy()) < 1e-8


def test_block_solve_refuses_what_is_not_block_diagonal():
    from paper_2306_15511_gb300 import Plan
    from paper_2306_15511_gb300._native import ShtgError
    L = 32
    g, prob, ninv, cl, bl, d, w1, w2 = _problem(L, False, nb=1)
    args = (_cuda(d[:, None], torch.float64), _cuda(w1[:, None], torch.complex128),
            _cuda(w2[:, None], torch.float64))
    # no block workspace
    plain = Plan(gauss=(L + 1, 2 * L + 2), lmax=L)
    with pytest.raises(ShtgError) as ei:
        plain.cg_sample(cl, bl, _cuda(ninv, torch.float64), *args, mode="block")
    assert ei.value.code == -1 and "SHTG_BLOCK_SOLVER" in str(ei.value)
    # N^-1 that varies along a ring
    plan = Plan(gauss=(L + 1, 2 * L + 2), lmax=L, block_solver=True)
    bumpy = ninv.copy()
    bumpy[g.ofs[3] + 1] *= 1.5
    with pytest.raises(ShtgError) as ei:
        plan.cg_sample(cl, bl, _cuda(bumpy, torch.float64), *args, mode="block")
    assert ei.value.code == -1 and "varies along a ring" in str(ei.value)
    # HEALPix polar rings have nphi < 2 lmax + 1 (their m alias)
    hp = Plan(nside=16, lmax=32, block_solver=True)
    p = C.fullsky_temperature(16, 32)
    with pytest.raises(ShtgError) as ei:
        hp.cg_sample(p.cl, p.bl, _cuda(p.ninv, torch.float64), _cuda(p.noise_map[None], torch.float64),
                     _cuda(p.w1[None], torch.complex128), _cuda(p.w2[None], torch.float64), mode="block")
    assert ei.value.code == -1 and "nphi" in str(ei.value)
    # the plan stays usable
    x, st = plan.cg_sample(cl, bl, _cuda(ninv, torch.float64), *args, mode="block", tol=1e-10)
    assert st["converged"] == 1

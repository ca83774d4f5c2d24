"""The benchmark workload at its full size, checked by the FP64 oracle.

8 T+E+B constrained realizations at N_side 1024, l_max 2048 (damped TT,
EE = 0.05 TT, BB = 1e-3 EE, TE = 0.3 sqrt(TT EE), 10' beam, 30 / 42 uK /
sqrt(hits) noise, |b| < 20 deg plus 200 holes) solved in one call in the
benchmark's launch configuration (mixed precision with the tensor-core
Legendre sums, batch 8) to a relative residual of 1e-6.  The oracle then
evaluates ||b - A x|| / ||b|| for realization 0 with its own right-hand side
and operator (about two FP64 T+E+B operator applications on the host).

Inputs never come from the CUDA path: the random fields are the seeded
Philox draws of inputs/, and realization 0's sky signal Y B a is the
oracle's synthesis.  The eight realizations observe that one sky, each with
its own noise and white-noise draws (d_k = Y B a_0 + n_k), so only one
oracle synthesis is needed.
"""
import numpy as np
import pytest

from inputs import configs as C
from oracle import sht as osht
from oracle import solver as osol

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NSIDE, LMAX, NB = 1024, 2048, 8


def test_teb_target_size_oracle_residual():
    from paper_2306_15511_gb300 import Plan
    dev = torch.device("cuda", 0)
    probs = C.teb_realizations(NB, NSIDE, LMAX, device=dev)
    p0 = probs[0]
    g = osht.healpix(NSIDE)
    ls = osht.ls_of(LMAX)
    a0 = p0.signal_alm.cpu().numpy() * p0.bl[ls][None]
    T = osht.alm2map(g, LMAX, a0[0])
    Q, U = osht.alm2map_spin2(g, LMAX, a0[1], a0[2])
    sky = torch.as_tensor(np.stack([T, Q, U]), device=dev)
    d = torch.stack([sky + p.noise_map for p in probs]).contiguous()
    w1 = torch.stack([p.w1 for p in probs]).contiguous()
    w2 = torch.stack([p.w2 for p in probs]).contiguous()
    ninv = torch.as_tensor(p0.ninv, device=dev).contiguous()
    plan = Plan(nside=NSIDE, lmax=LMAX, max_batch=NB, spin2=True)
    x, st = plan.cg_sample(p0.cl, p0.bl, ninv, d, w1, w2, tol=1e-6, mode="mixed_tc", maxiter=6000,
                           check_every=8)
    assert st["converged"] == 1, st
    x0 = x[0].cpu().numpy()
    d0 = d[0].cpu().numpy()
    del plan, x, d, w2
    torch.cuda.empty_cache()
    prob = osol.Problem(g, LMAX, p0.cl, p0.bl, p0.ninv)
    b0 = prob.rhs(d0, p0.w1.cpu().numpy(), p0.w2.cpu().numpy())
    res = osol.true_residual(prob, x0, b0)
    print(f"T+E+B N_side {NSIDE} / l_max {LMAX}, batch {NB}, mixed_tc: {st['iterations']} FP32 "
          f"iterations, {st['fp64_matvecs']} FP64-accurate operator applications, library "
          f"residual {st['rel_residual']:.3e}, oracle residual (realization 0) {res:.3e}")
    assert res <= 1.05e-6, (res, st)

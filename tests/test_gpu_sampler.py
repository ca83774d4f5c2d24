"""Sampler-level validation of the joint (C_l, a) move (Sect. 2.2.2) on the
full sky with uniform noise, where the marginal posterior of theta has the
closed form of Eq. (exact_harm).

A Gauss-Legendre grid (exact quadrature) with N^-1 proportional to the pixel
area gives noise of power N_l = sigma^2 per steradian, as Eq. (exact_harm)
assumes.  One parameter, an amplitude q with C_l(q) = q C_l^fid and a flat
prior on q > 0.  The chain runs entirely through the library (joint.py:
solves, rescaling, log pi, acceptance); the exact posterior of q is the
oracle's Eq. (exact_harm) on a grid.  Its mean and standard deviation must
agree with the chain's (after burn-in) to a quarter of the posterior width."""
import numpy as np
import pytest

from inputs import configs as C
from inputs import philox as px
from oracle import sht as osht
from oracle import solver as osol

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_joint_sampler_matches_exact_harmonic_posterior():
    from paper_2306_15511_gb300 import Plan
    from paper_2306_15511_gb300.joint import JointSampler
    L = 48
    g = osht.gauss_legendre(L + 1, 2 * L + 2)
    sig2 = 3.0                                   # noise power per steradian, uK^2
    ninv = g.pixel_weights() / sig2
    cl_fid = C.cl_flat(L)
    bl = C.gauss_beam(L, 2.0 * C.DEG)
    ls = osht.ls_of(L)
    a_true = np.sqrt(cl_fid)[ls] * C.white_alm(L, 7, px.STREAM_SIGNAL)
    d = osht.alm2map(g, L, a_true * bl[ls]) + C.white_map(g.npix, 7, px.STREAM_NOISE) / np.sqrt(ninv)
    # exact marginal posterior of q (flat prior), Eq. (exact_harm)
    r = sig2 * osht.alm2map_adjoint(g, L, ninv * d)
    co = osol.observed_spectrum(r, L)
    nl = np.full(L + 1, sig2)
    qs = np.linspace(0.2, 3.0, 5601)
    lk = np.array([osol.exact_harmonic_loglike(co, q * cl_fid, bl, nl) for q in qs])
    w = np.exp(lk - lk.max())
    mean = float(np.sum(w * qs) / np.sum(w))
    std = float(np.sqrt(np.sum(w * (qs - mean) ** 2) / np.sum(w)))
    assert std < 0.2 and qs[0] < mean - 6 * std and mean + 6 * std < qs[-1]
    # the chain
    plan = Plan(gauss=(L + 1, 2 * L + 2), lmax=L, max_batch=2)
    dev = torch.device("cuda", 0)
    sampler = JointSampler(plan, lambda th: th[0] * cl_fid if th[0] > 0 else None, bl,
                           torch.as_tensor(ninv, device=dev).contiguous(),
                           torch.as_tensor(d[None, None], device=dev).contiguous(), [1.0],
                           [[(2.4 * std) ** 2]], seed=0, log_prior=lambda th: 0.0, tol=1e-10, mode="fp64")
    chain = sampler.sample(3000)[300:, 0]
    rate = sampler.n_accepted / sampler.n_steps
    print(f"joint sampler: acceptance {rate:.3f}; q mean {chain.mean():.4f} std {chain.std():.4f}; "
          f"exact posterior mean {mean:.4f} std {std:.4f}")
    assert 0.15 < rate < 0.8
    assert abs(chain.mean() - mean) < 0.25 * std
    assert abs(chain.std() / std - 1.0) < 0.25

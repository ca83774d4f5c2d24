"""Joint (C_l, a) sampler of Sect. 2.2.2: Metropolis-Hastings in the
cosmological parameters theta with a Gaussian random-walk proposal and the
deterministic rescaling of the fluctuation term.

One step (the algorithm's steps 2-4):
  - propose theta' ~ N(theta, proposal covariance) and evaluate C_l(theta');
  - solve for the proposal's mean field a^' (right-hand side B Y^T N^-1 d,
    Eq. mean-field-map) and rescale the current fluctuation,
    f^scaled = (C'_l)^{1/2} (C_l)^{-1/2} f^;
  - accept with A = min[1, pi(theta') P(theta') / (pi(theta) P(theta))] (Eq.
    acceptance-rate), pi evaluated from a^' and f^scaled;
  - on acceptance solve for a new fluctuation f^ at theta' (Eq. fluc-map with
    fresh white noise) and re-evaluate pi(theta') with it.
The solves, the rescaling, log pi and the acceptance probability run in the
library (shtg_cg_sample, shtg_fluctuation_rescale, shtg_joint_log_target,
shtg_joint_acceptance); this class holds the chain's state and draws the
proposals, the acceptance uniforms and the white noise (torch generators).
Temperature or T+E+B; one realization of the data.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from .api import joint_acceptance


def white_noise(plan, ncomp: int, gen: torch.Generator):
    """Unit white noise of one realization: harmonic w1 [1, ncomp, nalm]
    complex128 (a_l0 ~ N(0, 1) real, real and imaginary parts N(0, 1/2) for
    m > 0) and pixel w2 [1, ncomp, npix] float64, on the plan's device."""
    dev = plan.device
    L = plan.lmax
    ms = torch.cat([torch.full((L + 1 - m,), m, dtype=torch.int64) for m in range(L + 1)]).to(dev)
    re = torch.randn(1, ncomp, plan.nalm, dtype=torch.float64, device=dev, generator=gen)
    im = torch.randn(1, ncomp, plan.nalm, dtype=torch.float64, device=dev, generator=gen)
    s = torch.where(ms == 0, 1.0, math.sqrt(0.5)).to(torch.float64)
    im = torch.where(ms == 0, torch.zeros_like(im), im * s)
    w1 = torch.complex(re * s, im).contiguous()
    w2 = torch.randn(1, ncomp, plan.npix, dtype=torch.float64, device=dev, generator=gen).contiguous()
    return w1, w2


class JointSampler:
    """Chain state: theta, C_l(theta), the mean field a^ and the fluctuation
    f^ at theta, and log pi(theta).

    cl_of_theta(theta) -> C_l array for cg_sample (return None for theta
    outside the prior's support); log_prior(theta) -> float (default flat).
    d: [1, ncomp, npix] float64 CUDA; ninv as for cg_sample.  mode and tol
    select the solver ("fp64", "mixed", "mixed_tc"); log pi uses
    FP64-accurate syntheses ("df64" by default)."""

    def __init__(self, plan, cl_of_theta, bl, ninv, d, theta0, proposal_cov, seed: int = 0,
                 log_prior=None, tol: float = 1e-8, mode: str = "fp64", maxiter: int = 4000,
                 logpi_precision: str = "df64"):
        self.plan, self.cl_of_theta, self.bl, self.ninv, self.d = plan, cl_of_theta, bl, ninv, d
        self.ncomp = int(d.shape[1])
        self.log_prior = log_prior or (lambda th: 0.0)
        self.kw = dict(tol=tol, mode=mode, maxiter=maxiter)
        self.prec = logpi_precision
        self.rng = np.random.default_rng(seed)
        self.gen = torch.Generator(device=plan.device)
        self.gen.manual_seed(seed)
        self.chol = np.linalg.cholesky(np.atleast_2d(np.asarray(proposal_cov, np.float64)))
        self.theta = np.atleast_1d(np.asarray(theta0, np.float64)).copy()
        self.cl = np.asarray(cl_of_theta(self.theta), np.float64)
        self.zero_d = torch.zeros_like(d)
        self.zero_w1 = torch.zeros(1, self.ncomp, plan.nalm, dtype=torch.complex128, device=plan.device)
        self.zero_w2 = torch.zeros_like(d)
        # step 1: mean field and fluctuation at theta0 in one split solve
        w1, w2 = white_noise(plan, self.ncomp, self.gen)
        x, _ = plan.cg_sample(self.cl, bl, ninv, d, w1, w2, split=True, **self.kw)
        self.a_hat, self.f_hat = x[0].contiguous().clone(), x[1].contiguous().clone()
        self.log_pi = self._log_pi(self.cl, self.a_hat, self.f_hat)
        self.n_steps = self.n_accepted = 0

    def _log_pi(self, cl, a_hat, f_hat) -> float:
        return float(self.plan.joint_log_target(cl, self.bl, self.ninv, self.d, a_hat, f_hat,
                                                precision=self.prec)[0])

    def step(self) -> bool:
        """One joint move; returns whether it was accepted."""
        self.n_steps += 1
        prop = self.theta + self.chol @ self.rng.standard_normal(self.theta.size)
        u = self.rng.uniform()
        cl_new = self.cl_of_theta(prop)
        if cl_new is None:
            return False
        cl_new = np.asarray(cl_new, np.float64)
        a_new, _ = self.plan.cg_sample(cl_new, self.bl, self.ninv, self.d, self.zero_w1, self.zero_w2, **self.kw)
        f_scaled = self.plan.fluctuation_rescale(self.cl, cl_new, self.f_hat)
        lp_new = self._log_pi(cl_new, a_new, f_scaled)
        acc = joint_acceptance(lp_new, self.log_pi, self.log_prior(prop), self.log_prior(self.theta))
        if u >= acc:
            return False
        # accepted: new state, and a new fluctuation at theta' (step 4)
        self.theta, self.cl, self.a_hat = prop, cl_new, a_new.contiguous()
        w1, w2 = white_noise(self.plan, self.ncomp, self.gen)
        f_new, _ = self.plan.cg_sample(cl_new, self.bl, self.ninv, self.zero_d, w1, w2, **self.kw)
        self.f_hat = f_new.contiguous()
        self.log_pi = self._log_pi(self.cl, self.a_hat, self.f_hat)
        self.n_accepted += 1
        return True

    def sample(self, n: int) -> np.ndarray:
        """n steps; returns the chain of theta, [n, ntheta]."""
        out = np.zeros((n, self.theta.size))
        for i in range(n):
            self.step()
            out[i] = self.theta
        return out

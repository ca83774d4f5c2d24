"""GB300-native constrained-realization sampler for CMB skies.

Hot path of the joint sampler of Eskilt et al. (arXiv 2306.15511), Sect.
2.2.1: PCG on Eq. (mapmakingeq) with spherical-harmonic-transform matvecs,
hand-written in CUDA for sm_103a (libshtg.so, C ABI in include/shtg.h).

The CUDA library is loaded on first use; there is no CPU fallback.
"""
from .api import Plan, chains_sample, joint_acceptance  # noqa: F401

__all__ = ["Plan", "chains_sample", "joint_acceptance"]

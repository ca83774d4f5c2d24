"""Plain FP64 CPU oracle for the constrained-realization sampler.

TEST INFRASTRUCTURE ONLY.  The tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import it; the product library never
does.  It shares no code with the CUDA path.

- ``oracle.c`` / :mod:`oracle.sht`: geometry, Legendre functions, spin-0 and
  spin-2 transforms by direct sums (App. A notation).
- :mod:`oracle.solver`: Eq. (mapmakingeq) operator and right-hand side, PCG,
  the full-sky closed form of Eqs. (hat_s_approx, hat_f_approx) and the
  Gaussian log-posterior of Eq. (joint-posterior) with its gradient.
"""
from . import sht, solver  # noqa: F401
from ._lib import build  # noqa: F401

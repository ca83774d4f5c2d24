"""Write the oracle's tightly converged solution of the masked temperature
workload (N_side 256, l_max 512, hits-weighted noise, |b| < 20 deg plus 50
holes) to tests/golden/masked_t_n256_l512_x.npy.

Only the FP64 CPU oracle and the seeded input generators are used: d is the
oracle's Y B a + n, b the oracle's right-hand side of Eq. (mapmakingeq), and
x the oracle's preconditioned conjugate gradients run to a relative residual
of 1e-11 (the stored solution's error is far below the 1e-5 that the GPU
mixed-precision solution is held to).  Run from the repository root:

    python tests/golden/make_masked_solution.py
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from inputs import configs as C  # noqa: E402
from oracle import sht as osht  # noqa: E402
from oracle import solver as osol  # noqa: E402

NSIDE, LMAX, TOL = 256, 512, 1e-11
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "masked_t_n256_l512_x.npy")


def main():
    t0 = time.time()
    p = C.masked_temperature(NSIDE, LMAX)
    g = osht.healpix(NSIDE)
    ls = osht.ls_of(LMAX)
    d = osht.alm2map(g, LMAX, p.signal_alm[0] * p.bl[ls]) + p.noise_map[0]
    prob = osol.Problem(g, LMAX, p.cl, p.bl, p.ninv)
    b = prob.rhs(d[None], p.w1, p.w2)
    x, it, hist = osol.pcg(prob, b, TOL, maxiter=20000)
    res = osol.true_residual(prob, x, b)
    np.save(OUT, x[0])
    print(f"{OUT}: {it} PCG iterations, recursive residual {hist[-1]:.3e}, "
          f"true residual {res:.3e}, {time.time() - t0:.0f} s")


if __name__ == "__main__":
    main()

"""Oracle constrained-realization solver (FP64, CPU).  Test infrastructure only.

Eq. (mapmakingeq) of Sect. 2.2.1, with the beam applied in harmonic space
and the synthesis Y written out:

    A a = b,   A = S^-1 + B Y^T N^-1 Y B,
    b = B Y^T (N^-1 d + N^-1/2 w2) + S^-1/2 w1.

- S is diagonal in (l, m) with C_l (temperature) or the 3x3 (T, E, B) block
  of Sect. 2.2.2 with EB = TB = 0.  Modes where S is singular (C_0 = C_1 = 0)
  are held at zero: there A acts as the identity and b is zero.
- B is the beam b_l; N^-1 is a diagonal pixel weight, 0 in the mask (App. A).
- S^-1/2 is the inverse of the symmetric principal square root of S.
- Solved by preconditioned conjugate gradients (Sect. 2.2.1 cites
  Shewchuk 1994) with the diagonal preconditioner of Sect. 4,
  M = S^-1 + b_l^2 D_lm, D_lm = sum_r g_lm(theta_r) sum_{p in r} N^-1_p.
All inner products use the metric of :func:`oracle.sht.dot_q6`.

Also here: the Gaussian log-posterior of Eq. (joint-posterior) with its
gradients, the pieces of the joint (C_l, a) move of Sect. 2.2.2 (the
fluctuation rescaling, log pi(theta) and the acceptance rule), and the
per-m dense block solve of App. A for azimuthally symmetric noise.
"""
from __future__ import annotations

import numpy as np

from . import sht


class Problem:
    """Operator data for one realization.

    cl: (lmax+1,) for temperature or (4, lmax+1) = TT, EE, BB, TE.
    ninv: (npix,) or (2, npix) = (N^-1 for T, N^-1 for Q and U).
    """

    def __init__(self, geom: sht.Geometry, lmax: int, cl, bl, ninv):
        self.g = geom
        self.lmax = lmax
        cl = np.asarray(cl, np.float64)
        self.ncomp = 1 if cl.ndim == 1 else 3
        self.bl = np.asarray(bl, np.float64)
        ninv = np.asarray(ninv, np.float64)
        self.ninv = ninv.reshape(1, -1) if ninv.ndim == 1 else ninv
        self.ls = sht.ls_of(lmax)
        L1 = lmax + 1
        # per-l inverse prior and inverse square root, as (ncomp, ncomp, L+1)
        sinv = np.zeros((self.ncomp, self.ncomp, L1))
        sinvh = np.zeros((self.ncomp, self.ncomp, L1))
        active = np.zeros(L1, bool)
        for l in range(L1):
            if self.ncomp == 1:
                S = np.array([[cl[l]]])
            else:
                tt, ee, bb, te = cl[:, l]
                S = np.array([[tt, te, 0.0], [te, ee, 0.0], [0.0, 0.0, bb]])
            w, V = np.linalg.eigh(S)
            if np.all(w > 0):
                active[l] = True
                sinv[:, :, l] = (V / w) @ V.T
                sinvh[:, :, l] = (V / np.sqrt(w)) @ V.T
            else:
                sinv[:, :, l] = np.eye(self.ncomp)
        self.sinv, self.sinvh, self.active = sinv, sinvh, active
        self.bmask = np.where(active, self.bl, 0.0)

    # -- pieces -------------------------------------------------------------
    def _per_l(self, mat, x):
        """Apply an (ncomp, ncomp, L+1) per-l matrix to x of shape (ncomp, nalm)."""
        M = mat[:, :, self.ls]
        return np.einsum("ijp,jp->ip", M, x)

    def Y(self, a):
        if self.ncomp == 1:
            return sht.alm2map(self.g, self.lmax, a[0])[None]
        T = sht.alm2map(self.g, self.lmax, a[0])
        Q, U = sht.alm2map_spin2(self.g, self.lmax, a[1], a[2])
        return np.stack([T, Q, U])

    def Yt(self, m):
        if self.ncomp == 1:
            return sht.alm2map_adjoint(self.g, self.lmax, m[0])[None]
        T = sht.alm2map_adjoint(self.g, self.lmax, m[0])
        E, B = sht.alm2map_spin2_adjoint(self.g, self.lmax, m[1], m[2])
        return np.stack([T, E, B])

    def ninv_maps(self):
        if self.ncomp == 1:
            return self.ninv[:1]
        return np.stack([self.ninv[0], self.ninv[1], self.ninv[1]])

    def beam(self, a):
        return a * self.bmask[self.ls][None]

    # -- operator -----------------------------------------------------------
    def matvec(self, x):
        x = np.asarray(x, np.complex128).reshape(self.ncomp, -1)
        y = self.Y(self.beam(x)) * self.ninv_maps()
        out = self.beam(self.Yt(y)) + self._per_l(self.sinv, x)
        return _zero_im_m0(out, self.lmax)

    def rhs(self, d, w1, w2):
        d = np.asarray(d, np.float64).reshape(self.ncomp, -1)
        w2 = np.asarray(w2, np.float64).reshape(self.ncomp, -1)
        w1 = np.asarray(w1, np.complex128).reshape(self.ncomp, -1)
        nv = self.ninv_maps()
        pix = nv * d + np.sqrt(nv) * w2
        b = self.beam(self.Yt(pix)) + self._per_l(self.sinvh, w1)
        return _zero_im_m0(b, self.lmax)

    def rhs_parts(self, d, w1, w2):
        """(mean-field part, fluctuation part) of the right-hand side, Eqs.
        (mean-field-map) and (fluc-map)."""
        z = np.zeros_like(np.asarray(d, np.float64).reshape(self.ncomp, -1))
        zw = np.zeros_like(np.asarray(w1, np.complex128).reshape(self.ncomp, -1))
        return self.rhs(d, zw, z), self.rhs(z, w1, w2)

    def precond_diag(self):
        """(ncomp, ncomp, nalm) block of M = S^-1 + b^2 D (D diagonal per comp)."""
        L = self.lmax
        nv = self.ninv
        wT = sht.ring_sums(self.g, nv[0])
        D = [sht.diag_ringsum(self.g, L, wT, 0)]
        if self.ncomp == 3:
            wP = sht.ring_sums(self.g, nv[1])
            dp = sht.diag_ringsum(self.g, L, wP, 2)
            D += [dp, dp]
        M = self.sinv[:, :, self.ls].copy()
        b2 = self.bmask[self.ls] ** 2
        for c in range(self.ncomp):
            M[c, c] += b2 * D[c]
        return M

    def dot(self, a, c):
        return sht.dot_q6(a, c, self.lmax)


def _zero_im_m0(a, lmax):
    a = np.array(a, np.complex128, copy=True)
    m0 = sht.ms_of(lmax) == 0
    a[..., m0] = a[..., m0].real
    return a


def apply_block_inverse(M, r):
    """Solve M z = r per alm index for an (nc, nc, nalm) block diagonal M."""
    nc = M.shape[0]
    if nc == 1:
        return r / M[0, 0][None]
    Mt = np.moveaxis(M, 2, 0)                          # (nalm, nc, nc)
    rt = np.moveaxis(r, 1, 0)[..., None]               # (nalm, nc, 1)
    zr = np.linalg.solve(Mt, rt.real)[..., 0]
    zi = np.linalg.solve(Mt, rt.imag)[..., 0]
    return np.moveaxis(zr + 1j * zi, 0, 1)


def pcg(prob: Problem, b, tol: float, maxiter: int = 1000, precond=True, x0=None):
    """Plain preconditioned conjugate gradients in FP64.

    precond: True (the diagonal preconditioner of Sect. 4), False (none) or a
    callable r -> z.  Stops when ||b - A x|| / ||b|| <= tol (recursively
    updated residual).  Returns (x, iterations, relative residual history)."""
    b = np.asarray(b, np.complex128).reshape(prob.ncomp, -1)
    if callable(precond):
        apply_m = precond
    elif precond:
        M = prob.precond_diag()
        apply_m = lambda r: apply_block_inverse(M, r)  # noqa: E731
    else:
        apply_m = lambda r: r.copy()  # noqa: E731
    x = np.zeros_like(b) if x0 is None else np.array(x0, np.complex128).reshape(b.shape)
    r = b - prob.matvec(x) if x0 is not None else b.copy()
    z = _zero_im_m0(apply_m(r), prob.lmax)
    p = z.copy()
    bn = np.sqrt(prob.dot(b, b))
    rz = prob.dot(r, z)
    hist = [np.sqrt(prob.dot(r, r)) / bn]
    it = 0
    while hist[-1] > tol and it < maxiter:
        q = prob.matvec(p)
        alpha = rz / prob.dot(p, q)
        x = x + alpha * p
        r = r - alpha * q
        z = _zero_im_m0(apply_m(r), prob.lmax)
        rz_new = prob.dot(r, z)
        p = z + (rz_new / rz) * p
        rz = rz_new
        it += 1
        hist.append(np.sqrt(prob.dot(r, r)) / bn)
    return x, it, np.array(hist)


# ----------------------------------------------------------------------------
# Two-level preconditioner: exact inverse on the low multipoles (Sect. 4 asks
# for preconditioners beyond the diagonal one)
# ----------------------------------------------------------------------------
def low_parameters(prob: Problem, lc: int):
    """Real parameters (l, m, comp, part) of the active multipoles l <= lc,
    a_lm = u + i v (part 0 = u, 1 = v; no v at m = 0), ordered by component,
    then l, m, part."""
    out = []
    for c in range(prob.ncomp):
        for l in range(lc + 1):
            if not prob.active[l]:
                continue
            for m in range(l + 1):
                for w in range(1 if m == 0 else 2):
                    out.append((l, m, c, w))
    return out


def low_block(prob: Problem, lc: int):
    """H = W A on the low parameters, one column per operator application:
    column j is A applied to the unit parameter e_j (a_lm = 1 or i), read
    back as real parts, times the metric weight w_i (1 for m = 0, else 2) of
    the row.  With the metric <a, c> = sum w (u u' + v v') of the inner
    products, H is symmetric.  Returns (parameters, H)."""
    L = prob.lmax
    params = low_parameters(prob, lc)
    n = len(params)
    nalm = (L + 1) * (L + 2) // 2
    idx = [m * (2 * L + 1 - m) // 2 + l for (l, m, _, _) in params]
    H = np.zeros((n, n))
    for j, (l, m, c, w) in enumerate(params):
        e = np.zeros((prob.ncomp, nalm), np.complex128)
        e[c, idx[j]] = 1.0 if w == 0 else 1j
        y = prob.matvec(e)
        for i, (l2, m2, c2, w2) in enumerate(params):
            v = y[c2, idx[i]]
            H[i, j] = (1.0 if m2 == 0 else 2.0) * (v.real if w2 == 0 else v.imag)
    return params, H


def two_level_precond(prob: Problem, lc: int):
    """z = M^-1 r with M^-1 the diagonal preconditioner's inverse outside
    the low block and A^-1 = H^-1 W on it (block Jacobi with one dense
    block).  Returns the callable for :func:`pcg`."""
    M = prob.precond_diag()
    params, H = low_block(prob, lc)
    L = prob.lmax
    comp = np.array([c for (_, _, c, _) in params], int)
    idx = np.array([m * (2 * L + 1 - m) // 2 + l for (l, m, _, _) in params], int)
    part = np.array([w for (_, _, _, w) in params], int)
    wgt = np.array([1.0 if m == 0 else 2.0 for (_, m, _, _) in params])

    def apply(r):
        z = apply_block_inverse(M, r)
        if not params:
            return z
        rv = r[comp, idx]
        g = wgt * np.where(part == 0, rv.real, rv.imag)
        zl = np.linalg.solve(H, g)
        z = np.array(z, np.complex128, copy=True)
        for k in range(len(params)):
            if part[k] == 0:
                z[comp[k], idx[k]] = zl[k] + 1j * z[comp[k], idx[k]].imag
            else:
                z[comp[k], idx[k]] = z[comp[k], idx[k]].real + 1j * zl[k]
        return z

    return apply


# ----------------------------------------------------------------------------
# Azimuthal block preconditioner: the per-m blocks of App. A built from the
# ring average of N^-1 (exact when N^-1 is constant along every ring)
# ----------------------------------------------------------------------------
def ring_sum_weights(prob: Problem):
    """sum over the pixels of each ring of N^-1: (ncomp_noise, nring) (T, and
    P for T+E+B), i.e. nphi_r times the ring average."""
    g = prob.g
    return np.stack([sht.ring_sums(g, prob.ninv[c]) for c in range(prob.ninv.shape[0])])


def azimuthal_te_block(prob: Problem, m: int, lb: int, wsum):
    """The m-block of A on the multipoles l = m .. lb of T (and E) with N^-1
    replaced by the ring weights wsum (per ring: sum of N^-1 over its pixels)
    and the aliasing of rings with nphi < 2 lmax + 1 left out:
      T-T: delta S^-1_TT + b_l b_l' sum_r wsum_T,r lambda_l lambda_l',
      E-E: delta S^-1_EE + b_l b_l' sum_r wsum_P,r (lw_l lw_l' + lx_l lx_l'),
      T-E: delta S^-1_TE;
    held multipoles (singular C_l block) give identity rows.  The E-B noise
    coupling at equal m (imaginary, sum_r wsum_P (lw lx' + lx lw')) and B are
    not part of the block.  Returns (l values, block) with rows [T l..] or
    [T l.., E l..]."""
    g = prob.g
    lr = np.arange(m, lb + 1)
    k = lr.size
    bm = prob.bmask[lr]
    act = prob.active[lr]
    lam = np.array([sht.lambda_lm(lb, m, g.cth[r], g.sth[r]) for r in range(g.nring)])   # (nring, k)
    GT = (lam * wsum[0][:, None]).T @ lam
    blocks = [[bm[:, None] * GT * bm[None, :] + np.diag(np.where(act, prob.sinv[0, 0][lr], 0.0))]]
    if prob.ncomp == 3:
        lw = np.zeros((g.nring, k))
        lx = np.zeros((g.nring, k))
        for r in range(g.nring):
            lw[r], lx[r] = sht.lambda_spin2(lb, m, g.cth[r], g.sth[r])
        GE = (lw * wsum[1][:, None]).T @ lw + (lx * wsum[1][:, None]).T @ lx
        te = np.diag(np.where(act, prob.sinv[0, 1][lr], 0.0))
        ee = bm[:, None] * GE * bm[None, :] + np.diag(np.where(act, prob.sinv[1, 1][lr], 0.0))
        blocks = [[blocks[0][0], te], [te, ee]]
    A = np.block(blocks)
    held = np.where(np.tile(~act, len(blocks)))[0]
    A[held, :] = 0.0
    A[:, held] = 0.0
    A[held, held] = 1.0
    return lr, A


def azimuthal_precond(prob: Problem, lb: int):
    """z = M^-1 r for the azimuthal block preconditioner: on the T (and E)
    multipoles l <= lb of every m <= lb the inverse of
    :func:`azimuthal_te_block` (real and imaginary parts alike), elsewhere
    (B, l > lb) the diagonal preconditioner.  A block Jacobi preconditioner:
    symmetric and positive definite.  Returns the callable for :func:`pcg`."""
    M = prob.precond_diag()
    L = prob.lmax
    wsum = ring_sum_weights(prob)
    ls, ms = sht.ls_of(L), sht.ms_of(L)
    nb = 1 if prob.ncomp == 1 else 2
    inv = {}
    for m in range(min(lb, L) + 1):
        _, A = azimuthal_te_block(prob, m, lb, wsum)
        inv[m] = (np.where((ms == m) & (ls <= lb))[0], np.linalg.inv(A))

    def apply(r):
        z = np.array(apply_block_inverse(M, r), np.complex128, copy=True)
        for m, (idx, Ai) in inv.items():
            v = np.concatenate([r[c, idx] for c in range(nb)])
            w = Ai @ v.real + 1j * (Ai @ v.imag)
            for c in range(nb):
                z[c, idx] = w[c * idx.size:(c + 1) * idx.size]
        return z

    return apply


# ----------------------------------------------------------------------------
# Per-m dense block solve for azimuthally symmetric noise (App. A)
# ----------------------------------------------------------------------------
def ring_weights(prob: Problem):
    """N^-1 of each ring when it is constant along every ring (App. A: a
    constant-latitude mask with noise that depends on latitude only), else
    None.  Temperature only."""
    g = prob.g
    w = np.zeros(g.nring)
    nv = prob.ninv[0]
    for r in range(g.nring):
        seg = nv[g.ofs[r]:g.ofs[r] + g.nphi[r]]
        if np.any(seg != seg[0]):
            return None
        w[r] = seg[0]
    return w


def azimuthal_block(prob: Problem, m: int, wring):
    """The m-block of A for ring-constant N^-1 (App. A, Eq. N_lml'm'_step in
    its discrete form): with every ring holding nphi >= 2 lmax + 1 pixels the
    phi sum of e^{-i (m - m') phi} vanishes unless m = m', so
    A^(m)_{l l'} = delta_{l l'} / C_l + b_l b_l' sum_r nphi_r w_r
    lambda_lm(theta_r) lambda_l'm(theta_r)
    for l, l' >= m; held multipoles (singular C_l) are identity rows.
    Returns (l values, dense block)."""
    L = prob.lmax
    g = prob.g
    lr = np.arange(m, L + 1)
    lam = np.array([sht.lambda_lm(L, m, g.cth[r], g.sth[r]) for r in range(g.nring)])  # (nring, nl)
    K = (lam * (g.nphi * wring)[:, None]).T @ lam
    bm = prob.bmask[lr]
    A = bm[:, None] * K * bm[None, :]
    act = prob.active[lr]
    A[np.ix_(act, act)] += np.diag(prob.sinv[0, 0][lr][act])
    held = np.where(~act)[0]
    A[held, :] = 0.0
    A[:, held] = 0.0
    A[held, held] = 1.0
    return lr, A


def block_solve(prob: Problem, b):
    """x = A^-1 b by one dense solve per m (App. A), for temperature with
    ring-constant N^-1 on a grid whose rings all have nphi >= 2 lmax + 1."""
    assert prob.ncomp == 1
    wring = ring_weights(prob)
    g = prob.g
    if wring is None or np.any(g.nphi < 2 * prob.lmax + 1):
        raise ValueError("block_solve needs ring-constant N^-1 and nphi >= 2 lmax + 1 on every ring")
    b = np.asarray(b, np.complex128).reshape(1, -1)
    x = np.zeros_like(b)
    ms = sht.ms_of(prob.lmax)
    for m in range(prob.lmax + 1):
        _, A = azimuthal_block(prob, m, wring)
        sel = ms == m
        rhs = b[0, sel]
        x[0, sel] = np.linalg.solve(A, rhs.real) + 1j * np.linalg.solve(A, rhs.imag)
    return _zero_im_m0(x, prob.lmax)


def true_residual(prob: Problem, x, b) -> float:
    b = np.asarray(b, np.complex128).reshape(prob.ncomp, -1)
    r = b - prob.matvec(x)
    return float(np.sqrt(prob.dot(r, r) / prob.dot(b, b)))


# ----------------------------------------------------------------------------
# Gaussian log-posterior (Eq. joint-posterior, a-dependent part)
# ----------------------------------------------------------------------------
def log_posterior(prob: Problem, a, d, cl_scale=None):
    """L(a) = -1/2 (d - Y B a)^T N^-1 (d - Y B a) - 1/2 sum_{l, m=-l..l} |a_lm|^2 / C_l
    for temperature (ncomp = 1), over active l.  ``cl_scale`` multiplies C_l
    per l (the exponent of the binned log C_l parameters)."""
    assert prob.ncomp == 1
    a = np.asarray(a, np.complex128).reshape(1, -1)
    res = np.asarray(d, np.float64).reshape(1, -1) - prob.Y(prob.beam(a))
    chi2 = float(np.sum(res * res * prob.ninv[:1]))
    ic = prob.sinv[0, 0].copy()
    ic[~prob.active] = 0.0
    if cl_scale is not None:
        ic = ic / cl_scale
    prior = prob.dot(a, a * ic[prob.ls][None])
    return -0.5 * chi2 - 0.5 * prior


def log_posterior_grad(prob: Problem, a, d, bins, cl_scale=None):
    """Gradient of :func:`log_posterior` in the metric dot_q6 with respect to
    a (B Y^T N^-1 (d - Y B a) - a / C_l) and with respect to the log C_l of
    each bin (1/2 sum_{l in bin} sum_{m=-l..l} |a_lm|^2 / C_l)."""
    a = np.asarray(a, np.complex128).reshape(1, -1)
    res = np.asarray(d, np.float64).reshape(1, -1) - prob.Y(prob.beam(a))
    ic = prob.sinv[0, 0].copy()
    ic[~prob.active] = 0.0
    if cl_scale is not None:
        ic = ic / cl_scale
    ga = prob.beam(prob.Yt(res * prob.ninv[:1])) - a * ic[prob.ls][None]
    ga = _zero_im_m0(ga, prob.lmax)
    w = np.where(sht.ms_of(prob.lmax) == 0, 1.0, 2.0)
    per_lm = 0.5 * w * np.abs(a[0]) ** 2 * ic[prob.ls]
    gl = np.array([per_lm[(prob.ls >= lo) & (prob.ls <= hi)].sum() for lo, hi in bins])
    return ga, gl


# ----------------------------------------------------------------------------
# Joint (C_l, a) move of Sect. 2.2.2 (Jewell et al. 2009, Racine et al. 2016)
# ----------------------------------------------------------------------------
def _cl_blocks(cl, lmax):
    """(L+1, n, n) per-l signal covariance: C_l (n = 1) or the T/E/B block
    with TE and EB = TB = 0 (n = 3) from (TT, EE, BB, TE)."""
    cl = np.asarray(cl, np.float64)
    if cl.ndim == 1:
        return cl[: lmax + 1, None, None].copy()
    tt, ee, bb, te = cl[:, : lmax + 1]
    C = np.zeros((lmax + 1, 3, 3))
    C[:, 0, 0], C[:, 1, 1], C[:, 2, 2] = tt, ee, bb
    C[:, 0, 1] = C[:, 1, 0] = te
    return C


def fluctuation_rescale(cl_old, cl_new, f, lmax):
    """f^scaled = (C^new_l)^{1/2} (C^old_l)^{-1/2} f_lm, the deterministic
    rescaling of the fluctuation term in the joint move.  Square roots are
    the symmetric principal ones (the reading used for S^-1/2 throughout);
    multipoles where either block is not positive definite (C_0 = C_1 = 0)
    are held at zero, as in the solver.  f: (n, nalm) with n = 1 or 3."""
    f = np.asarray(f, np.complex128)
    n = f.shape[0]
    Co, Cn = _cl_blocks(cl_old, lmax), _cl_blocks(cl_new, lmax)
    ls = sht.ls_of(lmax)
    M = np.zeros((lmax + 1, n, n))
    for l in range(lmax + 1):
        wo, Vo = np.linalg.eigh(Co[l])
        wn, Vn = np.linalg.eigh(Cn[l])
        if np.all(wo > 0) and np.all(wn > 0):
            M[l] = ((Vn * np.sqrt(wn)) @ Vn.T) @ ((Vo / np.sqrt(wo)) @ Vo.T)
    return np.einsum("pij,jp->ip", M[ls], f)


def joint_log_target(prob: Problem, d, a_hat, f_hat):
    """log pi(theta) of the joint move's acceptance rule:
    -1/2 (d - Y B a^)^T N^-1 (d - Y B a^) - 1/2 a^T S^-1 a^
    - 1/2 f^T B Y^T N^-1 Y B f^, with a^ the mean field and f^ the
    fluctuation term (the scaled one for a proposal).  Products in the
    alm metric of dot_q6; S^-1 acts on the active multipoles only."""
    nc = prob.ncomp
    a_hat = np.asarray(a_hat, np.complex128).reshape(nc, -1)
    f_hat = np.asarray(f_hat, np.complex128).reshape(nc, -1)
    nv = prob.ninv_maps()
    res = np.asarray(d, np.float64).reshape(nc, -1) - prob.Y(prob.beam(a_hat))
    chi2 = float(np.sum(res * res * nv))
    sinv = prob.sinv * prob.active[None, None, :]
    prior = prob.dot(a_hat, prob._per_l(sinv, a_hat))
    yf = prob.Y(prob.beam(f_hat))
    fl = float(np.sum(yf * yf * nv))
    return -0.5 * chi2 - 0.5 * prior - 0.5 * fl


def observed_spectrum(r, lmax):
    """C^o_l = 1/(2l+1) sum_{m=-l..l} |r_lm|^2 of a real field stored with
    m >= 0 (the m < 0 terms are the m > 0 ones conjugated)."""
    r = np.asarray(r, np.complex128).reshape(-1)
    ls, ms = sht.ls_of(lmax), sht.ms_of(lmax)
    w = np.where(ms == 0, 1.0, 2.0)
    p = np.bincount(ls, weights=w * np.abs(r) ** 2, minlength=lmax + 1)
    return p / (2.0 * np.arange(lmax + 1) + 1.0)


def exact_harmonic_loglike(cl_obs, cl_theta, bl, nl, lmin=2):
    """Eq. (exact_harm): ln P(theta | r) for full-sky temperature data with
    uniform noise, up to a theta-independent constant:
    sum_l -(2l+1)/2 [x_l - ln x_l], x_l = C^o_l / (b_l^2 C_l(theta) + N_l),
    over l >= lmin."""
    l = np.arange(len(cl_obs))
    sel = l >= lmin
    x = np.asarray(cl_obs)[sel] / (np.asarray(bl)[sel] ** 2 * np.asarray(cl_theta)[sel] + np.asarray(nl)[sel])
    return float(np.sum(-(2.0 * l[sel] + 1.0) / 2.0 * (x - np.log(x))))


def joint_acceptance(log_pi_new, log_pi_old, log_prior_new=0.0, log_prior_old=0.0):
    """A = min[1, pi(theta') P(theta') / (pi(theta) P(theta))] (Eq. acceptance-rate)."""
    return float(min(1.0, np.exp((log_pi_new + log_prior_new) - (log_pi_old + log_prior_old))))

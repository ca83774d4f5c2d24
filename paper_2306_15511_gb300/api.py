"""PyTorch binding of the shtg C ABI.

Tensors provide device memory and the current CUDA stream; every operation
is a call into libshtg.so with the same name as the C entry point.  This
layer only checks shapes, allocates output tensors and passes pointers.

Layouts (see include/shtg.h): alm complex, m-major, nalm = (L+1)(L+2)/2;
maps real in HEALPix RING order; batches outermost; spin-2 alm [.., 2, nalm]
(E, B) and maps [.., 2, npix] (Q, U); T+E+B problems [batch, 3, ...].
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _native as N

_PREC = {torch.complex128: N.FP64, torch.float64: N.FP64,
         torch.complex64: N.FP32, torch.float32: N.FP32}


def _prec(dtype, tensor_cores: bool, double_float: bool = False) -> int:
    if double_float:
        if tensor_cores or dtype not in (torch.complex128, torch.float64):
            raise ValueError("double_float needs complex128 alm / float64 maps (and no tensor_cores)")
        return N.DF64
    if not tensor_cores:
        return _PREC[dtype]
    if dtype not in (torch.complex64, torch.float32):
        raise ValueError("tensor_cores needs complex64 alm / float32 maps")
    return N.TC32


_ARITH = {"default": N.ARITH_DEFAULT, "fp64": N.ARITH_FP64, "df64": N.ARITH_DF64}


def _arith(fp64_arith: str) -> int:
    if fp64_arith not in _ARITH:
        raise ValueError(f"fp64_arith must be one of {sorted(_ARITH)}")
    return _ARITH[fp64_arith]


_PRECOND = {"none": N.PRECOND_NONE, "diag": N.PRECOND_DIAG, "lowl": N.PRECOND_LOWL, "azim": N.PRECOND_AZIM}


def _precond(precond) -> int:
    if precond is True or precond is False:
        return N.PRECOND_DIAG if precond else N.PRECOND_NONE
    if precond not in _PRECOND:
        raise ValueError(f"precond must be True, False or one of {sorted(_PRECOND)}")
    return _PRECOND[precond]


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t) -> C.c_void_p:
    if isinstance(t, np.ndarray):
        return C.c_void_p(t.ctypes.data)
    return C.c_void_p(t.data_ptr())


def _need_cuda(t: torch.Tensor, name: str):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


class Plan:
    """Geometry, tables and workspace for transforms and solves on one grid.

    Plan(nside=N, lmax=L)                      HEALPix RING grid
    Plan(gauss=(nring, nphi), lmax=L)          Gauss-Legendre grid
    max_batch: realizations per call; spin2: also Q/U transforms (T+E+B);
    block_solver: workspace of the exact per-m block solve (mode "block").
    """

    def __init__(self, nside: int | None = None, lmax: int = 0, max_batch: int = 1,
                 spin2: bool = False, gauss: tuple | None = None, block_solver: bool = False):
        lib = N.load()
        self._lib = lib
        h = C.c_void_p()
        flags = N.SPIN0 | (N.SPIN2 if spin2 else 0) | (N.BLOCK_SOLVER if block_solver else 0)
        if gauss is not None:
            rc = lib.shtg_plan_create(N.GEOM_GAUSS, int(gauss[0]), int(gauss[1]), int(lmax),
                                      int(max_batch), flags, C.byref(h))
        else:
            rc = lib.shtg_plan_create(N.GEOM_HEALPIX, int(nside), 0, int(lmax), int(max_batch),
                                      flags, C.byref(h))
        N.check(rc)
        self._h = h
        info = N.PlanInfo()
        N.check(lib.shtg_plan_get_info(h, C.byref(info)))
        self.info = info
        self.lmax, self.npix, self.nalm = info.lmax, int(info.npix), int(info.nalm)
        self.max_batch = info.max_batch
        self.spin2 = bool(info.flags & N.SPIN2)
        self.device = torch.device("cuda", torch.cuda.current_device())

    def close(self):
        if getattr(self, "_h", None):
            self._lib.shtg_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ----------------------------------------------------------- transforms
    def _batched(self, x, spin, inner):
        lead = x.shape[:-2] if spin == 2 else x.shape[:-1]
        nb = int(np.prod(lead)) if len(lead) else 1
        if x.shape[-1] != inner or (spin == 2 and x.shape[-2] != 2):
            raise ValueError(f"expected trailing shape {'(2, ' if spin == 2 else '('}{inner})")
        return lead, nb

    def alm2map(self, alm: torch.Tensor, spin: int = 0, tensor_cores: bool = False,
                double_float: bool = False) -> torch.Tensor:
        """Y: alm [..., nalm] (spin 0) or [..., 2, nalm] (E, B) -> maps.
        tensor_cores (complex64 only): Legendre sum on the tensor cores
        (bf16 hi/lo split products, FP32 accumulation).  double_float
        (complex128 only): FP64-accurate Legendre sum in double-FP32
        arithmetic on the FP32 pipe."""
        _need_cuda(alm, "alm")
        lead, nb = self._batched(alm, spin, self.nalm)
        real = torch.float64 if alm.dtype == torch.complex128 else torch.float32
        out = torch.empty(*lead, *((2,) if spin == 2 else ()), self.npix, dtype=real,
                          device=alm.device)
        N.check(self._lib.shtg_alm2map(self._h, spin, _prec(alm.dtype, tensor_cores, double_float), _ptr(alm), _ptr(out),
                                       nb, _stream()))
        return out

    def alm2map_adjoint(self, m: torch.Tensor, spin: int = 0, tensor_cores: bool = False,
                        double_float: bool = False) -> torch.Tensor:
        """Y^T (exact transpose, no pixel weights): maps -> alm.  tensor_cores
        (float32 only): Legendre sum on the tensor cores; double_float
        (float64 only): in double-FP32 arithmetic."""
        _need_cuda(m, "map")
        lead, nb = self._batched(m, spin, self.npix)
        cplx = torch.complex128 if m.dtype == torch.float64 else torch.complex64
        out = torch.empty(*lead, *((2,) if spin == 2 else ()), self.nalm, dtype=cplx,
                          device=m.device)
        N.check(self._lib.shtg_alm2map_adjoint(self._h, spin, _prec(m.dtype, tensor_cores, double_float), _ptr(m),
                                               _ptr(out), nb, _stream()))
        return out

    def alm2map_vjp(self, g: torch.Tensor, spin: int = 0, tensor_cores: bool = False,
                    double_float: bool = False) -> torch.Tensor:
        """Gradient of a real loss w.r.t. alm (torch convention) from dL/dmap."""
        _need_cuda(g, "map_grad")
        lead, nb = self._batched(g, spin, self.npix)
        cplx = torch.complex128 if g.dtype == torch.float64 else torch.complex64
        out = torch.empty(*lead, *((2,) if spin == 2 else ()), self.nalm, dtype=cplx,
                          device=g.device)
        N.check(self._lib.shtg_alm2map_vjp(self._h, spin, _prec(g.dtype, tensor_cores, double_float), _ptr(g), _ptr(out),
                                           nb, _stream()))
        return out

    def map2alm(self, m: torch.Tensor, spin: int = 0, niter: int = 0) -> torch.Tensor:
        """Quadrature analysis Y^T W with niter Jacobi refinements."""
        _need_cuda(m, "map")
        lead, nb = self._batched(m, spin, self.npix)
        cplx = torch.complex128 if m.dtype == torch.float64 else torch.complex64
        out = torch.empty(*lead, *((2,) if spin == 2 else ()), self.nalm, dtype=cplx,
                          device=m.device)
        N.check(self._lib.shtg_map2alm(self._h, spin, _PREC[m.dtype], _ptr(m), _ptr(out), nb,
                                       int(niter), _stream()))
        return out

    # ---------------------------------------------------------------- solver
    @staticmethod
    def _host_f64(a):
        return np.ascontiguousarray(np.asarray(a, dtype=np.float64))

    def _problem(self, cl, bl, ninv, d=None, w1=None, w2=None, nbatch=1, ncomp=1, cl_scale=None):
        self._keep = [self._host_f64(cl), self._host_f64(bl)]
        pr = N.Problem()
        pr.ncomp, pr.nbatch = ncomp, nbatch
        pr.cl, pr.bl = _ptr(self._keep[0]), _ptr(self._keep[1])
        pr.cl_scale = None
        if cl_scale is not None:
            sc = self._host_f64(cl_scale).reshape(-1)
            if sc.size != nbatch:
                raise ValueError("cl_scale needs one entry per realization")
            self._keep.append(sc)
            pr.cl_scale = _ptr(sc)
        pr.ninv = _ptr(ninv)
        pr.d = _ptr(d) if d is not None else None
        pr.w1 = _ptr(w1) if w1 is not None else None
        pr.w2 = _ptr(w2) if w2 is not None else None
        return pr

    def cg_sample(self, cl, bl, ninv, d, w1, w2, tol: float = 1e-6, mode: str = "mixed",
                  maxiter: int = 4000, precond=True, reliable_delta: float = 1e-2,
                  check_every: int = 4, out=None,
                  allow_not_converged: bool = False, profile: bool = False, graphs: bool = True,
                  cl_scale=None, fp64_arith: str = "default", split: bool = False, lowl_lmax: int = 0,
                  block_lmax: int = 0):
        """Constrained realization(s) of Eq. (mapmakingeq).

        mode: "fp64" (plain FP64 PCG), "mixed" / "mixed_tc" (FP32 PCG with
        FP64-accurate residual replacement; CUDA-core / tensor-core Legendre
        sums) or "block" (exact per-m dense solve of App. A for temperature
        with ring-constant N^-1 on a grid with nphi >= 2 lmax + 1 on every
        ring; the plan needs block_solver=True).

        cl_scale: optional [nbatch] amplitudes; realization b uses cl_scale[b] x cl.

        precond: True / "diag" (the diagonal preconditioner of Sect. 4),
        False / "none", "lowl" (two-level: the exact inverse of the
        operator on the multipoles l <= lowl_lmax, 0 = min(lmax, 32), plus
        the diagonal above) or "azim" (the exact per-m inverse of the
        operator with N^-1 averaged along every ring, App. A's blocks of T
        and E, for l <= block_lmax, 0 = min(lmax, 1024), plus the diagonal
        elsewhere); both built with the first realization's cl_scale and kept
        by the plan while N^-1, C_l, the beam and the scale are unchanged.
        The azimuthal blocks' set-up grows as block_lmax^3 (Gram sums) to
        block_lmax^4 (factorizations): a smaller block_lmax makes the first
        call cheaper and later ones take more iterations.

        split: solve the mean field (Eq. mean-field-map) and the fluctuation
        (Eq. fluc-map) as separate systems of one batch; the result is then
        [2, nbatch, ncomp, nalm] (mean fields, fluctuations) and the plan
        needs max_batch >= 2 nbatch.

        fp64_arith: arithmetic of the FP64-accurate steps (RHS, residual
        replacements; the whole solve in mode "fp64"): "default" (double-FP32
        in the mixed modes, native FP64 in mode "fp64"), "fp64" or "df64".

        graphs: replay one captured PCG iteration as a CUDA graph between the
        convergence checks (same results as eager launches; off while profiling).

        d, w2: [nbatch, ncomp, npix] float64; w1: [nbatch, ncomp, nalm] complex128;
        ninv: [npix] (T) or [2, npix] (T, P).  All CUDA tensors, or all host
        (numpy / pinned CPU tensors) for an end-to-end call with the copies
        inside the library.  Returns (alm [nbatch, ncomp, nalm], stats dict)."""
        host = not (isinstance(d, torch.Tensor) and d.is_cuda)
        nb, nc = int(d.shape[0]), int(d.shape[1])
        nsys = 2 * nb if split else nb
        if out is None:
            if host:
                out = torch.empty(nsys, nc, self.nalm, dtype=torch.complex128).pin_memory()
            else:
                out = torch.empty(nsys, nc, self.nalm, dtype=torch.complex128, device=d.device)
        if out.numel() != nsys * nc * self.nalm:
            raise ValueError("out must hold [2 nbatch if split else nbatch, ncomp, nalm] complex128")
        for t, name in ((d, "d"), (w1, "w1"), (w2, "w2"), (ninv, "ninv"), (out, "out")):
            if isinstance(t, torch.Tensor):
                if t.is_cuda == host:
                    raise ValueError(f"{name}: mix of host and device buffers")
                if not t.is_contiguous():
                    raise ValueError(f"{name} must be contiguous")
        pr = self._problem(cl, bl, ninv, d, w1, w2, nb, nc, cl_scale)
        o = N.CGOpts()
        o.tol, o.maxiter = float(tol), int(maxiter)
        modes = {"fp64": N.CG_FP64, "mixed": N.CG_MIXED, "mixed_tc": N.CG_MIXED_TC, "block": N.CG_BLOCK}
        if mode not in modes:
            raise ValueError(f"mode must be one of {sorted(modes)}")
        o.mode = modes[mode]
        o.precond = _precond(precond)
        o.lowl_lmax, o.block_lmax = int(lowl_lmax), int(block_lmax)
        o.reliable_delta, o.fp64_arith = float(reliable_delta), _arith(fp64_arith)
        o.check_every = int(check_every)
        o.flags = ((N.HOST_INPUTS if host else 0) | (N.PROFILE if profile else 0) |
                   (0 if graphs else N.NO_GRAPHS) | (N.SPLIT_RHS if split else 0))
        st = N.CGStats()
        rc = self._lib.shtg_cg_sample(self._h, C.byref(pr), _ptr(out), C.byref(o), C.byref(st),
                                      _stream())
        N.check(rc, allow=(-3,) if allow_not_converged else ())
        if split:
            out = out.view(2, nb, nc, self.nalm)
        return out, st.as_dict()

    # ----------------------------------------------------------- joint move
    def fluctuation_rescale(self, cl_old, cl_new, f: torch.Tensor, out=None) -> torch.Tensor:
        """f^scaled = (C'_l)^{1/2} (C_l)^{-1/2} f (Sect. 2.2.2) for f
        [nbatch, ncomp, nalm] complex128 (CUDA); cl as for cg_sample."""
        _need_cuda(f, "f")
        nb, nc = int(f.shape[0]), int(f.shape[1])
        if f.dtype != torch.complex128 or f.shape[-1] != self.nalm:
            raise ValueError("f must be [nbatch, ncomp, nalm] complex128")
        out = torch.empty_like(f) if out is None else out
        co, cn = self._host_f64(cl_old), self._host_f64(cl_new)
        N.check(self._lib.shtg_fluctuation_rescale(self._h, nc, _ptr(co), _ptr(cn), _ptr(f), _ptr(out), nb,
                                                   _stream()))
        return out

    def joint_log_target(self, cl, bl, ninv, d, a_hat: torch.Tensor, f_hat: torch.Tensor,
                         precision: str = "df64", cl_scale=None) -> np.ndarray:
        """log pi(theta) of Eq. (acceptance-rate) per realization: the data
        term of the mean field a_hat, its prior term and the noise term of the
        fluctuation f_hat (all CUDA, [nbatch, ncomp, nalm] complex128; d
        [nbatch, ncomp, npix] float64).  precision: "fp64" or "df64" transforms."""
        for t, n in ((a_hat, "a_hat"), (f_hat, "f_hat"), (d, "d"), (ninv, "ninv")):
            _need_cuda(t, n)
        nb, nc = int(d.shape[0]), int(d.shape[1])
        pr = self._problem(cl, bl, ninv, d, None, None, nb, nc, cl_scale)
        lp = np.zeros(nb)
        prec = {"fp64": N.FP64, "df64": N.DF64}[precision]
        N.check(self._lib.shtg_joint_log_target(self._h, C.byref(pr), prec, _ptr(a_hat), _ptr(f_hat),
                                                _ptr(lp), _stream()))
        return lp

    def lowl_block(self, cl, bl, ninv, ncomp: int = 1, lowl_lmax: int = 0, cl_scale=None):
        """The dense low-multipole block H of the two-level preconditioner
        (shtg_lowl_block): returns (H [n, n] float64, params [n, 4] int32 of
        (l, m, component, part)) for the active multipoles l <= l_c."""
        _need_cuda(ninv, "ninv")
        lc = int(lowl_lmax) if lowl_lmax > 0 else min(self.lmax, 32)
        cap = ncomp * (lc + 1) ** 2
        H = np.zeros(cap * cap)
        par = np.zeros(4 * cap, np.int32)
        n = C.c_int(0)
        pr = self._problem(cl, bl, ninv, nbatch=1, ncomp=ncomp, cl_scale=cl_scale)
        N.check(self._lib.shtg_lowl_block(self._h, C.byref(pr), int(lowl_lmax), _ptr(H), _ptr(par),
                                          C.byref(n), _stream()))
        k = n.value
        return H[:k * k].reshape(k, k).copy(), par[:4 * k].reshape(k, 4).copy()

    def precond_apply(self, cl, bl, ninv, r: torch.Tensor, precond="diag", lowl_lmax: int = 0,
                      block_lmax: int = 0, cl_scale=None, fp32: bool = False) -> torch.Tensor:
        """z = M^-1 r with the solver's preconditioner (shtg_precond_apply)
        for r [nbatch, ncomp, nalm] complex128 (CUDA); fp32: what the FP32
        iteration of the mixed solver applies."""
        _need_cuda(r, "r")
        z = torch.empty_like(r)
        pr = self._problem(cl, bl, ninv, nbatch=int(r.shape[0]), ncomp=int(r.shape[1]), cl_scale=cl_scale)
        o = N.CGOpts()
        o.precond = _precond(precond)
        o.lowl_lmax, o.block_lmax = int(lowl_lmax), int(block_lmax)
        o.mode = N.CG_MIXED if fp32 else N.CG_FP64
        N.check(self._lib.shtg_precond_apply(self._h, C.byref(pr), C.byref(o), _ptr(r.contiguous()), _ptr(z),
                                             _stream()))
        return z

    def apply_operator(self, cl, bl, ninv, x: torch.Tensor, cl_scale=None) -> torch.Tensor:
        """y = (S^-1 + B Y^T N^-1 Y B) x for x [nbatch, ncomp, nalm] complex128 (CUDA)."""
        _need_cuda(x, "x")
        y = torch.empty_like(x)
        pr = self._problem(cl, bl, ninv, nbatch=int(x.shape[0]), ncomp=int(x.shape[1]), cl_scale=cl_scale)
        N.check(self._lib.shtg_apply_operator(self._h, C.byref(pr), _ptr(x), _ptr(y), _stream()))
        return y

    def logpost_grad(self, cl, bl, alm: torch.Tensor, d: torch.Tensor, ninv: torch.Tensor,
                     bins=(), components: bool = False, want_grad: bool = True, theta=None):
        """Log-posterior of Eq. (joint-posterior) (temperature) with its
        gradient w.r.t. alm (complex64) and the log C_l of each bin.  theta:
        optional per-bin log offsets (C_l -> C_l exp(theta_k) on bin k, applied
        by the library)."""
        for t, n in ((alm, "alm"), (d, "d"), (ninv, "ninv")):
            _need_cuda(t, n)
        cl_h, bl_h = self._host_f64(cl), self._host_f64(bl)
        lo = np.ascontiguousarray([b[0] for b in bins], dtype=np.int32)
        hi = np.ascontiguousarray([b[1] for b in bins], dtype=np.int32)
        th = None
        if theta is not None:
            th = self._host_f64(theta).reshape(-1)
            if th.size != len(bins):
                raise ValueError("theta needs one entry per bin")
        g = torch.empty_like(alm) if want_grad else None
        gcl = np.zeros(len(bins))
        logp = C.c_double(0.0)
        N.check(self._lib.shtg_logpost_grad_binned(
            self._h, _ptr(cl_h), _ptr(bl_h), _ptr(alm), _ptr(d), _ptr(ninv), len(bins),
            _ptr(lo) if len(bins) else None, _ptr(hi) if len(bins) else None,
            _ptr(th) if th is not None else None,
            N.GRAD_COMPONENTS if components else 0, C.byref(logp),
            _ptr(g) if g is not None else None, _ptr(gcl) if len(bins) else None, _stream()))
        return logp.value, g, gcl


def joint_acceptance(log_pi_new: float, log_pi_old: float, log_prior_new: float = 0.0,
                     log_prior_old: float = 0.0) -> float:
    """Acceptance probability of the joint move, Eq. (acceptance-rate)."""
    a = C.c_double(0.0)
    N.check(N.load().shtg_joint_acceptance(float(log_pi_new), float(log_pi_old), float(log_prior_new),
                                           float(log_prior_old), C.byref(a)))
    return a.value


def fma_peak(precision: str = "fp32"):
    """Measured FMA throughput of the current GPU: (SM count, TFLOP/s) for
    precision "fp32" or "fp64" (2 flops per FMA)."""
    lib = N.load()
    sms, tf = C.c_int(0), C.c_double(0.0)
    N.check(lib.shtg_probe_fma_peak(N.FP32 if precision == "fp32" else N.FP64, C.byref(sms),
                                    C.byref(tf), _stream()))
    return sms.value, tf.value


def chains_sample(groups, tol: float = 1e-6, mode: str = "mixed_tc", maxiter: int = 4000,
                  precond=True, reliable_delta: float = 1e-2, check_every: int = 4,
                  allow_not_converged: bool = False, graphs: bool = True, fp64_arith: str = "default",
                  lowl_lmax: int = 0, block_lmax: int = 0, grouped: bool = False):
    """Constrained realizations of many chains of uneven geometry in one call.

    groups: list of dicts, one per geometry, with keys plan, cl, bl, ninv, d,
    w1, w2 (CUDA tensors shaped as for Plan.cg_sample) and optionally
    cl_scale (one amplitude per realization of the group).  Every group needs
    its own Plan.  grouped=True runs every stage of the FP32 iteration as one
    launch over all groups (SHTG_GROUPED) instead of the groups concurrently
    on their plans' streams.  Returns a list of (alm, stats) per group."""
    if not groups:
        raise ValueError("no groups")
    lib = N.load()
    n = len(groups)
    plans = (C.c_void_p * n)()
    probs = (N.Problem * n)()
    outs = (C.c_void_p * n)()
    stats = (N.CGStats * n)()
    keep, results = [], []
    for g, grp in enumerate(groups):
        plan, d = grp["plan"], grp["d"]
        for name in ("d", "w1", "w2", "ninv"):
            _need_cuda(grp[name], name)
        nb, nc = int(d.shape[0]), int(d.shape[1])
        out = torch.empty(nb, nc, plan.nalm, dtype=torch.complex128, device=d.device)
        pr = plan._problem(grp["cl"], grp["bl"], grp["ninv"], d, grp["w1"], grp["w2"], nb, nc,
                           grp.get("cl_scale"))
        keep.append(list(plan._keep))
        plans[g] = plan._h
        probs[g] = pr
        outs[g] = out.data_ptr()
        results.append(out)
    o = N.CGOpts()
    o.tol, o.maxiter = float(tol), int(maxiter)
    modes = {"fp64": N.CG_FP64, "mixed": N.CG_MIXED, "mixed_tc": N.CG_MIXED_TC}
    if mode not in modes:
        raise ValueError(f"mode must be one of {sorted(modes)}")
    o.mode = modes[mode]
    o.precond = _precond(precond)
    o.lowl_lmax, o.block_lmax = int(lowl_lmax), int(block_lmax)
    o.reliable_delta, o.fp64_arith = float(reliable_delta), _arith(fp64_arith)
    o.check_every = int(check_every)
    o.flags = (0 if graphs else N.NO_GRAPHS) | (N.GROUPED if grouped else 0)
    rc = lib.shtg_cg_sample_chains(n, plans, probs, outs, C.byref(o), stats, _stream())
    N.check(rc, allow=(-3,) if allow_not_converged else ())
    del keep
    return [(results[g], stats[g].as_dict()) for g in range(n)]


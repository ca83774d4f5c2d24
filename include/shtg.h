/*
 * shtg: GB300 (sm_103a) constrained-realization sampler for CMB skies.
 *
 * C ABI of the data-parallel hot path of Eskilt et al., "Cosmoglobe: Towards
 * end-to-end CMB cosmological parameter estimation without likelihood
 * approximations" (arXiv 2306.15511), Sect. 2.2.1: drawing a constrained
 * realization by preconditioned conjugate gradients on Eq. (mapmakingeq),
 *
 *     (S^-1 + B Y^T N^-1 Y B) a = B Y^T N^-1 d + S^-1/2 w1 + B Y^T N^-1/2 w2,
 *
 * where Y is the spherical-harmonic synthesis on the iso-latitude rings of a
 * HEALPix (or Gauss-Legendre) grid, B the harmonic beam b_l, S the signal
 * covariance C_l (or the 3x3 T/E/B block of Sect. 2.2.2 with EB = TB = 0) and
 * N^-1 a diagonal pixel weight that is 0 in the mask (App. A).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - alm: complex, interleaved (re, im), m-major with m >= 0 only:
 *   index(l, m) = m (2 lmax + 1 - m) / 2 + l, nalm = (lmax+1)(lmax+2)/2.
 *   Batches are outermost; T+E+B alm are [batch][3][nalm].  The imaginary
 *   part of a_l0 is ignored on input and written as 0 on output.
 * - Y_lm = lambda_lm(theta) e^{i m phi}, orthonormal, Condon-Shortley phase
 *   (App. A: P~_lm = Delta_lm P_lm with the (-1)^m in Delta_lm).
 *   Spin 2: Q +- iU = sum +-2a_lm +-2Y_lm with +-2a_lm = -(E_lm +- i B_lm),
 *   where +-2Y_lm = sqrt((l-2)!/(l+2)!) edth^2 (edth-bar^2) Y_lm.
 * - maps: real, RING order, [batch][npix] (spin 0) or [batch][2][npix] = Q, U.
 * - Y^T is the exact transpose of Y in the metric
 *   <a, c> = sum_l [a_l0 c_l0 + 2 Re sum_{m>0} conj(a_lm) c_lm]; every CG
 *   inner product and residual norm uses this metric.
 * - "precision" selects SHTG_FP64 or SHTG_DF64 (double / complex128 buffers;
 *   native FP64 or double-FP32 arithmetic in the Legendre sums) or SHTG_FP32
 *   or SHTG_TC32 (float / complex64 buffers; CUDA cores or tensor cores in
 *   the Legendre sums) for a transform.
 * - Device buffers are owned by the caller; the library never frees them.
 *   Plans own their tables and workspace.  No entry point allocates device
 *   memory after shtg_plan_create.  Calls on one plan must not overlap.
 * - stream: a cudaStream_t passed as void* (NULL = legacy default stream).
 *   Transforms are asynchronous on that stream; cg_sample synchronizes it.
 * - Every call returns SHTG_OK (0) or a negative error code; no call throws
 *   across the ABI.  shtg_last_error_string() describes the last failure on
 *   the calling thread.
 */
#ifndef SHTG_H
#define SHTG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ errors */
#define SHTG_OK 0
#define SHTG_ERR_ARG (-1)            /* invalid argument or unsupported size */
#define SHTG_ERR_CUDA (-2)           /* a CUDA runtime call failed */
#define SHTG_ERR_NOT_CONVERGED (-3)  /* maxiter reached; output holds the best iterate */
#define SHTG_ERR_TIMEOUT (-4)        /* a bounded device-side wait expired */
#define SHTG_ERR_NONFINITE (-5)      /* NaN or Inf met in inputs or iterates */
#define SHTG_ERR_NOT_SPD (-6)        /* C_l block not positive definite where b_l != 0 */
#define SHTG_ERR_NOMEM (-7)          /* plan creation could not allocate */

/* ---------------------------------------------------------------- options */
#define SHTG_GEOM_HEALPIX 0          /* nside_or_nring = N_side; 12 N_side^2 pixels */
#define SHTG_GEOM_GAUSS 1            /* nside_or_nring = rings; nphi_gauss pixels each */

#define SHTG_FP64 0
#define SHTG_FP32 1
#define SHTG_DF64 3                  /* FP64 buffers; Legendre sums of alm2map, alm2map_adjoint and
                                        alm2map_vjp in double-FP32 arithmetic (SHTG_ARITH_DF64);
                                        map2alm runs the FP64 path */
#define SHTG_TC32 2                  /* FP32 buffers; Legendre sums of alm2map, alm2map_adjoint
                                        and alm2map_vjp on the tensor cores (FP32 recurrence,
                                        bf16 hi/lo split products, FP32 accumulation: ~2^-16
                                        relative per term); map2alm runs the FP32 path; these
                                        calls synchronize the stream to check the kernels'
                                        bounded waits (SHTG_ERR_TIMEOUT if one expired) */

#define SHTG_SPIN0 1                 /* plan flag: temperature transforms */
#define SHTG_SPIN2 2                 /* plan flag: also spin-2 (Q, U) transforms */
#define SHTG_BLOCK_SOLVER 4          /* plan flag: also the workspace of SHTG_CG_BLOCK (per-m blocks of
                                        one chunk of m, at most 512 MB, and their recurrence values,
                                        at most 256 MB) */

#define SHTG_CG_FP64 0               /* plain FP64 PCG */
#define SHTG_CG_MIXED 1              /* FP32 PCG inside FP64-accurate iterative refinement
                                        (residual replacement; arithmetic: fp64_arith) */
#define SHTG_CG_MIXED_TC 2           /* as SHTG_CG_MIXED with the FP32 operator's Legendre
                                        sums on the tensor cores (SHTG_TC32) */
#define SHTG_CG_BLOCK 3              /* exact solve by one dense FP64 Cholesky per m (App. A): for
                                        temperature with N^-1 constant along every ring on a grid whose
                                        rings all have nphi >= 2 lmax + 1 (e.g. Gauss-Legendre with
                                        nphi_gauss >= 2 lmax + 1), where A is block-diagonal in m; the
                                        realizations share one C_l scale; the plan needs
                                        SHTG_BLOCK_SOLVER; SHTG_ERR_ARG when a condition fails */

#define SHTG_PRECOND_NONE 0          /* shtg_cg_opts.precond */
#define SHTG_PRECOND_DIAG 1
#define SHTG_PRECOND_LOWL 2
#define SHTG_PRECOND_AZIM 3
#define SHTG_ARITH_DEFAULT 0         /* shtg_cg_opts.fp64_arith */
#define SHTG_ARITH_FP64 1            /* native FP64 multiply-adds */
#define SHTG_ARITH_DF64 2            /* Legendre sums in double-FP32 (hi + lo float pairs, ~2^-47
                                        relative per operation) on the FP32 pipe, FP64 storage and
                                        FP64 ring FFTs; the transforms agree with SHTG_ARITH_FP64
                                        to 1e-12 relative (tested) */

#define SHTG_HOST_INPUTS 1           /* cg_sample flag: problem maps/alm and output are host pointers */
#define SHTG_PROFILE 2               /* cg_sample flag: time kernel classes with CUDA events */
#define SHTG_SPLIT_RHS 8             /* cg_sample flag: solve the mean field of Eq. (mean-field-map),
                                        A a^ = B Y^T N^-1 d, and the fluctuation of Eq. (fluc-map),
                                        A f^ = S^-1/2 w1 + B Y^T N^-1/2 w2, as 2 nbatch systems of one
                                        batch; alm_out is then [2][nbatch][ncomp][nalm] (the nbatch
                                        mean fields, then the nbatch fluctuations; a = a^ + f^) and the
                                        plan needs max_batch >= 2 nbatch */
#define SHTG_NO_GRAPHS 4             /* cg_sample flag: launch every PCG iteration eagerly instead of
                                        replaying one captured iteration as a CUDA graph (graphs are
                                        also off with SHTG_PROFILE, or with SHTG_GRAPHS=0 in the
                                        environment); results are identical either way */
#define SHTG_GROUPED 16              /* cg_sample_chains flag: run the FP32 PCG iterations of all
                                        groups together, each stage one launch over the work of every
                                        geometry (see shtg_cg_sample_chains) */

typedef struct shtg_plan shtg_plan;

typedef struct {
    int geom, nside, nring, lmax, max_batch, flags;
    int64_t npix, nalm;
    int64_t device_bytes;            /* device memory owned by the plan */
} shtg_plan_info;

/* Create a plan: ring geometry, FP64 start states of the Legendre recurrence
 * (the sectoral values lambda_mm and the first l at which lambda_lm(theta_r)
 * leaves the negligible range, computed once in FP64 with exponent
 * rescaling), recurrence coefficients, ring-FFT tables and the workspace for
 * up to max_batch maps (max_batch realizations of T, or of T+E+B when flags
 * has SHTG_SPIN2).  For SHTG_GEOM_GAUSS, nphi_gauss >= 2 lmax + 1 makes the
 * quadrature exact; it is ignored for HEALPix.  flags: SHTG_SPIN0 and/or
 * SHTG_SPIN2.  Limits (SHTG_ERR_ARG outside them): 0 <= lmax <= 8192,
 * 1 <= max_batch <= 4096; HEALPix 1 <= N_side <= 8192 and lmax <= 4 N_side;
 * Gauss-Legendre 1 <= rings <= 65536 and 1 <= nphi_gauss <= 65536; every
 * ring's FFT length within the ring stage's range of 2^13 points, Bluestein
 * lengths included (HEALPix N_side <= 1024; Gauss-Legendre nphi a power of
 * two <= 8192, or any nphi <= 4096).  Returns
 * SHTG_ERR_NOMEM if device memory is insufficient.  Sets *out on success. */
int shtg_plan_create(int geom, int nside_or_nring, int nphi_gauss, int lmax, int max_batch,
                     int flags, shtg_plan **out);
int shtg_plan_destroy(shtg_plan *plan);
int shtg_plan_get_info(const shtg_plan *plan, shtg_plan_info *info);
const char *shtg_last_error_string(void);
/* Interface version: 3 (2 + the flag SHTG_GROUPED of shtg_cg_sample_chains;
 * 2 = 1 + SHTG_DF64 and shtg_cg_opts.fp64_arith, which was a reserved field
 * set to 0 with the same layout). */
int shtg_version(void);

/* Y (Sect. 2.1, a(n) = sum a_lm Y_lm(n); App. A pixel sums):
 * alm [nbatch][nalm] -> map [nbatch][npix] for spin 0, or
 * alm [nbatch][2][nalm] (E, B) -> map [nbatch][2][npix] (Q, U) for spin 2.
 * Device pointers; nbatch <= max_batch (x2 components for spin 2 count
 * against 3 * max_batch maps). */
int shtg_alm2map(shtg_plan *plan, int spin, int precision, const void *alm, void *map,
                 int nbatch, void *stream);

/* Y^T, the exact transpose of shtg_alm2map (no pixel weights):
 * c_lm = sum_p map_p Y*_lm(p) (spin 0); the spin-2 form is the transpose of
 * the (E, B) -> (Q, U) map above.  This is the operator B Y^T of Eq.
 * (mapmakingeq) before the beam. */
int shtg_alm2map_adjoint(shtg_plan *plan, int spin, int precision, const void *map, void *alm,
                         int nbatch, void *stream);

/* Vector-Jacobian product of shtg_alm2map for autodiff: given dL/dmap,
 * returns dL/d(Re a_lm) + i dL/d(Im a_lm), which is w_m (Y^T dL/dmap)_lm with
 * w_0 = 1, w_m = 2 for m > 0 (the factor 2 accounts for the conjugate
 * coefficient a_l,-m that each stored a_lm stands for).  Same layouts as
 * shtg_alm2map_adjoint. */
int shtg_alm2map_vjp(shtg_plan *plan, int spin, int precision, const void *map_grad,
                     void *alm_grad, int nbatch, void *stream);

/* Quadrature analysis: Y^T W map with the geometry's pixel weights
 * (HEALPix 4 pi / N_pix; Gauss-Legendre w_k 2 pi / nphi), followed by niter
 * Jacobi refinements alm += Y^T W (map - Y alm).  Exact inverse of alm2map on
 * a Gauss-Legendre plan with nring >= lmax + 1, nphi >= 2 lmax + 1.
 * niter > 0 uses the plan's scratch map (single call at a time per plan). */
int shtg_map2alm(shtg_plan *plan, int spin, int precision, const void *map, void *alm,
                 int nbatch, int niter, void *stream);

/* Allocation-free Y^T for callers that cannot allocate device memory (code
 * that runs under a device-memory budget owned by another framework, or that
 * may not call cudaMalloc because it can synchronize the device).  The paper
 * has no counterpart.  Same result as shtg_alm2map_adjoint(spin 0, SHTG_FP64)
 * on a HEALPix plan, without a plan: map [12 nside^2] float64 and alm [nalm]
 * complex128 are device buffers owned by the caller; the ring geometry and
 * the Legendre recurrence are computed on the fly and the per-ring Fourier
 * sums go to a static 16 MiB device buffer inside the library.  Needs
 * 1 <= nside <= 8192, 0 <= lmax <= 4 nside and non-null buffers; sizes with
 * (4 nside - 1) (lmax + 1) 16 bytes > 16 MiB (e.g. nside 512, lmax 1024)
 * return SHTG_ERR_ARG like any other invalid argument.  The first call on a
 * device does the set-up: it looks the buffer's device address up
 * (cudaGetSymbolAddress) and caches it for that device.  With lazy module
 * loading (the CUDA default) that lookup also loads this part of the library
 * onto the device, which reserves the 16 MiB buffer and may synchronize the
 * device; so make the first call during set-up, outside any stream capture
 * and outside any region whose memory budget or timing must not be touched.
 * The cached address does not survive cudaDeviceReset: do not call this entry
 * point on a device after resetting it.  Every call on a device shares the
 * buffer: calls whose kernels may overlap on the GPU race on it.  Each c_lm is
 * accumulated from the ring pairs with FP64 atomic additions, whose order
 * varies from run to run, so two identical calls may differ by rounding
 * (results are not bitwise reproducible; the plan-based transpose is).
 * Allocates nothing after that set-up. */
int shtg_alm2map_adjoint_noalloc(int nside, int lmax, const double *map, double *alm, void *stream);

/* Measurement helper (the paper has no counterpart): the fused multiply-add
 * throughput of the current device at its current clocks, for the roofline
 * of the Legendre kernels.  precision: SHTG_FP32 or SHTG_FP64.  Each thread
 * of a grid that fills every SM runs 8 independent FMA chains; 2 flops per
 * FMA.  Writes the SM count and the measured TFLOP/s; synchronizes the
 * stream; allocates and frees a small output buffer (stream-ordered). */
int shtg_probe_fma_peak(int precision, int *sm_count, double *tflops, void *stream);

/* ------------------------------------------------- constrained realization */
typedef struct {
    int ncomp;        /* 1 = temperature; 3 = T, E, B (plan needs SHTG_SPIN2) */
    int nbatch;       /* realizations that share cl, bl and ninv (<= max_batch) */
    const double *cl; /* HOST. ncomp 1: [lmax+1] C_l; ncomp 3: [4][lmax+1] = TT, EE, BB, TE.
                         Multipoles whose block is singular (e.g. C_0 = C_1 = 0) are held at 0. */
    const double *bl; /* HOST. [lmax+1] beam transfer function b_l */
    const double *ninv; /* [npix] (T) or [2][npix] (T, then Q and U), N^-1 per pixel, 0 = masked */
    const double *d;  /* [nbatch][ncomp][npix] data maps (T or T, Q, U) */
    const double *w1; /* [nbatch][ncomp][nalm] complex128 unit white noise in harmonic space */
    const double *w2; /* [nbatch][ncomp][npix] unit white noise in pixel space */
    const double *cl_scale; /* HOST, optional. [nbatch]: realization b's C_l (the whole T/E/B
                               block) is cl_scale[b] x cl; null = all 1.  Independent chains of
                               one geometry with different signal amplitudes share one call.
                               Entries must be positive. */
} shtg_problem;

typedef struct {
    double tol;         /* stop when ||b - A x|| / ||b|| <= tol for every realization */
    int maxiter;        /* PCG iterations (FP64 mode) or FP32 iterations (mixed) */
    int mode;           /* SHTG_CG_FP64, SHTG_CG_MIXED, SHTG_CG_MIXED_TC or SHTG_CG_BLOCK */
    int precond;        /* SHTG_PRECOND_DIAG (1): diagonal preconditioner of Sect. 4 (default);
                           SHTG_PRECOND_NONE (0); SHTG_PRECOND_LOWL (2): two-level, the exact
                           inverse of the operator on l <= lowl_lmax plus the diagonal above;
                           SHTG_PRECOND_AZIM (3): azimuthal blocks, the exact per-m inverse of the
                           operator with N^-1 averaged along every ring (App. A's blocks of T and
                           E) for l <= block_lmax plus the diagonal elsewhere */
    double reliable_delta; /* mixed mode: an FP64 residual replacement happens when the FP32
                              residual has dropped by this factor since the last one (default 1e-2) */
    int fp64_arith;     /* arithmetic of the FP64-accurate steps (RHS, residual replacements,
                           the whole FP64 PCG): SHTG_ARITH_DEFAULT (0: double-FP32 in the mixed
                           modes, native FP64 in SHTG_CG_FP64), SHTG_ARITH_FP64 or
                           SHTG_ARITH_DF64 */
    int check_every;    /* iterations per CUDA graph launch between host convergence checks */
    int flags;          /* SHTG_HOST_INPUTS: ninv, d, w1, w2 and alm_out are host memory */
    int lowl_lmax;      /* SHTG_PRECOND_LOWL: l_c, the largest multipole of the dense block
                           (0: min(lmax, 32); at most min(lmax, 48)) */
    int block_lmax;     /* SHTG_PRECOND_AZIM: the largest multipole of the per-m blocks
                           (0: min(lmax, 1024); at most lmax) */
} shtg_cg_opts;

typedef struct {
    int iterations;     /* PCG iterations (mixed: FP32 iterations) */
    int outer_steps;    /* mixed mode: FP64 residual replacements */
    int fp64_matvecs;   /* FP64 operator applications, RHS excluded */
    int converged;      /* 1 if every realization met tol */
    double rel_residual;/* max over the batch of the FP64 ||b - A x|| / ||b|| at exit */
    double ms_setup, ms_rhs, ms_solve, ms_total;
    long long launches;        /* CUDA kernels the call launched */
    /* with SHTG_PROFILE: summed CUDA-event time and launch count per kernel
     * class: 0 Legendre synthesis FP32, 1 Legendre analysis FP32, 2 ring FFT
     * FP32, 3 Legendre synthesis FP64, 4 Legendre analysis FP64, 5 ring FFT
     * FP64, 6 vector / reduction kernels, 7 preconditioner diagonal */
    double kernel_ms[8];
    int kernel_launches[8];
} shtg_cg_stats;

/* Draw nbatch constrained realizations, a = x solving Eq. (mapmakingeq)
 * (Sect. 2.2.1): RHS b = B Y^T (N^-1 d + N^-1/2 w2) + S^-1/2 w1 with S^-1/2
 * the inverse symmetric square root of the C_l block; PCG with the
 * diagonal preconditioner M = S^-1 + b_l^2 D_lm, D_lm = sum_r g_lm(theta_r)
 * sum_{p in r} N^-1_p (g = lambda^2, or the spin-2 analogue).  Mixed mode
 * runs the PCG on FP32 vectors and transforms and replaces its residual by
 * the FP64 b - A x (FP64 transforms) each time it has dropped by
 * reliable_delta, keeping the search direction; x accumulates in FP64 and
 * convergence is judged on the FP64 residual.  alm_out:
 * [nbatch][ncomp][nalm] complex128.  Returns SHTG_ERR_NOT_CONVERGED (output =
 * last iterate, stats filled) if maxiter is hit.  opts may be NULL (tol 1e-6,
 * mixed, preconditioned). */
int shtg_cg_sample(shtg_plan *plan, const shtg_problem *prob, double *alm_out,
                   const shtg_cg_opts *opts, shtg_cg_stats *stats, void *stream);

/* Many independent chains of uneven geometry in one call (the batching of
 * Sect. 2.2 across Gibbs chains): group g's realizations share the geometry
 * of plans[g] (its N_side, l_max), its beam and N^-1, and are problems[g]
 * (nbatch realizations with their own amplitudes through cl_scale);
 * alm_out[g] as in shtg_cg_sample.  Every group needs its own plan.  Groups
 * run concurrently, each on its plan's own stream, after the work queued on
 * `stream` and before anything queued on it later; realizations that have
 * converged stop updating while the others go on.  stats: [ngroups] or
 * NULL.  Returns the first error other than SHTG_ERR_NOT_CONVERGED, else
 * SHTG_ERR_NOT_CONVERGED if a group did not converge, else SHTG_OK; the
 * error string names the group.
 *
 * With SHTG_GROUPED in opts->flags (batching of chains of uneven N_side and
 * l_max in one launch per stage): the groups run in lockstep on `stream`
 * instead of concurrently, and every stage of their FP32 PCG iteration is one
 * kernel launch over the work of all groups (Legendre synthesis and transpose
 * on the CUDA cores, the prior, the CG scalar and vector updates, the
 * azimuthal blocks; the ring stage is one launch per transform-length class,
 * at most five), replayed as one CUDA graph; a group whose realizations have
 * all converged is skipped on the device.  The FP64-accurate steps (the
 * right-hand sides, each group's residual replacements) stay per group.
 * Needs 1 <= ngroups <= 16, non-null opts with mode SHTG_CG_MIXED or
 * SHTG_CG_MIXED_TC (both run the CUDA-core FP32 Legendre sums here),
 * precond SHTG_PRECOND_NONE, SHTG_PRECOND_DIAG or SHTG_PRECOND_AZIM, the
 * same ncomp in every group and neither SHTG_SPLIT_RHS nor SHTG_PROFILE;
 * otherwise SHTG_ERR_ARG.  Uses each plan's workspace and d_flag slot as the
 * plain call does; allocates nothing beyond what the chosen preconditioner
 * allocates in a plain call. */
int shtg_cg_sample_chains(int ngroups, shtg_plan *const *plans, const shtg_problem *problems,
                          double *const *alm_out, const shtg_cg_opts *opts, shtg_cg_stats *stats,
                          void *stream);

/* Apply the operator A of Eq. (mapmakingeq) once: y = S^-1 x + B Y^T N^-1 Y B x
 * (x, y: device [nbatch][ncomp][nalm] complex128, FP64), using the problem's
 * cl, bl and ninv (d, w1, w2 unused).  Held multipoles pass through (y = x). */
int shtg_apply_operator(shtg_plan *plan, const shtg_problem *prob, const double *x, double *y,
                        void *stream);

/* The dense low-multipole block of SHTG_PRECOND_LOWL (the paper's Sect. 4
 * asks for preconditioners beyond the diagonal one; this is the coarse level
 * of a two-level one).  In the real parametrization a_lm = u + i v (no v at
 * m = 0) with the metric weight w = 1 for m = 0, 2 otherwise, the operator A
 * of Eq. (mapmakingeq) restricted to the active multipoles l <= l_c is
 * W^-1 H with the symmetric
 *   H_ij = b_l(i) b_l(j) sum_p N^-1_p phi_i(p) phi_j(p)
 *          + w_i [S^-1 / cl_scale[0]]_{comp(i) comp(j)} (same l, m, part),
 * phi_i the pixel field of a unit parameter (App. A's ring-pair sums with
 * each ring's Fourier coefficients of N^-1).  Writes H (HOST, [n][n] row
 * major; capacity (ncomp (l_c+1)^2)^2 doubles), params (HOST, [n][4] ints
 * l, m, component 0 T / 1 E / 2 B, part 0 u / 1 v; capacity 4 ncomp
 * (l_c+1)^2, may be NULL) and n.  Uses cl, bl, ninv (d, w1, w2 unused);
 * l_c = 0 is the default.  Inactive multipoles (singular C_l block) are left
 * out.  Synchronizes the stream; the workspace stays with the plan.
 * SHTG_ERR_NOT_SPD if the block is not positive definite. */
int shtg_lowl_block(shtg_plan *plan, const shtg_problem *prob, int lowl_lmax, double *H, int *params, int *n,
                    void *stream);

/* Apply the solver's preconditioner once (Sect. 4 and the options above):
 * z = M^-1 r for r, z device [nbatch][ncomp][nalm] complex128 (FP64, the
 * azimuthal blocks' FP64 inverses; with opts->mode SHTG_CG_MIXED or
 * SHTG_CG_MIXED_TC what the FP32 iteration applies: r rounded to FP32, FP32
 * diagonal and block inverses, z widened back), with the problem's cl, bl,
 * ninv and cl_scale (d, w1, w2 unused) and opts->precond, lowl_lmax and
 * block_lmax.  Builds what the preconditioner needs like shtg_cg_sample
 * (the workspace of SHTG_PRECOND_LOWL and SHTG_PRECOND_AZIM stays with the
 * plan).  Synchronizes the stream. */
int shtg_precond_apply(shtg_plan *plan, const shtg_problem *prob, const shtg_cg_opts *opts, const double *r,
                       double *z, void *stream);

/* ------------------------------------------- joint (C_l, a) move (Sect. 2.2.2) */
/* The deterministic rescaling of the fluctuation term,
 * f^scaled_lm = (C'_l)^{1/2} (C_l)^{-1/2} f^_lm, per l with the T/E/B block
 * of Sect. 2.2.2 (EB = TB = 0) and the symmetric principal square roots;
 * multipoles where either block is singular are set to 0.  cl_old, cl_new:
 * HOST, as shtg_problem.cl ([lmax+1] for ncomp 1, [4][lmax+1] = TT, EE, BB,
 * TE for ncomp 3).  f, f_out: device [nbatch][ncomp][nalm] complex128 (may be
 * the same buffer).  Synchronizes the stream. */
int shtg_fluctuation_rescale(shtg_plan *plan, int ncomp, const double *cl_old, const double *cl_new,
                             const double *f, double *f_out, int nbatch, void *stream);

/* log pi(theta) of the joint move's acceptance rule (Eq. acceptance-rate),
 * per realization b of prob (cl, bl, ninv, d, nbatch, ncomp, cl_scale used):
 * log pi = -1/2 (d - Y B a^)^T N^-1 (d - Y B a^) - 1/2 a^T S^-1 a^
 *          - 1/2 f^T B Y^T N^-1 Y B f^
 * with a^ the mean field and f^ the (scaled, for a proposal) fluctuation;
 * alm products in the metric above, S^-1 over the multipoles with a
 * non-singular block.  The prior term, printed with a and a^, is read as
 * a^T S^-1 a^.  a_hat, f_hat: device [nbatch][ncomp][nalm] complex128; d as in
 * shtg_problem (device).  precision SHTG_FP64 or SHTG_DF64 selects the
 * arithmetic of the synthesis (both FP64-accurate); sums in FP64.
 * log_pi: HOST [nbatch].  Synchronizes the stream. */
int shtg_joint_log_target(shtg_plan *plan, const shtg_problem *prob, int precision, const double *a_hat,
                          const double *f_hat, double *log_pi, void *stream);

/* Acceptance probability of the joint move (Eq. acceptance-rate):
 * A = min[1, pi(theta') P(theta') / (pi(theta) P(theta))] from the logs of
 * pi and of the prior P.  Host arithmetic only (no device work). */
int shtg_joint_acceptance(double log_pi_new, double log_pi_old, double log_prior_new, double log_prior_old,
                          double *accept);

/* --------------------------------------------------- log-posterior (grad) */
#define SHTG_GRAD_COMPONENTS 1   /* logpost flag: grad_alm as d/dRe + i d/dIm (x2 for m > 0) */

/* Gaussian log-posterior of Eq. (joint-posterior), a-dependent part, for
 * temperature: L = -1/2 (d - Y B a)^T N^-1 (d - Y B a) - 1/2 sum_{l, m=-l..l}
 * |a_lm|^2 / C_l over multipoles with C_l > 0.  FP32 transforms with FP64
 * reductions.  Inputs (device): alm [nalm] complex64, d [npix] float32,
 * ninv [npix] float32; host cl, bl [lmax+1].  Outputs: *logp (host),
 * grad_alm [nalm] complex64 (device; gradient in the metric above:
 * B Y^T N^-1 (d - Y B a) - a / C_l, or the component form with
 * SHTG_GRAD_COMPONENTS in flags), grad_logcl [nbins] (host; d L / d log C_l
 * for bins [bin_lo[k], bin_hi[k]]).  grad_alm or grad_logcl may be NULL. */
int shtg_logpost_grad(shtg_plan *plan, const double *cl, const double *bl, const float *alm,
                      const float *d, const float *ninv, int nbins, const int *bin_lo,
                      const int *bin_hi, int flags, double *logp, float *grad_alm,
                      double *grad_logcl, void *stream);

/* The same with the binned log C_l parameters of the joint posterior: C_l is
 * replaced by C_l exp(theta[k]) on the multipoles [bin_lo[k], bin_hi[k]]
 * (theta HOST [nbins], or NULL for theta = 0) before the evaluation, and
 * grad_theta[k] = d L / d theta_k.  Other arguments as shtg_logpost_grad. */
int shtg_logpost_grad_binned(shtg_plan *plan, const double *cl, const double *bl, const float *alm,
                             const float *d, const float *ninv, int nbins, const int *bin_lo,
                             const int *bin_hi, const double *theta, int flags, double *logp,
                             float *grad_alm, double *grad_theta, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* SHTG_H */

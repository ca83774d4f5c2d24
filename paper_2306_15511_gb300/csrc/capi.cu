// The exported C ABI (declared in include/shtg.h): argument checks, error
// reporting, and the composition of the Legendre and ring stages into the
// transforms Y, Y^T and the quadrature analysis.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "common.cuh"

namespace shtg {

static thread_local std::string g_err;

void set_error(const std::string &msg) { g_err = msg; }

int cuda_fail(cudaError_t e, const char *what, const char *file, int line) {
    set_error(std::string(what) + ": " + cudaGetErrorString(e) + " (" + file + ":" +
              std::to_string(line) + ")");
    return SHTG_ERR_CUDA;
}

template <typename T>
__global__ void k_sub(const T *__restrict__ a, const T *__restrict__ b, T *__restrict__ out, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = a[i] - b[i];
}
template <typename T>
__global__ void k_add(T *__restrict__ a, const T *__restrict__ b, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        a[i] += b[i];
}

static unsigned blocks_for(int64_t n) {
    int64_t g = (n + 255) / 256;
    return (unsigned)(g > 4096 ? 4096 : (g < 1 ? 1 : g));
}

// spin 0: alm rows [nbatch][nalm] -> maps [nbatch][npix]
// spin 2: alm rows [nbatch][2][nalm] -> maps [nbatch][2][npix]
template <typename T>
int transform_synth(Plan *p, int spin, const void *alm, void *map, int nbatch, cudaStream_t st) {
    typedef typename VT<T>::C C;
    C *F = sizeof(T) == 8 ? (C *)p->d_phase64 : (C *)p->d_phase32;
    const int rs = spin == 2 ? 2 : 1;
    SHTG_TRY(leg_synth<T>(p, spin, (const C *)alm, rs, nbatch, nullptr, F, st));
    SHTG_TRY(ring_synth<T>(p, F, nbatch * rs, (T *)map, st));
    return SHTG_OK;
}

template <typename T>
int transform_adjoint(Plan *p, int spin, const void *map, void *alm, int nbatch, int weighted,
                      cudaStream_t st, int vjp) {
    typedef typename VT<T>::C C;
    C *G = sizeof(T) == 8 ? (C *)p->d_phase64 : (C *)p->d_phase32;
    const int rs = spin == 2 ? 2 : 1;
    SHTG_TRY(ring_analysis<T>(p, (const T *)map, nbatch * rs, weighted, G, st));
    SHTG_TRY(leg_analysis<T>(p, spin, G, nbatch, nullptr, (C *)alm, rs, st, vjp));
    return SHTG_OK;
}
// Y and Y^T on FP64 buffers with the Legendre sums in double-FP32 arithmetic
static int transform_synth_df(Plan *p, int spin, const void *alm, void *map, int nbatch, cudaStream_t st) {
    const int rs = spin == 2 ? 2 : 1;
    SHTG_TRY(leg_synth_df(p, spin, (const double2 *)alm, rs, nbatch, nullptr, p->d_phase64, st));
    SHTG_TRY(ring_synth<double>(p, p->d_phase64, nbatch * rs, (double *)map, st));
    return SHTG_OK;
}
static int transform_adjoint_df(Plan *p, int spin, const void *map, void *alm, int nbatch, cudaStream_t st,
                                int vjp) {
    const int rs = spin == 2 ? 2 : 1;
    SHTG_TRY(ring_analysis<double>(p, (const double *)map, nbatch * rs, 0, p->d_phase64, st));
    SHTG_TRY(leg_analysis_df(p, spin, p->d_phase64, nbatch, nullptr, (double2 *)alm, rs, st, vjp));
    return SHTG_OK;
}

template int transform_synth<float>(Plan *, int, const void *, void *, int, cudaStream_t);
template int transform_synth<double>(Plan *, int, const void *, void *, int, cudaStream_t);
template int transform_adjoint<float>(Plan *, int, const void *, void *, int, int, cudaStream_t, int);
template int transform_adjoint<double>(Plan *, int, const void *, void *, int, int, cudaStream_t, int);

static int check_transform(const shtg_plan *plan, int spin, int precision, const void *a,
                           const void *b, int nbatch) {
    const Plan *p = reinterpret_cast<const Plan *>(plan);
    if (!p) {
        set_error("null plan");
        return SHTG_ERR_ARG;
    }
    if (spin != 0 && spin != 2) {
        set_error("spin must be 0 or 2");
        return SHTG_ERR_ARG;
    }
    if (spin == 2 && !(p->flags & SHTG_SPIN2)) {
        set_error("spin-2 transform on a plan created without SHTG_SPIN2");
        return SHTG_ERR_ARG;
    }
    if (precision != SHTG_FP64 && precision != SHTG_FP32 && precision != SHTG_TC32 && precision != SHTG_DF64) {
        set_error("precision must be SHTG_FP64, SHTG_FP32, SHTG_TC32 or SHTG_DF64");
        return SHTG_ERR_ARG;
    }
    if (!a || !b) {
        set_error("null buffer");
        return SHTG_ERR_ARG;
    }
    if (nbatch < 1 || nbatch > p->max_batch) {
        set_error("nbatch must be in [1, max_batch]");
        return SHTG_ERR_ARG;
    }
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != p->device) {
        cudaGetLastError();
        set_error("the current CUDA device is not the plan's device");
        return SHTG_ERR_ARG;
    }
    return SHTG_OK;
}

// Y^T with the Legendre stage on the tensor cores (FP32 buffers)
static int transform_adjoint_tc(Plan *p, int spin, const void *map, void *alm, int nbatch, cudaStream_t st,
                                int vjp) {
    const int rs = spin == 2 ? 2 : 1;
    SHTG_TRY(ring_analysis<float>(p, (const float *)map, nbatch * rs, 0, p->d_phase32, st));
    SHTG_TRY(leg_analysis_tc(p, spin, p->d_phase32, nbatch, nullptr, (float2 *)alm, rs, st, vjp));
    return check_device_flag(p, st);
}

int alm2map_vjp(Plan *p, int spin, int precision, const void *g, void *out, int nbatch,
                cudaStream_t st) {
    if (precision == SHTG_FP64) return transform_adjoint<double>(p, spin, g, out, nbatch, 0, st, 1);
    if (precision == SHTG_DF64) return transform_adjoint_df(p, spin, g, out, nbatch, st, 1);
    if (precision == SHTG_TC32) return transform_adjoint_tc(p, spin, g, out, nbatch, st, 1);
    return transform_adjoint<float>(p, spin, g, out, nbatch, 0, st, 1);
}

template <typename T>
int map2alm_t(Plan *p, int spin, const void *map, void *alm, int nbatch, int niter,
                     cudaStream_t st) {
    typedef typename VT<T>::C C;
    SHTG_TRY(transform_adjoint<T>(p, spin, map, alm, nbatch, 1, st));
    if (niter <= 0) return SHTG_OK;
    const int rows = spin == 2 ? 2 : 1;
    const int64_t nm = (int64_t)nbatch * rows * p->npix;
    const int64_t na = (int64_t)nbatch * rows * p->nalm;
    T *scratch = sizeof(T) == 8 ? (T *)p->d_map64 : (T *)p->d_map32;
    C *dalm = sizeof(T) == 8 ? (C *)p->v64[6] : (C *)p->v32[4];
    for (int it = 0; it < niter; ++it) {
        SHTG_TRY(transform_synth<T>(p, spin, alm, scratch, nbatch, st));
        k_sub<T><<<blocks_for(nm), 256, 0, st>>>((const T *)map, scratch, scratch, nm);
        SHTG_CHECK_LAUNCH("k_sub");
        SHTG_TRY(transform_adjoint<T>(p, spin, scratch, dalm, nbatch, 1, st));
        k_add<T><<<blocks_for(2 * na), 256, 0, st>>>((T *)alm, (const T *)dalm, 2 * na);
        SHTG_CHECK_LAUNCH("k_add");
    }
    return SHTG_OK;
}

}  // namespace shtg

using namespace shtg;

extern "C" {

int shtg_version(void) { return 3; }

const char *shtg_last_error_string(void) { return g_err.c_str(); }

int shtg_plan_create(int geom, int nside_or_nring, int nphi_gauss, int lmax, int max_batch,
                     int flags, shtg_plan **out) {
    if (!out) {
        set_error("out is null");
        return SHTG_ERR_ARG;
    }
    *out = nullptr;
    if (geom != SHTG_GEOM_HEALPIX && geom != SHTG_GEOM_GAUSS) {
        set_error("unknown geometry");
        return SHTG_ERR_ARG;
    }
    if (lmax < 0 || lmax > 8192 || max_batch < 1 || max_batch > 4096 || nside_or_nring < 1) {
        set_error("need 0 <= lmax <= 8192, 1 <= max_batch <= 4096 and a positive resolution");
        return SHTG_ERR_ARG;
    }
    if (geom == SHTG_GEOM_HEALPIX && (nside_or_nring > 8192 || lmax > 4 * nside_or_nring)) {
        set_error("HEALPix plans need nside <= 8192 and lmax <= 4 nside");
        return SHTG_ERR_ARG;
    }
    if (geom == SHTG_GEOM_GAUSS && (nphi_gauss < 1 || nphi_gauss > 65536 || nside_or_nring > 65536)) {
        set_error("Gauss-Legendre plans need 1 <= nphi_gauss <= 65536");
        return SHTG_ERR_ARG;
    }
    if (!(flags & (SHTG_SPIN0 | SHTG_SPIN2))) flags |= SHTG_SPIN0;
    Plan *p = new (std::nothrow) Plan();
    if (!p) {
        set_error("host allocation failed");
        return SHTG_ERR_NOMEM;
    }
    p->geom = geom;
    p->lmax = lmax;
    p->max_batch = max_batch;
    p->flags = flags;
    if (geom == SHTG_GEOM_HEALPIX) {
        p->nside = nside_or_nring;
    } else {
        p->nring = nside_or_nring;
        p->nphi_gauss = nphi_gauss;
    }
    if (cudaGetDevice(&p->device) != cudaSuccess) {
        cudaGetLastError();
        delete p;
        set_error("no CUDA device");
        return SHTG_ERR_CUDA;
    }
    const int rc = plan_build(p);
    if (rc != SHTG_OK) {
        plan_free(p);
        delete p;
        return rc;
    }
    *out = reinterpret_cast<shtg_plan *>(p);
    return SHTG_OK;
}

int shtg_plan_destroy(shtg_plan *plan) {
    if (!plan) return SHTG_OK;
    Plan *p = reinterpret_cast<Plan *>(plan);
    cudaDeviceSynchronize();
    plan_free(p);
    delete p;
    return SHTG_OK;
}

int shtg_plan_get_info(const shtg_plan *plan, shtg_plan_info *info) {
    if (!plan || !info) {
        set_error("null argument");
        return SHTG_ERR_ARG;
    }
    const Plan *p = reinterpret_cast<const Plan *>(plan);
    info->geom = p->geom;
    info->nside = p->nside;
    info->nring = p->nring;
    info->lmax = p->lmax;
    info->max_batch = p->max_batch;
    info->flags = p->flags;
    info->npix = p->npix;
    info->nalm = p->nalm;
    info->device_bytes = p->device_bytes;
    return SHTG_OK;
}

int shtg_alm2map(shtg_plan *plan, int spin, int precision, const void *alm, void *map,
                 int nbatch, void *stream) {
    SHTG_TRY(check_transform(plan, spin, precision, alm, map, nbatch));
    Plan *p = reinterpret_cast<Plan *>(plan);
    cudaStream_t st = (cudaStream_t)stream;
    if (precision == SHTG_FP64) return transform_synth<double>(p, spin, alm, map, nbatch, st);
    if (precision == SHTG_DF64) return transform_synth_df(p, spin, alm, map, nbatch, st);
    if (precision == SHTG_TC32) {
        float2 *F = p->d_phase32;
        const int rs = spin == 2 ? 2 : 1;
        SHTG_TRY(leg_synth_tc(p, spin, (const float2 *)alm, rs, nbatch, nullptr, F, st));
        SHTG_TRY(ring_synth<float>(p, F, nbatch * rs, (float *)map, st));
        return check_device_flag(p, st);
    }
    return transform_synth<float>(p, spin, alm, map, nbatch, st);
}

int shtg_alm2map_adjoint(shtg_plan *plan, int spin, int precision, const void *map, void *alm,
                         int nbatch, void *stream) {
    SHTG_TRY(check_transform(plan, spin, precision, map, alm, nbatch));
    Plan *p = reinterpret_cast<Plan *>(plan);
    cudaStream_t st = (cudaStream_t)stream;
    if (precision == SHTG_FP64) return transform_adjoint<double>(p, spin, map, alm, nbatch, 0, st);
    if (precision == SHTG_DF64) return transform_adjoint_df(p, spin, map, alm, nbatch, st, 0);
    if (precision == SHTG_TC32) return transform_adjoint_tc(p, spin, map, alm, nbatch, st, 0);
    return transform_adjoint<float>(p, spin, map, alm, nbatch, 0, st);
}

int shtg_alm2map_vjp(shtg_plan *plan, int spin, int precision, const void *map_grad,
                     void *alm_grad, int nbatch, void *stream) {
    SHTG_TRY(check_transform(plan, spin, precision, map_grad, alm_grad, nbatch));
    return alm2map_vjp(reinterpret_cast<Plan *>(plan), spin, precision, map_grad, alm_grad, nbatch,
                       (cudaStream_t)stream);
}

int shtg_map2alm(shtg_plan *plan, int spin, int precision, const void *map, void *alm,
                 int nbatch, int niter, void *stream) {
    SHTG_TRY(check_transform(plan, spin, precision, map, alm, nbatch));
    Plan *p = reinterpret_cast<Plan *>(plan);
    if (niter < 0 || niter > 100) {
        set_error("niter must be in [0, 100]");
        return SHTG_ERR_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    if (precision == SHTG_FP64 || precision == SHTG_DF64) return map2alm_t<double>(p, spin, map, alm, nbatch, niter, st);
    return map2alm_t<float>(p, spin, map, alm, nbatch, niter, st);
}

int shtg_cg_sample(shtg_plan *plan, const shtg_problem *prob, double *alm_out,
                   const shtg_cg_opts *opts, shtg_cg_stats *stats, void *stream) {
    if (!plan) {
        set_error("null plan");
        return SHTG_ERR_ARG;
    }
    return cg_sample(reinterpret_cast<Plan *>(plan), prob, alm_out, opts, stats,
                     (cudaStream_t)stream);
}

int shtg_cg_sample_chains(int ngroups, shtg_plan *const *plans, const shtg_problem *probs,
                          double *const *alm_out, const shtg_cg_opts *opts, shtg_cg_stats *stats,
                          void *stream) {
    if (ngroups < 1 || !plans || !probs || !alm_out) {
        set_error("chains: need ngroups >= 1, plans, problems and outputs");
        return SHTG_ERR_ARG;
    }
    for (int g = 0; g < ngroups; ++g) {
        if (!plans[g]) {
            set_error("chains: null plan");
            return SHTG_ERR_ARG;
        }
        for (int h = 0; h < g; ++h)
            if (plans[h] == plans[g]) {
                set_error("chains: every group needs its own plan (a plan's workspace serves one solve)");
                return SHTG_ERR_ARG;
            }
    }
    cudaStream_t st = (cudaStream_t)stream;
    if (opts && (opts->flags & SHTG_GROUPED)) {
        std::vector<Plan *> ps(ngroups);
        for (int g = 0; g < ngroups; ++g) ps[g] = reinterpret_cast<Plan *>(plans[g]);
        return cg_sample_grouped(ngroups, ps.data(), probs, alm_out, opts, stats, st);
    }
    if (ngroups == 1)
        return cg_sample(reinterpret_cast<Plan *>(plans[0]), &probs[0], alm_out[0], opts,
                         stats ? &stats[0] : nullptr, st);
    // fork: every group's work stream waits for the caller's stream
    cudaEvent_t fork;
    SHTG_CUDA(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
    SHTG_CUDA(cudaEventRecord(fork, st));
    for (int g = 0; g < ngroups; ++g)
        SHTG_CUDA(cudaStreamWaitEvent(reinterpret_cast<Plan *>(plans[g])->work_stream, fork, 0));
    // one host thread per group: a solve waits on the host at its convergence checks
    std::vector<int> rc(ngroups, SHTG_OK);
    std::vector<std::string> msg(ngroups);
    std::vector<std::thread> th;
    for (int g = 0; g < ngroups; ++g) {
        th.emplace_back([&, g]() {
            Plan *p = reinterpret_cast<Plan *>(plans[g]);
            if (cudaSetDevice(p->device) != cudaSuccess) {
                rc[g] = SHTG_ERR_CUDA;
                msg[g] = "cudaSetDevice failed";
                return;
            }
            rc[g] = cg_sample(p, &probs[g], alm_out[g], opts, stats ? &stats[g] : nullptr, p->work_stream);
            if (rc[g] != SHTG_OK) msg[g] = shtg_last_error_string();
        });
    }
    for (auto &t : th) t.join();
    // join: the caller's stream waits for every group
    for (int g = 0; g < ngroups; ++g) {
        SHTG_CUDA(cudaEventRecord(fork, reinterpret_cast<Plan *>(plans[g])->work_stream));
        SHTG_CUDA(cudaStreamWaitEvent(st, fork, 0));
    }
    cudaEventDestroy(fork);
    int worst = SHTG_OK;
    for (int g = 0; g < ngroups; ++g)
        if (rc[g] != SHTG_OK && (worst == SHTG_OK || worst == SHTG_ERR_NOT_CONVERGED)) {
            worst = rc[g];
            set_error("chain group " + std::to_string(g) + ": " + msg[g]);
        }
    return worst;
}

int shtg_apply_operator(shtg_plan *plan, const shtg_problem *prob, const double *x, double *y,
                        void *stream) {
    if (!plan || !x || !y) {
        set_error("null argument");
        return SHTG_ERR_ARG;
    }
    return apply_operator(reinterpret_cast<Plan *>(plan), prob, x, y, (cudaStream_t)stream);
}

int shtg_precond_apply(shtg_plan *plan, const shtg_problem *prob, const shtg_cg_opts *opts, const double *r,
                       double *z, void *stream) {
    if (!plan || !prob || !opts || !r || !z) {
        set_error("null argument");
        return SHTG_ERR_ARG;
    }
    return precond_apply(reinterpret_cast<Plan *>(plan), prob, opts, r, z, (cudaStream_t)stream);
}

int shtg_lowl_block(shtg_plan *plan, const shtg_problem *prob, int lowl_lmax, double *H, int *params, int *n,
                    void *stream) {
    if (!plan || !prob || !H || !n) {
        set_error("null argument");
        return SHTG_ERR_ARG;
    }
    return lowl_block(reinterpret_cast<Plan *>(plan), prob, lowl_lmax, H, params, n, (cudaStream_t)stream);
}

int shtg_logpost_grad(shtg_plan *plan, const double *cl, const double *bl, const float *alm,
                      const float *d, const float *ninv, int nbins, const int *bin_lo,
                      const int *bin_hi, int flags, double *logp, float *grad_alm,
                      double *grad_logcl, void *stream) {
    if (!plan || !cl || !bl || !alm || !d || !ninv || nbins < 0 ||
        (nbins > 0 && grad_logcl && (!bin_lo || !bin_hi))) {
        set_error("invalid argument");
        return SHTG_ERR_ARG;
    }
    return logpost_grad(reinterpret_cast<Plan *>(plan), cl, bl, alm, d, ninv, nbins, bin_lo,
                        bin_hi, flags, logp, grad_alm, grad_logcl, (cudaStream_t)stream);
}

int shtg_logpost_grad_binned(shtg_plan *plan, const double *cl, const double *bl, const float *alm,
                             const float *d, const float *ninv, int nbins, const int *bin_lo,
                             const int *bin_hi, const double *theta, int flags, double *logp,
                             float *grad_alm, double *grad_theta, void *stream) {
    if (!plan || !cl || !bl || !alm || !d || !ninv || nbins < 0 || (nbins > 0 && (!bin_lo || !bin_hi))) {
        set_error("logpost_grad_binned: null argument or negative nbins");
        return SHTG_ERR_ARG;
    }
    Plan *p = reinterpret_cast<Plan *>(plan);
    // C_l exp(theta_k) on the multipoles of bin k (Eq. joint-posterior with
    // binned log C_l parameters)
    std::vector<double> c(cl, cl + p->lmax + 1);
    if (theta)
        for (int k = 0; k < nbins; ++k) {
            const double f = std::exp(theta[k]);
            for (int l = std::max(0, bin_lo[k]); l <= std::min(p->lmax, bin_hi[k]); ++l) c[l] *= f;
        }
    return logpost_grad(p, c.data(), bl, alm, d, ninv, nbins, bin_lo, bin_hi, flags, logp, grad_alm,
                        grad_theta, (cudaStream_t)stream);
}

int shtg_fluctuation_rescale(shtg_plan *plan, int ncomp, const double *cl_old, const double *cl_new,
                             const double *f, double *f_out, int nbatch, void *stream) {
    if (!plan) {
        set_error("null plan");
        return SHTG_ERR_ARG;
    }
    Plan *p = reinterpret_cast<Plan *>(plan);
    if (nbatch > p->max_batch) {
        set_error("fluctuation_rescale: nbatch above max_batch");
        return SHTG_ERR_ARG;
    }
    return fluctuation_rescale(p, ncomp, cl_old, cl_new, f, f_out, nbatch, (cudaStream_t)stream);
}

int shtg_joint_log_target(shtg_plan *plan, const shtg_problem *prob, int precision, const double *a_hat,
                          const double *f_hat, double *log_pi, void *stream) {
    if (!plan) {
        set_error("null plan");
        return SHTG_ERR_ARG;
    }
    return joint_log_target(reinterpret_cast<Plan *>(plan), prob, precision, a_hat, f_hat, log_pi,
                            (cudaStream_t)stream);
}

int shtg_joint_acceptance(double log_pi_new, double log_pi_old, double log_prior_new, double log_prior_old,
                          double *accept) {
    if (!accept) {
        set_error("joint_acceptance: null output");
        return SHTG_ERR_ARG;
    }
    const double x = (log_pi_new + log_prior_new) - (log_pi_old + log_prior_old);
    if (std::isnan(x)) {
        set_error("joint_acceptance: NaN log ratio");
        return SHTG_ERR_NONFINITE;
    }
    *accept = x >= 0.0 ? 1.0 : std::exp(x);
    return SHTG_OK;
}

}  // extern "C"

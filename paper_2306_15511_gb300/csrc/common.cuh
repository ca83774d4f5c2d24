// Internal declarations shared by the shtg CUDA translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <string>
#include <vector>

#include "../../include/shtg.h"

namespace shtg {

// ----------------------------------------------------------------- errors
void set_error(const std::string &msg);
int cuda_fail(cudaError_t e, const char *what, const char *file, int line);

#define SHTG_CUDA(call)                                                           \
    do {                                                                          \
        cudaError_t e_ = (call);                                                  \
        if (e_ != cudaSuccess) return ::shtg::cuda_fail(e_, #call, __FILE__, __LINE__); \
    } while (0)

#define SHTG_CHECK_LAUNCH(name)                                                   \
    do {                                                                          \
        cudaError_t e_ = cudaGetLastError();                                      \
        if (e_ != cudaSuccess) return ::shtg::cuda_fail(e_, name, __FILE__, __LINE__); \
    } while (0)

#define SHTG_TRY(call)                                                            \
    do {                                                                          \
        int rc_ = (call);                                                         \
        if (rc_ != SHTG_OK) return rc_;                                           \
    } while (0)

// ----------------------------------------------------------- real types
// Allow a kernel the device's whole opt-in shared memory per block.  Every
// call sets the same value, so host threads that launch the kernel for
// plans of different sizes at once (chains) cannot lower the limit another
// thread's launch needs; occupancy follows the launch's own request.
template <typename K> inline cudaError_t allow_max_smem(K kern) {
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa;
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, kern);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
    return e;
}

template <typename T> struct VT;
template <> struct VT<float> { typedef float2 C; };
template <> struct VT<double> { typedef double2 C; };

__host__ __device__ __forceinline__ float2 cplx(float r, float i) { return make_float2(r, i); }
__host__ __device__ __forceinline__ double2 cplx(double r, double i) { return make_double2(r, i); }

// ------------------------------------------------------------------ plan
// Number of ring-FFT table entries per ring (see ringfft.cu).
struct RingFFT {
    int n;        // pixels on the ring
    int logM;     // log2 of the power-of-two transform length
    int blue;     // 1: Bluestein convolution of length M; 0: direct length n = M
    int shift;    // phi0 = shift * pi / n (0 or 1)
    int64_t chirp_off;  // offset of the n chirp values (Bluestein rings)
    int64_t bhat_off;   // offset of the M spectra of the convolution kernel
    int64_t ph_off;     // shifted rings: offset of e^{i pi k / n}, k = 0 .. min(lmax, n - 1)
};

// Ring FFT launches (ringfft.cu): threads per CTA for a launch whose
// longest buffer is 2^logm, and the butterflies per thread of the first
// radix-R pass (R = 2, 4, 8; log2 M not a multiple of four) that the kernel
// of that thread count is compiled for.  Launch buckets hold rings with
// M = 2^logm (and M = 2^(logm - 1) for aliased direct rings); the bucket of
// lengths <= 1024 runs 64 threads.
__host__ __device__ constexpr int ring_threads(int logm) {
    return logm >= 13 ? 512 : logm == 12 ? 256 : logm == 11 ? 128 : 64;
}
__host__ __device__ constexpr int ring_first_bpt(int R, int nt) {
    return nt >= 512 ? (R == 2 ? 8 : 1) : nt == 256 ? 1 : nt == 128 ? (R == 2 ? 1 : 2) : (R == 8 ? 1 : 4);
}

// grouped launches (chains of several geometries): plans per launch
#define SHTG_MAX_GROUPS 16

#define SHTG_FFT_LOGMAX 13   // longest ring transform (Bluestein length included): 8192

// l stride of the FP64 recurrence tile states
#define SHTG_TS64 32

// Kernel classes timed live with CUDA events (on the launching stream) when
// profiling is on; see shtg_cg_stats.kernel_ms.
enum KClass { K_LEG_SYN32 = 0, K_LEG_ANA32, K_RING32, K_LEG_SYN64, K_LEG_ANA64, K_RING64, K_VEC, K_DIAG };
#define SHTG_NCLASS 8

struct Prof {
    bool on = false;
    std::vector<cudaEvent_t> ev;   // pool created with the plan
    std::vector<int> cls;
    int n = 0;                     // recorded (begin, end) pairs
    int open_cls = -1;
    long long launches = 0;        // kernels launched by the library (always counted)
};

// two-level preconditioner (lowl.cu): workspace, the kept Gram matrix of the
// low multipoles and the inverse of the current low block
#define SHTG_LOWL_LCMAX 48
#define SHTG_LOWL_LC_DEFAULT 32
struct LowL {
    double2 *W = nullptr;          // [ch][ring][2 l_c + 1] Fourier coefficients of N^-1 per ring
    double *lam = nullptr;         // [lo(l, m)][pair] lambda_lm on the north ring
    double *lw = nullptr, *lx = nullptr;   // spin-2 profiles, same layout
    double *G = nullptr;           // [nfull][nfull] sum_p N^-1 phi_i phi_j (no beam, no prior)
    double *H = nullptr, *S = nullptr;     // ping-pong buffers of the sweep
    double *h64 = nullptr;         // H^-1 (one of H, S)
    float *h32 = nullptr;          // H^-1 in FP32
    int4 *par = nullptr;           // [nfull] (l, m, comp, part)
    int *sel = nullptr, *emap = nullptr;   // [n] active parameter -> full index / vector element
    float *wv = nullptr;           // [n] metric weight (1 for m = 0, else 2)
    double *part = nullptr;        // [max_batch][32] <r, z> corrections
    int *flag = nullptr, *shift = nullptr;
    double *ninv = nullptr;        // N^-1 the kept Gram matrix was built from
    int64_t bytes = 0;
    int cap_lc = -1, cap_nc = 0;   // workspace size
    int n = 0, lc = 0, nc = 0;     // current active block
    int gram_lc = -1, gram_nc = 0;
    bool gram_ok = false;
    std::vector<int4> params;      // host copy of the active parameters
    // the per-l table rows (beam, S^-1) and C_l scale H^-1 was built from
    std::vector<double> inv_ltab;
    double inv_isc = 0.0;
    bool inv_ok = false;
};

// azimuthal block preconditioner (azblk.cu): per-m blocks of T (and E) for
// l <= lb from the ring sums of N^-1, their Cholesky factors
#define SHTG_AZ_LB_DEFAULT 1024
struct AzBlk {
    int lb = -1, ncb = 0;          // block l max; components per block (T, or T and E)
    int64_t gsize = 0, hsize = 0, pcap = 0;
    double *G = nullptr;           // packed lower Gram matrices per m (T, then E), no beam, no prior
    double *H = nullptr;           // packed lower blocks per m; Cholesky factor R, then R^-1, in place
    double *M64 = nullptr;         // full-square block inverses per m (FP64)
    float *M32 = nullptr;          // their FP32 copy (the FP32 iteration)
    int64_t *goff = nullptr, *hoff = nullptr, *moff = nullptr, *poff = nullptr, *xoff = nullptr;
    double *Xg = nullptr;          // [m][q][row] right-hand sides of the blocks (FP32 or FP64 values)
    int ntile = 0;                 // 128-row tiles of the largest block
    double *w = nullptr;           // [ch][sum, diff][pair] ring sums of N^-1 over the pair's rings
    double *pl = nullptr, *pw = nullptr, *px = nullptr;   // profiles of a chunk of m
    double *slot = nullptr;        // [max_batch][lb + 1] <r, z> corrections
    int *flag = nullptr;
    double *ninv = nullptr;        // N^-1 the Gram matrices were built from
    int64_t bytes = 0;
    bool gram_ok = false, inv_ok = false;
    std::vector<double> inv_ltab;
    double inv_isc = 0.0;
};

struct Plan {
    int device = 0;
    Prof prof;
    std::map<long long, int> tuned;   // autotuned kernel variant per (precision, family, nmaps)
    int geom = 0, nside = 0, nring = 0, npairs = 0, lmax = 0, max_batch = 0, flags = 0;
    int nphi_gauss = 0;
    int64_t npix = 0, nalm = 0;
    int nmaps_max = 0;          // maps the workspace holds (max_batch * (spin2 ? 3 : 1))
    int64_t device_bytes = 0;

    // host geometry (rings north to south)
    std::vector<double> cth, sth, wring;
    std::vector<int> nphi, shift;
    std::vector<int64_t> ofs;

    // device geometry
    int *d_nphi = nullptr;
    int64_t *d_ofs = nullptr;
    double *d_wring = nullptr;    // quadrature weight of one pixel per ring
    double *d_u64 = nullptr;      // 1 - cos(theta) of the north ring of each pair
    float *d_u32 = nullptr;
    double *d_x64 = nullptr;      // cos(theta) of the north ring of each pair
    double *d_is2_64 = nullptr;   // 1 / sin^2(theta) per pair
    float *d_x32 = nullptr, *d_is2_32 = nullptr;
    int *d_lofidx = nullptr;      // l of each alm index
    int *d_mofidx = nullptr;      // m of each alm index

    // Legendre tables
    double2 *d_rec64 = nullptr;   // (a_lm, b_lm): lambda_l = a (1-u) lambda_{l-1} + b lambda_{l-2}
    float2 *d_rec32 = nullptr;
    int *d_ls64 = nullptr, *d_ls32 = nullptr;     // [m][pair] first significant l
    double2 *d_st64 = nullptr;    // [m][pair] (lambda_{ls-1}, lambda_ls)
    float2 *d_st32 = nullptr;
    double4_32a *d_s2c64 = nullptr;   // spin-2 recurrence (alpha, alpha+beta, alpha-beta, gamma)
    float4 *d_s2c32 = nullptr;
    int2 *d_ls2_64 = nullptr, *d_ls2_32 = nullptr;  // [m][pair] start l of (y+, y-)
    double4_32a *d_st2_64 = nullptr;  // [m][pair] (y+_{l-1}, y+_l, y-_{l-1}, y-_l) / 2
    float4 *d_st2_32 = nullptr;

    // ring FFT tables
    int fft_logmax = 0;
    RingFFT *d_rfft = nullptr;
    std::vector<RingFFT> h_rfft;
    // two-level twiddle table for e^{-2 pi i t / Mmax}, t = th 2^tw_blo + tl:
    // [lo: e^{-2 pi i tl / Mmax}, 2^tw_blo entries | hi: e^{-2 pi i th 2^tw_blo / Mmax}]
    double2 *d_tw64 = nullptr;
    float2 *d_tw32 = nullptr;
    int tw_blo = 0, tw_nlo = 0, tw_nhi = 0;
    double2 *d_chirp64 = nullptr, *d_bfwd64 = nullptr, *d_binv64 = nullptr;
    float2 *d_chirp32 = nullptr, *d_bfwd32 = nullptr, *d_binv32 = nullptr;
    // fixed-length launches (ringfft.cu): per-pass twiddles of the radix-16
    // passes for M = 2^logm, at twf_off[logm] (logm = 10 .. 13)
    double2 *d_twf64 = nullptr;
    float2 *d_twf32 = nullptr;
    int64_t twf_off[SHTG_FFT_LOGMAX + 1] = {};
    double2 *d_rph64 = nullptr;   // ring phase tables (RingFFT::ph_off)
    float2 *d_rph32 = nullptr;
    size_t fft_smem64 = 0, fft_smem32 = 0;
    int *d_ring_groups = nullptr;    // ring pairs, ordered by launch bucket
    struct RingLaunch {
        int off, count;   // slice of d_ring_groups
        int logm;         // log2 of the bucket's buffer length (every member's M, and 2n if aliased)
        int alias;        // bucket holds rings with n < 2 lmax
        int chirp;        // longest Bluestein ring of the bucket (its chirp is staged in shared memory)
        int fix;          // launches of 128 threads and more: log2 of every member's M (fixed-length passes); 0 = any
    };
    std::vector<RingLaunch> ring_launch;

    // workspace
    double2 *d_phase64 = nullptr;  // [nmaps_max][nring][lmax+1] Fourier coefficients per ring
    float2 *d_phase32 = nullptr;
    double *d_map64 = nullptr;     // [nmaps_max][npix] scratch maps
    float *d_map32 = nullptr;
    double *d_ninv64 = nullptr;    // [2][npix] problem weights (T, P)
    float *d_ninv32 = nullptr;

    // solver workspace (vectors hold max_batch realizations of all components)
    double2 *v64[7] = {};          // b, x, r, z, p, q, t
    float2 *v32[5] = {};           // r, z, p, q, x
    double *d_minv64 = nullptr;    // [max_batch][4][nalm] inverse preconditioner blocks per realization
    float *d_minv32 = nullptr;
    double *d_isc64 = nullptr;          // [max_batch] 1 / (C_l scale), 1 / sqrt(C_l scale)
    double *d_rsc64 = nullptr;
    float *d_isc32 = nullptr;
    float *d_diagT = nullptr, *d_diagP = nullptr;   // [nalm] ring-averaged diag of Y^T N^-1 Y
    float *d_wpairT = nullptr, *d_wpairP = nullptr; // [npairs] N^-1 summed over the ring pair
    double *d_ltab64 = nullptr;    // [9][lmax+1] beam, S^-1 (TT,TE,EE,BB), S^-1/2 (TT,TE,EE,BB)
    float *d_ltab32 = nullptr;     // [5][lmax+1] beam, S^-1 (TT,TE,EE,BB)
    double *d_scal = nullptr;      // [max_batch][16] per-realization PCG scalars
    double *d_part = nullptr;      // reduction partial sums
    int *d_flag = nullptr;         // [0]: set by a kernel whose bounded device wait expired
    cudaStream_t cap_stream = nullptr;   // non-blocking stream on which solver iterations are captured
    cudaStream_t work_stream = nullptr;  // non-blocking stream of this plan's solve in a chains call
    // ring-stage launch buckets after the first run on side streams, forked
    // from and joined back into the caller's stream with events
    static constexpr int RING_SIDE = 4;
    cudaStream_t ring_side[RING_SIDE] = {};
    cudaEvent_t ring_fork = nullptr, ring_join[RING_SIDE] = {};
    // FP32 recurrence states every 32 l (tensor-core transpose): entry
    // (m, t, pair) at (d_toff[m] + t) * npairs + pair is the state before
    // l = m + 32 t: (lambda_{l-1}, lambda_{l-2}) for spin 0, (y+_{l-1},
    // y+_{l-2}, y-_{l-1}, y-_{l-2}) for spin 2
    int64_t *d_toff = nullptr;
    float2 *d_tst0 = nullptr;
    float4 *d_tst2 = nullptr;
    // the same in FP64 every SHTG_TS64 l (FP64 and double-FP32 transposes),
    // [m][t][pair] at (d_toff64[m] + t) * npairs + pair
    int64_t *d_toff64 = nullptr;
    double2 *d_tst64_0 = nullptr;
    double4_32a *d_tst64_2 = nullptr;
    double *d_lsum = nullptr;      // [lmax+1] per-l sums (log-posterior)
    double *d_jtab = nullptr;      // [13][lmax+1] joint move: old and new spectra [2][4], rescaling rows [5]
    // per-m dense block solve (plans created with SHTG_BLOCK_SOLVER): blocks
    // and recurrence values of one chunk of m, ring-pair weights, offsets, flag
    double *d_blk = nullptr, *d_blklam = nullptr, *d_blkw = nullptr;
    int64_t *d_blkoff = nullptr;
    int *d_blkflag = nullptr;
    int64_t blk_cap = 0, lam_cap = 0;
    LowL lowl;
    AzBlk az;
    double *d_stage = nullptr;     // [nmaps_max][npix] staging for host inputs
    double *h_pinned = nullptr;    // pinned host scalars
};

// solver.cu
#define SHTG_RED_BLOCKS 128
int cg_sample(Plan *p, const shtg_problem *pr, double *alm_out, const shtg_cg_opts *o,
              shtg_cg_stats *stats, cudaStream_t st);
int apply_operator(Plan *p, const shtg_problem *pr, const double *x, double *y, cudaStream_t st);
// chains of several geometries with one grouped launch per stage of the FP32 iteration
int cg_sample_grouped(int ng, Plan *const *ps, const shtg_problem *prs, double *const *outs,
                      const shtg_cg_opts *o, shtg_cg_stats *stats, cudaStream_t st);
int fluctuation_rescale(Plan *p, int nc, const double *cl_old, const double *cl_new, const double *f,
                        double *g, int nbatch, cudaStream_t st);
int joint_log_target(Plan *p, const shtg_problem *pr, int precision, const double *a_hat,
                     const double *f_hat, double *logpi, cudaStream_t st);
// block.cu: per-m dense block solve for azimuthally symmetric noise (App. A)
int block_workspace(Plan *p);
int block_solve(Plan *p, const double2 *B, double2 *X, int nb, double isc, cudaStream_t st);
// lowl.cu: two-level preconditioner.  lowl_setup builds H^-1 for l_c
// (<= 0: the default) and nc components with 1 / (C_l scale) = isc (copying
// H to h_host first when given); lowl_apply replaces z on the low block of nb
// systems (r, z viewed as reals, per complex entries per system) and adds
// the change of <r, z> to the rz partials.
int lowl_setup(Plan *p, int lc, int nc, double isc, cudaStream_t st, double *h_host = nullptr);
template <typename T>
int lowl_apply(Plan *p, const T *r, T *z, int nb, int64_t per, double *part, cudaStream_t st);
void lowl_free(Plan *p);
// azblk.cu: azimuthal block preconditioner for l <= lb (<= 0: the default)
int az_setup(Plan *p, int lb, int nc, double isc, cudaStream_t st);
template <typename T>
int az_apply(Plan *p, const T *r, T *z, int nb, int64_t per, double *part, cudaStream_t st, bool fp64_factor);
void az_free(Plan *p);
// az_apply (FP32 factors) over ng plans whose blocks are set up, one launch
// per kernel for every group; groups whose device flag *active[g] is 0 are
// skipped
int az_apply_grp(int ng, Plan *const *ps, const float *const *r, float *const *z, const int *nb,
                 const int64_t *per, double *const *part, const int *const *active, cudaStream_t st);
int precond_apply(Plan *p, const shtg_problem *pr, const shtg_cg_opts *o, const double *r, double *z,
                  cudaStream_t st);
int lowl_block(Plan *p, const shtg_problem *pr, int lc, double *H, int *params, int *n, cudaStream_t st);
int logpost_grad(Plan *p, const double *cl, const double *bl, const float *alm, const float *d,
                 const float *ninv, int nbins, const int *blo, const int *bhi, int flags,
                 double *logp, float *grad, double *gcl, cudaStream_t st);

// plan.cu
int plan_build(Plan *p);
void plan_free(Plan *p);

// profiling: bracket one launch (or a group) of a kernel class
inline void prof_begin(Plan *p, int cls, cudaStream_t st) {
    Prof &f = p->prof;
    if (f.on && 2 * f.n + 1 < (int)f.ev.size()) {
        cudaEventRecord(f.ev[2 * f.n], st);
        f.open_cls = cls;
    }
}
inline void prof_end(Plan *p, cudaStream_t st, int nlaunch = 1) {
    Prof &f = p->prof;
    f.launches += nlaunch;
    if (f.open_cls >= 0) {
        cudaEventRecord(f.ev[2 * f.n + 1], st);
        if ((int)f.cls.size() <= f.n) f.cls.resize(f.n + 1);
        f.cls[f.n] = f.open_cls;
        f.n += 1;
        f.open_cls = -1;
    }
}
// after a stream synchronize: accumulate elapsed times per class and reset
void prof_collect(Plan *p, double *ms, int *count);

// legendre.cu: F[row][m][ring] <-> alm.  Map k of a call reads / writes the
// alm row k * rs (spin 0) or rows k * rs (E) and k * rs + 1 (B) (spin 2), each
// row nalm complex values; F rows are k (spin 0) or 2k (Q), 2k + 1 (U).
// beam: device [lmax+1] multiplying the alm side, or null.
template <typename T>
int leg_synth(Plan *p, int spin, const typename VT<T>::C *alm, int rs, int nmaps,
              const T *beam, typename VT<T>::C *F, cudaStream_t st);
// vjp = 1 doubles the m > 0 outputs (gradient in real-component convention).
template <typename T>
int leg_analysis(Plan *p, int spin, const typename VT<T>::C *G, int nmaps, const T *beam,
                 typename VT<T>::C *alm, int rs, cudaStream_t st, int vjp = 0);
// The FP32 CUDA-core Legendre sums of ng plans in one launch (chains of
// several geometries): group g works on plans[g] with its own buffers and
// arguments as leg_synth / leg_analysis would; groups whose device flag
// *active[g] is 0 are skipped (active, or an entry, may be null: always on).
int leg_synth_grp(int ng, Plan *const *ps, int spin, const float2 *const *alm, const int *rs, const int *nmaps,
                  const float *const *beam, float2 *const *F, const int *const *active, cudaStream_t st);
int leg_analysis_grp(int ng, Plan *const *ps, int spin, const float2 *const *G, const int *nmaps,
                     const float *const *beam, float2 *const *alm, const int *rs, const int *const *active,
                     cudaStream_t st);
// out[l, m] = sum_r w_r g_lm(theta_r) (g = lambda^2 or lw^2 + lx^2)
int leg_diag(Plan *p, int spin, const float *wring, float *out, cudaStream_t st);
// FP32 recurrence with the l-sum on the tensor cores (bf16 hi / lo split)
int leg_synth_tc(Plan *p, int spin, const float2 *alm, int rs, int nmaps, const float *beam, float2 *F,
                 cudaStream_t st);
// SHTG_ERR_TIMEOUT if a kernel recorded an expired device wait (clears the flag)
int check_device_flag(Plan *p, cudaStream_t st);
// tensor-core transpose (Y^T) Legendre stage; the tile-state tables it reads
int leg_analysis_tc(Plan *p, int spin, const float2 *G, int nmaps, const float *beam, float2 *alm, int rs,
                    cudaStream_t st, int vjp);
int build_tile_states(Plan *p);
// FP64 Legendre transpose as a register-blocked contraction; its FP64 tile states
int leg_analysis_g64(Plan *p, int spin, const double2 *G, int nmaps, const double *beam, double2 *alm, int rs,
                     cudaStream_t st, int vjp);
int build_tile_states64(Plan *p);
// FP64-accurate Legendre sums in double-FP32 arithmetic on FP64 buffers
// (legendre_df.cu); the transpose reads the FP64 tile states above
int leg_synth_df(Plan *p, int spin, const double2 *alm, int rs, int nmaps, const double *beam, double2 *F,
                 cudaStream_t st);
int leg_analysis_df(Plan *p, int spin, const double2 *G, int nmaps, const double *beam, double2 *alm, int rs,
                    cudaStream_t st, int vjp);

// ringfft.cu
// mode 0: F -> map (synthesis); mode 1: map -> G (adjoint, wmode 1 = quadrature weights);
// mode 2: F -> N^-1 -> G (fused, in place allowed).
template <typename T>
int ring_synth(Plan *p, const typename VT<T>::C *F, int nmaps, T *map, cudaStream_t st);
template <typename T>
int ring_analysis(Plan *p, const T *map, int nmaps, int weighted, typename VT<T>::C *G,
                  cudaStream_t st);
template <typename T>
int ring_fused(Plan *p, typename VT<T>::C *FG, int nmaps, int nT, const T *ninv,
               cudaStream_t st);
// ring_fused over ng plans (FP32), one launch per transform-length class
// (at most five) covering every plan; groups whose device flag *active[g]
// is 0 are skipped
template <typename T>
int ring_fused_grp(int ng, Plan *const *ps, typename VT<T>::C *const *FG, const int *nmaps, const int *nT,
                   const T *const *ninv, const int *const *active, cudaStream_t st);

int alm2map_vjp(Plan *p, int spin, int precision, const void *g, void *out, int nbatch,
                cudaStream_t st);

// capi.cu transforms used by the solver
template <typename T>
int transform_synth(Plan *p, int spin, const void *alm, void *map, int nbatch, cudaStream_t st);
template <typename T>
int transform_adjoint(Plan *p, int spin, const void *map, void *alm, int nbatch, int weighted,
                      cudaStream_t st, int vjp = 0);

inline int64_t alm_index(int l, int m, int lmax) {
    return (int64_t)m * (2 * lmax + 1 - m) / 2 + l;
}

}  // namespace shtg

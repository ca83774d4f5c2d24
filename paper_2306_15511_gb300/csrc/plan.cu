// Plan construction: ring geometry, Legendre recurrence tables, FP64 start
// states of the recurrence, ring-FFT tables and workspace.
//
// Legendre functions (App. A): Y_lm = lambda_lm(theta) e^{i m phi} with
// lambda_mm = (-1)^m sqrt((2m+1)/(4 pi) prod_{k<=m} (2k-1)/(2k)) sin^m theta,
// and for l > m the three-term recurrence written in u = 1 - cos theta,
//     lambda_l = a_l (1 - u) lambda_{l-1} + b_l lambda_{l-2},
//     a_l = sqrt((4l^2-1)/(l^2-m^2)),  b_l = -a_l sqrt(((l-1)^2-m^2)/(4(l-1)^2-1)),
// (a_{m+1} = sqrt(2m+3), b_{m+1} = 0).  Carrying u instead of cos theta keeps
// the near-polar rings exact in FP32, where cos theta rounds to 1.
#include <cmath>
#include <complex>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <functional>
#include <map>

#include "common.cuh"

namespace shtg {

static const double PI = 3.14159265358979323846264338327950288;

// ------------------------------------------------------------ start states
// For every (m, ring pair) walk the FP64 recurrence from lambda_mm with
// exponent rescaling (value = v * 2^(512 k)) until |lambda_lm| first reaches
// the significance threshold; record that l and (lambda_{l-1}, lambda_l).
// Terms below the threshold are dropped by the transform kernels, which then
// start their recurrence there without any rescaling logic.
__global__ void k_start_states(int lmax, int npairs, const double *__restrict__ u64,
                               const double *__restrict__ sect, const double2 *__restrict__ rec,
                               double thr64, double thr32, int *ls64, double2 *st64, int *ls32,
                               float2 *st32)
{
    const int pr = blockIdx.x * blockDim.x + threadIdx.x;
    const int m = blockIdx.y;
    if (pr >= npairs) return;
    const double u = u64[pr];
    const double s = sqrt(u * (2.0 - u));
    const int64_t o = (int64_t)m * npairs + pr;
    int l64 = lmax + 1, l32 = lmax + 1;
    double2 s64 = make_double2(0.0, 0.0);
    float2 s32 = make_float2(0.f, 0.f);
    if (s > 0.0) {
        // sectoral value by products, kept in [2^-256, 2^256] * 2^(512 k)
        double v = 0.28209479177387814347403972578;  // 1/sqrt(4 pi)
        int k = 0;
        for (int j = 1; j <= m; ++j) {
            v *= -sect[j] * s;
            if (fabs(v) < 0x1p-256) {
                v *= 0x1p512;
                k -= 1;
            }
        }
        double prev = 0.0;
        const int64_t base = (int64_t)m * (2 * lmax + 1 - m) / 2;
        for (int l = m;; ++l) {
            if (k == 0) {
                const double a = fabs(v);
                if (l32 > lmax && a >= thr32) {
                    l32 = l;
                    s32 = make_float2((float)prev, (float)v);
                }
                if (l64 > lmax && a >= thr64) {
                    l64 = l;
                    s64 = make_double2(prev, v);
                }
                if (l32 <= lmax && l64 <= lmax) break;
            }
            if (l == lmax) break;
            const double2 c = rec[base + l + 1];
            const double t = c.x * v;
            const double nv = fma(t, -u, fma(c.y, prev, t));
            prev = v;
            v = nv;
            if (fabs(v) > 0x1p256) {
                v *= 0x1p-512;
                prev *= 0x1p-512;
                k += 1;
            }
        }
    }
    ls64[o] = l64;
    st64[o] = s64;
    ls32[o] = l32;
    st32[o] = s32;
}

// Spin-2 start states.  The spin-2 kernels run two independent three-term
// recurrences (the Wigner d^l_{m,-+2} recurrence, normalized by
// sqrt((2l+1)/4pi)) for y+ = 2lambda_lm / 2 and y- = -2lambda_lm / 2, and form
// lw = y+ + y-, lx = y+ - y- on the fly.  Kept apart, each recurrence carries
// only its own rounding: near the poles the two differ by ~theta^4 and a
// combined recurrence would let the large one pollute the small one.
// Seeds at l0 = max(m, 2), free of cancellation (u = 1 - cos theta):
//   m >= 2: 2lambda_mm = N_m m (m-1) lambda_mm tan^2(theta/2),
//           -2lambda_mm = N_m m (m-1) lambda_mm cot^2(theta/2),
//           N_m = ((m-1) m (m+1) (m+2))^-1/2, tan^2(theta/2) = u / (2 - u);
//   m = 1:  +-2lambda_21 = -+sqrt(5/16pi) sin(theta) (1 -+ cos theta);
//   m = 0:  +-2lambda_20 = sqrt(15/32pi) sin^2(theta)
// (these follow from applying the spin-raising operator twice to Y_lm).
// Each recurrence is walked in FP64 with exponent rescaling up to its first
// significant l.
struct Scaled {
    double v;
    int k;   // value = v * 2^(512 k)
    __device__ void norm() {
        if (v == 0.0) return;
        while (fabs(v) < 0x1p-256) {
            v *= 0x1p512;
            k -= 1;
        }
        while (fabs(v) > 0x1p256) {
            v *= 0x1p-512;
            k += 1;
        }
    }
};

__global__ void k_start_spin2(int lmax, int npairs, const double *__restrict__ u64,
                              const double *__restrict__ sect, const double4_32a *__restrict__ s2c,
                              double thr64, double thr32, int2 *ls64, double4_32a *st64, int2 *ls32,
                              float4 *st32) {
    const int pr = blockIdx.x * blockDim.x + threadIdx.x;
    const int m = blockIdx.y;
    if (pr >= npairs) return;
    const double u = u64[pr];
    const double s = sqrt(u * (2.0 - u));
    const int64_t o = (int64_t)m * npairs + pr;
    int lp64 = lmax + 1, lp32 = lmax + 1, lm64 = lmax + 1, lm32 = lmax + 1;
    double sd[4] = {0, 0, 0, 0};
    float sf[4] = {0.f, 0.f, 0.f, 0.f};
    const int l0 = m > 2 ? m : 2;
    if (s > 0.0 && l0 <= lmax) {
        Scaled y0[2];
        if (m >= 2) {
            double v = 0.28209479177387814347403972578;
            int k = 0;
            for (int j = 1; j <= m; ++j) {
                v *= -sect[j] * s;
                if (fabs(v) < 0x1p-256) {
                    v *= 0x1p512;
                    k -= 1;
                }
            }
            const double dm = m;
            const double nm = dm * (dm - 1.0) / sqrt((dm - 1.0) * dm * (dm + 1.0) * (dm + 2.0));
            const double t2 = u / (2.0 - u);
            y0[0].v = v * nm * t2;
            y0[1].v = v * nm / t2;
            y0[0].k = y0[1].k = k;
        } else if (m == 1) {
            const double c = sqrt(5.0 / (16.0 * 3.14159265358979323846)) * s;
            y0[0].v = -c * u;
            y0[1].v = c * (2.0 - u);
            y0[0].k = y0[1].k = 0;
        } else {
            const double c = sqrt(15.0 / (32.0 * 3.14159265358979323846)) * s * s;
            y0[0].v = c;
            y0[1].v = c;
            y0[0].k = y0[1].k = 0;
        }
        const int64_t base = (int64_t)m * (2 * lmax + 1 - m) / 2;
        for (int sp = 0; sp < 2; ++sp) {   // sp 0: y+ (A = alpha + beta), 1: y- (alpha - beta)
            Scaled y = y0[sp];
            y.norm();
            double prev = 0.0;
            int got32 = 0, got64 = 0;
            for (int l = l0;; ++l) {
                if (y.k == 0) {
                    const double a = fabs(y.v);
                    if (!got32 && a >= thr32) {
                        got32 = 1;
                        (sp ? lm32 : lp32) = l;
                        sf[2 * sp] = (float)(0.5 * prev);
                        sf[2 * sp + 1] = (float)(0.5 * y.v);
                    }
                    if (!got64 && a >= thr64) {
                        got64 = 1;
                        (sp ? lm64 : lp64) = l;
                        sd[2 * sp] = 0.5 * prev;
                        sd[2 * sp + 1] = 0.5 * y.v;
                    }
                    if (got32 && got64) break;
                }
                if (l >= lmax) break;
                const double4_32a c = s2c[base + l + 1];
                const double t = fma(-c.x, u, sp ? c.z : c.y);
                const double nv = fma(t, y.v, -c.w * prev);
                prev = y.v;
                y.v = nv;
                if (fabs(y.v) > 0x1p256) {
                    y.v *= 0x1p-512;
                    prev *= 0x1p-512;
                    y.k += 1;
                }
            }
        }
    }
    ls64[o] = make_int2(lp64, lm64);
    ls32[o] = make_int2(lp32, lm32);
    st64[o] = make_double4_32a(sd[0], sd[1], sd[2], sd[3]);
    st32[o] = make_float4(sf[0], sf[1], sf[2], sf[3]);
}

// ----------------------------------------------------------------- host FFT
static int ilog2(int64_t n) {
    int l = 0;
    while ((int64_t(1) << l) < n) ++l;
    return l;
}
static uint32_t bitrev(uint32_t x, int bits) {
    uint32_t r = 0;
    for (int i = 0; i < bits; ++i) r |= ((x >> i) & 1u) << (bits - 1 - i);
    return r;
}
// in-place forward DFT (e^{-2 pi i jk / M}) of length M = 2^logM, natural order out
static void host_fft(std::vector<std::complex<double>> &a, int logM) {
    const int M = 1 << logM;
    for (int i = 0; i < M; ++i) {
        const uint32_t j = bitrev(i, logM);
        if (j > (uint32_t)i) std::swap(a[i], a[j]);
    }
    for (int len = 2; len <= M; len <<= 1) {
        for (int k = 0; k < len / 2; ++k) {
            const double ang = -2.0 * PI * k / len;
            const std::complex<double> w(cos(ang), sin(ang));
            for (int i = 0; i < M; i += len) {
                const std::complex<double> x = a[i + k], y = a[i + k + len / 2] * w;
                a[i + k] = x + y;
                a[i + k + len / 2] = x - y;
            }
        }
    }
}

template <typename P> static int dalloc(Plan *p, P **ptr, size_t count) {
    const size_t bytes = count * sizeof(P);
    if (bytes == 0) {
        *ptr = nullptr;
        return SHTG_OK;
    }
    cudaError_t e = cudaMalloc((void **)ptr, bytes);
    if (e != cudaSuccess) {
        *ptr = nullptr;
        cudaGetLastError();
        set_error(std::string("cudaMalloc of ") + std::to_string(bytes) + " bytes failed: " +
                  cudaGetErrorString(e));
        return SHTG_ERR_NOMEM;
    }
    p->device_bytes += (int64_t)bytes;
    return SHTG_OK;
}
template <typename P> static int upload(P *dst, const std::vector<P> &src) {
    if (src.empty()) return SHTG_OK;
    SHTG_CUDA(cudaMemcpy(dst, src.data(), src.size() * sizeof(P), cudaMemcpyHostToDevice));
    return SHTG_OK;
}

// ----------------------------------------------------------------- geometry
static void build_geometry(Plan *p, std::vector<double> &u_pair) {
    if (p->geom == SHTG_GEOM_HEALPIX) {
        const int N = p->nside;
        p->nring = 4 * N - 1;
        p->npix = 12LL * N * N;
        p->cth.resize(p->nring);
        p->sth.resize(p->nring);
        p->nphi.resize(p->nring);
        p->shift.resize(p->nring);
        p->ofs.resize(p->nring);
        p->wring.assign(p->nring, 4.0 * PI / (double)p->npix);
        std::vector<double> uring(p->nring);
        int64_t off = 0;
        for (int i = 1; i <= 4 * N - 1; ++i) {
            const int ii = (i <= 2 * N) ? i : 4 * N - i;
            double u;
            int np_, sh;
            if (ii < N) {
                u = (double)ii * ii / (3.0 * N * N);
                np_ = 4 * ii;
                sh = 1;
            } else {
                u = (2.0 * ii - N) / (3.0 * N);
                np_ = 4 * N;
                sh = ((ii - N) % 2 == 0) ? 1 : 0;
            }
            const int r = i - 1;
            uring[r] = u;
            p->cth[r] = (i <= 2 * N) ? 1.0 - u : -(1.0 - u);
            p->sth[r] = sqrt(u * (2.0 - u));
            p->nphi[r] = np_;
            p->shift[r] = sh;
            p->ofs[r] = off;
            off += np_;
        }
        p->npairs = 2 * N;
        u_pair.resize(p->npairs);
        for (int r = 0; r < p->npairs; ++r) u_pair[r] = uring[r];
    } else {
        const int n = p->nring;
        const int nphi = p->nphi_gauss;
        p->npix = (int64_t)n * nphi;
        p->cth.resize(n);
        p->sth.resize(n);
        p->nphi.assign(n, nphi);
        p->shift.assign(n, 0);
        p->ofs.resize(n);
        p->wring.resize(n);
        for (int k = 0; k < n; ++k) {
            // Newton iteration on the Legendre polynomial P_n
            double x = cos(PI * (k + 0.75) / (n + 0.5)), dp = 1.0;
            for (int it = 0; it < 100; ++it) {
                double p0 = 1.0, p1 = x;
                for (int j = 2; j <= n; ++j) {
                    const double p2 = ((2.0 * j - 1.0) * x * p1 - (j - 1.0) * p0) / j;
                    p0 = p1;
                    p1 = p2;
                }
                if (n == 1) p0 = 1.0, p1 = x;
                dp = n * (x * p1 - p0) / (x * x - 1.0);
                const double dx = p1 / dp;
                x -= dx;
                if (fabs(dx) < 1e-16) break;
            }
            double p0 = 1.0, p1 = x;
            for (int j = 2; j <= n; ++j) {
                const double p2 = ((2.0 * j - 1.0) * x * p1 - (j - 1.0) * p0) / j;
                p0 = p1;
                p1 = p2;
            }
            if (n == 1) p0 = 1.0, p1 = x;
            dp = n * (x * p1 - p0) / (x * x - 1.0);
            p->cth[k] = x;
            p->sth[k] = sqrt((1.0 - x) * (1.0 + x));
            p->ofs[k] = (int64_t)k * nphi;
            p->wring[k] = 2.0 / ((1.0 - x * x) * dp * dp) * 2.0 * PI / nphi;
        }
        // symmetric nodes: the south half mirrors the north half exactly
        for (int k = 0; k < n / 2; ++k) {
            p->cth[n - 1 - k] = -p->cth[k];
            p->sth[n - 1 - k] = p->sth[k];
            p->wring[n - 1 - k] = p->wring[k];
        }
        if (n % 2 == 1) p->cth[n / 2] = 0.0, p->sth[n / 2] = 1.0;
        p->npairs = (n + 1) / 2;
        u_pair.resize(p->npairs);
        for (int r = 0; r < p->npairs; ++r) u_pair[r] = 1.0 - p->cth[r];
    }
    p->nalm = (int64_t)(p->lmax + 1) * (p->lmax + 2) / 2;
}

static int build_legendre_tables(Plan *p, const std::vector<double> &u_pair) {
    const int L = p->lmax;
    const int64_t P = p->nalm;
    std::vector<double2> rec64(P);
    std::vector<float2> rec32(P);
    std::vector<int> lof(P), mof(P);
    std::vector<double4_32a> s2c64(P);
    std::vector<float4> s2c32(P);
    for (int m = 0; m <= L; ++m) {
        for (int l = m; l <= L; ++l) {
            const int64_t i = alm_index(l, m, L);
            double a = 0.0, b = 0.0;
            if (l == m + 1) {
                a = sqrt(2.0 * m + 3.0);
            } else if (l >= m + 2) {
                const double dl = l, dm = m;
                a = sqrt((4.0 * dl * dl - 1.0) / (dl * dl - dm * dm));
                b = -a * sqrt(((dl - 1.0) * (dl - 1.0) - dm * dm) / (4.0 * (dl - 1.0) * (dl - 1.0) - 1.0));
            }
            rec64[i] = make_double2(a, b);
            rec32[i] = make_float2((float)a, (float)b);
            lof[i] = l;
            mof[i] = m;
            // spin-2 recurrence (Wigner d^l_{m,-2}, normalized by sqrt((2l+1)/4pi)):
            //   y_l = (alpha (1 - u) + beta) y_{l-1} - gamma y_{l-2}
            // for y = 2lambda; -2lambda has -beta.  Coefficients of the step that
            // produces l (from l-1, l-2), defined for l - 1 >= max(m, 2).  With
            // k = l - 1, D = k sqrt((k+1)^2 - m^2) sqrt((k+1)^2 - 4),
            // f = sqrt((2k+3)/(2k+1)): alpha = f (2k+1) k (k+1) / D,
            // beta = 2 m f (2k+1) / D, gamma = f sqrt((2k+1)/(2k-1)) (k+1)
            // sqrt(k^2 - m^2) sqrt(k^2 - 4) / D.
            double al = 0, be = 0, ga = 0;
            const int k = l - 1;
            if (k >= 2 && k >= m) {
                const double dk = k, dm = m;
                const double D = dk * sqrt((dk + 1) * (dk + 1) - dm * dm) * sqrt((dk + 1) * (dk + 1) - 4.0);
                const double f = sqrt((2 * dk + 3) / (2 * dk + 1));
                al = f * (2 * dk + 1) * dk * (dk + 1) / D;
                be = f * (2 * dk + 1) * 2.0 * dm / D;
                ga = f * sqrt((2 * dk + 1) / (2 * dk - 1)) * (dk + 1) * sqrt(dk * dk - dm * dm) *
                     sqrt(dk * dk - 4.0) / D;
            }
            // stored as (alpha, alpha + beta, alpha - beta, gamma)
            s2c64[i] = make_double4_32a(al, al + be, al - be, ga);
            s2c32[i] = make_float4((float)al, (float)(al + be), (float)(al - be), (float)ga);
        }
    }
    SHTG_TRY(dalloc(p, &p->d_rec64, P));
    SHTG_TRY(dalloc(p, &p->d_rec32, P));
    SHTG_TRY(dalloc(p, &p->d_lofidx, P));
    SHTG_TRY(dalloc(p, &p->d_mofidx, P));
    SHTG_TRY(dalloc(p, &p->d_s2c64, P));
    SHTG_TRY(dalloc(p, &p->d_s2c32, P));
    SHTG_TRY(upload(p->d_rec64, rec64));
    SHTG_TRY(upload(p->d_rec32, rec32));
    SHTG_TRY(upload(p->d_lofidx, lof));
    SHTG_TRY(upload(p->d_mofidx, mof));
    SHTG_TRY(upload(p->d_s2c64, s2c64));
    SHTG_TRY(upload(p->d_s2c32, s2c32));

    // per-pair geometry
    const int NP = p->npairs;
    std::vector<double> x64(NP), is2_64(NP);
    std::vector<float> u32(NP), x32(NP), is2_32(NP);
    for (int r = 0; r < NP; ++r) {
        const double u = u_pair[r];
        const double s2 = u * (2.0 - u);
        x64[r] = 1.0 - u;
        is2_64[r] = 1.0 / s2;
        u32[r] = (float)u;
        x32[r] = (float)(1.0 - u);
        is2_32[r] = (float)(1.0 / s2);
    }
    SHTG_TRY(dalloc(p, &p->d_u64, NP));
    SHTG_TRY(dalloc(p, &p->d_u32, NP));
    SHTG_TRY(dalloc(p, &p->d_x64, NP));
    SHTG_TRY(dalloc(p, &p->d_x32, NP));
    SHTG_TRY(dalloc(p, &p->d_is2_64, NP));
    SHTG_TRY(dalloc(p, &p->d_is2_32, NP));
    SHTG_TRY(upload(p->d_u64, u_pair));
    SHTG_TRY(upload(p->d_u32, u32));
    SHTG_TRY(upload(p->d_x64, x64));
    SHTG_TRY(upload(p->d_x32, x32));
    SHTG_TRY(upload(p->d_is2_64, is2_64));
    SHTG_TRY(upload(p->d_is2_32, is2_32));

    // start states
    std::vector<double> sect(L + 2, 0.0);
    for (int k = 1; k <= L; ++k) sect[k] = sqrt((2.0 * k + 1.0) / (2.0 * k));
    double *d_sect = nullptr;
    SHTG_CUDA(cudaMalloc(&d_sect, sect.size() * sizeof(double)));
    cudaMemcpy(d_sect, sect.data(), sect.size() * sizeof(double), cudaMemcpyHostToDevice);
    const int64_t ns = (int64_t)(L + 1) * NP;
    SHTG_TRY(dalloc(p, &p->d_ls64, ns));
    SHTG_TRY(dalloc(p, &p->d_st64, ns));
    SHTG_TRY(dalloc(p, &p->d_ls32, ns));
    SHTG_TRY(dalloc(p, &p->d_st32, ns));
    dim3 grid((NP + 127) / 128, L + 1);
    // thresholds: terms below 2^-80 (FP64 kernels) / 2^-56 (FP32 kernels) are
    // dropped; both leave room for the 1/sin^2 factor of the spin-2 functions.
    k_start_states<<<grid, 128>>>(L, NP, p->d_u64, d_sect, p->d_rec64, 0x1p-80, 0x1p-56,
                                  p->d_ls64, p->d_st64, p->d_ls32, p->d_st32);
    if (p->flags & SHTG_SPIN2) {
        SHTG_TRY(dalloc(p, &p->d_ls2_64, ns));
        SHTG_TRY(dalloc(p, &p->d_st2_64, ns));
        SHTG_TRY(dalloc(p, &p->d_ls2_32, ns));
        SHTG_TRY(dalloc(p, &p->d_st2_32, ns));
        k_start_spin2<<<grid, 128>>>(L, NP, p->d_u64, d_sect, p->d_s2c64, 0x1p-80, 0x1p-56,
                                     p->d_ls2_64, p->d_st2_64, p->d_ls2_32, p->d_st2_32);
    }
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    cudaFree(d_sect);
    if (e != cudaSuccess) return cuda_fail(e, "k_start_states", __FILE__, __LINE__);
    return SHTG_OK;
}

static int build_fft_tables(Plan *p) {
    const int R = p->nring;
    p->h_rfft.resize(R);
    int logmax = 1;
    std::map<int, std::pair<int64_t, int64_t>> offs;  // n -> (chirp_off, bhat_off)
    int64_t chirp_total = 0, bhat_total = 0;
    for (int r = 0; r < R; ++r) {
        RingFFT f;
        f.n = p->nphi[r];
        f.shift = p->shift[r];
        const int lg = ilog2(f.n);
        if ((1 << lg) == f.n) {
            f.blue = 0;
            f.logM = lg;
            f.chirp_off = f.bhat_off = 0;
        } else {
            f.blue = 1;
            f.logM = ilog2(2 * (int64_t)f.n - 1);
            auto it = offs.find(f.n);
            if (it == offs.end()) {
                offs[f.n] = std::make_pair(chirp_total, bhat_total);
                f.chirp_off = chirp_total;
                f.bhat_off = bhat_total;
                chirp_total += f.n;
                bhat_total += (int64_t)1 << f.logM;
            } else {
                f.chirp_off = it->second.first;
                f.bhat_off = it->second.second;
            }
        }
        if (f.logM > logmax) logmax = f.logM;
        p->h_rfft[r] = f;
    }
    if (logmax > SHTG_FFT_LOGMAX) {
        set_error("ring transform length 2^" + std::to_string(logmax) + " above the supported 2^" +
                  std::to_string(SHTG_FFT_LOGMAX) + " (HEALPix N_side <= 1024; Gauss-Legendre nphi a "
                  "power of two <= 8192, or any nphi <= 4096)");
        return SHTG_ERR_ARG;
    }
    p->fft_logmax = logmax;
    const int Mmax = 1 << logmax;
    p->tw_blo = (logmax + 1) / 2;
    p->tw_nlo = 1 << p->tw_blo;
    p->tw_nhi = 1 << (logmax - p->tw_blo);
    std::vector<double2> tw64(p->tw_nlo + p->tw_nhi);
    std::vector<float2> tw32(tw64.size());
    for (int i = 0; i < p->tw_nlo + p->tw_nhi; ++i) {
        const int64_t t = i < p->tw_nlo ? i : (int64_t)(i - p->tw_nlo) << p->tw_blo;
        const double ang = -2.0 * PI * (double)t / (double)Mmax;
        tw64[i] = make_double2(cos(ang), sin(ang));
        tw32[i] = make_float2((float)cos(ang), (float)sin(ang));
    }
    // per-pass twiddles of the fixed-length FFT passes (ringfft.cu) for
    // M = 2^10 .. 2^13: radix-16 pass p with NS = 2^(logm mod 4) 16^p > 1 holds
    // e^{-2 pi i r k / (16 NS)} for r = 1 at k and r = 4 at NS + k, k < NS
    std::vector<double2> twf64;
    std::vector<float2> twf32;
    for (int lg = 10; lg <= SHTG_FFT_LOGMAX; ++lg) {
        p->twf_off[lg] = (int64_t)twf64.size();
        for (int ps = 0; ps < (lg >> 2); ++ps) {
            const int ns = (1 << (lg & 3)) << (4 * ps);
            if (ns == 1) continue;
            for (int r : {1, 4})
                for (int k = 0; k < ns; ++k) {
                    const int64_t t = ((int64_t)r * k) % (16 * (int64_t)ns);
                    const double ang = -2.0 * PI * (double)t / (16.0 * ns);
                    twf64.push_back(make_double2(cos(ang), sin(ang)));
                    twf32.push_back(make_float2((float)cos(ang), (float)sin(ang)));
                }
        }
    }
    std::vector<double2> ch64(chirp_total), bf64(bhat_total), bi64(bhat_total);
    std::vector<float2> ch32(chirp_total), bf32(bhat_total), bi32(bhat_total);
    for (auto &kv : offs) {
        const int n = kv.first;
        const int64_t co = kv.second.first, bo = kv.second.second;
        const int lgM = ilog2(2 * (int64_t)n - 1);
        const int M = 1 << lgM;
        std::vector<std::complex<double>> c(n);
        for (int j = 0; j < n; ++j) {
            const int64_t q = ((int64_t)j * j) % (2 * (int64_t)n);
            const double ang = -PI * (double)q / (double)n;   // c_j = e^{-i pi j^2 / n}
            c[j] = std::complex<double>(cos(ang), sin(ang));
            ch64[co + j] = make_double2(c[j].real(), c[j].imag());
            ch32[co + j] = make_float2((float)c[j].real(), (float)c[j].imag());
        }
        std::vector<std::complex<double>> bfw(M, 0.0), biv(M, 0.0);
        for (int j = 0; j < n; ++j) {
            bfw[j] = std::conj(c[j]);
            biv[j] = c[j];
            if (j > 0) {
                bfw[M - j] = std::conj(c[j]);
                biv[M - j] = c[j];
            }
        }
        host_fft(bfw, lgM);
        host_fft(biv, lgM);
        for (int i = 0; i < M; ++i) {
            const std::complex<double> a = bfw[i] / (double)M, b = biv[i] / (double)M;
            bf64[bo + i] = make_double2(a.real(), a.imag());
            bi64[bo + i] = make_double2(b.real(), b.imag());
            bf32[bo + i] = make_float2((float)a.real(), (float)a.imag());
            bi32[bo + i] = make_float2((float)b.real(), (float)b.imag());
        }
    }
    // e^{i pi k / n} (phi0 = pi / n) for k <= min(lmax, n - 1), one table per
    // distinct n of the shifted rings
    std::map<int, int64_t> phoffs;
    std::vector<double2> ph64;
    std::vector<float2> ph32;
    for (int r = 0; r < R; ++r) {
        RingFFT &f = p->h_rfft[r];
        f.ph_off = 0;
        if (!f.shift) continue;
        auto it = phoffs.find(f.n);
        if (it != phoffs.end()) {
            f.ph_off = it->second;
            continue;
        }
        f.ph_off = (int64_t)ph64.size();
        phoffs[f.n] = f.ph_off;
        const int kmax = std::min(p->lmax, f.n - 1);
        for (int k = 0; k <= kmax; ++k) {
            const double ang = PI * (double)k / (double)f.n;
            ph64.push_back(make_double2(cos(ang), sin(ang)));
            ph32.push_back(make_float2((float)cos(ang), (float)sin(ang)));
        }
    }
    if (ph64.empty()) {
        ph64.push_back(make_double2(1.0, 0.0));
        ph32.push_back(make_float2(1.0f, 0.0f));
    }
    SHTG_TRY(dalloc(p, &p->d_rph64, ph64.size()));
    SHTG_TRY(dalloc(p, &p->d_rph32, ph32.size()));
    SHTG_TRY(upload(p->d_rph64, ph64));
    SHTG_TRY(upload(p->d_rph32, ph32));
    SHTG_TRY(dalloc(p, &p->d_rfft, R));
    SHTG_TRY(upload(p->d_rfft, p->h_rfft));
    SHTG_TRY(dalloc(p, &p->d_twf64, twf64.size()));
    SHTG_TRY(dalloc(p, &p->d_twf32, twf32.size()));
    SHTG_TRY(upload(p->d_twf64, twf64));
    SHTG_TRY(upload(p->d_twf32, twf32));
    SHTG_TRY(dalloc(p, &p->d_tw64, tw64.size()));
    SHTG_TRY(dalloc(p, &p->d_tw32, tw32.size()));
    SHTG_TRY(upload(p->d_tw64, tw64));
    SHTG_TRY(upload(p->d_tw32, tw32));
    SHTG_TRY(dalloc(p, &p->d_chirp64, ch64.size()));
    SHTG_TRY(dalloc(p, &p->d_chirp32, ch32.size()));
    SHTG_TRY(dalloc(p, &p->d_bfwd64, bf64.size()));
    SHTG_TRY(dalloc(p, &p->d_binv64, bi64.size()));
    SHTG_TRY(dalloc(p, &p->d_bfwd32, bf32.size()));
    SHTG_TRY(dalloc(p, &p->d_binv32, bi32.size()));
    SHTG_TRY(upload(p->d_chirp64, ch64));
    SHTG_TRY(upload(p->d_chirp32, ch32));
    SHTG_TRY(upload(p->d_bfwd64, bf64));
    SHTG_TRY(upload(p->d_binv64, bi64));
    SHTG_TRY(upload(p->d_bfwd32, bf32));
    SHTG_TRY(upload(p->d_binv32, bi32));
    p->fft_smem64 = (size_t)Mmax * sizeof(double2);
    p->fft_smem32 = (size_t)Mmax * sizeof(float2);
    // Launch buckets by transform length, each launch with M / 16 threads
    // (one radix-16 butterfly per thread): Bluestein rings by their M, direct
    // rings without aliasing (n >= 2 lmax) by n, aliased direct rings by 2n so
    // that the south ring's folded spectrum fits in buf[n, 2n); buckets of
    // length 1024 and below share one launch.  Buckets above 1024 are split
    // by the members' own M (the aliased direct rings of a bucket have half
    // its length), so each of their launches runs one fixed transform length.
    std::vector<int> groups;
    {
        // (key, fix) -> ring pairs; key = launch length, fix = members' log2 M (0: mixed)
        std::map<std::pair<int, int>, std::vector<int>, std::greater<std::pair<int, int>>> bucket;
        std::map<int, int> keymax;
        for (int r = 0; r < p->npairs; ++r) {
            const RingFFT &f = p->h_rfft[r];
            const bool aliased = f.n < 2 * p->lmax;
            const int slot = (f.blue || !aliased) ? f.logM : f.logM + 1;
            const int key = std::max(slot, 10);
            bucket[std::make_pair(key, key > 10 ? f.logM : 0)].push_back(r);
            keymax[key] = std::max(keymax.count(key) ? keymax[key] : 0, slot);
        }
        p->ring_launch.clear();
        for (auto &kv : bucket) {
            Plan::RingLaunch g;
            g.off = (int)groups.size();
            g.count = (int)kv.second.size();
            g.logm = keymax[kv.first.first];
            g.fix = kv.first.second;
            g.alias = 0;
            g.chirp = 0;
            const int nt = g.fix ? (1 << g.fix) / 16 : ring_threads(g.logm);
            for (int r : kv.second) {
                const RingFFT &f = p->h_rfft[r];
                groups.push_back(r);
                if (f.n < 2 * p->lmax) g.alias = 1;
                if (f.blue) g.chirp = std::max(g.chirp, f.n);
                // the kernel's passes cover this ring: M / 16 butterflies per
                // radix-16 pass, M / R in the first pass
                const int M = 1 << f.logM, R = 1 << (f.logM & 3);
                // launches of buckets above 1024 run the fixed-length passes
                // of their members' one length, 2^logm or 2^(logm - 1)
                const bool fix_ok = g.fix == 0 ? g.logm <= 10
                                               : (g.fix == f.logM && (f.logM == g.logm || f.logM == g.logm - 1));
                const bool ok = fix_ok && M <= 16 * nt && (R == 1 || M / R <= nt * ring_first_bpt(R, nt)) &&
                                (f.n >= 2 * p->lmax || 2 * (int64_t)f.n <= ((int64_t)1 << g.logm));
                if (!ok) {
                    set_error("ring " + std::to_string(r) + ": transform length " + std::to_string(M) +
                              " does not fit its launch bucket 2^" + std::to_string(g.logm));
                    return SHTG_ERR_ARG;
                }
            }
            p->ring_launch.push_back(g);
        }
    }
    SHTG_TRY(dalloc(p, &p->d_ring_groups, groups.size()));
    SHTG_TRY(upload(p->d_ring_groups, groups));
    return SHTG_OK;
}

int plan_build(Plan *p) {
    std::vector<double> u_pair;
    build_geometry(p, u_pair);
    {
        std::vector<int> nph(p->nphi.begin(), p->nphi.end());
        SHTG_TRY(dalloc(p, &p->d_nphi, p->nring));
        SHTG_TRY(upload(p->d_nphi, nph));
        SHTG_TRY(dalloc(p, &p->d_ofs, p->nring));
        SHTG_TRY(upload(p->d_ofs, p->ofs));
        SHTG_TRY(dalloc(p, &p->d_wring, p->nring));
        SHTG_TRY(upload(p->d_wring, p->wring));
    }
    SHTG_TRY(build_legendre_tables(p, u_pair));
    SHTG_TRY(build_tile_states(p));
    SHTG_TRY(build_tile_states64(p));
    SHTG_TRY(build_fft_tables(p));
    // workspace
    const int spin2 = (p->flags & SHTG_SPIN2) ? 1 : 0;
    p->nmaps_max = p->max_batch * (spin2 ? 3 : 1);
    const int64_t nph = (int64_t)p->nmaps_max * (p->lmax + 1) * p->nring;
    SHTG_TRY(dalloc(p, &p->d_phase64, nph));
    SHTG_TRY(dalloc(p, &p->d_phase32, nph));
    const int64_t nmp = (int64_t)p->nmaps_max * p->npix;
    SHTG_TRY(dalloc(p, &p->d_map64, nmp));
    SHTG_TRY(dalloc(p, &p->d_map32, nmp));
    SHTG_TRY(dalloc(p, &p->d_ninv64, 2 * p->npix));
    SHTG_TRY(dalloc(p, &p->d_ninv32, 2 * p->npix));
    // solver workspace
    const int64_t nv = (int64_t)p->nmaps_max * p->nalm;
    for (int i = 0; i < 7; ++i) SHTG_TRY(dalloc(p, &p->v64[i], nv));
    for (int i = 0; i < 5; ++i) SHTG_TRY(dalloc(p, &p->v32[i], nv));
    SHTG_TRY(dalloc(p, &p->d_minv64, 4 * (int64_t)p->max_batch * p->nalm));
    SHTG_TRY(dalloc(p, &p->d_minv32, 4 * (int64_t)p->max_batch * p->nalm));
    SHTG_TRY(dalloc(p, &p->d_isc64, p->max_batch));
    SHTG_TRY(dalloc(p, &p->d_rsc64, p->max_batch));
    SHTG_TRY(dalloc(p, &p->d_isc32, p->max_batch));
    SHTG_TRY(dalloc(p, &p->d_diagT, p->nalm));
    SHTG_TRY(dalloc(p, &p->d_diagP, p->nalm));
    SHTG_TRY(dalloc(p, &p->d_wpairT, p->npairs));
    SHTG_TRY(dalloc(p, &p->d_wpairP, p->npairs));
    SHTG_TRY(dalloc(p, &p->d_ltab64, 9 * (int64_t)(p->lmax + 1)));
    SHTG_TRY(dalloc(p, &p->d_jtab, 13 * (int64_t)(p->lmax + 1)));
    if (p->flags & SHTG_BLOCK_SOLVER) {
        SHTG_TRY(block_workspace(p));
        SHTG_TRY(dalloc(p, &p->d_blk, p->blk_cap));
        SHTG_TRY(dalloc(p, &p->d_blklam, p->lam_cap));
        SHTG_TRY(dalloc(p, &p->d_blkw, 2 * (int64_t)p->npairs));
        SHTG_TRY(dalloc(p, &p->d_blkoff, 2 * (int64_t)(p->lmax + 1)));
        SHTG_TRY(dalloc(p, &p->d_blkflag, 4));
    }
    SHTG_TRY(dalloc(p, &p->d_ltab32, 5 * (int64_t)(p->lmax + 1)));
    SHTG_TRY(dalloc(p, &p->d_scal, 16 * (int64_t)p->max_batch));
    // reduction partials [4 max_batch][RED_BLOCKS], then per-realization scalars
    // of the mixed solver [4 max_batch] and per-realization sums [max_batch]
    SHTG_TRY(dalloc(p, &p->d_part, 4 * (int64_t)p->max_batch * SHTG_RED_BLOCKS + 5 * (int64_t)p->max_batch + 64));
    SHTG_TRY(dalloc(p, &p->d_lsum, (int64_t)p->lmax + 1));
    SHTG_CUDA(cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking));
    SHTG_CUDA(cudaStreamCreateWithFlags(&p->work_stream, cudaStreamNonBlocking));
    SHTG_CUDA(cudaEventCreateWithFlags(&p->ring_fork, cudaEventDisableTiming));
    for (int i = 0; i < Plan::RING_SIDE; ++i) {
        SHTG_CUDA(cudaStreamCreateWithFlags(&p->ring_side[i], cudaStreamNonBlocking));
        SHTG_CUDA(cudaEventCreateWithFlags(&p->ring_join[i], cudaEventDisableTiming));
    }
    SHTG_TRY(dalloc(p, &p->d_flag, 16));
    SHTG_CUDA(cudaMemset(p->d_flag, 0, 16 * sizeof(int)));
    // solver scalars and partials start defined (a fresh allocation may hold
    // what an earlier plan left there)
    SHTG_CUDA(cudaMemset(p->d_scal, 0, sizeof(double) * 16 * (size_t)p->max_batch));
    SHTG_CUDA(cudaMemset(p->d_part, 0,
                         sizeof(double) * (4 * (size_t)p->max_batch * SHTG_RED_BLOCKS + 5 * (size_t)p->max_batch + 64)));
    SHTG_TRY(dalloc(p, &p->d_stage, nmp));
    // pinned host scalars: the [max_batch][16] CG slots (host convergence
    // checks), then [max_batch] per-realization sums
    SHTG_CUDA(cudaMallocHost((void **)&p->h_pinned, (17 * (size_t)p->max_batch + 64) * sizeof(double)));
    p->prof.ev.resize(16384);
    for (auto &e : p->prof.ev) SHTG_CUDA(cudaEventCreate(&e));
    p->prof.cls.reserve(8192);
    SHTG_CUDA(cudaDeviceSynchronize());
    return SHTG_OK;
}

void plan_free(Plan *p) {
    lowl_free(p);
    az_free(p);
    void *ptrs[] = {p->d_nphi, p->d_ofs, p->d_wring, p->d_u64, p->d_u32, p->d_x64, p->d_is2_64,
                    p->d_x32, p->d_is2_32, p->d_lofidx, p->d_mofidx, p->d_rec64, p->d_rec32,
                    p->d_ls64, p->d_ls32, p->d_st64, p->d_st32, p->d_s2c64, p->d_s2c32,
                    p->d_rfft, p->d_tw64, p->d_tw32, p->d_chirp64, p->d_bfwd64, p->d_binv64,
                    p->d_chirp32, p->d_bfwd32, p->d_binv32, p->d_phase64, p->d_phase32,
                    p->d_map64, p->d_map32, p->d_ninv64, p->d_ninv32, p->d_minv64,
                    p->d_minv32, p->d_diagT, p->d_diagP, p->d_wpairT, p->d_wpairP,
                    p->d_ltab64, p->d_ltab32, p->d_scal, p->d_part, p->d_lsum, p->d_stage,
                    p->d_ls2_64, p->d_st2_64, p->d_ls2_32, p->d_st2_32, p->d_ring_groups, p->d_flag,
                    p->d_toff, p->d_tst0, p->d_tst2, p->d_isc64, p->d_rsc64, p->d_isc32,
                    p->d_toff64, p->d_tst64_0, p->d_tst64_2, p->d_rph64, p->d_rph32, p->d_twf64,
                    p->d_twf32, p->d_jtab, p->d_blk, p->d_blklam, p->d_blkw, p->d_blkoff,
                    p->d_blkflag};
    for (void *q : ptrs)
        if (q) cudaFree(q);
    for (int i = 0; i < 7; ++i)
        if (p->v64[i]) cudaFree(p->v64[i]);
    for (int i = 0; i < 5; ++i)
        if (p->v32[i]) cudaFree(p->v32[i]);
    if (p->h_pinned) cudaFreeHost(p->h_pinned);
    if (p->cap_stream) cudaStreamDestroy(p->cap_stream);
    if (p->work_stream) cudaStreamDestroy(p->work_stream);
    for (int i = 0; i < Plan::RING_SIDE; ++i) {
        if (p->ring_side[i]) cudaStreamDestroy(p->ring_side[i]);
        if (p->ring_join[i]) cudaEventDestroy(p->ring_join[i]);
    }
    if (p->ring_fork) cudaEventDestroy(p->ring_fork);
    for (auto &e : p->prof.ev)
        if (e) cudaEventDestroy(e);
    p->prof.ev.clear();
}

void prof_collect(Plan *p, double *ms, int *count) {
    Prof &f = p->prof;
    for (int i = 0; i < f.n; ++i) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, f.ev[2 * i], f.ev[2 * i + 1]) == cudaSuccess) {
            const int c = f.cls[i];
            if (ms) ms[c] += t;
            if (count) count[c] += 1;
        } else {
            cudaGetLastError();
        }
    }
    f.n = 0;
    f.open_cls = -1;
}

int check_device_flag(Plan *p, cudaStream_t st) {
    int h = 0;
    SHTG_CUDA(cudaMemcpyAsync(&h, p->d_flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    SHTG_CUDA(cudaStreamSynchronize(st));
    // Host-side fault injection for tests of the error path: with
    // SHTG_FAKE_WAIT_EXPIRY=1 in the environment the flag reads as set, as if
    // a kernel's bounded wait had expired (no device wait is forced to expire).
    {
        const char *e = getenv("SHTG_FAKE_WAIT_EXPIRY");
        if (e && e[0] == '1') h = 1;
    }
    if (h) {
        SHTG_CUDA(cudaMemsetAsync(p->d_flag, 0, sizeof(int), st));
        set_error("a tensor-core kernel gave up waiting for its MMAs (bounded mbarrier wait expired)");
        return SHTG_ERR_TIMEOUT;
    }
    return SHTG_OK;
}

}  // namespace shtg

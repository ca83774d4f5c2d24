// Legendre stage of the spherical-harmonic transforms (the l-sum of Y and
// its transpose), the compute-bound core of every operator application of
// Eq. (mapmakingeq).
//
// Synthesis:  F_r(m) = sum_l a_lm lambda_lm(theta_r)            (spin 0)
// Analysis:   c_lm   = sum_r lambda_lm(theta_r) G_r(m)           (transpose)
// Rings come in north/south pairs theta, pi - theta; lambda_lm(pi - theta) =
// (-1)^(l+m) lambda_lm(theta) (App. A), so one recurrence serves both rings:
// even and odd l - m partial sums E, O give F_N = E + O, F_S = E - O.
//
// Spin 2 (Q, U from E, B): with lw = (2Y + -2Y)/2, lx = (2Y - -2Y)/2 (theta
// parts; lw has parity (-1)^(l+m), lx the opposite one), obtained from their
// own coupled three-term recurrence (the Wigner d^l_{m,-+2} recurrence), which
// has no 1/sin^2 theta cancellation near the poles,
//   F_Q = - sum_l (E lw + i B lx),   F_U = sum_l (i E lx - B lw),
// and the analysis is the exact transpose
//   E^ = sum_r (-lw G_Q - i lx G_U),  B^ = sum_r (i lx G_Q - lw G_U).
//
// Work decomposition: one CTA per (m, block of ring pairs, group of maps);
// each thread owns NR ring pairs and keeps their recurrence in registers;
// the per-l coefficients and alm of the CTA's m are staged in shared memory
// and read as warp-wide broadcasts.  Each thread starts at the FP64-computed
// start state of its rings (first l above the significance threshold), so
// the loop carries no rescaling.  The analysis reduces over the warp's
// rings with a butterfly transpose-reduce of 8 consecutive l at a time.
#pragma once

#include <cstdlib>
#include <cstdio>

#include "common.cuh"

namespace shtg {

#define LEG_THREADS 128
#define LEG_CHUNK 128

// ------------------------------------------------------------- autotuner
// Key: (kernel kind, family, nmaps).  On the first call with a key every
// candidate runs twice on the caller's buffers (all compute the same
// result); the second run of each is timed with CUDA events on the stream
// and the fastest is kept.  SHTG_TUNE=0 in the environment, or profiling,
// keeps variant 0; SHTG_TUNE_LOG=1 prints every candidate's time to stderr.
inline bool tuning_enabled() {
    static int on = -1;
    if (on < 0) {
        const char *e = getenv("SHTG_TUNE");
        on = (e && e[0] == '0') ? 0 : 1;
    }
    return on == 1;
}
// SHTG_TUNE_FORCE=v: every tuned family runs its variant v (variant 0 where
// it has fewer), for profiling one shape or checking each shape on its own
inline int tuning_force() {
    static int v = -2;
    if (v == -2) {
        const char *e = getenv("SHTG_TUNE_FORCE");
        v = (e && e[0] >= '0' && e[0] <= '9') ? atoi(e) : -1;
    }
    return v;
}

inline bool tuning_log() {
    static int on = -1;
    if (on < 0) {
        const char *e = getenv("SHTG_TUNE_LOG");
        on = (e && e[0] == '1') ? 1 : 0;
    }
    return on == 1;
}

template <typename Run>
int tune(Plan *p, int key_prec, int family, int nmaps, int nvar, cudaStream_t st, Run run) {
    const long long key = ((long long)key_prec * 16 + family) * 65536 + nmaps;
    auto it = p->tuned.find(key);
    if (it != p->tuned.end()) return run(it->second);
    if (tuning_force() >= 0) {
        p->tuned[key] = tuning_force() < nvar ? tuning_force() : 0;
        return run(p->tuned[key]);
    }
    if (!tuning_enabled() || nvar <= 1 || p->prof.on) {
        p->tuned[key] = 0;
        return run(0);
    }
    cudaEvent_t e0, e1;
    SHTG_CUDA(cudaEventCreate(&e0));
    SHTG_CUDA(cudaEventCreate(&e1));
    int best = 0;
    float tbest = 1e30f;
    for (int v = 0; v < nvar; ++v) {
        int rc = run(v);
        if (rc != SHTG_OK) continue;
        cudaEventRecord(e0, st);
        rc = run(v);
        cudaEventRecord(e1, st);
        if (rc != SHTG_OK) continue;
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (tuning_log())
            fprintf(stderr, "shtg tune: kind %d family %d nmaps %d variant %d: %.3f ms\n", key_prec, family, nmaps,
                    v, ms);
        if (ms < tbest) {
            tbest = ms;
            best = v;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    p->tuned[key] = best;
    return run(best);
}

template <typename T> struct V4;
template <> struct V4<float> { typedef float4 t; };
template <> struct V4<double> { typedef double4_32a t; };

template <typename T> struct LegArgs {
    typedef typename VT<T>::C C;
    typedef typename V4<T>::t C4;
    int lmax, npairs, nring, nmaps;
    int rs;             // alm row stride (in rows of nalm) between maps
    int vjp;            // analysis: double the m > 0 outputs
    int64_t nalm;
    const C *alm;       // synthesis input / analysis output
    C *F;               // [map][ring][m]
    const T *beam;      // [lmax+1] or null
    const C *rec;       // (a, b) per alm index
    const C4 *s2c;      // spin-2 constants per alm index
    const int *ls;      // [m][pair]
    const C *st;        // [m][pair]
    const int2 *ls2;    // [m][pair] start l of the y+ / y- recurrences
    const C4 *st2;      // [m][pair] (y+_{l-1}, y+_l, y-_{l-1}, y-_l), y = +-2lambda / 2
    const T *u;
    const float *wpair; // diag kernel: ring weights summed over the pair
    float *diag;        // diag kernel output
    int *err;           // tensor-core kernels: set to 1 when a bounded wait expires
    const int64_t *toff;  // tensor-core transpose: recurrence states every 32 l (FP32 plans)
    const float2 *tst0;
    const float4 *tst2;
    const int64_t *toff64;    // FP64 recurrence states every SHTG_TS64 l (FP64 and double-FP32 transposes)
    const double2 *tst64_0;
    const double4_32a *tst64_2;
};

// one recurrence step: (l1, l2) = (lambda_{l-1}, lambda_{l-2}) -> (lambda_l, lambda_{l-1})
template <typename T>
__device__ __forceinline__ void rstep(T &l1, T &l2, const T a, const T b, const T u) {
    const T t = a * l1;
    const T n = fma(t, -u, fma(b, l2, t));
    l2 = l1;
    l1 = n;
}

template <typename T, int NR>
struct PairState {
    int pr[NR];
    T u[NR];
    int ls[NR], lsb[NR];                // start l (spin 2: of y+ and of y-)
    T s0[NR], s1[NR], s2[NR], s3[NR];   // start values
    T a1[NR], a2[NR];   // spin 0: lambda_l, lambda_{l-1}; spin 2: y+_l, y+_{l-1}
    T b1[NR], b2[NR];   // spin 2: y-_l, y-_{l-1}
};

// Load the per-pair geometry and start states; returns the warp's l range.
template <typename T, int NR, int SPIN>
__device__ __forceinline__ void load_pairs(const LegArgs<T> &a, int bx, int m, PairState<T, NR> &S,
                                           int &warp_lo, int &warp_hi) {
    const int L = a.lmax;
    int lo = L + 1, hi = -1;
#pragma unroll
    for (int j = 0; j < NR; ++j) {
        const int pr = bx * (LEG_THREADS * NR) + j * LEG_THREADS + threadIdx.x;
        S.pr[j] = pr;
        S.a1[j] = S.a2[j] = S.b1[j] = S.b2[j] = T(0);
        S.u[j] = T(1);
        S.ls[j] = L + 1;
        S.lsb[j] = L + 1;
        S.s0[j] = S.s1[j] = S.s2[j] = S.s3[j] = T(0);
        if (pr < a.npairs) {
            S.u[j] = a.u[pr];
            const int64_t o = (int64_t)m * a.npairs + pr;
            if (SPIN == 2) {
                const int2 q = a.ls2[o];
                S.ls[j] = q.x;
                S.lsb[j] = q.y;
                const typename LegArgs<T>::C4 s = a.st2[o];
                S.s0[j] = s.x;
                S.s1[j] = s.y;
                S.s2[j] = s.z;
                S.s3[j] = s.w;
            } else {
                S.ls[j] = a.ls[o];
                const typename VT<T>::C s = a.st[o];
                S.s0[j] = s.x;
                S.s1[j] = s.y;
            }
        }
        lo = min(lo, min(S.ls[j], S.lsb[j]));
        if (S.ls[j] <= L) hi = max(hi, S.ls[j]);
        if (S.lsb[j] <= L) hi = max(hi, S.lsb[j]);
    }
    warp_lo = __reduce_min_sync(0xffffffffu, lo);
    warp_hi = __reduce_max_sync(0xffffffffu, hi);
}

// spin 0: lambda_l = a (1 - u) lambda_{l-1} + b lambda_{l-2}
template <typename T, int NR, bool INJ>
__device__ __forceinline__ void step0(PairState<T, NR> &S, const typename VT<T>::C cf, int l) {
#pragma unroll
    for (int j = 0; j < NR; ++j) {
        rstep(S.a1[j], S.a2[j], cf.x, cf.y, S.u[j]);
        if (INJ) {
            if (l == S.ls[j]) {
                S.a2[j] = S.s0[j];
                S.a1[j] = S.s1[j];
            }
        }
    }
}

// spin 2: y+-_l = (alpha (1-u) +- beta) y+-_{l-1} - gamma y+-_{l-2}
template <typename T, int NR, bool INJ, typename C4>
__device__ __forceinline__ void step2(PairState<T, NR> &S, const C4 cf, int l) {
#pragma unroll
    for (int j = 0; j < NR; ++j) {
        const T tp = fma(-cf.x, S.u[j], cf.y);
        const T tm = fma(-cf.x, S.u[j], cf.z);
        const T pn = fma(tp, S.a1[j], -cf.w * S.a2[j]);
        const T mn = fma(tm, S.b1[j], -cf.w * S.b2[j]);
        S.a2[j] = S.a1[j];
        S.a1[j] = pn;
        S.b2[j] = S.b1[j];
        S.b1[j] = mn;
        if (INJ) {
            if (l == S.ls[j]) {
                S.a2[j] = S.s0[j];
                S.a1[j] = S.s1[j];
            }
            if (l == S.lsb[j]) {
                S.b2[j] = S.s2[j];
                S.b1[j] = S.s3[j];
            }
        }
    }
}

template <typename T, int NR, int SPIN, bool INJ>
__device__ __forceinline__ void stepx(PairState<T, NR> &S, const typename VT<T>::C *s_rec,
                                      const typename V4<T>::t *s_s2c, int i, int l) {
    if (SPIN == 2) step2<T, NR, INJ>(S, s_s2c[i], l);
    else step0<T, NR, INJ>(S, s_rec[i], l);
}

// CTA-wide minimum of the warps' start l (all threads must call).
__device__ __forceinline__ int cta_min(int v, int *s) {
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) s[w] = v;
    __syncthreads();
    int r = s[0];
#pragma unroll
    for (int i = 1; i < LEG_THREADS / 32; ++i) r = min(r, s[i]);
    __syncthreads();
    return r;
}

// =========================================================== synthesis
// The work of one CTA: ring-pair block bx, order m, map group bz.  Called by
// the plan's kernel (the three block indices) and by the grouped kernel
// (one work item of a list that spans several geometries).
template <typename T, int NR, int NM, int SPIN>
__device__ __forceinline__ void leg_synth_cta(const LegArgs<T> &a, const int bx, const int m, const int bz) {
    typedef typename VT<T>::C C;
    typedef typename V4<T>::t C4;
    constexpr int NA = (SPIN == 2) ? 2 * NM : NM;   // alm rows staged (E, B per map)
    constexpr int NACC = (SPIN == 2) ? 8 : 2;        // reals per parity class per map
    __shared__ C s_rec[LEG_CHUNK];
    __shared__ C4 s_s2c[SPIN == 2 ? LEG_CHUNK : 1];
    __shared__ C s_alm[NA][LEG_CHUNK];
    __shared__ int s_red[LEG_THREADS / 32];

    const int L = a.lmax;
    const int map0 = bz * NM;
    const int nm = min(NM, a.nmaps - map0);
    const int64_t base = (int64_t)m * (2 * L + 1 - m) / 2;

    PairState<T, NR> S;
    int warp_lo, warp_hi;
    load_pairs<T, NR, SPIN>(a, bx, m, S, warp_lo, warp_hi);
    const int lo = cta_min(warp_lo, s_red);

    T accE[NR][NM][NACC], accO[NR][NM][NACC];
#pragma unroll
    for (int j = 0; j < NR; ++j)
#pragma unroll
        for (int k = 0; k < NM; ++k)
#pragma unroll
            for (int q = 0; q < NACC; ++q) accE[j][k][q] = accO[j][k][q] = T(0);

    auto accumulate = [&](const int i, T(&acc)[NR][NM][NACC]) {
        if (SPIN == 0) {
#pragma unroll
            for (int k = 0; k < NM; ++k) {
                const C av = s_alm[k][i];
#pragma unroll
                for (int j = 0; j < NR; ++j) {
                    acc[j][k][0] = fma(S.a1[j], av.x, acc[j][k][0]);
                    acc[j][k][1] = fma(S.a1[j], av.y, acc[j][k][1]);
                }
            }
        } else {
#pragma unroll
            for (int j = 0; j < NR; ++j) {
                const T lw = S.a1[j] + S.b1[j], lx = S.a1[j] - S.b1[j];
#pragma unroll
                for (int k = 0; k < NM; ++k) {
                    const C e = s_alm[2 * k][i];
                    const C b = s_alm[2 * k + 1][i];
                    // W parts: Q = -E lw, U = -B lw ; X parts: Q = -i B lx, U = i E lx
                    acc[j][k][0] = fma(-e.x, lw, acc[j][k][0]);
                    acc[j][k][1] = fma(-e.y, lw, acc[j][k][1]);
                    acc[j][k][2] = fma(-b.x, lw, acc[j][k][2]);
                    acc[j][k][3] = fma(-b.y, lw, acc[j][k][3]);
                    acc[j][k][4] = fma(b.y, lx, acc[j][k][4]);
                    acc[j][k][5] = fma(-b.x, lx, acc[j][k][5]);
                    acc[j][k][6] = fma(-e.y, lx, acc[j][k][6]);
                    acc[j][k][7] = fma(e.x, lx, acc[j][k][7]);
                }
            }
        }
    };

    // rings with no significant l in this CTA still get their (zero) output
    for (int c0 = lo; c0 <= L; c0 += LEG_CHUNK) {
        const int c1 = min(c0 + LEG_CHUNK, L + 1);
        __syncthreads();
        for (int i = threadIdx.x; i < c1 - c0; i += LEG_THREADS) {
            const int l = c0 + i;
            const int64_t idx = base + l;
            if (SPIN == 2) s_s2c[i] = a.s2c[idx];
            else s_rec[i] = a.rec[idx];
            const T bm = a.beam ? a.beam[l] : T(1);
#pragma unroll
            for (int k = 0; k < NA; ++k) {
                C v = cplx(T(0), T(0));
                const int mk = (SPIN == 2) ? k / 2 : k;
                if (mk < nm) {
                    const int64_t row = (int64_t)(map0 + mk) * a.rs + ((SPIN == 2) ? (k & 1) : 0);
                    v = a.alm[row * a.nalm + idx];
                    if (m == 0) v.y = T(0);
                    v.x *= bm;
                    v.y *= bm;
                }
                s_alm[k][i] = v;
            }
        }
        __syncthreads();
        int l = max(c0, warp_lo);
        const int la_end = min(c1 - 1, warp_hi);
        for (; l <= la_end; ++l) {   // start states still being injected
            stepx<T, NR, SPIN, true>(S, s_rec, s_s2c, l - c0, l);
            if ((l - m) & 1) accumulate(l - c0, accO);
            else accumulate(l - c0, accE);
        }
        if (l < c1 && ((l - m) & 1)) {
            stepx<T, NR, SPIN, false>(S, s_rec, s_s2c, l - c0, l);
            accumulate(l - c0, accO);
            ++l;
        }
        for (; l + 1 < c1; l += 2) {
            stepx<T, NR, SPIN, false>(S, s_rec, s_s2c, l - c0, l);
            accumulate(l - c0, accE);
            stepx<T, NR, SPIN, false>(S, s_rec, s_s2c, l + 1 - c0, l + 1);
            accumulate(l + 1 - c0, accO);
        }
        if (l < c1) {
            stepx<T, NR, SPIN, false>(S, s_rec, s_s2c, l - c0, l);
            accumulate(l - c0, accE);
        }
    }

#pragma unroll
    for (int j = 0; j < NR; ++j) {
        const int pr = S.pr[j];
        if (pr >= a.npairs) continue;
        const int rn = pr, rs = a.nring - 1 - pr;
#pragma unroll
        for (int k = 0; k < NM; ++k) {
            if (k >= nm) break;
            if (SPIN == 0) {
                C *out = a.F + (int64_t)(map0 + k) * a.nring * (L + 1) + m;
                out[(int64_t)rn * (L + 1)] = cplx(accE[j][k][0] + accO[j][k][0], accE[j][k][1] + accO[j][k][1]);
                if (rs != rn)
                    out[(int64_t)rs * (L + 1)] = cplx(accE[j][k][0] - accO[j][k][0], accE[j][k][1] - accO[j][k][1]);
            } else {
                const T *E = accE[j][k], *O = accO[j][k];
                // north: W + X over both classes; south: even W - X, odd X - W
                C *oq = a.F + (int64_t)(2 * (map0 + k)) * a.nring * (L + 1) + m;
                C *ou = a.F + (int64_t)(2 * (map0 + k) + 1) * a.nring * (L + 1) + m;
                oq[(int64_t)rn * (L + 1)] = cplx(E[0] + O[0] + E[4] + O[4], E[1] + O[1] + E[5] + O[5]);
                ou[(int64_t)rn * (L + 1)] = cplx(E[2] + O[2] + E[6] + O[6], E[3] + O[3] + E[7] + O[7]);
                if (rs != rn) {
                    oq[(int64_t)rs * (L + 1)] = cplx(E[0] - O[0] - E[4] + O[4], E[1] - O[1] - E[5] + O[5]);
                    ou[(int64_t)rs * (L + 1)] = cplx(E[2] - O[2] - E[6] + O[6], E[3] - O[3] - E[7] + O[7]);
                }
            }
        }
    }
}

template <typename T, int NR, int NM, int SPIN>
__global__ void __launch_bounds__(LEG_THREADS) k_leg_synth(const LegArgs<T> a) {
    leg_synth_cta<T, NR, NM, SPIN>(a, blockIdx.x, blockIdx.y, blockIdx.z);
}

// =========================================================== analysis
// butterfly transpose-reduce of 8 values over the warp: afterwards every lane
// holds the warp sum of value index 4*b4 + 2*b3 + b2 (b = lane bits).
template <typename T>
__device__ __forceinline__ T treduce8(T (&v)[8], const int lane) {
    const bool b4 = (lane >> 4) & 1, b3 = (lane >> 3) & 1, b2 = (lane >> 2) & 1;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const T send = b4 ? v[i] : v[i + 4];
        const T keep = b4 ? v[i + 4] : v[i];
        v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const T send = b3 ? v[i] : v[i + 2];
        const T keep = b3 ? v[i + 2] : v[i];
        v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
    {
        const T send = b2 ? v[0] : v[1];
        const T keep = b2 ? v[1] : v[0];
        v[0] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
    }
    v[0] += __shfl_xor_sync(0xffffffffu, v[0], 2);
    v[0] += __shfl_xor_sync(0xffffffffu, v[0], 1);
    return v[0];
}

// The work of one CTA (as leg_synth_cta); single: the CTA covers every ring
// pair of its m, so it stores its sums instead of adding them atomically
template <typename T, int NR, int NM, int SPIN>
__device__ __forceinline__ void leg_analysis_cta(const LegArgs<T> &a, const int bx, const int m, const int bz,
                                                 const bool single) {
    typedef typename VT<T>::C C;
    typedef typename V4<T>::t C4;
    constexpr int NO = (SPIN == 2) ? 4 : 2;     // reals out per map per l (E, B or a)
    __shared__ C s_rec[LEG_CHUNK];
    __shared__ C4 s_s2c[SPIN == 2 ? LEG_CHUNK : 1];
    __shared__ int s_red[LEG_THREADS / 32];
    extern __shared__ unsigned char s_dyn[];
    T *s_acc = reinterpret_cast<T *>(s_dyn);     // [(lmax+1-m)][NM][NO]

    const int L = a.lmax;
    const int map0 = bz * NM;
    const int nm = min(NM, a.nmaps - map0);
    const int64_t base = (int64_t)m * (2 * L + 1 - m) / 2;
    const int nl = L + 1 - m;
    const int lane = threadIdx.x & 31;

    for (int i = threadIdx.x; i < nl * NM * NO; i += LEG_THREADS) s_acc[i] = T(0);

    PairState<T, NR> S;
    int warp_lo, warp_hi;
    load_pairs<T, NR, SPIN>(a, bx, m, S, warp_lo, warp_hi);

    // per-pair even / odd combinations of the north and south ring data
    T gE[NR][NM][2 * (NO / 2)], gO[NR][NM][2 * (NO / 2)];
#pragma unroll
    for (int j = 0; j < NR; ++j) {
        const int pr = S.pr[j];
        const bool ok = pr < a.npairs;
        const int rn = pr, rs = a.nring - 1 - pr;
#pragma unroll
        for (int k = 0; k < NM; ++k) {
#pragma unroll
            for (int c = 0; c < NO / 2; ++c) {
                C gn = cplx(T(0), T(0)), gs = cplx(T(0), T(0));
                if (ok && k < nm) {
                    const int row = (SPIN == 2) ? 2 * (map0 + k) + c : map0 + k;
                    const C *g = a.F + (int64_t)row * a.nring * (L + 1) + m;
                    gn = g[(int64_t)rn * (L + 1)];
                    if (rs != rn) gs = g[(int64_t)rs * (L + 1)];
                }
                // l - m even uses gE, odd gO; the l loop below runs over groups
                // of 8 starting at a multiple of 8, so (l - m) & 1 = (v & 1) ^ (m & 1):
                // for odd m the two sets swap once here and the parity of
                // every unrolled step is a compile-time constant
                const T sgn = (m & 1) ? T(-1) : T(1);
                gE[j][k][2 * c] = gn.x + sgn * gs.x;
                gE[j][k][2 * c + 1] = gn.y + sgn * gs.y;
                gO[j][k][2 * c] = gn.x - sgn * gs.x;
                gO[j][k][2 * c + 1] = gn.y - sgn * gs.y;
            }
        }
    }
    const int lo = cta_min(warp_lo, s_red) & ~7;
    if (lo <= L) {
        for (int c0 = lo; c0 <= L; c0 += LEG_CHUNK) {
            const int c1 = min(c0 + LEG_CHUNK, L + 1);
            __syncthreads();
            for (int i = threadIdx.x; i < c1 - c0; i += LEG_THREADS) {
                const int64_t idx = base + c0 + i;
                if (SPIN == 2) s_s2c[i] = (c0 + i >= m) ? a.s2c[idx] : C4();
                else s_rec[i] = (c0 + i >= m) ? a.rec[idx] : cplx(T(0), T(0));
            }
            __syncthreads();
            for (int g0 = c0; g0 < c1; g0 += 8) {
                if (g0 + 7 < warp_lo) continue;      // warp-uniform
                T part[NM][NO][8];
#pragma unroll
                for (int v = 0; v < 8; ++v) {
                    const int l = g0 + v;
                    const bool live = (l >= warp_lo) && (l < c1);
                    if (live) {
                        if (l <= warp_hi) stepx<T, NR, SPIN, true>(S, s_rec, s_s2c, l - c0, l);
                        else stepx<T, NR, SPIN, false>(S, s_rec, s_s2c, l - c0, l);
                    }
                    const bool odd = v & 1;   // (l - m) & 1 after the swap for odd m
#pragma unroll
                    for (int k = 0; k < NM; ++k)
#pragma unroll
                        for (int q = 0; q < NO; ++q) part[k][q][v] = T(0);
                    if (live) {
                        if (SPIN == 0) {
#pragma unroll
                            for (int j = 0; j < NR; ++j)
#pragma unroll
                                for (int k = 0; k < NM; ++k) {
                                    const T gr = odd ? gO[j][k][0] : gE[j][k][0];
                                    const T gi = odd ? gO[j][k][1] : gE[j][k][1];
                                    part[k][0][v] = fma(S.a1[j], gr, part[k][0][v]);
                                    part[k][1][v] = fma(S.a1[j], gi, part[k][1][v]);
                                }
                        } else {
#pragma unroll
                            for (int j = 0; j < NR; ++j) {
                                const T lw = S.a1[j] + S.b1[j], lx = S.a1[j] - S.b1[j];
#pragma unroll
                                for (int k = 0; k < NM; ++k) {
                                    // even: W-terms use (Q_N + Q_S, U_N + U_S), X-terms the odd sums
                                    const T *gw = odd ? gO[j][k] : gE[j][k];
                                    const T *gx = odd ? gE[j][k] : gO[j][k];
                                    // E^ += -lw GQ - i lx GU ; B^ += i lx GQ - lw GU
                                    part[k][0][v] = fma(-lw, gw[0], fma(lx, gx[3], part[k][0][v]));
                                    part[k][1][v] = fma(-lw, gw[1], fma(-lx, gx[2], part[k][1][v]));
                                    part[k][2][v] = fma(-lw, gw[2], fma(-lx, gx[1], part[k][2][v]));
                                    part[k][3][v] = fma(-lw, gw[3], fma(lx, gx[0], part[k][3][v]));
                                }
                            }
                        }
                    }
                }
                const int vsel = 4 * ((lane >> 4) & 1) + 2 * ((lane >> 3) & 1) + ((lane >> 2) & 1);
                const int l = g0 + vsel;
#pragma unroll
                for (int k = 0; k < NM; ++k)
#pragma unroll
                    for (int q = 0; q < NO; ++q) {
                        const T r = treduce8<T>(part[k][q], lane);
                        if ((lane & 3) == 0 && l >= m && l <= L && k < nm)
                            atomicAdd(&s_acc[((l - m) * NM + k) * NO + q], r);
                    }
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nl * nm; i += LEG_THREADS) {
        const int li = i / nm, k = i % nm;
        const int l = m + li;
        const T bm = (a.beam ? a.beam[l] : T(1)) * ((a.vjp && m > 0) ? T(2) : T(1));
#pragma unroll
        for (int c = 0; c < NO / 2; ++c) {
            T re = s_acc[(li * NM + k) * NO + 2 * c] * bm;
            T im = (m == 0) ? T(0) : s_acc[(li * NM + k) * NO + 2 * c + 1] * bm;
            const int64_t row = (int64_t)(map0 + k) * a.rs + c;
            C *dst = const_cast<C *>(a.alm) + row * a.nalm + base + l;
            if (single) {
                *dst = cplx(re, im);
            } else {
                atomicAdd(&dst->x, re);
                atomicAdd(&dst->y, im);
            }
        }
    }
}

template <typename T, int NR, int NM, int SPIN>
__global__ void __launch_bounds__(LEG_THREADS) k_leg_analysis(const LegArgs<T> a) {
    leg_analysis_cta<T, NR, NM, SPIN>(a, blockIdx.x, blockIdx.y, blockIdx.z, gridDim.x == 1);
}

// ======================================================= grouped launches
// One launch over the CTAs of several plans (chains of different N_side and
// l_max): entry g holds one plan's arguments (the launcher orders them by
// decreasing l_max); flat CTA i belongs to the entry with first[g] <= i <
// first[g+1]; within an entry the CTA index runs over (ring-pair block, m,
// map group), ring-pair blocks fastest and m ascending, so the long low-m
// recurrences start first.  An entry whose device flag *active[g] is 0 (a
// null pointer: always active) is skipped.
template <typename T> struct LegGroups {
    int ng;
    int first[SHTG_MAX_GROUPS + 1];
    int gx[SHTG_MAX_GROUPS];     // ring-pair blocks of the group
    int gy[SHTG_MAX_GROUPS];     // orders m of the group (l_max + 1)
    const int *active[SHTG_MAX_GROUPS];
    LegArgs<T> a[SHTG_MAX_GROUPS];
};

__device__ __forceinline__ int group_of(const int *first, const int ng, const int i) {
    int g = 0;
    while (g + 1 < ng && i >= first[g + 1]) ++g;
    return g;
}

template <typename T, int NR, int NM, int SPIN>
__global__ void __launch_bounds__(LEG_THREADS) k_leg_synth_grp(const __grid_constant__ LegGroups<T> G) {
    const int i = blockIdx.x;
    const int g = group_of(G.first, G.ng, i);
    if (G.active[g] && *G.active[g] == 0) return;
    const int li = i - G.first[g], t = li / G.gx[g];
    leg_synth_cta<T, NR, NM, SPIN>(G.a[g], li % G.gx[g], t % G.gy[g], t / G.gy[g]);
}

template <typename T, int NR, int NM, int SPIN>
__global__ void __launch_bounds__(LEG_THREADS) k_leg_analysis_grp(const __grid_constant__ LegGroups<T> G) {
    const int i = blockIdx.x;
    const int g = group_of(G.first, G.ng, i);
    if (G.active[g] && *G.active[g] == 0) return;
    const int li = i - G.first[g], t = li / G.gx[g];
    leg_analysis_cta<T, NR, NM, SPIN>(G.a[g], li % G.gx[g], t % G.gy[g], t / G.gy[g], G.gx[g] == 1);
}

// ====================================================== preconditioner
// diag_lm = sum_pairs wpair_r g_lm(theta_r), g = lambda^2 (spin 0) or
// lw^2 + lx^2 (spin 2); g has the same value on both rings of a pair.
template <int NR, int SPIN>
__global__ void __launch_bounds__(LEG_THREADS) k_leg_diag(const LegArgs<float> a) {
    __shared__ float2 s_rec[LEG_CHUNK];
    __shared__ float4 s_s2c[LEG_CHUNK];
    __shared__ int s_red[LEG_THREADS / 32];
    extern __shared__ unsigned char s_dyn[];
    float *s_acc = reinterpret_cast<float *>(s_dyn);
    const int m = blockIdx.y;
    const int L = a.lmax;
    const int64_t base = (int64_t)m * (2 * L + 1 - m) / 2;
    const int nl = L + 1 - m;
    const int lane = threadIdx.x & 31;
    for (int i = threadIdx.x; i < nl; i += LEG_THREADS) s_acc[i] = 0.f;
    PairState<float, NR> S;
    int warp_lo, warp_hi;
    load_pairs<float, NR, SPIN>(a, blockIdx.x, m, S, warp_lo, warp_hi);
    float w[NR];
#pragma unroll
    for (int j = 0; j < NR; ++j) w[j] = S.pr[j] < a.npairs ? a.wpair[S.pr[j]] : 0.f;
    const int lo = cta_min(warp_lo, s_red) & ~7;
    if (lo <= L) {
        for (int c0 = lo; c0 <= L; c0 += LEG_CHUNK) {
            const int c1 = min(c0 + LEG_CHUNK, L + 1);
            __syncthreads();
            for (int i = threadIdx.x; i < c1 - c0; i += LEG_THREADS) {
                const int64_t idx = base + c0 + i;
                if (SPIN == 2) s_s2c[i] = (c0 + i >= m) ? a.s2c[idx] : make_float4(0.f, 0.f, 0.f, 0.f);
                else s_rec[i] = (c0 + i >= m) ? a.rec[idx] : make_float2(0.f, 0.f);
            }
            __syncthreads();
            for (int g0 = c0; g0 < c1; g0 += 8) {
                if (g0 + 7 < warp_lo) continue;
                float part[8];
#pragma unroll
                for (int v = 0; v < 8; ++v) {
                    const int l = g0 + v;
                    part[v] = 0.f;
                    if (l >= warp_lo && l < c1) {
                        if (l <= warp_hi) stepx<float, NR, SPIN, true>(S, s_rec, s_s2c, l - c0, l);
                        else stepx<float, NR, SPIN, false>(S, s_rec, s_s2c, l - c0, l);
#pragma unroll
                        for (int j = 0; j < NR; ++j) {
                            // spin 2: lw^2 + lx^2 = 2 (y+^2 + y-^2)
                            const float g = (SPIN == 0) ? S.a1[j] * S.a1[j]
                                                        : 2.f * (S.a1[j] * S.a1[j] + S.b1[j] * S.b1[j]);
                            part[v] = fmaf(w[j], g, part[v]);
                        }
                    }
                }
                const int vsel = 4 * ((lane >> 4) & 1) + 2 * ((lane >> 3) & 1) + ((lane >> 2) & 1);
                const int l = g0 + vsel;
                const float r = treduce8<float>(part, lane);
                if ((lane & 3) == 0 && l >= m && l <= L) atomicAdd(&s_acc[l - m], r);
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nl; i += LEG_THREADS) {
        float *dst = a.diag + base + m + i;
        if (gridDim.x == 1) *dst = s_acc[i];
        else atomicAdd(dst, s_acc[i]);
    }
}

// ============================================================ launchers
template <typename T> LegArgs<T> leg_make_args(Plan *p);
template <> LegArgs<float> leg_make_args<float>(Plan *p);
template <> LegArgs<double> leg_make_args<double>(Plan *p);

template <typename T, int SPIN, int NR, int NM>
int launch_synth_v(Plan *p, const typename VT<T>::C *alm, int rs, int nmaps, const T *beam,
                   typename VT<T>::C *F, cudaStream_t st) {
    LegArgs<T> a = leg_make_args<T>(p);
    a.alm = alm;
    a.rs = rs;
    a.F = F;
    a.beam = beam;
    a.nmaps = nmaps;
    dim3 grid((p->npairs + LEG_THREADS * NR - 1) / (LEG_THREADS * NR), p->lmax + 1,
              (nmaps + NM - 1) / NM);
    prof_begin(p, sizeof(T) == 8 ? K_LEG_SYN64 : K_LEG_SYN32, st);
    k_leg_synth<T, NR, NM, SPIN><<<grid, LEG_THREADS, 0, st>>>(a);
    prof_end(p, st);
    SHTG_CHECK_LAUNCH("k_leg_synth");
    return SHTG_OK;
}

template <typename T, int SPIN, int NR, int NM>
int launch_analysis_v(Plan *p, const typename VT<T>::C *G, int nmaps, const T *beam,
                      typename VT<T>::C *alm, int rs, cudaStream_t st, int vjp) {
    constexpr int NO = (SPIN == 2) ? 4 : 2;
    LegArgs<T> a = leg_make_args<T>(p);
    a.alm = alm;
    a.rs = rs;
    a.vjp = vjp;
    a.F = const_cast<typename VT<T>::C *>(G);
    a.beam = beam;
    a.nmaps = nmaps;
    const int gx = (p->npairs + LEG_THREADS * NR - 1) / (LEG_THREADS * NR);
    const int comps = (SPIN == 2) ? 2 : 1;
    if (gx > 1) {
        const size_t cs = sizeof(typename VT<T>::C) * (size_t)p->nalm;
        SHTG_CUDA(cudaMemset2DAsync(alm, cs * rs, 0, cs * comps, nmaps, st));
    }
    const size_t smem = sizeof(T) * (size_t)(p->lmax + 1) * NM * NO;
    auto kern = k_leg_analysis<T, NR, NM, SPIN>;
    if (smem > 48 * 1024) SHTG_CUDA(allow_max_smem(kern));
    dim3 grid(gx, p->lmax + 1, (nmaps + NM - 1) / NM);
    prof_begin(p, sizeof(T) == 8 ? K_LEG_ANA64 : K_LEG_ANA32, st);
    kern<<<grid, LEG_THREADS, smem, st>>>(a);
    prof_end(p, st);
    SHTG_CHECK_LAUNCH("k_leg_analysis");
    return SHTG_OK;
}

// variant tables (one per precision translation unit)
typedef int (*SynthFn32)(Plan *, const float2 *, int, int, const float *, float2 *, cudaStream_t);
typedef int (*SynthFn64)(Plan *, const double2 *, int, int, const double *, double2 *, cudaStream_t);
typedef int (*AnaFn32)(Plan *, const float2 *, int, const float *, float2 *, int, cudaStream_t, int);
typedef int (*AnaFn64)(Plan *, const double2 *, int, const double *, double2 *, int, cudaStream_t, int);
struct Variants32 {
    int n[4];                // synth0, synth2, ana0, ana2
    SynthFn32 syn[2][8];
    AnaFn32 ana[2][8];
    int shape[4][8][2];      // (NR, NM) per variant, for reporting
};
struct Variants64 {
    int n[4];
    SynthFn64 syn[2][8];
    AnaFn64 ana[2][8];
    int shape[4][8][2];
};
const Variants32 &variants32();
const Variants64 &variants64();

}  // namespace shtg

// FP64-accurate Legendre sums in double-FP32 arithmetic (df.cuh).
//
// The same sums as the FP64 kernels: synthesis F_r(m) = sum_l a_lm
// lambda_lm(theta_r) with the even / odd split of App. A, and the transpose
// c_lm = sum_r lambda_lm(theta_r) G_r(m).  Inputs and outputs stay FP64 in
// HBM (the plan's FP64 recurrence coefficients, start states and tile
// states, FP64 alm and ring data); values are rounded to df when they are
// staged, and every multiply-add of the recurrence and the contraction runs
// in df on the FP32 pipe.  GB300 issues 64 FP32 operations per FP64
// operation, and a df multiply-add costs about twelve, so the FP64-accurate
// transforms (RHS and residual replacements of the mixed solver, the
// SHTG_DF64 transforms) leave the narrow FP64 pipe.  Rounding: ~2^-47
// relative per operation against 2^-53 for FP64; the recurrence carries O(l)
// of them, far below the 1e-10 the FP64 transforms are held to.
//
// Synthesis: one thread per ring pair (NR of them) and NM maps, as the
// CUDA-core kernels, the recurrence in registers.  Transpose: the
// register-blocked contraction of the FP64 transpose (legendre_g64.cu) with
// stages of 32 ring pairs, whose recurrences all four warps generate in
// 32-l segments from the plan's FP64 tile states (every SHTG_TS64 l).
#include "df.cuh"
#include "legendre_kernels.cuh"

namespace shtg {
namespace {

struct __align__(16) dfc2 {   // spin-0 coefficients (a, b)
    df a, b;
};
struct __align__(16) dfc4 {   // spin-2 coefficients (alpha, alpha + beta, alpha - beta, gamma)
    df x, y, z, w;
};

__device__ __forceinline__ dfc2 dfc2_from(double2 v) {
    dfc2 r;
    r.a = df_from(v.x);
    r.b = df_from(v.y);
    return r;
}
__device__ __forceinline__ dfc4 dfc4_from(double4_32a v) {
    dfc4 r;
    r.x = df_from(v.x);
    r.y = df_from(v.y);
    r.z = df_from(v.z);
    r.w = df_from(v.w);
    return r;
}

template <int NR> struct DfPair {
    int pr[NR];
    df u[NR];   // u = 1 - cos theta
    int ls[NR], lsb[NR];
    df s0[NR], s1[NR], s2[NR], s3[NR];
    df a1[NR], a2[NR], b1[NR], b2[NR];
};

template <int NR>
__device__ __forceinline__ void df_pair_reset(DfPair<NR> &S, int j, int L) {
    S.a1[j] = S.a2[j] = S.b1[j] = S.b2[j] = df_zero();
    S.s0[j] = S.s1[j] = S.s2[j] = S.s3[j] = df_zero();
    S.u[j] = df_make(1.f, 0.f);
    S.ls[j] = S.lsb[j] = L + 1;
}

// geometry and FP64 start states of ring pair pr for m, rounded to df
template <int NR, int SPIN>
__device__ __forceinline__ void df_pair_load(const LegArgs<double> &a, int m, int pr, DfPair<NR> &S, int j) {
    S.pr[j] = pr;
    df_pair_reset(S, j, a.lmax);
    if (pr >= a.npairs) return;
    const double u = a.u[pr];
    S.u[j] = df_from(u);
    const int64_t o = (int64_t)m * a.npairs + pr;
    if (SPIN == 2) {
        const int2 q = a.ls2[o];
        S.ls[j] = q.x;
        S.lsb[j] = q.y;
        const double4_32a s = a.st2[o];
        S.s0[j] = df_from(s.x);
        S.s1[j] = df_from(s.y);
        S.s2[j] = df_from(s.z);
        S.s3[j] = df_from(s.w);
    } else {
        S.ls[j] = a.ls[o];
        const double2 s = a.st[o];
        S.s0[j] = df_from(s.x);
        S.s1[j] = df_from(s.y);
    }
}

// spin 0: lambda_l = a (1 - u) lambda_{l-1} + b lambda_{l-2}, formed as
// t + b lambda_{l-2} - t u with t = a lambda_{l-1} (as the FP64 kernels do):
// near the poles u ~ 1e-6 keeps its full relative precision, which a
// rounded cos(theta) = 1 - u would not (2^-48 absolute on cos(theta) is
// 1e-8 relative on u at the first HEALPix ring of N_side 1024)
template <int NR, bool INJ>
__device__ __forceinline__ void df_step0(DfPair<NR> &S, const dfc2 cf, int l) {
#pragma unroll
    for (int j = 0; j < NR; ++j) {
        const df t = df_mul(cf.a, S.a1[j]);
        const df n = df_sub(df_add(t, df_mul(cf.b, S.a2[j])), df_mul(t, S.u[j]));
        S.a2[j] = S.a1[j];
        S.a1[j] = n;
        if (INJ && l == S.ls[j]) {
            S.a2[j] = S.s0[j];
            S.a1[j] = S.s1[j];
        }
    }
}

// spin 2: y+-_l = ((alpha + -beta) - alpha u) y+-_{l-1} - gamma y+-_{l-2}
template <int NR, bool INJ>
__device__ __forceinline__ void df_step2(DfPair<NR> &S, const dfc4 cf, int l) {
#pragma unroll
    for (int j = 0; j < NR; ++j) {
        const df au = df_mul(cf.x, S.u[j]);
        const df tp = df_sub(cf.y, au), tm = df_sub(cf.z, au);
        const df pn = df_sub(df_mul(tp, S.a1[j]), df_mul(cf.w, S.a2[j]));
        const df mn = df_sub(df_mul(tm, S.b1[j]), df_mul(cf.w, S.b2[j]));
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

template <int NR, int SPIN, bool INJ>
__device__ __forceinline__ void df_stepx(DfPair<NR> &S, const dfc2 *s_rec, const dfc4 *s_s2c, int i, int l) {
    if (SPIN == 2) df_step2<NR, INJ>(S, s_s2c[i], l);
    else df_step0<NR, INJ>(S, s_rec[i], l);
}

// =========================================================== synthesis
template <int NR, int NM, int SPIN>
__global__ void __launch_bounds__(LEG_THREADS) k_leg_synth_df(const LegArgs<double> a) {
    constexpr int NA = (SPIN == 2) ? 2 * NM : NM;   // alm rows staged (E, B per map)
    constexpr int NACC = (SPIN == 2) ? 8 : 2;        // reals per parity class per map
    __shared__ dfc2 s_rec[SPIN == 2 ? 1 : LEG_CHUNK];
    __shared__ dfc4 s_s2c[SPIN == 2 ? LEG_CHUNK : 1];
    __shared__ dfc s_alm[NA][LEG_CHUNK];
    __shared__ int s_red[LEG_THREADS / 32];

    const int m = blockIdx.y;
    const int L = a.lmax;
    const int map0 = blockIdx.z * NM;
    const int nm = min(NM, a.nmaps - map0);
    const int64_t base = (int64_t)m * (2 * L + 1 - m) / 2;

    DfPair<NR> S;
    int lo = L + 1, hi = -1;
#pragma unroll
    for (int j = 0; j < NR; ++j) {
        df_pair_load<NR, SPIN>(a, m, blockIdx.x * (LEG_THREADS * NR) + j * LEG_THREADS + threadIdx.x, S, j);
        lo = min(lo, min(S.ls[j], S.lsb[j]));
        if (S.ls[j] <= L) hi = max(hi, S.ls[j]);
        if (S.lsb[j] <= L) hi = max(hi, S.lsb[j]);
    }
    const int warp_lo = __reduce_min_sync(0xffffffffu, lo);
    const int warp_hi = __reduce_max_sync(0xffffffffu, hi);
    const int clo = cta_min(warp_lo, s_red);

    dfacc accE[NR][NM][NACC], accO[NR][NM][NACC];
#pragma unroll
    for (int j = 0; j < NR; ++j)
#pragma unroll
        for (int k = 0; k < NM; ++k)
#pragma unroll
            for (int q = 0; q < NACC; ++q) {
                df_acc_zero(accE[j][k][q]);
                df_acc_zero(accO[j][k][q]);
            }

    auto accumulate = [&](const int i, dfacc(&acc)[NR][NM][NACC]) {
        if (SPIN == 0) {
#pragma unroll
            for (int k = 0; k < NM; ++k) {
                const dfc av = s_alm[k][i];
#pragma unroll
                for (int j = 0; j < NR; ++j) {
                    df_fma(acc[j][k][0], S.a1[j], av.re);
                    df_fma(acc[j][k][1], S.a1[j], av.im);
                }
            }
        } else {
#pragma unroll
            for (int j = 0; j < NR; ++j) {
                const df lw = df_add(S.a1[j], S.b1[j]), lx = df_sub(S.a1[j], S.b1[j]);
                const df nlw = df_neg(lw), nlx = df_neg(lx);
#pragma unroll
                for (int k = 0; k < NM; ++k) {
                    const dfc e = s_alm[2 * k][i];
                    const dfc b = s_alm[2 * k + 1][i];
                    // W parts: Q = -E lw, U = -B lw ; X parts: Q = -i B lx, U = i E lx
                    df_fma(acc[j][k][0], nlw, e.re);
                    df_fma(acc[j][k][1], nlw, e.im);
                    df_fma(acc[j][k][2], nlw, b.re);
                    df_fma(acc[j][k][3], nlw, b.im);
                    df_fma(acc[j][k][4], lx, b.im);
                    df_fma(acc[j][k][5], nlx, b.re);
                    df_fma(acc[j][k][6], nlx, e.im);
                    df_fma(acc[j][k][7], lx, e.re);
                }
            }
        }
    };
    auto renorm = [&]() {
#pragma unroll
        for (int j = 0; j < NR; ++j)
#pragma unroll
            for (int k = 0; k < NM; ++k)
#pragma unroll
                for (int q = 0; q < NACC; ++q) {
                    df_acc_norm(accE[j][k][q]);
                    df_acc_norm(accO[j][k][q]);
                }
    };

    for (int c0 = clo; c0 <= L; c0 += LEG_CHUNK) {
        const int c1 = min(c0 + LEG_CHUNK, L + 1);
        __syncthreads();
        for (int i = threadIdx.x; i < c1 - c0; i += LEG_THREADS) {
            const int l = c0 + i;
            const int64_t idx = base + l;
            if (SPIN == 2) s_s2c[i] = dfc4_from(a.s2c[idx]);
            else s_rec[i] = dfc2_from(a.rec[idx]);
            const double bm = a.beam ? a.beam[l] : 1.0;
#pragma unroll
            for (int k = 0; k < NA; ++k) {
                double2 v = make_double2(0.0, 0.0);
                const int mk = (SPIN == 2) ? k / 2 : k;
                if (mk < nm) {
                    const int64_t row = (int64_t)(map0 + mk) * a.rs + ((SPIN == 2) ? (k & 1) : 0);
                    v = a.alm[row * a.nalm + idx];
                    if (m == 0) v.y = 0.0;
                    v.x *= bm;
                    v.y *= bm;
                }
                dfc d;
                d.re = df_from(v.x);
                d.im = df_from(v.y);
                s_alm[k][i] = d;
            }
        }
        __syncthreads();
        int l = max(c0, warp_lo);
        const int la_end = min(c1 - 1, warp_hi);
        for (; l <= la_end; ++l) {   // start states still being injected
            df_stepx<NR, SPIN, true>(S, s_rec, s_s2c, l - c0, l);
            if ((l - m) & 1) accumulate(l - c0, accO);
            else accumulate(l - c0, accE);
        }
        if (l < c1 && ((l - m) & 1)) {
            df_stepx<NR, SPIN, false>(S, s_rec, s_s2c, l - c0, l);
            accumulate(l - c0, accO);
            ++l;
        }
        for (; l + 1 < c1; l += 2) {
            df_stepx<NR, SPIN, false>(S, s_rec, s_s2c, l - c0, l);
            accumulate(l - c0, accE);
            df_stepx<NR, SPIN, false>(S, s_rec, s_s2c, l + 1 - c0, l + 1);
            accumulate(l + 1 - c0, accO);
        }
        if (l < c1) {
            df_stepx<NR, SPIN, false>(S, s_rec, s_s2c, l - c0, l);
            accumulate(l - c0, accE);
        }
        renorm();   // at most 64 terms per class since the last one
    }

#pragma unroll
    for (int j = 0; j < NR; ++j) {
        const int pr = S.pr[j];
        if (pr >= a.npairs) continue;
        const int rn = pr, rs = a.nring - 1 - pr;
#pragma unroll
        for (int k = 0; k < NM; ++k) {
            if (k >= nm) break;
            double E[NACC], O[NACC];
#pragma unroll
            for (int q = 0; q < NACC; ++q) {
                E[q] = df_acc_to(accE[j][k][q]);
                O[q] = df_acc_to(accO[j][k][q]);
            }
            if (SPIN == 0) {
                double2 *out = a.F + (int64_t)(map0 + k) * a.nring * (L + 1) + m;
                out[(int64_t)rn * (L + 1)] = make_double2(E[0] + O[0], E[1] + O[1]);
                if (rs != rn) out[(int64_t)rs * (L + 1)] = make_double2(E[0] - O[0], E[1] - O[1]);
            } else {
                // north: W + X over both classes; south: even W - X, odd X - W
                double2 *oq = a.F + (int64_t)(2 * (map0 + k)) * a.nring * (L + 1) + m;
                double2 *ou = a.F + (int64_t)(2 * (map0 + k) + 1) * a.nring * (L + 1) + m;
                oq[(int64_t)rn * (L + 1)] = make_double2(E[0] + O[0] + E[4] + O[4], E[1] + O[1] + E[5] + O[5]);
                ou[(int64_t)rn * (L + 1)] = make_double2(E[2] + O[2] + E[6] + O[6], E[3] + O[3] + E[7] + O[7]);
                if (rs != rn) {
                    oq[(int64_t)rs * (L + 1)] = make_double2(E[0] - O[0] - E[4] + O[4], E[1] - O[1] - E[5] + O[5]);
                    ou[(int64_t)rs * (L + 1)] = make_double2(E[2] - O[2] - E[6] + O[6], E[3] - O[3] - E[7] + O[7]);
                }
            }
        }
    }
}

// =========================================================== transpose
constexpr int D_LR = 128;   // l per CTA (rows): four 32-l segments, one per warp
constexpr int D_KP = 32;    // ring pairs per stage (a warp's lanes)
constexpr int D_NT = 128;   // threads
constexpr int D_NMT = 8;    // maps per CTA (grid.z covers more)
constexpr int D_LS = D_KP + 1;   // row stride of the value tile (odd: rows in distinct banks)
constexpr int D_GS = 9;          // map stride of the ring-data sets

template <int SPIN> struct DfT {
    static constexpr int NV = SPIN == 2 ? 2 : 1;   // value tiles: lambda, or (lw, lx)
    static constexpr int NO = SPIN == 2 ? 4 : 2;   // outputs per map
    static constexpr int COEF = SPIN == 2 ? 32 : 16;
    static constexpr int LAM = 0;
    static constexpr int GSET = LAM + NV * D_LR * D_LS * 8;
    static constexpr int CO = GSET + D_KP * D_NMT * D_GS * 8;
    static constexpr int RED = CO + D_LR * COEF;
    static constexpr int BYTES = RED + 16;
};

template <int SPIN>
__global__ void __launch_bounds__(D_NT) k_leg_analysis_df(const LegArgs<double> a) {
    typedef DfT<SPIN> Ly;
    constexpr int NO = Ly::NO;
    extern __shared__ __align__(16) unsigned char smem[];
    df *lam = reinterpret_cast<df *>(smem + Ly::LAM);      // [NV][D_LR][D_LS]
    df *gset = reinterpret_cast<df *>(smem + Ly::GSET);    // [D_KP][D_NMT][D_GS]
    dfc2 *s_rec = reinterpret_cast<dfc2 *>(smem + Ly::CO);
    dfc4 *s_s2c = reinterpret_cast<dfc4 *>(smem + Ly::CO);
    int *s_first = reinterpret_cast<int *>(smem + Ly::RED);

    const int tid = threadIdx.x;
    const int m = blockIdx.y;
    const int L = a.lmax;
    const int lbase = m + blockIdx.x * D_LR;
    if (lbase > L) return;
    const int lend = min(L, lbase + D_LR - 1);
    const int map0 = blockIdx.z * D_NMT;
    const int nm = min(D_NMT, a.nmaps - map0);
    const int64_t base = (int64_t)m * (2 * L + 1 - m) / 2;
    const int64_t rowsz = (int64_t)a.nring * (L + 1);

    for (int i = tid; i < D_LR; i += D_NT) {
        const int l = lbase + i;
        const bool in = l <= L;
        if (SPIN == 2) s_s2c[i] = dfc4_from(in ? a.s2c[base + l] : make_double4_32a(0.0, 0.0, 0.0, 0.0));
        else s_rec[i] = dfc2_from(in ? a.rec[base + l] : make_double2(0.0, 0.0));
    }
    // first ring pair whose recurrence starts at or before lend (later pairs
    // without significant values add exact zeros)
    if (tid == 0) *s_first = a.npairs;
    __syncthreads();
    for (int pr = tid; pr < a.npairs; pr += D_NT) {
        const int64_t o = (int64_t)m * a.npairs + pr;
        int lsp;
        if (SPIN == 2) {
            const int2 q = a.ls2[o];
            lsp = min(q.x, q.y);
        } else {
            lsp = a.ls[o];
        }
        if (lsp <= lend) {
            atomicMin(s_first, pr);
            break;
        }
    }
    __syncthreads();
    const int s0 = *s_first / D_KP;
    const int nps = (a.npairs + D_KP - 1) / D_KP;

    // this thread's outputs: map k, class c, rows i = c + 2 (rg + 8 j)
    const int k = tid & 7, c = (tid >> 3) & 1, rg = tid >> 4;
    dfacc acc[8][NO];
#pragma unroll
    for (int j = 0; j < 8; ++j)
#pragma unroll
        for (int q = 0; q < NO; ++q) df_acc_zero(acc[j][q]);

    for (int s = s0; s < nps; ++s) {
        __syncthreads();   // the previous stage's tiles are consumed
        {
            // ---- recurrences of the stage's 32 ring pairs: warp w runs rows
            // 32 w .. 32 w + 31 of pair s * 32 + lane from the FP64 state
            // tabulated at l0 = lbase + 32 w
            const int pp = tid & 31, seg = tid >> 5;
            const int pr = s * D_KP + pp;
            const int l0 = lbase + 32 * seg;
            DfPair<1> S;
            df_pair_load<1, SPIN>(a, m, pr, S, 0);
            const bool live = pr < a.npairs && l0 <= L;
            if (live) {
                const int64_t e = (a.toff64[m] + (l0 - m) / SHTG_TS64) * a.npairs + pr;
                if (SPIN == 2) {
                    const double4_32a t4 = a.tst64_2[e];
                    S.a1[0] = df_from(t4.x);
                    S.a2[0] = df_from(t4.y);
                    S.b1[0] = df_from(t4.z);
                    S.b2[0] = df_from(t4.w);
                } else {
                    const double2 t2 = a.tst64_0[e];
                    S.a1[0] = df_from(t2.x);
                    S.a2[0] = df_from(t2.y);
                }
            }
            // injection steps only if some pair of the warp starts in this segment
            const bool inj = __any_sync(0xffffffffu, live && ((S.ls[0] >= l0 && S.ls[0] < l0 + 32) ||
                                                              (SPIN == 2 && S.lsb[0] >= l0 && S.lsb[0] < l0 + 32)));
            for (int i = 32 * seg; i < 32 * seg + 32; ++i) {
                df v0 = df_zero(), v1 = df_zero();
                if (live) {
                    if (inj) df_stepx<1, SPIN, true>(S, s_rec, s_s2c, i, lbase + i);
                    else df_stepx<1, SPIN, false>(S, s_rec, s_s2c, i, lbase + i);
                    if (SPIN == 2) {
                        v0 = df_add(S.a1[0], S.b1[0]);
                        v1 = df_sub(S.a1[0], S.b1[0]);
                    } else {
                        v0 = S.a1[0];
                    }
                }
                lam[i * D_LS + pp] = v0;
                if (SPIN == 2) lam[D_LR * D_LS + i * D_LS + pp] = v1;
            }
        }
        // ---- ring data of the stage: per (pair, map) the even / odd sets
        for (int it = tid; it < D_KP * D_NMT; it += D_NT) {
            const int pp = it >> 3, kk = it & 7;
            const int pr = s * D_KP + pp;
            df *g = gset + (pp * D_NMT + kk) * D_GS;
            double2 z[4] = {make_double2(0.0, 0.0), make_double2(0.0, 0.0), make_double2(0.0, 0.0),
                            make_double2(0.0, 0.0)};
            if (pr < a.npairs && kk < nm) {
                const int rn = pr, rs = a.nring - 1 - pr;
                const int nrow = SPIN == 2 ? 2 : 1;
                for (int cc = 0; cc < nrow; ++cc) {
                    const int64_t row = SPIN == 2 ? 2 * (map0 + kk) + cc : map0 + kk;
                    const double2 *gr = a.F + row * rowsz + m;
                    const double2 gn = gr[(int64_t)rn * (L + 1)];
                    const double2 gs = rs != rn ? gr[(int64_t)rs * (L + 1)] : make_double2(0.0, 0.0);
                    z[2 * cc] = make_double2(gn.x + gs.x, gn.y + gs.y);       // even set
                    z[2 * cc + 1] = make_double2(gn.x - gs.x, gn.y - gs.y);   // odd set
                }
            }
            // spin 0: [E re, E im, O re, O im]; spin 2: [QE re, QE im, QO re, QO im, UE re, UE im, UO re, UO im]
            for (int q = 0; q < (SPIN == 2 ? 4 : 2); ++q) {
                g[2 * q] = df_from(z[q].x);
                g[2 * q + 1] = df_from(z[q].y);
            }
        }
        __syncthreads();
        // ---- contraction over the stage's ring pairs
#pragma unroll 2
        for (int p = 0; p < D_KP; ++p) {
            const df *g = gset + (p * D_NMT + k) * D_GS;
            if (SPIN == 0) {
                const df gre = g[2 * c], gim = g[2 * c + 1];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const df lv = lam[(c + 2 * (rg + 8 * j)) * D_LS + p];
                    df_fma(acc[j][0], lv, gre);
                    df_fma(acc[j][1], lv, gim);
                }
            } else {
                // lw terms take the row's set, lx terms the other one:
                //   E^ = -lw G_Q - i lx G_U,  B^ = i lx G_Q - lw G_U
                const df qr = g[2 * c], qi = g[2 * c + 1], ur = g[4 + 2 * c], ui = g[4 + 2 * c + 1];
                const df xqr = g[2 * (1 - c)], xqi = g[2 * (1 - c) + 1], xur = g[4 + 2 * (1 - c)],
                         xui = g[4 + 2 * (1 - c) + 1];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int i = c + 2 * (rg + 8 * j);
                    const df lw = lam[i * D_LS + p], lx = lam[D_LR * D_LS + i * D_LS + p];
                    const df nlw = df_neg(lw), nlx = df_neg(lx);
                    df_fma(acc[j][0], lx, xui);
                    df_fma(acc[j][0], nlw, qr);
                    df_fma(acc[j][1], nlx, xur);
                    df_fma(acc[j][1], nlw, qi);
                    df_fma(acc[j][2], nlx, xqi);
                    df_fma(acc[j][2], nlw, ur);
                    df_fma(acc[j][3], lx, xqr);
                    df_fma(acc[j][3], nlw, ui);
                }
            }
        }
#pragma unroll
        for (int j = 0; j < 8; ++j)
#pragma unroll
            for (int q = 0; q < NO; ++q) df_acc_norm(acc[j][q]);   // 64 terms at most since the last
    }
    // ---- epilogue: every alm of this CTA's l range written once
    if (k >= nm) return;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int l = lbase + c + 2 * (rg + 8 * j);
        if (l > L) continue;
        const double bm = (a.beam ? a.beam[l] : 1.0) * ((a.vjp && m > 0) ? 2.0 : 1.0);
#pragma unroll
        for (int cc = 0; cc < NO / 2; ++cc) {
            const int64_t row = (int64_t)(map0 + k) * a.rs + cc;
            double2 *dst = const_cast<double2 *>(a.alm) + row * a.nalm + base + l;
            *dst = make_double2(df_acc_to(acc[j][2 * cc]) * bm, m == 0 ? 0.0 : df_acc_to(acc[j][2 * cc + 1]) * bm);
        }
    }
}

template <int NR, int NM, int SPIN>
int launch_synth_df(Plan *p, const double2 *alm, int rs, int nmaps, const double *beam, double2 *F,
                    cudaStream_t st) {
    LegArgs<double> a = leg_make_args<double>(p);
    a.alm = alm;
    a.rs = rs;
    a.F = F;
    a.beam = beam;
    a.nmaps = nmaps;
    dim3 grid((p->npairs + LEG_THREADS * NR - 1) / (LEG_THREADS * NR), p->lmax + 1, (nmaps + NM - 1) / NM);
    prof_begin(p, K_LEG_SYN64, st);
    k_leg_synth_df<NR, NM, SPIN><<<grid, LEG_THREADS, 0, st>>>(a);
    prof_end(p, st);
    SHTG_CHECK_LAUNCH("k_leg_synth_df");
    return SHTG_OK;
}

template <int SPIN>
int launch_analysis_df(Plan *p, const double2 *G, int nmaps, const double *beam, double2 *alm, int rs,
                       cudaStream_t st, int vjp) {
    LegArgs<double> a = leg_make_args<double>(p);
    a.alm = alm;
    a.rs = rs;
    a.vjp = vjp;
    a.F = const_cast<double2 *>(G);
    a.beam = beam;
    a.nmaps = nmaps;
    if (!a.toff64 || !a.tst64_0 || (SPIN == 2 && !a.tst64_2)) {
        set_error("double-FP32 transpose: the plan has no FP64 recurrence tile states");
        return SHTG_ERR_ARG;
    }
    const int smem = DfT<SPIN>::BYTES;
    if (smem > 48 * 1024)
        SHTG_CUDA(cudaFuncSetAttribute(k_leg_analysis_df<SPIN>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    dim3 grid((p->lmax + D_LR) / D_LR, p->lmax + 1, (nmaps + D_NMT - 1) / D_NMT);
    prof_begin(p, K_LEG_ANA64, st);
    k_leg_analysis_df<SPIN><<<grid, D_NT, smem, st>>>(a);
    prof_end(p, st);
    SHTG_CHECK_LAUNCH("k_leg_analysis_df");
    return SHTG_OK;
}

}  // namespace

// Autotuned (key kind 3): synthesis (ring pairs per thread, maps per pass)
// spin 0: (1, 8), (1, 4), (2, 4); spin 2: (1, 4), (1, 2), (2, 1) (the first
// of each was the fastest at N_side 1024, l_max 2048, 8 maps).  The
// transpose has one shape.
int leg_synth_df(Plan *p, int spin, const double2 *alm, int rs, int nmaps, const double *beam, double2 *F,
                 cudaStream_t st) {
    return tune(p, 3, spin == 2 ? 1 : 0, nmaps, 3, st, [&](int v) {
        if (spin == 2) {
            if (v == 1) return launch_synth_df<1, 2, 2>(p, alm, rs, nmaps, beam, F, st);
            if (v == 2) return launch_synth_df<2, 1, 2>(p, alm, rs, nmaps, beam, F, st);
            return launch_synth_df<1, 4, 2>(p, alm, rs, nmaps, beam, F, st);
        }
        if (v == 1) return launch_synth_df<1, 4, 0>(p, alm, rs, nmaps, beam, F, st);
        if (v == 2) return launch_synth_df<2, 4, 0>(p, alm, rs, nmaps, beam, F, st);
        return launch_synth_df<1, 8, 0>(p, alm, rs, nmaps, beam, F, st);
    });
}

int leg_analysis_df(Plan *p, int spin, const double2 *G, int nmaps, const double *beam, double2 *alm, int rs,
                    cudaStream_t st, int vjp) {
    if (spin == 2) return launch_analysis_df<2>(p, G, nmaps, beam, alm, rs, st, vjp);
    return launch_analysis_df<0>(p, G, nmaps, beam, alm, rs, st, vjp);
}

}  // namespace shtg

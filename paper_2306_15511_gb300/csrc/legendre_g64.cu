// FP64 Legendre transpose (Y^T) as a register-blocked contraction.
//
// c_lm = sum_r lambda_lm(theta_r) G_r(m): for one m and a range of 128 l,
// the recurrence values of 16 ring pairs at a time are generated once into
// shared memory ([row = l - lbase][pair]) and every thread accumulates a
// block of outputs over all ring pairs in registers: 8 rows of one parity
// class of l - m (App. A: lambda_lm(pi - theta) = (-1)^(l+m) lambda_lm(theta),
// so class-E rows take G_N + G_S and class-O rows G_N - G_S) times the 2
// (spin 0) or 4 (spin 2: E re, E im, B re, B im) outputs of one map.  Each
// recurrence runs once per (l, ring pair) for all maps, and the sum over
// ring pairs needs no cross-thread reduction: per (l, ring pair, map) the
// FP64 pipe sees the 2 (spin 0) or 8 (spin 2) multiply-adds of the
// contraction and nothing else.  The recurrence restarts every 128 l from
// FP64 states tabulated (every SHTG_TS64 l) at plan creation by the same
// steps, so its values equal those of one continuous run.
#include <string>
#include <vector>

#include "legendre_kernels.cuh"

namespace shtg {
namespace {

constexpr int G_LR = 128;   // l per CTA (rows)
constexpr int G_KP = 16;    // ring pairs per stage
constexpr int G_NT = 128;   // threads
constexpr int G_NMT = 8;    // maps per CTA (grid.z covers more)
constexpr int G_LS = G_KP + 1;   // row stride of the value tile (odd: rows in distinct banks)
constexpr int G_GS = 9;          // map stride of the ring-data sets

// FP64 recurrence state before every l = m + SHTG_TS64 t of every (m, ring
// pair), [m][t][pair]: the steps of the Legendre kernels, one thread per
// (m, pair).
template <int SPIN>
__global__ void __launch_bounds__(LEG_THREADS) k_tile_states64(const LegArgs<double> a, const int64_t *toff,
                                                               double2 *out0, double4_32a *out2) {
    const int m = blockIdx.y;
    const int L = a.lmax;
    PairState<double, 1> S;
    int wlo, whi;
    load_pairs<double, 1, SPIN>(a, blockIdx.x, m, S, wlo, whi);
    const int pr = S.pr[0];
    if (pr >= a.npairs) return;
    const int64_t base = (int64_t)m * (2 * L + 1 - m) / 2;
    const int64_t o = toff[m] * a.npairs + pr;
    for (int l = m; l <= L; ++l) {
        if (((l - m) & (SHTG_TS64 - 1)) == 0) {
            const int64_t e = o + (int64_t)((l - m) / SHTG_TS64) * a.npairs;
            if (SPIN == 2) out2[e] = make_double4_32a(S.a1[0], S.a2[0], S.b1[0], S.b2[0]);
            else out0[e] = make_double2(S.a1[0], S.a2[0]);
        }
        stepx<double, 1, SPIN, true>(S, a.rec + base, a.s2c + base, l, l);
    }
}

template <int SPIN> struct G64 {
    static constexpr int NV = SPIN == 2 ? 2 : 1;    // value tiles: lambda, or (lw, lx)
    static constexpr int NO = SPIN == 2 ? 4 : 2;    // outputs per map
    static constexpr int COEF = SPIN == 2 ? 32 : 16;
    static constexpr int LAM = 0;
    static constexpr int GSET = LAM + NV * G_LR * G_LS * 8;
    static constexpr int CO = GSET + G_KP * G_NMT * G_GS * 8;
    static constexpr int RED = CO + G_LR * COEF;
    static constexpr int BYTES = RED + 16;
};

template <int SPIN>
__global__ void __launch_bounds__(G_NT) k_leg_analysis_g64(const LegArgs<double> a) {
    typedef G64<SPIN> Ly;
    constexpr int NO = Ly::NO;
    extern __shared__ __align__(16) unsigned char smem[];
    double *lam = reinterpret_cast<double *>(smem + Ly::LAM);      // [NV][G_LR][G_LS]
    double *gset = reinterpret_cast<double *>(smem + Ly::GSET);    // [G_KP][G_NMT][G_GS]
    double2 *s_rec = reinterpret_cast<double2 *>(smem + Ly::CO);
    double4_32a *s_s2c = reinterpret_cast<double4_32a *>(smem + Ly::CO);
    int *s_first = reinterpret_cast<int *>(smem + Ly::RED);

    const int tid = threadIdx.x;
    const int m = blockIdx.y;
    const int L = a.lmax;
    const int lbase = m + blockIdx.x * G_LR;
    if (lbase > L) return;
    const int lend = min(L, lbase + G_LR - 1);
    const int map0 = blockIdx.z * G_NMT;
    const int nm = min(G_NMT, a.nmaps - map0);
    const int64_t base = (int64_t)m * (2 * L + 1 - m) / 2;
    const int64_t rowsz = (int64_t)a.nring * (L + 1);

    for (int i = tid; i < G_LR; i += G_NT) {
        const int l = lbase + i;
        const bool in = l <= L;
        if (SPIN == 2) s_s2c[i] = in ? a.s2c[base + l] : make_double4_32a(0.0, 0.0, 0.0, 0.0);
        else s_rec[i] = in ? a.rec[base + l] : make_double2(0.0, 0.0);
    }
    // first ring pair whose recurrence starts at or before lend (the start l
    // falls towards the equator; a later pair without significant values
    // only adds exact zeros)
    if (tid == 0) *s_first = a.npairs;
    __syncthreads();
    {
        for (int pr = tid; pr < a.npairs; pr += G_NT) {
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
    }
    __syncthreads();
    const int s0 = *s_first / G_KP;
    const int nps = (a.npairs + G_KP - 1) / G_KP;

    // this thread's outputs: map k, class c, rows i = c + 2 (rg + 8 j)
    const int k = tid & 7, c = (tid >> 3) & 1, rg = tid >> 4;
    double acc[8][NO];
#pragma unroll
    for (int j = 0; j < 8; ++j)
#pragma unroll
        for (int q = 0; q < NO; ++q) acc[j][q] = 0.0;

    for (int s = s0; s < nps; ++s) {
        __syncthreads();   // the previous stage's tiles are consumed
        if (tid < G_KP) {
            // ---- recurrence of pair s * 16 + tid over the 128 rows
            const int pr = s * G_KP + tid;
            PairState<double, 1> S;
            S.a1[0] = S.a2[0] = S.b1[0] = S.b2[0] = 0.0;
            S.u[0] = 1.0;
            S.ls[0] = S.lsb[0] = L + 1;
            S.s0[0] = S.s1[0] = S.s2[0] = S.s3[0] = 0.0;
            const bool live = pr < a.npairs;
            if (live) {
                const int64_t o = (int64_t)m * a.npairs + pr;
                const int64_t e = (a.toff64[m] + (lbase - m) / SHTG_TS64) * a.npairs + pr;
                S.u[0] = a.u[pr];
                if (SPIN == 2) {
                    const int2 q = a.ls2[o];
                    S.ls[0] = q.x;
                    S.lsb[0] = q.y;
                    const double4_32a s4 = a.st2[o];
                    S.s0[0] = s4.x;
                    S.s1[0] = s4.y;
                    S.s2[0] = s4.z;
                    S.s3[0] = s4.w;
                    const double4_32a t4 = a.tst64_2[e];
                    S.a1[0] = t4.x;
                    S.a2[0] = t4.y;
                    S.b1[0] = t4.z;
                    S.b2[0] = t4.w;
                } else {
                    S.ls[0] = a.ls[o];
                    const double2 s2 = a.st[o];
                    S.s0[0] = s2.x;
                    S.s1[0] = s2.y;
                    const double2 t2 = a.tst64_0[e];
                    S.a1[0] = t2.x;
                    S.a2[0] = t2.y;
                }
            }
            for (int i = 0; i < G_LR; ++i) {
                double v0 = 0.0, v1 = 0.0;
                if (live) {
                    stepx<double, 1, SPIN, true>(S, s_rec, s_s2c, i, lbase + i);
                    if (SPIN == 2) {
                        v0 = S.a1[0] + S.b1[0];
                        v1 = S.a1[0] - S.b1[0];
                    } else {
                        v0 = S.a1[0];
                    }
                }
                lam[i * G_LS + tid] = v0;
                if (SPIN == 2) lam[G_LR * G_LS + i * G_LS + tid] = v1;
            }
        }
        {
            // ---- ring data of the stage: per (pair, map) the even / odd sets
            const int pp = tid >> 3, kk = tid & 7;
            const int pr = s * G_KP + pp;
            double *g = gset + (pp * G_NMT + kk) * G_GS;
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
                g[2 * q] = z[q].x;
                g[2 * q + 1] = z[q].y;
            }
        }
        __syncthreads();
        // ---- contraction over the stage's ring pairs
#pragma unroll 4
        for (int p = 0; p < G_KP; ++p) {
            const double *g = gset + (p * G_NMT + k) * G_GS;
            if (SPIN == 0) {
                const double gre = g[2 * c], gim = g[2 * c + 1];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const double lv = lam[(c + 2 * (rg + 8 * j)) * G_LS + p];
                    acc[j][0] = fma(lv, gre, acc[j][0]);
                    acc[j][1] = fma(lv, gim, acc[j][1]);
                }
            } else {
                // lw terms take the row's set, lx terms the other one:
                //   E^ = -lw G_Q - i lx G_U,  B^ = i lx G_Q - lw G_U
                const double qr = g[2 * c], qi = g[2 * c + 1], ur = g[4 + 2 * c], ui = g[4 + 2 * c + 1];
                const double xqr = g[2 * (1 - c)], xqi = g[2 * (1 - c) + 1], xur = g[4 + 2 * (1 - c)],
                             xui = g[4 + 2 * (1 - c) + 1];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int i = c + 2 * (rg + 8 * j);
                    const double lw = lam[i * G_LS + p], lx = lam[G_LR * G_LS + i * G_LS + p];
                    acc[j][0] = fma(-lw, qr, fma(lx, xui, acc[j][0]));
                    acc[j][1] = fma(-lw, qi, fma(-lx, xur, acc[j][1]));
                    acc[j][2] = fma(-lw, ur, fma(-lx, xqi, acc[j][2]));
                    acc[j][3] = fma(-lw, ui, fma(lx, xqr, acc[j][3]));
                }
            }
        }
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
            *dst = make_double2(acc[j][2 * cc] * bm, m == 0 ? 0.0 : acc[j][2 * cc + 1] * bm);
        }
    }
}

template <int SPIN>
int launch_g64(Plan *p, const double2 *G, int nmaps, const double *beam, double2 *alm, int rs, cudaStream_t st,
               int vjp) {
    LegArgs<double> a = leg_make_args<double>(p);
    a.alm = alm;
    a.rs = rs;
    a.vjp = vjp;
    a.F = const_cast<double2 *>(G);
    a.beam = beam;
    a.nmaps = nmaps;
    if (!a.toff64 || !a.tst64_0 || (SPIN == 2 && !a.tst64_2)) {
        set_error("FP64 transpose: the plan has no FP64 recurrence tile states");
        return SHTG_ERR_ARG;
    }
    const int smem = G64<SPIN>::BYTES;
    if (smem > 48 * 1024)
        SHTG_CUDA(cudaFuncSetAttribute(k_leg_analysis_g64<SPIN>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    dim3 grid((p->lmax + G_LR) / G_LR, p->lmax + 1, (nmaps + G_NMT - 1) / G_NMT);
    prof_begin(p, K_LEG_ANA64, st);
    k_leg_analysis_g64<SPIN><<<grid, G_NT, smem, st>>>(a);
    prof_end(p, st);
    SHTG_CHECK_LAUNCH("k_leg_analysis_g64");
    return SHTG_OK;
}

}  // namespace

int build_tile_states64(Plan *p) {
    const int L = p->lmax;
    std::vector<int64_t> toff(L + 2);
    toff[0] = 0;
    for (int m = 0; m <= L; ++m) toff[m + 1] = toff[m] + (L + 1 - m + SHTG_TS64 - 1) / SHTG_TS64;
    const size_t nent = (size_t)toff[L + 1] * p->npairs;
    auto alloc = [&](void **ptr, size_t bytes) -> int {
        cudaError_t e = cudaMalloc(ptr, bytes);
        if (e != cudaSuccess) {
            *ptr = nullptr;
            cudaGetLastError();
            set_error(std::string("cudaMalloc of ") + std::to_string(bytes) +
                      " bytes (FP64 recurrence tile states) failed: " + cudaGetErrorString(e));
            return SHTG_ERR_NOMEM;
        }
        p->device_bytes += (int64_t)bytes;
        return SHTG_OK;
    };
    SHTG_TRY(alloc((void **)&p->d_toff64, sizeof(int64_t) * toff.size()));
    SHTG_CUDA(cudaMemcpy(p->d_toff64, toff.data(), sizeof(int64_t) * toff.size(), cudaMemcpyHostToDevice));
    SHTG_TRY(alloc((void **)&p->d_tst64_0, sizeof(double2) * nent));
    LegArgs<double> a = leg_make_args<double>(p);
    dim3 grid((p->npairs + LEG_THREADS - 1) / LEG_THREADS, L + 1);
    k_tile_states64<0><<<grid, LEG_THREADS>>>(a, p->d_toff64, p->d_tst64_0, nullptr);
    SHTG_CHECK_LAUNCH("k_tile_states64");
    if (p->flags & SHTG_SPIN2) {
        SHTG_TRY(alloc((void **)&p->d_tst64_2, sizeof(double4_32a) * nent));
        k_tile_states64<2><<<grid, LEG_THREADS>>>(a, p->d_toff64, nullptr, p->d_tst64_2);
        SHTG_CHECK_LAUNCH("k_tile_states64");
    }
    SHTG_CUDA(cudaDeviceSynchronize());
    return SHTG_OK;
}

int leg_analysis_g64(Plan *p, int spin, const double2 *G, int nmaps, const double *beam, double2 *alm, int rs,
                     cudaStream_t st, int vjp) {
    if (spin == 2) return launch_g64<2>(p, G, nmaps, beam, alm, rs, st, vjp);
    return launch_g64<0>(p, G, nmaps, beam, alm, rs, st, vjp);
}

}  // namespace shtg

// Dispatch of the Legendre kernels: argument set-up, the diag kernel and an
// autotuner that picks the (ring pairs per thread, maps per pass) shape of
// each kernel family on first use.
#include <algorithm>
#include <map>
#include <string>

#include "legendre_kernels.cuh"

namespace shtg {

template <> LegArgs<float> leg_make_args<float>(Plan *p) {
    LegArgs<float> a{};
    a.lmax = p->lmax;
    a.npairs = p->npairs;
    a.nring = p->nring;
    a.nalm = p->nalm;
    a.rec = p->d_rec32;
    a.s2c = p->d_s2c32;
    a.ls = p->d_ls32;
    a.st = p->d_st32;
    a.ls2 = p->d_ls2_32;
    a.st2 = p->d_st2_32;
    a.u = p->d_u32;
    a.toff = p->d_toff;
    a.tst0 = p->d_tst0;
    a.tst2 = p->d_tst2;
    return a;
}
template <> LegArgs<double> leg_make_args<double>(Plan *p) {
    LegArgs<double> a{};
    a.lmax = p->lmax;
    a.npairs = p->npairs;
    a.nring = p->nring;
    a.nalm = p->nalm;
    a.rec = p->d_rec64;
    a.s2c = p->d_s2c64;
    a.ls = p->d_ls64;
    a.st = p->d_st64;
    a.ls2 = p->d_ls2_64;
    a.st2 = p->d_st2_64;
    a.u = p->d_u64;
    a.toff64 = p->d_toff64;
    a.tst64_0 = p->d_tst64_0;
    a.tst64_2 = p->d_tst64_2;
    return a;
}

template <>
int leg_synth<float>(Plan *p, int spin, const float2 *alm, int rs, int nmaps, const float *beam,
                     float2 *F, cudaStream_t st) {
    const Variants32 &V = variants32();
    const int s = spin == 2 ? 1 : 0;
    return tune(p, 1, s, nmaps, V.n[s], st, [&](int v) { return V.syn[s][v](p, alm, rs, nmaps, beam, F, st); });
}
template <>
int leg_synth<double>(Plan *p, int spin, const double2 *alm, int rs, int nmaps, const double *beam,
                      double2 *F, cudaStream_t st) {
    const Variants64 &V = variants64();
    const int s = spin == 2 ? 1 : 0;
    return tune(p, 0, s, nmaps, V.n[s], st, [&](int v) { return V.syn[s][v](p, alm, rs, nmaps, beam, F, st); });
}
template <>
int leg_analysis<float>(Plan *p, int spin, const float2 *G, int nmaps, const float *beam, float2 *alm,
                        int rs, cudaStream_t st, int vjp) {
    const Variants32 &V = variants32();
    const int s = spin == 2 ? 1 : 0;
    return tune(p, 1, 2 + s, nmaps, V.n[2 + s], st,
                [&](int v) { return V.ana[s][v](p, G, nmaps, beam, alm, rs, st, vjp); });
}
template <>
int leg_analysis<double>(Plan *p, int spin, const double2 *G, int nmaps, const double *beam,
                         double2 *alm, int rs, cudaStream_t st, int vjp) {
    // candidates: the register-blocked contraction (legendre_g64.cu, about
    // half the FP64 instructions of the warp-reduction kernels when several
    // maps share a recurrence; the default), then the warp-reduction shapes
    const Variants64 &V = variants64();
    const int s = spin == 2 ? 1 : 0;
    return tune(p, 0, 2 + s, nmaps, V.n[2 + s] + 1, st, [&](int v) {
        if (v == 0) return leg_analysis_g64(p, spin, G, nmaps, beam, alm, rs, st, vjp);
        return V.ana[s][v - 1](p, G, nmaps, beam, alm, rs, st, vjp);
    });
}

// ------------------------------------------------------- grouped launches
// FP32 Legendre sums on the CUDA cores over several plans in one launch (the
// chains of several geometries), each group with the shape of variant 0 of
// its family (the shape the tuner keeps at batches of about ten maps).
namespace {
template <int SPIN, bool SYN> struct GrpShape;
template <> struct GrpShape<0, true> { static constexpr int NR = 4, NM = 2; };
template <> struct GrpShape<2, true> { static constexpr int NR = 2, NM = 2; };
template <> struct GrpShape<0, false> { static constexpr int NR = 4, NM = 2; };
template <> struct GrpShape<2, false> { static constexpr int NR = 2, NM = 2; };

template <int SPIN, bool SYN>
int launch_grp(int ng, Plan *const *ps, const float2 *const *in, const int *rs, const int *nmaps,
               const float *const *beam, float2 *const *out, const int *const *active, cudaStream_t st) {
    constexpr int NR = GrpShape<SPIN, SYN>::NR, NM = GrpShape<SPIN, SYN>::NM, NO = SPIN == 2 ? 4 : 2;
    if (ng < 1 || ng > SHTG_MAX_GROUPS) {
        set_error("grouped Legendre launch: 1 to " + std::to_string(SHTG_MAX_GROUPS) + " groups");
        return SHTG_ERR_ARG;
    }
    LegGroups<float> G{};
    G.ng = ng;
    size_t smem = 0;
    int64_t total = 0;
    // entries in the order of decreasing l_max (the longest recurrences per
    // CTA first, so the launch does not end on them)
    int order[SHTG_MAX_GROUPS];
    for (int g = 0; g < ng; ++g) order[g] = g;
    std::stable_sort(order, order + ng, [&](int x, int y) { return ps[x]->lmax > ps[y]->lmax; });
    for (int e = 0; e < ng; ++e) {
        const int g = order[e];
        Plan *p = ps[g];
        LegArgs<float> a = leg_make_args<float>(p);
        a.rs = rs[g];
        a.beam = beam[g];
        a.nmaps = nmaps[g];
        if (SYN) {
            a.alm = in[g];
            a.F = out[g];
        } else {
            a.F = const_cast<float2 *>(in[g]);
            a.alm = out[g];
        }
        G.a[e] = a;
        G.active[e] = active ? active[g] : nullptr;
        G.gx[e] = (p->npairs + LEG_THREADS * NR - 1) / (LEG_THREADS * NR);
        G.gy[e] = p->lmax + 1;
        G.first[e] = (int)total;
        total += (int64_t)G.gx[e] * G.gy[e] * ((nmaps[g] + NM - 1) / NM);
        if (!SYN) {
            smem = std::max(smem, sizeof(float) * (size_t)(p->lmax + 1) * NM * NO);
            if (G.gx[e] > 1) {   // CTAs of one m add their sums atomically
                const size_t cs = sizeof(float2) * (size_t)p->nalm;
                SHTG_CUDA(cudaMemset2DAsync(out[g], cs * rs[g], 0, cs * (SPIN == 2 ? 2 : 1), nmaps[g], st));
            }
        }
    }
    if (total > 0x7fffffff) {
        set_error("grouped Legendre launch: too many CTAs");
        return SHTG_ERR_ARG;
    }
    G.first[ng] = (int)total;
    if (total == 0) return SHTG_OK;
    Plan *acct = ps[0];
    prof_begin(acct, SYN ? K_LEG_SYN32 : K_LEG_ANA32, st);
    if (SYN) {
        k_leg_synth_grp<float, NR, NM, SPIN><<<(unsigned)total, LEG_THREADS, 0, st>>>(G);
    } else {
        auto kern = k_leg_analysis_grp<float, NR, NM, SPIN>;
        if (smem > 48 * 1024) SHTG_CUDA(allow_max_smem(kern));
        kern<<<(unsigned)total, LEG_THREADS, smem, st>>>(G);
    }
    prof_end(acct, st);
    SHTG_CHECK_LAUNCH(SYN ? "k_leg_synth_grp" : "k_leg_analysis_grp");
    return SHTG_OK;
}
}  // namespace

int leg_synth_grp(int ng, Plan *const *ps, int spin, const float2 *const *alm, const int *rs, const int *nmaps,
                  const float *const *beam, float2 *const *F, const int *const *active, cudaStream_t st) {
    if (spin == 2) return launch_grp<2, true>(ng, ps, alm, rs, nmaps, beam, F, active, st);
    return launch_grp<0, true>(ng, ps, alm, rs, nmaps, beam, F, active, st);
}
int leg_analysis_grp(int ng, Plan *const *ps, int spin, const float2 *const *G, const int *nmaps,
                     const float *const *beam, float2 *const *alm, const int *rs, const int *const *active,
                     cudaStream_t st) {
    if (spin == 2) return launch_grp<2, false>(ng, ps, G, rs, nmaps, beam, alm, active, st);
    return launch_grp<0, false>(ng, ps, G, rs, nmaps, beam, alm, active, st);
}

int leg_diag(Plan *p, int spin, const float *wpair, float *out, cudaStream_t st) {
    constexpr int NR = 4;
    LegArgs<float> a = leg_make_args<float>(p);
    a.wpair = wpair;
    a.diag = out;
    const int gx = (p->npairs + LEG_THREADS * NR - 1) / (LEG_THREADS * NR);
    if (gx > 1) SHTG_CUDA(cudaMemsetAsync(out, 0, sizeof(float) * p->nalm, st));
    const size_t smem = sizeof(float) * (size_t)(p->lmax + 1);
    dim3 grid(gx, p->lmax + 1, 1);
    prof_begin(p, K_DIAG, st);
    if (spin == 2) {
        if (smem > 48 * 1024) SHTG_CUDA(allow_max_smem(k_leg_diag<NR, 2>));
        k_leg_diag<NR, 2><<<grid, LEG_THREADS, smem, st>>>(a);
    } else {
        if (smem > 48 * 1024) SHTG_CUDA(allow_max_smem(k_leg_diag<NR, 0>));
        k_leg_diag<NR, 0><<<grid, LEG_THREADS, smem, st>>>(a);
    }
    prof_end(p, st);
    SHTG_CHECK_LAUNCH("k_leg_diag");
    return SHTG_OK;
}

}  // namespace shtg

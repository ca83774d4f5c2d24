// Dispatch of the Legendre kernels: argument set-up, the diag kernel and an
// autotuner that picks the (ring pairs per thread, maps per pass) shape of
// each kernel family on first use.
#include <map>

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

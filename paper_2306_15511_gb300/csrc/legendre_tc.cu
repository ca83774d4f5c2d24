// Legendre synthesis on the 5th-generation tensor cores (tcgen05).
//
// F_r(m) = sum_l lambda_lm(theta_r) a_lm is, for one m and a block of 128
// ring pairs, the product of a [pair x l] matrix (the recurrence values,
// generated on the fly) with an [l x column] matrix (the alm of all maps),
// split by the parity of l - m into the even / odd sums E, O (App. A:
// lambda_lm(pi - theta) = (-1)^(l+m) lambda_lm(theta)), F_N = E + O,
// F_S = E - O.  Spin 2 uses the two Wigner recurrences y+, y- with
// lw = y+ + y-, lx = y+ - y- as two A matrices and the (E, B) -> (Q, U)
// sign pattern folded into the B matrices.
//
// Precision: every thread runs the FP32 recurrence of its ring pair exactly
// as the FP32 CUDA-core kernels do (same FP64 start states), and each value
// x is split into bf16 x_hi + x_lo (x_lo = bf16(x - x_hi)); the alm are split
// the same way.  Three products hi*hi + lo*hi + hi*lo are accumulated in
// FP32 in tensor memory, which keeps ~16 of the 24 mantissa bits of every
// product (relative error ~2^-17 per term) at bf16 tensor-core rates.
//
// Pipeline per CTA (one m, 128 ring pairs, up to 8 maps): the l range is cut
// into chunks of 32 (16 per parity class, one MMA K of 16 each).  All 128
// threads generate the A tiles of chunk c (bf16 hi / lo, K-major core
// matrices in shared memory) and the B tiles, then one thread issues the
// tcgen05.mma of chunk c and commits them to an mbarrier.  With two stages
// the threads go on with chunk c + 1 in the other stage while the tensor
// core works; with one stage (half the shared memory, twice the resident
// CTAs) they wait for the commit and the other CTAs on the SM fill the gap.
// The accumulators stay in tensor memory until the last chunk and are read
// back with tcgen05.ld for the F_N / F_S epilogue.
#include <cuda_bf16.h>

#include "legendre_kernels.cuh"

namespace shtg {
namespace {

constexpr int TC_M = 128;        // ring pairs per CTA = MMA M = threads
constexpr int TC_NMT = 8;        // maps per CTA (grid.z covers more)
constexpr int TC_ATILE = 4096;   // one A tile: 128 rows x 16 bf16 (K-major core matrices)
constexpr uint32_t TC_WAIT_LIMIT = 1u << 22;   // bounded mbarrier polling

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor, no swizzle: start address, LBO = byte
// stride between core matrices adjacent in K, SBO = byte stride between
// core matrices adjacent in M (or N); version 1 at bit 46.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor of kind::f16 with bf16 A and B (both K-major) and an
// FP32 accumulator: D format bit 4, A / B format 1 (bf16) at bits 7 / 10,
// N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t idesc_bf16(int m, int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t da, uint64_t db, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(da), "l"(db), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
        smem_u32(bar)));
}

// Wait (bounded) for the completion of the mbarrier phase with the given
// parity; false if the limit ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
    uint32_t done = 0;
    for (uint32_t it = 0; it < TC_WAIT_LIMIT && !done; ++it) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(smem_u32(bar)), "r"(parity));
    }
    return done != 0;
}

// 32 consecutive TMEM columns of this warp's 32 lanes: thread = lane
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
          "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
          "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
          "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// (a, b) -> bf16x2 hi and lo words, element a in the low half
__device__ __forceinline__ void split2(float a, float b, uint32_t &hi, uint32_t &lo) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    const float2 hf = __bfloat1622float2(h);
    const __nv_bfloat162 l = __floats2bfloat162_rn(a - hf.x, b - hf.y);
    hi = *reinterpret_cast<const uint32_t *>(&h);
    lo = *reinterpret_cast<const uint32_t *>(&l);
}

// 8 values -> one 16-byte core-matrix row of hi and one of lo
__device__ __forceinline__ void store_row8(unsigned char *hi_row, unsigned char *lo_row, const float (&x)[8]) {
    uint4 h, l;
    split2(x[0], x[1], h.x, l.x);
    split2(x[2], x[3], h.y, l.y);
    split2(x[4], x[5], h.z, l.z);
    split2(x[6], x[7], h.w, l.w);
    *reinterpret_cast<uint4 *>(hi_row) = h;
    *reinterpret_cast<uint4 *>(lo_row) = l;
}

// Per-spin tile configuration.  NCOL: B rows of one product block (spin 0:
// re, im of 8 maps; spin 2: Q re, Q im, U re, U im of 8 maps); a B tile holds
// NCOL hi rows then NCOL lo rows, 16 K (l of one parity class) each.
template <int SPIN> struct TcCfg;
template <> struct TcCfg<0> {
    static constexpr int NCOL = 16, NA = TC_NMT, NTA = 4, NTB = 2, TMEM = 64;
};
template <> struct TcCfg<2> {
    static constexpr int NCOL = 32, NA = 2 * TC_NMT, NTA = 8, NTB = 4, TMEM = 128;
};
// Shared memory of the synthesis CTA: NSTG operand stages (A and B tiles of
// one 32-l chunk each), the alm and recurrence coefficients of SCH l, two
// mbarriers, the TMEM address and scratch.  One stage halves the footprint
// (spin 2: 50 KB instead of 99 KB with SCH = 64), so four CTAs instead of two
// share an SM; the MMA of a chunk then has to finish before the CTA writes
// the next chunk's tiles, and the other CTAs fill that gap.
template <int SPIN, int NSTG, int SCH> struct TcLayout {
    static constexpr int ALMS = SCH + 1;   // staged alm row stride (odd: rows fall in distinct banks)
    static constexpr int BTILE = 2 * TcCfg<SPIN>::NCOL * 32;
    static constexpr int STAGE = TcCfg<SPIN>::NTA * TC_ATILE + TcCfg<SPIN>::NTB * BTILE;
    static constexpr int ALM = NSTG * STAGE;                                // staged alm [NA][ALMS] float2
    static constexpr int COEF = ALM + ((TcCfg<SPIN>::NA * ALMS * 8 + 15) & ~15);   // staged coefficients
    static constexpr int BARS = COEF + SCH * (SPIN == 2 ? 16 : 8);          // 2 mbarriers
    static constexpr int TMEMA = BARS + 16;                                 // TMEM base address
    static constexpr int RED = TMEMA + 16;                                  // cta_min scratch
    static constexpr int BYTES = RED + 16;
};

// Recurrence over one chunk of 32 l (l = q0 .. q0 + 31, staged coefficient
// index i0 + (l - q0)); values of the even class (l - m even, K index
// (l - q0) / 2) and the odd class go to their A tiles as bf16 hi / lo.
// Row = this thread's ring pair; K group h = 0, 1 holds K 0..7, 8..15.
template <int SPIN, bool INJ>
__device__ __forceinline__ void gen_atiles(PairState<float, 1> &S, const float2 *s_rec, const float4 *s_s2c,
                                           const int i0, const int q0, unsigned char *stg) {
    const int rofs = threadIdx.x * 16;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        unsigned char *t = stg + h * 2048 + rofs;
        if (SPIN == 0) {
            float e[8], o[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int d = 16 * h + 2 * i;
                stepx<float, 1, 0, INJ>(S, s_rec, s_s2c, i0 + d, q0 + d);
                e[i] = S.a1[0];
                stepx<float, 1, 0, INJ>(S, s_rec, s_s2c, i0 + d + 1, q0 + d + 1);
                o[i] = S.a1[0];
            }
            store_row8(t, t + TC_ATILE, e);                   // E hi, E lo
            store_row8(t + 2 * TC_ATILE, t + 3 * TC_ATILE, o); // O hi, O lo
        } else {
            float wE[8], wO[8], xE[8], xO[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int d = 16 * h + 2 * i;
                stepx<float, 1, 2, INJ>(S, s_rec, s_s2c, i0 + d, q0 + d);
                wE[i] = S.a1[0] + S.b1[0];
                xE[i] = S.a1[0] - S.b1[0];
                stepx<float, 1, 2, INJ>(S, s_rec, s_s2c, i0 + d + 1, q0 + d + 1);
                wO[i] = S.a1[0] + S.b1[0];
                xO[i] = S.a1[0] - S.b1[0];
            }
            // tiles: lwE hi, lo | lwO hi, lo | lxE hi, lo | lxO hi, lo
            store_row8(t, t + TC_ATILE, wE);
            store_row8(t + 2 * TC_ATILE, t + 3 * TC_ATILE, wO);
            store_row8(t + 4 * TC_ATILE, t + 5 * TC_ATILE, xE);
            store_row8(t + 6 * TC_ATILE, t + 7 * TC_ATILE, xO);
        }
    }
}

// B tiles of one chunk from the staged alm (already times the beam).  Tile
// b: spin 0 -> class b (0 even, 1 odd); spin 2 -> b = 2 w + class with
// W columns (-E re, -E im, -B re, -B im) and X columns (B im, -B re, -E im,
// E re) per map, feeding (Q re, Q im, U re, U im).  Column c, K index k:
// hi at row c, lo at row NCOL + c (K-major core matrices, LBO = 32 NCOL).
template <int SPIN, int ALMS>
__device__ __forceinline__ void gen_btiles(const float2 *s_alm, const int i0, unsigned char *bt) {
    constexpr int NCOL = TcCfg<SPIN>::NCOL, NTB = TcCfg<SPIN>::NTB;
    constexpr int BTILE = 2 * NCOL * 32;
    // item = (tile b, K group kg, column c): one 16-byte core-matrix row of
    // hi and one of lo (the 8 K values, l = i0 + off + 16 kg + 2 j, of column
    // c), consecutive threads on consecutive rows.  Column c of tile b reads
    // one component of one staged alm row: spin 0 (re, im) of map c / 2;
    // spin 2 W tiles (b < 2) -(E re, E im, B re, B im), X tiles (B im, -B re,
    // -E im, E re) of map c / 4, component c % 4.
    for (int it = threadIdx.x; it < NTB * 2 * NCOL; it += TC_M) {
        const int c = it % NCOL, kg = (it / NCOL) & 1, b = it / (2 * NCOL);
        const int off = b & 1;
        int row, ri;
        float sg;
        if (SPIN == 0) {
            row = c >> 1;
            ri = c & 1;
            sg = 1.f;
        } else {
            const int mk = c >> 2, comp = c & 3;
            if (b < 2) {
                row = 2 * mk + (comp >= 2 ? 1 : 0);
                ri = comp & 1;
                sg = -1.f;
            } else {
                row = 2 * mk + (comp < 2 ? 1 : 0);
                ri = (comp & 1) ^ 1;
                sg = (comp == 1 || comp == 2) ? -1.f : 1.f;
            }
        }
        const float *src = reinterpret_cast<const float *>(s_alm + row * ALMS + i0 + off + 16 * kg) + ri;
        float x[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) x[j] = sg * src[4 * j];
        unsigned char *r = bt + b * BTILE + kg * (32 * NCOL) + c * 16;
        store_row8(r, r + NCOL * 16, x);
    }
}

template <int SPIN, int NSTG, int SCH>
__global__ void __launch_bounds__(TC_M) k_leg_synth_tc(const LegArgs<float> a) {
    typedef TcCfg<SPIN> Cfg;
    typedef TcLayout<SPIN, NSTG, SCH> Lay;
    constexpr int NCOL = Cfg::NCOL;
    extern __shared__ __align__(1024) unsigned char smem[];
    float2 *s_alm = reinterpret_cast<float2 *>(smem + Lay::ALM);
    float2 *s_rec = reinterpret_cast<float2 *>(smem + Lay::COEF);
    float4 *s_s2c = reinterpret_cast<float4 *>(smem + Lay::COEF);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + Lay::BARS);
    uint32_t *s_tmem = reinterpret_cast<uint32_t *>(smem + Lay::TMEMA);
    int *s_red = reinterpret_cast<int *>(smem + Lay::RED);

    const int tid = threadIdx.x, warp = tid >> 5;
    const int m = blockIdx.y;
    const int L = a.lmax;
    const int map0 = blockIdx.z * TC_NMT;
    const int nm = min(TC_NMT, a.nmaps - map0);
    const int64_t base = (int64_t)m * (2 * L + 1 - m) / 2;

    PairState<float, 1> S;
    int warp_lo, warp_hi;
    load_pairs<float, 1, SPIN>(a, blockIdx.x, m, S, warp_lo, warp_hi);
    const int lo = cta_min(warp_lo, s_red);
    const int pr = S.pr[0];
    const int rn = pr, rs = a.nring - 1 - pr;

    if (lo > L) {   // no significant l for any pair of this CTA: zero output
        if (pr < a.npairs) {
            for (int k = 0; k < nm; ++k) {
                for (int c = 0; c < (SPIN == 2 ? 2 : 1); ++c) {
                    const int row = SPIN == 2 ? 2 * (map0 + k) + c : map0 + k;
                    float2 *out = a.F + (int64_t)row * a.nring * (L + 1) + m;
                    out[(int64_t)rn * (L + 1)] = make_float2(0.f, 0.f);
                    if (rs != rn) out[(int64_t)rs * (L + 1)] = make_float2(0.f, 0.f);
                }
            }
        }
        return;
    }

    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bars[0])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bars[1])));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(s_tmem)),
                     "r"(Cfg::TMEM));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = *s_tmem;

    bool ok = true;
    int chunk = 0;
    const int l_begin = m + ((lo - m) & ~31);   // chunks start at l - m = 0 mod 32
    for (int c0 = l_begin; c0 <= L; c0 += SCH) {
        // ---- stage coefficients and beam-weighted alm of l = c0 .. c0 + SCH - 1
        __syncthreads();
        for (int i = tid; i < SCH; i += TC_M) {
            const int l = c0 + i;
            const bool in = l <= L;
            const int64_t idx = base + l;
            if (SPIN == 2) s_s2c[i] = in ? a.s2c[idx] : make_float4(0.f, 0.f, 0.f, 0.f);
            else s_rec[i] = in ? a.rec[idx] : make_float2(0.f, 0.f);
            const float bm = (in && a.beam) ? a.beam[l] : 1.f;
#pragma unroll
            for (int k = 0; k < Cfg::NA; ++k) {
                float2 v = make_float2(0.f, 0.f);
                const int mk = SPIN == 2 ? k / 2 : k;
                if (in && mk < nm) {
                    const int64_t row = (int64_t)(map0 + mk) * a.rs + (SPIN == 2 ? (k & 1) : 0);
                    v = a.alm[row * a.nalm + idx];
                    if (m == 0) v.y = 0.f;
                    v.x *= bm;
                    v.y *= bm;
                }
                s_alm[k * Lay::ALMS + i] = v;
            }
        }
        __syncthreads();
        for (int q0 = c0; q0 < c0 + SCH && q0 <= L; q0 += 32, ++chunk) {
            const int sidx = chunk % NSTG;
            unsigned char *stg = smem + sidx * Lay::STAGE;
            // the MMAs of chunk - NSTG read this stage: wait for their commit
            // (the k-th commit on a barrier completes its phase k)
            if (chunk >= NSTG) ok = mbar_wait(&bars[sidx], ((chunk - NSTG) / NSTG) & 1) && ok;
            const int i0 = q0 - c0;
            // injection steps only where some pair of the warp starts in this chunk
            const bool starts = (S.ls[0] >= q0 && S.ls[0] < q0 + 32) ||
                                (SPIN == 2 && S.lsb[0] >= q0 && S.lsb[0] < q0 + 32);
            if (q0 <= warp_hi && __any_sync(0xffffffffu, starts)) gen_atiles<SPIN, true>(S, s_rec, s_s2c, i0, q0, stg);
            else gen_atiles<SPIN, false>(S, s_rec, s_s2c, i0, q0, stg);
            gen_btiles<SPIN, Lay::ALMS>(s_alm, i0, stg + Cfg::NTA * TC_ATILE);
            asm volatile("fence.proxy.async.shared::cta;");
            __syncthreads();
            if (tid == 0) {
                asm volatile("tcgen05.fence::after_thread_sync;");
                const uint32_t sa = smem_u32(stg);
                const uint32_t sb = sa + Cfg::NTA * TC_ATILE;
                const uint32_t full = idesc_bf16(TC_M, 2 * NCOL), half = idesc_bf16(TC_M, NCOL);
                const uint32_t acc = chunk > 0;
                auto A = [&](int t) { return sdesc(sa + t * TC_ATILE, 2048, 128); };
                auto B = [&](int t) { return sdesc(sb + t * Lay::BTILE, 32 * NCOL, 128); };
                if (SPIN == 0) {
                    // D_E (columns 0 .. 2 NCOL) and D_O (2 NCOL .. 4 NCOL)
                    mma_bf16(tmem, A(0), B(0), full, acc);
                    mma_bf16(tmem, A(1), B(0), half, 1);
                    mma_bf16(tmem + 2 * NCOL, A(2), B(1), full, acc);
                    mma_bf16(tmem + 2 * NCOL, A(3), B(1), half, 1);
                } else {
                    // symmetric part: lw even with W even, lx odd with X odd;
                    // antisymmetric part: lw odd with W odd, lx even with X even
                    mma_bf16(tmem, A(0), B(0), full, acc);
                    mma_bf16(tmem, A(1), B(0), half, 1);
                    mma_bf16(tmem, A(6), B(3), full, 1);
                    mma_bf16(tmem, A(7), B(3), half, 1);
                    mma_bf16(tmem + 2 * NCOL, A(2), B(1), full, acc);
                    mma_bf16(tmem + 2 * NCOL, A(3), B(1), half, 1);
                    mma_bf16(tmem + 2 * NCOL, A(4), B(2), full, 1);
                    mma_bf16(tmem + 2 * NCOL, A(5), B(2), half, 1);
                }
                mma_commit(&bars[sidx]);
            }
        }
    }
    // ---- the last commit covers every MMA issued before it
    const int last = chunk - 1;
    ok = mbar_wait(&bars[last % NSTG], (last / NSTG) & 1) && ok;
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (!ok && tid == 0 && a.err) atomicExch(a.err, 1);

    // ---- epilogue: this thread's TMEM lane is its ring pair
    const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
    float d0[32], d1[32];
    if (SPIN == 0) {
        tmem_ld32(trow, d0);        // D_E: [0, 16) hi*hi + lo*hi, [16, 32) hi*lo
        tmem_ld32(trow + 32, d1);   // D_O
        if (ok && pr < a.npairs) {
#pragma unroll
            for (int k = 0; k < TC_NMT; ++k) {
                if (k >= nm) break;
                const float er = d0[2 * k] + d0[NCOL + 2 * k], ei = d0[2 * k + 1] + d0[NCOL + 2 * k + 1];
                const float orr = d1[2 * k] + d1[NCOL + 2 * k], oi = d1[2 * k + 1] + d1[NCOL + 2 * k + 1];
                float2 *out = a.F + (int64_t)(map0 + k) * a.nring * (L + 1) + m;
                out[(int64_t)rn * (L + 1)] = make_float2(er + orr, ei + oi);
                if (rs != rn) out[(int64_t)rs * (L + 1)] = make_float2(er - orr, ei - oi);
            }
        }
    } else {
        // symmetric part S (columns 0 .. 64), antisymmetric part X (64 .. 128)
        float s2[32], x2[32];
        tmem_ld32(trow, d0);         // S hi*hi + lo*hi
        tmem_ld32(trow + 32, d1);    // S hi*lo
#pragma unroll
        for (int c = 0; c < 32; ++c) s2[c] = d0[c] + d1[c];
        tmem_ld32(trow + 64, d0);
        tmem_ld32(trow + 96, d1);
#pragma unroll
        for (int c = 0; c < 32; ++c) x2[c] = d0[c] + d1[c];
        if (ok && pr < a.npairs) {
#pragma unroll
            for (int k = 0; k < TC_NMT; ++k) {
                if (k >= nm) break;
                float2 *oq = a.F + (int64_t)(2 * (map0 + k)) * a.nring * (L + 1) + m;
                float2 *ou = a.F + (int64_t)(2 * (map0 + k) + 1) * a.nring * (L + 1) + m;
                const int c = 4 * k;
                oq[(int64_t)rn * (L + 1)] = make_float2(s2[c] + x2[c], s2[c + 1] + x2[c + 1]);
                ou[(int64_t)rn * (L + 1)] = make_float2(s2[c + 2] + x2[c + 2], s2[c + 3] + x2[c + 3]);
                if (rs != rn) {
                    oq[(int64_t)rs * (L + 1)] = make_float2(s2[c] - x2[c], s2[c + 1] - x2[c + 1]);
                    ou[(int64_t)rs * (L + 1)] = make_float2(s2[c + 2] - x2[c + 2], s2[c + 3] - x2[c + 3]);
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(Cfg::TMEM));
}

template <int SPIN, int NSTG, int SCH>
int launch_synth_tc(Plan *p, const float2 *alm, int rs, int nmaps, const float *beam, float2 *F,
                    cudaStream_t st) {
    LegArgs<float> a = leg_make_args<float>(p);
    a.alm = alm;
    a.rs = rs;
    a.F = F;
    a.beam = beam;
    a.nmaps = nmaps;
    a.err = p->d_flag;
    const int smem = TcLayout<SPIN, NSTG, SCH>::BYTES;
    auto kern = k_leg_synth_tc<SPIN, NSTG, SCH>;
    SHTG_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    dim3 grid((p->npairs + TC_M - 1) / TC_M, p->lmax + 1, (nmaps + TC_NMT - 1) / TC_NMT);
    prof_begin(p, K_LEG_SYN32, st);
    kern<<<grid, TC_M, smem, st>>>(a);
    prof_end(p, st);
    SHTG_CHECK_LAUNCH("k_leg_synth_tc");
    return SHTG_OK;
}

// FP32 recurrence state before every l = m + 32 t of every (m, ring pair):
// the same steps (rstep / step2 with the same injections) as the Legendre
// kernels, so a kernel that restarts from an entry reproduces the values of
// one continuous run bit for bit.  One thread per (m, pair); entries
// [m][t][pair] so that a warp's stores are contiguous.
template <int SPIN>
__global__ void __launch_bounds__(LEG_THREADS) k_tile_states(const LegArgs<float> a, const int64_t *toff,
                                                             float2 *out0, float4 *out2) {
    const int m = blockIdx.y;
    const int L = a.lmax;
    PairState<float, 1> S;
    int wlo, whi;
    load_pairs<float, 1, SPIN>(a, blockIdx.x, m, S, wlo, whi);
    const int pr = S.pr[0];
    if (pr >= a.npairs) return;
    const int64_t base = (int64_t)m * (2 * L + 1 - m) / 2;
    const int64_t o = toff[m] * a.npairs + pr;
    for (int l = m; l <= L; ++l) {
        if (((l - m) & 31) == 0) {
            const int64_t e = o + (int64_t)((l - m) >> 5) * a.npairs;
            if (SPIN == 2) out2[e] = make_float4(S.a1[0], S.a2[0], S.b1[0], S.b2[0]);
            else out0[e] = make_float2(S.a1[0], S.a2[0]);
        }
        stepx<float, 1, SPIN, true>(S, a.rec + base, a.s2c + base, l, l);
    }
}

}  // namespace

int build_tile_states(Plan *p) {
    const int L = p->lmax;
    std::vector<int64_t> toff(L + 2);
    toff[0] = 0;
    for (int m = 0; m <= L; ++m) toff[m + 1] = toff[m] + (L + 1 - m + 31) / 32;
    const size_t nent = (size_t)toff[L + 1] * p->npairs;
    auto alloc = [&](void **ptr, size_t bytes) -> int {
        cudaError_t e = cudaMalloc(ptr, bytes);
        if (e != cudaSuccess) {
            *ptr = nullptr;
            cudaGetLastError();
            set_error(std::string("cudaMalloc of ") + std::to_string(bytes) +
                      " bytes (recurrence tile states) failed: " + cudaGetErrorString(e));
            return SHTG_ERR_NOMEM;
        }
        p->device_bytes += (int64_t)bytes;
        return SHTG_OK;
    };
    SHTG_TRY(alloc((void **)&p->d_toff, sizeof(int64_t) * toff.size()));
    SHTG_CUDA(cudaMemcpy(p->d_toff, toff.data(), sizeof(int64_t) * toff.size(), cudaMemcpyHostToDevice));
    SHTG_TRY(alloc((void **)&p->d_tst0, sizeof(float2) * nent));
    LegArgs<float> a = leg_make_args<float>(p);
    dim3 grid((p->npairs + LEG_THREADS - 1) / LEG_THREADS, L + 1);
    k_tile_states<0><<<grid, LEG_THREADS>>>(a, p->d_toff, p->d_tst0, nullptr);
    SHTG_CHECK_LAUNCH("k_tile_states");
    if (p->flags & SHTG_SPIN2) {
        SHTG_TRY(alloc((void **)&p->d_tst2, sizeof(float4) * nent));
        k_tile_states<2><<<grid, LEG_THREADS>>>(a, p->d_toff, nullptr, p->d_tst2);
        SHTG_CHECK_LAUNCH("k_tile_states");
    }
    SHTG_CUDA(cudaDeviceSynchronize());
    return SHTG_OK;
}

namespace {

// ===================================================== transpose (Y^T)
// c_lm = sum_r lambda_lm(theta_r) G_r(m) for one m and a range of 512 l:
// rows = l (two 128-row tiles per 256 l: l - m even, l - m odd), K = ring
// pairs in stages of 16, columns = (map, output) with the north / south
// combination G_N + G_S (rows with the parity of lambda) or G_N - G_S
// folded into the B tiles.  A tiles hold the recurrence values l-major
// (MN-major core matrices: 8 pairs x 8 consecutive rows of one class), which
// is how a thread produces them: thread (pair p, segment s) runs the FP32
// recurrence of pair p over 32 l from the tabulated state at l = m + 32 t.
// The CTA accumulates over all ring pairs in tensor memory, so every alm is
// written once, by one CTA, without atomics.
constexpr int TA_K = 16;        // ring pairs per stage (MMA K)
template <int SPIN> struct TaCfg;
template <> struct TaCfg<0> {
    static constexpr int NO = 16, NAT = 4, NBT = 2, TMEM = 64;
};
template <> struct TaCfg<2> {
    static constexpr int NO = 32, NAT = 8, NBT = 4, TMEM = 128;
};
// Shared memory of the transpose CTA (TR 256-l tiles): NAS A buffers (the
// tiles of one (stage, 256-l tile) unit), NBS B buffers (one per stage of 16
// pairs), the ring data of one stage, the coefficients of 256 TR l, two
// mbarriers and the TMEM address.  The ring data are consumed when the
// stage's B tiles are built, so the next stage's copy is issued right after
// (it overlaps with the stage's A generation) and one buffer suffices.
// Fewer buffers shrink the CTA (spin 2 with one A and one B buffer: 53 KB
// with two 256-l tiles, 49 KB with one) so that four CTAs share an SM.
template <int SPIN, int NAS, int NBS, int TR> struct TaLayout {
    static constexpr int BT = 64 * TaCfg<SPIN>::NO;                         // B tile: 2 NO rows x 16 K bf16
    static constexpr int ASTAGE = TaCfg<SPIN>::NAT * TC_ATILE;
    static constexpr int BSTAGE = TaCfg<SPIN>::NBT * BT;
    static constexpr int BOFF = NAS * ASTAGE;
    // ring data of one stage: [pair][north rows | south rows] float2 with pair
    // stride GS = 2 NROW + 2: the B-tile builder's warp reads 8 consecutive
    // floats per K pair and its four K pairs sit 4 GS = 8 (mod 32) floats
    // apart, so every load hits 32 distinct banks
    static constexpr int NROW = SPIN == 2 ? 2 * TC_NMT : TC_NMT;
    static constexpr int GS = 2 * NROW + 2;
    static constexpr int GBUF = ((TA_K * GS * 8) + 15) & ~15;
    static constexpr int GOFF = BOFF + NBS * BSTAGE;
    static constexpr int COEF = GOFF + GBUF;
    // coefficients of 256 TR l, one padding entry after every 32 (ta_cpad)
    static constexpr int BARS = COEF + 264 * TR * (SPIN == 2 ? 16 : 8);
    static constexpr int TMEM = TR * TaCfg<SPIN>::TMEM / 2;   // 2 NO columns per 256-l tile
    static constexpr int TMEMA = BARS + 16;
    static constexpr int BYTES = TMEMA + 16;
};

// Shared index of the recurrence coefficients of l = lbase + i in the
// transpose: one padding entry after every 32, so the two 32-l segments that
// a warp's threads step through at once (256 or 512 bytes apart unpadded,
// the same banks) read distinct banks.
__device__ __forceinline__ int ta_cpad(int i) { return i + (i >> 5); }

// MN-major A (bit 15), K-major B, bf16 in, FP32 accumulator
__host__ __device__ constexpr uint32_t idesc_bf16_amn(int m, int n) {
    return idesc_bf16(m, n) | (1u << 15);
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
          "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Start data of one ring pair for m (from the FP64 start states) and the
// tabulated FP32 recurrence state before l0 = m + 32 t.
struct PairStart {
    int ls, lsb;
    float s0, s1, s2, s3, u;
};
template <int SPIN>
__device__ __forceinline__ PairStart load_pair_start(const LegArgs<float> &a, int m, int pr) {
    PairStart q;
    q.ls = q.lsb = a.lmax + 1;
    q.s0 = q.s1 = q.s2 = q.s3 = 0.f;
    q.u = 1.f;
    if (pr < a.npairs) {
        const int64_t o = (int64_t)m * a.npairs + pr;
        q.u = a.u[pr];
        if (SPIN == 2) {
            const int2 l2 = a.ls2[o];
            const float4 s4 = a.st2[o];
            q.ls = l2.x;
            q.lsb = l2.y;
            q.s0 = s4.x;
            q.s1 = s4.y;
            q.s2 = s4.z;
            q.s3 = s4.w;
        } else {
            const float2 s2 = a.st[o];
            q.ls = a.ls[o];
            q.s0 = s2.x;
            q.s1 = s2.y;
        }
    }
    return q;
}
template <int SPIN>
__device__ __forceinline__ float4 load_tile_state(const LegArgs<float> &a, int m, int pr, int l0) {
    if (pr >= a.npairs || l0 > a.lmax) return make_float4(0.f, 0.f, 0.f, 0.f);
    const int64_t e = (a.toff[m] + ((l0 - m) >> 5)) * a.npairs + pr;
    if (SPIN == 2) return a.tst2[e];
    const float2 t = a.tst0[e];
    return make_float4(t.x, t.y, 0.f, 0.f);
}

// A tiles of one (stage, 256-l tile): this thread's pair (column pin of the
// K = 16 slice) over l = l0 .. l0 + 31, l0 = tstart + 32 seg, from state ts;
// values of class E (l - m even) go to rows 16 seg + j of the E tiles, class
// O to the same rows of the O tiles.  Pairs beyond npairs and l beyond lmax
// give 0.  INJ: some pair of the warp starts its recurrence inside the
// segment (the tabulated state already holds every earlier start).
template <int SPIN, bool INJ>
__device__ __forceinline__ void gen_atiles_ana(const PairStart &q, const float4 ts, const bool live, const int pin,
                                               const int seg, const int l0, const int lbase,
                                               const float2 *s_rec, const float4 *s_s2c, unsigned char *at) {
    PairState<float, 1> S;
    S.u[0] = q.u;
    S.ls[0] = q.ls;
    S.lsb[0] = q.lsb;
    S.s0[0] = q.s0;
    S.s1[0] = q.s1;
    S.s2[0] = q.s2;
    S.s3[0] = q.s3;
    S.a1[0] = ts.x;
    S.a2[0] = ts.y;
    S.b1[0] = ts.z;
    S.b2[0] = ts.w;
    const int kg = pin >> 3, krow = pin & 7;
    // padded shared index of l0 + d: l0 - lbase is a multiple of 32 and d <= 31,
    // so ta_cpad(l0 - lbase + d) = ta_cpad(l0 - lbase) + d
    const int cb = ta_cpad(l0 - lbase);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        // rows 16 seg + 8 h .. + 7: core matrix (M group 2 seg + h, K group kg)
        unsigned char *t = at + (kg * 16 + 2 * seg + h) * 128 + krow * 16;
        if (SPIN == 0) {
            float e[8], o[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int d = 16 * h + 2 * i;
                e[i] = o[i] = 0.f;
                if (live) {
                    stepx<float, 1, 0, INJ>(S, s_rec, s_s2c, cb + d, l0 + d);
                    e[i] = S.a1[0];
                    stepx<float, 1, 0, INJ>(S, s_rec, s_s2c, cb + d + 1, l0 + d + 1);
                    o[i] = S.a1[0];
                }
            }
            store_row8(t, t + TC_ATILE, e);                    // E hi, E lo
            store_row8(t + 2 * TC_ATILE, t + 3 * TC_ATILE, o);  // O hi, O lo
        } else {
            float wE[8], wO[8], xE[8], xO[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int d = 16 * h + 2 * i;
                wE[i] = wO[i] = xE[i] = xO[i] = 0.f;
                if (live) {
                    stepx<float, 1, 2, INJ>(S, s_rec, s_s2c, cb + d, l0 + d);
                    wE[i] = S.a1[0] + S.b1[0];
                    xE[i] = S.a1[0] - S.b1[0];
                    stepx<float, 1, 2, INJ>(S, s_rec, s_s2c, cb + d + 1, l0 + d + 1);
                    wO[i] = S.a1[0] + S.b1[0];
                    xO[i] = S.a1[0] - S.b1[0];
                }
            }
            store_row8(t, t + TC_ATILE, wE);
            store_row8(t + 2 * TC_ATILE, t + 3 * TC_ATILE, wO);
            store_row8(t + 4 * TC_ATILE, t + 5 * TC_ATILE, xE);
            store_row8(t + 6 * TC_ATILE, t + 7 * TC_ATILE, xO);
        }
    }
}

// Asynchronous copy (cp.async) of the ring data of stage ps into sg:
// element (pair p, row q, ring z) at sg[p GS + z NROW + q]; rows are the maps of
// this CTA (spin 2: Q, U of each); zeros for pairs beyond npairs, missing
// maps and the south ring of the equator pair.
template <int SPIN>
__device__ __forceinline__ void stage_ring_data(const LegArgs<float> &a, const int m, const int ps, const int map0,
                                                const int nm, float2 *sg) {
    typedef TaLayout<SPIN, 1, 1, 1> Lay;   // (ring-data geometry only)
    const int L = a.lmax;
    const int64_t rowsz = (int64_t)a.nring * (L + 1);
    const int nrow = SPIN == 2 ? 2 * nm : nm;
    for (int it = threadIdx.x; it < TA_K * Lay::NROW * 2; it += TC_M) {
        const int z = it & 1;
        const int q = (it >> 1) % Lay::NROW;
        const int pp = it / (2 * Lay::NROW);
        const int pr = ps * TA_K + pp;
        float2 *dst = sg + pp * Lay::GS + z * Lay::NROW + q;
        const int rn = pr, rs = a.nring - 1 - pr;
        if (pr < a.npairs && q < nrow && !(z && rs == rn)) {
            const int64_t grow = (SPIN == 2 ? 2 * map0 : map0) + q;
            const float2 *src = a.F + grow * rowsz + (int64_t)(z ? rs : rn) * (L + 1) + m;
            asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
        } else {
            *dst = make_float2(0.f, 0.f);
        }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}

// B tiles of one stage from the staged ring data.  Tile b: spin 0 -> rows
// for class b (0: G_N + G_S, 1: G_N - G_S) with columns (re, im) per map;
// spin 2 -> b = 2 x + class' with lw columns (x = 0, class' = b) and lx
// columns (x = 1, class' = the other one):
//   E^ = -lw G_Q - i lx G_U,  B^ = i lx G_Q - lw G_U
// (columns E re, E im, B re, B im per map).  hi at row c, lo at row NO + c.
// One thread per (K group kg, K pair kq, column c) writes that column's word
// (two consecutive ring pairs) in every tile: a warp covers 8 consecutive
// columns x 4 K pairs, i.e. 32 distinct banks per store, and reads only the
// two scalars per ring pair that its column needs.
template <int SPIN>
__device__ __forceinline__ void gen_btiles_ana(const float2 *sg, unsigned char *bt) {
    typedef TaLayout<SPIN, 1, 1, 1> Lay;   // (tile geometry only)
    constexpr int NO = TaCfg<SPIN>::NO, BT = Lay::BT;
    const float *sgf = reinterpret_cast<const float *>(sg);
    for (int it = threadIdx.x; it < 8 * NO; it += TC_M) {
        const int kq = it & 3;
        const int c = (it >> 2) % NO;
        const int kg = it / (4 * NO);
        const int k0 = 8 * kg + 2 * kq;
        unsigned char *tile = bt + kg * (32 * NO) + kq * 4;
        if (SPIN == 0) {
            // column c: component c & 1 of map c >> 1, i.e. float c of the
            // north rows and float 2 NROW + c (the south rows)
            float vp[2], vm[2];
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const float *g = sgf + 2 * (k0 + q) * Lay::GS;
                const float gn = g[c], gs = g[2 * Lay::NROW + c];
                vp[q] = gn + gs;
                vm[q] = gn + (-1.f) * gs;
            }
            uint32_t hi, lo;
            split2(vp[0], vp[1], hi, lo);
            *reinterpret_cast<uint32_t *>(tile + c * 16) = hi;
            *reinterpret_cast<uint32_t *>(tile + (NO + c) * 16) = lo;
            split2(vm[0], vm[1], hi, lo);
            *reinterpret_cast<uint32_t *>(tile + BT + c * 16) = hi;
            *reinterpret_cast<uint32_t *>(tile + BT + (NO + c) * 16) = lo;
        } else {
            // column c = 4 k + comp of map k; the lw tiles take w = (-Q re,
            // -Q im, -U re, -U im)[comp], the lx tiles x = (U im, -U re,
            // -Q im, Q re)[comp], each as N + S or N - S
            const int k = c >> 2, comp = c & 3;
            const int wf = comp < 2 ? 0 : 1, wc = comp & 1;            // field (Q 0, U 1), re / im
            const int xf = comp < 2 ? 1 : 0, xc = (comp & 1) ^ 1;
            const float xs = (comp == 1 || comp == 2) ? -1.f : 1.f;
            // (row 2 k + field of the north rows at float 2 (2 k + field) + re/im,
            // the south rows 2 NROW floats later)
            float wp[2], wm[2], xp[2], xm[2];
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const float *g = sgf + 2 * (k0 + q) * Lay::GS + 4 * k;
                const float wn = g[2 * wf + wc], wsv = g[2 * Lay::NROW + 2 * wf + wc];
                const float xn = g[2 * xf + xc], xsv = g[2 * Lay::NROW + 2 * xf + xc];
                wp[q] = -(wn + wsv);
                wm[q] = -(wn + (-1.f) * wsv);
                xp[q] = xs * (xn + xsv);
                xm[q] = xs * (xn + (-1.f) * xsv);
            }
            uint32_t hi, lo;
            split2(wp[0], wp[1], hi, lo);   // b = 0: lw, class 0
            *reinterpret_cast<uint32_t *>(tile + c * 16) = hi;
            *reinterpret_cast<uint32_t *>(tile + (NO + c) * 16) = lo;
            split2(wm[0], wm[1], hi, lo);   // b = 1: lw, class 1
            *reinterpret_cast<uint32_t *>(tile + BT + c * 16) = hi;
            *reinterpret_cast<uint32_t *>(tile + BT + (NO + c) * 16) = lo;
            split2(xm[0], xm[1], hi, lo);   // b = 2: lx, class 1
            *reinterpret_cast<uint32_t *>(tile + 2 * BT + c * 16) = hi;
            *reinterpret_cast<uint32_t *>(tile + 2 * BT + (NO + c) * 16) = lo;
            split2(xp[0], xp[1], hi, lo);   // b = 3: lx, class 0
            *reinterpret_cast<uint32_t *>(tile + 3 * BT + c * 16) = hi;
            *reinterpret_cast<uint32_t *>(tile + 3 * BT + (NO + c) * 16) = lo;
        }
    }
}

template <int SPIN, int NAS, int NBS, int TR>
__global__ void __launch_bounds__(TC_M) k_leg_analysis_tc(const LegArgs<float> a) {
    typedef TaCfg<SPIN> Cfg;
    typedef TaLayout<SPIN, NAS, NBS, TR> Lay;
    constexpr int NO = Cfg::NO;
    extern __shared__ __align__(1024) unsigned char smem[];
    float2 *s_rec = reinterpret_cast<float2 *>(smem + Lay::COEF);
    float4 *s_s2c = reinterpret_cast<float4 *>(smem + Lay::COEF);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + Lay::BARS);
    uint32_t *s_tmem = reinterpret_cast<uint32_t *>(smem + Lay::TMEMA);

    const int tid = threadIdx.x, warp = tid >> 5;
    const int m = blockIdx.y;
    const int L = a.lmax;
    const int lbase = m + blockIdx.x * (256 * TR);
    if (lbase > L) return;
    const int ntile = min(TR, (L - lbase) / 256 + 1);
    const int lend = min(L, lbase + 256 * TR - 1);
    const int map0 = blockIdx.z * TC_NMT;
    const int nm = min(TC_NMT, a.nmaps - map0);
    const int64_t base = (int64_t)m * (2 * L + 1 - m) / 2;

    for (int i = tid; i < 256 * TR; i += TC_M) {
        const int l = lbase + i;
        const bool in = l <= L;
        if (SPIN == 2) s_s2c[ta_cpad(i)] = in ? a.s2c[base + l] : make_float4(0.f, 0.f, 0.f, 0.f);
        else s_rec[ta_cpad(i)] = in ? a.rec[base + l] : make_float2(0.f, 0.f);
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bars[0])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bars[1])));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(s_tmem)),
                     "r"(Lay::TMEM));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = *s_tmem;

    const int pin = tid & (TA_K - 1), seg = tid >> 4;
    const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
    float2 *sgb = reinterpret_cast<float2 *>(smem + Lay::GOFF);
    int *s_first = reinterpret_cast<int *>(smem + Lay::TMEMA + 4);

    // first stage with a pair whose recurrence starts at or before lend; the
    // start l falls towards the equator, so every later stage is worked too
    // (a stage without significant values contributes exact zeros)
    if (tid == 0) *s_first = a.npairs;
    __syncthreads();
    {
        int first = a.npairs;
        for (int pr = tid; pr < a.npairs; pr += TC_M) {
            const int64_t o = (int64_t)m * a.npairs + pr;
            int lsp;
            if (SPIN == 2) {
                const int2 q = a.ls2[o];
                lsp = min(q.x, q.y);
            } else {
                lsp = a.ls[o];
            }
            if (lsp <= lend) {
                first = pr;
                break;
            }
        }
        if (first < a.npairs) atomicMin(s_first, first);
    }
    __syncthreads();
    const int s0 = *s_first / TA_K;
    const int nps = (a.npairs + TA_K - 1) / TA_K;
    const int nst = s0 < nps ? nps - s0 : 0;

    bool ok = true;
    int unit = 0, waited = -1;
    int last_unit[NBS];            // last unit that read each B buffer
#pragma unroll
    for (int i = 0; i < NBS; ++i) last_unit[i] = -1;
    PairStart pst{}, pnext{};
    float4 tcur = make_float4(0.f, 0.f, 0.f, 0.f);
    if (nst > 0) {
        stage_ring_data<SPIN>(a, m, s0, map0, nm, sgb);
        pst = load_pair_start<SPIN>(a, m, s0 * TA_K + pin);
        tcur = load_tile_state<SPIN>(a, m, s0 * TA_K + pin, lbase + 32 * seg);
    }
    for (int si = 0; si < nst; ++si) {
        const int ps = s0 + si;
        const int pr = ps * TA_K + pin;
        const bool more = si + 1 < nst;
        if (more) pnext = load_pair_start<SPIN>(a, m, pr + TA_K);   // in flight during this stage
        asm volatile("cp.async.wait_group 0;" ::: "memory");          // this stage's ring data
        __syncthreads();
        // unit u commits to barrier u % NAS, completing its phase u / NAS; the
        // commits complete in order, so waiting for u covers every unit before it
        const int bsel = si % NBS;
        unsigned char *bt = smem + Lay::BOFF + bsel * Lay::BSTAGE;
        if (last_unit[bsel] > waited) {   // the stage NBS back read this B buffer
            const int u = last_unit[bsel];
            ok = mbar_wait(&bars[u % NAS], (u / NAS) & 1) && ok;
            waited = u;
        }
        gen_btiles_ana<SPIN>(sgb, bt);
        for (int r = 0; r < ntile; ++r) {
            const int asel = unit % NAS;
            unsigned char *at = smem + asel * Lay::ASTAGE;
            if (unit >= NAS && unit - NAS > waited) {   // the unit NAS back read this A buffer
                ok = mbar_wait(&bars[asel], ((unit - NAS) / NAS) & 1) && ok;
                waited = unit - NAS;
            }
            const int tstart = lbase + 256 * r;
            const int l0 = tstart + 32 * seg;
            // state of the next unit: (this stage, next tile) or (next stage, first tile)
            float4 tnext = make_float4(0.f, 0.f, 0.f, 0.f);
            if (r + 1 < ntile) tnext = load_tile_state<SPIN>(a, m, pr, l0 + 256);
            else if (more) tnext = load_tile_state<SPIN>(a, m, pr + TA_K, lbase + 32 * seg);
            const bool live = pr < a.npairs && l0 <= L;
            const bool starts = (pst.ls >= l0 && pst.ls < l0 + 32) || (SPIN == 2 && pst.lsb >= l0 && pst.lsb < l0 + 32);
            if (__any_sync(0xffffffffu, live && starts))
                gen_atiles_ana<SPIN, true>(pst, tcur, live, pin, seg, l0, lbase, s_rec, s_s2c, at);
            else
                gen_atiles_ana<SPIN, false>(pst, tcur, live, pin, seg, l0, lbase, s_rec, s_s2c, at);
            tcur = tnext;
            asm volatile("fence.proxy.async.shared::cta;");
            __syncthreads();
            // every thread has built this stage's B tiles: the ring-data buffer
            // takes the next stage's copy, in flight during the stage's units
            if (r == 0 && more) stage_ring_data<SPIN>(a, m, ps + 1, map0, nm, sgb);
            if (tid == 0) {
                asm volatile("tcgen05.fence::after_thread_sync;");
                const uint32_t sa = smem_u32(at), sb = smem_u32(bt);
                const uint32_t id = idesc_bf16_amn(TC_M, NO);
                const uint32_t acc = si > 0;
                auto A = [&](int t) { return sdesc(sa + t * TC_ATILE, 2048, 128); };
                auto Bh = [&](int t) { return sdesc(sb + t * Lay::BT, 32 * NO, 128); };
                auto Bl = [&](int t) { return sdesc(sb + t * Lay::BT + (NO / 8) * 128, 32 * NO, 128); };
                const uint32_t dE = tmem + r * 2 * NO, dO = dE + NO;
                if (SPIN == 0) {
                    mma_bf16(dE, A(0), Bh(0), id, acc);
                    mma_bf16(dE, A(0), Bl(0), id, 1);
                    mma_bf16(dE, A(1), Bh(0), id, 1);
                    mma_bf16(dO, A(2), Bh(1), id, acc);
                    mma_bf16(dO, A(2), Bl(1), id, 1);
                    mma_bf16(dO, A(3), Bh(1), id, 1);
                } else {
                    mma_bf16(dE, A(0), Bh(0), id, acc);   // lw even rows, W from G_N + G_S
                    mma_bf16(dE, A(0), Bl(0), id, 1);
                    mma_bf16(dE, A(1), Bh(0), id, 1);
                    mma_bf16(dE, A(4), Bh(2), id, 1);     // lx even rows, X from G_N - G_S
                    mma_bf16(dE, A(4), Bl(2), id, 1);
                    mma_bf16(dE, A(5), Bh(2), id, 1);
                    mma_bf16(dO, A(2), Bh(1), id, acc);
                    mma_bf16(dO, A(2), Bl(1), id, 1);
                    mma_bf16(dO, A(3), Bh(1), id, 1);
                    mma_bf16(dO, A(6), Bh(3), id, 1);
                    mma_bf16(dO, A(6), Bl(3), id, 1);
                    mma_bf16(dO, A(7), Bh(3), id, 1);
                }
                mma_commit(&bars[asel]);
            }
            last_unit[bsel] = unit;
            ++unit;
        }
        pst = pnext;
    }
    if (unit > 0 && unit - 1 > waited) ok = mbar_wait(&bars[(unit - 1) % NAS], ((unit - 1) / NAS) & 1) && ok;
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (!ok && tid == 0 && a.err) atomicExch(a.err, 1);

    // ---- epilogue: lane = row i, l = tstart + 2 i (E tile) and + 1 (O tile)
#pragma unroll
    for (int r = 0; r < TR; ++r) {
        if (r >= ntile) break;
        const int tstart = lbase + 256 * r;
#pragma unroll
        for (int cls = 0; cls < 2; ++cls) {
            const int l = tstart + 2 * tid + cls;
            float d[NO];
            if (SPIN == 0) tmem_ld16(trow + r * 2 * NO + cls * NO, *reinterpret_cast<float(*)[16]>(d));
            else tmem_ld32(trow + r * 2 * NO + cls * NO, *reinterpret_cast<float(*)[32]>(d));
            if (!ok || l > L) continue;
            const float bm = (a.beam ? a.beam[l] : 1.f) * ((a.vjp && m > 0) ? 2.f : 1.f);
#pragma unroll
            for (int k = 0; k < TC_NMT; ++k) {
                if (k >= nm) break;
#pragma unroll
                for (int c = 0; c < (SPIN == 2 ? 2 : 1); ++c) {
                    const int j = SPIN == 2 ? 4 * k + 2 * c : 2 * k;
                    float re = 0.f, im = 0.f;
                    if (nst > 0) {
                        re = d[j] * bm;
                        im = m == 0 ? 0.f : d[j + 1] * bm;
                    }
                    const int64_t row = (int64_t)(map0 + k) * a.rs + c;
                    float2 *dst = const_cast<float2 *>(a.alm) + row * a.nalm + base + l;
                    *dst = make_float2(re, im);
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(Lay::TMEM));
}

template <int SPIN, int NAS, int NBS, int TR>
int launch_analysis_tc(Plan *p, const float2 *G, int nmaps, const float *beam, float2 *alm, int rs,
                       cudaStream_t st, int vjp) {
    LegArgs<float> a = leg_make_args<float>(p);
    a.alm = alm;
    a.rs = rs;
    a.vjp = vjp;
    a.F = const_cast<float2 *>(G);
    a.beam = beam;
    a.nmaps = nmaps;
    a.err = p->d_flag;
    if (!a.toff || !a.tst0 || (SPIN == 2 && !a.tst2)) {
        set_error("tensor-core transpose: the plan has no recurrence tile states");
        return SHTG_ERR_ARG;
    }
    const int smem = TaLayout<SPIN, NAS, NBS, TR>::BYTES;
    auto kern = k_leg_analysis_tc<SPIN, NAS, NBS, TR>;
    SHTG_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    dim3 grid((p->lmax + 256 * TR) / (256 * TR), p->lmax + 1, (nmaps + TC_NMT - 1) / TC_NMT);
    prof_begin(p, K_LEG_ANA32, st);
    kern<<<grid, TC_M, smem, st>>>(a);
    prof_end(p, st);
    SHTG_CHECK_LAUNCH("k_leg_analysis_tc");
    return SHTG_OK;
}
}  // namespace

// Shapes tried by the autotuner (key kind 2): synthesis (stages, staged l)
// = (1, 64) [four CTAs per SM at spin 2], (2, 128), (1, 128); transpose
// (A buffers, B buffers, 256-l tiles) = (1, 1, 2) [three CTAs per SM; the
// fastest at N_side 1024, l_max 2048, 8 maps], (1, 2, 2), (2, 2, 2),
// (1, 1, 1) [four CTAs per SM], (1, 2, 1), (2, 2, 1).
// Every shape sums the same products in the same order, so the choice does
// not change a bit of the result.
int leg_synth_tc(Plan *p, int spin, const float2 *alm, int rs, int nmaps, const float *beam, float2 *F,
                 cudaStream_t st) {
    return tune(p, 2, spin == 2 ? 1 : 0, nmaps, 3, st, [&](int v) {
        if (spin == 2) {
            if (v == 1) return launch_synth_tc<2, 2, 128>(p, alm, rs, nmaps, beam, F, st);
            if (v == 2) return launch_synth_tc<2, 1, 128>(p, alm, rs, nmaps, beam, F, st);
            return launch_synth_tc<2, 1, 64>(p, alm, rs, nmaps, beam, F, st);
        }
        if (v == 1) return launch_synth_tc<0, 2, 128>(p, alm, rs, nmaps, beam, F, st);
        if (v == 2) return launch_synth_tc<0, 1, 128>(p, alm, rs, nmaps, beam, F, st);
        return launch_synth_tc<0, 1, 64>(p, alm, rs, nmaps, beam, F, st);
    });
}

template <int SPIN>
static int analysis_tc_shape(int v, Plan *p, const float2 *G, int nmaps, const float *beam, float2 *alm, int rs,
                             cudaStream_t st, int vjp) {
    switch (v) {
        case 1: return launch_analysis_tc<SPIN, 1, 2, 2>(p, G, nmaps, beam, alm, rs, st, vjp);
        case 2: return launch_analysis_tc<SPIN, 2, 2, 2>(p, G, nmaps, beam, alm, rs, st, vjp);
        case 3: return launch_analysis_tc<SPIN, 1, 1, 1>(p, G, nmaps, beam, alm, rs, st, vjp);
        case 4: return launch_analysis_tc<SPIN, 1, 2, 1>(p, G, nmaps, beam, alm, rs, st, vjp);
        case 5: return launch_analysis_tc<SPIN, 2, 2, 1>(p, G, nmaps, beam, alm, rs, st, vjp);
        default: return launch_analysis_tc<SPIN, 1, 1, 2>(p, G, nmaps, beam, alm, rs, st, vjp);
    }
}

int leg_analysis_tc(Plan *p, int spin, const float2 *G, int nmaps, const float *beam, float2 *alm, int rs,
                    cudaStream_t st, int vjp) {
    return tune(p, 2, spin == 2 ? 3 : 2, nmaps, 6, st, [&](int v) {
        if (spin == 2) return analysis_tc_shape<2>(v, p, G, nmaps, beam, alm, rs, st, vjp);
        return analysis_tc_shape<0>(v, p, G, nmaps, beam, alm, rs, st, vjp);
    });
}

}  // namespace shtg

// Ring stage of the spherical-harmonic transforms: on each iso-latitude ring
// the field is f(phi_j) = sum_{m=-L..L} F(m) e^{i m (phi0 + 2 pi j / n)} with
// F(-m) = conj(F(m)) (a real field), phi0 = shift * pi / n.
//
// One CTA per ring pair.  The north and south rings of a pair have the same
// n and phi0, so one complex FFT of z = f_N + i f_S serves both.  Frequencies
// are folded modulo n (rings with n < 2L + 1 alias).  The length-n DFT is a
// Stockham autosort FFT in shared memory (natural order in and out): every
// pass loads R elements per butterfly into registers, applies the twiddles,
// does the radix-R DFT in registers and writes the R outputs to their sorted
// places (Govindaraju et al. 2008, "High performance discrete Fourier
// transforms on graphics processors", with one radix-2, -4 or -8 pass first,
// where it needs no twiddles, and radix-16 passes after it).  The buffer is
// padded by one element per 16 so that the
// scattered writes of the early passes hit distinct banks.  Rings whose n is
// not a power of two (HEALPix polar caps) use Bluestein's chirp convolution
// with precomputed kernel spectra.  The fused variant applies N^-1 between
// the inverse and the forward transform, so the pixel map never goes to
// global memory inside an operator application.
#include <algorithm>
#include <string>

#include "common.cuh"

namespace shtg {

// Threads per CTA: M / 16 for the launch's longest transform M (every
// radix-16 pass then has one butterfly per thread), at least 64; resident
// CTAs per SM for a budget of 128 registers a thread in FP32 (the inlined
// passes do not spill; the fixed-length launches, M = 16 NT: 64 registers,
// so twice as many threads share an SM), 255 in FP64 up to 256 threads (the
// FP64 passes spill at 128).
template <typename T, int NT, int FIX> struct RingBlocks {
    static constexpr int v = sizeof(T) == 8 ? (NT >= 256 ? 1 : 256 / NT) : (FIX > 0 ? 1024 : 512) / NT;
};

__device__ __forceinline__ int rpad(int i) { return i + (i >> 4); }

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }

// v * e^{-+2 pi i k / 16} (minus sign: forward transform, plus: inverse); k is
// a compile-time constant after unrolling, so the switch folds away
template <bool INV, typename C>
__device__ __forceinline__ C rot16(const C v, const int k) {
    typedef decltype(v.x) T;
    const T c1 = T(0.92387953251128675613), s1 = T(0.38268343236508977173), h = T(0.70710678118654752440);
    T c, s;   // cos, sin of k pi / 8
    switch (k & 15) {
        case 0: return v;
        case 4: return INV ? C{-v.y, v.x} : C{v.y, -v.x};
        case 8: return C{-v.x, -v.y};
        case 12: return INV ? C{v.y, -v.x} : C{-v.y, v.x};
        case 1: c = c1; s = s1; break;
        case 2: c = h; s = h; break;
        case 3: c = s1; s = c1; break;
        case 5: c = -s1; s = c1; break;
        case 6: c = -h; s = h; break;
        case 7: c = -c1; s = s1; break;
        case 9: c = -c1; s = -s1; break;
        case 10: c = -h; s = -h; break;
        case 11: c = -s1; s = -c1; break;
        case 13: c = s1; s = -c1; break;
        case 14: c = h; s = -h; break;
        default: c = c1; s = -s1; break;   // 15
    }
    if (INV) return C{v.x * c - v.y * s, v.x * s + v.y * c};
    return C{v.x * c + v.y * s, v.y * c - v.x * s};
}

template <bool INV, typename C>
__device__ __forceinline__ void dft2(C &a, C &b) {
    const C t = a;
    a = cadd(t, b);
    b = csub(t, b);
}

// natural order in and out: X_s = sum_r x_r e^{-+2 pi i r s / 4}
template <bool INV, typename C>
__device__ __forceinline__ void dft4(C &x0, C &x1, C &x2, C &x3) {
    const C t0 = cadd(x0, x2), t1 = csub(x0, x2), t2 = cadd(x1, x3);
    const C d = csub(x1, x3);
    const C t3 = INV ? C{-d.y, d.x} : C{d.y, -d.x};
    x0 = cadd(t0, t2);
    x2 = csub(t0, t2);
    x1 = cadd(t1, t3);
    x3 = csub(t1, t3);
}

// Composite radix-R DFT in registers, natural order in and out: with
// r = N2 r1 + r2 and s = s1 + N1 s2, X_s = sum_r2 w_R^{r2 s1} w_N2^{r2 s2}
// (sum_r1 x_r w_N1^{r1 s1}): N2 DFTs of length N1, twiddles, N1 DFTs of length N2.
template <int R, bool INV, typename C> struct Dft;
template <bool INV, typename C> struct Dft<2, INV, C> {
    static __device__ __forceinline__ void run(C *v) { dft2<INV>(v[0], v[1]); }
};
template <bool INV, typename C> struct Dft<4, INV, C> {
    static __device__ __forceinline__ void run(C *v) { dft4<INV>(v[0], v[1], v[2], v[3]); }
};
template <bool INV, typename C> struct Dft<8, INV, C> {   // N1 = 2, N2 = 4
    static __device__ __forceinline__ void run(C *v) {
        C y[4][2];
#pragma unroll
        for (int r2 = 0; r2 < 4; ++r2) {
            y[r2][0] = v[r2];
            y[r2][1] = v[4 + r2];
            dft2<INV>(y[r2][0], y[r2][1]);
            y[r2][1] = rot16<INV>(y[r2][1], 2 * r2);   // w_8^{r2} = w_16^{2 r2}
        }
#pragma unroll
        for (int s1 = 0; s1 < 2; ++s1) {
            dft4<INV>(y[0][s1], y[1][s1], y[2][s1], y[3][s1]);
#pragma unroll
            for (int s2 = 0; s2 < 4; ++s2) v[s1 + 2 * s2] = y[s2][s1];
        }
    }
};
template <bool INV, typename C> struct Dft<16, INV, C> {   // N1 = N2 = 4
    static __device__ __forceinline__ void run(C *v) {
        C y[4][4];
#pragma unroll
        for (int r2 = 0; r2 < 4; ++r2) {
            y[r2][0] = v[r2];
            y[r2][1] = v[4 + r2];
            y[r2][2] = v[8 + r2];
            y[r2][3] = v[12 + r2];
            dft4<INV>(y[r2][0], y[r2][1], y[r2][2], y[r2][3]);
#pragma unroll
            for (int s1 = 1; s1 < 4; ++s1) y[r2][s1] = rot16<INV>(y[r2][s1], r2 * s1);
        }
#pragma unroll
        for (int s1 = 0; s1 < 4; ++s1) {
            dft4<INV>(y[0][s1], y[1][s1], y[2][s1], y[3][s1]);
#pragma unroll
            for (int s2 = 0; s2 < 4; ++s2) v[s1 + 4 * s2] = y[s2][s1];
        }
    }
};

// Twiddles from the two-level table in shared memory: e^{-2 pi i t / Mmax}
template <typename C> struct TwTab {
    const C *lo, *hi;
    int blo, logmax;
    __device__ __forceinline__ C at(int t) const {
        return cmul(hi[t >> blo], lo[t & ((1 << blo) - 1)]);
    }
};

// One Stockham pass of radix R over a length-M transform whose sub-transforms
// of length Ns are done: butterfly j (k = j mod Ns) takes x[j + r M/R],
// multiplies element r by w^{r k} (w = e^{-+2 pi i / (Ns R)}), does a radix-R
// DFT and writes output s to (j - k) R + k + s Ns.  Each thread handles BPT
// butterflies; all reads finish (barrier) before any write, so the pass runs
// in place.  With post != null the outputs are multiplied by post[index];
// with cj they are conjugated (after the multiplication).
template <int R, int BPT, int NT, bool TW, typename C>
__device__ __forceinline__ void spass(C *buf, const int M, const int Ns, const TwTab<C> &tw,
                                      const C *__restrict__ post, const bool cj) {
    const int nb = M / R;
    C v[BPT][R];
#pragma unroll
    for (int b = 0; b < BPT; ++b) {
        const int j = threadIdx.x + b * NT;
        if (j < nb) {
#pragma unroll
            for (int r = 0; r < R; ++r) v[b][r] = buf[rpad(j + r * nb)];
        }
    }
    __syncthreads();
    int lsr = 0;   // log2(Ns R)
    while ((1 << lsr) < Ns * R) ++lsr;
    const int lshift = tw.logmax - lsr;
#pragma unroll
    for (int b = 0; b < BPT; ++b) {
        const int j = threadIdx.x + b * NT;
        if (j < nb) {
            const int k = j & (Ns - 1);
            if (TW && Ns > 1) {
                // w^r = w^{4a} w^b (r = 4a + b): table values at r = 1, 2, 4, 8,
                // products elsewhere (at most three roundings per twiddle)
                const int t = k << lshift;
                C wb[4], wa[4];
                wb[1] = tw.at(t);
                if (R >= 4) {
                    wb[2] = tw.at(2 * t);
                    wb[3] = cmul(wb[2], wb[1]);
                }
                if (R >= 8) wa[1] = tw.at(4 * t);
                if (R >= 16) {
                    wa[2] = tw.at(8 * t);
                    wa[3] = cmul(wa[2], wa[1]);
                }
#pragma unroll
                for (int r = 1; r < R; ++r) {
                    const int ra = r >> 2, rb = r & 3;
                    const C w = ra == 0 ? wb[rb] : (rb == 0 ? wa[ra] : cmul(wa[ra], wb[rb]));
                    v[b][r] = cmul(v[b][r], w);
                }
            }
            Dft<R, false, C>::run(v[b]);
            const int d = (j - k) * R + k;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int o = d + r * Ns;
                C y = post ? cmul(v[b][r], post[o]) : v[b][r];
                if (cj) y.y = -y.y;
                buf[rpad(o)] = y;
            }
        }
    }
    __syncthreads();
}

// Length-2^logM forward DFT (e^{-2 pi i jk/M}, unnormalized) of buf in
// place, natural order in and out; the last pass multiplies by post (if not
// null) and conjugates when cj is set.  The inverse transform is
// conj(DFT(conj x)): callers conjugate on the way in and out.  Passes: one
// radix-8, -4 or -2 pass when log2 M is not a multiple of four, then radix
// 16.  Each kernel calls it from one place, so it is inlined once.
template <int NT, typename C>
__device__ __forceinline__ void fft_stockham(C *buf, const int logM, const TwTab<C> tw,
                                          const C *__restrict__ post, const bool cj) {
    // M <= 16 NT.  A radix-2, -4 or -8 pass (when log2 M is not a multiple of
    // four) goes first, where it needs no twiddles (Ns = 1), with
    // ring_first_bpt butterflies per thread (the plan checks that this covers
    // M / R for every ring of the launch); the radix-16 passes follow with at
    // most one butterfly per thread, the last of them applying post / cj.
    const int M = 1 << logM;
    int Ns = 1, rem = logM;
    const int r0 = logM & 3;
    if (r0 != 0) {
        const bool last = rem == r0;
        if (r0 == 3) spass<8, ring_first_bpt(8, NT), NT, false>(buf, M, 1, tw, last ? post : nullptr, last && cj);
        else if (r0 == 2) spass<4, ring_first_bpt(4, NT), NT, false>(buf, M, 1, tw, last ? post : nullptr, last && cj);
        else spass<2, ring_first_bpt(2, NT), NT, false>(buf, M, 1, tw, last ? post : nullptr, last && cj);
        Ns = 1 << r0;
        rem -= r0;
    }
    while (rem > 0) {
        const bool last = rem == 4;
        spass<16, 1, NT, true>(buf, M, Ns, tw, last ? post : nullptr, last && cj);
        Ns <<= 4;
        rem -= 4;
    }
}

// ---------------------------------------------------------------------------
// Fixed-length Stockham FFT (M = 2^LOGM known at compile time), used by the
// launches of the long rings.  Same passes as fft_stockham (one radix-2, -4 or
// -8 pass when log2 M is not a multiple of four, then radix-16 passes), but
// every shared-memory address of a pass is a per-thread base plus a
// compile-time offset, and the twiddles of each radix-16 pass come from a
// precomputed table (twf_*): entries k and NS + k of pass p hold w^1 and w^4
// for w = e^{-2 pi i k / (16 NS)}, k < NS = 2^(LOGM mod 4) 16^p (passes with
// NS = 1 need none), rounded once from FP64; the other powers are products
// of those.  A warp's 32 consecutive k read 32 consecutive entries.
//
// Padded addresses: rpad(i) = i + i / 16.  For a pass with NB = M / R
// butterflies (NB a multiple of 16), butterfly j reads j + r NB, whose padded
// address is rpad(j) + r (NB + NB / 16).  Radix-16 outputs go to
// o = d + r NS with d = 16 (j - k) + k: for NS >= 16, rpad(o) = d + (j - k) +
// k / 16 + r (NS + NS / 16); for NS = 1, 2, 4, 8 (NS divides 16, k < NS),
// rpad(o) = d + (j - k) + r NS + (r NS) / 16.  The first pass (NS = 1)
// writes o = R j + r at rpad(R j) + r.
__host__ __device__ constexpr int twf_pass_ns(int logm, int p) { return (1 << (logm & 3)) << (4 * p); }
__host__ __device__ constexpr int twf_pass_off(int logm, int p) {
    int o = 0;
    for (int q = 0; q < p; ++q)
        if (twf_pass_ns(logm, q) > 1) o += 2 * twf_pass_ns(logm, q);
    return o;
}

// Radix-16 DFT in place with its outputs left transposed: X[s] ends at
// v[4 (s mod 4) + s / 4] (the same 4 x 4 decomposition as Dft<16>: DFT-4 down
// the columns r2, twiddles w16^(r2 s1), DFT-4 along the rows s1), so no second
// array of 16 values is live; callers read the outputs through the
// compile-time permutation dft16_at.
__host__ __device__ constexpr int dft16_at(int s) { return 4 * (s & 3) + (s >> 2); }
template <typename C>
__device__ __forceinline__ void dft16_tp(C *v) {
#pragma unroll
    for (int r2 = 0; r2 < 4; ++r2) {
        dft4<false>(v[r2], v[r2 + 4], v[r2 + 8], v[r2 + 12]);
        v[r2 + 4] = rot16<false>(v[r2 + 4], r2);
        v[r2 + 8] = rot16<false>(v[r2 + 8], 2 * r2);
        v[r2 + 12] = rot16<false>(v[r2 + 12], 3 * r2);
    }
#pragma unroll
    for (int s1 = 0; s1 < 4; ++s1) dft4<false>(v[4 * s1], v[4 * s1 + 1], v[4 * s1 + 2], v[4 * s1 + 3]);
}

__host__ __device__ constexpr int twf_len(int logm) { return twf_pass_off(logm, logm >> 2); }

template <int R, int LOGM, int NT, typename C>
__device__ __forceinline__ void fpass_first(C *buf) {
    constexpr int M = 1 << LOGM, NB = M / R, BPT = (NB + NT - 1) / NT;
    constexpr int SIN = NB + NB / 16;
    static_assert(NB % 16 == 0, "first pass needs M / R to be a multiple of 16");
    C v[BPT][R];
#pragma unroll
    for (int b = 0; b < BPT; ++b) {
        const int j = threadIdx.x + b * NT;
        if (NB % NT == 0 || j < NB) {
            const int bi = j + (j >> 4);
#pragma unroll
            for (int r = 0; r < R; ++r) v[b][r] = buf[bi + r * SIN];
        }
    }
    __syncthreads();
#pragma unroll
    for (int b = 0; b < BPT; ++b) {
        const int j = threadIdx.x + b * NT;
        if (NB % NT == 0 || j < NB) {
            Dft<R, false, C>::run(v[b]);
            const int o0 = j * R;
            const int bo = o0 + (o0 >> 4);
#pragma unroll
            for (int r = 0; r < R; ++r) buf[bo + r] = v[b][r];
        }
    }
    __syncthreads();
}

template <int LOGM, int NS, int NT, typename C>
__device__ __forceinline__ void fpass16(C *buf, const C *__restrict__ twp) {
    constexpr int M = 1 << LOGM, NB = M / 16, BPT = (NB + NT - 1) / NT;
    constexpr int SIN = NB + NB / 16;
    static_assert(NB % 16 == 0, "radix-16 pass needs M / 16 to be a multiple of 16");
    C v[BPT][16];
#pragma unroll
    for (int b = 0; b < BPT; ++b) {
        const int j = threadIdx.x + b * NT;
        if (NB % NT == 0 || j < NB) {
            const int bi = j + (j >> 4);
#pragma unroll
            for (int r = 0; r < 16; ++r) v[b][r] = buf[bi + r * SIN];
        }
    }
    __syncthreads();
#pragma unroll
    for (int b = 0; b < BPT; ++b) {
        const int j = threadIdx.x + b * NT;
        if (NB % NT == 0 || j < NB) {
            const int k = j & (NS - 1);
            if (NS > 1) {
                // w^r for r = 4a + c from the two table values w and w^4:
                // w^2, w^3 = w^2 w; w^8 = (w^4)^2, w^12 = w^8 w^4; w^(4a + c) =
                // w^(4a) w^c: at most five roundings, ten live registers
                const C w1 = twp[k], w4 = twp[NS + k];
                const C w2 = cmul(w1, w1), w3 = cmul(w2, w1);
                v[b][1] = cmul(v[b][1], w1);
                v[b][2] = cmul(v[b][2], w2);
                v[b][3] = cmul(v[b][3], w3);
                C wa = w4;
#pragma unroll
                for (int a = 1; a < 4; ++a) {
                    if (a > 1) wa = cmul(wa, w4);
                    v[b][4 * a] = cmul(v[b][4 * a], wa);
                    v[b][4 * a + 1] = cmul(v[b][4 * a + 1], cmul(wa, w1));
                    v[b][4 * a + 2] = cmul(v[b][4 * a + 2], cmul(wa, w2));
                    v[b][4 * a + 3] = cmul(v[b][4 * a + 3], cmul(wa, w3));
                }
            }
            dft16_tp(v[b]);
            const int d = 16 * (j - k) + k;
            const int bo = NS >= 16 ? d + (j - k) + (k >> 4) : d + (j - k);
#pragma unroll
            for (int r = 0; r < 16; ++r) {
                const int off = NS >= 16 ? r * (NS + NS / 16) : r * NS + (r * NS) / 16;
                buf[bo + off] = v[b][dft16_at(r)];
            }
        }
    }
    __syncthreads();
}

template <int LOGM, int NT, int P, typename C>
__device__ __forceinline__ void fft16_passes(C *buf, const C *__restrict__ tw) {
    if constexpr (P < (LOGM >> 2)) {
        fpass16<LOGM, twf_pass_ns(LOGM, P), NT>(buf, tw + twf_pass_off(LOGM, P));
        fft16_passes<LOGM, NT, P + 1>(buf, tw);
    }
}

// Length-2^LOGM forward DFT of buf in place (natural order in and out).
template <int LOGM, int NT, typename C>
__device__ __forceinline__ void fft_fixed(C *buf, const C *__restrict__ tw) {
    static_assert(LOGM >= 8, "fixed-length passes need M >= 256");
    constexpr int R0L = LOGM & 3;
    if constexpr (R0L != 0) fpass_first<(1 << R0L), LOGM, NT>(buf);
    fft16_passes<LOGM, NT, 0>(buf, tw);
}

// One transform direction with the fixed-length FFT (see transform_dir)
// (the Bluestein spectrum multiply is a separate sweep over the buffer with
// coalesced loads of the spectrum, so no pass keeps sixteen of them in flight)
template <int LOGM, int NT, typename C>
__device__ __forceinline__ void transform_dir_fixed(C *buf, const C *__restrict__ tw, const C *__restrict__ bh) {
    constexpr int M = 1 << LOGM;
    if (bh) {
        fft_fixed<LOGM, NT>(buf, tw);
#pragma unroll 4
        for (int i = threadIdx.x; i < M; i += NT) {
            C y = cmul(buf[rpad(i)], __ldg(bh + i));
            y.y = -y.y;
            buf[rpad(i)] = y;
        }
        __syncthreads();
    }
    fft_fixed<LOGM, NT>(buf, tw);
}

template <typename T> struct RingArgs {
    typedef typename VT<T>::C C;
    int lmax, nring, npairs, nmaps;
    int64_t npix;
    const RingFFT *rf;
    const int64_t *ofs;
    const double *wring;
    const C *tw;      // two-level twiddle table [lo | hi]
    int tw_blo, tw_nlo, tw_nhi, logmax;
    const C *chirp, *bfwd, *binv;
    const C *rph;     // ring phase tables e^{i pi k / n}
    const C *twf;     // fixed-length launches: pass twiddles for M = 2^FIX
    int mpg;          // maps per CTA: CTA (pair, y) handles maps [y mpg, min(nmaps, (y + 1) mpg))
    C *FG;            // [map][ring][m]
    T *map;           // [map][npix]
    const T *ninv;    // fused: [comp][npix]
    int nT;           // fused: rows [0, nT) use N^-1 component 0 (T), later rows component 1 (Q, U)
    int weighted;     // analysis: multiply by the quadrature weight
    int buf_len;      // shared transform buffer length (padded) of this launch
    int chirp_len;    // shared chirp buffer length (longest Bluestein ring of the launch)
    const int *pairs; // ring pairs handled by this launch (one CTA each)
};

// One transform direction in place: a DFT for power-of-two rings (bh null),
// a Bluestein convolution with kernel spectrum bh otherwise (buf then holds
// its conjugate).  One FFT call site.
template <int NT, typename C>
__device__ __forceinline__ void transform_dir(C *buf, const int logM, const TwTab<C> &tw, const C *__restrict__ bh) {
    const int nf = bh ? 2 : 1;
    for (int k = 0; k < nf; ++k) fft_stockham<NT>(buf, logM, tw, k == 0 ? bh : nullptr, bh != nullptr && k == 0);
}

// The transforms of one map: [fold or load] -> one (MODE 0, 1) or two
// (MODE 2, with the N^-1 weighting between) transform directions -> [write
// map or unfold].  A direction is one FFT (power-of-two rings) or, for
// Bluestein rings, a convolution = DFT, times the kernel spectrum and
// conjugated in the last pass, DFT again: buf then holds the conjugate of the
// convolution.  The directions run in a loop, so the FFT is inlined once.
// The work of one CTA: ring pair a.pairs[pidx], maps [y mpg, (y + 1) mpg).
// Called by the plan's kernel (the block indices) and by the grouped kernel
// (one work item of a list that spans several geometries).
template <typename T, int MODE, int NT, int FIX>
__device__ __forceinline__ void ring_cta(const RingArgs<T> &a, const int pidx, const int y) {
    typedef typename VT<T>::C C;
    extern __shared__ __align__(16) unsigned char s_raw[];
    // FIX > 0: every ring of the launch has M = 2^FIX and the fixed-length
    // passes run (twiddles from twf, no shared twiddle table)
    constexpr bool fixed = FIX > 0;
    // FP32 fixed-length launches stage their pass twiddles in shared memory
    // (at most 1092 entries); FP64 ones read them through L1 (the FP64
    // 8192-point buffer and chirp leave no room)
    constexpr bool twf_smem = fixed && sizeof(T) == 4;
    const int ntw = fixed ? (twf_smem ? twf_len(FIX > 0 ? FIX : 8) : 0) : a.tw_nlo + a.tw_nhi;
    C *s_tw = reinterpret_cast<C *>(s_raw);
    C *buf = s_tw + ntw;
    C *s_chirp = buf + a.buf_len;          // this ring's chirp (Bluestein rings)
    C *scr_p = s_chirp + a.chirp_len;      // aliased fold: partial sums [north | south][NT] (generic launches)
    const C *tw_src = fixed ? a.twf : a.tw;
    for (int i = threadIdx.x; i < ntw; i += NT) s_tw[i] = tw_src[i];
    const C *twf = twf_smem ? s_tw : a.twf;
    TwTab<C> tw;
    tw.lo = s_tw;
    tw.hi = s_tw + a.tw_nlo;
    tw.blo = a.tw_blo;
    tw.logmax = a.logmax;
    // (the first FFT pass starts after a barrier that follows the fill below)

    const int pr = a.pairs[pidx];
    const int rn = pr, rs = a.nring - 1 - pr;
    const bool single = (rn == rs);
    const RingFFT f = a.rf[rn];
    const int n = f.n, logM = f.logM, M = 1 << logM;
    const int L = a.lmax;
    // the chirp is read up to five times per element and map: stage it once
    const C *chirp = a.chirp + f.chirp_off;
    if (f.blue) {
        for (int i = threadIdx.x; i < n; i += NT) s_chirp[i] = chirp[i];
        chirp = s_chirp;
    }
    __syncthreads();
    const C *ph = a.rph + f.ph_off;   // e^{i pi k / n} (shifted rings)
    const C zero = {T(0), T(0)};
    constexpr int NDIR = MODE == 2 ? 2 : 1;

    const int q0 = y * a.mpg, q1 = min(a.nmaps, q0 + a.mpg);
    for (int q = q0; q < q1; ++q) {
        if (MODE != 1 && n >= 2 * L) {
            // ---- fold without aliasing (n >= 2 l_max): F(m) alone fills bin m
            // and conj F(m) bin n - m (phase e^{+-i pi s m / n}); with n = 2 l_max
            // both land in bin n / 2 = l_max; bins strictly between l_max and
            // n - l_max are zero.  One thread per m: independent loads.
            const C *Fn = a.FG + ((int64_t)q * a.nring + rn) * (L + 1);
            const C *Fs = a.FG + ((int64_t)q * a.nring + rs) * (L + 1);
#pragma unroll 4
            for (int mm = threadIdx.x; mm <= L; mm += NT) {
                C hn = Fn[mm], hs = single ? zero : Fs[mm];
                if (f.shift) {
                    const C phk = ph[mm];
                    hn = cmul(hn, phk);
                    hs = cmul(hs, phk);
                }
                C z1 = {hn.x - hs.y, hn.y + hs.x};      // bin mm
                C z2 = {hn.x + hs.y, -hn.y + hs.x};     // bin n - mm: conj(hn) + i conj(hs)
                if (mm == 0) z2 = zero;
                const int k2 = n - mm;
                if (2 * mm == n) {                      // bin n / 2 collects both
                    z1.x += z2.x;
                    z1.y += z2.y;
                }
                buf[rpad(mm)] = f.blue ? cmul(z1, cconj(chirp[mm])) : cconj(z1);
                if (mm > 0 && 2 * mm != n)
                    buf[rpad(k2)] = f.blue ? cmul(z2, cconj(chirp[k2])) : cconj(z2);
            }
            for (int k = L + 1 + threadIdx.x; k < n - L; k += NT) buf[rpad(k)] = zero;
        } else if (MODE != 1) {
            // ---- aliased fold (n < 2 l_max) into the length-n spectrum of
            // z = f_N + i f_S.  Per residue r: Q(r) = sum_t (-1)^{s t} F(r + t n)
            // (phi0 = s pi / n); then H(k) = e^{i pi s k / n} [Q(k) + (-1)^s
            // conj Q(n - k)] for k > 0 and H(0) = Q(0) + conj(Q(0) - F(0)).
            // Rings with n < NT / 2 split each residue's sum over S = NT / n
            // thread segments (coalesced reads, fixed summation order), so a
            // small polar ring costs no more time than a long one.
            const C *Fn = a.FG + ((int64_t)q * a.nring + rn) * (L + 1);
            const C *Fs = a.FG + ((int64_t)q * a.nring + rs) * (L + 1);
            // Q of the south ring in buf[n, 2n) (the launch's buffer holds 2n
            // for every aliased ring; Bluestein rings: M >= 2n)
            auto qsr = [&](int k) -> C & { return buf[rpad(n + k)]; };
            const int S = (!fixed && n <= NT / 2) ? NT / n : 1;   // fixed launches: n > NT / 2
            if (S > 1) {
                const int k = threadIdx.x % n, s = threadIdx.x / n;
                if (s < S) {
                    C pn = zero, ps = zero;
                    T sg = (f.shift && (s & 1)) ? T(-1) : T(1);   // (-1)^{s t}, t = s + j S
                    const bool flip = f.shift && (S & 1);
                    for (int mm = k + s * n; mm <= L; mm += S * n) {
                        const C vn = Fn[mm];
                        pn.x += sg * vn.x;
                        pn.y += sg * vn.y;
                        if (!single) {
                            const C vs = Fs[mm];
                            ps.x += sg * vs.x;
                            ps.y += sg * vs.y;
                        }
                        if (flip) sg = -sg;
                    }
                    scr_p[s * n + k] = pn;
                    scr_p[NT + s * n + k] = ps;
                }
                __syncthreads();
                for (int kk = threadIdx.x; kk < n; kk += NT) {
                    C qn = zero, qq = zero;
                    for (int s2 = 0; s2 < S; ++s2) {
                        qn = cadd(qn, scr_p[s2 * n + kk]);
                        qq = cadd(qq, scr_p[NT + s2 * n + kk]);
                    }
                    buf[rpad(kk)] = qn;
                    qsr(kk) = qq;
                }
            } else {
                for (int k = threadIdx.x; k < n; k += NT) {
                    C qn = zero, qq = zero;
                    T sg = T(1);
                    for (int mm = k; mm <= L; mm += n) {
                        const C vn = Fn[mm];
                        qn.x += sg * vn.x;
                        qn.y += sg * vn.y;
                        if (!single) {
                            const C vs = Fs[mm];
                            qq.x += sg * vs.x;
                            qq.y += sg * vs.y;
                        }
                        if (f.shift) sg = -sg;
                    }
                    buf[rpad(k)] = qn;
                    qsr(k) = qq;
                }
            }
            __syncthreads();
            // bins k and n - k from one thread, in place over Q_N
            const T sig = f.shift ? T(-1) : T(1);
            for (int j = threadIdx.x; 2 * j <= n; j += NT) {
                const int k1 = j, k2 = j ? n - j : 0;
                const C qn1 = buf[rpad(k1)], qn2 = buf[rpad(k2)];
                const C qs1 = qsr(k1), qs2 = qsr(k2);
                C hn1, hs1, hn2, hs2;
                if (j == 0) {
                    const C f0n = Fn[0], f0s = single ? zero : Fs[0];
                    hn1 = {qn1.x + (qn1.x - f0n.x), qn1.y - (qn1.y - f0n.y)};
                    hs1 = {qs1.x + (qs1.x - f0s.x), qs1.y - (qs1.y - f0s.y)};
                } else {
                    hn1 = {qn1.x + sig * qn2.x, qn1.y - sig * qn2.y};
                    hs1 = {qs1.x + sig * qs2.x, qs1.y - sig * qs2.y};
                }
                hn2 = {qn2.x + sig * qn1.x, qn2.y - sig * qn1.y};
                hs2 = {qs2.x + sig * qs1.x, qs2.y - sig * qs1.y};
                if (f.shift) {
                    // e^{i pi (n - k) / n} = -conj e^{i pi k / n}
                    const C ph1 = ph[k1];
                    const C ph2 = {-ph1.x, ph1.y};
                    hn1 = cmul(hn1, ph1);
                    hs1 = cmul(hs1, ph1);
                    hn2 = cmul(hn2, ph2);
                    hs2 = cmul(hs2, ph2);
                }
                const C z1 = {hn1.x - hs1.y, hn1.y + hs1.x};
                buf[rpad(k1)] = f.blue ? cmul(z1, cconj(chirp[k1])) : cconj(z1);
                if (k2 != k1) {
                    const C z2 = {hn2.x - hs2.y, hn2.y + hs2.x};
                    buf[rpad(k2)] = f.blue ? cmul(z2, cconj(chirp[k2])) : cconj(z2);
                }
            }
            // (Bluestein rings keep Q_S in buf[n, 2n): zero the tail only after)
            if (f.blue) __syncthreads();
        } else {
            // ---- load z = w (m_N + i m_S)
            const T *mn = a.map + (int64_t)q * a.npix + a.ofs[rn];
            const T *ms = a.map + (int64_t)q * a.npix + a.ofs[rs];
            const T w = a.weighted ? T(a.wring[rn]) : T(1);
#pragma unroll 4
            for (int j = threadIdx.x; j < n; j += NT) {
                const C z = {mn[j] * w, single ? T(0) : ms[j] * w};
                buf[rpad(j)] = f.blue ? cmul(z, chirp[j]) : z;
            }
        }
        if (f.blue)
            for (int k = n + threadIdx.x; k < M; k += NT) buf[rpad(k)] = zero;
        __syncthreads();
#pragma unroll 1
        for (int dir = 0; dir < NDIR; ++dir) {
            // inverse (e^{+2 pi i jk/n}) for MODE 0 and the first direction of
            // MODE 2, forward (e^{-2 pi i jk/n}) otherwise
            const bool fwd = MODE == 1 || dir == 1;
            const C *bh = f.blue ? (fwd ? a.bfwd : a.binv) + f.bhat_off : nullptr;
            if constexpr (fixed) {
                transform_dir_fixed<(fixed ? FIX : 8), NT>(buf, twf, bh);
            } else {
                transform_dir<NT>(buf, logM, tw, bh);
            }
            if (MODE == 2 && dir == 0) {
                // ---- N^-1 weighting (each thread rewrites the elements it reads)
                const int comp = q < a.nT ? 0 : 1;
                const T *wn = a.ninv + (int64_t)comp * a.npix + a.ofs[rn];
                const T *ws = a.ninv + (int64_t)comp * a.npix + a.ofs[rs];
#pragma unroll 4
                for (int j = threadIdx.x; j < n; j += NT) {
                    C z = buf[rpad(j)];
                    if (f.blue) z = cmul(z, chirp[j]);
                    z.y = -z.y;
                    C y = {z.x * wn[j], single ? T(0) : z.y * ws[j]};
                    if (f.blue) y = cmul(y, chirp[j]);
                    buf[rpad(j)] = y;
                }
                if (f.blue)
                    for (int k = n + threadIdx.x; k < M; k += NT) buf[rpad(k)] = zero;
                __syncthreads();
            }
        }
        if (MODE == 0) {
            // ---- ring pixels: z = conj(buf) (direct) or conj(buf c) (Bluestein)
            T *mn = a.map + (int64_t)q * a.npix + a.ofs[rn];
            T *ms = a.map + (int64_t)q * a.npix + a.ofs[rs];
            for (int j = threadIdx.x; j < n; j += NT) {
                C z = buf[rpad(j)];
                if (f.blue) z = cmul(z, chirp[j]);
                z.y = -z.y;
                mn[j] = z.x;
                if (!single) ms[j] = z.y;
            }
        } else {
            // ---- unfold: G(m) = e^{-i m phi0} Y(m mod n), split north / south
            C *Gn = a.FG + ((int64_t)q * a.nring + rn) * (L + 1);
            C *Gs = a.FG + ((int64_t)q * a.nring + rs) * (L + 1);
            // G(k + t n) = (-1)^{s t} e^{-i pi s k / n} Y(k), one phase per bin
            if (n > L) {
                for (int k = threadIdx.x; k <= L; k += NT) {
                    const int k2 = k ? n - k : 0;
                    C w1 = buf[rpad(k)], w2 = buf[rpad(k2)];
                    if (f.blue) {
                        w1 = cmul(cconj(w1), chirp[k]);
                        w2 = cmul(cconj(w2), chirp[k2]);
                    }
                    C yn = {T(0.5) * (w1.x + w2.x), T(0.5) * (w1.y - w2.y)};
                    C ys = {T(0.5) * (w1.y + w2.y), T(-0.5) * (w1.x - w2.x)};
                    if (f.shift) {
                        const C phk = cconj(ph[k]);
                        yn = cmul(yn, phk);
                        ys = cmul(ys, phk);
                    }
                    Gn[k] = yn;
                    if (!single) Gs[k] = ys;
                }
            } else {
                // aliased rings: Y_N(k), Y_S(k) for bins k and n - k from one
                // thread (Y_N in place over buf, Y_S beside it), then every m
                // written once, coalesced
                auto ysr = [&](int k) -> C & { return buf[rpad(n + k)]; };
                for (int j = threadIdx.x; 2 * j <= n; j += NT) {
                    const int k1 = j, k2 = j ? n - j : 0;
                    C w1 = buf[rpad(k1)], w2 = buf[rpad(k2)];
                    if (f.blue) {
                        w1 = cmul(cconj(w1), chirp[k1]);
                        w2 = cmul(cconj(w2), chirp[k2]);
                    }
                    C yn1 = {T(0.5) * (w1.x + w2.x), T(0.5) * (w1.y - w2.y)};
                    C ys1 = {T(0.5) * (w1.y + w2.y), T(-0.5) * (w1.x - w2.x)};
                    C yn2 = {yn1.x, -yn1.y};
                    C ys2 = {ys1.x, -ys1.y};
                    if (f.shift) {
                        // e^{-i pi (n - k) / n} = -conj e^{-i pi k / n}
                        const C ph1 = cconj(ph[k1]);
                        const C ph2 = {-ph1.x, ph1.y};
                        yn1 = cmul(yn1, ph1);
                        ys1 = cmul(ys1, ph1);
                        yn2 = cmul(yn2, ph2);
                        ys2 = cmul(ys2, ph2);
                    }
                    buf[rpad(k1)] = yn1;
                    ysr(k1) = ys1;
                    if (k2 != k1) {
                        buf[rpad(k2)] = yn2;
                        ysr(k2) = ys2;
                    }
                }
                __syncthreads();
                int k = threadIdx.x % n, t = threadIdx.x / n;
                const int dk = NT % n, dt = NT / n;
                for (int mm = threadIdx.x; mm <= L; mm += NT) {
                    C yn = buf[rpad(k)], ys = ysr(k);
                    if (f.shift && (t & 1)) {
                        yn = {-yn.x, -yn.y};
                        ys = {-ys.x, -ys.y};
                    }
                    Gn[mm] = yn;
                    if (!single) Gs[mm] = ys;
                    k += dk;
                    t += dt;
                    if (k >= n) {
                        k -= n;
                        t += 1;
                    }
                }
            }
        }
        __syncthreads();
    }
}

template <typename T, int MODE, int NT, int FIX>
__global__ void __launch_bounds__(NT, (RingBlocks<T, NT, FIX>::v)) k_ring(const RingArgs<T> a) {
    ring_cta<T, MODE, NT, FIX>(a, blockIdx.x, blockIdx.y);
}

// Grouped launch (chains of several geometries): one launch per
// transform-length class (the template's NT and FIX) over the launch buckets
// of that class of every plan; entry e is one (plan, bucket) with its own
// arguments, flat CTA i belongs to the entry with first[e] <= i <
// first[e + 1] and runs ring pair i' % count[e], map group i' / count[e]
// (i' = i - first[e]).  Entries whose plan group's device flag is 0 are
// skipped.
#define SHTG_RING_ENTRIES (2 * SHTG_MAX_GROUPS)
template <typename T> struct RingGroups {
    int ne;
    int first[SHTG_RING_ENTRIES + 1];
    int count[SHTG_RING_ENTRIES];
    const int *active[SHTG_RING_ENTRIES];   // the entry's plan group flag (null: always active)
    RingArgs<T> a[SHTG_RING_ENTRIES];
};

template <typename T, int MODE, int NT, int FIX>
__global__ void __launch_bounds__(NT, (RingBlocks<T, NT, FIX>::v)) k_ring_grp(const __grid_constant__ RingGroups<T> G) {
    const int i = blockIdx.x;
    int e = 0;
    while (e + 1 < G.ne && i >= G.first[e + 1]) ++e;
    if (G.active[e] && *G.active[e] == 0) return;
    const int li = i - G.first[e];
    ring_cta<T, MODE, NT, FIX>(G.a[e], li % G.count[e], li / G.count[e]);
}

template <typename T> static const typename VT<T>::C *ring_twf(Plan *p);
template <> const float2 *ring_twf<float>(Plan *p) { return p->d_twf32; }
template <> const double2 *ring_twf<double>(Plan *p) { return p->d_twf64; }

template <typename T> static RingArgs<T> ring_args(Plan *p);
template <> RingArgs<float> ring_args<float>(Plan *p) {
    RingArgs<float> a{};
    a.tw = p->d_tw32;
    a.chirp = p->d_chirp32;
    a.rph = p->d_rph32;
    a.bfwd = p->d_bfwd32;
    a.binv = p->d_binv32;
    return a;
}
template <> RingArgs<double> ring_args<double>(Plan *p) {
    RingArgs<double> a{};
    a.tw = p->d_tw64;
    a.chirp = p->d_chirp64;
    a.rph = p->d_rph64;
    a.bfwd = p->d_bfwd64;
    a.binv = p->d_binv64;
    return a;
}

template <typename T, int MODE, int NT, int FIX>
static int launch_ring_nt(RingArgs<T> a, int ctas, size_t smem, cudaStream_t st) {
    auto kern = k_ring<T, MODE, NT, FIX>;
    if (smem > 48 * 1024) SHTG_CUDA(allow_max_smem(kern));
    // The maps of a ring pair are split over grid.y when the pairs alone give
    // fewer than four waves of resident CTAs (a CTA still handles at least
    // two maps, so its chirp and twiddle staging stay amortized)
    int dev = 0, nsm = 0, per = 0;
    SHTG_CUDA(cudaGetDevice(&dev));
    SHTG_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    SHTG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, NT, smem));
    const int want = 4 * nsm * (per > 0 ? per : 1);
    int groups = (want + ctas - 1) / ctas;
    groups = std::max(1, std::min(groups, (a.nmaps + 1) / 2));
    a.mpg = (a.nmaps + groups - 1) / groups;
    groups = (a.nmaps + a.mpg - 1) / a.mpg;
    kern<<<dim3(ctas, groups), NT, smem, st>>>(a);
    return SHTG_OK;
}

template <typename T, int MODE>
static int launch_ring(Plan *p, RingArgs<T> a, cudaStream_t st) {
    typedef typename VT<T>::C C;
    a.lmax = p->lmax;
    a.nring = p->nring;
    a.npairs = p->npairs;
    a.npix = p->npix;
    a.rf = p->d_rfft;
    a.ofs = p->d_ofs;
    a.wring = p->d_wring;
    a.logmax = p->fft_logmax;
    a.tw_blo = p->tw_blo;
    a.tw_nlo = p->tw_nlo;
    a.tw_nhi = p->tw_nhi;
    // one launch per length bucket, each with the thread count and shared
    // memory of its longest transform.  The buckets touch disjoint ring
    // pairs, so all but the first run on the plan's side streams, forked from
    // and joined back into st with events (parallel branches when st is
    // being captured into a graph): the short single-wave launches of the
    // small polar rings then overlap with the long ones.
    prof_begin(p, sizeof(T) == 8 ? K_RING64 : K_RING32, st);
    int nl = 0, nside = 0;
    const int nb = (int)p->ring_launch.size();
    if (nb > 1) SHTG_CUDA(cudaEventRecord(p->ring_fork, st));
    for (int gi = 0; gi < nb; ++gi) {
        const Plan::RingLaunch &g = p->ring_launch[gi];
        if (g.count == 0) continue;
        cudaStream_t ls = st;
        if (gi > 0 && nside < Plan::RING_SIDE) {
            ls = p->ring_side[nside];
            SHTG_CUDA(cudaStreamWaitEvent(ls, p->ring_fork, 0));
        }
        const int M = 1 << g.logm;
        // launches of buckets above 1024 hold rings of one transform length
        // M = 2^g.fix (2^logm, or 2^(logm - 1) for aliased direct rings, whose
        // buffer still holds 2^logm: checked at plan creation) and run the
        // fixed-length passes with M / 16 threads
        const bool fix = g.fix > 0;
        const int nt = fix ? (1 << g.fix) / 16 : ring_threads(g.logm);
        a.buf_len = M + M / 16;
        a.chirp_len = g.chirp;
        a.twf = fix ? ring_twf<T>(p) + p->twf_off[g.fix] : nullptr;
        // shared memory: twiddles (generic: two-level table; FP32 fixed: the
        // pass tables), buffer, chirp, and the aliased fold's partial sums
        // (generic launches only: a fixed launch's rings have n >= M / 2 >
        // NT / 2, so they never split a residue's sum)
        const size_t ntw = fix ? (sizeof(T) == 4 ? (size_t)twf_len(g.fix) : 0) : (size_t)p->tw_nlo + p->tw_nhi;
        const size_t smem = sizeof(C) * (ntw + a.buf_len + a.chirp_len + ((g.alias && !fix) ? 2 * nt : 0));
        a.pairs = p->d_ring_groups + g.off;
        int rc = SHTG_OK;
        switch (g.fix) {
            case 10: rc = launch_ring_nt<T, MODE, 64, 10>(a, g.count, smem, ls); break;
            case 11: rc = launch_ring_nt<T, MODE, 128, 11>(a, g.count, smem, ls); break;
            case 12: rc = launch_ring_nt<T, MODE, 256, 12>(a, g.count, smem, ls); break;
            case 13: rc = launch_ring_nt<T, MODE, 512, 13>(a, g.count, smem, ls); break;
            default: rc = launch_ring_nt<T, MODE, 64, 0>(a, g.count, smem, ls); break;
        }
        if (rc != SHTG_OK) return rc;
        if (ls != st) {
            SHTG_CUDA(cudaEventRecord(p->ring_join[nside], ls));
            SHTG_CUDA(cudaStreamWaitEvent(st, p->ring_join[nside], 0));
            ++nside;
        }
        ++nl;
    }
    prof_end(p, st, nl);
    SHTG_CHECK_LAUNCH("k_ring");
    return SHTG_OK;
}

// launch arguments of one bucket of plan p (the fields launch_ring sets)
template <typename T>
static void ring_bucket_args(Plan *p, const Plan::RingLaunch &g, RingArgs<T> &a, size_t &smem) {
    typedef typename VT<T>::C C;
    a.lmax = p->lmax;
    a.nring = p->nring;
    a.npairs = p->npairs;
    a.npix = p->npix;
    a.rf = p->d_rfft;
    a.ofs = p->d_ofs;
    a.wring = p->d_wring;
    a.logmax = p->fft_logmax;
    a.tw_blo = p->tw_blo;
    a.tw_nlo = p->tw_nlo;
    a.tw_nhi = p->tw_nhi;
    const int M = 1 << g.logm;
    const bool fix = g.fix > 0;
    const int nt = fix ? (1 << g.fix) / 16 : ring_threads(g.logm);
    a.buf_len = M + M / 16;
    a.chirp_len = g.chirp;
    a.twf = fix ? ring_twf<T>(p) + p->twf_off[g.fix] : nullptr;
    const size_t ntw = fix ? (sizeof(T) == 4 ? (size_t)twf_len(g.fix) : 0) : (size_t)p->tw_nlo + p->tw_nhi;
    smem = sizeof(C) * (ntw + a.buf_len + a.chirp_len + ((g.alias && !fix) ? 2 * nt : 0));
    a.pairs = p->d_ring_groups + g.off;
}

template <typename T, int MODE, int NT, int FIX>
static int launch_ring_grp(RingGroups<T> &G, size_t smem, int64_t total, cudaStream_t st) {
    auto kern = k_ring_grp<T, MODE, NT, FIX>;
    if (smem > 48 * 1024) SHTG_CUDA(allow_max_smem(kern));
    kern<<<(unsigned)total, NT, smem, st>>>(G);
    return SHTG_OK;
}

template <typename T>
int ring_fused_grp(int ng, Plan *const *ps, typename VT<T>::C *const *FG, const int *nmaps, const int *nT,
                   const T *const *ninv, const int *const *active, cudaStream_t st) {
    if (ng < 1 || ng > SHTG_MAX_GROUPS) {
        set_error("grouped ring launch: 1 to " + std::to_string(SHTG_MAX_GROUPS) + " groups");
        return SHTG_ERR_ARG;
    }
    Plan *acct = ps[0];
    int dev = 0, nsm = 0;
    SHTG_CUDA(cudaGetDevice(&dev));
    SHTG_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    prof_begin(acct, sizeof(T) == 8 ? K_RING64 : K_RING32, st);
    int nl = 0;
    // classes by FIX (0: the generic passes of the buckets <= 1024, 64 threads)
    for (int fix : {13, 12, 11, 10, 0}) {
        RingGroups<T> G{};
        size_t smem = 0;
        int npair = 0;
        for (int g = 0; g < ng; ++g)
            for (const Plan::RingLaunch &b : ps[g]->ring_launch)
                if (b.fix == fix && b.count > 0) {
                    if (G.ne == SHTG_RING_ENTRIES) {
                        set_error("grouped ring launch: more than " + std::to_string(SHTG_RING_ENTRIES) +
                                  " launch buckets of one length");
                        return SHTG_ERR_ARG;
                    }
                    RingArgs<T> a = ring_args<T>(ps[g]);
                    size_t sm = 0;
                    ring_bucket_args<T>(ps[g], b, a, sm);
                    a.FG = FG[g];
                    a.nmaps = nmaps[g];
                    a.nT = nT[g];
                    a.ninv = ninv[g];
                    smem = std::max(smem, sm);
                    G.a[G.ne] = a;
                    G.count[G.ne] = b.count;
                    G.active[G.ne] = active ? active[g] : nullptr;
                    G.ne += 1;
                    npair += b.count;
                }
        if (G.ne == 0) continue;
        // maps per CTA as in the plan's launches: enough CTAs for about four
        // waves, at least two maps per CTA
        const int nt = fix ? (1 << fix) / 16 : 64;
        const int per = std::max(1, (sizeof(T) == 4 ? (fix > 0 ? 1024 : 512) : 256) / nt);
        const int want = 4 * nsm * per;
        int64_t total = 0;
        for (int e = 0; e < G.ne; ++e) {
            RingArgs<T> &a = G.a[e];
            int groups = (want + npair - 1) / npair;
            groups = std::max(1, std::min(groups, (a.nmaps + 1) / 2));
            a.mpg = (a.nmaps + groups - 1) / groups;
            groups = (a.nmaps + a.mpg - 1) / a.mpg;
            G.first[e] = (int)total;
            total += (int64_t)G.count[e] * groups;
            if (total > 0x7fffffff) {
                set_error("grouped ring launch: too many CTAs");
                return SHTG_ERR_ARG;
            }
        }
        G.first[G.ne] = (int)total;
        int rc = SHTG_OK;
        switch (fix) {
            case 10: rc = launch_ring_grp<T, 2, 64, 10>(G, smem, total, st); break;
            case 11: rc = launch_ring_grp<T, 2, 128, 11>(G, smem, total, st); break;
            case 12: rc = launch_ring_grp<T, 2, 256, 12>(G, smem, total, st); break;
            case 13: rc = launch_ring_grp<T, 2, 512, 13>(G, smem, total, st); break;
            default: rc = launch_ring_grp<T, 2, 64, 0>(G, smem, total, st); break;
        }
        if (rc != SHTG_OK) return rc;
        ++nl;
    }
    prof_end(acct, st, nl);
    SHTG_CHECK_LAUNCH("k_ring_grp");
    return SHTG_OK;
}
template int ring_fused_grp<float>(int, Plan *const *, float2 *const *, const int *, const int *,
                                   const float *const *, const int *const *, cudaStream_t);

template <typename T>
int ring_synth(Plan *p, const typename VT<T>::C *F, int nmaps, T *map, cudaStream_t st) {
    RingArgs<T> a = ring_args<T>(p);
    a.FG = const_cast<typename VT<T>::C *>(F);
    a.map = map;
    a.nmaps = nmaps;
    return launch_ring<T, 0>(p, a, st);
}
template <typename T>
int ring_analysis(Plan *p, const T *map, int nmaps, int weighted, typename VT<T>::C *G,
                  cudaStream_t st) {
    RingArgs<T> a = ring_args<T>(p);
    a.FG = G;
    a.map = const_cast<T *>(map);
    a.nmaps = nmaps;
    a.weighted = weighted;
    return launch_ring<T, 1>(p, a, st);
}
template <typename T>
int ring_fused(Plan *p, typename VT<T>::C *FG, int nmaps, int nT, const T *ninv,
               cudaStream_t st) {
    RingArgs<T> a = ring_args<T>(p);
    a.FG = FG;
    a.nmaps = nmaps;
    a.nT = nT;
    a.ninv = ninv;
    return launch_ring<T, 2>(p, a, st);
}

template int ring_synth<float>(Plan *, const float2 *, int, float *, cudaStream_t);
template int ring_synth<double>(Plan *, const double2 *, int, double *, cudaStream_t);
template int ring_analysis<float>(Plan *, const float *, int, int, float2 *, cudaStream_t);
template int ring_analysis<double>(Plan *, const double *, int, int, double2 *, cudaStream_t);
template int ring_fused<float>(Plan *, float2 *, int, int, const float *, cudaStream_t);
template int ring_fused<double>(Plan *, double2 *, int, int, const double *, cudaStream_t);

}  // namespace shtg

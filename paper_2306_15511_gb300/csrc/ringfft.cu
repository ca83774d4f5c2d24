// Ring stage of the spherical-harmonic transforms: on each iso-latitude ring
// the field is f(phi_j) = sum_{m=-L..L} F(m) e^{i m (phi0 + 2 pi j / n)} with
// F(-m) = conj(F(m)) (a real field), phi0 = shift * pi / n.
//
// One CTA per ring pair.  The north and south rings of a pair have the same
// n and phi0, so one complex FFT of z = f_N + i f_S serves both.  Frequencies
// are folded modulo n (rings with n < 2L + 1 alias), the length-n DFT runs in
// shared memory as a radix-2 decimation-in-frequency / decimation-in-time
// pair (bit-reversed order never has to be undone), and rings whose n is not
// a power of two use Bluestein's chirp convolution with precomputed kernel
// spectra.  The fused variant applies N^-1 between the inverse and the
// forward transform, so the pixel map never goes to global memory inside an
// operator application.
#include "common.cuh"

namespace shtg {

#define RFFT_THREADS 512

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }

// e^{i pi q / n} for integer q in [0, n)
__device__ __forceinline__ float2 phase_pi(int q, int n, float) {
    float s, c;
    sincospif((float)q / (float)n, &s, &c);
    return make_float2(c, s);
}
__device__ __forceinline__ double2 phase_pi(int q, int n, double) {
    double s, c;
    sincospi((double)q / (double)n, &s, &c);
    return make_double2(c, s);
}

template <typename T> struct RingArgs {
    typedef typename VT<T>::C C;
    int lmax, nring, npairs, nmaps;
    int64_t npix;
    const RingFFT *rf;
    const int64_t *ofs;
    const double *wring;
    const C *tw;
    int logmax;
    const C *chirp, *bfwd, *binv;
    C *FG;            // [map][ring][m]
    T *map;           // [map][npix]
    const T *ninv;    // fused: [comp][npix]
    int nT;           // fused: rows [0, nT) use N^-1 component 0 (T), later rows component 1 (Q, U)
    int weighted;     // analysis: multiply by the quadrature weight
    const int *pairs; // ring pairs handled by this launch (one CTA each)
};

// radix-2 DIF: natural order in, bit-reversed order out
template <typename C>
__device__ __forceinline__ void fft_dif(C *buf, const int logM, const C *__restrict__ tw,
                                        const int logmax, const bool inv) {
    const int M = 1 << logM;
    for (int s = 0; s < logM; ++s) {
        const int lh = logM - 1 - s;
        const int half = 1 << lh;
        for (int b = threadIdx.x; b < (M >> 1); b += blockDim.x) {
            const int k = b & (half - 1);
            const int i0 = ((b >> lh) << (lh + 1)) + k;
            const int i1 = i0 + half;
            C w = tw[k << (logmax - 1 - lh)];
            if (inv) w.y = -w.y;
            const C x0 = buf[i0], x1 = buf[i1];
            buf[i0] = cadd(x0, x1);
            buf[i1] = cmul(csub(x0, x1), w);
        }
        __syncthreads();
    }
}

// radix-2 DIT: bit-reversed order in, natural order out
template <typename C>
__device__ __forceinline__ void fft_dit(C *buf, const int logM, const C *__restrict__ tw,
                                        const int logmax, const bool inv) {
    const int M = 1 << logM;
    for (int lh = 0; lh < logM; ++lh) {
        const int half = 1 << lh;
        for (int b = threadIdx.x; b < (M >> 1); b += blockDim.x) {
            const int k = b & (half - 1);
            const int i0 = ((b >> lh) << (lh + 1)) + k;
            const int i1 = i0 + half;
            C w = tw[k << (logmax - 1 - lh)];
            if (inv) w.y = -w.y;
            const C x0 = buf[i0];
            const C x1 = cmul(buf[i1], w);
            buf[i0] = cadd(x0, x1);
            buf[i1] = csub(x0, x1);
        }
        __syncthreads();
    }
}

__device__ __forceinline__ int brev(int i, int logM) {
    return logM ? (int)(__brev((unsigned)i) >> (32 - logM)) : 0;
}

// Bluestein convolution core: buf holds a (natural, zero padded); on return buf
// holds the circular convolution with the kernel whose scaled spectrum is bh
// (bit-reversed order).
template <typename C>
__device__ __forceinline__ void blue_conv(C *buf, const int logM, const C *__restrict__ bh,
                                          const C *__restrict__ tw, const int logmax) {
    fft_dif(buf, logM, tw, logmax, false);
    for (int i = threadIdx.x; i < (1 << logM); i += blockDim.x) buf[i] = cmul(buf[i], bh[i]);
    __syncthreads();
    fft_dit(buf, logM, tw, logmax, true);
}

template <typename T, int MODE>
__global__ void __launch_bounds__(RFFT_THREADS) k_ring(const RingArgs<T> a) {
    typedef typename VT<T>::C C;
    extern __shared__ unsigned char s_raw[];
    C *buf = reinterpret_cast<C *>(s_raw);
    const int pr = a.pairs[blockIdx.x];
    const int rn = pr, rs = a.nring - 1 - pr;
    const bool single = (rn == rs);
    const RingFFT f = a.rf[rn];
    const int n = f.n, logM = f.logM, M = 1 << logM;
    const int L = a.lmax;
    const C *chirp = a.chirp + f.chirp_off;
    const C zero = {T(0), T(0)};

    for (int q = 0; q < a.nmaps; ++q) {
        if (MODE == 0 || MODE == 2) {
            // ---- fold F into the length-n spectrum of z = f_N + i f_S
            const C *Fn = a.FG + ((int64_t)q * a.nring + rn) * (L + 1);
            const C *Fs = a.FG + ((int64_t)q * a.nring + rs) * (L + 1);
            // H(k) = e^{i pi s k / n} [ sum_t (-1)^{s t} F(k + t n)
            //                         + sum_t (-1)^{s (t+1)} conj F(n - k + t n) ]
            // (phi0 = s pi / n): one phase per bin, a sign per folded term.
            for (int k = threadIdx.x; k < n; k += blockDim.x) {
                C hn = zero, hs = zero;
                T sg = T(1);
                for (int mm = k; mm <= L; mm += n) {
                    const C vn = Fn[mm];
                    hn.x += sg * vn.x;
                    hn.y += sg * vn.y;
                    if (!single) {
                        const C vs = Fs[mm];
                        hs.x += sg * vs.x;
                        hs.y += sg * vs.y;
                    }
                    if (f.shift) sg = -sg;
                }
                sg = f.shift ? T(-1) : T(1);
                for (int mm = (k == 0 ? n : n - k); mm <= L; mm += n) {
                    const C vn = Fn[mm];
                    hn.x += sg * vn.x;
                    hn.y -= sg * vn.y;
                    if (!single) {
                        const C vs = Fs[mm];
                        hs.x += sg * vs.x;
                        hs.y -= sg * vs.y;
                    }
                    if (f.shift) sg = -sg;
                }
                if (f.shift) {
                    const C ph = phase_pi(k, n, T(0));
                    hn = cmul(hn, ph);
                    hs = cmul(hs, ph);
                }
                const C z = {hn.x - hs.y, hn.y + hs.x};
                buf[k] = f.blue ? cmul(z, cconj(chirp[k])) : z;
            }
            if (f.blue)
                for (int k = n + threadIdx.x; k < M; k += blockDim.x) buf[k] = zero;
            __syncthreads();
            // ---- inverse DFT (e^{+2 pi i jk/n})
            if (f.blue) blue_conv(buf, logM, a.binv + f.bhat_off, a.tw, a.logmax);
            else fft_dif(buf, logM, a.tw, a.logmax, true);   // z_j at buf[brev(j)]
            if (MODE == 0) {
                T *mn = a.map + (int64_t)q * a.npix + a.ofs[rn];
                T *ms = a.map + (int64_t)q * a.npix + a.ofs[rs];
                for (int j = threadIdx.x; j < n; j += blockDim.x) {
                    const C z = f.blue ? cmul(buf[j], cconj(chirp[j])) : buf[brev(j, logM)];
                    mn[j] = z.x;
                    if (!single) ms[j] = z.y;
                }
                __syncthreads();
                continue;
            }
            // ---- fused N^-1 weighting
            const int comp = q < a.nT ? 0 : 1;
            const T *wn = a.ninv + (int64_t)comp * a.npix + a.ofs[rn];
            const T *ws = a.ninv + (int64_t)comp * a.npix + a.ofs[rs];
            if (f.blue) {
                for (int j = threadIdx.x; j < n; j += blockDim.x) {
                    const C c = chirp[j];
                    const C z = cmul(buf[j], cconj(c));
                    const C y = {z.x * wn[j], single ? T(0) : z.y * ws[j]};
                    buf[j] = cmul(y, c);
                }
                for (int k = n + threadIdx.x; k < M; k += blockDim.x) buf[k] = zero;
            } else {
                for (int i = threadIdx.x; i < n; i += blockDim.x) {
                    const int j = brev(i, logM);
                    const C z = buf[i];
                    buf[i] = C{z.x * wn[j], single ? T(0) : z.y * ws[j]};
                }
            }
            __syncthreads();
        } else {
            // ---- MODE 1: load z = w (m_N + i m_S)
            const T *mn = a.map + (int64_t)q * a.npix + a.ofs[rn];
            const T *ms = a.map + (int64_t)q * a.npix + a.ofs[rs];
            const T w = a.weighted ? T(a.wring[rn]) : T(1);
            for (int j = threadIdx.x; j < n; j += blockDim.x) {
                const C z = {mn[j] * w, single ? T(0) : ms[j] * w};
                if (f.blue) buf[j] = cmul(z, chirp[j]);
                else buf[brev(j, logM)] = z;
            }
            if (f.blue)
                for (int k = n + threadIdx.x; k < M; k += blockDim.x) buf[k] = zero;
            __syncthreads();
        }
        // ---- forward DFT (e^{-2 pi i jk/n}) of the bit-reversed (direct) or
        //      chirped (Bluestein) buffer; result W in natural order
        if (f.blue) blue_conv(buf, logM, a.bfwd + f.bhat_off, a.tw, a.logmax);
        else fft_dit(buf, logM, a.tw, a.logmax, false);
        // ---- unfold: G(m) = e^{-i m phi0} Y(m mod n), split north / south
        C *Gn = a.FG + ((int64_t)q * a.nring + rn) * (L + 1);
        C *Gs = a.FG + ((int64_t)q * a.nring + rs) * (L + 1);
        // G(k + t n) = (-1)^{s t} e^{-i pi s k / n} Y(k), one phase per bin
        const int nk = min(n, L + 1);
        for (int k = threadIdx.x; k < nk; k += blockDim.x) {
            const int k2 = (n - k) % n;
            C w1 = buf[k], w2 = buf[k2];
            if (f.blue) {
                w1 = cmul(w1, chirp[k]);
                w2 = cmul(w2, chirp[k2]);
            }
            C yn = {T(0.5) * (w1.x + w2.x), T(0.5) * (w1.y - w2.y)};
            C ys = {T(0.5) * (w1.y + w2.y), T(-0.5) * (w1.x - w2.x)};
            if (f.shift) {
                const C ph = cconj(phase_pi(k, n, T(0)));
                yn = cmul(yn, ph);
                ys = cmul(ys, ph);
            }
            for (int mm = k; mm <= L; mm += n) {
                Gn[mm] = yn;
                if (!single) Gs[mm] = ys;
                if (f.shift) {
                    yn.x = -yn.x;
                    yn.y = -yn.y;
                    ys.x = -ys.x;
                    ys.y = -ys.y;
                }
            }
        }
        __syncthreads();
    }
}

template <typename T> static RingArgs<T> ring_args(Plan *p);
template <> RingArgs<float> ring_args<float>(Plan *p) {
    RingArgs<float> a{};
    a.tw = p->d_tw32;
    a.chirp = p->d_chirp32;
    a.bfwd = p->d_bfwd32;
    a.binv = p->d_binv32;
    return a;
}
template <> RingArgs<double> ring_args<double>(Plan *p) {
    RingArgs<double> a{};
    a.tw = p->d_tw64;
    a.chirp = p->d_chirp64;
    a.bfwd = p->d_bfwd64;
    a.binv = p->d_binv64;
    return a;
}

template <typename T, int MODE>
static int launch_ring(Plan *p, RingArgs<T> a, cudaStream_t st) {
    a.lmax = p->lmax;
    a.nring = p->nring;
    a.npairs = p->npairs;
    a.npix = p->npix;
    a.rf = p->d_rfft;
    a.ofs = p->d_ofs;
    a.wring = p->d_wring;
    a.logmax = p->fft_logmax;
    auto kern = k_ring<T, MODE>;
    // direct (power-of-two) and Bluestein ring pairs run as separate launches so
    // that each gets the shared memory its own transform length needs
    prof_begin(p, sizeof(T) == 8 ? K_RING64 : K_RING32, st);
    for (int g = 0; g < 2; ++g) {
        const int cnt = p->ring_group_count[g];
        if (cnt == 0) continue;
        const size_t smem = sizeof(typename VT<T>::C) << p->ring_group_logm[g];
        if (smem > 48 * 1024)
            SHTG_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        a.pairs = p->d_ring_groups + (g ? p->ring_group_count[0] : 0);
        kern<<<cnt, RFFT_THREADS, smem, st>>>(a);
    }
    prof_end(p, st, (p->ring_group_count[0] > 0) + (p->ring_group_count[1] > 0));
    SHTG_CHECK_LAUNCH("k_ring");
    return SHTG_OK;
}

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

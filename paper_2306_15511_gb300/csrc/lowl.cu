// Two-level preconditioner: the exact inverse of the operator of Eq.
// (mapmakingeq) on the low multipoles l <= l_c (every m and component) plus
// the diagonal preconditioner on the rest, i.e. block Jacobi with one dense
// block.  Sect. 4 names preconditioners beyond the diagonal one as the way
// to cut the cost of the CG solves; under a mask the slowest modes are the
// large scales that the mask couples, which this block treats exactly.
//
// Real parametrization.  A stored a_lm = u + i v (m >= 0; no v at m = 0)
// enters a field channel (T, or Q and U) as c Re(zeta F(m) e^{i m phi}),
// c = 1 for m = 0 and 2 otherwise, zeta = 1 for u and i for v, F(m) the
// ring's Legendre term of a unit a_lm (the convention of the synthesis:
// spin 0 F_T = lambda; spin 2 F_Q = -(E lw + i B lx), F_U = i E lx - B lw).
// In the metric <a, c> = sum w (u u' + v v') (w = c) the transpose Y^T of the
// library is W^-1 Phi^T, so on the low parameters A = W^-1 H with the
// symmetric
//
//   H_ij = b_l(i) b_l(j) G_ij + w_i [S^-1]_{comp(i) comp(j)}(l) delta_(l m part),
//   G_ij = sum_p N^-1_p phi_i(p) phi_j(p),
//
// and the preconditioner applies z = A^-1 r = H^-1 (w r) there.  G is exact,
// done per ring with the ring's Fourier coefficients of N^-1,
// W_r(k) = sum_j N^-1_j e^{-i k phi_j}:  with rho = zeta F,
//
//   sum_j N^-1_j Re(rho_i e^{i a phi_j}) Re(rho_j e^{i b phi_j})
//       = Re[rho_i rho_j conj W(a + b) + rho_i conj(rho_j) conj W(a - b)] / 2,
//
// W(-k) = conj W(k), summed over the channels the two parameters share (Q
// and U share one N^-1; temperature and polarization share none).  The south
// ring of a pair takes the parity of the Legendre functions (App. A):
// lambda(pi - theta) = (-1)^(l-m) lambda(theta); lw has that parity and lx
// the opposite one.  G depends on N^-1 and the geometry only and is kept
// between calls while N^-1 stays bitwise the same.  H is inverted in FP64 by
// the sweep operator (Gauss-Jordan in place on a symmetric positive definite
// matrix, no pivoting, one launch per pivot).
#include <algorithm>
#include <string>
#include <vector>

#include "common.cuh"

namespace shtg {
namespace {

constexpr int LT = 32;      // Gram tile edge
constexpr int LPC = 4;      // ring pairs staged per Gram chunk
constexpr int LOWB = 32;    // CTAs per system of the apply kernel

__host__ __device__ __forceinline__ int lo_idx(int l, int m) { return l * (l + 1) / 2 + m; }

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cmulc(double2 a, double2 b) {   // a conj(b)
    return make_double2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}

// W[ch][ring][k] = sum_j N^-1_j e^{-i k phi_j}, k = 0 .. kmax, phi_j =
// pi (shift + 2 j) / n with the argument reduced exactly in integers; one
// warp per k, lanes over the ring's pixels.
__global__ void __launch_bounds__(256) k_lowl_dft(const double *__restrict__ ninv, int64_t npix,
                                                  const int *__restrict__ nphi, const int64_t *__restrict__ ofs,
                                                  const int *__restrict__ shift, int nring, int kmax,
                                                  double2 *__restrict__ W) {
    const int r = blockIdx.x, ch = blockIdx.y;
    const int n = nphi[r];
    const double *v = ninv + (int64_t)ch * npix + ofs[r];
    const int s = shift[r];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int k = warp; k <= kmax; k += 8) {
        double re = 0.0, im = 0.0;
        for (int j = lane; j < n; j += 32) {
            const int64_t q = ((int64_t)k * (s + 2 * j)) % (2 * (int64_t)n);
            double sn, cs;
            sincospi((double)q / (double)n, &sn, &cs);
            const double x = v[j];
            re = fma(x, cs, re);
            im = fma(-x, sn, im);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            re += __shfl_xor_sync(0xffffffffu, re, o);
            im += __shfl_xor_sync(0xffffffffu, im, o);
        }
        if (lane == 0) W[((int64_t)ch * nring + r) * (kmax + 1) + k] = make_double2(re, im);
    }
}

// Legendre profiles on the north ring of each pair, l <= lc, from the
// plan's FP64 recurrence tables with the steps and start-state injection of
// the synthesis: spin 0 lam[lo][pair]; spin 2 lw, lx [lo][pair].
__global__ void k_lowl_prof0(int lmax, int lc, int npairs, const double *__restrict__ u64,
                             const double2 *__restrict__ rec, const int *__restrict__ ls,
                             const double2 *__restrict__ st, double *__restrict__ lam) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    const int m = blockIdx.y;
    if (p >= npairs) return;
    const int64_t base = (int64_t)m * (2 * lmax + 1 - m) / 2;
    const int64_t o = (int64_t)m * npairs + p;
    const int l0 = ls[o];
    const double2 s = st[o];
    const double u = u64[p];
    double a1 = 0.0, a2 = 0.0;
    for (int l = m; l <= lc; ++l) {
        const double2 cf = rec[base + l];
        const double t = cf.x * a1;
        const double v = fma(t, -u, fma(cf.y, a2, t));
        a2 = a1;
        a1 = v;
        if (l == l0) {
            a2 = s.x;
            a1 = s.y;
        }
        lam[(int64_t)lo_idx(l, m) * npairs + p] = a1;
    }
}

__global__ void k_lowl_prof2(int lmax, int lc, int npairs, const double *__restrict__ u64,
                             const double4_32a *__restrict__ s2c, const int2 *__restrict__ ls2,
                             const double4_32a *__restrict__ st2, double *__restrict__ lw,
                             double *__restrict__ lx) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    const int m = blockIdx.y;
    if (p >= npairs) return;
    const int64_t base = (int64_t)m * (2 * lmax + 1 - m) / 2;
    const int64_t o = (int64_t)m * npairs + p;
    const int2 q = ls2[o];
    const double4_32a s = st2[o];
    const double u = u64[p];
    double a1 = 0.0, a2 = 0.0, b1 = 0.0, b2 = 0.0;   // y+, y-
    for (int l = m; l <= lc; ++l) {
        const double4_32a cf = s2c[base + l];
        const double tp = fma(-cf.x, u, cf.y), tm = fma(-cf.x, u, cf.z);
        const double pn = fma(tp, a1, -cf.w * a2), mn = fma(tm, b1, -cf.w * b2);
        a2 = a1;
        a1 = pn;
        b2 = b1;
        b1 = mn;
        if (l == q.x) {
            a2 = s.x;
            a1 = s.y;
        }
        if (l == q.y) {
            b2 = s.z;
            b1 = s.w;
        }
        const int64_t e = (int64_t)lo_idx(l, m) * npairs + p;
        lw[e] = a1 + b1;
        lx[e] = a1 - b1;
    }
}

// rho of parameter par = (l, m, comp, part) on the north (z = 0) or south
// (z = 1) ring of pair p: (c0, c1) = (rho_T, 0) or (rho_Q, rho_U)
__device__ __forceinline__ void lowl_rho(int4 par, int p, int z, int npairs, const double *__restrict__ lam,
                                         const double *__restrict__ lw, const double *__restrict__ lx,
                                         double2 &c0, double2 &c1) {
    const int64_t e = (int64_t)lo_idx(par.x, par.y) * npairs + p;
    const double sg = (z && ((par.x - par.y) & 1)) ? -1.0 : 1.0;   // parity on the south ring
    if (par.z == 0) {
        c0 = make_double2(sg * lam[e], 0.0);
        c1 = make_double2(0.0, 0.0);
    } else {
        const double w = sg * lw[e], x = (z ? -sg : 1.0) * lx[e];
        if (par.z == 1) {   // E: Q = -lw, U = i lx
            c0 = make_double2(-w, 0.0);
            c1 = make_double2(0.0, x);
        } else {            // B: Q = -i lx, U = -lw
            c0 = make_double2(0.0, -x);
            c1 = make_double2(-w, 0.0);
        }
    }
    if (par.w) {   // zeta = i
        c0 = make_double2(-c0.y, c0.x);
        c1 = make_double2(-c1.y, c1.x);
    }
}

// G over the full parameter list: lower-triangle 32 x 32 tiles (mirrored),
// 16 x 16 threads with 2 x 2 entries each; W [ch][ring][kw]
__global__ void __launch_bounds__(256) k_lowl_gram(int n, int npairs, int nring, int kw, int nch,
                                                   const int4 *__restrict__ par, const double *__restrict__ lam,
                                                   const double *__restrict__ lw, const double *__restrict__ lx,
                                                   const double2 *__restrict__ W, double *__restrict__ G) {
    __shared__ double2 si[2][LPC][2][LT], sj[2][LPC][2][LT];   // [side][pair][c0 / c1][param]
    __shared__ double2 sw[2][LPC][2][2 * SHTG_LOWL_LCMAX + 1];   // [ch][pair][side][k]
    const int t = blockIdx.x;
    int ti = (int)((sqrt(8.0 * t + 1.0) - 1.0) / 2.0);
    while (ti * (ti + 1) / 2 > t) --ti;
    while ((ti + 1) * (ti + 2) / 2 <= t) ++ti;
    const int tj = t - ti * (ti + 1) / 2;
    const int i0 = ti * LT, j0 = tj * LT;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    int4 pi[2], pj[2];
    for (int a = 0; a < 2; ++a) {
        const int i = i0 + 2 * ty + a, j = j0 + 2 * tx + a;
        pi[a] = i < n ? par[i] : make_int4(0, 0, -1, 0);
        pj[a] = j < n ? par[j] : make_int4(0, 0, -1, 0);
    }
    // a tile whose rows are all temperature and columns all polarization (or
    // the reverse) shares no channel: zero
    const int ci0 = par[i0].z != 0, ci1 = par[min(i0 + LT, n) - 1].z != 0;
    const int cj0 = par[j0].z != 0, cj1 = par[min(j0 + LT, n) - 1].z != 0;
    const bool any = !(ci0 == ci1 && cj0 == cj1 && ci0 != cj0);
    double acc[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
    const int kmax = kw - 1;
    for (int p0 = 0; any && p0 < npairs; p0 += LPC) {
        __syncthreads();
        for (int e = threadIdx.x; e < 2 * LPC * LT; e += 256) {
            const int z = e / (LPC * LT), q = (e / LT) % LPC, c = e % LT;
            const int p = p0 + q;
            const bool live = p < npairs && !(z && nring - 1 - p == p);
            double2 a0 = make_double2(0.0, 0.0), a1 = a0, b0 = a0, b1 = a0;
            if (live && i0 + c < n) lowl_rho(par[i0 + c], p, z, npairs, lam, lw, lx, a0, a1);
            if (live && j0 + c < n) lowl_rho(par[j0 + c], p, z, npairs, lam, lw, lx, b0, b1);
            si[z][q][0][c] = a0;
            si[z][q][1][c] = a1;
            sj[z][q][0][c] = b0;
            sj[z][q][1][c] = b1;
        }
        for (int e = threadIdx.x; e < nch * LPC * 2 * kw; e += 256) {
            const int ch = e / (LPC * 2 * kw), q = (e / (2 * kw)) % LPC, z = (e / kw) & 1, k = e % kw;
            const int p = p0 + q;
            double2 v = make_double2(0.0, 0.0);
            if (p < npairs) {
                const int r = z ? nring - 1 - p : p;
                if (!(z && r == p)) v = W[((int64_t)ch * nring + r) * kw + k];
            }
            sw[ch][q][z][k] = v;
        }
        __syncthreads();
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int b = 0; b < 2; ++b) {
                const int4 I = pi[a], J = pj[b];
                const int chi = I.z != 0;
                if (I.z < 0 || J.z < 0 || chi != (J.z != 0)) continue;
                const int ks = I.y + J.y, kd = I.y - J.y;
                if (ks > kmax) continue;
                double s = 0.0;
#pragma unroll
                for (int z = 0; z < 2; ++z)
#pragma unroll
                    for (int q = 0; q < LPC; ++q) {
                        const double2 x0 = si[z][q][0][2 * ty + a], x1 = si[z][q][1][2 * ty + a];
                        const double2 y0 = sj[z][q][0][2 * tx + b], y1 = sj[z][q][1][2 * tx + b];
                        const double2 p00 = cmul(x0, y0), p11 = cmul(x1, y1);
                        const double2 c00 = cmulc(x0, y0), c11 = cmulc(x1, y1);
                        const double2 ws = sw[chi][q][z][ks];
                        double2 wd = sw[chi][q][z][kd >= 0 ? kd : -kd];
                        if (kd < 0) wd.y = -wd.y;
                        // Re(A conj W(a + b)) + Re(B conj W(a - b))
                        s += (p00.x + p11.x) * ws.x + (p00.y + p11.y) * ws.y + (c00.x + c11.x) * wd.x +
                             (c00.y + c11.y) * wd.y;
                    }
                acc[a][b] += s;
            }
    }
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const int i = i0 + 2 * ty + a, j = j0 + 2 * tx + b;
            if (i >= n || j >= n) continue;
            const double ci = pi[a].y ? 2.0 : 1.0, cj = pj[b].y ? 2.0 : 1.0;
            const double v = 0.5 * ci * cj * acc[a][b];
            G[(int64_t)i * n + j] = v;
            G[(int64_t)j * n + i] = v;
        }
}

// H over the active parameters (sel[a] indexes the full list); flag bit 1
// if a diagonal entry is not positive
__global__ void k_lowl_assemble(int n, int nfull, const int *__restrict__ sel, const int4 *__restrict__ par,
                                const double *__restrict__ G, const double *__restrict__ ltab, int lmax1,
                                double isc, double *__restrict__ H, int *__restrict__ flag) {
    const int64_t nn = (int64_t)n * n;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nn; e += (int64_t)gridDim.x * blockDim.x) {
        const int a = (int)(e / n), b = (int)(e % n);
        const int fa = sel[a], fb = sel[b];
        const int4 I = par[fa], J = par[fb];
        double v = ltab[I.x] * ltab[J.x] * G[(int64_t)fa * nfull + fb];
        if (I.x == J.x && I.y == J.y && I.w == J.w) {
            const int c1 = min(I.z, J.z), c2 = max(I.z, J.z);
            int row = 0;   // S^-1 rows of the per-l table: 1 TT, 2 TE, 3 EE, 4 BB
            if (c1 == 0 && c2 == 0) row = 1;
            else if (c1 == 0 && c2 == 1) row = 2;
            else if (c1 == 1 && c2 == 1) row = 3;
            else if (c1 == 2 && c2 == 2) row = 4;
            if (row) v += (I.y ? 2.0 : 1.0) * ltab[row * lmax1 + I.x] * isc;
        }
        H[e] = v;
        if (a == b && !(v > 0.0)) atomicOr(flag, 1);
    }
}

// one pivot of the sweep operator, out = sweep_k(in) (flag bit 2 if the
// pivot is not positive); after every pivot, out = -H^-1
__global__ void k_lowl_sweep(int n, int k, const double *__restrict__ in, double *__restrict__ out,
                             int *__restrict__ flag) {
    const int64_t nn = (int64_t)n * n;
    const double d = in[(int64_t)k * n + k];
    if (blockIdx.x == 0 && threadIdx.x == 0 && !(d > 0.0)) atomicOr(flag, 2);
    const double id = 1.0 / d;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nn; e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / n), j = (int)(e % n);
        double v;
        if (i == k && j == k) v = -id;
        else if (i == k || j == k) v = in[e] * id;
        else v = fma(-in[(int64_t)i * n + k] * id, in[(int64_t)k * n + j], in[e]);
        out[e] = v;
    }
}

// H^-1 = -sweep (in place) and its FP32 copy
__global__ void k_lowl_finish(int64_t nn, double *__restrict__ S, float *__restrict__ h32) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nn; e += (int64_t)gridDim.x * blockDim.x) {
        const double v = -S[e];
        S[e] = v;
        h32[e] = (float)v;
    }
}

// flag |= 1 if a and b differ anywhere (bitwise)
__global__ void k_lowl_cmp(const unsigned long long *__restrict__ a, const unsigned long long *__restrict__ b,
                           int64_t n, int *__restrict__ flag) {
    int d = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        d |= a[i] != b[i];
    if (__syncthreads_or(d) && threadIdx.x == 0) atomicOr(flag, 1);
}

// z <- H^-1 (w r) on the active low parameters of system blockIdx.y (r, z
// as reals: element e of a system is entry e of its [ncomp][nalm] complex
// vector viewed as 2 ncomp nalm reals), and that system's change of <r, z>
// in lowpart[b][blockIdx.x]
template <typename T>
__global__ void __launch_bounds__(256) k_lowl_apply(int n, const int *__restrict__ emap,
                                                    const float *__restrict__ wv, const T *__restrict__ Hinv,
                                                    const T *__restrict__ r, T *__restrict__ z, int64_t per,
                                                    double *__restrict__ lowpart) {
    extern __shared__ __align__(16) unsigned char s_raw[];
    T *g = reinterpret_cast<T *>(s_raw);
    __shared__ double sm[8];
    const int b = blockIdx.y;
    const T *rb = r + 2 * (int64_t)b * per;
    T *zb = z + 2 * (int64_t)b * per;
    for (int i = threadIdx.x; i < n; i += blockDim.x) g[i] = (T)wv[i] * rb[emap[i]];
    __syncthreads();
    double corr = 0.0;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int i = blockIdx.x * nw + warp; i < n; i += gridDim.x * nw) {
        const T *h = Hinv + (int64_t)i * n;
        T s = T(0);
        for (int j = lane; j < n; j += 32) s = fma(h[j], g[j], s);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) {
            const int e = emap[i];
            const T zold = zb[e];
            zb[e] = s;
            corr += (double)wv[i] * (double)rb[e] * ((double)s - (double)zold);
        }
    }
    if (lane == 0) sm[warp] = corr;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < nw; ++w) t += sm[w];
        lowpart[b * LOWB + blockIdx.x] = t;
    }
}

// add each system's low-block change of <r, z> to its first rz partial, in a
// fixed order (graph replays stay bitwise equal to eager launches)
__global__ void k_lowl_addpart(int nb, const double *__restrict__ lowpart, double *__restrict__ part, int rb) {
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
        double t = 0.0;
        for (int c = 0; c < LOWB; ++c) t += lowpart[b * LOWB + c];
        part[((int64_t)b * 2 + 0) * rb + 0] += t;
    }
}

template <typename P> int lalloc(Plan *p, P **ptr, size_t count) {
    const size_t bytes = sizeof(P) * std::max<size_t>(count, 1);
    const cudaError_t e = cudaMalloc((void **)ptr, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *ptr = nullptr;
        set_error("two-level preconditioner: cannot allocate " + std::to_string(bytes) + " bytes");
        return SHTG_ERR_NOMEM;
    }
    p->device_bytes += (int64_t)bytes;
    p->lowl.bytes += (int64_t)bytes;
    return SHTG_OK;
}

unsigned blocks_for(int64_t n) {
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 8192));
}

// workspace for l_c and nc (kept while a later call needs no more)
int lowl_reserve(Plan *p, int lc, int nc, cudaStream_t st) {
    LowL &q = p->lowl;
    if (q.cap_lc >= lc && q.cap_nc >= nc) return SHTG_OK;
    lowl_free(p);
    const int64_t nfull = (int64_t)nc * (lc + 1) * (lc + 1), nlo = (int64_t)(lc + 1) * (lc + 2) / 2;
    const int nch = nc == 3 ? 2 : 1;
    SHTG_TRY(lalloc(p, &q.W, (size_t)nch * p->nring * (2 * lc + 1)));
    SHTG_TRY(lalloc(p, &q.lam, (size_t)(nlo * p->npairs)));
    SHTG_TRY(lalloc(p, &q.lw, (size_t)(nc == 3 ? nlo * p->npairs : 1)));
    SHTG_TRY(lalloc(p, &q.lx, (size_t)(nc == 3 ? nlo * p->npairs : 1)));
    SHTG_TRY(lalloc(p, &q.G, (size_t)(nfull * nfull)));
    SHTG_TRY(lalloc(p, &q.H, (size_t)(nfull * nfull)));
    SHTG_TRY(lalloc(p, &q.S, (size_t)(nfull * nfull)));
    SHTG_TRY(lalloc(p, &q.h32, (size_t)(nfull * nfull)));
    SHTG_TRY(lalloc(p, &q.par, (size_t)nfull));
    SHTG_TRY(lalloc(p, &q.sel, (size_t)nfull));
    SHTG_TRY(lalloc(p, &q.emap, (size_t)nfull));
    SHTG_TRY(lalloc(p, &q.wv, (size_t)nfull));
    SHTG_TRY(lalloc(p, &q.part, (size_t)p->max_batch * LOWB));
    SHTG_TRY(lalloc(p, &q.flag, 4));
    SHTG_TRY(lalloc(p, &q.shift, (size_t)p->nring));
    SHTG_TRY(lalloc(p, &q.ninv, (size_t)nch * p->npix));
    // ordered on the solve's stream (not the legacy default stream), complete
    // before returning
    SHTG_CUDA(cudaMemcpyAsync(q.shift, p->shift.data(), sizeof(int) * p->nring, cudaMemcpyHostToDevice, st));
    SHTG_CUDA(cudaStreamSynchronize(st));
    q.cap_lc = lc;
    q.cap_nc = nc;
    return SHTG_OK;
}

}  // namespace

void lowl_free(Plan *p) {
    LowL &q = p->lowl;
    void *bufs[] = {q.W, q.lam, q.lw, q.lx, q.G, q.H, q.S, q.h32, q.par, q.sel, q.emap, q.wv,
                    q.part, q.flag, q.shift, q.ninv};
    for (void *b : bufs)
        if (b) cudaFree(b);
    p->device_bytes -= q.bytes;
    q = LowL{};
}

int lowl_setup(Plan *p, int lc, int nc, double isc, cudaStream_t st, double *h_host) {
    const int lcmax = std::min(p->lmax, SHTG_LOWL_LCMAX);
    if (lc <= 0) lc = std::min(lcmax, SHTG_LOWL_LC_DEFAULT);
    if (lc > lcmax) {
        set_error("two-level preconditioner: l_c must be at most " + std::to_string(lcmax));
        return SHTG_ERR_ARG;
    }
    SHTG_TRY(lowl_reserve(p, lc, nc, st));
    LowL &q = p->lowl;
    const int L1 = p->lmax + 1;
    const int nch = nc == 3 ? 2 : 1;
    // the full parameter list (component-major, then l, m, part) and its
    // active subset (multipoles whose C_l block is not singular)
    std::vector<int4> par;
    for (int c = 0; c < nc; ++c)
        for (int l = 0; l <= lc; ++l)
            for (int m = 0; m <= l; ++m)
                for (int w = 0; w < (m ? 2 : 1); ++w) par.push_back(make_int4(l, m, c, w));
    const int nf = (int)par.size();
    // per-l rows 0 (beam), 1-4 (S^-1) and 5 (S^-1/2 TT: zero where held)
    std::vector<double> tab(6 * (size_t)L1);
    SHTG_CUDA(cudaMemcpyAsync(tab.data(), p->d_ltab64, sizeof(double) * tab.size(), cudaMemcpyDeviceToHost, st));
    SHTG_CUDA(cudaStreamSynchronize(st));
    const double *sh = tab.data() + 5 * (size_t)L1;
    std::vector<int> sel, emap;
    std::vector<float> wv;
    q.params.clear();
    for (int i = 0; i < nf; ++i) {
        const int4 a = par[i];
        if (!(sh[a.x] > 0.0)) continue;
        sel.push_back(i);
        emap.push_back((int)(2 * ((int64_t)a.z * p->nalm + alm_index(a.x, a.y, p->lmax)) + a.w));
        wv.push_back(a.y ? 2.f : 1.f);
        q.params.push_back(a);
    }
    const int n = (int)sel.size();
    const bool same = q.inv_ok && q.n == n && q.lc == lc && q.nc == nc && q.inv_isc == isc && q.inv_ltab == tab;
    q.inv_ok = false;
    q.n = n;
    q.lc = lc;
    q.nc = nc;
    if (n == 0) return SHTG_OK;
    SHTG_CUDA(cudaMemcpyAsync(q.sel, sel.data(), sizeof(int) * n, cudaMemcpyHostToDevice, st));
    SHTG_CUDA(cudaMemcpyAsync(q.emap, emap.data(), sizeof(int) * n, cudaMemcpyHostToDevice, st));
    SHTG_CUDA(cudaMemcpyAsync(q.wv, wv.data(), sizeof(float) * n, cudaMemcpyHostToDevice, st));
    // ---- G, kept while N^-1, l_c and the components are unchanged
    const int64_t nin = (int64_t)nch * p->npix;
    bool rebuild = !q.gram_ok || q.gram_lc != lc || q.gram_nc != nc;
    if (!rebuild) {
        int h = 0;
        SHTG_CUDA(cudaMemsetAsync(q.flag, 0, sizeof(int), st));
        k_lowl_cmp<<<blocks_for(nin), 256, 0, st>>>(reinterpret_cast<const unsigned long long *>(p->d_ninv64),
                                                     reinterpret_cast<const unsigned long long *>(q.ninv), nin,
                                                     q.flag);
        SHTG_CHECK_LAUNCH("k_lowl_cmp");
        SHTG_CUDA(cudaMemcpyAsync(&h, q.flag, sizeof(int), cudaMemcpyDeviceToHost, st));
        SHTG_CUDA(cudaStreamSynchronize(st));
        p->prof.launches += 1;
        rebuild = h != 0;
    }
    if (rebuild) {
        q.gram_ok = false;
        SHTG_CUDA(cudaMemcpyAsync(q.par, par.data(), sizeof(int4) * nf, cudaMemcpyHostToDevice, st));
        const int kmax = 2 * lc;
        k_lowl_dft<<<dim3(p->nring, nch), 256, 0, st>>>(p->d_ninv64, p->npix, p->d_nphi, p->d_ofs, q.shift,
                                                       p->nring, kmax, q.W);
        SHTG_CHECK_LAUNCH("k_lowl_dft");
        const dim3 pg((p->npairs + 127) / 128, lc + 1);
        k_lowl_prof0<<<pg, 128, 0, st>>>(p->lmax, lc, p->npairs, p->d_u64, p->d_rec64, p->d_ls64, p->d_st64,
                                         q.lam);
        SHTG_CHECK_LAUNCH("k_lowl_prof0");
        if (nc == 3) {
            k_lowl_prof2<<<pg, 128, 0, st>>>(p->lmax, lc, p->npairs, p->d_u64, p->d_s2c64, p->d_ls2_64,
                                             p->d_st2_64, q.lw, q.lx);
            SHTG_CHECK_LAUNCH("k_lowl_prof2");
        }
        const int nt = (nf + LT - 1) / LT;
        k_lowl_gram<<<nt * (nt + 1) / 2, 256, 0, st>>>(nf, p->npairs, p->nring, kmax + 1, nch, q.par, q.lam,
                                                       q.lw, q.lx, q.W, q.G);
        SHTG_CHECK_LAUNCH("k_lowl_gram");
        SHTG_CUDA(cudaMemcpyAsync(q.ninv, p->d_ninv64, sizeof(double) * nin, cudaMemcpyDeviceToDevice, st));
        p->prof.launches += 3 + (nc == 3);
        q.gram_ok = true;
        q.gram_lc = lc;
        q.gram_nc = nc;
    }
    // ---- H and its inverse (kept while G, the per-l table and the C_l scale
    // are unchanged, e.g. across the calls of one chain state)
    if (same && !rebuild && !h_host) {
        q.inv_ok = true;
        return SHTG_OK;
    }
    const int64_t nn = (int64_t)n * n;
    SHTG_CUDA(cudaMemsetAsync(q.flag, 0, sizeof(int), st));
    k_lowl_assemble<<<blocks_for(nn), 256, 0, st>>>(n, nf, q.sel, q.par, q.G, p->d_ltab64, L1, isc, q.H, q.flag);
    SHTG_CHECK_LAUNCH("k_lowl_assemble");
    if (h_host) SHTG_CUDA(cudaMemcpyAsync(h_host, q.H, sizeof(double) * nn, cudaMemcpyDeviceToHost, st));
    double *a = q.H, *b = q.S;
    for (int k = 0; k < n; ++k) {
        k_lowl_sweep<<<blocks_for(nn), 256, 0, st>>>(n, k, a, b, q.flag);
        std::swap(a, b);
    }
    SHTG_CHECK_LAUNCH("k_lowl_sweep");
    k_lowl_finish<<<blocks_for(nn), 256, 0, st>>>(nn, a, q.h32);
    SHTG_CHECK_LAUNCH("k_lowl_finish");
    q.h64 = a;
    p->prof.launches += 2 + n;
    int h = 0;
    SHTG_CUDA(cudaMemcpyAsync(&h, q.flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    SHTG_CUDA(cudaStreamSynchronize(st));
    if (h) {
        q.n = 0;
        set_error("two-level preconditioner: the low-l block is not positive definite");
        return SHTG_ERR_NOT_SPD;
    }
    q.inv_ltab = tab;
    q.inv_isc = isc;
    q.inv_ok = true;
    // the apply kernel stages n values per system in shared memory (at most
    // 3 x 49^2 doubles = 57.6 KB)
    if (sizeof(double) * (size_t)n > 48 * 1024) {
        SHTG_CUDA(allow_max_smem(k_lowl_apply<double>));
        SHTG_CUDA(allow_max_smem(k_lowl_apply<float>));
    }
    return SHTG_OK;
}

template <typename T>
int lowl_apply(Plan *p, const T *r, T *z, int nb, int64_t per, double *part, cudaStream_t st) {
    const LowL &q = p->lowl;
    if (q.n == 0) return SHTG_OK;
    const T *H = sizeof(T) == 8 ? reinterpret_cast<const T *>(q.h64) : reinterpret_cast<const T *>(q.h32);
    k_lowl_apply<T><<<dim3(LOWB, nb), 256, sizeof(T) * (size_t)q.n, st>>>(q.n, q.emap, q.wv, H, r, z, per, q.part);
    k_lowl_addpart<<<1, 256, 0, st>>>(nb, q.part, part, SHTG_RED_BLOCKS);
    p->prof.launches += 2;
    SHTG_CHECK_LAUNCH("k_lowl_apply");
    return SHTG_OK;
}

template int lowl_apply<float>(Plan *, const float *, float *, int, int64_t, double *, cudaStream_t);
template int lowl_apply<double>(Plan *, const double *, double *, int, int64_t, double *, cudaStream_t);

}  // namespace shtg

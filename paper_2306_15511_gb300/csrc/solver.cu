// Constrained-realization solver of Eq. (mapmakingeq), Sect. 2.2.1:
//
//     (S^-1 + B Y^T N^-1 Y B) a = B Y^T (N^-1 d + N^-1/2 w2) + S^-1/2 w1
//
// solved by preconditioned conjugate gradients (the paper uses CG with the
// diagonal preconditioner of Sect. 4).  nbatch realizations share the
// operator; each keeps its own CG scalars in device memory so that an
// iteration is a fixed launch sequence with no host round trip, and a
// realization that has converged is frozen (alpha = beta = 0) while the
// others continue.
//
// Modes: plain FP64 PCG, or FP32 PCG on A delta = r inside FP64 iterative
// refinement (r = b - A x evaluated with the FP64 transforms), which reaches
// the FP64 residual target with FP32 operator applications.
//
// Inner products use <a, c> = sum_l [a_l0 c_l0 + 2 Re sum_{m>0} conj(a_lm) c_lm],
// the metric in which Y^T is the transpose of Y and A is symmetric.
#include <chrono>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include <cstdio>

#include "common.cuh"

namespace shtg {

#define RT 256
#define RB SHTG_RED_BLOCKS

// scalar slots per realization
enum { S_RZ = 0, S_PQ, S_RR, S_BB, S_ALPHA, S_BETA, S_ACTIVE, S_ITERS, S_TOL2, S_BAD, S_SCALE, S_RESTART };

__device__ __forceinline__ double cdot(double2 a, double2 b) { return a.x * b.x + a.y * b.y; }

// Per-element partial dot products.  FP32 vectors sum the component
// products of one alm index (at most three complex terms) in FP32: one
// rounding of ~2^-24 relative per element that does not grow with the
// vector length; the caller adds the element's sum into an FP64
// accumulator.  This keeps the reductions of the FP32 iteration to two FP64
// operations per element (GB300's FP64 pipe is narrow).  FP64 vectors stay
// in FP64 throughout.
template <typename C> struct DotAcc;
template <> struct DotAcc<float2> {
    typedef float t;
    static __device__ __forceinline__ float add(float acc, float2 a, float2 b) {
        return fmaf(a.x, b.x, fmaf(a.y, b.y, acc));
    }
};
template <> struct DotAcc<double2> {
    typedef double t;
    static __device__ __forceinline__ double add(double acc, double2 a, double2 b) { return acc + cdot(a, b); }
};

__device__ double block_sum(double v, double *sm) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) sm[w] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) r += sm[i];
    return r;
}

// --------------------------------------------------------------- pixel side
// out rows [T_0 .. T_{nt-1}, Q_0, U_0, Q_1, U_1, ...] (the transform's row
// order for nt realizations) from inputs in [b][c][npix] order: realization
// b of the inputs goes to realization boff + b of the output;
// out (=|+=) N^-1 d (+ sqrt(N^-1) w2).
__global__ void k_rhs_pix(const double *__restrict__ d, const double *__restrict__ w2,
                          const double *__restrict__ ninv, int nt, int boff, int nc, int64_t npix,
                          int accumulate, double *__restrict__ out) {
    const int row = blockIdx.y;
    const int b = row / nc, c = row % nc;
    const int ob = boff + b;
    const int orow = (c == 0) ? ob : nt + 2 * ob + (c - 1);
    const double *wv = ninv + (c == 0 ? 0 : npix);
    double *o = out + (int64_t)orow * npix;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < npix;
         p += (int64_t)gridDim.x * blockDim.x) {
        // explicit roundings: host-staged inputs (two passes) and device inputs
        // (one pass) give bit-identical sums
        const double w = wv[p];
        const double t1 = d ? __dmul_rn(w, d[(int64_t)row * npix + p]) : 0.0;
        const double t2 = w2 ? __dmul_rn(sqrt(w), w2[(int64_t)row * npix + p]) : 0.0;
        double v = accumulate ? o[p] : 0.0;
        if (d) v = __dadd_rn(v, t1);
        if (w2) v = __dadd_rn(v, t2);
        o[p] = v;
    }
}

__global__ void k_to_double(const float *__restrict__ a, double *__restrict__ b, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        b[i] = (double)a[i];
}
__global__ void k_to_float(const double *__restrict__ a, float *__restrict__ b, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        b[i] = (float)a[i];
}

// sum of N^-1 over both rings of every pair
__global__ void k_wpair(const double *__restrict__ ninv, const int64_t *__restrict__ ofs,
                        const int *__restrict__ nphi, int nring, float *__restrict__ out) {
    __shared__ double sm[RT / 32];
    const int pr = blockIdx.x;
    const int rn = pr, rs = nring - 1 - pr;
    double s = 0.0;
    for (int j = threadIdx.x; j < nphi[rn]; j += blockDim.x) s += ninv[ofs[rn] + j];
    if (rs != rn)
        for (int j = threadIdx.x; j < nphi[rs]; j += blockDim.x) s += ninv[ofs[rs] + j];
    s = block_sum(s, sm);
    if (threadIdx.x == 0) out[pr] = (float)s;
}

// ------------------------------------------------------------ harmonic side
template <typename T> struct HT;
template <> struct HT<float> { typedef float2 C; };
template <> struct HT<double> { typedef double2 C; };

// y += S^-1 x (per-l 1x1 or T/E 2x2 + B block); sinv rows TT, TE, EE, BB.
// DOT: also the partial <x, y> of the result per realization (the PCG's
// <p, A p>, the operator's last kernel doing the dot's reads), launched on
// the reduction grid (RB blocks per realization) with the per-element sums
// of k_dot, so alpha is the same bit for bit.
// (the rows of realization b handled by block bx of nbx: the plan's kernel
// passes its block indices, the grouped kernel those of its group)
template <typename T, bool DOT>
__device__ __forceinline__ void prior_add_rows(const typename HT<T>::C *__restrict__ x,
                                               typename HT<T>::C *__restrict__ y, int nc, int64_t nalm,
                                               int lmax1, const int *__restrict__ lof,
                                               const T *__restrict__ sinv, const T *__restrict__ isc,
                                               const int *__restrict__ mof, double *__restrict__ part,
                                               const int b, const int bx, const int nbx) {
    typedef typename HT<T>::C C;
    __shared__ double sm[DOT ? RT / 32 : 1];
    const int64_t off = (int64_t)b * nc * nalm;
    const T sc = isc[b];   // 1 / (C_l scale of realization b)
    double s = 0.0;
    for (int64_t i = bx * (int64_t)blockDim.x + threadIdx.x; i < nalm; i += (int64_t)nbx * blockDim.x) {
        const int l = lof[i];
        const T tt = sinv[l] * sc;
        typename DotAcc<C>::t t = 0;
        if (nc == 1) {
            const C xv = x[off + i];
            C yv = y[off + i];
            yv.x += tt * xv.x;
            yv.y += tt * xv.y;
            y[off + i] = yv;
            if (DOT) t = DotAcc<C>::add(t, xv, yv);
        } else {
            const T te = sinv[lmax1 + l] * sc, ee = sinv[2 * lmax1 + l] * sc, bb = sinv[3 * lmax1 + l] * sc;
            const C xt = x[off + i], xe = x[off + nalm + i], xb = x[off + 2 * nalm + i];
            C yt = y[off + i], ye = y[off + nalm + i], yb = y[off + 2 * nalm + i];
            yt.x += tt * xt.x + te * xe.x;
            yt.y += tt * xt.y + te * xe.y;
            ye.x += te * xt.x + ee * xe.x;
            ye.y += te * xt.y + ee * xe.y;
            yb.x += bb * xb.x;
            yb.y += bb * xb.y;
            y[off + i] = yt;
            y[off + nalm + i] = ye;
            y[off + 2 * nalm + i] = yb;
            if (DOT) {
                t = DotAcc<C>::add(t, xt, yt);
                t = DotAcc<C>::add(t, xe, ye);
                t = DotAcc<C>::add(t, xb, yb);
            }
        }
        if (DOT) s += (mof[i] ? 2.0 : 1.0) * (double)t;
    }
    if (DOT) {
        s = block_sum(s, sm);
        if (threadIdx.x == 0) part[(int64_t)b * RB + bx] = s;
    }
}
template <typename T, bool DOT>
__global__ void k_prior_add(const typename HT<T>::C *__restrict__ x, typename HT<T>::C *__restrict__ y,
                            int nc, int64_t nalm, int lmax1, const int *__restrict__ lof,
                            const T *__restrict__ sinv, const T *__restrict__ isc,
                            const int *__restrict__ mof, double *__restrict__ part) {
    prior_add_rows<T, DOT>(x, y, nc, nalm, lmax1, lof, sinv, isc, mof, part, blockIdx.y, blockIdx.x, gridDim.x);
}

// Preconditioner M = S^-1 + b_l^2 diag(D_T, D_P, D_P), stored as its inverse:
// nc = 1: minv[0] = 1 / M; nc = 3: minv[0..2] = inverse T/E block (11, 12, 22), minv[3] = 1 / M_BB.
__global__ void k_precond(const float *__restrict__ dT, const float *__restrict__ dP,
                          const double *__restrict__ ltab, int nc, int64_t nalm, int lmax1,
                          const int *__restrict__ lof, int use_diag, const double *__restrict__ isc,
                          double *__restrict__ m64, float *__restrict__ m32) {
    // realization b = blockIdx.y: S^-1 / (its C_l scale); one [4][nalm] block each
    const int b = blockIdx.y;
    const double sc = isc[b];
    m64 += (int64_t)b * 4 * nalm;
    m32 += (int64_t)b * 4 * nalm;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nalm;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int l = lof[i];
        const double b2 = use_diag ? ltab[l] * ltab[l] : 0.0;
        const double tt = ltab[lmax1 + l] * sc, te = ltab[2 * lmax1 + l] * sc, ee = ltab[3 * lmax1 + l] * sc,
                     bb = ltab[4 * lmax1 + l] * sc;
        double v[4];
        const double gT = use_diag ? b2 * (double)dT[i] : 0.0;
        const double gP = (use_diag && nc == 3) ? b2 * (double)dP[i] : 0.0;
        if (nc == 1) {
            v[0] = 1.0 / (tt + gT);
            v[1] = v[2] = v[3] = 0.0;
        } else {
            const double a11 = tt + gT, a12 = te, a22 = ee + gP;
            const double det = a11 * a22 - a12 * a12;
            v[0] = a22 / det;
            v[1] = -a12 / det;
            v[2] = a11 / det;
            v[3] = 1.0 / (bb + gP);
        }
        for (int k = 0; k < 4; ++k) {
            m64[k * nalm + i] = v[k];
            m32[k * nalm + i] = (float)v[k];
        }
    }
}

// RHS: b += S^-1/2 w1 (sinvh rows TT, TE, EE, BB)
__global__ void k_rhs_alm(const double2 *__restrict__ w1, double2 *__restrict__ bvec, int nc,
                          int64_t nalm, int lmax1, const int *__restrict__ lof,
                          const int *__restrict__ mof, const double *__restrict__ sh,
                          const double *__restrict__ rsc) {
    const int b = blockIdx.y;
    const int64_t off = (int64_t)b * nc * nalm;
    const double sc = rsc[b];   // 1 / sqrt(C_l scale of realization b)
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nalm;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int l = lof[i];
        const bool m0 = mof[i] == 0;
        const double tt = sh[l] * sc;
        if (nc == 1) {
            double2 w = w1[off + i], v = bvec[off + i];
            v.x += tt * w.x;
            v.y = m0 ? 0.0 : v.y + tt * w.y;
            bvec[off + i] = v;
        } else {
            const double te = sh[lmax1 + l] * sc, ee = sh[2 * lmax1 + l] * sc, bb = sh[3 * lmax1 + l] * sc;
            const double2 wt = w1[off + i], we = w1[off + nalm + i], wb = w1[off + 2 * nalm + i];
            double2 vt = bvec[off + i], ve = bvec[off + nalm + i], vb = bvec[off + 2 * nalm + i];
            vt.x += tt * wt.x + te * we.x;
            vt.y += tt * wt.y + te * we.y;
            ve.x += te * wt.x + ee * we.x;
            ve.y += te * wt.y + ee * we.y;
            vb.x += bb * wb.x;
            vb.y += bb * wb.y;
            if (m0) vt.y = ve.y = vb.y = 0.0;
            bvec[off + i] = vt;
            bvec[off + nalm + i] = ve;
            bvec[off + 2 * nalm + i] = vb;
        }
    }
}

// --------------------------------------------------------------- PCG kernels
// partial <a, c> per realization
template <typename C>
__global__ void k_dot(const C *__restrict__ a, const C *__restrict__ c, int nc, int64_t nalm,
                      const int *__restrict__ mof, double *__restrict__ part, int slot, int nslot) {
    __shared__ double sm[RT / 32];
    const int b = blockIdx.y;
    const int64_t off = (int64_t)b * nc * nalm;
    double s = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nalm;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double w = mof[i] ? 2.0 : 1.0;
        typename DotAcc<C>::t t = 0;
        for (int k = 0; k < nc; ++k) t = DotAcc<C>::add(t, a[off + k * nalm + i], c[off + k * nalm + i]);
        s += w * (double)t;
    }
    s = block_sum(s, sm);
    if (threadIdx.x == 0) part[((int64_t)b * nslot + slot) * RB + blockIdx.x] = s;
}

// out[b] = sum over the RB partials of realization b (slot 0 of 1), in the
// order in which the host sums them
__global__ void k_row_sums(const double *__restrict__ part, int nb, double *__restrict__ out) {
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
        double s = 0.0;
        for (int k = 0; k < RB; ++k) s += part[(int64_t)b * RB + k];
        out[b] = s;
    }
}

__device__ __forceinline__ double sum_part(const double *part, int b, int nslot, int slot) {
    double s = 0.0;
    for (int k = 0; k < RB; ++k) s += part[((int64_t)b * nslot + slot) * RB + k];
    return s;
}

// apply the preconditioner inverse block to (r_T, r_E, r_B) at alm index i
template <typename T, typename C>
__device__ __forceinline__ void apply_minv(const T *minv, int64_t nalm, int64_t i, int nc,
                                           const C *r, C *z) {
    if (nc == 1) {
        const T m = minv[i];
        z[0].x = m * r[0].x;
        z[0].y = m * r[0].y;
    } else {
        const T a = minv[i], b = minv[nalm + i], c = minv[2 * nalm + i], d = minv[3 * nalm + i];
        z[0].x = a * r[0].x + b * r[1].x;
        z[0].y = a * r[0].y + b * r[1].y;
        z[1].x = b * r[0].x + c * r[1].x;
        z[1].y = b * r[0].y + c * r[1].y;
        z[2].x = d * r[2].x;
        z[2].y = d * r[2].y;
    }
}

// INIT: z = M^-1 r and partial (rz, rr).  Otherwise x += alpha p, r -= alpha q,
// then the same.
template <typename T, bool INIT>
__device__ __forceinline__ void update_rows(typename HT<T>::C *__restrict__ x, typename HT<T>::C *__restrict__ r,
                                            typename HT<T>::C *__restrict__ z,
                                            const typename HT<T>::C *__restrict__ p,
                                            const typename HT<T>::C *__restrict__ q, const T *__restrict__ minv,
                                            int nc, int64_t nalm, const int *__restrict__ mof,
                                            const double *__restrict__ scal, double *__restrict__ part,
                                            const int b, const int bx, const int nbx) {
    typedef typename HT<T>::C C;
    __shared__ double sm[RT / 32];
    const int64_t off = (int64_t)b * nc * nalm;
    const T alpha = INIT ? T(0) : (T)scal[b * 16 + S_ALPHA];
    double srz = 0.0, srr = 0.0;
    for (int64_t i = bx * (int64_t)blockDim.x + threadIdx.x; i < nalm; i += (int64_t)nbx * blockDim.x) {
        C rv[3], zv[3];
        for (int k = 0; k < nc; ++k) {
            const int64_t e = off + k * nalm + i;
            C rr = r[e];
            if (!INIT) {
                const C pv = p[e], qv = q[e];
                C xv = x[e];
                xv.x += alpha * pv.x;
                xv.y += alpha * pv.y;
                x[e] = xv;
                rr.x -= alpha * qv.x;
                rr.y -= alpha * qv.y;
                r[e] = rr;
            }
            rv[k] = rr;
        }
        apply_minv<T, C>(minv + (int64_t)b * 4 * nalm, nalm, i, nc, rv, zv);
        const double w = mof[i] ? 2.0 : 1.0;
        typename DotAcc<C>::t a1 = 0, a2 = 0;
        for (int k = 0; k < nc; ++k) {
            z[off + k * nalm + i] = zv[k];
            a1 = DotAcc<C>::add(a1, rv[k], zv[k]);
            a2 = DotAcc<C>::add(a2, rv[k], rv[k]);
        }
        srz += w * (double)a1;
        srr += w * (double)a2;
    }
    srz = block_sum(srz, sm);
    srr = block_sum(srr, sm);
    if (threadIdx.x == 0) {
        part[((int64_t)b * 2 + 0) * RB + bx] = srz;
        part[((int64_t)b * 2 + 1) * RB + bx] = srr;
    }
}
template <typename T, bool INIT>
__global__ void k_update(typename HT<T>::C *__restrict__ x, typename HT<T>::C *__restrict__ r,
                         typename HT<T>::C *__restrict__ z, const typename HT<T>::C *__restrict__ p,
                         const typename HT<T>::C *__restrict__ q, const T *__restrict__ minv,
                         int nc, int64_t nalm, const int *__restrict__ mof,
                         const double *__restrict__ scal, double *__restrict__ part) {
    update_rows<T, INIT>(x, r, z, p, q, minv, nc, nalm, mof, scal, part, blockIdx.y, blockIdx.x, gridDim.x);
}

// The scalar kernels run one block; thread t serves realizations t, t +
// blockDim.x, ... (a plan holds up to 4096).
__global__ void k_scal_init(const double *__restrict__ part, double *__restrict__ scal, int nb,
                            double tol2) {
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
        const double rz = sum_part(part, b, 2, 0), rr = sum_part(part, b, 2, 1);
        double *s = scal + b * 16;
        s[S_RZ] = rz;
        s[S_RR] = rr;
        s[S_BB] = rr;
        s[S_TOL2] = tol2;
        s[S_ACTIVE] = (rr > 0.0) ? 1.0 : 0.0;
        s[S_ITERS] = 0.0;
        s[S_BAD] = (isfinite(rr) && isfinite(rz)) ? 0.0 : 1.0;
        s[S_ALPHA] = s[S_BETA] = 0.0;
    }
}

// floor2: the FP32 iteration of the mixed solver passes the squared
// relative residual at which its recursion reaches FP32 rounding; a finite
// non-positive curvature there (p made of rounding noise, e.g. after a
// preconditioner close to the exact inverse) ends the stage instead of
// failing it, and the FP64 residual replacement judges convergence.  The
// FP64 PCG passes 0 (any non-positive curvature is a failure).
__device__ __forceinline__ void scal_alpha_one(const double *__restrict__ part, double *__restrict__ scal,
                                               const int b, const double floor2) {
    double *s = scal + b * 16;
    const double pq = sum_part(part, b, 1, 0);
    s[S_PQ] = pq;
    double alpha = 0.0;
    if (s[S_ACTIVE] != 0.0) {
        if (pq > 0.0 && isfinite(pq)) {
            alpha = s[S_RZ] / pq;
        } else {
            s[S_ACTIVE] = 0.0;
            if (isfinite(pq) && s[S_RR] <= floor2 * s[S_BB]) s[S_RESTART] = 1.0;   // next stage: p = z
            else s[S_BAD] = 1.0;
        }
    }
    s[S_ALPHA] = alpha;
}
__global__ void k_scal_alpha(const double *__restrict__ part, double *__restrict__ scal, int nb, double floor2) {
    for (int b = threadIdx.x; b < nb; b += blockDim.x) scal_alpha_one(part, scal, b, floor2);
}

__device__ __forceinline__ void scal_beta_one(const double *__restrict__ part, double *__restrict__ scal,
                                              const int b) {
    double *s = scal + b * 16;
    const double rz = sum_part(part, b, 2, 0), rr = sum_part(part, b, 2, 1);
    double beta = 0.0;
    if (s[S_ACTIVE] != 0.0) {
        s[S_ITERS] += 1.0;
        if (!isfinite(rz) || !isfinite(rr)) {
            s[S_BAD] = 1.0;
            s[S_ACTIVE] = 0.0;
        } else {
            beta = (s[S_RZ] != 0.0) ? rz / s[S_RZ] : 0.0;
            s[S_RZ] = rz;
            s[S_RR] = rr;
            if (rr <= s[S_TOL2] * s[S_BB]) s[S_ACTIVE] = 0.0;
        }
    }
    s[S_BETA] = beta;
}
__global__ void k_scal_beta(const double *__restrict__ part, double *__restrict__ scal, int nb) {
    for (int b = threadIdx.x; b < nb; b += blockDim.x) scal_beta_one(part, scal, b);
}

template <typename C>
__device__ __forceinline__ void pupdate_rows(C *__restrict__ p, const C *__restrict__ z, int nc, int64_t nalm,
                                             const double *__restrict__ scal, const int b, const int bx,
                                             const int nbx) {
    const int64_t off = (int64_t)b * nc * nalm;
    const double beta = scal[b * 16 + S_BETA];
    const int64_t n = (int64_t)nc * nalm;
    for (int64_t i = bx * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)nbx * blockDim.x) {
        C pv = p[off + i];
        const C zv = z[off + i];
        pv.x = zv.x + (decltype(pv.x))beta * pv.x;
        pv.y = zv.y + (decltype(pv.y))beta * pv.y;
        p[off + i] = pv;
    }
}
template <typename C>
__global__ void k_pupdate(C *__restrict__ p, const C *__restrict__ z, int nc, int64_t nalm,
                          const double *__restrict__ scal) {
    pupdate_rows<C>(p, z, nc, nalm, scal, blockIdx.y, blockIdx.x, gridDim.x);
}

// ----------------------------------------------- grouped FP32 PCG kernels
// The vector kernels of the FP32 iteration over several plans in one
// launch (chains of several geometries): flat realization row = blockIdx.y
// (row kernels) or group = blockIdx.x (scalar kernels); each group's
// vectors, tables and scalars are its own plan's.
struct VecGrp {
    float2 *x, *r, *z, *p, *q;
    const float *minv, *sinv, *isc;
    const int *lof, *mof;
    double *scal, *part;
    const int *active;   // device flag: 0 = the group is skipped
    int64_t nalm;
    int nc, nb, lmax1;
};
struct VecGroups {
    int ng;
    int firstb[SHTG_MAX_GROUPS + 1];   // first flat realization row of each group
    VecGrp v[SHTG_MAX_GROUPS];
};

__device__ __forceinline__ int vgroup(const VecGroups &G, const int row) {
    int g = 0;
    while (g + 1 < G.ng && row >= G.firstb[g + 1]) ++g;
    return g;
}

__global__ void k_prior_add_grp(const __grid_constant__ VecGroups G) {
    const int g = vgroup(G, blockIdx.y);
    const VecGrp &v = G.v[g];
    if (*v.active == 0) return;
    prior_add_rows<float, true>(v.p, v.q, v.nc, v.nalm, v.lmax1, v.lof, v.sinv, v.isc, v.mof, v.part,
                                blockIdx.y - G.firstb[g], blockIdx.x, gridDim.x);
}
__global__ void k_scal_alpha_grp(const __grid_constant__ VecGroups G, double floor2) {
    const VecGrp &v = G.v[blockIdx.x];
    if (*v.active == 0) return;
    for (int b = threadIdx.x; b < v.nb; b += blockDim.x) scal_alpha_one(v.part, v.scal, b, floor2);
}
__global__ void k_update_grp(const __grid_constant__ VecGroups G) {
    const int g = vgroup(G, blockIdx.y);
    const VecGrp &v = G.v[g];
    if (*v.active == 0) return;
    update_rows<float, false>(v.x, v.r, v.z, v.p, v.q, v.minv, v.nc, v.nalm, v.mof, v.scal, v.part,
                              blockIdx.y - G.firstb[g], blockIdx.x, gridDim.x);
}
__global__ void k_scal_beta_grp(const __grid_constant__ VecGroups G) {
    const VecGrp &v = G.v[blockIdx.x];
    if (*v.active == 0) return;
    for (int b = threadIdx.x; b < v.nb; b += blockDim.x) scal_beta_one(v.part, v.scal, b);
}
__global__ void k_pupdate_grp(const __grid_constant__ VecGroups G) {
    const int g = vgroup(G, blockIdx.y);
    const VecGrp &v = G.v[g];
    if (*v.active == 0) return;
    pupdate_rows<float2>(v.p, v.z, v.nc, v.nalm, v.scal, blockIdx.y - G.firstb[g], blockIdx.x, gridDim.x);
}

// mixed precision helpers
__global__ void k_resid(const double2 *__restrict__ b, const double2 *__restrict__ t,
                        double2 *__restrict__ r, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double2 bv = b[i], tv = t[i];
        r[i] = make_double2(bv.x - tv.x, bv.y - tv.y);
    }
}
// r32 = r64 / scale_b (0 for realizations already converged)
__global__ void k_scale_down(const double2 *__restrict__ r, float2 *__restrict__ r32, int64_t per,
                             const double *__restrict__ inv_scale) {
    const int b = blockIdx.y;
    const double s = inv_scale[b];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < per;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double2 v = r[(int64_t)b * per + i];
        r32[(int64_t)b * per + i] = make_float2((float)(v.x * s), (float)(v.y * s));
    }
}
// x64 += scale_b * d32
__global__ void k_correct(double2 *__restrict__ x, const float2 *__restrict__ d, int64_t per,
                          const double *__restrict__ scale) {
    const int b = blockIdx.y;
    const double s = scale[b];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < per;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float2 v = d[(int64_t)b * per + i];
        double2 xv = x[(int64_t)b * per + i];
        xv.x += s * (double)v.x;
        xv.y += s * (double)v.y;
        x[(int64_t)b * per + i] = xv;
    }
}

// v *= f_b per realization (FP32 search direction after a residual replacement)
__global__ void k_scale_vec(float2 *__restrict__ v, int64_t per, const double *__restrict__ f) {
    const int b = blockIdx.y;
    const float s = (float)f[b];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < per;
         i += (int64_t)gridDim.x * blockDim.x) {
        float2 x = v[(int64_t)b * per + i];
        x.x *= s;
        x.y *= s;
        v[(int64_t)b * per + i] = x;
    }
}

// after a residual replacement: new rz, rr from the partials; tol2 per realization
__global__ void k_scal_reliable(const double *__restrict__ part, double *__restrict__ scal, int nb,
                                const double *__restrict__ tol2) {
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
        double *s = scal + b * 16;
        const double rz = sum_part(part, b, 2, 0), rr = sum_part(part, b, 2, 1);
        s[S_RZ] = rz;
        s[S_RR] = rr;
        s[S_BB] = 1.0;                       // the FP32 residual is normalized to 1
        s[S_TOL2] = tol2[b];
        s[S_ACTIVE] = (tol2[b] >= 0.0 && rr > 0.0) ? 1.0 : 0.0;
        // set, not accumulated: the first replacement of a solve runs on scalar
        // slots that hold whatever an earlier call (or a fresh allocation) left,
        // and a bad FP32 stage already ended the solve at its host check
        s[S_BAD] = (isfinite(rr) && isfinite(rz)) ? 0.0 : 1.0;
        s[S_ITERS] = 0.0;
        s[S_RESTART] = 0.0;
        s[S_ALPHA] = s[S_BETA] = 0.0;
    }
}

// a stage that ended at its rounding floor restarts its direction: p = z
__global__ void k_restart_dir(float2 *__restrict__ p, const float2 *__restrict__ z, int64_t per,
                              const double *__restrict__ scal) {
    const int b = blockIdx.y;
    if (scal[b * 16 + S_RESTART] == 0.0) return;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < per; i += (int64_t)gridDim.x * blockDim.x)
        p[(int64_t)b * per + i] = z[(int64_t)b * per + i];
}

// ------------------------------------------------------------ log-posterior
// per-l sums of the prior term: lsum[l] += w_m |a_lm|^2 / C_l (active l)
__global__ void k_prior_lsum(const float2 *__restrict__ a, int64_t nalm, const int *__restrict__ lof,
                             const int *__restrict__ mof, const float *__restrict__ icl,
                             double *__restrict__ lsum) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nalm;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int l = lof[i];
        const float c = icl[l];
        if (c == 0.f) continue;
        const double w = mof[i] ? 2.0 : 1.0;
        const float2 v = a[i];
        atomicAdd(&lsum[l], w * ((double)v.x * v.x + (double)v.y * v.y) * (double)c);
    }
}
// res = d - m (in place in m); chi2 partial = sum ninv res^2; m <- ninv res
__global__ void k_resid_pix(const float *__restrict__ d, const float *__restrict__ ninv,
                            float *__restrict__ m, int64_t npix, double *__restrict__ part) {
    __shared__ double sm[RT / 32];
    double s = 0.0;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < npix;
         p += (int64_t)gridDim.x * blockDim.x) {
        const float r = d[p] - m[p];
        const float w = ninv[p];
        s += (double)w * (double)r * (double)r;
        m[p] = w * r;
    }
    s = block_sum(s, sm);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}
// grad -= a / C_l (active l), zero at held multipoles
__global__ void k_grad_prior(const float2 *__restrict__ a, float2 *__restrict__ g, int64_t nalm,
                             const int *__restrict__ lof, const int *__restrict__ mof,
                             const float *__restrict__ icl, int components) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nalm;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float c = icl[lof[i]];
        float2 v = g[i];
        const float2 av = a[i];
        if (c == 0.f) {
            v = make_float2(0.f, 0.f);
        } else {
            v.x -= c * av.x;
            v.y -= c * av.y;
        }
        if (mof[i] == 0) {
            v.y = 0.f;
        } else if (components) {
            v.x *= 2.f;
            v.y *= 2.f;
        }
        g[i] = v;
    }
}

// ------------------------------------------------------------- joint move
// Joint (C_l, a) move of Sect. 2.2.2.
//
// Rescaling matrix of the fluctuation term per l: R_l = (C'_l)^{1/2}
// (C_l)^{-1/2} with the symmetric principal square roots of the T/E block
// (closed form for 2 x 2: sqrt(M) = (M + sqrt(det) I) / sqrt(tr + 2 sqrt(det)),
// whose determinant is sqrt(det), so its inverse is adj(M + sqrt(det) I) /
// (sqrt(tr + 2 sqrt(det)) sqrt(det))) and the scalar B part; R_l = 0 where
// either block is singular (those multipoles are held at zero).  cl rows:
// [TT, EE, BB, TE] x L1 for old then new (nc = 1: TT rows only).
// out rows: R_TT, R_TE, R_ET, R_EE, R_BB.
__global__ void k_rescale_table(const double *__restrict__ cold, const double *__restrict__ cnew, int nc,
                                int L1, double *__restrict__ out) {
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= L1) return;
    double r[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    if (nc == 1) {
        const double a = cold[l], b = cnew[l];
        if (a > 0.0 && b > 0.0) r[0] = sqrt(b / a);
    } else {
        const double at = cold[l], ae = cold[L1 + l], ab = cold[2 * L1 + l], ax = cold[3 * L1 + l];
        const double bt = cnew[l], be = cnew[L1 + l], bb = cnew[2 * L1 + l], bx = cnew[3 * L1 + l];
        const double dold = at * ae - ax * ax, dnew = bt * be - bx * bx;
        if (at > 0.0 && dold > 0.0 && ab > 0.0 && bt > 0.0 && dnew > 0.0 && bb > 0.0) {
            const double so = sqrt(dold), to = sqrt(at + ae + 2.0 * so);
            const double sn = sqrt(dnew), tn = sqrt(bt + be + 2.0 * sn);
            // (C')^{1/2} = [[bt + sn, bx], [bx, be + sn]] / tn
            const double p11 = (bt + sn) / tn, p12 = bx / tn, p22 = (be + sn) / tn;
            // C^{-1/2} = [[ae + so, -ax], [-ax, at + so]] / (to so)
            const double q = 1.0 / (to * so);
            const double q11 = (ae + so) * q, q12 = -ax * q, q22 = (at + so) * q;
            r[0] = p11 * q11 + p12 * q12;
            r[1] = p11 * q12 + p12 * q22;
            r[2] = p12 * q11 + p22 * q12;
            r[3] = p12 * q12 + p22 * q22;
            r[4] = sqrt(bb / ab);
        }
    }
    for (int k = 0; k < 5; ++k) out[k * L1 + l] = r[k];
}

// g = R_l f per alm index (T, E, B of one realization; imaginary part of
// m = 0 written as 0)
__global__ void k_rescale(const double2 *__restrict__ f, double2 *__restrict__ g, int nc, int64_t nalm,
                          const int *__restrict__ lof, const int *__restrict__ mof,
                          const double *__restrict__ R, int L1) {
    const int64_t off = (int64_t)blockIdx.y * nc * nalm;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nalm;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int l = lof[i];
        const bool m0 = mof[i] == 0;
        if (nc == 1) {
            double2 v = f[off + i];
            v.x *= R[l];
            v.y = m0 ? 0.0 : v.y * R[l];
            g[off + i] = v;
        } else {
            const double2 t = f[off + i], e = f[off + nalm + i], b = f[off + 2 * nalm + i];
            const double r11 = R[l], r12 = R[L1 + l], r21 = R[2 * L1 + l], r22 = R[3 * L1 + l];
            const double rb = R[4 * L1 + l];
            double2 vt = {r11 * t.x + r12 * e.x, r11 * t.y + r12 * e.y};
            double2 ve = {r21 * t.x + r22 * e.x, r21 * t.y + r22 * e.y};
            double2 vb = {rb * b.x, rb * b.y};
            if (m0) vt.y = ve.y = vb.y = 0.0;
            g[off + i] = vt;
            g[off + nalm + i] = ve;
            g[off + 2 * nalm + i] = vb;
        }
    }
}

// Pixel sums of the log target per realization (grid RB x nb): mode 0:
// sum_c sum_p N^-1_c,p (d - m)^2; mode 1: sum_c sum_p N^-1_c,p m^2.  d is in
// [b][c][npix] order, m in the transform's row order (T rows, then Q, U
// pairs), N^-1 [T, P] with Q and U sharing P.
__global__ void k_joint_pix(const double *__restrict__ d, const double *__restrict__ m,
                            const double *__restrict__ ninv, int nb, int nc, int64_t npix, int mode,
                            double *__restrict__ part) {
    __shared__ double sm[RT / 32];
    const int b = blockIdx.y;
    double acc = 0.0;
    for (int c = 0; c < nc; ++c) {
        const int row = (c == 0) ? b : nb + 2 * b + (c - 1);
        const double *mv = m + (int64_t)row * npix;
        const double *dv = d ? d + ((int64_t)b * nc + c) * npix : nullptr;
        const double *wv = ninv + (c == 0 ? 0 : npix);
        for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < npix;
             p += (int64_t)gridDim.x * blockDim.x) {
            const double v = mode == 0 ? dv[p] - mv[p] : mv[p];
            acc += wv[p] * v * v;
        }
    }
    acc = block_sum(acc, sm);
    if (threadIdx.x == 0) part[b * RB + blockIdx.x] = acc;
}

// Prior term per realization (grid RB x nb): sum over active multipoles of
// w_m Re(conj(a) S^-1 a) (w_0 = 1, w_m = 2), S^-1 the per-l block scaled by
// the realization's 1 / (C_l scale); sinv rows TT, TE, EE, BB; a multipole
// is active where the inverse square root's TT entry sh is positive.
__global__ void k_prior_quad(const double2 *__restrict__ a, int nc, int64_t nalm, int L1,
                             const int *__restrict__ lof, const int *__restrict__ mof,
                             const double *__restrict__ sinv, const double *__restrict__ sh,
                             const double *__restrict__ isc, double *__restrict__ part) {
    __shared__ double sm[RT / 32];
    const int b = blockIdx.y;
    const double2 *ab = a + (int64_t)b * nc * nalm;
    double acc = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nalm;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int l = lof[i];
        if (!(sh[l] > 0.0)) continue;
        const bool m0 = mof[i] == 0;
        const double w = m0 ? 1.0 : 2.0;
        double2 t = ab[i];
        if (m0) t.y = 0.0;
        double q;
        if (nc == 1) {
            q = sinv[l] * (t.x * t.x + t.y * t.y);
        } else {
            double2 e = ab[nalm + i], bb = ab[2 * nalm + i];
            if (m0) e.y = bb.y = 0.0;
            q = sinv[l] * (t.x * t.x + t.y * t.y) + 2.0 * sinv[L1 + l] * (t.x * e.x + t.y * e.y) +
                sinv[2 * L1 + l] * (e.x * e.x + e.y * e.y) + sinv[3 * L1 + l] * (bb.x * bb.x + bb.y * bb.y);
        }
        acc += w * q;
    }
    acc = block_sum(acc, sm) * isc[b];
    if (threadIdx.x == 0) part[b * RB + blockIdx.x] = acc;
}

// ====================================================================== host
// One PCG iteration (operator application + vector updates) captured as a
// CUDA graph and replayed between the host's convergence checks: the
// iteration's pointers and per-realization scalars live on the device, so
// every iteration launches the same work.
struct IterGraph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    long long launches = 0;   // library launches in one replay
    void release() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        exec = nullptr;
        graph = nullptr;
    }
    ~IterGraph() { release(); }
};

struct Solve {
    Plan *p;
    cudaStream_t st;
    int nb, nc;
    int tc = 0;      // FP32 operator: Legendre sums on the tensor cores
    int df = 0;      // FP64 operator: Legendre sums in double-FP32 arithmetic
    int graphs = 1;  // replay captured iterations (off while profiling)
    int pc = SHTG_PRECOND_DIAG;   // preconditioner: the low block (LOWL) or the azimuthal blocks (AZIM)
                                  // replace z on their rows after every update of the diagonal one
    int64_t nalm, per, nvec;
    dim3 vgrid;   // (blocks, nb)
    dim3 rgrid;   // (RB, nb)
};

static dim3 grid_1d(int64_t n) {
    int64_t g = (n + RT - 1) / RT;
    if (g > 4096) g = 4096;
    if (g < 1) g = 1;
    return dim3((unsigned)g);
}

template <typename T> struct Vec;
template <> struct Vec<double> {
    static double2 *r(Plan *p) { return p->v64[2]; }
    static double2 *z(Plan *p) { return p->v64[3]; }
    static double2 *pp(Plan *p) { return p->v64[4]; }
    static double2 *q(Plan *p) { return p->v64[5]; }
    static double *minv(Plan *p) { return p->d_minv64; }
    static double *beam(Plan *p) { return p->d_ltab64; }
    static double *sinv(Plan *p) { return p->d_ltab64 + (p->lmax + 1); }
    static double *isc(Plan *p) { return p->d_isc64; }
    static double *ninv(Plan *p) { return p->d_ninv64; }
    static double2 *phase(Plan *p) { return p->d_phase64; }
};
template <> struct Vec<float> {
    static float2 *r(Plan *p) { return p->v32[0]; }
    static float2 *z(Plan *p) { return p->v32[1]; }
    static float2 *pp(Plan *p) { return p->v32[2]; }
    static float2 *q(Plan *p) { return p->v32[3]; }
    static float *minv(Plan *p) { return p->d_minv32; }
    static float *beam(Plan *p) { return p->d_ltab32; }
    static float *sinv(Plan *p) { return p->d_ltab32 + (p->lmax + 1); }
    static float *isc(Plan *p) { return p->d_isc32; }
    static float *ninv(Plan *p) { return p->d_ninv32; }
    static float2 *phase(Plan *p) { return p->d_phase32; }
};

// Legendre synthesis of the operator: FP64 (s.df: double-FP32), FP32 or
// (s.tc) tensor-core FP32
static int op_synth(Solve &s, int spin, const double2 *x, int rs, const double *beam, double2 *F) {
    if (s.df) return leg_synth_df(s.p, spin, x, rs, s.nb, beam, F, s.st);
    return leg_synth<double>(s.p, spin, x, rs, s.nb, beam, F, s.st);
}
static int op_synth(Solve &s, int spin, const float2 *x, int rs, const float *beam, float2 *F) {
    if (s.tc) return leg_synth_tc(s.p, spin, x, rs, s.nb, beam, F, s.st);
    return leg_synth<float>(s.p, spin, x, rs, s.nb, beam, F, s.st);
}

// Legendre transpose of the operator: FP64 (s.df: double-FP32), FP32 or
// (s.tc) tensor-core FP32
static int op_analysis(Solve &s, int spin, const double2 *G, const double *beam, double2 *y, int rs) {
    if (s.df) return leg_analysis_df(s.p, spin, G, s.nb, beam, y, rs, s.st, 0);
    return leg_analysis<double>(s.p, spin, G, s.nb, beam, y, rs, s.st);
}
static int op_analysis(Solve &s, int spin, const float2 *G, const float *beam, float2 *y, int rs) {
    if (s.tc) return leg_analysis_tc(s.p, spin, G, s.nb, beam, y, rs, s.st, 0);
    return leg_analysis<float>(s.p, spin, G, s.nb, beam, y, rs, s.st);
}

// y = A x = S^-1 x + B Y^T N^-1 Y B x for all realizations
template <typename T>
static int matvec(Solve &s, const typename HT<T>::C *x, typename HT<T>::C *y, bool dot = false) {
    typedef typename HT<T>::C C;
    Plan *p = s.p;
    C *F = Vec<T>::phase(p);
    const T *beam = Vec<T>::beam(p);
    const int64_t rowsz = (int64_t)(p->lmax + 1) * p->nring;
    SHTG_TRY(op_synth(s, 0, x, s.nc, beam, F));
    if (s.nc == 3) SHTG_TRY(op_synth(s, 2, x + s.nalm, 3, beam, F + s.nb * rowsz));
    SHTG_TRY(ring_fused<T>(p, F, s.nb * s.nc, s.nb, Vec<T>::ninv(p), s.st));
    SHTG_TRY(op_analysis(s, 0, F, beam, y, s.nc));
    if (s.nc == 3) SHTG_TRY(op_analysis(s, 2, F + s.nb * rowsz, beam, y + s.nalm, 3));
    prof_begin(p, K_VEC, s.st);
    if (dot)   // y's final values and <x, y> partials (slot 0) in one pass
        k_prior_add<T, true><<<s.rgrid, RT, 0, s.st>>>(x, y, s.nc, s.nalm, p->lmax + 1, p->d_lofidx,
                                                       Vec<T>::sinv(p), Vec<T>::isc(p), p->d_mofidx, p->d_part);
    else
        k_prior_add<T, false><<<dim3(grid_1d(s.nalm).x, s.nb), RT, 0, s.st>>>(
            x, y, s.nc, s.nalm, p->lmax + 1, p->d_lofidx, Vec<T>::sinv(p), Vec<T>::isc(p), nullptr, nullptr);
    prof_end(p, s.st);
    SHTG_CHECK_LAUNCH("k_prior_add");
    return SHTG_OK;
}

// The preconditioner beyond the diagonal: z on the rows of the low block or
// of the azimuthal blocks, and the change of <r, z> in the rz partials.
template <typename T>
static int precond_fix(Solve &s, const typename HT<T>::C *r, typename HT<T>::C *z) {
    if (s.pc == SHTG_PRECOND_LOWL)
        return lowl_apply<T>(s.p, reinterpret_cast<const T *>(r), reinterpret_cast<T *>(z), s.nb, s.per,
                             s.p->d_part, s.st);
    if (s.pc == SHTG_PRECOND_AZIM)
        return az_apply<T>(s.p, reinterpret_cast<const T *>(r), reinterpret_cast<T *>(z), s.nb, s.per,
                           s.p->d_part, s.st, false);
    return SHTG_OK;
}

// One PCG iteration on the device: q = A p, alpha, x/r/z update, beta, p.
template <typename T>
static int pcg_iteration(Solve &s, typename HT<T>::C *x, typename HT<T>::C *r, typename HT<T>::C *z,
                         typename HT<T>::C *pv, typename HT<T>::C *q, const T *minv) {
    typedef typename HT<T>::C C;
    Plan *p = s.p;
    SHTG_TRY(matvec<T>(s, pv, q, true));   // q = A p and the partials of <p, q>
    prof_begin(p, K_VEC, s.st);
    // FP32 recursion: below 1e-3 of the stage's start a breakdown ends the stage
    k_scal_alpha<<<1, 1024, 0, s.st>>>(p->d_part, p->d_scal, s.nb, sizeof(T) == 4 ? 1e-6 : 0.0);
    k_update<T, false><<<s.rgrid, RT, 0, s.st>>>(x, r, z, pv, q, minv, s.nc, s.nalm, p->d_mofidx,
                                                 p->d_scal, p->d_part);
    SHTG_TRY(precond_fix<T>(s, r, z));
    k_scal_beta<<<1, 1024, 0, s.st>>>(p->d_part, p->d_scal, s.nb);
    k_pupdate<C><<<dim3(grid_1d(s.per).x, s.nb), RT, 0, s.st>>>(pv, z, s.nc, s.nalm, p->d_scal);
    prof_end(p, s.st, 4);
    SHTG_CHECK_LAUNCH("pcg iteration");
    return SHTG_OK;
}

// nrun iterations.  With graphs on (and profiling off) the first call runs
// one iteration eagerly (any autotuning happens there), captures the next
// one into g and replays it for the rest; later calls only replay.
template <typename T>
static int run_iterations(Solve &s, IterGraph &g, int nrun, typename HT<T>::C *x, typename HT<T>::C *r,
                          typename HT<T>::C *z, typename HT<T>::C *pv, typename HT<T>::C *q,
                          const T *minv) {
    Plan *p = s.p;
    if (!s.graphs || p->prof.on) {
        for (int k = 0; k < nrun; ++k) SHTG_TRY(pcg_iteration<T>(s, x, r, z, pv, q, minv));
        return SHTG_OK;
    }
    if (!g.exec && nrun > 0) {
        SHTG_TRY(pcg_iteration<T>(s, x, r, z, pv, q, minv));
        --nrun;
        if (nrun == 0) return SHTG_OK;
        // capture on the plan's own stream (the caller's may be the legacy
        // default stream, which cannot be captured); capturing runs nothing,
        // and the replays go to the caller's stream
        const long long l0 = p->prof.launches;
        const cudaStream_t caller = s.st;
        s.st = p->cap_stream;
        SHTG_CUDA(cudaStreamBeginCapture(s.st, cudaStreamCaptureModeRelaxed));
        const int rc = pcg_iteration<T>(s, x, r, z, pv, q, minv);
        cudaGraph_t graph = nullptr;
        const cudaError_t e = cudaStreamEndCapture(s.st, &graph);
        s.st = caller;
        g.launches = p->prof.launches - l0;
        p->prof.launches = l0;
        if (rc != SHTG_OK) {
            if (graph) cudaGraphDestroy(graph);
            return rc;
        }
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture", __FILE__, __LINE__);
        g.graph = graph;
        SHTG_CUDA(cudaGraphInstantiate(&g.exec, graph, 0));
    }
    for (int k = 0; k < nrun; ++k) {
        SHTG_CUDA(cudaGraphLaunch(g.exec, s.st));
        p->prof.launches += g.launches;
    }
    return SHTG_OK;
}

// PCG on A x = b for T vectors; x starts at 0.  Per-realization convergence
// at ||r|| <= tol ||b||.  Returns the number of iterations run.
template <typename T>
static int pcg(Solve &s, const typename HT<T>::C *b, typename HT<T>::C *x, double tol, int maxiter,
               int check_every, int *iters, int *all_converged) {
    typedef typename HT<T>::C C;
    Plan *p = s.p;
    C *r = Vec<T>::r(p), *z = Vec<T>::z(p), *pv = Vec<T>::pp(p), *q = Vec<T>::q(p);
    const T *minv = Vec<T>::minv(p);
    const size_t vb = sizeof(C) * (size_t)s.nvec;
    IterGraph graph;
    SHTG_CUDA(cudaMemsetAsync(x, 0, vb, s.st));
    SHTG_CUDA(cudaMemcpyAsync(r, b, vb, cudaMemcpyDeviceToDevice, s.st));
    k_update<T, true><<<s.rgrid, RT, 0, s.st>>>(nullptr, r, z, nullptr, nullptr, minv, s.nc, s.nalm,
                                                p->d_mofidx, p->d_scal, p->d_part);
    SHTG_CHECK_LAUNCH("k_update init");
    SHTG_TRY(precond_fix<T>(s, r, z));
    k_scal_init<<<1, 1024, 0, s.st>>>(p->d_part, p->d_scal, s.nb, tol * tol);
    p->prof.launches += 2;
    SHTG_CHECK_LAUNCH("k_scal_init");
    SHTG_CUDA(cudaMemcpyAsync(pv, z, vb, cudaMemcpyDeviceToDevice, s.st));
    int it = 0;
    *all_converged = 0;
    if (check_every < 1) check_every = 1;
    while (it < maxiter) {
        // host check first: every realization may already be done (b = 0)
        SHTG_CUDA(cudaMemcpyAsync(p->h_pinned, p->d_scal, sizeof(double) * 16 * s.nb,
                                  cudaMemcpyDeviceToHost, s.st));
        SHTG_CUDA(cudaStreamSynchronize(s.st));
        int active = 0, bad = 0;
        for (int k = 0; k < s.nb; ++k) {
            active += p->h_pinned[k * 16 + S_ACTIVE] != 0.0;
            bad += p->h_pinned[k * 16 + S_BAD] != 0.0;
        }
        if (bad) {
            set_error("non-finite or non-positive curvature in PCG");
            *iters = it;
            return SHTG_ERR_NONFINITE;
        }
        if (!active) {
            *all_converged = 1;
            break;
        }
        const int nrun = std::min(check_every, maxiter - it);
        SHTG_TRY(run_iterations<T>(s, graph, nrun, x, r, z, pv, q, minv));
        it += nrun;
    }
    if (!*all_converged) {
        SHTG_CUDA(cudaMemcpyAsync(p->h_pinned, p->d_scal, sizeof(double) * 16 * s.nb,
                                  cudaMemcpyDeviceToHost, s.st));
        SHTG_CUDA(cudaStreamSynchronize(s.st));
        int active = 0;
        for (int k = 0; k < s.nb; ++k) active += p->h_pinned[k * 16 + S_ACTIVE] != 0.0;
        *all_converged = active == 0;
    }
    int mx = 0;
    for (int k = 0; k < s.nb; ++k) mx = std::max(mx, (int)p->h_pinned[k * 16 + S_ITERS]);
    *iters = it;
    (void)mx;
    return SHTG_OK;
}

// per-realization <v, v> into host array
static int norms2(Solve &s, const double2 *v, std::vector<double> &out) {
    Plan *p = s.p;
    k_dot<double2><<<s.rgrid, RT, 0, s.st>>>(v, v, s.nc, s.nalm, p->d_mofidx, p->d_part, 0, 1);
    p->prof.launches += 1;
    SHTG_CHECK_LAUNCH("k_dot");
    std::vector<double> h((size_t)s.nb * RB);
    SHTG_CUDA(cudaMemcpyAsync(h.data(), p->d_part, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, s.st));
    SHTG_CUDA(cudaStreamSynchronize(s.st));
    out.assign(s.nb, 0.0);
    for (int b = 0; b < s.nb; ++b)
        for (int k = 0; k < RB; ++k) out[b] += h[(size_t)b * RB + k];
    return SHTG_OK;
}

static double now_ms() {
    return std::chrono::duration<double, std::milli>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

// Per-l tables from host C_l and b_l, copied on the solve's stream (the
// kernels that read them run there; a copy on the legacy default stream is
// not ordered with a non-blocking stream).  Returns SHTG_ERR_NOT_SPD for an
// indefinite block.
static int build_ltab(Plan *p, int nc, const double *cl, const double *bl, cudaStream_t st) {
    const int L1 = p->lmax + 1;
    std::vector<double> t64(9 * (size_t)L1, 0.0);
    std::vector<float> t32(5 * (size_t)L1, 0.f);
    for (int l = 0; l < L1; ++l) {
        double tt, te = 0, ee = 1, bb = 1;
        bool active;
        double s[4] = {1, 0, 1, 1}, h[4] = {0, 0, 0, 0};
        if (nc == 1) {
            tt = cl[l];
            if (!(tt >= 0.0)) {
                set_error("C_l < 0 at l = " + std::to_string(l));
                return SHTG_ERR_NOT_SPD;
            }
            active = tt > 0.0;
            if (active) {
                s[0] = 1.0 / tt;
                h[0] = 1.0 / sqrt(tt);
            }
        } else {
            tt = cl[l];
            ee = cl[L1 + l];
            bb = cl[2 * L1 + l];
            te = cl[3 * L1 + l];
            const double det = tt * ee - te * te;
            if (!(tt >= 0 && ee >= 0 && bb >= 0 && det >= -1e-300)) {
                set_error("C_l block not positive semi-definite at l = " + std::to_string(l));
                return SHTG_ERR_NOT_SPD;
            }
            active = tt > 0 && bb > 0 && det > 0;
            if (active) {
                s[0] = ee / det;
                s[1] = -te / det;
                s[2] = tt / det;
                s[3] = 1.0 / bb;
                // inverse of the symmetric square root of [[tt, te], [te, ee]]:
                // sqrt(M) = (M + sqrt(det) I) / sqrt(tr + 2 sqrt(det))
                const double sd = sqrt(det), tq = sqrt(tt + ee + 2.0 * sd);
                const double r11 = (tt + sd) / tq, r12 = te / tq, r22 = (ee + sd) / tq;
                const double rd = r11 * r22 - r12 * r12;
                h[0] = r22 / rd;
                h[1] = -r12 / rd;
                h[2] = r11 / rd;
                h[3] = 1.0 / sqrt(bb);
            }
        }
        const double beam = active ? bl[l] : 0.0;
        t64[l] = beam;
        for (int k = 0; k < 4; ++k) {
            t64[(1 + k) * (size_t)L1 + l] = s[k];
            t64[(5 + k) * (size_t)L1 + l] = h[k];
            t32[(1 + k) * (size_t)L1 + l] = (float)s[k];
        }
        t32[l] = (float)beam;
    }
    SHTG_CUDA(cudaMemcpyAsync(p->d_ltab64, t64.data(), sizeof(double) * t64.size(), cudaMemcpyHostToDevice, st));
    SHTG_CUDA(cudaMemcpyAsync(p->d_ltab32, t32.data(), sizeof(float) * t32.size(), cudaMemcpyHostToDevice, st));
    SHTG_CUDA(cudaStreamSynchronize(st));   // the host tables go out of scope
    return SHTG_OK;
}

// Copy N^-1 into the plan (FP64 + FP32 copies), build the preconditioner.
// nsys systems: system k belongs to realization k mod prob->nbatch (the
// split right-hand sides of a realization share its C_l scale).
static int setup_operator(Plan *p, const shtg_problem *pr, int host_inputs, int precond,
                          cudaStream_t st, int nsys = 0) {
    const int nc = pr->ncomp;
    if (nsys <= 0) nsys = pr->nbatch;
    SHTG_TRY(build_ltab(p, nc, pr->cl, pr->bl, st));
    {
        // realization b's C_l is cl_scale[b] x cl: S^-1 scales by 1/s, S^-1/2 by 1/sqrt(s)
        std::vector<double> i64(nsys), r64(nsys);
        std::vector<float> i32(nsys);
        for (int k = 0; k < nsys; ++k) {
            const int b = k % pr->nbatch;
            const double sc = pr->cl_scale ? pr->cl_scale[b] : 1.0;
            i64[k] = 1.0 / sc;
            r64[k] = 1.0 / sqrt(sc);
            i32[k] = (float)i64[k];
        }
        SHTG_CUDA(cudaMemcpyAsync(p->d_isc64, i64.data(), sizeof(double) * nsys, cudaMemcpyHostToDevice, st));
        SHTG_CUDA(cudaMemcpyAsync(p->d_rsc64, r64.data(), sizeof(double) * nsys, cudaMemcpyHostToDevice, st));
        SHTG_CUDA(cudaMemcpyAsync(p->d_isc32, i32.data(), sizeof(float) * nsys, cudaMemcpyHostToDevice, st));
        SHTG_CUDA(cudaStreamSynchronize(st));   // the host vectors go out of scope
    }
    const int ncomp_ninv = nc == 3 ? 2 : 1;
    const size_t nb = sizeof(double) * (size_t)p->npix * ncomp_ninv;
    SHTG_CUDA(cudaMemcpyAsync(p->d_ninv64, pr->ninv, nb,
                              host_inputs ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, st));
    k_to_float<<<grid_1d(p->npix * ncomp_ninv), RT, 0, st>>>(p->d_ninv64, p->d_ninv32,
                                                           p->npix * ncomp_ninv);
    p->prof.launches += 1;
    SHTG_CHECK_LAUNCH("k_to_float");
    if (precond) {
        k_wpair<<<p->npairs, RT, 0, st>>>(p->d_ninv64, p->d_ofs, p->d_nphi, p->nring, p->d_wpairT);
        p->prof.launches += 1;
        SHTG_CHECK_LAUNCH("k_wpair");
        SHTG_TRY(leg_diag(p, 0, p->d_wpairT, p->d_diagT, st));
        if (nc == 3) {
            k_wpair<<<p->npairs, RT, 0, st>>>(p->d_ninv64 + p->npix, p->d_ofs, p->d_nphi, p->nring,
                                              p->d_wpairP);
            p->prof.launches += 1;
            SHTG_CHECK_LAUNCH("k_wpair");
            SHTG_TRY(leg_diag(p, 2, p->d_wpairP, p->d_diagP, st));
        }
    }
    k_precond<<<dim3(grid_1d(p->nalm).x, nsys), RT, 0, st>>>(
        p->d_diagT, nc == 3 ? p->d_diagP : p->d_diagT, p->d_ltab64, nc, p->nalm, p->lmax + 1, p->d_lofidx,
        precond, p->d_isc64, p->d_minv64, p->d_minv32);
    p->prof.launches += 1;
    SHTG_CHECK_LAUNCH("k_precond");
    return SHTG_OK;
}

static int check_problem(Plan *p, const shtg_problem *pr) {
    if (!pr || !pr->cl || !pr->bl || !pr->ninv) {
        set_error("problem, cl, bl and ninv are required");
        return SHTG_ERR_ARG;
    }
    if (pr->ncomp != 1 && pr->ncomp != 3) {
        set_error("ncomp must be 1 or 3");
        return SHTG_ERR_ARG;
    }
    if (pr->ncomp == 3 && !(p->flags & SHTG_SPIN2)) {
        set_error("ncomp = 3 needs a plan created with SHTG_SPIN2");
        return SHTG_ERR_ARG;
    }
    if (pr->nbatch < 1 || pr->nbatch > p->max_batch) {
        set_error("nbatch must be in [1, max_batch]");
        return SHTG_ERR_ARG;
    }
    if (pr->cl_scale)
        for (int b = 0; b < pr->nbatch; ++b)
            if (!(pr->cl_scale[b] > 0.0) || !std::isfinite(pr->cl_scale[b])) {
                set_error("cl_scale entries must be positive and finite");
                return SHTG_ERR_ARG;
            }
    return SHTG_OK;
}

static Solve make_solve(Plan *p, int nb, int nc, cudaStream_t st) {
    Solve s;
    s.p = p;
    s.st = st;
    s.nb = nb;
    s.nc = nc;
    s.nalm = p->nalm;
    s.per = (int64_t)nc * p->nalm;
    s.nvec = (int64_t)nb * s.per;
    s.vgrid = dim3(grid_1d(s.per).x, nb);
    s.rgrid = dim3(RB, nb);
    return s;
}

// FP32 PCG with reliable updates (residual replacement).  The iteration runs
// on FP32 vectors normalized per realization; x accumulates in FP64.  When a
// realization's FP32 residual has dropped by the factor delta (or reached the
// target), the FP64 residual r = b - A x is recomputed with the FP64
// transforms and replaces the FP32 one; the search direction is kept
// (rescaled), so the Krylov progress survives the update.  Converged
// realizations are frozen.  On return rr holds the final FP64 ||r||^2.
static int mixed_solve(Solve &s, const shtg_cg_opts &opt, const std::vector<double> &bb,
                       std::vector<double> &rr, shtg_cg_stats *stt) {
    Plan *p = s.p;
    cudaStream_t st = s.st;
    const int nb = s.nb;
    double2 *B = p->v64[0], *X = p->v64[1], *R = p->v64[2], *Tt = p->v64[6];
    float2 *r32 = p->v32[0], *z32 = p->v32[1], *p32 = p->v32[2], *q32 = p->v32[3], *x32 = p->v32[4];
    const float *minv = p->d_minv32;
    // per-realization scalars on the device: [0,nb) 1/scale, [nb,2nb) FP32 target^2,
    // [2nb,3nb) direction rescale, [3nb,4nb) scale
    double *d_sc = p->d_part + 4 * (int64_t)p->max_batch * SHTG_RED_BLOCKS;
    const size_t vb32 = sizeof(float2) * (size_t)s.nvec;
    const double delta = opt.reliable_delta;
    std::vector<double> scale(nb, 0.0), sc(4 * nb);
    std::vector<char> done(nb, 0);
    SHTG_CUDA(cudaMemsetAsync(X, 0, sizeof(double2) * (size_t)s.nvec, st));
    SHTG_CUDA(cudaMemcpyAsync(R, B, sizeof(double2) * (size_t)s.nvec, cudaMemcpyDeviceToDevice, st));
    rr = bb;
    IterGraph graph;
    int it = 0, first = 1;
    for (;;) {
        // ---- residual replacement (the first pass starts the iteration)
        int active = 0;
        for (int b = 0; b < nb; ++b) {
            done[b] = bb[b] == 0.0 || rr[b] <= opt.tol * opt.tol * bb[b];
            const double nr = sqrt(rr[b]);
            const double old = scale[b];
            scale[b] = done[b] ? 0.0 : nr;
            sc[b] = done[b] ? 0.0 : 1.0 / nr;
            // the FP32 stage runs until a realization has reduced its residual by
            // delta (the host's check); each one stops on its own at 0.1 delta, well
            // above the FP32 rounding floor: a preconditioner close to the exact
            // inverse takes the residual there in one or two iterations, and CG on
            // rounding noise until the next check can diverge; -1 = frozen
            sc[nb + b] = done[b] ? -1.0 : (0.1 * delta) * (0.1 * delta);
            sc[2 * nb + b] = (done[b] || old == 0.0) ? 0.0 : old / nr;
            sc[3 * nb + b] = scale[b];
            active += !done[b];
        }
        if (!active || it >= opt.maxiter) break;
        SHTG_CUDA(cudaMemcpyAsync(d_sc, sc.data(), sizeof(double) * 4 * nb, cudaMemcpyHostToDevice, st));
        k_scale_down<<<s.vgrid, RT, 0, st>>>(R, r32, s.per, d_sc);
        if (first) SHTG_CUDA(cudaMemsetAsync(x32, 0, vb32, st));
        else k_scale_vec<<<s.vgrid, RT, 0, st>>>(p32, s.per, d_sc + 2 * nb);
        k_update<float, true><<<s.rgrid, RT, 0, st>>>(nullptr, r32, z32, nullptr, nullptr, minv, s.nc,
                                                     s.nalm, p->d_mofidx, p->d_scal, p->d_part);
        SHTG_TRY(precond_fix<float>(s, r32, z32));
        if (!first) k_restart_dir<<<s.vgrid, RT, 0, st>>>(p32, z32, s.per, p->d_scal);
        k_scal_reliable<<<1, 1024, 0, st>>>(p->d_part, p->d_scal, nb, d_sc + nb);
        p->prof.launches += first ? 3 : 5;
        SHTG_CHECK_LAUNCH("reliable update");
        // the search direction is kept (rescaled to the new normalization); only
        // the first pass starts it from z
        if (first) SHTG_CUDA(cudaMemcpyAsync(p32, z32, vb32, cudaMemcpyDeviceToDevice, st));
        first = 0;
        // ---- FP32 iterations until a realization is ready for a replacement
        int since = 0;
        for (;;) {
            const int nrun = std::min(std::max(1, opt.check_every), opt.maxiter - it);
            SHTG_TRY(run_iterations<float>(s, graph, nrun, x32, r32, z32, p32, q32, minv));
            it += nrun;
            SHTG_CUDA(cudaMemcpyAsync(p->h_pinned, p->d_scal, sizeof(double) * 16 * nb,
                                      cudaMemcpyDeviceToHost, st));
            SHTG_CUDA(cudaStreamSynchronize(st));
            int ready = 0, still = 0;
            for (int b = 0; b < nb; ++b) {
                const double *h = p->h_pinned + b * 16;
                if (h[S_BAD] != 0.0) {
                    if (s.tc) SHTG_TRY(check_device_flag(p, s.st));   // an expired wait explains it
                    char buf[256];
                    snprintf(buf, sizeof buf,
                             "non-finite or non-positive curvature in the FP32 PCG (system %d, stage iteration %g: "
                             "<p, Ap> = %.3e, <r, z> = %.3e, |r|^2 = %.3e of the stage's start)",
                             b, h[S_ITERS], h[S_PQ], h[S_RZ], h[S_RR]);
                    set_error(buf);
                    return SHTG_ERR_NONFINITE;
                }
                if (done[b]) continue;
                const bool act = h[S_ACTIVE] != 0.0;
                still += act;
                if (act && h[S_RR] <= delta * delta) ready += 1;
            }
            since += nrun;
            // replace as soon as one realization has dropped by delta: waiting
            // for all lets the FP32 recursion drift and costs more iterations
            // than the extra FP64 applications save
            if (ready || !still || it >= opt.maxiter || since >= 400) break;
        }
        stt->iterations = it;
        // ---- x += scale * x32 ; R = B - A X in FP64
        k_correct<<<s.vgrid, RT, 0, st>>>(X, x32, s.per, d_sc + 3 * nb);
        p->prof.launches += 1;
        SHTG_CHECK_LAUNCH("k_correct");
        SHTG_CUDA(cudaMemsetAsync(x32, 0, vb32, st));
        SHTG_TRY(matvec<double>(s, X, Tt));
        stt->fp64_matvecs++;
        stt->outer_steps++;
        k_resid<<<grid_1d(s.nvec), RT, 0, st>>>(B, Tt, R, s.nvec);
        p->prof.launches += 1;
        SHTG_TRY(norms2(s, R, rr));
    }
    stt->iterations = it;
    return SHTG_OK;
}

// The low block or the azimuthal blocks, built for every system with the
// first realization's C_l scale (for the others the preconditioner is still
// symmetric positive definite, only not the exact block inverse).
static int precond_setup(Solve &s, const shtg_cg_opts &opt, const shtg_problem *pr) {
    s.pc = opt.precond;
    const double isc = pr->cl_scale ? 1.0 / pr->cl_scale[0] : 1.0;
    if (opt.precond == SHTG_PRECOND_LOWL) return lowl_setup(s.p, opt.lowl_lmax, s.nc, isc, s.st);
    if (opt.precond == SHTG_PRECOND_AZIM) return az_setup(s.p, opt.block_lmax, s.nc, isc, s.st);
    return SHTG_OK;
}

int precond_apply(Plan *p, const shtg_problem *pr, const shtg_cg_opts *o, const double *r, double *z,
                  cudaStream_t st) {
    SHTG_TRY(check_problem(p, pr));
    if (!o || o->precond < SHTG_PRECOND_NONE || o->precond > SHTG_PRECOND_AZIM) {
        set_error("precond must be SHTG_PRECOND_NONE, SHTG_PRECOND_DIAG, SHTG_PRECOND_LOWL or SHTG_PRECOND_AZIM");
        return SHTG_ERR_ARG;
    }
    SHTG_TRY(setup_operator(p, pr, 0, o->precond, st));
    Solve s = make_solve(p, pr->nbatch, pr->ncomp, st);
    SHTG_TRY(precond_setup(s, *o, pr));
    double2 *R = p->v64[2];
    SHTG_CUDA(cudaMemcpyAsync(R, r, sizeof(double2) * (size_t)s.nvec, cudaMemcpyDeviceToDevice, st));
    double2 *Z = reinterpret_cast<double2 *>(z);
    if (o->mode == SHTG_CG_MIXED || o->mode == SHTG_CG_MIXED_TC) {
        // what the FP32 iteration applies: FP32 vectors, FP32 diagonal and blocks
        float2 *r32 = p->v32[0], *z32 = p->v32[1];
        const int64_t n2 = 2 * s.nvec;
        k_to_float<<<grid_1d(n2), RT, 0, st>>>(reinterpret_cast<const double *>(R), reinterpret_cast<float *>(r32), n2);
        k_update<float, true><<<s.rgrid, RT, 0, st>>>(nullptr, r32, z32, nullptr, nullptr, p->d_minv32, s.nc, s.nalm,
                                                      p->d_mofidx, p->d_scal, p->d_part);
        p->prof.launches += 2;
        SHTG_CHECK_LAUNCH("k_update");
        SHTG_TRY(precond_fix<float>(s, r32, z32));
        k_to_double<<<grid_1d(n2), RT, 0, st>>>(reinterpret_cast<const float *>(z32), z, n2);
        p->prof.launches += 1;
        SHTG_CHECK_LAUNCH("k_to_double");
        SHTG_CUDA(cudaStreamSynchronize(st));
        return SHTG_OK;
    }
    k_update<double, true><<<s.rgrid, RT, 0, st>>>(nullptr, R, Z, nullptr, nullptr, p->d_minv64, s.nc, s.nalm,
                                                   p->d_mofidx, p->d_scal, p->d_part);
    SHTG_CHECK_LAUNCH("k_update");
    p->prof.launches += 1;
    if (s.pc == SHTG_PRECOND_LOWL)
        SHTG_TRY(lowl_apply<double>(p, reinterpret_cast<const double *>(R), z, s.nb, s.per, p->d_part, st));
    if (s.pc == SHTG_PRECOND_AZIM)
        SHTG_TRY(az_apply<double>(p, reinterpret_cast<const double *>(R), z, s.nb, s.per, p->d_part, st, true));
    SHTG_CUDA(cudaStreamSynchronize(st));
    return SHTG_OK;
}

// One cg_sample call between its phases: cg_begin checks the arguments,
// sets up the operator and the preconditioner and forms the right-hand
// sides; the solve runs; cg_end reports the FP64 residuals, copies the
// solution out and fills the stats.  The grouped chains solve runs the
// phases of several plans around one grouped iteration.
struct CgCall {
    shtg_cg_opts opt;
    shtg_cg_stats stt;
    Solve s;
    std::vector<double> bb, rr;
    int host = 0;
    double t0 = 0.0, t1 = 0.0;
    long long launches0 = 0;
};

static int cg_begin(Plan *p, const shtg_problem *pr, const double *alm_out, const shtg_cg_opts *o,
                    cudaStream_t st, CgCall &c) {
    SHTG_TRY(check_problem(p, pr));
    shtg_cg_opts &opt = c.opt;
    if (o) {
        opt = *o;
    } else {
        memset(&opt, 0, sizeof(opt));
        opt.tol = 1e-6;
        opt.maxiter = 1000;
        opt.mode = SHTG_CG_MIXED;
        opt.precond = SHTG_PRECOND_DIAG;
    }
    if (!(opt.tol > 0)) opt.tol = 1e-6;
    if (opt.maxiter <= 0) opt.maxiter = 1000;
    if (!(opt.reliable_delta > 0 && opt.reliable_delta < 1)) opt.reliable_delta = 1e-2;
    if (opt.check_every <= 0) opt.check_every = 4;
    if (opt.mode != SHTG_CG_FP64 && opt.mode != SHTG_CG_MIXED && opt.mode != SHTG_CG_MIXED_TC &&
        opt.mode != SHTG_CG_BLOCK) {
        set_error("mode must be SHTG_CG_FP64, SHTG_CG_MIXED, SHTG_CG_MIXED_TC or SHTG_CG_BLOCK");
        return SHTG_ERR_ARG;
    }
    if (opt.mode == SHTG_CG_BLOCK) {
        // the conditions of App. A's block-diagonal form (the ring-constant
        // N^-1 is checked on the device once it is staged)
        if (!(p->flags & SHTG_BLOCK_SOLVER)) {
            set_error("SHTG_CG_BLOCK needs a plan created with SHTG_BLOCK_SOLVER");
            return SHTG_ERR_ARG;
        }
        if (pr->ncomp != 1) {
            set_error("SHTG_CG_BLOCK solves temperature problems only");
            return SHTG_ERR_ARG;
        }
        for (int r = 0; r < p->nring; ++r)
            if (p->nphi[r] < 2 * p->lmax + 1) {
                set_error("SHTG_CG_BLOCK needs nphi >= 2 lmax + 1 on every ring (ring " + std::to_string(r) +
                          " has " + std::to_string(p->nphi[r]) + ")");
                return SHTG_ERR_ARG;
            }
        if (pr->cl_scale)
            for (int b = 1; b < pr->nbatch; ++b)
                if (pr->cl_scale[b] != pr->cl_scale[0]) {
                    set_error("SHTG_CG_BLOCK: the realizations must share one C_l scale");
                    return SHTG_ERR_ARG;
                }
    }
    if (opt.precond < SHTG_PRECOND_NONE || opt.precond > SHTG_PRECOND_AZIM) {
        set_error("precond must be SHTG_PRECOND_NONE, SHTG_PRECOND_DIAG, SHTG_PRECOND_LOWL or SHTG_PRECOND_AZIM");
        return SHTG_ERR_ARG;
    }
    if (opt.fp64_arith != SHTG_ARITH_DEFAULT && opt.fp64_arith != SHTG_ARITH_FP64 &&
        opt.fp64_arith != SHTG_ARITH_DF64) {
        set_error("fp64_arith must be SHTG_ARITH_DEFAULT, SHTG_ARITH_FP64 or SHTG_ARITH_DF64");
        return SHTG_ERR_ARG;
    }
    const int host = (opt.flags & SHTG_HOST_INPUTS) ? 1 : 0;
    c.host = host;
    const int split = (opt.flags & SHTG_SPLIT_RHS) ? 1 : 0;
    if (!pr->d || !pr->w1 || !pr->w2 || !alm_out) {
        set_error("d, w1, w2 and alm_out are required");
        return SHTG_ERR_ARG;
    }
    if (split && 2 * pr->nbatch > p->max_batch) {
        set_error("SHTG_SPLIT_RHS solves 2 nbatch systems: needs max_batch >= 2 nbatch");
        return SHTG_ERR_ARG;
    }
    shtg_cg_stats &stt = c.stt;
    memset(&stt, 0, sizeof(stt));
    p->prof.on = (opt.flags & SHTG_PROFILE) != 0;
    p->prof.n = 0;
    p->prof.open_cls = -1;
    c.launches0 = p->prof.launches;
    const double t0 = now_ms();
    c.t0 = t0;
    // nb systems: the realizations, or (split) their mean-field right-hand
    // sides followed by their fluctuation right-hand sides
    const int nr = pr->nbatch, nb = split ? 2 * nr : nr, nc = pr->ncomp;
    c.s = make_solve(p, nb, nc, st);
    Solve &s = c.s;
    s.tc = opt.mode == SHTG_CG_MIXED_TC;
    s.df = opt.fp64_arith == SHTG_ARITH_DF64 ||
           (opt.fp64_arith == SHTG_ARITH_DEFAULT && opt.mode != SHTG_CG_FP64 && opt.mode != SHTG_CG_BLOCK);
    {
        const char *e = getenv("SHTG_GRAPHS");
        s.graphs = !(opt.flags & SHTG_NO_GRAPHS) && !(e && e[0] == '0');
    }
    SHTG_TRY(setup_operator(p, pr, host, opt.mode == SHTG_CG_BLOCK ? 0 : opt.precond, st, nb));
    if (opt.mode != SHTG_CG_BLOCK) SHTG_TRY(precond_setup(s, opt, pr));
    const double ts = now_ms();
    double2 *B = p->v64[0], *Tt = p->v64[6];
    // ---- RHS: B Y^T (N^-1 d + N^-1/2 w2) + S^-1/2 w1 in FP64; split: the
    // mean field's B Y^T N^-1 d (Eq. mean-field-map) for systems [0, nr) and
    // the fluctuation's S^-1/2 w1 + B Y^T N^-1/2 w2 (Eq. fluc-map) for [nr, 2 nr)
    const int64_t npix = p->npix;
    const size_t mapbytes = sizeof(double) * (size_t)nr * nc * npix;
    const dim3 pgrid(grid_1d(npix).x, nr * nc);
    const int wofs = split ? nr : 0;   // first system that receives w2 (and w1)
    if (host) {
        SHTG_CUDA(cudaMemcpyAsync(p->d_stage, pr->d, mapbytes, cudaMemcpyHostToDevice, st));
        k_rhs_pix<<<pgrid, RT, 0, st>>>(p->d_stage, nullptr, p->d_ninv64, nb, 0, nc, npix, 0, p->d_map64);
        SHTG_CUDA(cudaMemcpyAsync(p->d_stage, pr->w2, mapbytes, cudaMemcpyHostToDevice, st));
        k_rhs_pix<<<pgrid, RT, 0, st>>>(nullptr, p->d_stage, p->d_ninv64, nb, wofs, nc, npix, !split,
                                        p->d_map64);
        p->prof.launches += 2;
    } else if (split) {
        k_rhs_pix<<<pgrid, RT, 0, st>>>(pr->d, nullptr, p->d_ninv64, nb, 0, nc, npix, 0, p->d_map64);
        k_rhs_pix<<<pgrid, RT, 0, st>>>(nullptr, pr->w2, p->d_ninv64, nb, nr, nc, npix, 0, p->d_map64);
        p->prof.launches += 2;
    } else {
        k_rhs_pix<<<pgrid, RT, 0, st>>>(pr->d, pr->w2, p->d_ninv64, nb, 0, nc, npix, 0, p->d_map64);
        p->prof.launches += 1;
    }
    SHTG_CHECK_LAUNCH("k_rhs_pix");
    {
        const int64_t rowsz = (int64_t)(p->lmax + 1) * p->nring;
        SHTG_TRY(ring_analysis<double>(p, p->d_map64, nb * nc, 0, p->d_phase64, st));
        SHTG_TRY(op_analysis(s, 0, p->d_phase64, p->d_ltab64, B, nc));
        if (nc == 3) SHTG_TRY(op_analysis(s, 2, p->d_phase64 + nb * rowsz, p->d_ltab64, B + p->nalm, 3));
        const double2 *w1 = reinterpret_cast<const double2 *>(pr->w1);
        const size_t w1n = (size_t)nr * nc * p->nalm;
        if (host) {
            SHTG_CUDA(cudaMemcpyAsync(Tt, pr->w1, sizeof(double2) * w1n, cudaMemcpyHostToDevice, st));
            w1 = Tt;
        }
        k_rhs_alm<<<dim3(grid_1d(s.per).x, nr), RT, 0, st>>>(w1, B + wofs * s.per, nc, p->nalm, p->lmax + 1,
                                                             p->d_lofidx, p->d_mofidx,
                                                             p->d_ltab64 + 5 * (p->lmax + 1),
                                                             p->d_rsc64 + wofs);
        p->prof.launches += 1;
        SHTG_CHECK_LAUNCH("k_rhs_alm");
    }
    std::vector<double> &bb = c.bb;
    SHTG_TRY(norms2(s, B, bb));
    for (int b = 0; b < nb; ++b)
        if (!std::isfinite(bb[b])) {
            set_error("non-finite right-hand side in realization " + std::to_string(b) +
                      ": d, w1, w2 or N^-1 holds NaN or Inf");
            return SHTG_ERR_NONFINITE;
        }
    const double t1 = now_ms();
    c.t1 = t1;
    stt.ms_setup = ts - t0;
    stt.ms_rhs = t1 - ts;
    return SHTG_OK;
}

static int cg_end(Plan *p, CgCall &c, double *alm_out, shtg_cg_stats *stats, cudaStream_t st) {
    const shtg_cg_opts &opt = c.opt;
    shtg_cg_stats &stt = c.stt;
    Solve &s = c.s;
    const int nb = s.nb;
    double2 *X = p->v64[1];
    double worst = 0.0;
    int conv_all = 1;
    for (int b = 0; b < nb; ++b) {
        const double rel = c.bb[b] > 0 ? sqrt(c.rr[b] / c.bb[b]) : 0.0;
        worst = std::max(worst, rel);
        if (rel > opt.tol) conv_all = 0;
    }
    stt.rel_residual = worst;
    stt.converged = conv_all;
    SHTG_CUDA(cudaMemcpyAsync(alm_out, X, sizeof(double2) * (size_t)s.nvec,
                              c.host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, st));
    SHTG_CUDA(cudaStreamSynchronize(st));
    const double t2 = now_ms();
    stt.ms_solve = t2 - c.t1;
    stt.ms_total = t2 - c.t0;
    prof_collect(p, stt.kernel_ms, stt.kernel_launches);
    p->prof.on = false;
    stt.launches = p->prof.launches - c.launches0;
    if (stats) *stats = stt;
    if (!conv_all) {
        set_error("maximum iterations reached before the tolerance");
        return SHTG_ERR_NOT_CONVERGED;
    }
    return SHTG_OK;
}

int cg_sample(Plan *p, const shtg_problem *pr, double *alm_out, const shtg_cg_opts *o,
              shtg_cg_stats *stats, cudaStream_t st) {
    CgCall c;
    SHTG_TRY(cg_begin(p, pr, alm_out, o, st, c));
    const shtg_cg_opts &opt = c.opt;
    shtg_cg_stats &stt = c.stt;
    Solve &s = c.s;
    const int nb = s.nb;
    double2 *B = p->v64[0], *X = p->v64[1], *R = p->v64[2], *Tt = p->v64[6];
    int rc = SHTG_OK;
    std::vector<double> &rr = c.rr;
    if (opt.mode == SHTG_CG_BLOCK) {
        SHTG_TRY(block_solve(p, B, X, nb, pr->cl_scale ? 1.0 / pr->cl_scale[0] : 1.0, st));
        // the FP64 residual of the exact solve, for the stats
        SHTG_TRY(matvec<double>(s, X, Tt));
        stt.fp64_matvecs = 1;
        k_resid<<<grid_1d(s.nvec), RT, 0, st>>>(B, Tt, R, s.nvec);
        p->prof.launches += 1;
        SHTG_TRY(norms2(s, R, rr));
    } else if (opt.mode == SHTG_CG_FP64) {
        int iters = 0, conv = 0;
        rc = pcg<double>(s, B, X, opt.tol, opt.maxiter, opt.check_every, &iters, &conv);
        stt.iterations = iters;
        if (rc != SHTG_OK) return rc;
        SHTG_TRY(matvec<double>(s, X, Tt));
        stt.fp64_matvecs = 1;
        k_resid<<<grid_1d(s.nvec), RT, 0, st>>>(B, Tt, R, s.nvec);
        p->prof.launches += 1;
        SHTG_TRY(norms2(s, R, rr));
    } else {
        SHTG_TRY(mixed_solve(s, opt, c.bb, rr, &stt));
        if (s.tc) SHTG_TRY(check_device_flag(p, st));
    }
    (void)nb;
    return cg_end(p, c, alm_out, stats, st);
}

// ================================================== chains: grouped solve
// Chains of several geometries solved together (flag SHTG_GROUPED of
// shtg_cg_sample_chains): every stage of the FP32 PCG iteration (Legendre
// synthesis, ring stage with N^-1, Legendre transpose, prior and <p, Ap>,
// the scalar and vector updates, the azimuthal blocks) is one launch over
// the work of every group (the ring stage: one per transform-length class),
// and the iteration is replayed as one CUDA graph.  Each group keeps its own
// plan, vectors and per-realization scalars; a group whose realizations have
// all converged is skipped through a device flag (its plan's d_flag[1]).
// The FP64-accurate steps (right-hand side, residual replacements) stay per
// group: a group's replacement runs at the host check after one of its
// realizations has dropped by reliable_delta, while the others go on.
struct GroupIter {
    int ng = 0, nc = 1, nbtot = 0, pc = SHTG_PRECOND_DIAG;
    std::vector<Plan *> ps;
    std::vector<const float2 *> xin, xin2;
    std::vector<float2 *> F, F2, q, q2, r32, z32;
    std::vector<const float *> beam, ninv;
    std::vector<int> rs0, rs2, nmaps, nring_maps, nT, nb;
    std::vector<int64_t> per;
    std::vector<double *> part;
    std::vector<const int *> act;
    VecGroups V{};
};

static int pcg_iteration_grp(GroupIter &G, cudaStream_t st) {
    Plan *const *ps = G.ps.data();
    const int *const *act = G.act.data();
    SHTG_TRY(leg_synth_grp(G.ng, ps, 0, G.xin.data(), G.rs0.data(), G.nmaps.data(), G.beam.data(), G.F.data(), act,
                           st));
    if (G.nc == 3)
        SHTG_TRY(leg_synth_grp(G.ng, ps, 2, G.xin2.data(), G.rs2.data(), G.nmaps.data(), G.beam.data(), G.F2.data(),
                               act, st));
    SHTG_TRY(ring_fused_grp<float>(G.ng, ps, G.F.data(), G.nring_maps.data(), G.nT.data(), G.ninv.data(), act, st));
    SHTG_TRY(leg_analysis_grp(G.ng, ps, 0, G.F.data(), G.nmaps.data(), G.beam.data(), G.q.data(), G.rs0.data(), act,
                              st));
    if (G.nc == 3)
        SHTG_TRY(leg_analysis_grp(G.ng, ps, 2, G.F2.data(), G.nmaps.data(), G.beam.data(), G.q2.data(),
                                  G.rs2.data(), act, st));
    Plan *acct = ps[0];
    prof_begin(acct, K_VEC, st);
    const dim3 rows(RB, G.nbtot);
    k_prior_add_grp<<<rows, RT, 0, st>>>(G.V);
    k_scal_alpha_grp<<<G.ng, 1024, 0, st>>>(G.V, 1e-6);
    k_update_grp<<<rows, RT, 0, st>>>(G.V);
    if (G.pc == SHTG_PRECOND_AZIM)
        SHTG_TRY(az_apply_grp(G.ng, ps, reinterpret_cast<const float *const *>(G.r32.data()),
                              reinterpret_cast<float *const *>(G.z32.data()), G.nb.data(), G.per.data(),
                              G.part.data(), act, st));
    k_scal_beta_grp<<<G.ng, 1024, 0, st>>>(G.V);
    k_pupdate_grp<<<rows, RT, 0, st>>>(G.V);
    prof_end(acct, st, 5);
    SHTG_CHECK_LAUNCH("grouped pcg iteration");
    return SHTG_OK;
}

// nrun grouped iterations; the first call runs one eagerly, captures the
// next one on the first plan's capture stream and replays it
static int run_iterations_grp(GroupIter &G, IterGraph &graph, int nrun, bool graphs, cudaStream_t st) {
    Plan *p = G.ps[0];
    if (!graphs || p->prof.on) {
        for (int k = 0; k < nrun; ++k) SHTG_TRY(pcg_iteration_grp(G, st));
        return SHTG_OK;
    }
    if (!graph.exec && nrun > 0) {
        SHTG_TRY(pcg_iteration_grp(G, st));
        if (--nrun == 0) return SHTG_OK;
        const long long l0 = p->prof.launches;
        cudaStream_t cs = p->cap_stream;
        SHTG_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed));
        const int rc = pcg_iteration_grp(G, cs);
        cudaGraph_t g = nullptr;
        const cudaError_t e = cudaStreamEndCapture(cs, &g);
        graph.launches = p->prof.launches - l0;
        p->prof.launches = l0;
        if (rc != SHTG_OK) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture", __FILE__, __LINE__);
        graph.graph = g;
        SHTG_CUDA(cudaGraphInstantiate(&graph.exec, g, 0));
    }
    for (int k = 0; k < nrun; ++k) {
        SHTG_CUDA(cudaGraphLaunch(graph.exec, st));
        p->prof.launches += graph.launches;
    }
    return SHTG_OK;
}

// The grouped mixed solve: mixed_solve's stages, with the FP32 iterations of
// every group in one grouped iteration.
static int mixed_solve_grp(int ng, Plan *const *ps, std::vector<CgCall> &c, cudaStream_t st) {
    const shtg_cg_opts &opt = c[0].opt;
    const double delta = opt.reliable_delta;
    struct GState {
        std::vector<double> scale, sc;
        std::vector<char> done;
        double *d_sc = nullptr;
        bool first = true, finished = false, replace = true;
        int since = 0;
    };
    std::vector<GState> gs(ng);
    GroupIter G;
    G.ng = ng;
    G.nc = c[0].s.nc;
    G.pc = opt.precond;
    G.ps.assign(ps, ps + ng);
    G.V.ng = ng;
    for (int g = 0; g < ng; ++g) {
        Plan *p = ps[g];
        Solve &s = c[g].s;
        s.st = st;
        const int nb = s.nb;
        const int64_t rowsz = (int64_t)(p->lmax + 1) * p->nring;
        float2 *r32 = p->v32[0], *z32 = p->v32[1], *p32 = p->v32[2], *q32 = p->v32[3], *x32 = p->v32[4];
        G.xin.push_back(p32);
        G.xin2.push_back(p32 + s.nalm);
        G.F.push_back(p->d_phase32);
        G.F2.push_back(p->d_phase32 + nb * rowsz);
        G.q.push_back(q32);
        G.q2.push_back(q32 + s.nalm);
        G.r32.push_back(r32);
        G.z32.push_back(z32);
        G.beam.push_back(p->d_ltab32);
        G.ninv.push_back(p->d_ninv32);
        G.rs0.push_back(s.nc);
        G.rs2.push_back(3);
        G.nmaps.push_back(nb);
        G.nring_maps.push_back(nb * s.nc);
        G.nT.push_back(nb);
        G.nb.push_back(nb);
        G.per.push_back(s.per);
        G.part.push_back(p->d_part);
        G.act.push_back(p->d_flag + 1);
        VecGrp &v = G.V.v[g];
        v.x = x32;
        v.r = r32;
        v.z = z32;
        v.p = p32;
        v.q = q32;
        v.minv = p->d_minv32;
        v.sinv = p->d_ltab32 + (p->lmax + 1);
        v.isc = p->d_isc32;
        v.lof = p->d_lofidx;
        v.mof = p->d_mofidx;
        v.scal = p->d_scal;
        v.part = p->d_part;
        v.active = p->d_flag + 1;
        v.nalm = s.nalm;
        v.nc = s.nc;
        v.nb = nb;
        v.lmax1 = p->lmax + 1;
        G.V.firstb[g] = G.nbtot;
        G.nbtot += nb;
        GState &q = gs[g];
        q.scale.assign(nb, 0.0);
        q.sc.assign(4 * nb, 0.0);
        q.done.assign(nb, 0);
        q.d_sc = p->d_part + 4 * (int64_t)p->max_batch * SHTG_RED_BLOCKS;
        double2 *B = p->v64[0], *X = p->v64[1], *R = p->v64[2];
        SHTG_CUDA(cudaMemsetAsync(X, 0, sizeof(double2) * (size_t)s.nvec, st));
        SHTG_CUDA(cudaMemcpyAsync(R, B, sizeof(double2) * (size_t)s.nvec, cudaMemcpyDeviceToDevice, st));
        c[g].rr = c[g].bb;
    }
    G.V.firstb[ng] = G.nbtot;
    bool graphs = true;
    {
        const char *e = getenv("SHTG_GRAPHS");
        graphs = !(opt.flags & SHTG_NO_GRAPHS) && !(e && e[0] == '0');
    }
    IterGraph graph;
    // fork / join events of the concurrent replacements
    struct Events {
        cudaEvent_t fork = nullptr;
        std::vector<cudaEvent_t> join;
        ~Events() {
            if (fork) cudaEventDestroy(fork);
            for (cudaEvent_t e : join)
                if (e) cudaEventDestroy(e);
        }
    } ev;
    SHTG_CUDA(cudaEventCreateWithFlags(&ev.fork, cudaEventDisableTiming));
    ev.join.assign(ng, nullptr);
    for (int g = 0; g < ng; ++g) SHTG_CUDA(cudaEventCreateWithFlags(&ev.join[g], cudaEventDisableTiming));
    int it = 0;
    for (;;) {
        // ---- stage starts (after a residual replacement, or the first one)
        int live = 0;
        for (int g = 0; g < ng; ++g) {
            GState &q = gs[g];
            if (q.finished) continue;
            if (!q.replace) {
                ++live;
                continue;
            }
            q.replace = false;
            Plan *p = ps[g];
            Solve &s = c[g].s;
            const int nb = s.nb;
            const std::vector<double> &bb = c[g].bb, &rr = c[g].rr;
            int active = 0;
            for (int b = 0; b < nb; ++b) {
                q.done[b] = bb[b] == 0.0 || rr[b] <= opt.tol * opt.tol * bb[b];
                const double nr = sqrt(rr[b]);
                const double old = q.scale[b];
                q.scale[b] = q.done[b] ? 0.0 : nr;
                q.sc[b] = q.done[b] ? 0.0 : 1.0 / nr;
                q.sc[nb + b] = q.done[b] ? -1.0 : (0.1 * delta) * (0.1 * delta);
                q.sc[2 * nb + b] = (q.done[b] || old == 0.0) ? 0.0 : old / nr;
                q.sc[3 * nb + b] = q.scale[b];
                active += !q.done[b];
            }
            if (!active || it >= opt.maxiter) {
                q.finished = true;
                SHTG_CUDA(cudaMemsetAsync(p->d_flag + 1, 0, sizeof(int), st));
                continue;
            }
            ++live;
            float2 *r32 = p->v32[0], *z32 = p->v32[1], *p32 = p->v32[2], *x32 = p->v32[4];
            const size_t vb32 = sizeof(float2) * (size_t)s.nvec;
            SHTG_CUDA(cudaMemcpyAsync(q.d_sc, q.sc.data(), sizeof(double) * 4 * nb, cudaMemcpyHostToDevice, st));
            k_scale_down<<<s.vgrid, RT, 0, st>>>(p->v64[2], r32, s.per, q.d_sc);
            if (q.first) SHTG_CUDA(cudaMemsetAsync(x32, 0, vb32, st));
            else k_scale_vec<<<s.vgrid, RT, 0, st>>>(p32, s.per, q.d_sc + 2 * nb);
            k_update<float, true><<<s.rgrid, RT, 0, st>>>(nullptr, r32, z32, nullptr, nullptr, p->d_minv32, s.nc,
                                                         s.nalm, p->d_mofidx, p->d_scal, p->d_part);
            if (G.pc == SHTG_PRECOND_AZIM)
                SHTG_TRY(az_apply<float>(p, reinterpret_cast<const float *>(r32), reinterpret_cast<float *>(z32), nb,
                                         s.per, p->d_part, st, false));
            if (!q.first) k_restart_dir<<<s.vgrid, RT, 0, st>>>(p32, z32, s.per, p->d_scal);
            k_scal_reliable<<<1, 1024, 0, st>>>(p->d_part, p->d_scal, nb, q.d_sc + nb);
            p->prof.launches += q.first ? 3 : 5;
            SHTG_CHECK_LAUNCH("reliable update");
            if (q.first) SHTG_CUDA(cudaMemcpyAsync(p32, z32, vb32, cudaMemcpyDeviceToDevice, st));
            q.first = false;
            SHTG_CUDA(cudaMemsetAsync(p->d_flag + 1, 1, sizeof(int), st));
        }
        if (!live) break;
        // ---- grouped FP32 iterations
        const int nrun = std::min(std::max(1, opt.check_every), opt.maxiter - it);
        SHTG_TRY(run_iterations_grp(G, graph, nrun, graphs, st));
        it += nrun;
        for (int g = 0; g < ng; ++g)
            if (!gs[g].finished) {
                Plan *p = ps[g];
                SHTG_CUDA(cudaMemcpyAsync(p->h_pinned, p->d_scal, sizeof(double) * 16 * c[g].s.nb,
                                          cudaMemcpyDeviceToHost, st));
            }
        SHTG_CUDA(cudaStreamSynchronize(st));
        // ---- host check per group: which groups are due for a replacement
        std::vector<int> due;
        for (int g = 0; g < ng; ++g) {
            GState &q = gs[g];
            if (q.finished) continue;
            Plan *p = ps[g];
            Solve &s = c[g].s;
            const int nb = s.nb;
            c[g].stt.iterations += nrun;
            int ready = 0, still = 0;
            for (int b = 0; b < nb; ++b) {
                const double *h = p->h_pinned + b * 16;
                if (h[S_BAD] != 0.0) {
                    char buf[256];
                    snprintf(buf, sizeof buf,
                             "non-finite or non-positive curvature in the FP32 PCG (group %d, system %d, stage "
                             "iteration %g: <p, Ap> = %.3e, <r, z> = %.3e, |r|^2 = %.3e of the stage's start)",
                             g, b, h[S_ITERS], h[S_PQ], h[S_RZ], h[S_RR]);
                    set_error(buf);
                    return SHTG_ERR_NONFINITE;
                }
                if (q.done[b]) continue;
                const bool act = h[S_ACTIVE] != 0.0;
                still += act;
                if (act && h[S_RR] <= delta * delta) ready += 1;
            }
            q.since += nrun;
            if (ready || !still || it >= opt.maxiter || q.since >= 400) due.push_back(g);
        }
        if (due.empty()) continue;
        // ---- the due groups' replacements, concurrently on their plans' own
        // streams (forked from and joined back into st): x += scale x32,
        // R = B - A X with the group's FP64-accurate operator, ||R||^2 per
        // realization summed on the device in the order of norms2
        SHTG_CUDA(cudaEventRecord(ev.fork, st));
        for (int g : due) {
            Plan *p = ps[g];
            Solve &s = c[g].s;
            const int nb = s.nb;
            cudaStream_t ws = p->work_stream;
            SHTG_CUDA(cudaStreamWaitEvent(ws, ev.fork, 0));
            s.st = ws;
            double2 *B = p->v64[0], *X = p->v64[1], *R = p->v64[2], *Tt = p->v64[6];
            float2 *x32 = p->v32[4];
            k_correct<<<s.vgrid, RT, 0, ws>>>(X, x32, s.per, gs[g].d_sc + 3 * nb);
            SHTG_CHECK_LAUNCH("k_correct");
            SHTG_CUDA(cudaMemsetAsync(x32, 0, sizeof(float2) * (size_t)s.nvec, ws));
            SHTG_TRY(matvec<double>(s, X, Tt));
            k_resid<<<grid_1d(s.nvec), RT, 0, ws>>>(B, Tt, R, s.nvec);
            k_dot<double2><<<s.rgrid, RT, 0, ws>>>(R, R, s.nc, s.nalm, p->d_mofidx, p->d_part, 0, 1);
            double *rsum = p->d_part + 4 * (int64_t)p->max_batch * SHTG_RED_BLOCKS + 4 * (int64_t)p->max_batch;
            k_row_sums<<<1, 256, 0, ws>>>(p->d_part, nb, rsum);
            p->prof.launches += 4;
            SHTG_CHECK_LAUNCH("grouped replacement");
            SHTG_CUDA(cudaMemcpyAsync(p->h_pinned + 16 * (size_t)p->max_batch, rsum, sizeof(double) * nb,
                                      cudaMemcpyDeviceToHost, ws));
            SHTG_CUDA(cudaEventRecord(ev.join[g], ws));
            SHTG_CUDA(cudaStreamWaitEvent(st, ev.join[g], 0));
            s.st = st;
            c[g].stt.fp64_matvecs++;
            c[g].stt.outer_steps++;
        }
        SHTG_CUDA(cudaStreamSynchronize(st));
        for (int g : due) {
            Plan *p = ps[g];
            const int nb = c[g].s.nb;
            c[g].rr.assign(p->h_pinned + 16 * (size_t)p->max_batch, p->h_pinned + 16 * (size_t)p->max_batch + nb);
            gs[g].since = 0;
            gs[g].replace = true;
        }
    }
    return SHTG_OK;
}

int cg_sample_grouped(int ng, Plan *const *ps, const shtg_problem *prs, double *const *outs,
                      const shtg_cg_opts *o, shtg_cg_stats *stats, cudaStream_t st) {
    if (ng < 1 || ng > SHTG_MAX_GROUPS) {
        set_error("SHTG_GROUPED: 1 to " + std::to_string(SHTG_MAX_GROUPS) + " geometry groups per call");
        return SHTG_ERR_ARG;
    }
    if (!o || (o->mode != SHTG_CG_MIXED && o->mode != SHTG_CG_MIXED_TC)) {
        set_error("SHTG_GROUPED needs options with mode SHTG_CG_MIXED or SHTG_CG_MIXED_TC");
        return SHTG_ERR_ARG;
    }
    if (o->precond != SHTG_PRECOND_NONE && o->precond != SHTG_PRECOND_DIAG && o->precond != SHTG_PRECOND_AZIM) {
        set_error("SHTG_GROUPED supports SHTG_PRECOND_NONE, SHTG_PRECOND_DIAG and SHTG_PRECOND_AZIM");
        return SHTG_ERR_ARG;
    }
    if (o->flags & (SHTG_SPLIT_RHS | SHTG_PROFILE)) {
        set_error("SHTG_GROUPED does not combine with SHTG_SPLIT_RHS or SHTG_PROFILE");
        return SHTG_ERR_ARG;
    }
    for (int g = 0; g < ng; ++g)
        if (prs[g].ncomp != prs[0].ncomp) {
            set_error("SHTG_GROUPED: every group needs the same ncomp");
            return SHTG_ERR_ARG;
        }
    int64_t nbtot = 0;
    for (int g = 0; g < ng; ++g) nbtot += (prs[g].nbatch > 0 ? prs[g].nbatch : 0);
    if (nbtot > 65535) {
        set_error("SHTG_GROUPED: at most 65535 realizations over all groups");
        return SHTG_ERR_ARG;
    }
    std::vector<CgCall> c(ng);
    for (int g = 0; g < ng; ++g) {
        const int rc = cg_begin(ps[g], &prs[g], outs[g], o, st, c[g]);
        if (rc != SHTG_OK) {
            set_error("chain group " + std::to_string(g) + ": " + shtg_last_error_string());
            return rc;
        }
    }
    SHTG_TRY(mixed_solve_grp(ng, ps, c, st));
    int worst = SHTG_OK;
    for (int g = 0; g < ng; ++g) {
        const int rc = cg_end(ps[g], c[g], outs[g], stats ? &stats[g] : nullptr, st);
        if (rc != SHTG_OK && (worst == SHTG_OK || worst == SHTG_ERR_NOT_CONVERGED)) {
            worst = rc;
            set_error("chain group " + std::to_string(g) + ": " + shtg_last_error_string());
        }
    }
    return worst;
}

}  // namespace shtg

namespace shtg {

int apply_operator(Plan *p, const shtg_problem *pr, const double *x, double *y, cudaStream_t st) {
    SHTG_TRY(check_problem(p, pr));
    SHTG_TRY(setup_operator(p, pr, 0, 0, st));
    Solve s = make_solve(p, pr->nbatch, pr->ncomp, st);
    return matvec<double>(s, reinterpret_cast<const double2 *>(x), reinterpret_cast<double2 *>(y));
}

int lowl_block(Plan *p, const shtg_problem *pr, int lc, double *H, int *params, int *n, cudaStream_t st) {
    SHTG_TRY(check_problem(p, pr));
    SHTG_TRY(setup_operator(p, pr, 0, 1, st));
    SHTG_TRY(lowl_setup(p, lc, pr->ncomp, pr->cl_scale ? 1.0 / pr->cl_scale[0] : 1.0, st, H));
    const LowL &q = p->lowl;
    *n = q.n;
    if (params)
        for (int i = 0; i < q.n; ++i) {
            params[4 * i + 0] = q.params[i].x;
            params[4 * i + 1] = q.params[i].y;
            params[4 * i + 2] = q.params[i].z;
            params[4 * i + 3] = q.params[i].w;
        }
    return SHTG_OK;
}

int logpost_grad(Plan *p, const double *cl, const double *bl, const float *alm, const float *d,
                 const float *ninv, int nbins, const int *blo, const int *bhi, int flags,
                 double *logp, float *grad, double *gcl, cudaStream_t st) {
    const int L1 = p->lmax + 1;
    SHTG_TRY(build_ltab(p, 1, cl, bl, st));
    // row 2 of the FP32 per-l table (unused by temperature problems) holds 1 / C_l, 0 where held
    std::vector<float> icl(L1);
    for (int l = 0; l < L1; ++l) icl[l] = cl[l] > 0 ? (float)(1.0 / cl[l]) : 0.f;
    float *d_icl = p->d_ltab32 + 2 * L1;
    SHTG_CUDA(cudaMemcpyAsync(d_icl, icl.data(), sizeof(float) * L1, cudaMemcpyHostToDevice, st));
    const float *beam = p->d_ltab32;
    const float2 *a = reinterpret_cast<const float2 *>(alm);
    SHTG_TRY(leg_synth<float>(p, 0, a, 1, 1, beam, p->d_phase32, st));
    SHTG_TRY(ring_synth<float>(p, p->d_phase32, 1, p->d_map32, st));
    k_resid_pix<<<RB, RT, 0, st>>>(d, ninv, p->d_map32, p->npix, p->d_part);
    SHTG_CHECK_LAUNCH("k_resid_pix");
    if (grad) {
        float2 *g = reinterpret_cast<float2 *>(grad);
        SHTG_TRY(ring_analysis<float>(p, p->d_map32, 1, 0, p->d_phase32, st));
        SHTG_TRY(leg_analysis<float>(p, 0, p->d_phase32, 1, beam, g, 1, st));
        k_grad_prior<<<grid_1d(p->nalm), RT, 0, st>>>(a, g, p->nalm, p->d_lofidx, p->d_mofidx, d_icl,
                                                     (flags & SHTG_GRAD_COMPONENTS) ? 1 : 0);
        SHTG_CHECK_LAUNCH("k_grad_prior");
    }
    SHTG_CUDA(cudaMemsetAsync(p->d_lsum, 0, sizeof(double) * L1, st));
    k_prior_lsum<<<grid_1d(p->nalm), RT, 0, st>>>(a, p->nalm, p->d_lofidx, p->d_mofidx, d_icl, p->d_lsum);
    SHTG_CHECK_LAUNCH("k_prior_lsum");
    std::vector<double> part(RB), ls(L1);
    SHTG_CUDA(cudaMemcpyAsync(part.data(), p->d_part, sizeof(double) * RB, cudaMemcpyDeviceToHost, st));
    SHTG_CUDA(cudaMemcpyAsync(ls.data(), p->d_lsum, sizeof(double) * L1, cudaMemcpyDeviceToHost, st));
    SHTG_CUDA(cudaStreamSynchronize(st));
    double chi2 = 0.0, prior = 0.0;
    for (double v : part) chi2 += v;
    for (double v : ls) prior += v;
    if (logp) *logp = -0.5 * chi2 - 0.5 * prior;
    if (gcl)
        for (int k = 0; k < nbins; ++k) {
            double s = 0.0;
            for (int l = std::max(0, blo[k]); l <= std::min(p->lmax, bhi[k]); ++l) s += ls[l];
            gcl[k] = 0.5 * s;
        }
    return SHTG_OK;
}

}  // namespace shtg

namespace shtg {

int fluctuation_rescale(Plan *p, int nc, const double *cl_old, const double *cl_new, const double *f,
                        double *g, int nbatch, cudaStream_t st) {
    if ((nc != 1 && nc != 3) || (nc == 3 && !(p->flags & SHTG_SPIN2)) || !cl_old || !cl_new || !f || !g ||
        nbatch < 1) {
        set_error("fluctuation_rescale: ncomp 1 or 3 (3 needs SHTG_SPIN2), non-null C_l and buffers, nbatch >= 1");
        return SHTG_ERR_ARG;
    }
    const int L1 = p->lmax + 1;
    const int rows = nc == 1 ? 1 : 4;
    // old and new spectra staged in the plan's joint table, then R_l
    double *cl = p->d_jtab, *R = p->d_jtab + 8 * (int64_t)L1;
    SHTG_CUDA(cudaMemcpyAsync(cl, cl_old, sizeof(double) * rows * L1, cudaMemcpyHostToDevice, st));
    SHTG_CUDA(cudaMemcpyAsync(cl + 4 * (int64_t)L1, cl_new, sizeof(double) * rows * L1, cudaMemcpyHostToDevice, st));
    k_rescale_table<<<(L1 + 127) / 128, 128, 0, st>>>(cl, cl + 4 * (int64_t)L1, nc, L1, R);
    SHTG_CHECK_LAUNCH("k_rescale_table");
    k_rescale<<<dim3(grid_1d(p->nalm).x, nbatch), RT, 0, st>>>(
        reinterpret_cast<const double2 *>(f), reinterpret_cast<double2 *>(g), nc, p->nalm, p->d_lofidx,
        p->d_mofidx, R, L1);
    SHTG_CHECK_LAUNCH("k_rescale");
    p->prof.launches += 2;
    // the host spectra must stay valid until the copies ran (pageable memory)
    SHTG_CUDA(cudaStreamSynchronize(st));
    return SHTG_OK;
}

int joint_log_target(Plan *p, const shtg_problem *pr, int precision, const double *a_hat,
                     const double *f_hat, double *logpi, cudaStream_t st) {
    SHTG_TRY(check_problem(p, pr));
    if (!pr->d || !a_hat || !f_hat || !logpi || (precision != SHTG_FP64 && precision != SHTG_DF64)) {
        set_error("joint_log_target: d, a_hat, f_hat and log_pi are required; precision SHTG_FP64 or SHTG_DF64");
        return SHTG_ERR_ARG;
    }
    SHTG_TRY(setup_operator(p, pr, 0, 0, st));
    const int nb = pr->nbatch, nc = pr->ncomp, L1 = p->lmax + 1;
    Solve s = make_solve(p, nb, nc, st);
    s.df = precision == SHTG_DF64;
    double2 *F = p->d_phase64;
    const int64_t rowsz = (int64_t)L1 * p->nring;
    const double *beam = p->d_ltab64;
    auto synth = [&](const double *x) -> int {
        const double2 *a = reinterpret_cast<const double2 *>(x);
        SHTG_TRY(op_synth(s, 0, a, nc, beam, F));
        if (nc == 3) SHTG_TRY(op_synth(s, 2, a + p->nalm, 3, beam, F + nb * rowsz));
        return ring_synth<double>(p, F, nb * nc, p->d_map64, st);
    };
    double *part = p->d_part;   // [3][nb][RB]: chi^2, fluctuation, prior
    SHTG_TRY(synth(a_hat));
    k_joint_pix<<<dim3(RB, nb), RT, 0, st>>>(pr->d, p->d_map64, p->d_ninv64, nb, nc, p->npix, 0, part);
    SHTG_CHECK_LAUNCH("k_joint_pix");
    SHTG_TRY(synth(f_hat));
    k_joint_pix<<<dim3(RB, nb), RT, 0, st>>>(nullptr, p->d_map64, p->d_ninv64, nb, nc, p->npix, 1,
                                              part + nb * RB);
    SHTG_CHECK_LAUNCH("k_joint_pix");
    k_prior_quad<<<dim3(RB, nb), RT, 0, st>>>(reinterpret_cast<const double2 *>(a_hat), nc, p->nalm, L1,
                                               p->d_lofidx, p->d_mofidx, p->d_ltab64 + L1,
                                               p->d_ltab64 + 5 * (int64_t)L1, p->d_isc64, part + 2 * nb * RB);
    SHTG_CHECK_LAUNCH("k_prior_quad");
    p->prof.launches += 3;
    std::vector<double> h(3 * (size_t)nb * RB);
    SHTG_CUDA(cudaMemcpyAsync(h.data(), part, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, st));
    SHTG_CUDA(cudaStreamSynchronize(st));
    for (int b = 0; b < nb; ++b) {
        double t[3] = {0.0, 0.0, 0.0};
        for (int q = 0; q < 3; ++q)
            for (int k = 0; k < RB; ++k) t[q] += h[((size_t)q * nb + b) * RB + k];
        logpi[b] = -0.5 * t[0] - 0.5 * t[2] - 0.5 * t[1];
        if (!std::isfinite(logpi[b])) {
            set_error("joint_log_target: non-finite value in realization " + std::to_string(b));
            return SHTG_ERR_NONFINITE;
        }
    }
    return SHTG_OK;
}

}  // namespace shtg

// Azimuthal block preconditioner: the per-m blocks of App. A built from
// the ring sums of N^-1 (the noise averaged along every ring), inverted
// exactly, as the preconditioner of the PCG on Eq. (mapmakingeq).
//
// When N^-1 is constant along every ring the operator is block-diagonal in
// m (App. A): per m and l, l' >= m
//
//   T-T: delta S^-1_TT + b_l b_l' sum_r W_T,r lambda_lm(theta_r) lambda_l'm(theta_r)
//   E-E: delta S^-1_EE + b_l b_l' sum_r W_P,r (lw_l lw_l' + lx_l lx_l')
//   T-E: delta S^-1_TE
//
// with W_r the sum of N^-1 over ring r (the aliasing of rings with
// nphi < 2 l_max + 1 left out).  For any N^-1 these blocks, with W_r the
// ring sums of the actual N^-1, approximate the operator by its azimuthal
// average; under a constant-latitude mask with holes and a scan pattern they
// capture the mask exactly and leave only the holes and the pattern to the
// iteration.  The imaginary E-B coupling at equal m (sum_r W_P (lw lx' + lx
// lw')) and the B rows are left to the diagonal preconditioner, as are all
// multipoles above l_b: a block Jacobi preconditioner, symmetric and
// positive definite.  Each block serves the real and the imaginary parts of
// every realization.
//
// Over a north / south ring pair lambda(pi - theta) = (-1)^(l-m) lambda
// (App. A), lw has the same parity and lx the opposite one, so every product
// of two profiles sums over pairs with W_N + W_S (l + l' even) or W_N - W_S
// (l + l' odd).  The profiles come from the plan's FP64 recurrence tables
// (the steps and start states of the transforms).  The Gram matrices depend
// on N^-1 only and are kept while it stays bitwise the same; the blocks are
// assembled with the beam and S^-1, factored by Cholesky and the factor
// inverted in FP64 (one CTA per m, packed lower triangles, row i at
// i (i + 1) / 2), and each block's inverse M^-1 = R^-T R^-1 formed as a full
// square by a tiled product (FP64, and an FP32 copy for the FP32 iteration);
// all of it kept while the per-l table and the C_l scale stay the same.  In
// the iteration z = M^-1 r is a row-parallel product over (m, 32-row tile)
// with every realization's real and imaginary parts as right-hand sides.
#include <algorithm>
#include <string>
#include <vector>

#include "common.cuh"

namespace shtg {
namespace {

constexpr int GT = 32;      // Gram tile and pair chunk
constexpr int AZT = 256;    // threads of the ring-sum kernel
constexpr int AZF = 1024;   // threads of the factor kernels (one CTA per m: the largest block alone
                            // bounds the launch, so its rank-1 updates need every warp of the SM)

__host__ __device__ __forceinline__ int64_t tri(int64_t i) { return i * (i + 1) / 2; }

// per ring pair: the sums of N^-1 over its rings (channel ch: T, P) as
// W_N + W_S and W_N - W_S
__global__ void k_az_weights(const double *__restrict__ ninv, int64_t npix, const int64_t *__restrict__ ofs,
                             const int *__restrict__ nphi, int nring, int npairs, double *__restrict__ w) {
    __shared__ double sm[AZT / 32][2];
    const int pr = blockIdx.x, ch = blockIdx.y;
    const int rn = pr, rs = nring - 1 - pr;
    const double *v = ninv + (int64_t)ch * npix;
    double sn = 0.0, ss = 0.0;
    for (int j = threadIdx.x; j < nphi[rn]; j += blockDim.x) sn += v[ofs[rn] + j];
    if (rs != rn)
        for (int j = threadIdx.x; j < nphi[rs]; j += blockDim.x) ss += v[ofs[rs] + j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sn += __shfl_xor_sync(0xffffffffu, sn, o);
        ss += __shfl_xor_sync(0xffffffffu, ss, o);
    }
    const int wp = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        sm[wp][0] = sn;
        sm[wp][1] = ss;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
            a += sm[k][0];
            b += sm[k][1];
        }
        w[((int64_t)ch * 2 + 0) * npairs + pr] = a + b;
        w[((int64_t)ch * 2 + 1) * npairs + pr] = a - b;
    }
}

// profiles of the m values [m0, m0 + nm) for l = m .. lb on the north ring
// of every pair: prof[poff[m - m0] + (l - m) npairs + p]; spin 0 lambda in
// pl, spin 2 lw in pw and lx in px (nc = 3 only)
__global__ void k_az_prof(int lmax, int lb, int npairs, int m0, int spin2, const int64_t *__restrict__ poff,
                          const double *__restrict__ u64, const double2 *__restrict__ rec,
                          const int *__restrict__ ls, const double2 *__restrict__ st,
                          const double4_32a *__restrict__ s2c, const int2 *__restrict__ ls2,
                          const double4_32a *__restrict__ st2, double *__restrict__ pl, double *__restrict__ pw,
                          double *__restrict__ px) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    const int m = m0 + blockIdx.y;
    if (p >= npairs) return;
    const int64_t base = (int64_t)m * (2 * lmax + 1 - m) / 2;
    const int64_t o = (int64_t)m * npairs + p;
    const double u = u64[p];
    const int64_t po = poff[blockIdx.y] + p;
    {
        const int l0 = ls[o];
        const double2 s = st[o];
        double a1 = 0.0, a2 = 0.0;
        for (int l = m; l <= lb; ++l) {
            const double2 cf = rec[base + l];
            const double t = cf.x * a1;
            const double v = fma(t, -u, fma(cf.y, a2, t));
            a2 = a1;
            a1 = v;
            if (l == l0) {
                a2 = s.x;
                a1 = s.y;
            }
            pl[po + (int64_t)(l - m) * npairs] = a1;
        }
    }
    if (spin2) {
        const int2 q = ls2[o];
        const double4_32a s = st2[o];
        double a1 = 0.0, a2 = 0.0, b1 = 0.0, b2 = 0.0;
        for (int l = m; l <= lb; ++l) {
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
            pw[po + (int64_t)(l - m) * npairs] = a1 + b1;
            px[po + (int64_t)(l - m) * npairs] = a1 - b1;
        }
    }
}

// Gram matrices of a chunk, packed lower triangles: grid.x the 32 x 32
// tiles (I >= J) of the largest block, grid.y the m of the chunk, grid.z the
// component (0: T from lambda with the T weights; 1: E from lw, lx with the
// P weights); 16 x 16 threads with 2 x 2 entries each.  The I rows of a pair
// chunk are staged already multiplied by the pair weights of both parities
// (W_N + W_S for l + l' even, W_N - W_S for odd; the tile offsets are even,
// so a thread's entry (a, b) has parity (a + b) & 1), which leaves one FP64
// multiply-add per profile product on GB300's narrow FP64 pipe.
__global__ void __launch_bounds__(256) k_az_gram(int lb, int npairs, int m0, const int64_t *__restrict__ poff,
                                                 const int64_t *__restrict__ goff, const double *__restrict__ pl,
                                                 const double *__restrict__ pw, const double *__restrict__ px,
                                                 const double *__restrict__ w, double *__restrict__ G) {
    // dynamic: sIw[par][prof][GT][GT] then sJ[prof][GT][GT + 1]
    extern __shared__ __align__(16) unsigned char az_raw[];
    double(*sIw)[2][GT][GT] = reinterpret_cast<double(*)[2][GT][GT]>(az_raw);
    double(*sJ)[GT][GT + 1] = reinterpret_cast<double(*)[GT][GT + 1]>(az_raw + sizeof(double) * 4 * GT * GT);
    const int m = m0 + blockIdx.y, c = blockIdx.z;
    const int k = lb + 1 - m;
    const int nt = (k + GT - 1) / GT;
    int t = blockIdx.x, I = 0;
    while (t > I) {
        t -= I + 1;
        ++I;
    }
    const int J = t;
    if (I >= nt) return;
    const double *A0 = (c == 0 ? pl : pw) + poff[blockIdx.y];
    const double *A1 = px + poff[blockIdx.y];
    const double *wc = w + (int64_t)c * 2 * npairs;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    double acc[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
    const int nprof = c == 0 ? 1 : 2;
    for (int p0 = 0; p0 < npairs; p0 += GT) {
        for (int e = threadIdx.x; e < GT * GT; e += 256) {
            const int r = e / GT, q = e % GT;
            const int p = p0 + q;
            const int li = I * GT + r, lj = J * GT + r;
            const bool pi = p < npairs && li < k, pj = p < npairs && lj < k;
            const double w0 = p < npairs ? wc[p] : 0.0, w1 = p < npairs ? wc[npairs + p] : 0.0;
            const double a0 = pi ? A0[(int64_t)li * npairs + p] : 0.0;
            sIw[0][0][r][q] = a0 * w0;
            sIw[1][0][r][q] = a0 * w1;
            sJ[0][r][q] = pj ? A0[(int64_t)lj * npairs + p] : 0.0;
            if (nprof == 2) {
                const double a1 = pi ? A1[(int64_t)li * npairs + p] : 0.0;
                sIw[0][1][r][q] = a1 * w0;
                sIw[1][1][r][q] = a1 * w1;
                sJ[1][r][q] = pj ? A1[(int64_t)lj * npairs + p] : 0.0;
            }
        }
        __syncthreads();
        const int r0 = 2 * ty, r1 = 2 * ty + 1, c0 = 2 * tx, c1 = 2 * tx + 1;
        if (nprof == 1) {
#pragma unroll 8
            for (int q = 0; q < GT; ++q) {
                const double j0 = sJ[0][c0][q], j1 = sJ[0][c1][q];
                acc[0][0] = fma(sIw[0][0][r0][q], j0, acc[0][0]);
                acc[0][1] = fma(sIw[1][0][r0][q], j1, acc[0][1]);
                acc[1][0] = fma(sIw[1][0][r1][q], j0, acc[1][0]);
                acc[1][1] = fma(sIw[0][0][r1][q], j1, acc[1][1]);
            }
        } else {
#pragma unroll 4
            for (int q = 0; q < GT; ++q) {
                const double j0 = sJ[0][c0][q], j1 = sJ[0][c1][q], k0 = sJ[1][c0][q], k1 = sJ[1][c1][q];
                acc[0][0] = fma(sIw[0][1][r0][q], k0, fma(sIw[0][0][r0][q], j0, acc[0][0]));
                acc[0][1] = fma(sIw[1][1][r0][q], k1, fma(sIw[1][0][r0][q], j1, acc[0][1]));
                acc[1][0] = fma(sIw[1][1][r1][q], k0, fma(sIw[1][0][r1][q], j0, acc[1][0]));
                acc[1][1] = fma(sIw[0][1][r1][q], k1, fma(sIw[0][0][r1][q], j1, acc[1][1]));
            }
        }
        __syncthreads();
    }
    double *Gm = G + goff[m] + (int64_t)c * tri(k);
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const int i = I * GT + 2 * ty + a, j = J * GT + 2 * tx + b;
            if (i < k && j <= i) Gm[tri(i) + j] = acc[a][b];
        }
}
constexpr size_t AZ_GRAM_SMEM = sizeof(double) * (4 * GT * GT + 2 * GT * (GT + 1));

// H_m = b b G + S^-1 (isc) over the rows [T l = m .. lb, E l = m .. lb];
// held multipoles give identity rows
__global__ void k_az_assemble(int lb, int ncb, const int64_t *__restrict__ goff, const int64_t *__restrict__ hoff,
                              const double *__restrict__ G, const double *__restrict__ ltab, int lmax1, double isc,
                              double *__restrict__ H) {
    const int m = blockIdx.y;
    const int k = lb + 1 - m, n = ncb * k;
    const int64_t ne = tri(n);
    const double *Gm = G + goff[m];
    double *Hm = H + hoff[m];
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < ne; e += (int64_t)gridDim.x * blockDim.x) {
        // packed (i, j), j <= i
        int i = (int)((sqrt(8.0 * (double)e + 1.0) - 1.0) / 2.0);
        while (tri(i) > e) --i;
        while (tri(i + 1) <= e) ++i;
        const int j = (int)(e - tri(i));
        const int ci = i / k, cj = j / k, ii = i % k, jj = j % k;
        const int li = m + ii, lj = m + jj;
        const bool ai = ltab[5 * lmax1 + li] > 0.0, aj = ltab[5 * lmax1 + lj] > 0.0;
        double v;
        if (!ai || !aj) {
            v = i == j ? 1.0 : 0.0;
        } else {
            v = 0.0;
            if (ci == cj) v = ltab[li] * ltab[lj] * Gm[(int64_t)ci * tri(k) + tri(ii) + jj];
            if (li == lj) {
                const int row = (ci == 0 && cj == 0) ? 1 : (ci == 1 && cj == 1) ? 3 : 2;   // TT, EE, TE
                v += ltab[row * lmax1 + li] * isc;
            }
        }
        Hm[e] = v;
    }
}

// One CTA per m: Cholesky H = R R^T in place (packed lower, right-looking;
// column j of the trailing update staged in shared memory).  flag bit 1: a
// pivot was not positive.
__global__ void __launch_bounds__(AZF) k_az_chol(int lb, int ncb, const int64_t *__restrict__ hoff, double *H,
                                                 int *__restrict__ flag) {
    extern __shared__ __align__(16) unsigned char az_raw[];
    double *col = reinterpret_cast<double *>(az_raw);
    __shared__ double s_d;
    const int m = blockIdx.x;
    const int n = ncb * (lb + 1 - m);
    double *A = H + hoff[m];
    for (int j = 0; j < n; ++j) {
        if (threadIdx.x == 0) {
            const double d = A[tri(j) + j];
            if (!(d > 0.0)) atomicOr(flag, 1);
            s_d = d > 0.0 ? sqrt(d) : 1.0;
            A[tri(j) + j] = s_d;
        }
        __syncthreads();
        const double id = 1.0 / s_d;
        for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) {
            const double v = A[tri(i) + j] * id;
            A[tri(i) + j] = v;
            col[i] = v;
        }
        __syncthreads();
        // A_ik -= R_ij R_kj for j < k <= i: one warp per row, lanes over k
        // (unrolled, so that each lane has several independent loads in flight)
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        for (int i = j + 1 + warp; i < n; i += blockDim.x >> 5) {
            const double rij = col[i];
            double *row = A + tri(i);
#pragma unroll 4
            for (int kk = j + 1 + lane; kk <= i; kk += 32) row[kk] = fma(-rij, col[kk], row[kk]);
        }
        __syncthreads();
    }
}

// One CTA per m: R <- R^-1 in place (packed lower), column by column from
// the last: X_jj = 1 / R_jj, X_kj = -X_jj sum_{j < t <= k} X_kt R_tj for
// k > j (the trailing block already inverted; column j of R staged in
// shared memory, one warp per row k).
__global__ void __launch_bounds__(AZF) k_az_trinv(int lb, int ncb, const int64_t *__restrict__ hoff, double *H) {
    extern __shared__ __align__(16) unsigned char az_raw[];
    double *col = reinterpret_cast<double *>(az_raw);
    __shared__ double s_d;
    const int m = blockIdx.x;
    const int n = ncb * (lb + 1 - m);
    double *A = H + hoff[m];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int j = n - 1; j >= 0; --j) {
        if (threadIdx.x == 0) {
            s_d = 1.0 / A[tri(j) + j];
            A[tri(j) + j] = s_d;
        }
        for (int t = j + 1 + threadIdx.x; t < n; t += blockDim.x) col[t] = A[tri(t) + j];
        __syncthreads();
        const double d = s_d;
        for (int k = j + 1 + warp; k < n; k += blockDim.x >> 5) {
            const double *row = A + tri(k);
            double s = 0.0;
#pragma unroll 4
            for (int t = j + 1 + lane; t <= k; t += 32) s = fma(row[t], col[t], s);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) A[tri(k) + j] = -d * s;
        }
        __syncthreads();
    }
}

// M^-1 = X^T X (X = R^-1, packed lower) as full squares: grid.x the 32 x 32
// tiles (I >= J) of the largest block, grid.y = m; M_ij = sum_{k >= i} X_ki
// X_kj for i >= j, mirrored; FP64 into M64 and its FP32 copy into M32.
__global__ void __launch_bounds__(256) k_az_minv(int lb, int ncb, const int64_t *__restrict__ hoff,
                                                 const int64_t *__restrict__ moff, const double *__restrict__ H,
                                                 double *__restrict__ M64, float *__restrict__ M32) {
    __shared__ double sI[GT][GT + 1], sJ[GT][GT + 1];
    const int m = blockIdx.y;
    const int n = ncb * (lb + 1 - m);
    const int nt = (n + GT - 1) / GT;
    int t = blockIdx.x, I = 0;
    while (t > I) {
        t -= I + 1;
        ++I;
    }
    const int J = t;
    if (I >= nt) return;
    const double *X = H + hoff[m];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    double acc[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
    for (int k0 = I * GT; k0 < n; k0 += GT) {
        for (int e = threadIdx.x; e < GT * GT; e += 256) {
            const int kk = e / GT, c = e % GT;
            const int k = k0 + kk, i = I * GT + c, j = J * GT + c;
            sI[kk][c] = (k < n && i <= k) ? X[tri(k) + i] : 0.0;
            sJ[kk][c] = (k < n && j <= k) ? X[tri(k) + j] : 0.0;
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < GT; ++kk)
#pragma unroll
            for (int a = 0; a < 2; ++a)
#pragma unroll
                for (int b = 0; b < 2; ++b) acc[a][b] = fma(sI[kk][2 * ty + a], sJ[kk][2 * tx + b], acc[a][b]);
        __syncthreads();
    }
    double *Mm = M64 + moff[m];
    float *Fm = M32 + moff[m];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const int i = I * GT + 2 * ty + a, j = J * GT + 2 * tx + b;
            if (i >= n || j > i) continue;
            Mm[(int64_t)i * n + j] = acc[a][b];
            Mm[(int64_t)j * n + i] = acc[a][b];
            Fm[(int64_t)i * n + j] = (float)acc[a][b];
            Fm[(int64_t)j * n + i] = (float)acc[a][b];
        }
}

// The right-hand sides of every block as dense rows: Xg[xoff[m] + q n + j]
// = r at row j (component j / k, l = m + j % k) of right-hand side q = 2 b +
// part (m = 0: q = b, real parts); grid (m, q), threads over the rows.
template <typename T, typename TF>
__device__ __forceinline__ void az_gather_cta(int lb, int ncb, int lmax, int nb, const int64_t *__restrict__ xoff,
                                              const T *__restrict__ r, int64_t nalm, int64_t per,
                                              TF *__restrict__ Xg, const int m, const int q) {
    const int nparts = m ? 2 : 1;
    if (q >= nb * nparts) return;
    const int k = lb + 1 - m, n = ncb * k;
    const int b = q / nparts, part = q % nparts;
    const int64_t base = (int64_t)m * (2 * lmax + 1 - m) / 2 + m;
    TF *dst = Xg + xoff[m] + (int64_t)q * n;
    for (int c = 0; c < ncb; ++c) {
        const T *src = r + 2 * ((int64_t)b * per + (int64_t)c * nalm + base) + part;
        for (int ll = threadIdx.x; ll < k; ll += blockDim.x) dst[c * k + ll] = (TF)src[2 * (int64_t)ll];
    }
}
template <typename T, typename TF>
__global__ void k_az_gather(int lb, int ncb, int lmax, int nb, const int64_t *__restrict__ xoff,
                            const T *__restrict__ r, int64_t nalm, int64_t per, TF *__restrict__ Xg) {
    az_gather_cta<T, TF>(lb, ncb, lmax, nb, xoff, r, nalm, per, Xg, blockIdx.x, blockIdx.y);
}

// z <- M^-1 r on the block rows, as a tall-skinny product Z = M X per m
// (X: the staged right-hand sides, up to 16 per pass): grid.x = m, grid.y =
// tile of MR = 128 rows; 128 threads, thread t computes rows 4 (t / 4) ..
// + 3 for right-hand sides 4 (t % 4) .. + 3.  The columns run in steps of KT:
// the step's 128 x KT piece of M is loaded into registers (one row per
// thread, the next step's loads in flight during this step's products) and
// stored transposed in shared memory, so each k reads four rows and four
// right-hand sides with two 16-byte loads.  q = 2 b + part (part 0 real, 1
// imaginary; m = 0 real only).  slot[((b (lb + 1) + m) ntile + tile) 2 +
// part] = the change of sum w r z of system b's part on these rows (every
// slot of an existing tile is written by every application; the others stay
// zero).
constexpr int MR = 128, KT = 32;
template <typename T, typename TF>
__device__ __forceinline__ void az_mapply_cta(int lb, int ncb, int lmax, int nb, int ntile,
                                              const int64_t *__restrict__ moff, const TF *__restrict__ M,
                                              const int64_t *__restrict__ xoff, const TF *__restrict__ Xg,
                                              const T *__restrict__ r, T *__restrict__ z, int64_t nalm,
                                              int64_t per, double *__restrict__ slot, const int m,
                                              const int tile) {
    __shared__ __align__(16) TF As[KT][MR];
    __shared__ __align__(16) TF Xs[KT][16];
    __shared__ double sred[16][33];
    const int k = lb + 1 - m, n = ncb * k;
    const int i0 = tile * MR;
    if (i0 >= n) return;
    const TF *Mm = M + moff[m];
    const int nparts = m ? 2 : 1;
    const int nq = nb * nparts;
    const int64_t base = (int64_t)m * (2 * lmax + 1 - m) / 2 + m;   // alm index of l = m
    const double wm = m ? 2.0 : 1.0;
    const int tid = threadIdx.x, rg = tid >> 2, qg = tid & 3;
    // this thread's row of the staged piece of M
    const int ri = min(i0 + tid, n - 1);
    const TF *mrow = Mm + (int64_t)ri * n;
    const bool rlive = i0 + tid < n;
    for (int q0 = 0; q0 < nq; q0 += 16) {
        const int qn = min(16, nq - q0);
        TF acc[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[a][c] = TF(0);
        TF nxt[KT];
        auto load_piece = [&](int j0) {
#pragma unroll
            for (int kk = 0; kk < KT; ++kk) nxt[kk] = (rlive && j0 + kk < n) ? mrow[j0 + kk] : TF(0);
        };
        load_piece(0);
        for (int j0 = 0; j0 < n; j0 += KT) {
            __syncthreads();
#pragma unroll
            for (int kk = 0; kk < KT; ++kk) As[kk][tid] = nxt[kk];
            for (int e = tid; e < KT * 16; e += 128) {
                const int kk = e / 16, q = e % 16;
                Xs[kk][q] = (j0 + kk < n && q < qn) ? Xg[xoff[m] + (int64_t)(q0 + q) * n + j0 + kk] : TF(0);
            }
            __syncthreads();
            if (j0 + KT < n) load_piece(j0 + KT);
#pragma unroll
            for (int kk = 0; kk < KT; ++kk) {
                TF a4[4], x4[4];
#pragma unroll
                for (int a = 0; a < 4; ++a) a4[a] = As[kk][4 * rg + a];
#pragma unroll
                for (int c = 0; c < 4; ++c) x4[c] = Xs[kk][4 * qg + c];
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int c = 0; c < 4; ++c) acc[a][c] = fma(a4[a], x4[c], acc[a][c]);
            }
        }
        // write z and this thread's change of w r z per right-hand side
        double ds[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            const int i = i0 + 4 * rg + a;
            if (i >= n) continue;
            const int c = i / k, ll = i % k;
#pragma unroll
            for (int cq = 0; cq < 4; ++cq) {
                const int q = 4 * qg + cq;
                if (q >= qn) continue;
                const int gq = q0 + q, b = gq / nparts, part = gq % nparts;
                const int64_t el = 2 * ((int64_t)b * per + (int64_t)c * nalm + base + ll) + part;
                const double rv = (double)r[el], zo = (double)z[el];
                ds[cq] += wm * rv * ((double)acc[a][cq] - zo);
                z[el] = (T)acc[a][cq];
            }
        }
#pragma unroll
        for (int cq = 0; cq < 4; ++cq) sred[4 * qg + cq][rg] = ds[cq];
        __syncthreads();
        if (tid < qn) {
            const int gq = q0 + tid, b = gq / nparts, part = gq % nparts;
            double s = 0.0;
            for (int g = 0; g < 32; ++g) s += sred[tid][g];
            slot[(((int64_t)b * (lb + 1) + m) * ntile + tile) * 2 + part] = s;
        }
        __syncthreads();
    }
}
template <typename T, typename TF>
__global__ void __launch_bounds__(128) k_az_mapply(int lb, int ncb, int lmax, int nb, int ntile,
                                                   const int64_t *__restrict__ moff, const TF *__restrict__ M,
                                                   const int64_t *__restrict__ xoff, const TF *__restrict__ Xg,
                                                   const T *__restrict__ r, T *__restrict__ z, int64_t nalm,
                                                   int64_t per, double *__restrict__ slot) {
    az_mapply_cta<T, TF>(lb, ncb, lmax, nb, ntile, moff, M, xoff, Xg, r, z, nalm, per, slot, blockIdx.x,
                         blockIdx.y);
}

// per system b: the sum of its slots in a fixed order (each thread a fixed
// strided subset, then the threads in order), added to its first rz partial
__device__ __forceinline__ void az_addpart_cta(int nslot, const double *__restrict__ slot,
                                               double *__restrict__ part, int rb, const int b) {
    __shared__ double sm[256];
    const double *s = slot + (int64_t)b * nslot;
    double t = 0.0;
    for (int e = threadIdx.x; e < nslot; e += 256) t += s[e];
    sm[threadIdx.x] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        double u = 0.0;
        for (int w = 0; w < 256; ++w) u += sm[w];
        part[((int64_t)b * 2 + 0) * rb + 0] += u;
    }
}
__global__ void k_az_addpart(int nslot, const double *__restrict__ slot, double *__restrict__ part, int rb) {
    az_addpart_cta(nslot, slot, part, rb, blockIdx.x);
}

// Grouped application (chains of several geometries, FP32 iteration): the
// three kernels above over every group's blocks in one launch each; flat
// block i belongs to the group g with first[g] <= i < first[g + 1] and runs
// (m, y) = (i' % (lb + 1), i' / (lb + 1)), i' = i - first[g] (addpart: the
// system b = i').  Groups whose device flag is 0 are skipped.
struct AzGrp {
    int lb, ncb, lmax, nb, ntile;
    const int64_t *xoff, *moff;
    const float *M;
    float *Xg;
    const float *r;
    float *z;
    int64_t nalm, per;
    double *slot, *part;
    const int *active;
};
struct AzGroups {
    int ng;
    int first[SHTG_MAX_GROUPS + 1];
    AzGrp a[SHTG_MAX_GROUPS];
};
__device__ __forceinline__ int az_group(const AzGroups &G, const int i) {
    int g = 0;
    while (g + 1 < G.ng && i >= G.first[g + 1]) ++g;
    return g;
}
__global__ void k_az_gather_grp(const __grid_constant__ AzGroups G) {
    const int g = az_group(G, blockIdx.x);
    const AzGrp &a = G.a[g];
    if (*a.active == 0) return;
    const int li = blockIdx.x - G.first[g];
    az_gather_cta<float, float>(a.lb, a.ncb, a.lmax, a.nb, a.xoff, a.r, a.nalm, a.per, a.Xg, li % (a.lb + 1),
                                li / (a.lb + 1));
}
__global__ void __launch_bounds__(128) k_az_mapply_grp(const __grid_constant__ AzGroups G) {
    const int g = az_group(G, blockIdx.x);
    const AzGrp &a = G.a[g];
    if (*a.active == 0) return;
    const int li = blockIdx.x - G.first[g];
    az_mapply_cta<float, float>(a.lb, a.ncb, a.lmax, a.nb, a.ntile, a.moff, a.M, a.xoff, a.Xg, a.r, a.z, a.nalm,
                                a.per, a.slot, li % (a.lb + 1), li / (a.lb + 1));
}
__global__ void k_az_addpart_grp(const __grid_constant__ AzGroups G) {
    const int g = az_group(G, blockIdx.x);
    const AzGrp &a = G.a[g];
    if (*a.active == 0) return;
    az_addpart_cta((a.lb + 1) * a.ntile * 2, a.slot, a.part, SHTG_RED_BLOCKS, blockIdx.x - G.first[g]);
}
__global__ void k_az_cmp(const unsigned long long *__restrict__ a, const unsigned long long *__restrict__ b,
                         int64_t n, int *__restrict__ flag) {
    int d = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        d |= a[i] != b[i];
    if (__syncthreads_or(d) && threadIdx.x == 0) atomicOr(flag, 1);
}

template <typename P> int aalloc(Plan *p, P **ptr, size_t count) {
    const size_t bytes = sizeof(P) * std::max<size_t>(count, 1);
    const cudaError_t e = cudaMalloc((void **)ptr, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *ptr = nullptr;
        set_error("azimuthal block preconditioner: cannot allocate " + std::to_string(bytes) + " bytes");
        return SHTG_ERR_NOMEM;
    }
    p->device_bytes += (int64_t)bytes;
    p->az.bytes += (int64_t)bytes;
    return SHTG_OK;
}

unsigned az_blocks(int64_t n) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 4096)); }

int az_reserve(Plan *p, int lb, int ncb, cudaStream_t st) {
    AzBlk &q = p->az;
    if (q.lb == lb && q.ncb == ncb && q.H) return SHTG_OK;
    az_free(p);
    q.lb = lb;
    q.ncb = ncb;
    std::vector<int64_t> goff(lb + 1), hoff(lb + 1), moff(lb + 1), xoff(lb + 1);
    int64_t gs = 0, hs = 0, ms = 0, xs = 0;
    for (int m = 0; m <= lb; ++m) {
        const int64_t k = lb + 1 - m, n = ncb * k;
        goff[m] = gs;
        hoff[m] = hs;
        moff[m] = ms;
        xoff[m] = xs;
        gs += ncb * tri(k);
        hs += tri(n);
        ms += n * n;
        xs += n * 2 * (int64_t)p->max_batch;
    }
    q.ntile = (ncb * (lb + 1) + MR - 1) / MR;
    // profiles of a chunk of m: at most 2^25 values per profile (one block always fits)
    const int64_t ptot = (int64_t)(lb + 1) * (lb + 2) / 2 * p->npairs;
    q.pcap = std::min(ptot, std::max<int64_t>((int64_t)1 << 25, (int64_t)(lb + 1) * p->npairs));
    const int nch = ncb == 2 ? 2 : 1;
    SHTG_TRY(aalloc(p, &q.G, (size_t)gs));
    SHTG_TRY(aalloc(p, &q.H, (size_t)hs));
    SHTG_TRY(aalloc(p, &q.M64, (size_t)ms));
    SHTG_TRY(aalloc(p, &q.M32, (size_t)ms));
    SHTG_TRY(aalloc(p, &q.goff, (size_t)(lb + 1)));
    SHTG_TRY(aalloc(p, &q.hoff, (size_t)(lb + 1)));
    SHTG_TRY(aalloc(p, &q.moff, (size_t)(lb + 1)));
    SHTG_TRY(aalloc(p, &q.xoff, (size_t)(lb + 1)));
    SHTG_TRY(aalloc(p, &q.Xg, (size_t)xs));
    SHTG_TRY(aalloc(p, &q.poff, (size_t)(lb + 1)));
    SHTG_TRY(aalloc(p, &q.w, (size_t)4 * p->npairs));
    SHTG_TRY(aalloc(p, &q.pl, (size_t)q.pcap));
    SHTG_TRY(aalloc(p, &q.pw, (size_t)(ncb == 2 ? q.pcap : 1)));
    SHTG_TRY(aalloc(p, &q.px, (size_t)(ncb == 2 ? q.pcap : 1)));
    const size_t nslot = (size_t)p->max_batch * (lb + 1) * q.ntile * 2;
    SHTG_TRY(aalloc(p, &q.slot, nslot));
    SHTG_TRY(aalloc(p, &q.flag, 4));
    SHTG_TRY(aalloc(p, &q.ninv, (size_t)nch * p->npix));
    // ordered on the solve's stream (a chains group's stream is not ordered
    // with the legacy default stream), complete before the host vectors go
    SHTG_CUDA(cudaMemcpyAsync(q.goff, goff.data(), sizeof(int64_t) * (lb + 1), cudaMemcpyHostToDevice, st));
    SHTG_CUDA(cudaMemcpyAsync(q.hoff, hoff.data(), sizeof(int64_t) * (lb + 1), cudaMemcpyHostToDevice, st));
    SHTG_CUDA(cudaMemcpyAsync(q.moff, moff.data(), sizeof(int64_t) * (lb + 1), cudaMemcpyHostToDevice, st));
    SHTG_CUDA(cudaMemcpyAsync(q.xoff, xoff.data(), sizeof(int64_t) * (lb + 1), cudaMemcpyHostToDevice, st));
    SHTG_CUDA(cudaMemsetAsync(q.slot, 0, sizeof(double) * nslot, st));
    SHTG_CUDA(cudaStreamSynchronize(st));
    return SHTG_OK;
}

}  // namespace

void az_free(Plan *p) {
    AzBlk &q = p->az;
    void *bufs[] = {q.G, q.H, q.M64, q.M32, q.goff, q.hoff, q.moff, q.xoff, q.Xg, q.poff, q.w, q.pl, q.pw, q.px,
                    q.slot, q.flag, q.ninv};
    for (void *b : bufs)
        if (b) cudaFree(b);
    p->device_bytes -= q.bytes;
    q = AzBlk{};
}

int az_setup(Plan *p, int lb, int nc, double isc, cudaStream_t st) {
    const int L = p->lmax, L1 = L + 1, np = p->npairs;
    if (lb <= 0) lb = std::min(L, SHTG_AZ_LB_DEFAULT);
    if (lb > L) {
        set_error("azimuthal block preconditioner: block_lmax must be at most lmax");
        return SHTG_ERR_ARG;
    }
    const int ncb = nc == 3 ? 2 : 1;
    SHTG_TRY(az_reserve(p, lb, ncb, st));
    AzBlk &q = p->az;
    const int nch = ncb == 2 ? 2 : 1;
    const int64_t nin = (int64_t)nch * p->npix;
    // ---- Gram matrices, kept while N^-1 is bitwise unchanged
    bool rebuild = !q.gram_ok;
    if (!rebuild) {
        int h = 0;
        SHTG_CUDA(cudaMemsetAsync(q.flag, 0, sizeof(int), st));
        k_az_cmp<<<az_blocks(nin), 256, 0, st>>>(reinterpret_cast<const unsigned long long *>(p->d_ninv64),
                                                  reinterpret_cast<const unsigned long long *>(q.ninv), nin, q.flag);
        SHTG_CHECK_LAUNCH("k_az_cmp");
        SHTG_CUDA(cudaMemcpyAsync(&h, q.flag, sizeof(int), cudaMemcpyDeviceToHost, st));
        SHTG_CUDA(cudaStreamSynchronize(st));
        p->prof.launches += 1;
        rebuild = h != 0;
    }
    if (rebuild) {
        q.gram_ok = false;
        q.inv_ok = false;
        if (AZ_GRAM_SMEM > 48 * 1024) SHTG_CUDA(allow_max_smem(k_az_gram));
        k_az_weights<<<dim3(np, nch), AZT, 0, st>>>(p->d_ninv64, p->npix, p->d_ofs, p->d_nphi, p->nring, np, q.w);
        SHTG_CHECK_LAUNCH("k_az_weights");
        p->prof.launches += 1;
        int m0 = 0;
        std::vector<int64_t> poff;
        while (m0 <= lb) {
            int m1 = m0;
            int64_t used = 0;
            poff.clear();
            while (m1 <= lb) {
                const int64_t need = (int64_t)(lb + 1 - m1) * np;
                if (m1 > m0 && (used + need > q.pcap || m1 - m0 >= 65535)) break;
                poff.push_back(used);
                used += need;
                ++m1;
            }
            const int nm = m1 - m0;
            SHTG_CUDA(cudaMemcpyAsync(q.poff, poff.data(), sizeof(int64_t) * nm, cudaMemcpyHostToDevice, st));
            k_az_prof<<<dim3((np + 127) / 128, nm), 128, 0, st>>>(L, lb, np, m0, ncb == 2, q.poff, p->d_u64,
                                                                 p->d_rec64, p->d_ls64, p->d_st64, p->d_s2c64,
                                                                 p->d_ls2_64, p->d_st2_64, q.pl, q.pw, q.px);
            SHTG_CHECK_LAUNCH("k_az_prof");
            const int nt = (lb + 1 - m0 + GT - 1) / GT;
            k_az_gram<<<dim3(nt * (nt + 1) / 2, nm, ncb), 256, AZ_GRAM_SMEM, st>>>(lb, np, m0, q.poff, q.goff, q.pl,
                                                                                   q.pw, q.px, q.w, q.G);
            SHTG_CHECK_LAUNCH("k_az_gram");
            p->prof.launches += 2;
            // the offsets are read by this chunk's kernels before the next copy
            SHTG_CUDA(cudaStreamSynchronize(st));
            m0 = m1;
        }
        SHTG_CUDA(cudaMemcpyAsync(q.ninv, p->d_ninv64, sizeof(double) * nin, cudaMemcpyDeviceToDevice, st));
        q.gram_ok = true;
    }
    // ---- blocks, factors and inverses, kept while the per-l table and the scale are unchanged
    std::vector<double> tab(6 * (size_t)L1);
    SHTG_CUDA(cudaMemcpyAsync(tab.data(), p->d_ltab64, sizeof(double) * tab.size(), cudaMemcpyDeviceToHost, st));
    SHTG_CUDA(cudaStreamSynchronize(st));
    if (q.inv_ok && q.inv_isc == isc && q.inv_ltab == tab) return SHTG_OK;
    q.inv_ok = false;
    k_az_assemble<<<dim3(64, lb + 1), 256, 0, st>>>(lb, ncb, q.goff, q.hoff, q.G, p->d_ltab64, L1, isc, q.H);
    SHTG_CHECK_LAUNCH("k_az_assemble");
    SHTG_CUDA(cudaMemsetAsync(q.flag, 0, sizeof(int), st));
    const size_t csm = sizeof(double) * (size_t)ncb * (lb + 1);
    if (csm > 48 * 1024) {
        SHTG_CUDA(allow_max_smem(k_az_chol));
        SHTG_CUDA(allow_max_smem(k_az_trinv));
    }
    k_az_chol<<<lb + 1, AZF, csm, st>>>(lb, ncb, q.hoff, q.H, q.flag);
    SHTG_CHECK_LAUNCH("k_az_chol");
    k_az_trinv<<<lb + 1, AZF, csm, st>>>(lb, ncb, q.hoff, q.H);
    SHTG_CHECK_LAUNCH("k_az_trinv");
    const int nt = (ncb * (lb + 1) + GT - 1) / GT;
    k_az_minv<<<dim3(nt * (nt + 1) / 2, lb + 1), 256, 0, st>>>(lb, ncb, q.hoff, q.moff, q.H, q.M64, q.M32);
    SHTG_CHECK_LAUNCH("k_az_minv");
    p->prof.launches += 4;
    int h = 0;
    SHTG_CUDA(cudaMemcpyAsync(&h, q.flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    SHTG_CUDA(cudaStreamSynchronize(st));
    if (h) {
        set_error("azimuthal block preconditioner: a block is not positive definite");
        return SHTG_ERR_NOT_SPD;
    }
    q.inv_ltab = tab;
    q.inv_isc = isc;
    q.inv_ok = true;
    return SHTG_OK;
}

template <typename T, typename TF>
static int az_apply_t(Plan *p, const T *r, T *z, int nb, int64_t per, double *part, cudaStream_t st) {
    const AzBlk &q = p->az;
    const TF *M = sizeof(TF) == 4 ? reinterpret_cast<const TF *>(q.M32) : reinterpret_cast<const TF *>(q.M64);
    TF *Xg = reinterpret_cast<TF *>(q.Xg);
    k_az_gather<T, TF><<<dim3(q.lb + 1, 2 * nb), 256, 0, st>>>(q.lb, q.ncb, p->lmax, nb, q.xoff, r, p->nalm, per, Xg);
    k_az_mapply<T, TF><<<dim3(q.lb + 1, q.ntile), 128, 0, st>>>(q.lb, q.ncb, p->lmax, nb, q.ntile, q.moff, M, q.xoff,
                                                                Xg, r, z, p->nalm, per, q.slot);
    k_az_addpart<<<nb, 256, 0, st>>>((q.lb + 1) * q.ntile * 2, q.slot, part, SHTG_RED_BLOCKS);
    p->prof.launches += 3;
    SHTG_CHECK_LAUNCH("k_az_mapply");
    return SHTG_OK;
}

template <typename T>
int az_apply(Plan *p, const T *r, T *z, int nb, int64_t per, double *part, cudaStream_t st, bool fp64_factor) {
    if (sizeof(T) == 8 && fp64_factor)
        return az_apply_t<double, double>(p, reinterpret_cast<const double *>(r), reinterpret_cast<double *>(z), nb,
                                          per, part, st);
    return az_apply_t<T, float>(p, r, z, nb, per, part, st);
}

int az_apply_grp(int ng, Plan *const *ps, const float *const *r, float *const *z, const int *nb,
                 const int64_t *per, double *const *part, const int *const *active, cudaStream_t st) {
    if (ng < 1 || ng > SHTG_MAX_GROUPS) {
        set_error("grouped azimuthal blocks: 1 to " + std::to_string(SHTG_MAX_GROUPS) + " groups");
        return SHTG_ERR_ARG;
    }
    AzGroups G[3] = {};
    int64_t tot[3] = {0, 0, 0};
    for (int g = 0; g < ng; ++g) {
        const AzBlk &q = ps[g]->az;
        if (!q.inv_ok || !q.M32 || !active[g]) {
            set_error("grouped azimuthal blocks: group " + std::to_string(g) + " has no factored blocks");
            return SHTG_ERR_ARG;
        }
        AzGrp a;
        a.lb = q.lb;
        a.ncb = q.ncb;
        a.lmax = ps[g]->lmax;
        a.nb = nb[g];
        a.ntile = q.ntile;
        a.xoff = q.xoff;
        a.moff = q.moff;
        a.M = q.M32;
        a.Xg = reinterpret_cast<float *>(q.Xg);
        a.r = r[g];
        a.z = z[g];
        a.nalm = ps[g]->nalm;
        a.per = per[g];
        a.slot = q.slot;
        a.part = part[g];
        a.active = active[g];
        const int64_t n[3] = {(int64_t)(q.lb + 1) * 2 * nb[g], (int64_t)(q.lb + 1) * q.ntile, (int64_t)nb[g]};
        for (int k = 0; k < 3; ++k) {
            G[k].ng = ng;
            G[k].a[g] = a;
            G[k].first[g] = (int)tot[k];
            tot[k] += n[k];
        }
    }
    for (int k = 0; k < 3; ++k) {
        if (tot[k] > 0x7fffffff) {
            set_error("grouped azimuthal blocks: too many blocks");
            return SHTG_ERR_ARG;
        }
        G[k].first[ng] = (int)tot[k];
    }
    k_az_gather_grp<<<(unsigned)tot[0], 256, 0, st>>>(G[0]);
    k_az_mapply_grp<<<(unsigned)tot[1], 128, 0, st>>>(G[1]);
    k_az_addpart_grp<<<(unsigned)tot[2], 256, 0, st>>>(G[2]);
    ps[0]->prof.launches += 3;
    SHTG_CHECK_LAUNCH("k_az_mapply_grp");
    return SHTG_OK;
}

template int az_apply<float>(Plan *, const float *, float *, int, int64_t, double *, cudaStream_t, bool);
template int az_apply<double>(Plan *, const double *, double *, int, int64_t, double *, cudaStream_t, bool);

}  // namespace shtg

// Exact per-m dense solve of the constrained-realization system for
// azimuthally symmetric noise (App. A).
//
// When N^-1 is constant along every ring and every ring has nphi >= 2 lmax + 1
// pixels, the phi sum of e^{-i (m - m') phi} over a ring vanishes unless
// m = m', so A = S^-1 + B Y^T N^-1 Y B is block-diagonal in m (App. A, Eq.
// N_lml'm'_step in its discrete form):
//
//   A^(m)_{l l'} = delta_{l l'} / C_l + b_l b_l' sum_r nphi_r w_r lambda_lm(theta_r) lambda_l'm(theta_r).
//
// Over a north / south ring pair lambda_lm(pi - theta) = (-1)^(l+m)
// lambda_lm(theta) (App. A), so the ring sum is a sum over pairs with the
// weight nphi (w_N + w_S) for l + l' even and nphi (w_N - w_S) for l + l'
// odd.  Each block is built in FP64 (the recurrence values of one m for all
// pairs, then a parity-weighted Gram product), factored by Cholesky and
// solved for the real and imaginary parts of every realization's right-hand
// side.  Temperature only.  The m values are processed in chunks whose
// blocks and recurrence values fit the plan's block workspace.
#include <algorithm>

#include "common.cuh"

namespace shtg {
namespace {

constexpr int BT = 32;   // Gram tile (l x l') and pair chunk

// Per ring pair: sum and difference of nphi w over its rings, and a flag if
// N^-1 varies along a ring (then the operator is not block-diagonal).
__global__ void k_blk_weights(const double *__restrict__ ninv, const int64_t *__restrict__ ofs,
                              const int *__restrict__ nphi, int nring, int npairs, double *__restrict__ wsum,
                              double *__restrict__ wdiff, int *__restrict__ flag) {
    const int pr = blockIdx.x;
    if (pr >= npairs) return;
    const int rn = pr, rs = nring - 1 - pr;
    const double wn = ninv[ofs[rn]];
    const double ws = rs != rn ? ninv[ofs[rs]] : 0.0;
    bool bad = false;
    for (int j = threadIdx.x; j < nphi[rn]; j += blockDim.x) bad |= ninv[ofs[rn] + j] != wn;
    if (rs != rn)
        for (int j = threadIdx.x; j < nphi[rs]; j += blockDim.x) bad |= ninv[ofs[rs] + j] != ws;
    if (bad) atomicOr(flag, 1);
    if (threadIdx.x == 0) {
        const double n = (double)nphi[rn];
        wsum[pr] = n * (wn + ws);
        wdiff[pr] = n * (wn - ws);
    }
}

// lambda_lm(theta_p) for the m values [m0, m0 + nm) of a chunk and all pairs:
// row l - m of block m at lam[loff[m - m0] + (l - m) npairs + p].  FP64
// recurrence lambda_l = a_lm (1 - u) lambda_{l-1} + b_lm lambda_{l-2} from
// zero, with the pair's FP64 start state injected at its first significant l.
__global__ void k_blk_lambda(int lmax, int npairs, int m0, const int64_t *__restrict__ loff,
                             const double *__restrict__ u64, const double2 *__restrict__ rec,
                             const int *__restrict__ ls, const double2 *__restrict__ st,
                             double *__restrict__ lam) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    const int m = m0 + blockIdx.y;
    if (p >= npairs) return;
    const int64_t base = (int64_t)m * (2 * lmax + 1 - m) / 2;
    const int64_t o = (int64_t)m * npairs + p;
    const int l0 = ls[o];
    const double2 s = st[o];
    const double u = u64[p];
    double a1 = 0.0, a2 = 0.0;
    double *out = lam + loff[blockIdx.y] + p;
    for (int l = m; l <= lmax; ++l) {
        const double2 cf = rec[base + l];
        // a (1 - u) lambda_{l-1} + b lambda_{l-2}, rounded as in the transforms
        const double t = cf.x * a1;
        const double v = fma(t, -u, fma(cf.y, a2, t));
        a2 = a1;
        a1 = v;
        if (l == l0) {
            a2 = s.x;
            a1 = s.y;
        }
        out[(int64_t)(l - m) * npairs] = a1;
    }
}

// Lower-triangle 32 x 32 tiles of the blocks of a chunk: grid.x enumerates
// the tiles (I >= J) of the largest block, grid.y the m of the chunk; each
// of the 256 threads owns 2 x 2 entries.  A_{l l'} = delta / C_l +
// b_l b_l' sum_p lambda_l lambda_l' (l + l' even ? wsum : wdiff); held
// multipoles (inactive C_l) give identity rows and columns.  isc: 1 / (the
// realizations' common C_l scale).
__global__ void __launch_bounds__(256) k_blk_gram(int lmax, int npairs, int m0, const int64_t *__restrict__ loff,
                                                  const int64_t *__restrict__ aoff, const double *__restrict__ lam,
                                                  const double *__restrict__ wsum, const double *__restrict__ wdiff,
                                                  const double *__restrict__ ltab, double isc,
                                                  double *__restrict__ A) {
    __shared__ double sI[BT][BT + 1], sJ[BT][BT + 1], sw[2][BT];
    const int m = m0 + blockIdx.y;
    const int n = lmax + 1 - m;
    const int nt = (n + BT - 1) / BT;
    // tile index -> (I, J), I >= J, row-major over the lower triangle
    int t = blockIdx.x, I = 0;
    while (t > I) {
        t -= I + 1;
        ++I;
    }
    const int J = t;
    if (I >= nt) return;
    const double *lm = lam + loff[blockIdx.y];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int i0 = I * BT + 2 * ty, j0 = J * BT + 2 * tx;
    double acc[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
    for (int p0 = 0; p0 < npairs; p0 += BT) {
        for (int e = threadIdx.x; e < BT * BT; e += 256) {
            const int r = e / BT, c = e % BT;   // r: l within the tile, c: pair within the chunk
            const int p = p0 + c;
            const int li = I * BT + r, lj = J * BT + r;
            sI[r][c] = (p < npairs && li < n) ? lm[(int64_t)li * npairs + p] : 0.0;
            sJ[r][c] = (p < npairs && lj < n) ? lm[(int64_t)lj * npairs + p] : 0.0;
        }
        for (int e = threadIdx.x; e < BT; e += 256) {
            const int p = p0 + e;
            sw[0][e] = p < npairs ? wsum[p] : 0.0;
            sw[1][e] = p < npairs ? wdiff[p] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int b = 0; b < 2; ++b) {
                const int par = (2 * ty + a + 2 * tx + b) & 1;   // parity of l + l' (same as of the tile offsets)
                double s = 0.0;
#pragma unroll 8
                for (int c = 0; c < BT; ++c) s = fma(sI[2 * ty + a][c] * sJ[2 * tx + b][c], sw[par][c], s);
                acc[a][b] += s;
            }
        __syncthreads();
    }
    const int L1 = lmax + 1;
    double *Am = A + aoff[blockIdx.y];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const int i = i0 + a, j = j0 + b;
            if (i >= n || j >= n || j > i) continue;
            const int li = m + i, lj = m + j;
            // active multipoles: the inverse square root's TT entry is positive
            const bool ai = ltab[5 * L1 + li] > 0.0, aj = ltab[5 * L1 + lj] > 0.0;
            double v;
            if (!ai || !aj) v = (i == j) ? 1.0 : 0.0;
            else v = ltab[li] * ltab[lj] * acc[a][b] + (i == j ? ltab[L1 + li] * isc : 0.0);
            Am[(int64_t)i * n + j] = v;
        }
}

// One CTA per m of the chunk: Cholesky factorization A = R R^T in place
// (lower triangle, right-looking, one column at a time) and the solve of
// R R^T x = b for the real and the imaginary part of every realization's
// right-hand side (B, X: [nb][nalm] complex, block m at alm index base_m + l).
__global__ void __launch_bounds__(256) k_blk_chol(int lmax, int m0, const int64_t *__restrict__ aoff, double *A,
                                                  const double2 *__restrict__ B, double2 *__restrict__ X, int nb,
                                                  int64_t nalm, int *__restrict__ flag) {
    __shared__ double s_d;
    const int m = m0 + blockIdx.x;
    const int n = lmax + 1 - m;
    double *Am = A + aoff[blockIdx.x];
    const int64_t base = (int64_t)m * (2 * lmax + 1 - m) / 2 + m;   // alm index of l = m
    for (int j = 0; j < n; ++j) {
        if (threadIdx.x == 0) {
            const double d = Am[(int64_t)j * n + j];
            if (!(d > 0.0)) atomicOr(flag, 2);
            s_d = d > 0.0 ? sqrt(d) : 1.0;
            Am[(int64_t)j * n + j] = s_d;
        }
        __syncthreads();
        const double d = s_d;
        for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) Am[(int64_t)i * n + j] /= d;
        __syncthreads();
        // trailing update of the lower triangle, A_ik -= R_ij R_kj for
        // j < k <= i: one warp per row i, its lanes over consecutive k
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        for (int i = j + 1 + warp; i < n; i += blockDim.x >> 5) {
            const double rij = Am[(int64_t)i * n + j];
            for (int k = j + 1 + lane; k <= i; k += 32) Am[(int64_t)i * n + k] -= rij * Am[(int64_t)k * n + j];
        }
        __syncthreads();
    }
    // right-hand sides: column q = 2 b + (0: real, 1: imaginary part)
    const int nrhs = 2 * nb;
    auto xr = [&](int i, int q) -> double & {
        double2 *x = X + (int64_t)(q >> 1) * nalm + base + i;
        return (q & 1) ? x->y : x->x;
    };
    for (int e = threadIdx.x; e < n * nrhs; e += blockDim.x) {
        const int i = e / nrhs, q = e % nrhs;
        const double2 b = B[(int64_t)(q >> 1) * nalm + base + i];
        xr(i, q) = (q & 1) ? (m == 0 ? 0.0 : b.y) : b.x;
    }
    __syncthreads();
    // forward: R y = b
    for (int j = 0; j < n; ++j) {
        const double d = Am[(int64_t)j * n + j];
        for (int q = threadIdx.x; q < nrhs; q += blockDim.x) xr(j, q) /= d;
        __syncthreads();
        for (int e = threadIdx.x; e < (n - j - 1) * nrhs; e += blockDim.x) {
            const int i = j + 1 + e / nrhs, q = e % nrhs;
            xr(i, q) -= Am[(int64_t)i * n + j] * xr(j, q);
        }
        __syncthreads();
    }
    // backward: R^T x = y
    for (int j = n - 1; j >= 0; --j) {
        const double d = Am[(int64_t)j * n + j];
        for (int q = threadIdx.x; q < nrhs; q += blockDim.x) xr(j, q) /= d;
        __syncthreads();
        for (int e = threadIdx.x; e < j * nrhs; e += blockDim.x) {
            const int i = e / nrhs, q = e % nrhs;
            xr(i, q) -= Am[(int64_t)j * n + i] * xr(j, q);
        }
        __syncthreads();
    }
}

}  // namespace

int block_workspace(Plan *p) {
    const int L = p->lmax;
    int64_t nblk = 0, nlam = 0;
    for (int m = 0; m <= L; ++m) {
        const int64_t n = L + 1 - m;
        nblk += n * n;
        nlam += n * p->npairs;
    }
    // chunks of m bounded by 2^26 block entries and 2^25 recurrence values
    p->blk_cap = std::min<int64_t>(nblk, (int64_t)1 << 26);
    p->lam_cap = std::min<int64_t>(nlam, (int64_t)1 << 25);
    const int64_t n0 = L + 1;
    p->blk_cap = std::max(p->blk_cap, n0 * n0);
    p->lam_cap = std::max(p->lam_cap, n0 * p->npairs);
    return SHTG_OK;
}

int block_solve(Plan *p, const double2 *B, double2 *X, int nb, double isc, cudaStream_t st) {
    const int L = p->lmax, np = p->npairs;
    if (!p->d_blk) {
        set_error("SHTG_CG_BLOCK needs a plan created with SHTG_BLOCK_SOLVER");
        return SHTG_ERR_ARG;
    }
    SHTG_CUDA(cudaMemsetAsync(p->d_blkflag, 0, sizeof(int), st));
    double *wsum = p->d_blkw, *wdiff = p->d_blkw + np;
    k_blk_weights<<<np, 256, 0, st>>>(p->d_ninv64, p->d_ofs, p->d_nphi, p->nring, np, wsum, wdiff, p->d_blkflag);
    SHTG_CHECK_LAUNCH("k_blk_weights");
    int h = 0;
    SHTG_CUDA(cudaMemcpyAsync(&h, p->d_blkflag, sizeof(int), cudaMemcpyDeviceToHost, st));
    SHTG_CUDA(cudaStreamSynchronize(st));
    if (h) {
        set_error("SHTG_CG_BLOCK: N^-1 varies along a ring (the operator is not block-diagonal in m)");
        return SHTG_ERR_ARG;
    }
    p->prof.launches += 1;
    std::vector<int64_t> offs;
    int m0 = 0;
    while (m0 <= L) {
        // the chunk [m0, m1): blocks and recurrence values within the workspace
        int64_t ab = 0, al = 0;
        int m1 = m0;
        offs.clear();
        std::vector<int64_t> loff, aoff;
        while (m1 <= L) {
            const int64_t n = L + 1 - m1;
            if (m1 > m0 && (ab + n * n > p->blk_cap || al + n * np > p->lam_cap || m1 - m0 >= 65535)) break;
            aoff.push_back(ab);
            loff.push_back(al);
            ab += n * n;
            al += n * np;
            ++m1;
        }
        const int nm = m1 - m0;
        SHTG_CUDA(cudaMemcpyAsync(p->d_blkoff, aoff.data(), sizeof(int64_t) * nm, cudaMemcpyHostToDevice, st));
        SHTG_CUDA(cudaMemcpyAsync(p->d_blkoff + nm, loff.data(), sizeof(int64_t) * nm, cudaMemcpyHostToDevice, st));
        k_blk_lambda<<<dim3((np + 127) / 128, nm), 128, 0, st>>>(L, np, m0, p->d_blkoff + nm, p->d_u64, p->d_rec64,
                                                                p->d_ls64, p->d_st64, p->d_blklam);
        SHTG_CHECK_LAUNCH("k_blk_lambda");
        const int nt = (L + 1 - m0 + BT - 1) / BT;
        k_blk_gram<<<dim3(nt * (nt + 1) / 2, nm), 256, 0, st>>>(L, np, m0, p->d_blkoff + nm, p->d_blkoff,
                                                                p->d_blklam, wsum, wdiff, p->d_ltab64, isc, p->d_blk);
        SHTG_CHECK_LAUNCH("k_blk_gram");
        k_blk_chol<<<nm, 256, 0, st>>>(L, m0, p->d_blkoff, p->d_blk, B, X, nb, p->nalm, p->d_blkflag);
        SHTG_CHECK_LAUNCH("k_blk_chol");
        p->prof.launches += 3;
        // the offsets are read by the kernels of this chunk before the next copy
        SHTG_CUDA(cudaStreamSynchronize(st));
        m0 = m1;
    }
    SHTG_CUDA(cudaMemcpyAsync(&h, p->d_blkflag, sizeof(int), cudaMemcpyDeviceToHost, st));
    SHTG_CUDA(cudaStreamSynchronize(st));
    if (h & 2) {
        set_error("SHTG_CG_BLOCK: a block is not positive definite");
        return SHTG_ERR_NOT_SPD;
    }
    return SHTG_OK;
}

}  // namespace shtg

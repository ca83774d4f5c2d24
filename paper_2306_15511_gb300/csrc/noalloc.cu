// Allocation-free transpose transform Y^T (HEALPix, FP64, spin 0) for callers
// that cannot allocate device memory: code that runs under a device-memory
// budget owned by another framework, or that may not call cudaMalloc because
// it can synchronize the device and stall concurrent work.  Those callers
// cannot create a plan (plan creation allocates its tables and workspace), so
// this entry point needs no plan: the ring geometry and the Legendre
// recurrence are computed on the fly, and the only intermediate (the per-ring
// Fourier sums G_r(m)) lives in a fixed static device buffer.
//
// The buffer is shared by every call on a device and keeps the last call's
// contents; each call overwrites every element it reads, and the output is
// zeroed before it is accumulated.  Calls whose kernels overlap on the GPU
// (different streams, or different host threads) race on the buffer.
//
// The buffer's device address is looked up once per device, on the first
// call; under lazy module loading that lookup also loads this module onto the
// device and so reserves the 16 MiB.  A cudaDeviceReset invalidates the cached
// address, so the entry point is not for use on a device after a reset.  The
// transpose accumulates each c_lm from all ring pairs with FP64 atomic
// additions; their order is not fixed, so repeated calls agree only to
// rounding.
#include <mutex>

#include "common.cuh"

namespace shtg {
namespace {

constexpr size_t NOALLOC_SCRATCH_BYTES = size_t(16) << 20;   // 16 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

constexpr int NOALLOC_MAX_DEVICES = 64;
std::mutex g_noalloc_mu;
void *g_noalloc_addr[NOALLOC_MAX_DEVICES] = {};

// device address of the static buffer for the current device (host code may
// not use the symbol itself: on the host it only names a stand-in object)
int scratch_address(void **out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice", __FILE__, __LINE__);
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) {
        set_error("device index out of range for the static scratch table");
        return SHTG_ERR_ARG;
    }
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress", __FILE__, __LINE__);
        g_noalloc_addr[dev] = p;
    }
    *out = g_noalloc_addr[dev];
    return SHTG_OK;
}

// HEALPix ring r (0-based, north to south): 1 - cos(theta) of its northern
// mirror, pixels, first-pixel offset and the half-pixel shift flag.
__device__ void hp_ring(int N, int r, double &u, int &nphi, long long &ofs, int &shift) {
    const int i = r + 1;
    const int ii = (i <= 2 * N) ? i : 4 * N - i;
    if (ii < N) {
        u = (double)ii * ii / (3.0 * N * N);
        nphi = 4 * ii;
        shift = 1;
    } else {
        u = (2.0 * ii - N) / (3.0 * N);
        nphi = 4 * N;
        shift = ((ii - N) % 2 == 0) ? 1 : 0;
    }
    if (i < N) {
        ofs = 2LL * i * (i - 1);
    } else if (i <= 3 * N) {
        ofs = 2LL * N * (N - 1) + 4LL * N * (i - N);
    } else {
        const long long npix = 12LL * N * N;
        const int k = 4 * N - i;   // rings counted from the south pole
        ofs = npix - 2LL * k * (k + 1);
    }
}

__global__ void k_na_zero(double *a, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        a[i] = 0.0;
}

// G_r(m) = sum_j map_j e^{-i m (phi0 + 2 pi j / n)}, phi0 = shift pi / n
__global__ void k_na_ring_dft(int N, int lmax, const double *__restrict__ map, double2 *G) {
    const int r = blockIdx.y;
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m > lmax) return;
    double u;
    int n, sh;
    long long ofs;
    hp_ring(N, r, u, n, ofs, sh);
    double gr = 0.0, gi = 0.0;
    for (int j = 0; j < n; ++j) {
        const long long q = ((long long)m * (sh + 2LL * j)) % (2LL * n);
        double s, c;
        sincospi((double)q / (double)n, &s, &c);
        const double v = map[ofs + j];
        gr += v * c;
        gi -= v * s;
    }
    G[(long long)r * (lmax + 1) + m] = make_double2(gr, gi);
}

// c_lm += sum over the ring pair of lambda_lm (G_N + (-1)^(l+m) G_S); one
// thread per (m, ring pair), FP64 recurrence with exponent rescaling
__global__ void k_na_legendre(int N, int lmax, const double2 *__restrict__ G, double *alm) {
    const int m = blockIdx.y;
    const int pr = blockIdx.x * blockDim.x + threadIdx.x;
    const int npairs = 2 * N;
    if (pr >= npairs || m > lmax) return;
    const int nring = 4 * N - 1;
    const int rn = pr, rs = nring - 1 - pr;
    double u;
    int n, sh;
    long long ofs;
    hp_ring(N, rn, u, n, ofs, sh);
    const double x = 1.0 - u, s = sqrt(u * (2.0 - u));
    const double2 gn = G[(long long)rn * (lmax + 1) + m];
    const double2 gs = (rs != rn) ? G[(long long)rs * (lmax + 1) + m] : make_double2(0.0, 0.0);
    double v = 0.28209479177387814347403972578;   // lambda_00 = 1/sqrt(4 pi)
    int k = 0;                                     // value = v * 2^(512 k)
    for (int j = 1; j <= m; ++j) {
        v *= -sqrt((2.0 * j + 1.0) / (2.0 * j)) * s;
        if (v != 0.0 && fabs(v) < 0x1p-256) {
            v *= 0x1p512;
            k -= 1;
        }
    }
    double prev = 0.0;
    const long long base = (long long)m * (2 * lmax + 1 - m) / 2;
    for (int l = m; l <= lmax; ++l) {
        if (l > m) {
            const double dl = l, dm = m;
            const double a = sqrt((4.0 * dl * dl - 1.0) / (dl * dl - dm * dm));
            const double b = (l == m + 1) ? 0.0
                : sqrt(((dl - 1.0) * (dl - 1.0) - dm * dm) / (4.0 * (dl - 1.0) * (dl - 1.0) - 1.0));
            const double nv = a * (x * v - b * prev);
            prev = v;
            v = nv;
            if (fabs(v) > 0x1p256) {
                v *= 0x1p-512;
                prev *= 0x1p-512;
                k += 1;
            }
        }
        if (k == 0) {   // below that the terms are under 2^-256 and negligible
            const double sg = ((l + m) & 1) ? -1.0 : 1.0;
            const double re = v * (gn.x + sg * gs.x);
            const double im = (m == 0) ? 0.0 : v * (gn.y + sg * gs.y);
            atomicAdd(&alm[2 * (base + l)], re);
            atomicAdd(&alm[2 * (base + l) + 1], im);
        }
    }
}

}  // namespace
}  // namespace shtg

using namespace shtg;

extern "C" int shtg_alm2map_adjoint_noalloc(int nside, int lmax, const double *map, double *alm,
                                            void *stream) {
    if (nside < 1 || nside > 8192 || lmax < 0 || lmax > 4 * nside || !map || !alm) {
        set_error("noalloc adjoint: need 1 <= nside <= 8192, 0 <= lmax <= 4 nside and non-null buffers");
        return SHTG_ERR_ARG;
    }
    const long long nring = 4LL * nside - 1;
    const unsigned long long need = (unsigned long long)nring * (lmax + 1) * sizeof(double2);
    if (need > NOALLOC_SCRATCH_BYTES) {
        set_error("noalloc adjoint: needs " + std::to_string(need) + " bytes of scratch (n_ring x "
                  "(lmax+1) x 16); the static buffer holds " +
                  std::to_string((unsigned long long)NOALLOC_SCRATCH_BYTES) + " bytes");
        return SHTG_ERR_ARG;
    }
    void *scratch = nullptr;
    SHTG_TRY(scratch_address(&scratch));
    double2 *G = reinterpret_cast<double2 *>(scratch);
    cudaStream_t st = (cudaStream_t)stream;
    const long long nalm2 = 2LL * (lmax + 1) * (lmax + 2) / 2;
    k_na_zero<<<256, 256, 0, st>>>(alm, nalm2);
    SHTG_CHECK_LAUNCH("k_na_zero");
    k_na_ring_dft<<<dim3((lmax + 128) / 128, (unsigned)nring), 128, 0, st>>>(nside, lmax, map, G);
    SHTG_CHECK_LAUNCH("k_na_ring_dft");
    k_na_legendre<<<dim3((2 * nside + 127) / 128, lmax + 1), 128, 0, st>>>(nside, lmax, G, alm);
    SHTG_CHECK_LAUNCH("k_na_legendre");
    return SHTG_OK;
}

/*
 * FP64 CPU oracle for the constrained-realization sampler of Eskilt et al.
 * (arXiv 2306.15511).  TEST INFRASTRUCTURE ONLY: the test suite, the smoke
 * check and the CPU-baseline leg of the benchmark may call it; the product
 * path never does.  It shares no code with the CUDA library.
 *
 * What it computes, written out from the definitions:
 *   - HEALPix RING geometry (Gorski et al. 2005) and Gauss-Legendre rings.
 *   - lambda_lm(theta), the theta part of Y_lm = lambda_lm e^{i m phi},
 *     orthonormal with the Condon-Shortley phase; App. A defines
 *     P~_lm = Delta_lm P_lm(cos theta) with the (-1)^m factor.
 *   - spin-2 harmonics from the spin-raising operator applied twice to Y_lm
 *     (2Y_lm ~ edth^2 Y_lm), expressed through lambda_lm and lambda_{l-1,m}.
 *   - Y (alm -> map) as a direct sum over l followed by a direct DFT over m
 *     on every ring; Y^T as its literal transpose.
 *
 * Layouts: alm complex interleaved (re, im), m-major,
 * index(l, m) = m(2L+1-m)/2 + l; maps real in ring order with per-ring
 * offsets.  The imaginary part of a_l0 is ignored (treated as zero).
 *
 * The order of operations follows the definitions: no blocking, no fusion.
 * OpenMP only distributes independent rings or independent m values.
 */
#include <math.h>
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_PI 3.14159265358979323846264338327950288

int orc_abi_version(void) { return 4; }

/* Worker threads of the OpenMP loops below (n > 0 sets them; every call
 * returns the count in force).  Used only to time the oracle on one core. */
int orc_set_threads(int n)
{
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
}

/* ------------------------------------------------------------------------- */
/* geometry                                                                  */
/* ------------------------------------------------------------------------- */
int orc_healpix_nring(int nside) { return 4 * nside - 1; }

/* Rings i = 1 .. 4N-1 from north to south.  Polar rings (i < N):
 * z = 1 - i^2/(3N^2), 4i pixels, first pixel at phi0 = pi/(4i).
 * Equatorial rings (N <= i <= 3N): z = 4/3 - 2i/(3N), 4N pixels,
 * phi0 = pi/(4N) when i - N is even, else 0.  The south cap mirrors the
 * north one.  sin(theta) is computed from 1 - z without cancellation. */
void orc_healpix_geom(int nside, double *cth, double *sth, int64_t *nphi,
                      double *phi0, int64_t *ofs)
{
    const int n = nside;
    int64_t off = 0;
    for (int i = 1; i <= 4 * n - 1; ++i) {
        const int ii = (i <= 2 * n) ? i : 4 * n - i;
        double z, s, shift;
        int64_t np_;
        if (ii < n) {
            const double t = (double)ii * ii / (3.0 * n * n); /* 1 - z */
            z = 1.0 - t;
            s = sqrt(t * (2.0 - t));
            np_ = 4 * (int64_t)ii;
            shift = 1.0;
        } else {
            z = 4.0 / 3.0 - 2.0 * ii / (3.0 * n);
            s = sqrt((1.0 - z) * (1.0 + z));
            np_ = 4 * (int64_t)n;
            shift = ((ii - n) % 2 == 0) ? 1.0 : 0.0;
        }
        if (i > 2 * n) z = -z;
        cth[i - 1] = z;
        sth[i - 1] = s;
        nphi[i - 1] = np_;
        phi0[i - 1] = shift * ORC_PI / (double)np_;
        ofs[i - 1] = off;
        off += np_;
    }
}

/* Gauss-Legendre nodes x_k (descending, i.e. north to south) and weights
 * w_k = 2 / ((1 - x^2) P_n'(x)^2), by Newton iteration on P_n. */
void orc_gl_geom(int nring, double *cth, double *sth, double *wgt)
{
    const int n = nring;
    for (int k = 0; k < n; ++k) {
        double x = cos(ORC_PI * (k + 0.75) / (n + 0.5));
        double dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = x;
            for (int j = 2; j <= n; ++j) {
                const double p2 = ((2.0 * j - 1.0) * x * p1 - (j - 1.0) * p0) / j;
                p0 = p1;
                p1 = p2;
            }
            if (n == 1) { p1 = x; p0 = 1.0; }
            dp = n * (x * p1 - p0) / (x * x - 1.0);
            const double dx = p1 / dp;
            x -= dx;
            if (fabs(dx) < 1e-16) break;
        }
        {
            double p0 = 1.0, p1 = x;
            for (int j = 2; j <= n; ++j) {
                const double p2 = ((2.0 * j - 1.0) * x * p1 - (j - 1.0) * p0) / j;
                p0 = p1;
                p1 = p2;
            }
            if (n == 1) { p1 = x; p0 = 1.0; }
            dp = n * (x * p1 - p0) / (x * x - 1.0);
        }
        cth[k] = x;
        sth[k] = sqrt((1.0 - x) * (1.0 + x));
        wgt[k] = 2.0 / ((1.0 - x * x) * dp * dp);
    }
}

/* ------------------------------------------------------------------------- */
/* associated Legendre functions                                             */
/* ------------------------------------------------------------------------- */
/* Recurrence coefficients for fixed m, l = m+2 .. lmax:
 *   lambda_l = alpha_l (x lambda_{l-1} - beta_l lambda_{l-2}),
 *   alpha_l = sqrt((4l^2-1)/(l^2-m^2)), beta_l = sqrt(((l-1)^2-m^2)/(4(l-1)^2-1)). */
static void rec_coef(int lmax, int m, double *alpha, double *beta)
{
    for (int l = m + 2; l <= lmax; ++l) {
        const double dl = l, dm = m;
        alpha[l] = sqrt((4.0 * dl * dl - 1.0) / (dl * dl - dm * dm));
        beta[l] = sqrt(((dl - 1.0) * (dl - 1.0) - dm * dm) / (4.0 * (dl - 1.0) * (dl - 1.0) - 1.0));
    }
}

/* lambda_lm(theta) for l = m .. lmax into out[l - m].
 * Sectoral start: lambda_00 = 1/sqrt(4 pi),
 *   lambda_kk = -sqrt((2k+1)/(2k)) sin(theta) lambda_{k-1,k-1},
 * then lambda_{m+1,m} = sqrt(2m+3) cos(theta) lambda_mm and the three-term
 * recurrence.  Values are carried as v * 2^e so that the tiny sectoral values
 * near the poles and at large m neither underflow nor lose the l-growth that
 * follows; the stored result is ldexp(v, e) (0 when below the FP64 range). */
static void lambda_row_c(int lmax, int m, double x, double s, const double *alpha,
                         const double *beta, double *out)
{
    double v = 1.0 / sqrt(4.0 * ORC_PI);
    int e = 0;
    for (int k = 1; k <= m; ++k) {
        v *= -sqrt((2.0 * k + 1.0) / (2.0 * k)) * s;
        if (v != 0.0 && fabs(v) < 0x1p-200) {
            v *= 0x1p200;
            e -= 200;
        }
    }
    out[0] = ldexp(v, e);
    if (lmax == m) return;
    double p2 = v, p1 = sqrt(2.0 * m + 3.0) * x * v;
    out[1] = ldexp(p1, e);
    for (int l = m + 2; l <= lmax; ++l) {
        const double pn = alpha[l] * (x * p1 - beta[l] * p2);
        p2 = p1;
        p1 = pn;
        if (fabs(p1) > 0x1p200) {
            p1 *= 0x1p-200;
            p2 *= 0x1p-200;
            e += 200;
        }
        out[l - m] = ldexp(p1, e);
    }
}

void orc_lambda(int lmax, int m, double cth, double sth, double *out)
{
    double *al = (double *)calloc(lmax + 2, sizeof(double));
    double *be = (double *)calloc(lmax + 2, sizeof(double));
    rec_coef(lmax, m, al, be);
    lambda_row_c(lmax, m, cth, sth, al, be, out);
    free(al);
    free(be);
}

/* Spin-2 functions for fixed m from lambda_l and lambda_{l-1} (l >= 2):
 * with N_l = ((l-1) l (l+1) (l+2))^{-1/2}, f_lm = sqrt((2l+1)(l^2-m^2)/(2l-1)),
 *   lw = ( 2Y + (-2)Y ) / 2 = 2 N_l [ -((l - m^2)/s^2 + l(l-1)/2) lambda_l
 *                                     + f_lm x / s^2 lambda_{l-1} ]
 *   lx = ( 2Y - (-2)Y ) / 2 = 2 m N_l / s^2 [ -(l-1) x lambda_l + f_lm lambda_{l-1} ]
 * These follow from applying the spin-raising (lowering) operator twice to
 * lambda_lm e^{imphi}, eliminating lambda'' with the Legendre equation and
 * lambda' with s lambda'_l = l x lambda_l - f_lm lambda_{l-1}.  Both vanish
 * for l < 2.  lam[] holds lambda_lm for l = m..lmax (index l - m). */
static void spin2_from_lambda(int lmax, int m, double x, double s, const double *lam,
                              double *lw, double *lx)
{
    const double is2 = 1.0 / (s * s);
    for (int l = m; l <= lmax; ++l) {
        if (l < 2) {
            lw[l - m] = 0.0;
            lx[l - m] = 0.0;
            continue;
        }
        const double dl = l, dm = m;
        const double nl = 1.0 / sqrt((dl - 1.0) * dl * (dl + 1.0) * (dl + 2.0));
        const double f = sqrt((2.0 * dl + 1.0) * (dl * dl - dm * dm) / (2.0 * dl - 1.0));
        const double lc = lam[l - m];
        const double lp = (l > m) ? lam[l - m - 1] : 0.0;
        lw[l - m] = 2.0 * nl * (-((dl - dm * dm) * is2 + 0.5 * dl * (dl - 1.0)) * lc + f * x * is2 * lp);
        lx[l - m] = 2.0 * dm * nl * is2 * (-(dl - 1.0) * x * lc + f * lp);
    }
}

void orc_lambda_spin2(int lmax, int m, double cth, double sth, double *lw, double *lx)
{
    double *lam = (double *)malloc(sizeof(double) * (lmax - m + 1));
    orc_lambda(lmax, m, cth, sth, lam);
    spin2_from_lambda(lmax, m, cth, sth, lam, lw, lx);
    free(lam);
}

/* ------------------------------------------------------------------------- */
/* ring DFTs                                                                 */
/* ------------------------------------------------------------------------- */
/* f_j = Re F(0) + 2 Re sum_{m=1}^{L} F(m) e^{i m (phi0 + 2 pi j / n)},
 * j = 0..n-1: the real field whose Fourier coefficients for m >= 0 are F(m)
 * and for m < 0 are conj(F(-m)).  Direct sum; the twiddle table holds
 * e^{2 pi i k/n} and the exponent m j is reduced modulo n exactly. */
static void ring_tables(int L, int64_t n, double phi0, double *tw, double *ph)
{
    for (int64_t k = 0; k < n; ++k) {
        tw[2 * k] = cos(2.0 * ORC_PI * (double)k / (double)n);
        tw[2 * k + 1] = sin(2.0 * ORC_PI * (double)k / (double)n);
    }
    for (int m = 0; m <= L; ++m) {
        ph[2 * m] = cos(m * phi0);
        ph[2 * m + 1] = sin(m * phi0);
    }
}

static void ring_synth(int L, const double *F /* 2(L+1) */, int64_t n, double phi0,
                       double *out, double *tw /* 2n + 2(L+1) scratch */)
{
    double *ph = tw + 2 * n;
    ring_tables(L, n, phi0, tw, ph);
    for (int64_t j = 0; j < n; ++j) {
        double acc = F[0];
        for (int m = 1; m <= L; ++m) {
            const double pr = ph[2 * m], pi_ = ph[2 * m + 1];
            const int64_t k = ((int64_t)m * j) % n;
            const double er = pr * tw[2 * k] - pi_ * tw[2 * k + 1];
            const double ei = pr * tw[2 * k + 1] + pi_ * tw[2 * k];
            acc += 2.0 * (F[2 * m] * er - F[2 * m + 1] * ei);
        }
        out[j] = acc;
    }
}

/* G(m) = sum_j y_j e^{-i m (phi0 + 2 pi j / n)}, m = 0..L (the transpose of
 * ring_synth up to the factor 2 on m > 0, which the Q6 metric absorbs). */
static void ring_analy(int L, const double *y, int64_t n, double phi0, double *G,
                       double *tw /* 2n + 2(L+1) scratch */, int nm, const int *mlist)
{
    double *ph = tw + 2 * n;
    ring_tables(L, n, phi0, tw, ph);
    const int cnt = nm < 0 ? L + 1 : nm;
    for (int q = 0; q < cnt; ++q) {
        const int m = nm < 0 ? q : mlist[q];
        const double pr = ph[2 * m], pi_ = ph[2 * m + 1];
        double gr = 0.0, gi = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            const int64_t k = ((int64_t)m * j) % n;
            const double er = pr * tw[2 * k] - pi_ * tw[2 * k + 1];
            const double ei = pr * tw[2 * k + 1] + pi_ * tw[2 * k];
            gr += y[j] * er;
            gi -= y[j] * ei;
        }
        G[2 * m] = gr;
        G[2 * m + 1] = gi;
    }
}

static inline int64_t aidx(int l, int m, int L) { return (int64_t)m * (2 * L + 1 - m) / 2 + l; }

static int64_t max_nphi(int nring, const int64_t *nphi)
{
    int64_t mx = 1;
    for (int r = 0; r < nring; ++r)
        if (nphi[r] > mx) mx = nphi[r];
    return mx;
}

/* ------------------------------------------------------------------------- */
/* spin-0 transforms                                                         */
/* ------------------------------------------------------------------------- */
/* map = Y alm:  F_r(m) = sum_l a_lm lambda_lm(theta_r), then ring_synth. */
void orc_alm2map(int nring, const double *cth, const double *sth, const int64_t *nphi,
                 const double *phi0, const int64_t *ofs, int L, const double *alm,
                 double *map)
{
    double *F = (double *)calloc((size_t)nring * 2 * (L + 1), sizeof(double));
#pragma omp parallel
    {
        double *lam = (double *)malloc(sizeof(double) * (L + 1));
        double *al = (double *)calloc(L + 2, sizeof(double));
        double *be = (double *)calloc(L + 2, sizeof(double));
#pragma omp for schedule(dynamic, 1)
        for (int m = 0; m <= L; ++m) {
            rec_coef(L, m, al, be);
            for (int r = 0; r < nring; ++r) {
                lambda_row_c(L, m, cth[r], sth[r], al, be, lam);
                double fr = 0.0, fi = 0.0;
                for (int l = m; l <= L; ++l) {
                    const int64_t i = aidx(l, m, L);
                    fr += alm[2 * i] * lam[l - m];
                    fi += (m == 0 ? 0.0 : alm[2 * i + 1]) * lam[l - m];
                }
                F[((size_t)r * (L + 1) + m) * 2] = fr;
                F[((size_t)r * (L + 1) + m) * 2 + 1] = fi;
            }
        }
        free(lam);
        free(al);
        free(be);
    }
    const int64_t nmx = max_nphi(nring, nphi);
#pragma omp parallel
    {
        double *tw = (double *)malloc(sizeof(double) * (2 * nmx + 2 * (L + 1)));
#pragma omp for schedule(dynamic, 1)
        for (int r = 0; r < nring; ++r)
            ring_synth(L, F + (size_t)r * 2 * (L + 1), nphi[r], phi0[r], map + ofs[r], tw);
        free(tw);
    }
    free(F);
}

/* alm = Y^T map:  G_r(m) = sum_{p in r} map_p e^{-i m phi_p},
 * c_lm = sum_r lambda_lm(theta_r) G_r(m).  ``mlist`` (length nm) restricts the
 * output to those m (other entries untouched); pass nm < 0 for all m. */
void orc_alm2map_adjoint_m(int nring, const double *cth, const double *sth,
                           const int64_t *nphi, const double *phi0, const int64_t *ofs,
                           int L, const double *map, double *alm, int nm, const int *mlist)
{
    double *G = (double *)calloc((size_t)nring * 2 * (L + 1), sizeof(double));
    const int64_t nmx = max_nphi(nring, nphi);
#pragma omp parallel
    {
        double *tw = (double *)malloc(sizeof(double) * (2 * nmx + 2 * (L + 1)));
#pragma omp for schedule(dynamic, 1)
        for (int r = 0; r < nring; ++r)
            ring_analy(L, map + ofs[r], nphi[r], phi0[r], G + (size_t)r * 2 * (L + 1), tw, nm, mlist);
        free(tw);
    }
    const int cnt = nm < 0 ? L + 1 : nm;
#pragma omp parallel
    {
        double *lam = (double *)malloc(sizeof(double) * (L + 1));
        double *al = (double *)calloc(L + 2, sizeof(double));
        double *be = (double *)calloc(L + 2, sizeof(double));
        double *acc = (double *)malloc(sizeof(double) * 2 * (L + 1));
#pragma omp for schedule(dynamic, 1)
        for (int q = 0; q < cnt; ++q) {
            const int m = nm < 0 ? q : mlist[q];
            rec_coef(L, m, al, be);
            memset(acc, 0, sizeof(double) * 2 * (L + 1));
            for (int r = 0; r < nring; ++r) {
                lambda_row_c(L, m, cth[r], sth[r], al, be, lam);
                const double gr = G[((size_t)r * (L + 1) + m) * 2];
                const double gi = G[((size_t)r * (L + 1) + m) * 2 + 1];
                for (int l = m; l <= L; ++l) {
                    acc[2 * l] += lam[l - m] * gr;
                    acc[2 * l + 1] += lam[l - m] * gi;
                }
            }
            for (int l = m; l <= L; ++l) {
                const int64_t i = aidx(l, m, L);
                alm[2 * i] = acc[2 * l];
                alm[2 * i + 1] = (m == 0) ? 0.0 : acc[2 * l + 1];
            }
        }
        free(lam);
        free(al);
        free(be);
        free(acc);
    }
    free(G);
}

void orc_alm2map_adjoint(int nring, const double *cth, const double *sth,
                         const int64_t *nphi, const double *phi0, const int64_t *ofs, int L,
                         const double *map, double *alm)
{
    orc_alm2map_adjoint_m(nring, cth, sth, nphi, phi0, ofs, L, map, alm, -1, NULL);
}

/* ------------------------------------------------------------------------- */
/* spin-2 transforms (E, B) <-> (Q, U)                                       */
/* ------------------------------------------------------------------------- */
/* With 2a_lm = -(E_lm + i B_lm), -2a_lm = -(E_lm - i B_lm) and
 * Q +- iU = sum +-2a_lm +-2Y_lm, the Fourier coefficients on a ring are
 *   F_Q(m) = - sum_l ( E_lm lw + i B_lm lx ),
 *   F_U(m) =   sum_l ( i E_lm lx - B_lm lw ),
 * and Q, U follow by ring_synth. */
void orc_alm2map_spin2(int nring, const double *cth, const double *sth, const int64_t *nphi,
                       const double *phi0, const int64_t *ofs, int L, const double *almE,
                       const double *almB, double *Q, double *U)
{
    const size_t fsz = (size_t)nring * 2 * (L + 1);
    double *FQ = (double *)calloc(fsz, sizeof(double));
    double *FU = (double *)calloc(fsz, sizeof(double));
#pragma omp parallel
    {
        double *lam = (double *)malloc(sizeof(double) * (L + 1));
        double *lw = (double *)malloc(sizeof(double) * (L + 1));
        double *lx = (double *)malloc(sizeof(double) * (L + 1));
        double *al = (double *)calloc(L + 2, sizeof(double));
        double *be = (double *)calloc(L + 2, sizeof(double));
#pragma omp for schedule(dynamic, 1)
        for (int m = 0; m <= L; ++m) {
            rec_coef(L, m, al, be);
            for (int r = 0; r < nring; ++r) {
                lambda_row_c(L, m, cth[r], sth[r], al, be, lam);
                spin2_from_lambda(L, m, cth[r], sth[r], lam, lw, lx);
                double qr = 0, qi = 0, ur = 0, ui = 0;
                for (int l = m; l <= L; ++l) {
                    const int64_t i = aidx(l, m, L);
                    const double er = almE[2 * i], ei = (m == 0) ? 0.0 : almE[2 * i + 1];
                    const double br = almB[2 * i], bi = (m == 0) ? 0.0 : almB[2 * i + 1];
                    const double w = lw[l - m], x = lx[l - m];
                    /* -(E w + i B x) */
                    qr += -(er * w - bi * x);
                    qi += -(ei * w + br * x);
                    /* i E x - B w */
                    ur += -ei * x - br * w;
                    ui += er * x - bi * w;
                }
                const size_t o = ((size_t)r * (L + 1) + m) * 2;
                FQ[o] = qr;
                FQ[o + 1] = qi;
                FU[o] = ur;
                FU[o + 1] = ui;
            }
        }
        free(lam);
        free(lw);
        free(lx);
        free(al);
        free(be);
    }
    const int64_t nmx = max_nphi(nring, nphi);
#pragma omp parallel
    {
        double *tw = (double *)malloc(sizeof(double) * (2 * nmx + 2 * (L + 1)));
#pragma omp for schedule(dynamic, 1)
        for (int r = 0; r < nring; ++r) {
            ring_synth(L, FQ + (size_t)r * 2 * (L + 1), nphi[r], phi0[r], Q + ofs[r], tw);
            ring_synth(L, FU + (size_t)r * 2 * (L + 1), nphi[r], phi0[r], U + ofs[r], tw);
        }
        free(tw);
    }
    free(FQ);
    free(FU);
}

/* Transpose of orc_alm2map_spin2 in the Q6 metric:
 *   E^_lm = sum_r [ -lw G_Q(m) - i lx G_U(m) ],
 *   B^_lm = sum_r [  i lx G_Q(m) - lw G_U(m) ]. */
void orc_alm2map_spin2_adjoint_m(int nring, const double *cth, const double *sth,
                                 const int64_t *nphi, const double *phi0, const int64_t *ofs,
                                 int L, const double *Q, const double *U, double *almE,
                                 double *almB, int nm, const int *mlist)
{
    const size_t fsz = (size_t)nring * 2 * (L + 1);
    double *GQ = (double *)calloc(fsz, sizeof(double));
    double *GU = (double *)calloc(fsz, sizeof(double));
    const int64_t nmx = max_nphi(nring, nphi);
#pragma omp parallel
    {
        double *tw = (double *)malloc(sizeof(double) * (2 * nmx + 2 * (L + 1)));
#pragma omp for schedule(dynamic, 1)
        for (int r = 0; r < nring; ++r) {
            ring_analy(L, Q + ofs[r], nphi[r], phi0[r], GQ + (size_t)r * 2 * (L + 1), tw, nm, mlist);
            ring_analy(L, U + ofs[r], nphi[r], phi0[r], GU + (size_t)r * 2 * (L + 1), tw, nm, mlist);
        }
        free(tw);
    }
    const int cnt = nm < 0 ? L + 1 : nm;
#pragma omp parallel
    {
        double *lam = (double *)malloc(sizeof(double) * (L + 1));
        double *lw = (double *)malloc(sizeof(double) * (L + 1));
        double *lx = (double *)malloc(sizeof(double) * (L + 1));
        double *al = (double *)calloc(L + 2, sizeof(double));
        double *be = (double *)calloc(L + 2, sizeof(double));
        double *acc = (double *)malloc(sizeof(double) * 4 * (L + 1));
#pragma omp for schedule(dynamic, 1)
        for (int q = 0; q < cnt; ++q) {
            const int m = nm < 0 ? q : mlist[q];
            rec_coef(L, m, al, be);
            memset(acc, 0, sizeof(double) * 4 * (L + 1));
            for (int r = 0; r < nring; ++r) {
                lambda_row_c(L, m, cth[r], sth[r], al, be, lam);
                spin2_from_lambda(L, m, cth[r], sth[r], lam, lw, lx);
                const size_t o = ((size_t)r * (L + 1) + m) * 2;
                const double qr = GQ[o], qi = GQ[o + 1], ur = GU[o], ui = GU[o + 1];
                for (int l = m; l <= L; ++l) {
                    const double w = lw[l - m], x = lx[l - m];
                    /* -w GQ - i x GU */
                    acc[4 * l + 0] += -w * qr + x * ui;
                    acc[4 * l + 1] += -w * qi - x * ur;
                    /* i x GQ - w GU */
                    acc[4 * l + 2] += -x * qi - w * ur;
                    acc[4 * l + 3] += x * qr - w * ui;
                }
            }
            for (int l = m; l <= L; ++l) {
                const int64_t i = aidx(l, m, L);
                almE[2 * i] = acc[4 * l + 0];
                almE[2 * i + 1] = (m == 0) ? 0.0 : acc[4 * l + 1];
                almB[2 * i] = acc[4 * l + 2];
                almB[2 * i + 1] = (m == 0) ? 0.0 : acc[4 * l + 3];
            }
        }
        free(lam);
        free(lw);
        free(lx);
        free(al);
        free(be);
        free(acc);
    }
    free(GQ);
    free(GU);
}

/* ------------------------------------------------------------------------- */
/* ring-averaged diagonal of Y^T N^-1 Y (preconditioner)                     */
/* ------------------------------------------------------------------------- */
/* out_lm = sum_r w_r * g(l, m, theta_r) where g = lambda_lm^2 (spin 0) or
 * lw^2 + lx^2 (spin 2) and w_r = sum_{p in r} N^-1_p. */
void orc_diag_ringsum(int nring, const double *cth, const double *sth, int L, int spin,
                      const double *wring, double *out)
{
#pragma omp parallel
    {
        double *lam = (double *)malloc(sizeof(double) * (L + 1));
        double *lw = (double *)malloc(sizeof(double) * (L + 1));
        double *lx = (double *)malloc(sizeof(double) * (L + 1));
        double *al = (double *)calloc(L + 2, sizeof(double));
        double *be = (double *)calloc(L + 2, sizeof(double));
#pragma omp for schedule(dynamic, 1)
        for (int m = 0; m <= L; ++m) {
            rec_coef(L, m, al, be);
            for (int l = m; l <= L; ++l) out[aidx(l, m, L)] = 0.0;
            for (int r = 0; r < nring; ++r) {
                lambda_row_c(L, m, cth[r], sth[r], al, be, lam);
                if (spin == 2) spin2_from_lambda(L, m, cth[r], sth[r], lam, lw, lx);
                for (int l = m; l <= L; ++l) {
                    const double g = (spin == 2) ? lw[l - m] * lw[l - m] + lx[l - m] * lx[l - m]
                                                 : lam[l - m] * lam[l - m];
                    out[aidx(l, m, L)] += wring[r] * g;
                }
            }
        }
        free(lam);
        free(lw);
        free(lx);
        free(al);
        free(be);
    }
}

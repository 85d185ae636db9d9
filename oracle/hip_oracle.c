/*
 * FP64 brute-force oracle for the windowed periodic-box pair-count estimators of
 * Philcox (arXiv:2005.01739): power-spectrum multipoles (Sec. 3, Eq. pk-binned and
 * its binned estimator) and isotropic bispectrum multipoles (Sec. 4, Eq. AC-def and
 * the binned summary of Sec. 4.5).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference leg of bench.py may load this library.  The product
 * path (paper_2005_01739_gb300) never calls, links or imports anything here, and
 * this file shares no code, header, table or constant generator with it.
 *
 * Everything is written as the plain definition, in double precision:
 *   - every ordered pair (i, j != i) is visited by brute force over all N
 *     particles with the minimum-image separation (periodic box, R0 < L/2);
 *   - the bin-averaged Bessel function is evaluated per bin from its two edges
 *     (Eq. jla-def), with D_l from a power series at small argument and from the
 *     recursion of App. C above it;
 *   - spherical harmonics are the complex Y_lm from associated Legendre functions.
 * OpenMP parallelises over primaries only; per-thread partial sums are reduced at
 * the end, so the arithmetic per primary follows the definition exactly.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <complex.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_LMAX 4
#define ORC_PI 3.14159265358979323846264338327950288

/* ---------------------------------------------------------------- window --- */
/* Pair-separation window of Eq. window_defn (Sec. 2), x = |r| / R0. */
double orc_window(double x)
{
    if (x < 0.0) return 0.0;
    if (x < 0.5) return 1.0;
    if (x < 0.75) {
        double y = 2.0 * x - 1.0;
        return 1.0 - 8.0 * y * y * y + 8.0 * y * y * y * y;
    }
    if (x < 1.0) {
        double y = x - 1.0;
        return -64.0 * y * y * y - 128.0 * y * y * y * y;
    }
    return 0.0;
}

/* ------------------------------------------------------------ Legendre ----- */
double orc_legendre(int l, double mu)
{
    double p0 = 1.0, p1 = mu;
    if (l == 0) return p0;
    for (int n = 1; n < l; ++n) {
        double p2 = ((2.0 * n + 1.0) * mu * p1 - n * p0) / (n + 1.0);
        p0 = p1;
        p1 = p2;
    }
    return p1;
}

/* --------------------------------------------------------- sine integral --- */
/* Si(u) = int_0^u sin(t)/t dt.  Power series for u <= 4; above that
 * Si(u) = pi/2 + Im E1(i u), with E1 from its continued fraction
 * E1(z) = e^{-z} / (z + 1 - 1^2/(z + 3 - 2^2/(z + 5 - ...))) evaluated by the
 * modified Lentz method.  Odd in u. */
double orc_si(double u)
{
    if (u < 0.0) return -orc_si(-u);
    if (u <= 4.0) {
        double sum = 0.0, term = u; /* term = (-1)^n u^(2n+1)/(2n+1)! */
        for (int n = 0; n < 60; ++n) {
            double add = term / (2.0 * n + 1.0);
            sum += add;
            if (fabs(add) < 1e-18 * fabs(sum)) break;
            term *= -u * u / ((2.0 * n + 2.0) * (2.0 * n + 3.0));
        }
        return sum;
    }
    double complex z = I * u;
    const double tiny = 1e-300;
    double complex b = z + 1.0;
    double complex f = 1.0 / b; /* value of the fraction 1/(b0 - a1/(b1 - ...)) */
    double complex c = 1.0 / tiny;
    double complex d = 1.0 / b;
    for (int n = 1; n < 100000; ++n) {
        double complex a = -(double)n * (double)n;
        b += 2.0;
        d = 1.0 / (a * d + b);
        c = b + a / c;
        double complex del = c * d;
        f *= del;
        if (cabs(del - 1.0) < 1e-17) break;
    }
    double complex e1 = cexp(-z) * f;
    return 0.5 * ORC_PI + cimag(e1);
}

/* ------------------------------------------------- spherical Bessel j_n ---- */
/* j_0..j_nmax at x by upward recurrence from the closed forms of j_0, j_1
 * (stable enough for x >= 2 and n <= 6, the only use below).  At x == 0 the
 * limits j_n(0) = delta_{n0} are returned. */
static void orc_sph_jn_up(int nmax, double x, double *j)
{
    if (x == 0.0) {
        for (int n = 0; n <= nmax; ++n) j[n] = (n == 0) ? 1.0 : 0.0;
        return;
    }
    double s = sin(x), c = cos(x);
    j[0] = s / x;
    if (nmax >= 1) j[1] = s / (x * x) - c / x;
    for (int n = 1; n < nmax; ++n) j[n + 1] = (2.0 * n + 1.0) / x * j[n] - j[n - 1];
}

/* Series j_n(x) = sum_s (-1)^s x^(n+2s) / (2^s s! (2n+2s+1)!!), for small x. */
static double orc_sph_jn_series(int n, double x)
{
    double dfac = 1.0; /* (2n+1)!! */
    for (int k = 1; k <= 2 * n + 1; k += 2) dfac *= k;
    double term = pow(x, n) / dfac, sum = 0.0;
    for (int s = 0; s < 200; ++s) {
        sum += term;
        if (fabs(term) < 1e-18 * fabs(sum)) break;
        term *= -x * x / (2.0 * (s + 1) * (2.0 * n + 2.0 * s + 3.0));
    }
    return sum;
}

double orc_sph_jn(int n, double x)
{
    if (fabs(x) < 2.0 + n) return orc_sph_jn_series(n, x);
    double j[16];
    orc_sph_jn_up(n, x, j);
    return j[n];
}

/* ----------------------------------------------------------- D_l(u) -------- */
/* Dhat_l(u) = int_0^u t^2 j_l(t) dt (the D_l of Eq. jla-def taken as the definite
 * integral from 0, App. C).
 *   u <  4 : term-by-term integral of the j_l power series,
 *            sum_s (-1)^s u^(2s+l+3) / (2^s s! (2l+2s+1)!! (2s+l+3));
 *   u >= 4 : the App. C recursion
 *            D_l = u^2 j_{l+1} - l u j_l + l(l+1) I_l,
 *            l I_l = (l-1) I_{l-2} - (2l-1) j_{l-1},  I_0 = Si,  I_1 = -j_0,
 *            minus the same expression at u = 0 (the arbitrary constant of
 *            integration; zero for even l, -2 for l = 1, -8 for l = 3). */
#define ORC_DSWITCH 4.0

static void orc_I_rec(int l, double si0, const double *j, double *Iout)
{
    /* I_0..I_l from the recursion, given I_0 = si0 and j_0..j_{l} */
    double Iv[ORC_LMAX + 2];
    Iv[0] = si0;
    if (l >= 1) Iv[1] = -j[0];
    for (int n = 2; n <= l; ++n) Iv[n] = ((n - 1.0) * Iv[n - 2] - (2.0 * n - 1.0) * j[n - 1]) / n;
    for (int n = 0; n <= l; ++n) Iout[n] = Iv[n];
}

double orc_dhat(int l, double u)
{
    if (u < ORC_DSWITCH) {
        double dfac = 1.0; /* (2l+1)!! */
        for (int k = 1; k <= 2 * l + 1; k += 2) dfac *= k;
        double upow = pow(u, l + 3); /* u^(2s+l+3) */
        double coef = 1.0 / dfac;   /* (-1)^s / (2^s s! (2l+2s+1)!!) */
        double sum = 0.0;
        for (int s = 0; s < 200; ++s) {
            double add = coef * upow / (2.0 * s + l + 3.0);
            sum += add;
            if (fabs(add) < 1e-19 * fabs(sum) || add == 0.0) break;
            coef *= -1.0 / (2.0 * (s + 1) * (2.0 * l + 2.0 * s + 3.0));
            upow *= u * u;
        }
        return sum;
    }
    double j[ORC_LMAX + 3], Iv[ORC_LMAX + 2];
    orc_sph_jn_up(l + 1, u, j);
    orc_I_rec(l, orc_si(u), j, Iv);
    double val = u * u * j[l + 1] - l * u * j[l] + l * (l + 1.0) * Iv[l];
    /* constant of the same closed form at u = 0 */
    double j0[ORC_LMAX + 3], I0[ORC_LMAX + 2];
    orc_sph_jn_up(l + 1, 0.0, j0);
    orc_I_rec(l, 0.0, j0, I0);
    double c0 = l * (l + 1.0) * I0[l];
    return val - c0;
}

/* Bin-averaged spherical Bessel function of Eq. jla-def:
 * jbar = 3 [D_l(r k_hi) - D_l(r k_lo)] / (r^3 (k_hi^3 - k_lo^3)); its r -> 0
 * limit is delta_{l0}. */
double orc_jbar(int l, double r, double klo, double khi)
{
    if (r == 0.0) return (l == 0) ? 1.0 : 0.0;
    return 3.0 * (orc_dhat(l, r * khi) - orc_dhat(l, r * klo)) / (r * r * r * (khi * khi * khi - klo * klo * klo));
}

/* ------------------------------------------------- spherical harmonics ----- */
/* Complex Y_lm(theta, phi) with the Condon-Shortley phase, for 0 <= l <= 4,
 * -l <= m <= l, written into Y[l*l + l + m]; input is a unit vector. */
static void orc_ylm(double ux, double uy, double uz, double complex *Y)
{
    double ct = uz;
    double st = sqrt(fmax(0.0, 1.0 - ct * ct));
    double phi = atan2(uy, ux);
    /* associated Legendre P_l^m(ct), m >= 0, standard recurrences */
    double P[ORC_LMAX + 1][ORC_LMAX + 1];
    memset(P, 0, sizeof(P));
    P[0][0] = 1.0;
    for (int m = 1; m <= ORC_LMAX; ++m) P[m][m] = -(2.0 * m - 1.0) * st * P[m - 1][m - 1];
    for (int m = 0; m < ORC_LMAX; ++m) P[m + 1][m] = (2.0 * m + 1.0) * ct * P[m][m];
    for (int m = 0; m <= ORC_LMAX; ++m)
        for (int l = m + 2; l <= ORC_LMAX; ++l)
            P[l][m] = ((2.0 * l - 1.0) * ct * P[l - 1][m] - (l + m - 1.0) * P[l - 2][m]) / (l - m);
    for (int l = 0; l <= ORC_LMAX; ++l) {
        for (int m = 0; m <= l; ++m) {
            double fr = 1.0; /* (l-m)!/(l+m)! */
            for (int k = l - m + 1; k <= l + m; ++k) fr /= k;
            double norm = sqrt((2.0 * l + 1.0) / (4.0 * ORC_PI) * fr);
            double complex y = norm * P[l][m] * cexp(I * m * phi);
            Y[l * l + l + m] = y;
            if (m > 0) Y[l * l + l - m] = ((m & 1) ? -1.0 : 1.0) * conj(y);
        }
    }
}

void orc_ylm_export(double ux, double uy, double uz, double *re, double *im)
{
    double complex Y[(ORC_LMAX + 1) * (ORC_LMAX + 1)];
    orc_ylm(ux, uy, uz, Y);
    for (int k = 0; k < (ORC_LMAX + 1) * (ORC_LMAX + 1); ++k) {
        re[k] = creal(Y[k]);
        im[k] = cimag(Y[k]);
    }
}

/* --------------------------------------------------------- helpers --------- */
static inline double orc_minimage(double d, double L)
{
    return d - L * round(d / L);
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ----------------------------------------------------------- P pair sum ---- */
/* DD[il][a] = sum_{i in prim} sum_{j != i} w_i w_j W(r_ij/R0) jbar^a_l(r_ij) L_l(mu_ij)
 * for l = 2*il (il = 0..n_ell-1), over ordered pairs with 0 < r_ij < R0, where
 * r_ij = minimum image of x_i - x_j and mu = r_z / r (line of sight along axis
 * `los`).  This is the pair sum inside the binned estimator of Sec. 3 (the sum
 * over i != j in Eq. pk-binned's estimator form).  With prim = all particles it
 * is the full ordered sum.  npairs receives the number of ordered pairs counted.
 * pos is [N][3], w is [N] (NULL means unit weights), prim is [nprim] indices. */
int orc_power_pairs(const double *pos, const double *w, int64_t N, double L, double R0,
                    const double *edges, int nk, int n_ell, int los,
                    const int64_t *prim, int64_t nprim, double *DD, int64_t *npairs)
{
    if (N < 1 || nk < 1 || n_ell < 1 || n_ell > 3 || !(L > 0) || !(R0 > 0) || R0 >= 0.5 * L) return -1;
    int nthr = orc_num_threads();
    double *acc = (double *)calloc((size_t)nthr * n_ell * nk, sizeof(double));
    int64_t *cnt = (int64_t *)calloc((size_t)nthr, sizeof(int64_t));
    if (!acc || !cnt) { free(acc); free(cnt); return -2; }
    double R02 = R0 * R0;
#pragma omp parallel
    {
        int t = 0;
#ifdef _OPENMP
        t = omp_get_thread_num();
#endif
        double *my = acc + (size_t)t * n_ell * nk;
#pragma omp for schedule(dynamic, 16)
        for (int64_t pi = 0; pi < nprim; ++pi) {
            int64_t i = prim[pi];
            double wi = w ? w[i] : 1.0;
            for (int64_t j = 0; j < N; ++j) {
                if (j == i) continue;
                double d[3];
                for (int k = 0; k < 3; ++k) d[k] = orc_minimage(pos[3 * i + k] - pos[3 * j + k], L);
                double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                if (r2 >= R02 || r2 == 0.0) continue;
                double r = sqrt(r2);
                double mu = d[los] / r;
                double wgt = wi * (w ? w[j] : 1.0) * orc_window(r / R0);
                cnt[t] += 1;
                for (int il = 0; il < n_ell; ++il) {
                    int l = 2 * il;
                    double lw = wgt * orc_legendre(l, mu);
                    for (int a = 0; a < nk; ++a) my[il * nk + a] += lw * orc_jbar(l, r, edges[a], edges[a + 1]);
                }
            }
        }
    }
    memset(DD, 0, sizeof(double) * n_ell * nk);
    int64_t tot = 0;
    for (int t = 0; t < nthr; ++t) {
        for (int k = 0; k < n_ell * nk; ++k) DD[k] += acc[(size_t)t * n_ell * nk + k];
        tot += cnt[t];
    }
    if (npairs) *npairs = tot;
    free(acc);
    free(cnt);
    return 0;
}

/* ------------------------------------------------------ B primary sums ----- */
/* For each primary p (rows of ppos, weight pw[p]) form, over data j with
 * 0 < |x_p - x_j| < R0 (minimum image; a primary that is itself data row
 * `pself[p]` skips that row; pself may be NULL or hold -1):
 *   A^a_lm(p) = sum_j w_j jbar^a_l(r) W(r/R0) Y_lm(rhat),  rhat = (x_p - x_j)/r
 *   C^ab_l(p) = sum_j w_j^2 jbar^a_l(r) jbar^b_l(r) W(r/R0)^2
 * (Eq. AC-def with the k-space binning of Sec. 4.4) and accumulate
 *   T[l][a][b] += pw[p] * [ 4pi/(2l+1) Re sum_m A^a_lm conj(A^b_lm) - C^ab_l ].
 * T is [(lmax+1) * nk * nk].  npairs counts (primary, data) pairs. */
int orc_bispec_primaries(const double *ppos, const double *pw, const int64_t *pself, int64_t nprim,
                         const double *dpos, const double *dw, int64_t N, double L, double R0,
                         const double *edges, int nk, int lmax, double *T, int64_t *npairs)
{
    if (lmax < 0 || lmax > ORC_LMAX || nk < 1 || !(L > 0) || !(R0 > 0) || R0 >= 0.5 * L) return -1;
    int nl = lmax + 1;
    int nlm = nl * nl;
    size_t tsz = (size_t)nl * nk * nk;
    int nthr = orc_num_threads();
    double *acc = (double *)calloc((size_t)nthr * tsz, sizeof(double));
    int64_t *cnt = (int64_t *)calloc((size_t)nthr, sizeof(int64_t));
    if (!acc || !cnt) { free(acc); free(cnt); return -2; }
    double R02 = R0 * R0;
#pragma omp parallel
    {
        int t = 0;
#ifdef _OPENMP
        t = omp_get_thread_num();
#endif
        double *my = acc + (size_t)t * tsz;
        double complex *A = (double complex *)malloc(sizeof(double complex) * nlm * nk);
        double *C = (double *)malloc(sizeof(double) * tsz);
        double *jb = (double *)malloc(sizeof(double) * nl * nk);
        double complex Y[(ORC_LMAX + 1) * (ORC_LMAX + 1)];
#pragma omp for schedule(dynamic, 8)
        for (int64_t p = 0; p < nprim; ++p) {
            memset(A, 0, sizeof(double complex) * nlm * nk);
            memset(C, 0, sizeof(double) * tsz);
            int64_t self = pself ? pself[p] : -1;
            for (int64_t j = 0; j < N; ++j) {
                if (j == self) continue;
                double d[3];
                for (int k = 0; k < 3; ++k) d[k] = orc_minimage(ppos[3 * p + k] - dpos[3 * j + k], L);
                double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                if (r2 >= R02 || r2 == 0.0) continue;
                double r = sqrt(r2);
                cnt[t] += 1;
                double wj = dw ? dw[j] : 1.0;
                double W = orc_window(r / R0);
                orc_ylm(d[0] / r, d[1] / r, d[2] / r, Y);
                for (int l = 0; l < nl; ++l)
                    for (int a = 0; a < nk; ++a) jb[l * nk + a] = orc_jbar(l, r, edges[a], edges[a + 1]);
                for (int l = 0; l < nl; ++l)
                    for (int m = -l; m <= l; ++m)
                        for (int a = 0; a < nk; ++a)
                            A[(l * l + l + m) * nk + a] += wj * jb[l * nk + a] * W * Y[l * l + l + m];
                for (int l = 0; l < nl; ++l)
                    for (int a = 0; a < nk; ++a)
                        for (int b = 0; b < nk; ++b)
                            C[((size_t)l * nk + a) * nk + b] += wj * wj * jb[l * nk + a] * jb[l * nk + b] * W * W;
            }
            for (int l = 0; l < nl; ++l)
                for (int a = 0; a < nk; ++a)
                    for (int b = 0; b < nk; ++b) {
                        double complex s = 0.0;
                        for (int m = -l; m <= l; ++m)
                            s += A[(l * l + l + m) * nk + a] * conj(A[(l * l + l + m) * nk + b]);
                        my[((size_t)l * nk + a) * nk + b] +=
                            pw[p] * (4.0 * ORC_PI / (2.0 * l + 1.0) * creal(s) - C[((size_t)l * nk + a) * nk + b]);
                    }
        }
        free(A);
        free(C);
        free(jb);
    }
    memset(T, 0, sizeof(double) * tsz);
    int64_t tot = 0;
    for (int t = 0; t < nthr; ++t) {
        for (size_t k = 0; k < tsz; ++k) T[k] += acc[(size_t)t * tsz + k];
        tot += cnt[t];
    }
    if (npairs) *npairs = tot;
    free(acc);
    free(cnt);
    return 0;
}

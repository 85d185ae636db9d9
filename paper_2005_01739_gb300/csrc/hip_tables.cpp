// Host-side FP64 construction of the small coefficient tables used by the pair
// kernels (see hip_math.cuh):
//   * Taylor coefficients of F_l(u) = D_l(u)/u^3, from term-by-term integration of
//     the power series of j_l (D_l as defined under Eq. jla-def, App. C);
//   * the power series of the sine integral Si(u) / u in u^2;
//   * polynomial fits of the sine-integral auxiliary functions
//         u f(u)   = int_0^inf e^{-s} / (1 + s^2/u^2) ds,
//         u^2 g(u) = int_0^inf s e^{-s} / (1 + s^2/u^2) ds,
//     (Laplace-transform representations of f and g; Si = pi/2 - f cos - g sin),
//     by Chebyshev interpolation in t = (u0/u)^2 on (0, 1], converted to monomials.
// The integrals are done by composite Gauss-Legendre quadrature with nodes from
// Newton iteration on the Legendre polynomial.
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "hip_math.cuh"

namespace {

void legendre_pd(int n, double z, double &p, double &dp)
{
    double p0 = 1.0, p1 = z;
    for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
    }
    p = p1;
    dp = n * (z * p1 - p0) / (z * z - 1.0);
}

void gauss_legendre(int n, std::vector<double> &x, std::vector<double> &w)
{
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    for (int i = 0; i < n; ++i) {
        double z = std::cos(M_PI * (i + 0.75) / (n + 0.5)), p, dp;
        for (int it = 0; it < 100; ++it) {
            legendre_pd(n, z, p, dp);
            double dz = p / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        legendre_pd(n, z, p, dp);
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

// u f(u) and u^2 g(u) by composite Gauss-Legendre on s in [0, 60].
void aux_fg(double u, double &uf, double &u2g)
{
    static std::vector<double> gx, gw;
    static std::once_flag once;
    std::call_once(once, [] { gauss_legendre(20, gx, gw); });
    const int panels = 120;
    const double smax = 60.0, h = smax / panels;
    double a = 0.0, b = 0.0;
    for (int p = 0; p < panels; ++p) {
        double lo = p * h;
        for (size_t q = 0; q < gx.size(); ++q) {
            double s = lo + 0.5 * h * (gx[q] + 1.0);
            double wq = 0.5 * h * gw[q];
            double den = 1.0 + (s / u) * (s / u);
            double e = std::exp(-s) / den;
            a += wq * e;
            b += wq * s * e;
        }
    }
    uf = a;
    u2g = b;
}

// Chebyshev interpolation of v(t) on [0,1] at deg+1 first-kind nodes, returned as
// monomial coefficients in t.
template <typename Fn>
void cheb_fit_monomial(int deg, Fn fn, std::vector<double> &mono)
{
    int n = deg + 1;
    std::vector<double> fv(n), tnode(n);
    for (int i = 0; i < n; ++i) {
        double y = std::cos(M_PI * (i + 0.5) / n);
        tnode[i] = 0.5 * (y + 1.0);
        fv[i] = fn(tnode[i]);
    }
    std::vector<double> cc(n, 0.0);
    for (int k = 0; k < n; ++k) {
        double s = 0.0;
        for (int i = 0; i < n; ++i) s += fv[i] * std::cos(M_PI * k * (i + 0.5) / n);
        cc[k] = (k == 0 ? 1.0 : 2.0) * s / n;
    }
    // T_k(2t - 1) as monomials in t
    std::vector<std::vector<double>> T(n, std::vector<double>(n, 0.0));
    T[0][0] = 1.0;
    if (n > 1) {
        T[1][0] = -1.0;
        T[1][1] = 2.0;
    }
    for (int k = 2; k < n; ++k) {
        for (int j = 0; j < n; ++j) {
            double v = -2.0 * T[k - 1][j] - T[k - 2][j];
            if (j > 0) v += 4.0 * T[k - 1][j - 1];
            T[k][j] = v;
        }
    }
    mono.assign(n, 0.0);
    for (int k = 0; k < n; ++k)
        for (int j = 0; j < n; ++j) mono[j] += cc[k] * T[k][j];
}

}  // namespace

void hip_build_coeffs(HipCoeffs *C)
{
    std::memset(C, 0, sizeof(*C));
    // Taylor coefficients of F_l(u)/u^l in x = u^2:
    //   (-1)^s / (2^s s! (2l+2s+1)!! (2s+l+3))
    for (int l = 0; l <= HIP_LMAX; ++l) {
        double dfac = 1.0;
        for (int k = 1; k <= 2 * l + 1; k += 2) dfac *= k;
        double coef = 1.0 / dfac;
        for (int s = 0; s < HIP_F64_NSER; ++s) {
            double c = coef / (2.0 * s + l + 3.0);
            C->ser64[l][s] = c;
            if (s < HIP_F32_NSER) {
                C->ser32[l][s] = (float)c;
                C->ser32lo[l][s] = (float)(c - (double)C->ser32[l][s]);
            }
            coef *= -1.0 / (2.0 * (s + 1) * (2.0 * l + 2.0 * s + 3.0));
        }
    }
    // Si(u)/u = sum_n (-1)^n x^n / ((2n+1) (2n+1)!)
    {
        double fac = 1.0;  // (2n+1)!
        for (int n = 0; n < HIP_F64_NSISER; ++n) {
            if (n > 0) fac *= (2.0 * n) * (2.0 * n + 1.0);
            C->siser64[n] = ((n & 1) ? -1.0 : 1.0) / ((2.0 * n + 1.0) * fac);
        }
    }
    std::vector<double> m;
    auto fit = [&](double u0, int deg, int which, std::vector<double> &out) {
        cheb_fit_monomial(deg, [&](double t) {
            double tt = t < 1e-300 ? 1e-300 : t;
            double u = u0 / std::sqrt(tt);
            double uf, u2g;
            if (t <= 0.0) {
                uf = 1.0;
                u2g = 1.0;
            } else {
                aux_fg(u, uf, u2g);
            }
            return which == 0 ? uf : u2g;
        }, out);
    };
    fit(6.0, HIP_F32_SIDEG, 0, m);
    for (int q = 0; q <= HIP_F32_SIDEG; ++q) C->sif32[q] = (float)m[q];
    fit(6.0, HIP_F32_SIDEG, 1, m);
    for (int q = 0; q <= HIP_F32_SIDEG; ++q) C->sig32[q] = (float)m[q];
    fit(4.0, HIP_FB_SIDEG, 0, m);
    for (int q = 0; q <= HIP_FB_SIDEG; ++q) C->fbsif[q] = (float)m[q];
    fit(4.0, HIP_FB_SIDEG, 1, m);
    for (int q = 0; q <= HIP_FB_SIDEG; ++q) C->fbsig[q] = (float)m[q];
    // F_l(u)/u^l on x = u^2 in [0, 16]: Chebyshev interpolation of degree 6 of
    // its Taylor series (40 terms, FP64), returned as monomials in x
    for (int l = 0; l <= HIP_LMAX; ++l) {
        cheb_fit_monomial(HIP_FB_NPOLY - 1, [&](double tt) {
            const double x = 16.0 * tt;
            double dfac = 1.0;
            for (int k = 1; k <= 2 * l + 1; k += 2) dfac *= k;
            double coef = 1.0 / dfac, xs = 1.0, sum = 0.0;
            for (int q = 0; q < 40; ++q) {
                sum += coef / (2.0 * q + l + 3.0) * xs;
                coef *= -1.0 / (2.0 * (q + 1) * (2.0 * l + 2.0 * q + 3.0));
                xs *= x;
            }
            return sum;
        }, m);
        // monomials in t = x / 16 -> monomials in x
        double sc = 1.0;
        for (int q = 0; q < HIP_FB_NPOLY; ++q) {
            C->fbpoly[l][q] = (float)(m[q] * sc);
            sc /= 16.0;
        }
    }
    fit(HIP_F64_USI, HIP_F64_SIDEG, 0, m);
    for (int q = 0; q <= HIP_F64_SIDEG; ++q) C->sif64[q] = m[q];
    fit(HIP_F64_USI, HIP_F64_SIDEG, 1, m);
    for (int q = 0; q <= HIP_F64_SIDEG; ++q) C->sig64[q] = m[q];
}

// Nodes and weights of n-point Gauss-Legendre quadrature on [-1, 1].
void hip_gauss_legendre(int n, std::vector<double> &x, std::vector<double> &w) { gauss_legendre(n, x, w); }

const HipCoeffs &hip_host_coeffs()
{
    static HipCoeffs C;
    static std::once_flag once;
    std::call_once(once, [] { hip_build_coeffs(&C); });
    return C;
}

// Per-pair special functions of the estimators of arXiv:2005.01739, shared by the
// pair kernels (device) and by host self-checks (the same source compiles for both).
//
// The bin-averaged spherical Bessel function of Eq. jla-def is evaluated through
// its edge form
//     jbar^a_l(r) = 3 [ k_{a+1}^3 F_l(r k_{a+1}) - k_a^3 F_l(r k_a) ] / (k_{a+1}^3 - k_a^3),
//     F_l(u) = D_l(u) / u^3,   D_l(u) = int_0^u t^2 j_l(t) dt,
// so one F_l evaluation per (pair, bin edge) serves the two bins that share the
// edge and the r^-3 of Eq. jla-def never appears.  D_l comes from the recursion
// of App. C, which for l <= 4 collapses to (s = sin u, c = cos u, Si = sine integral)
//     D_0 = s - u c
//     D_1 = 2 - 2c - u s
//     D_2 = -4 s + u c + 3 Si
//     D_3 = (u - 15/u) s + 7 c + 8
//     D_4 = (11 - 52.5/u^2) s + (52.5/u - u) c + 7.5 Si
// (constants of integration chosen so that D_l(0) = 0).  These forms cancel
// catastrophically for small u, where the Taylor series of F_l in x = u^2 is used
// instead.  Si(u) for large u is pi/2 - f(u) cos u - g(u) sin u with the auxiliary
// functions f, g replaced by polynomial fits of u f(u) and u^2 g(u) in
// t = (u0/u)^2, fitted in FP64 on the host at library initialisation.
#pragma once

#include <math.h>
#include <stdint.h>

#ifndef __CUDACC__
#define __host__
#define __device__
#define __forceinline__ inline
#endif

#define HIP_F32_USMALL 6.0f    // FP32: series below, closed form above
#define HIP_F32_NSER 15        // Taylor terms of F_l in x = u^2 (u < 6)
#define HIP_F32_NSERLO 9       // terms of the low-half coefficient chain
#define HIP_F32_SIDEG 8        // degree of the u f(u), u^2 g(u) fits in t = (6/u)^2
#define HIP_F32_UASYM 24.0f    // FP32: asymptotic f, g (four terms each) when u >= this

#define HIP_F64_USMALL 2.5     // FP64: series below
#define HIP_F64_USI 12.0       // FP64: Si by its power series below, fitted auxiliaries above
#define HIP_F64_NSER 16
#define HIP_F64_NSISER 32
#define HIP_F64_SIDEG 16

#define HIP_LMAX 4

// FP32 edge functions of the bispectrum pass: a short polynomial below HIP_FB_U
// and the closed forms above (see hip_F_b32)
#define HIP_FB_U 4.0f          // polynomial below, closed form above
#define HIP_FB_NPOLY 7         // terms of F_l(u)/u^l as a polynomial in x = u^2 on [0, 16]
#define HIP_FB_SIDEG 10        // degree of the u f(u), u^2 g(u) fits in t = (4/u)^2

// The FP32 series coefficients are stored as unevaluated sums hi + lo of two
// floats; the lo halves are evaluated by a second, shorter Horner chain whose
// result is accumulated separately (see hip_F_f32).  Rounding a coefficient to a
// single float would bias F_l(u) by a smooth function of u, the same for every
// pair; summed over ~1e9 pairs such a bias does not average out, while the
// rounding of the arithmetic itself varies from pair to pair and does.
struct HipCoeffs {
    // Taylor coefficients of F_l(u) / u^l in x = u^2
    float ser32[HIP_LMAX + 1][HIP_F32_NSER];
    float ser32lo[HIP_LMAX + 1][HIP_F32_NSER];
    double ser64[HIP_LMAX + 1][HIP_F64_NSER];
    // monomial coefficients in t of u f(u) and u^2 g(u) (FP32: t = (6/u)^2; FP64: t = (12/u)^2)
    float sif32[HIP_F32_SIDEG + 1];
    float sig32[HIP_F32_SIDEG + 1];
    double sif64[HIP_F64_SIDEG + 1];
    double sig64[HIP_F64_SIDEG + 1];
    // Si(u) / u = sum_n a_n x^n (FP64 middle range)
    double siser64[HIP_F64_NSISER];
    // bispectrum pass: F_l(u)/u^l on u < 4 as monomials in x = u^2 (Chebyshev
    // interpolant of degree 6), and the f, g fits in t = (4/u)^2 for u >= 4
    float fbpoly[HIP_LMAX + 1][HIP_FB_NPOLY];
    float fbsif[HIP_FB_SIDEG + 1];
    float fbsig[HIP_FB_SIDEG + 1];
};

#define HIP_HALF_PI_F 1.57079632679489661923f
#define HIP_HALF_PI_F_LO (-4.37113900018624283e-8f)  // pi/2 - (float)(pi/2)
#define HIP_HALF_PI_D 1.57079632679489661923

// ---------------------------------------------------------------- window ----
// Eq. window_defn (Sec. 2); x = r / R0.
template <typename T>
__host__ __device__ __forceinline__ T hip_W(T x)
{
    if (x < T(0.5)) return T(1);
    if (x < T(0.75)) {
        T y = T(2) * x - T(1);
        T y3 = y * y * y;
        return T(1) - T(8) * y3 + T(8) * y3 * y;
    }
    if (x < T(1)) {
        T y = x - T(1);
        T y3 = y * y * y;
        return T(-64) * y3 - T(128) * y3 * y;
    }
    return T(0);
}

// ------------------------------------------------- scaled Legendre series ----
// R_m(t) = d_m P_m(t) with d_0 = 1 and d_{m+1} = d_m (m + 1) / 2^{k_m},
// k_m = floor(log2(m + 1)).  Bonnet's recurrence becomes
//     R_{m+1} = alpha_m t R_m - beta_m R_{m-1},
//     alpha_m = (2m + 1) / 2^{k_m},  beta_m = m^2 / 2^{k_m + k_{m-1}},
// whose constants are exact in binary floating point: the recursion in FP32 then
// has no error common to all its inputs (a rounded (2m+1)/(m+1) would scale every
// P_{m+1} by the same factor).  d_m stays between 1 and 2^m.
__host__ __device__ constexpr int hip_leg_k(int m)
{
    int k = 0;
    while ((2 << k) <= m + 1) ++k;
    return k;
}
template <typename T>
__host__ __device__ constexpr T hip_leg_alpha(int m)
{
    return T(2 * m + 1) / T(1 << hip_leg_k(m));
}
template <typename T>
__host__ __device__ constexpr T hip_leg_beta(int m)
{
    return T(m * m) / T(1 << (hip_leg_k(m) + hip_leg_k(m - 1)));
}
__host__ __device__ constexpr double hip_leg_scale(int m)  // d_m (exact)
{
    double d = 1.0;
    for (int j = 0; j < m; ++j) d = d * (j + 1) / (1 << hip_leg_k(j));
    return d;
}

template <typename T>
__host__ __device__ __forceinline__ void hip_legendre24(T mu, T &l2, T &l4)
{
    T m2 = mu * mu;
    l2 = T(1.5) * m2 - T(0.5);
    l4 = (T(4.375) * m2 - T(3.75)) * m2 + T(0.375);
}

// ------------------------------------------------------------ F_l (FP32) ---
// Evaluates F_l(u) for the l in MASK (bit l) as an unevaluated sum
//     F_l(u) = Fm[l] + Fc[l] + (series && l == 0 ? C.ser32[0][0] : 0),
// where the caller accumulates the three parts separately:
//   Fm  -- the float-rounded main value;
//   Fc  -- the tiny correction carried by the low halves of the series
//          coefficients (zero on the closed-form branch);
//   the constant 1/3 of F_0 (as its float C.ser32[0][0]) on the series branch,
//   returned through `series` so that the caller adds omega * (1/3)_float as its
//   own FMA.
// Keeping the constant out of Fm matters: near u = 0, F_0 = 1/3 - u^2/30 + ...
// is flat, so rounding 1/3 + small to a float gives the same rounding error for
// every close pair, a bias that does not average out over many pairs.
template <int MASK>
__host__ __device__ __forceinline__ void hip_F_f32_series(float u, const HipCoeffs &C, float *Fm, float *Fc)
{
    const float x = u * u;
#pragma unroll
    for (int l = 0; l <= HIP_LMAX; ++l) {
        if (!(MASK & (1 << l))) continue;
        float acc = C.ser32[l][HIP_F32_NSER - 1];
#pragma unroll
        for (int s = HIP_F32_NSER - 2; s >= 1; --s) acc = fmaf(acc, x, C.ser32[l][s]);
        float cor = C.ser32lo[l][HIP_F32_NSERLO - 1];
#pragma unroll
        for (int s = HIP_F32_NSERLO - 2; s >= 0; --s) cor = fmaf(cor, x, C.ser32lo[l][s]);
        float ul = 1.0f;
#pragma unroll
        for (int q = 0; q < l; ++q) ul *= u;
        if (l == 0) {
            Fm[0] = acc * x;
        } else {
            Fm[l] = fmaf(acc, x, C.ser32[l][0]) * ul;
        }
        Fc[l] = cor * ul;
    }
}

// Closed forms of F_l = D_l / u^3 given s = sin u, c = cos u.
template <int MASK>
__host__ __device__ __forceinline__ void hip_F_f32_closed(float u, float s, float c, const HipCoeffs &C, float *Fm)
{
#ifdef __CUDA_ARCH__
    const float w = __fdividef(1.0f, u);
#else
    const float w = 1.0f / u;
#endif
    const float w2 = w * w;
    const float w3 = w2 * w;
    float si = 0.0f;
    if (MASK & ((1 << 2) | (1 << 4))) {
        const float t = 36.0f * w2;
        float pf = C.sif32[HIP_F32_SIDEG], pg = C.sig32[HIP_F32_SIDEG];
#pragma unroll
        for (int q = HIP_F32_SIDEG - 1; q >= 0; --q) {
            pf = fmaf(pf, t, C.sif32[q]);
            pg = fmaf(pg, t, C.sig32[q]);
        }
        // Si = pi/2 - f cos - g sin, f = w pf, g = w^2 pg
        si = HIP_HALF_PI_F - fmaf(w, fmaf(pf, c, w * pg * s), -HIP_HALF_PI_F_LO);
    }
    if (MASK & 1) Fm[0] = fmaf(w3, s, -w2 * c);
    if (MASK & 2) Fm[1] = fmaf(w3, 2.0f - 2.0f * c, -w2 * s);
    if (MASK & 4) Fm[2] = fmaf(w3, fmaf(3.0f, si, -4.0f * s), w2 * c);
    if (MASK & 8) Fm[3] = fmaf(w2, s, w3 * fmaf(7.0f, c, 8.0f - 15.0f * w * s));
    if (MASK & 16) Fm[4] = fmaf(w3, fmaf(fmaf(-52.5f, w2, 11.0f), s, 7.5f * si), w2 * fmaf(52.5f, w2, -1.0f) * c);
}

// ----------------------------------------------------- D_l (FP32 pair path) ---
// The FP32 pair kernels accumulate omega D_l(r k_e) / r^3 = omega k_e^3 F_l(r k_e)
// per edge, so the closed forms are used without their 1/u^3 factor.
//
// Closed forms given s = sin u, c = cos u (u >= HIP_F32_USMALL).  Si(u) =
// pi/2 - f(u) cos u - g(u) sin u with the auxiliary functions f, g either from
// the fits used by hip_F_f32_closed (any u >= 6) or, when ASYM, from the first
// four terms of their asymptotic series,
//     f = (1/u) (1 - 2!/u^2 + 4!/u^4 - 6!/u^6),  g = (1/u^2) (1 - 3!/u^2 + 5!/u^4 - 7!/u^6),
// whose remainders are below the first omitted terms 8!/u^9 and 9!/u^10:
// 1.5e-8 and 6e-9 at u = 24, against |D_l| ~ u.
//
// w is 1/u as the caller has it (the pair kernels form it as (1/r)(1/k_e)).
template <int MASK, bool ASYM>
__host__ __device__ __forceinline__ void hip_D_f32_closed(float u, float w, float s, float c, const HipCoeffs &C,
                                                          float *D)
{
    float w2 = 0.0f, si = 0.0f;
    if (MASK & ((1 << 2) | (1 << 3) | (1 << 4))) w2 = w * w;
    if (MASK & ((1 << 2) | (1 << 4))) {
        float pf, pg;
        if (ASYM) {
            pf = fmaf(fmaf(fmaf(-720.0f, w2, 24.0f), w2, -2.0f), w2, 1.0f);
            pg = fmaf(fmaf(fmaf(-5040.0f, w2, 120.0f), w2, -6.0f), w2, 1.0f);
        } else {
            const float t = 36.0f * w2;
            pf = C.sif32[HIP_F32_SIDEG];
            pg = C.sig32[HIP_F32_SIDEG];
#pragma unroll
            for (int q = HIP_F32_SIDEG - 1; q >= 0; --q) {
                pf = fmaf(pf, t, C.sif32[q]);
                pg = fmaf(pg, t, C.sig32[q]);
            }
        }
        // Si = pi/2 - f cos - g sin, f = w pf, g = w^2 pg
        si = HIP_HALF_PI_F - fmaf(w, fmaf(pf, c, w * pg * s), -HIP_HALF_PI_F_LO);
    }
    if (MASK & 1) D[0] = fmaf(-u, c, s);
    if (MASK & 2) D[1] = fmaf(-u, s, 2.0f - 2.0f * c);
    if (MASK & 4) D[2] = fmaf(u, c, fmaf(3.0f, si, -4.0f * s));
    if (MASK & 8) D[3] = fmaf(fmaf(-15.0f, w, u), s, fmaf(7.0f, c, 8.0f));
    if (MASK & 16) D[4] = fmaf(fmaf(-52.5f, w2, 11.0f), s, fmaf(fmaf(52.5f, w, -u), c, 7.5f * si));
}

// Series below HIP_F32_USMALL: D_l = u^(3 + l) (c_l0 + x P_l(x) + low-half chain),
// x = u^2.  The constant's low half rides in the low chain, so that the 1/3 of
// D_0 is not rounded to a float once for every pair.
template <int MASK>
__host__ __device__ __forceinline__ void hip_D_f32_series(float u, const HipCoeffs &C, float *D)
{
    const float x = u * u;
    const float u3 = x * u;
#pragma unroll
    for (int l = 0; l <= HIP_LMAX; ++l) {
        if (!(MASK & (1 << l))) continue;
        float acc = C.ser32[l][HIP_F32_NSER - 1];
#pragma unroll
        for (int s = HIP_F32_NSER - 2; s >= 1; --s) acc = fmaf(acc, x, C.ser32[l][s]);
        float cor = C.ser32lo[l][HIP_F32_NSERLO - 1];
#pragma unroll
        for (int s = HIP_F32_NSERLO - 2; s >= 0; --s) cor = fmaf(cor, x, C.ser32lo[l][s]);
        float ul = u3;
#pragma unroll
        for (int q = 0; q < l; ++q) ul *= u;
        D[l] = (fmaf(acc, x, C.ser32[l][0]) + cor) * ul;
    }
}

template <int MASK>
__host__ __device__ __forceinline__ void hip_F_f32(float u, const HipCoeffs &C, float *Fm, float *Fc, bool &series)
{
    if (u < HIP_F32_USMALL) {
        series = true;
        hip_F_f32_series<MASK>(u, C, Fm, Fc);
        return;
    }
    series = false;
    float s, c;
#ifdef __CUDA_ARCH__
    sincosf(u, &s, &c);
#else
    s = sinf(u);
    c = cosf(u);
#endif
    hip_F_f32_closed<MASK>(u, s, c, C, Fm);
#pragma unroll
    for (int l = 0; l <= HIP_LMAX; ++l) Fc[l] = 0.0f;
}

// ------------------------------------------------- F_l (FP32, bispectrum) ---
// F_l(u), l = 0..4, for the bispectrum's a_lm pass, where every lane of a warp
// evaluates one bin edge of the same pair and the two branches below diverge
// whenever some edges fall below the switch: the branches are kept short.
//   u < 4:  F_l(u) = u^l p_l(u^2), p_l the degree-6 Chebyshev interpolant of
//           F_l(u)/u^l on x in [0, 16] (made in FP64 at library load), evaluated
//           by Horner in x: ~2e-7 relative in FP32;
//   u >= 4: the closed forms with Si = pi/2 - f cos - g sin from degree-10 fits
//           of u f(u), u^2 g(u) in t = (4/u)^2: ~1.5e-7 absolute in Si; the
//           closed forms cancel by at most ~10x at u = 4 for l = 4.
// Unlike hip_F_f32 (the power spectrum's direct pass, held to 1e-5 on sums of
// 1e9 pairs) there is no low-order correction chain: the bispectrum's budget is
// 1e-4.
#ifdef __CUDA_ARCH__
// sin and cos of u >= 0 for the bispectrum's edge functions: Cody-Waite reduction
// u = k pi/2 + x with pi/2 split into three floats (A + B + C, each product k A,
// k B, k C taken exactly inside an FMA; reduction error < 3e-8 for u < 1500), then
// the hardware approximations on |x| <= pi/4 (absolute error below 4e-7 there),
// and the quadrant k mod 4.  Cheaper than sincosf, whose full-range accuracy the
// 1e-4 budget of B does not need.
__device__ __forceinline__ void hip_sincos_b32(float u, float *s, float *c)
{
    const float k = rintf(u * 0.636619746685028f);  // 2 / pi
    float x = fmaf(k, -1.5707963705062866f, u);
    x = fmaf(k, 4.371138828673793e-08f, x);
    x = fmaf(k, 1.7151245100058819e-15f, x);
    const float sx = __sinf(x), cx = __cosf(x);
    const int q = (int)k & 3;
    *s = (q & 1) ? cx : sx;
    *c = (q & 1) ? sx : cx;
    if (q == 1 || q == 2) *c = -*c;
    if (q >= 2) *s = -*s;
}
#endif

__host__ __device__ __forceinline__ void hip_F_b32(float u, const HipCoeffs &C, float *F)
{
    if (u < HIP_FB_U) {
        const float x = u * u;
        float ul = 1.0f;
#pragma unroll
        for (int l = 0; l <= HIP_LMAX; ++l) {
            float acc = C.fbpoly[l][HIP_FB_NPOLY - 1];
#pragma unroll
            for (int q = HIP_FB_NPOLY - 2; q >= 0; --q) acc = fmaf(acc, x, C.fbpoly[l][q]);
            F[l] = acc * ul;
            ul *= u;
        }
        return;
    }
    float s, c;
#ifdef __CUDA_ARCH__
    hip_sincos_b32(u, &s, &c);
    const float w = __fdividef(1.0f, u);
#else
    s = sinf(u);
    c = cosf(u);
    const float w = 1.0f / u;
#endif
    const float w2 = w * w;
    const float w3 = w2 * w;
    const float t = 16.0f * w2;
    float pf = C.fbsif[HIP_FB_SIDEG], pg = C.fbsig[HIP_FB_SIDEG];
#pragma unroll
    for (int q = HIP_FB_SIDEG - 1; q >= 0; --q) {
        pf = fmaf(pf, t, C.fbsif[q]);
        pg = fmaf(pg, t, C.fbsig[q]);
    }
    const float si = HIP_HALF_PI_F - fmaf(w, fmaf(pf, c, w * pg * s), -HIP_HALF_PI_F_LO);
    F[0] = fmaf(w3, s, -w2 * c);
    F[1] = fmaf(w3, 2.0f - 2.0f * c, -w2 * s);
    F[2] = fmaf(w3, fmaf(3.0f, si, -4.0f * s), w2 * c);
    F[3] = fmaf(w2, s, w3 * fmaf(7.0f, c, 8.0f - 15.0f * w * s));
    F[4] = fmaf(w3, fmaf(fmaf(-52.5f, w2, 11.0f), s, 7.5f * si), w2 * fmaf(52.5f, w2, -1.0f) * c);
}

// Total F_l(u) of the FP32 path (host self-checks).
template <int MASK>
__host__ __device__ __forceinline__ void hip_F_f32_total(float u, const HipCoeffs &C, double *F)
{
    float Fm[5] = {0, 0, 0, 0, 0}, Fc[5] = {0, 0, 0, 0, 0};
    bool series = false;
    hip_F_f32<MASK>(u, C, Fm, Fc, series);
    for (int l = 0; l <= HIP_LMAX; ++l)
        F[l] = (double)Fm[l] + (double)Fc[l] + ((series && l == 0) ? (double)C.ser32[0][0] : 0.0);
}

// ------------------------------------------------------------ F_l (FP64) ---
template <int MASK>
__host__ __device__ __forceinline__ void hip_F_f64_series(double u, const HipCoeffs &C, double *F)
{
    const double x = u * u;
#pragma unroll
    for (int l = 0; l <= HIP_LMAX; ++l) {
        if (!(MASK & (1 << l))) continue;
        double acc = C.ser64[l][HIP_F64_NSER - 1];
#pragma unroll
        for (int s = HIP_F64_NSER - 2; s >= 0; --s) acc = fma(acc, x, C.ser64[l][s]);
        double ul = 1.0;
#pragma unroll
        for (int q = 0; q < l; ++q) ul *= u;
        F[l] = acc * ul;
    }
}

template <int MASK>
__host__ __device__ __forceinline__ void hip_F_f64_closed(double u, double s, double c, const HipCoeffs &C, double *F)
{
    const double w = 1.0 / u;
    const double w2 = w * w;
    const double w3 = w2 * w;
    double si = 0.0;
    if (MASK & ((1 << 2) | (1 << 4))) {
        if (u < HIP_F64_USI) {
            const double x = u * u;
            double acc = C.siser64[HIP_F64_NSISER - 1];
#pragma unroll 4
            for (int n = HIP_F64_NSISER - 2; n >= 0; --n) acc = fma(acc, x, C.siser64[n]);
            si = acc * u;
        } else {
            const double t = (HIP_F64_USI * HIP_F64_USI) * w2;
            double pf = C.sif64[HIP_F64_SIDEG], pg = C.sig64[HIP_F64_SIDEG];
#pragma unroll
            for (int q = HIP_F64_SIDEG - 1; q >= 0; --q) {
                pf = fma(pf, t, C.sif64[q]);
                pg = fma(pg, t, C.sig64[q]);
            }
            si = HIP_HALF_PI_D - w * fma(pf, c, w * pg * s);
        }
    }
    if (MASK & 1) F[0] = fma(w3, s, -w2 * c);
    if (MASK & 2) F[1] = fma(w3, 2.0 - 2.0 * c, -w2 * s);
    if (MASK & 4) F[2] = fma(w3, fma(3.0, si, -4.0 * s), w2 * c);
    if (MASK & 8) F[3] = fma(w2, s, w3 * fma(7.0, c, 8.0 - 15.0 * w * s));
    if (MASK & 16) F[4] = fma(w3, fma(fma(-52.5, w2, 11.0), s, 7.5 * si), w2 * fma(52.5, w2, -1.0) * c);
}

template <int MASK>
__host__ __device__ __forceinline__ void hip_F_f64(double u, const HipCoeffs &C, double *F)
{
    if (u < HIP_F64_USMALL) {
        hip_F_f64_series<MASK>(u, C, F);
        return;
    }
    double s, c;
#ifdef __CUDA_ARCH__
    sincos(u, &s, &c);
#else
    s = sin(u);
    c = cos(u);
#endif
    hip_F_f64_closed<MASK>(u, s, c, C, F);
}

// Host-side construction of the coefficient table (FP64 fits; hip_tables.cpp).
void hip_build_coeffs(HipCoeffs *C);
const HipCoeffs &hip_host_coeffs();

// Power-spectrum pair pass by Legendre moments of the separation.
//
// The pair sum of Sec. 3 asks, for every bin edge k_e and multipole l, for
//     S_l(k_e) = sum_pairs omega L_l(mu) f_e(r),   f_e(r) = k_e^3 F_l(r k_e),
// (omega = w_i w_j W(r/R0); the edge sums the direct kernel accumulates).  f_e is
// an entire function of r, so on a short interval [c dc, (c+1) dc) it is a
// rapidly converging Legendre series f_e(r) = sum_m a^{e}_{c m} P_m(t), t the
// position in the interval mapped to [-1, 1].  Hence
//     S_l(k_e) = sum_c sum_m a^{e l}_{c m} M^l_{c m},  M^l_{c m} = sum_{pairs in c} omega L_l(mu) P_m(t),
// and the pair loop only accumulates the moments M (HIP_PM_M per bin and l)
// instead of evaluating every edge: O(M n_l) per pair instead of O(n_e n_l).
// The coefficients a come from 24-point Gauss-Legendre projection of f_e in FP64
// (once per call), the final contraction is FP64.  f_e is band-limited (F_l(u)
// is an average of j_l(u y) over y in [0, 1], so its spectrum in r lies in
// [-k_e, k_e]); on an interval of half-width h its m-th Legendre coefficient is
// therefore at most (2m+1) max|j_m(k h)| ~ (2m+1) (k h)^m / (2m+1)!! times the
// spectral mass.  With dc = R0 / n_c (rounded up to 16 significant bits) and
// n_c >= R0 k_max / 4, k h <= 2 and the first neglected term (m = 16) is below
// ~4e-13 of f: exact for both precisions.  The moments are those of the scaled
// polynomials R_m = d_m P_m, whose recurrence has exact constants.  The FP32
// path keeps per CTA in shared memory each moment as an exact fixed-point sum
// (two 32-bit integer words, hip_pm_add), folded into FP64 every HIP_PM_FOLD
// pairs; the per-pair terms are formed without an error common to many pairs
// (exact interval origins, split reciprocals, exact recurrence constants), so
// what FP32 leaves is rounding that averages out over the pairs.
#define HIP_PAIR_UPLOAD hip_upload_coeffs_moments
#include "hip_pair_kernel.cuh"

#include <vector>

#include "hip_moments.h"

#define HIP_PM_NG 24
#define HIP_PM_MAXW 8      // warps of a CTA: 4 or 8 (template NW, chosen at launch)
#define HIP_PM_FOLD 16384  // most pairs a CTA adds into its FP32 moments before folding them to FP64
#define HIP_PM_TILE 128    // particles per staged tile of a cell
// an epoch (the pairs between two folds) holds at most HIP_PM_FOLD - 1 + one tile pair
static_assert(HIP_PM_FOLD + HIP_PM_TILE * HIP_PM_TILE <= 32768, "fixed-point moment words could overflow");
#define HIP_PM_QCAP 64     // queue ring: < 32 pairs plus one ballot round of <= 32
#define HIP_PM_PST 17      // row stride of the P_m(t) table (odd: conflict-free stores by row)

__constant__ double c_pm_gw[HIP_PM_NG];           // Gauss-Legendre weights on [-1, 1]
__constant__ double c_pm_gx[HIP_PM_NG];           // and nodes
__constant__ double c_pm_P[HIP_PM_NG][HIP_PM_M];  // P_m at the nodes

cudaError_t hip_upload_pm_tables()
{
    void hip_gauss_legendre(int n, std::vector<double> &x, std::vector<double> &w);
    std::vector<double> x, w;
    hip_gauss_legendre(HIP_PM_NG, x, w);
    double P[HIP_PM_NG][HIP_PM_M];
    for (int g = 0; g < HIP_PM_NG; ++g) {
        P[g][0] = 1.0;
        P[g][1] = x[g];
        for (int m = 1; m + 1 < HIP_PM_M; ++m) P[g][m + 1] = ((2.0 * m + 1.0) * x[g] * P[g][m] - m * P[g][m - 1]) / (m + 1.0);
    }
    cudaError_t e = cudaMemcpyToSymbol(c_pm_gw, w.data(), sizeof(double) * HIP_PM_NG);
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_pm_gx, x.data(), sizeof(double) * HIP_PM_NG);
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_pm_P, P, sizeof(P));
    return e;
}

// a[((il n_e + e) n_c + c) M + m] = (2m+1)/2 int_{-1}^{1} f_e(r(t)) P_m(t) dt / d_m,
// one thread per (edge, interval): the coefficients of the scaled polynomials
// R_m = d_m P_m whose moments the pair pass accumulates.
__global__ void k_pm_coeffs(const double *__restrict__ kedge, int n_e, int n_c, double dc, int n_ell, double *a)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n_e * n_c) return;
    const int e = idx / n_c, c = idx - e * n_c;
    const double k = kedge[e], k3 = k * k * k;
    double acc[3][HIP_PM_M];
#pragma unroll
    for (int il = 0; il < 3; ++il)
#pragma unroll
        for (int m = 0; m < HIP_PM_M; ++m) acc[il][m] = 0.0;
    for (int g = 0; g < HIP_PM_NG; ++g) {
        const double r = (c + 0.5 * (1.0 + c_pm_gx[g])) * dc;
        double F[5];
        hip_F_f64<21>(r * k, c_coeffs, F);
        const double s = k3 * c_pm_gw[g];
        const double f0 = s * F[0], f2 = s * F[2], f4 = s * F[4];
#pragma unroll
        for (int m = 0; m < HIP_PM_M; ++m) {
            const double p = c_pm_P[g][m];
            acc[0][m] = fma(f0, p, acc[0][m]);
            acc[1][m] = fma(f2, p, acc[1][m]);
            acc[2][m] = fma(f4, p, acc[2][m]);
        }
    }
    for (int il = 0; il < n_ell; ++il)
#pragma unroll
        for (int m = 0; m < HIP_PM_M; ++m)
            a[(((size_t)il * n_e + e) * n_c + c) * HIP_PM_M + m] = 0.5 * (2.0 * m + 1.0) * acc[il][m] / hip_leg_scale(m);
}

// Staging of the pair pass: tiles of the two cells (shared by the CTA: offsets
// and primary flag packed for one 16-byte load, weights apart) and, per warp, a
// ring queue of accepted pairs (tile indices only) and the stage of one drain:
// the pairs in interval order with omega L_l, their interval, and P_m(t).
template <typename T>
struct __align__(16) PmPt {
    T x, y, z;
    T in;  // 1 if the particle is in the primary range, else 0
};
template <typename T>
struct PmTiles {
    PmPt<T> h[HIP_PM_TILE], n[HIP_PM_TILE];
    float hw[HIP_PM_TILE], nw[HIP_PM_TILE];
};
template <typename T>
struct __align__(16) PmRow {
    T o0, o2, o4;  // omega L_0, omega L_2, omega L_4
    int c;         // interval
};
template <typename T>
struct PmStage {
    PmRow<T> row[32];
    T P[32 * HIP_PM_PST];  // P_m(t) of row s at s HIP_PM_PST + m
    int q[HIP_PM_QCAP];    // queued pairs: home index << 9 | neighbour index << 2 | ordered pairs counted
};

// Accumulator of the CTA's moments in shared memory.  FP64: the sums.  FP32: a
// 64-bit fixed-point sum per moment held in two 32-bit words, so that every add
// is a native 32-bit integer atomic and the CTA's sums are exact (independent
// of the order of the adds); the unit is fixed per catalog (hip_pm_units).
template <typename T>
struct PmAcc {
    using type = double;
    static constexpr int words = 1;
};
template <>
struct PmAcc<float> {
    using type = unsigned;
    static constexpr int words = 2;
};
template <typename T>
using PmA = typename PmAcc<T>::type;

// Words of the CTA's moment array for n_cp intervals: [3][M][n_cp], and for FP32
// the low words after the high ones.
template <typename T>
__host__ __device__ constexpr int hip_pm_words(int n_cp)
{
    return 3 * HIP_PM_M * n_cp * PmAcc<T>::words;
}

// Shared moment add of a run sum v.  FP32: x = v C (C = 2^s, the catalog's
// units per value of this moment order, so x is exact); for |x| <= 2^33 it is
// rounded to the integer 2^17 a + b with a = rint(x 2^-17) and b = rint(x - 2^17 a)
// in [-2^16, 2^16]: a goes to the word at M, b to the word at M + lo_off (both
// signed), and with fewer than 2^15 adds between folds neither sum leaves the
// int32 range.  Both roundings are additions of 1.5 2^23 (the integer lands in
// the low significand bits, read back by one integer subtraction), and
// x - 2^17 a is exact (at most 2^16 in magnitude and a multiple of x's last
// place).  With CHECK a larger run sum (far above the catalog's typical term)
// goes to the FP64 total G[gi] instead; the drain takes the unchecked form when
// a bound on its run sums rules that out (hip_pm_walk).
template <bool CHECK>
__device__ __forceinline__ void hip_pm_add(unsigned *M, float v, int lo_off, float C, double *G, int gi)
{
    const float x = __fmul_rn(v, C);
    if (CHECK && !(fabsf(x) <= 8589934592.0f)) {  // 2^33
        atomicAdd(G + gi, (double)v);
        return;
    }
    const float ab = fmaf(x, 7.62939453125e-06f, 12582912.0f);  // 1.5 2^23 + rint(x 2^-17)
    const float a = __fsub_rn(ab, 12582912.0f);                  // exact
    const float bb = __fadd_rn(fmaf(a, -131072.0f, x), 12582912.0f);
    atomicAdd(reinterpret_cast<int *>(M), __float_as_int(ab) - 0x4B400000);
    atomicAdd(reinterpret_cast<int *>(M) + lo_off, __float_as_int(bb) - 0x4B400000);
}
// The same add shared by the two lanes of a pair that hold the same v (the l = 4
// sums of moment m sit in lanes m and 16 + m): lane g = 0 adds the word at M,
// g = 1 the word at M + lo_off, so one atomic instruction of the warp covers
// both words of all 16 sums.
template <bool CHECK>
__device__ __forceinline__ void hip_pm_add_half(unsigned *M, float v, int lo_off, float C, double *G, int gi, int g)
{
    const float x = __fmul_rn(v, C);
    if (CHECK && !(fabsf(x) <= 8589934592.0f)) {  // 2^33
        if (g == 0) atomicAdd(G + gi, (double)v);
        return;
    }
    const float ab = fmaf(x, 7.62939453125e-06f, 12582912.0f);
    const float a = __fsub_rn(ab, 12582912.0f);
    const float bb = __fadd_rn(fmaf(a, -131072.0f, x), 12582912.0f);
    atomicAdd(reinterpret_cast<int *>(M) + (g ? lo_off : 0), __float_as_int(g ? bb : ab) - 0x4B400000);
}
template <bool CHECK>
__device__ __forceinline__ void hip_pm_add_half(double *M, double v, int, float, double *, int, int g)
{
    if (g == 0) atomicAdd(M, v);
}
template <bool CHECK>
__device__ __forceinline__ void hip_pm_add(double *M, double v, int, float, double *, int)
{
    atomicAdd(M, v);
}

// Value of moment word i (n words per part) as FP64, clearing it.
__device__ __forceinline__ double hip_pm_take(unsigned *M, int i, int n, float C)
{
    const double v = ((double)(int)M[i] * 131072.0 + (double)(int)M[i + n]) * (double)(1.0f / C);  // C = 2^s
    M[i] = 0u;
    M[i + n] = 0u;
    return v;
}
__device__ __forceinline__ double hip_pm_take(double *M, int i, int, float)
{
    const double v = M[i];
    M[i] = 0.0;
    return v;
}

// Per-launch constants of the drain: the interval width dc (a 16-bit significand,
// so c dc is exact in FP32 for c < 256), 1 / dc, and 2 / dc and 1 / R0 each as a
// rounded value plus its residual, so that t and r / R0 carry no bias common to
// all pairs.
template <typename T>
struct PmScale {
    T dc, inv_dc, ihd, ihd_lo, iR, iR_lo;
    __device__ PmScale(T dc_, T R0)
    {
        dc = dc_;
        inv_dc = T(1) / dc;
        ihd = T(2) / dc;
        ihd_lo = fma(-dc, ihd, T(2)) / dc;
        iR = T(1) / R0;
        iR_lo = fma(-R0, iR, T(1)) / R0;
    }
};

// Shared state of a CTA's FP32 moment sums: the fixed-point scales C[m] of the
// current catalog and the per-warp pair counts since the last count.
struct PmEpoch {
    int drained[HIP_PM_MAXW];
    int row;  // next home row of the current tile pair (taken by the warps one at a time)
    float C[HIP_PM_M];
    float Smax;  // a drain whose sum of |omega| is at most this keeps every run sum below 2^32 units
};

// Frame of one work item: the neighbour cell's offset from the home cell (hi + lo).
template <typename T>
struct PmShift {
    T x, y, z, xl, yl, zl;
};

// The moment walk of a drain: lane 16 g + m runs over the n staged pairs in
// interval order with register sums and adds a sum to the moment array once per
// interval run (g = 0: l = 0, g = 1: l = 2, and both l = 4, whose two words the
// lane pair m, 16 + m adds with one atomic instruction), unrolled UNR times (the
// batched kernel, short of registers, takes 4, the single-catalog one 8).
template <typename T, int MASK, bool CHECK, int UNR>
__device__ __forceinline__ void hip_pm_walk(const PmStage<T> &sg, int n, int lane, PmA<T> *M, int n_cp, int n_c,
                                            const float *Cg, double *Mg)
{
    const int m = lane & 15, g = lane >> 4;
    PmA<T> *Ma = M + (size_t)(g * HIP_PM_M + m) * n_cp;
    PmA<T> *Mb = M + (size_t)(2 * HIP_PM_M + m) * n_cp;
    const bool use_a = (g == 0) || (MASK & 4);
    const bool use_b = (MASK & 16) != 0;  // both lanes m and 16 + m sum l = 4 of moment m
    const int lo_off = 3 * HIP_PM_M * n_cp;
    const float C = Cg[m];
    const int ga = (g * HIP_PM_M + m) * n_c, gb = (2 * HIP_PM_M + m) * n_c;  // rows of the FP64 totals
    T sa = T(0), sb = T(0);
    int cur = sg.row[0].c;
#pragma unroll UNR
    for (int s = 0; s < n; ++s) {
        const PmRow<T> r = sg.row[s];
        if (r.c != cur) {  // warp-uniform
            if (use_a) hip_pm_add<CHECK>(Ma + cur, sa, lo_off, C, Mg, ga + cur);
            if (use_b) hip_pm_add_half<CHECK>(Mb + cur, sb, lo_off, C, Mg, gb + cur, g);
            sa = T(0);
            sb = T(0);
            cur = r.c;
        }
        const T p = sg.P[s * HIP_PM_PST + m];
        sa += (g ? r.o2 : r.o0) * p;
        sb += r.o4 * p;
    }
    if (use_a) hip_pm_add<CHECK>(Ma + cur, sa, lo_off, C, Mg, ga + cur);
    if (use_b) hip_pm_add_half<CHECK>(Mb + cur, sb, lo_off, C, Mg, gb + cur, g);
}

// Moments of the n (1..32) queued pairs at ring positions head, head + 1, ...:
// M[(il M + m) n_cp + c] += omega L_l P_m(t).  Lane p first evaluates queued
// pair p from the tiles (exact separation, mu, W, interval, t); the pairs are
// then sorted by interval across the warp (bitonic network on (interval, lane)
// keys), lane s tabulates P_m(t) of the s-th pair, and finally the lanes run
// over the moments (lane = 16 g + m: g = 0 sums l = 0 and l = 4, g = 1 sums
// l = 2), walk the sorted pairs with register sums, and add a sum to the shared
// array once per interval run, at 48 distinct addresses.
template <typename T, int MASK, int UNR>
__device__ __forceinline__ void hip_pm_drain(PmStage<T> &sg, const PmTiles<T> &tl, const PmShift<T> &sh, int los,
                                             int head, int n, int lane, PmA<T> *M, int n_cp, int n_c,
                                             const PmScale<T> &ps, const float *Cg, float Smax, double *Mg,
                                             unsigned long long &cnt)
{
    int key = ((HIP_PM_NCMAX + 1) << 5) | lane;  // empty lanes sort last
    T t = T(0), o0 = T(0), o2 = T(0), o4 = T(0);
    if (lane < n) {
        const int e = sg.q[(head + lane) & (HIP_PM_QCAP - 1)];
        const int il = e >> 9, jl = (e >> 2) & 127, mult = e & 3;
        const PmPt<T> h = tl.h[il], nb = tl.n[jl];
        const T xi = h.x - sh.x, yi = h.y - sh.y, zi = h.z - sh.z;
        const T xil = hip_low(h.x, -sh.x, xi) - sh.xl, yil = hip_low(h.y, -sh.y, yi) - sh.yl,
                zil = hip_low(h.z, -sh.z, zi) - sh.zl;
        const T ddx = xi - nb.x, ddy = yi - nb.y, ddz = zi - nb.z;
        T r, rl, dlo;
        hip_pair_sep(xi, xil, yi, yil, zi, zil, nb.x, nb.y, nb.z, ddx, ddy, ddz, los, &r, &rl, &dlo);
        // mu and W from the full separation (hi + lo): the low parts carry the cell
        // shift's rounding, common to all pairs across a periodic face
        const T rr = r + rl;
        const T mu = ((los == 0 ? ddx : (los == 1 ? ddy : ddz)) + dlo) / rr;
        T l2, l4;
        hip_legendre24<T>(mu, l2, l4);
        // w_i w_j times the ordered pairs counted, formed in T (exact in FP64), then W
        o0 = (T(tl.hw[il]) * T(tl.nw[jl]) * T(mult)) * hip_W<T>(fma(rr, ps.iR_lo, rr * ps.iR));
        o2 = o0 * l2;
        o4 = o0 * l4;
        const int c = min((int)(r * ps.inv_dc), n_c - 1);
        // t in [-1, 1]: c dc is exact and r - c dc too for c >= 1 (Sterbenz), the low part rl added after
        const T d = (r - T(c) * ps.dc) + rl;
        t = fma(d, ps.ihd_lo, d * ps.ihd) - T(1);
        key = (c << 5) | lane;
        cnt += (unsigned long long)mult;
    }
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1)
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            const int other = __shfl_xor_sync(0xffffffffu, key, j);
            const bool keep_min = ((lane & j) == 0) == ((lane & k) == 0);
            key = keep_min ? min(key, other) : max(key, other);
        }
    const int src = key & 31;
    const T ts = __shfl_sync(0xffffffffu, t, src);
    PmRow<T> rw;
    rw.o0 = __shfl_sync(0xffffffffu, o0, src);
    rw.o2 = __shfl_sync(0xffffffffu, o2, src);
    rw.o4 = __shfl_sync(0xffffffffu, o4, src);
    rw.c = key >> 5;
    if (lane < n) {
        T *P = sg.P + lane * HIP_PM_PST;
        T p0 = T(1), p1 = ts;
        P[0] = p0;
        P[1] = p1;
#pragma unroll
        for (int m = 1; m + 1 < HIP_PM_M; ++m) {
            // the scaled polynomials R_m = d_m P_m (exact recurrence constants)
            const T p2 = hip_leg_alpha<T>(m) * ts * p1 - hip_leg_beta<T>(m) * p0;
            p0 = p1;
            p1 = p2;
            P[m + 1] = p2;
        }
        sg.row[lane] = rw;
    }
    // |run sum| <= S d_m with S the drain's sum of |omega| (|L_l| <= 1, |R_m| <= d_m)
    T S = o0 < T(0) ? -o0 : o0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) S += __shfl_xor_sync(0xffffffffu, S, o);
    __syncwarp();
    if (sizeof(T) == 8 || S <= T(Smax))  // warp-uniform
        hip_pm_walk<T, MASK, false, UNR>(sg, n, lane, M, n_cp, n_c, Cg, Mg);
    else
        hip_pm_walk<T, MASK, true, UNR>(sg, n, lane, M, n_cp, n_c, Cg, Mg);
    __syncwarp();
}

// Adds the CTA's moment array into the FP64 totals Mg ([3 M][n_c]) and clears it.
template <typename T>
__device__ __forceinline__ void hip_pm_fold(PmA<T> *M, int n_cp, int n_c, double *Mg, const float *C)
{
    const int n = 3 * HIP_PM_M * n_cp;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int row = i / n_cp, c = i - row * n_cp;
        const double v = hip_pm_take(M, i, n, C[row & (HIP_PM_M - 1)]);
        if (c < n_c && v != 0.0) atomicAdd(&Mg[(size_t)row * n_c + c], v);
    }
}

// Adds the per-warp pair counts (written before the barrier that precedes this
// call) into since_fold and, at `fold` pairs (<= HIP_PM_FOLD), folds the FP32 moments; called by
// all threads between a tile pair's barriers, when no warp is draining.  A tile
// pair adds at most HIP_PM_TILE^2 pairs, so a fold epoch holds fewer than 2^15.
// (The FP64 path folds once per catalog.)
template <typename T>
__device__ __forceinline__ void hip_pm_count(PmEpoch &ep, PmA<T> *M, int n_cp, int n_c, double *Mg, int &since_fold,
                                             int fold)
{
    if (sizeof(T) == 4) {
#pragma unroll
        for (int w = 0; w < HIP_PM_MAXW; ++w) since_fold += ep.drained[w];  // unused entries stay 0
        if (since_fold >= fold) {  // CTA-uniform
            hip_pm_fold<T>(M, n_cp, n_c, Mg, ep.C);
            since_fold = 0;
        }
    }
}

// Fixed-point scales of a catalog from the mean |w| of its particles (wabs =
// sum |w|, n particles): with mean |w|^2 < 2^e and d_m <= 2^D, C_m = 2^(25 - e - D)
// puts a typical term omega L_l R_m at ~2^23 units (rounding below FP32's, and
// unbiased); a drain whose sum of |omega| stays below Smax (2^7 mean |w|^2 and
// more: 32 pairs of weight products up to ~4 mean |w|^2) keeps every run sum
// within the 2^32-unit range of one add.  Called by threads 0..15; the caller
// synchronises.
__device__ __forceinline__ void hip_pm_units(PmEpoch &ep, const double *wabs, long long n)
{
    const int m = threadIdx.x;
    const double wm = n > 0 ? *wabs / (double)n : 0.0;
    int e = 0;
    frexp(wm > 0.0 ? wm * wm : 1.0, &e);
    int D = 0;
    while ((double)(1 << D) < hip_leg_scale(m)) ++D;
    const int s = min(max(25 - e - D, -126), 127);
    ep.C[m] = ldexpf(1.0f, s);
    if (m == 0) {  // S d_k 2^s_k <= S 2^(D_k + s_k) <= 2^32 for every order k (a factor 2 to spare
                   // for |t| a rounding beyond 1 and the FP32 sum S)
        int smax = -1000;
        for (int k = 0; k < HIP_PM_M; ++k) {
            int Dk = 0;
            while ((double)(1 << Dk) < hip_leg_scale(k)) ++Dk;
            smax = max(smax, Dk + min(max(25 - e - Dk, -126), 127));
        }
        ep.Smax = ldexpf(1.0f, min(max(32 - smax, -126), 127));
    }
}

// One work item (home cell, half-shell shift; item counts within the catalog):
// the CTA stages the two cells' tiles, its warps take the home particles (DYN:
// one at a time from a shared counter, so that they reach the next barrier
// together; else warp w takes w, w + NW, ...: cheaper on small tiles), test
// candidates one per lane and queue the accepted ones as tile indices; 32
// queued pairs (and whatever is queued when a tile pair is done) are drained
// into the CTA's moment array M.  Called by all threads of the CTA.
template <typename T, int MASK, int NW, bool DYN>
__device__ __forceinline__ void hip_pm_item(const CellList<T> &cl, long long p0, long long p1, int los, int item,
                                            PmTiles<T> &tl, PmStage<T> &sg, PmEpoch &ep, PmA<T> *M, int n_cp, int n_c,
                                            T R0, T dc, double *Mg, unsigned long long &cnt, int &drained,
                                            int &since_fold, int fold)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned lt_mask = (1u << lane) - 1u;
    const T R0sq = R0 * R0;
    const PmScale<T> ps(dc, R0);
    const int n_c3 = cl.n_c;
    const int c = item / HIP_NSHIFT, q = item - c * HIP_NSHIFT;
    const int cx = c / (n_c3 * n_c3), cy = (c / n_c3) % n_c3, cz = c % n_c3;
    const int dx = c_shift[q][0], dy = c_shift[q][1], dz = c_shift[q][2];
    const int nb = (((cx + dx + n_c3) % n_c3) * n_c3 + (cy + dy + n_c3) % n_c3) * n_c3 + (cz + dz + n_c3) % n_c3;
    PmShift<T> sh;
    hip_cell_shift(cl, cx, dx, sh.x, sh.xl);
    hip_cell_shift(cl, cy, dy, sh.y, sh.yl);
    hip_cell_shift(cl, cz, dz, sh.z, sh.zl);
    const int a0 = cl.cell_start[c], a1 = cl.cell_start[c + 1];
    const int b0 = cl.cell_start[nb], b1 = cl.cell_start[nb + 1];
    const bool self = (q == 0);
    for (int hb = a0; hb < a1; hb += HIP_PM_TILE) {
        const int hn = min(HIP_PM_TILE, a1 - hb);
        __syncthreads();
        for (int i = threadIdx.x; i < hn; i += blockDim.x) {
            const long long oi = cl.idx[hb + i];
            PmPt<T> p;
            p.x = cl.x[hb + i];
            p.y = cl.y[hb + i];
            p.z = cl.z[hb + i];
            p.in = (oi >= p0 && oi < p1) ? T(1) : T(0);
            tl.h[i] = p;
            tl.hw[i] = cl.w[hb + i];
        }
        for (int nbs = self ? hb : b0; nbs < b1; nbs += HIP_PM_TILE) {
            const int nn = min(HIP_PM_TILE, b1 - nbs);
            if (lane == 0) ep.drained[warp] = drained;
            drained = 0;
            __syncthreads();
            hip_pm_count<T>(ep, M, n_cp, n_c, Mg, since_fold, fold);
            if (threadIdx.x == 0) ep.row = 0;
            for (int i = threadIdx.x; i < nn; i += blockDim.x) {
                const long long oi = cl.idx[nbs + i];
                PmPt<T> p;
                p.x = cl.x[nbs + i];
                p.y = cl.y[nbs + i];
                p.z = cl.z[nbs + i];
                p.in = (oi >= p0 && oi < p1) ? T(1) : T(0);
                tl.n[i] = p;
                tl.nw[i] = cl.w[nbs + i];
            }
            __syncthreads();
            const bool same = self && (nbs == hb);
            int qn = 0;  // queued pairs of this warp (ring head 0 after each partial drain)
            int qh = 0;
            for (int il = warp;;) {  // DYN: home rows one at a time from the shared counter
                if (DYN) {
                    if (lane == 0) il = atomicAdd(&ep.row, 1);
                    il = __shfl_sync(0xffffffffu, il, 0);
                }
                if (il >= hn) break;
                const PmPt<T> h = tl.h[il];
                const T xi = h.x - sh.x, yi = h.y - sh.y, zi = h.z - sh.z;
                const int ini = (int)h.in;
                for (int jb = same ? il + 1 : 0; jb < nn; jb += 32) {
                    const int jl = jb + lane;
                    bool ok = false;
                    int mult = 0;
                    if (jl < nn) {
                        const PmPt<T> p = tl.n[jl];
                        const T ddx = xi - p.x, ddy = yi - p.y, ddz = zi - p.z;
                        const T r2 = ddx * ddx + ddy * ddy + ddz * ddz;
                        mult = ini + (int)p.in;
                        ok = (r2 < R0sq) && (r2 > T(0)) && (mult > 0);
                    }
                    const unsigned bal = __ballot_sync(0xffffffffu, ok);
                    if (ok) sg.q[(qh + qn + __popc(bal & lt_mask)) & (HIP_PM_QCAP - 1)] = (il << 9) | (jl << 2) | mult;
                    qn += __popc(bal);
                    if (qn >= 32) {
                        __syncwarp();
                        hip_pm_drain<T, MASK, DYN ? 8 : 4>(sg, tl, sh, los, qh, 32, lane, M, n_cp, n_c, ps, ep.C,
                                                           ep.Smax, Mg, cnt);
                        qh = (qh + 32) & (HIP_PM_QCAP - 1);
                        qn -= 32;
                        drained += 32;
                    }
                }
                if (!DYN) il += NW;
            }
            if (qn > 0) {  // the tiles change after this tile pair
                __syncwarp();
                hip_pm_drain<T, MASK, DYN ? 8 : 4>(sg, tl, sh, los, qh, qn, lane, M, n_cp, n_c, ps, ep.C, ep.Smax, Mg, cnt);
                drained += qn;
            }
        }
    }
}

// The pair pass of one catalog: persistent CTAs take work items from the
// counter (hip_pm_item).  The moment array lives in dynamic shared memory
// ([3][M][n_cp], T, n_cp = n_c rounded up to odd so the 16 moments of one
// interval fall in distinct banks; FP32 adds the remainder terms after it) and
// is folded into the FP64 totals Mg every HIP_PM_FOLD pairs and when the weight
// bound rises (FP32, at tile-pair boundaries), and at the end.
template <typename T, int MASK, int NW>
__global__ void __launch_bounds__(NW * 32, 32 / NW)  // <= 64 registers: 32 warps per SM fit
    k_power_moments(CellList<T> cl, PowerKernelArgs a, T R0, int n_c, T dc, double *Mg)
{
    __shared__ PmTiles<T> tl;
    __shared__ PmStage<T> stages[NW];
    __shared__ int s_item;
    __shared__ PmEpoch ep;
    extern __shared__ __align__(16) unsigned char pm_raw[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int n_cp = n_c | 1;
    PmA<T> *M = reinterpret_cast<PmA<T> *>(pm_raw);
    for (int i = threadIdx.x; i < hip_pm_words<T>(n_cp); i += blockDim.x) M[i] = PmA<T>(0);
    if (threadIdx.x < HIP_PM_M) hip_pm_units(ep, Mg + hip_pm_mg_doubles(n_c) - 1, a.n_part);
    double *Mr = Mg + (size_t)(blockIdx.x % HIP_PM_REPL) * 3 * HIP_PM_M * n_c;  // this CTA's replica
    if (threadIdx.x < HIP_PM_MAXW) ep.drained[threadIdx.x] = 0;
    unsigned long long cnt = 0;
    int since_fold = 0, drained = 0;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_item = atomicAdd(a.work_counter, 1);
        __syncthreads();
        const int item = s_item;
        if (item >= a.n_items) break;
        hip_pm_item<T, MASK, NW, true>(cl, a.p0, a.p1, a.los, item, tl, stages[warp], ep, M, n_cp, n_c, R0, dc, Mr, cnt,
                                 drained, since_fold, HIP_PM_FOLD);
    }
    __syncthreads();
    hip_pm_fold<T>(M, n_cp, n_c, Mr, ep.C);
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    if (lane == 0 && cnt) atomicAdd(a.npairs, cnt);
}

// The batched pair pass: all catalogs' work items end to end in one persistent
// launch (l = 0, 2, 4 always).  A CTA's items increase, so it moves through the
// catalogs in order; when it moves on it folds its moments and pair count into
// the catalog it leaves.  The dynamic array is sized for the largest n_c.
template <typename T, int NW>
__global__ void __launch_bounds__(NW * 32, 32 / NW)
    k_power_moments_batched(const PmCat<T> *__restrict__ cats, int n_cats, int n_items, int n_c_max, int *counter,
                            int fold)
{
    __shared__ PmTiles<T> tl;
    __shared__ PmStage<T> stages[NW];
    __shared__ int s_item;
    __shared__ PmEpoch ep;
    extern __shared__ __align__(16) unsigned char pm_raw[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    PmA<T> *M = reinterpret_cast<PmA<T> *>(pm_raw);
    for (int i = threadIdx.x; i < hip_pm_words<T>(n_c_max | 1); i += blockDim.x) M[i] = PmA<T>(0);
    if (threadIdx.x < HIP_PM_MAXW) ep.drained[threadIdx.x] = 0;
    unsigned long long cnt = 0;
    int since_fold = 0, drained = 0;
    int ci = -1;
    __shared__ PmCat<T> cat;  // the current catalog (shared: frees the registers it would take)
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
        __syncthreads();
        const int item = s_item;
        const bool done = item >= n_items;
        int nci = ci < 0 ? 0 : ci;
        if (!done)
            while (nci < n_cats - 1 && item >= cats[nci].item_end) ++nci;
        if (done || nci != ci) {  // CTA-uniform
            if (ci >= 0) {
                __syncthreads();
                hip_pm_fold<T>(M, cat.n_c | 1, cat.n_c, cat.Mg + (size_t)(blockIdx.x % HIP_PM_REPL) * 3 * HIP_PM_M * cat.n_c,
                               ep.C);  // leaves M zero
                unsigned long long c2 = cnt;
                for (int o = 16; o > 0; o >>= 1) c2 += __shfl_xor_sync(0xffffffffu, c2, o);
                if (lane == 0 && c2) atomicAdd(cat.npairs, c2);
                cnt = 0;
                since_fold = 0;
            }
            if (done) break;
            ci = nci;
            __syncthreads();  // the fold above has read the previous catalog and its scales
            if (threadIdx.x == 0) cat = cats[ci];
            __syncthreads();
            if (threadIdx.x < HIP_PM_M) hip_pm_units(ep, cat.Mg + hip_pm_mg_doubles(cat.n_c) - 1, cat.n_part);
        }
        hip_pm_item<T, 21, NW, false>(cat.cl, cat.p0, cat.p1, cat.los, item - cat.item_begin, tl, stages[warp], ep, M,
                           cat.n_c | 1, cat.n_c, cat.R0, cat.dc,
                           cat.Mg + (size_t)(blockIdx.x % HIP_PM_REPL) * 3 * HIP_PM_M * cat.n_c, cnt, drained,
                           since_fold, fold);
    }
}

// S[il][e] = sum_c sum_m a[il][e][c][m] Mg[il][m][c] by one 256-thread block,
// written as row[il n_e + e] (one partial row [3][n_e] of the power finalize).
__device__ __forceinline__ void hip_pm_contract_block(const double *__restrict__ a, const double *__restrict__ Mg,
                                                      int n_e, int n_c, int il, int e, double *row)
{
    __shared__ double red[256];
    const double *ae = a + ((size_t)il * n_e + e) * n_c * HIP_PM_M;
    const double *mg = Mg + (size_t)il * HIP_PM_M * n_c;
    const size_t rs = (size_t)3 * HIP_PM_M * n_c;  // replica stride
    double acc = 0.0;
    for (int i = threadIdx.x; i < n_c * HIP_PM_M; i += 256) {
        const int c = i / HIP_PM_M, m = i - c * HIP_PM_M;
        double v = 0.0;
        for (int r = 0; r < HIP_PM_REPL; ++r) v += mg[r * rs + (size_t)m * n_c + c];
        acc = fma(ae[i], v, acc);
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) row[il * n_e + e] = red[0];
}

// one block per (il, e)
__global__ void __launch_bounds__(256) k_pm_contract(const double *__restrict__ a, const double *__restrict__ Mg,
                                                     int n_e, int n_c, double *row)
{
    const int il = blockIdx.x / n_e, e = blockIdx.x - il * n_e;
    hip_pm_contract_block(a, Mg, n_e, n_c, il, e, row);
}

// blockIdx.y = catalog, blockIdx.x = il n_e_max + e
__global__ void __launch_bounds__(256) k_pm_contract_batched(const PmContractCat *__restrict__ cc, int n_e_max)
{
    const PmContractCat c = cc[blockIdx.y];
    const int il = blockIdx.x / n_e_max, e = blockIdx.x - il * n_e_max;
    if (il >= c.n_ell || e >= c.n_e) return;
    hip_pm_contract_block(c.coef, c.Mg, c.n_e, c.n_c, il, e, c.row);
}

// Sum of |w| over n particles into *out (zeroed before), for the fixed-point
// scales of the FP32 moment sums.
__device__ __forceinline__ void hip_pm_wabs_part(const float *__restrict__ w, long long n, long long i0,
                                                 long long step, double *out)
{
    __shared__ double red[32];
    double s = 0.0;
    for (long long i = i0; i < n; i += step) s += (double)fabsf(w[i]);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0 && v != 0.0) atomicAdd(out, v);
    }
}
__global__ void __launch_bounds__(256) k_pm_wabs(const float *__restrict__ w, long long n, double *out)
{
    hip_pm_wabs_part(w, n, blockIdx.x * 256ll + threadIdx.x, (long long)gridDim.x * 256, out);
}
// blockIdx.y = catalog
template <typename T>
__global__ void __launch_bounds__(256) k_pm_wabs_batched(const PmCat<T> *__restrict__ cats)
{
    const PmCat<T> &c = cats[blockIdx.y];
    hip_pm_wabs_part(c.cl.w, c.n_part, blockIdx.x * 256ll + threadIdx.x, (long long)gridDim.x * 256,
                     c.Mg + hip_pm_mg_doubles(c.n_c) - 1);
}

// ------------------------------------------------------------------ host ----
int hip_pm_intervals(double R0, double k_max)
{
    const int n = (int)std::ceil(R0 * k_max / 4.0);
    return n < 8 ? 8 : n;
}

double hip_pm_width(double R0, int n_c)
{
    int ex = 0;
    const double f = std::frexp(R0 / n_c, &ex);  // [0.5, 1)
    return std::ldexp(std::ceil(f * 65536.0) / 65536.0, ex);
}

size_t hip_pm_coef_doubles(int n_e, int n_c) { return (size_t)3 * n_e * n_c * HIP_PM_M; }

cudaError_t hip_pm_coeffs(const double *d_kedges, int n_e, int n_ell, double R0, double k_max, double *coef,
                          cudaStream_t st)
{
    const int n_c = hip_pm_intervals(R0, k_max);
    k_pm_coeffs<<<(n_e * n_c + 127) / 128, 128, 0, st>>>(d_kedges, n_e, n_c, hip_pm_width(R0, n_c), n_ell, coef);
    return cudaGetLastError();
}

size_t hip_pm_scratch_bytes(int n_e, int n_c)
{
    return sizeof(double) * ((size_t)n_e + (size_t)3 * n_e * n_c * HIP_PM_M + hip_pm_mg_doubles(n_c)) + 256;
}

template <typename T>
static size_t pm_dyn_smem(int n_c)
{
    return sizeof(PmA<T>) * (size_t)hip_pm_words<T>(n_c | 1);
}

bool hip_pm_applicable(double R0, double k_max, bool fp32)
{
    const int n_c = hip_pm_intervals(R0, k_max);
    if (n_c > HIP_PM_NCMAX) return false;
    const size_t dyn = fp32 ? pm_dyn_smem<float>(n_c) : pm_dyn_smem<double>(n_c);
    const size_t stat = sizeof(PmTiles<double>) + sizeof(PmStage<double>) * HIP_PM_MAXW;
    return dyn + stat <= 220 * 1024;
}

// Warps per CTA: 8 when the cells hold enough particles to keep them busy (the
// shared tiles and moment array then serve more warps, raising occupancy), else
// 4 (sparse catalogs: fewer idle warps at each tile pair's barriers).
static int pm_warps(double per_cell) { return per_cell >= 24.0 ? 8 : 4; }

template <typename T, int MASK, int NW>
static cudaError_t pm_launch_nw(const CellList<T> &cl, const PowerKernelArgs &a, T R0, int n_c, T dc, double *Mg,
                                cudaStream_t st)
{
    const size_t dyn = pm_dyn_smem<T>(n_c);
    cudaError_t e = cudaFuncSetAttribute(k_power_moments<T, MASK, NW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)dyn);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, nb = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_power_moments<T, MASK, NW>, NW * 32, dyn);
    const int grid = sms * (nb < 1 ? 1 : nb);
    k_power_moments<T, MASK, NW><<<grid, NW * 32, dyn, st>>>(cl, a, R0, n_c, dc, Mg);
    return cudaGetLastError();
}
template <typename T, int MASK>
static cudaError_t pm_launch(const CellList<T> &cl, const PowerKernelArgs &a, T R0, int n_c, T dc, double *Mg,
                             cudaStream_t st)
{
    const double per_cell = (double)a.n_part * HIP_NSHIFT / (a.n_items > 0 ? a.n_items : 1);
    return pm_warps(per_cell) == 8 ? pm_launch_nw<T, MASK, 8>(cl, a, R0, n_c, dc, Mg, st)
                                   : pm_launch_nw<T, MASK, 4>(cl, a, R0, n_c, dc, Mg, st);
}

template <typename T>
cudaError_t hip_power_moments(const CellList<T> &cl, const PowerKernelArgs &a, const double *kedges, int n_ell,
                              double R0, void *scratch, double *row, cudaStream_t st)
{
    const int n_e = a.n_e;
    const int n_c = hip_pm_intervals(R0, kedges[n_e - 1]);
    const double dc = hip_pm_width(R0, n_c);  // exact in T
    double *ke = (double *)scratch;
    double *coef = ke + n_e;
    double *Mg = coef + (size_t)3 * n_e * n_c * HIP_PM_M;
    cudaError_t e;
    if ((e = cudaMemcpyAsync(ke, kedges, sizeof(double) * n_e, cudaMemcpyHostToDevice, st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(Mg, 0, sizeof(double) * hip_pm_mg_doubles(n_c), st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(row, 0, sizeof(double) * 3 * n_e, st)) != cudaSuccess) return e;
    k_pm_coeffs<<<(n_e * n_c + 127) / 128, 128, 0, st>>>(ke, n_e, n_c, dc, n_ell, coef);
    if (sizeof(T) == 4) {
        const long long nb = std::min<long long>((a.n_part + 255) / 256, 4 * 152);
        k_pm_wabs<<<(int)(nb < 1 ? 1 : nb), 256, 0, st>>>(cl.w, a.n_part, Mg + hip_pm_mg_doubles(n_c) - 1);
    }
    if (n_ell == 3)
        e = pm_launch<T, 21>(cl, a, (T)R0, n_c, (T)dc, Mg, st);
    else if (n_ell == 2)
        e = pm_launch<T, 5>(cl, a, (T)R0, n_c, (T)dc, Mg, st);
    else
        e = pm_launch<T, 1>(cl, a, (T)R0, n_c, (T)dc, Mg, st);
    if (e != cudaSuccess) return e;
    k_pm_contract<<<n_ell * n_e, 256, 0, st>>>(coef, Mg, n_e, n_c, row);
    return cudaGetLastError();
}
template cudaError_t hip_power_moments<float>(const CellList<float> &, const PowerKernelArgs &, const double *, int,
                                              double, void *, double *, cudaStream_t);
template cudaError_t hip_power_moments<double>(const CellList<double> &, const PowerKernelArgs &, const double *,
                                               int, double, void *, double *, cudaStream_t);

template <typename T, int NW>
static cudaError_t pm_batched_nw(const PmCat<T> *cats, int n_cats, int n_items, int n_c_max, int *counter, int fold,
                                 cudaStream_t st)
{
    if (sizeof(T) == 4) k_pm_wabs_batched<T><<<dim3(64, n_cats), 256, 0, st>>>(cats);
    const size_t dyn = pm_dyn_smem<T>(n_c_max);
    cudaError_t e = cudaFuncSetAttribute(k_power_moments_batched<T, NW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)dyn);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, nb = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_power_moments_batched<T, NW>, NW * 32, dyn);
    const int grid = sms * (nb < 1 ? 1 : nb);
    k_power_moments_batched<T, NW><<<grid, NW * 32, dyn, st>>>(cats, n_cats, n_items, n_c_max, counter, fold);
    return cudaGetLastError();
}

template <typename T>
cudaError_t hip_power_moments_batched(const PmCat<T> *cats, int n_cats, int n_items, int n_c_max, int *counter,
                                      const PmContractCat *cc, int n_e_max, double per_cell, int warps, int fold,
                                      cudaStream_t st)
{
    const int nw = warps == 4 || warps == 8 ? warps : pm_warps(per_cell);
    const int fo = fold >= 1024 && fold <= HIP_PM_FOLD ? fold : HIP_PM_FOLD;
    cudaError_t e = nw == 8 ? pm_batched_nw<T, 8>(cats, n_cats, n_items, n_c_max, counter, fo, st)
                            : pm_batched_nw<T, 4>(cats, n_cats, n_items, n_c_max, counter, fo, st);
    if (e != cudaSuccess) return e;
    k_pm_contract_batched<<<dim3(3 * n_e_max, n_cats), 256, 0, st>>>(cc, n_e_max);
    return cudaGetLastError();
}
template cudaError_t hip_power_moments_batched<float>(const PmCat<float> *, int, int, int, int *,
                                                      const PmContractCat *, int, double, int, int, cudaStream_t);
template cudaError_t hip_power_moments_batched<double>(const PmCat<double> *, int, int, int, int *,
                                                       const PmContractCat *, int, double, int, int, cudaStream_t);

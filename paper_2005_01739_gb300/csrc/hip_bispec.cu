// Bispectrum kernels (Sec. 4 of arXiv:2005.01739).
//
// For every primary p (data particles, then the random catalog) the kernel
// forms, over data neighbours j with 0 < |x_p - x_j| < R0,
//     A^a_lm(p) = sum_j w_j W(r/R0) jbar^a_l(r) R_lm(rhat)        (Eq. AC-def, binned)
//     C^ab_l(p) = sum_j w_j^2 W^2 jbar^a_l(r) jbar^b_l(r)
// with real spherical harmonics R_lm scaled so that sum_m R_lm(u) R_lm(v) =
// L_l(u.v) (the addition theorem with the 4 pi / (2l+1) absorbed; real and
// complex harmonics give the same sum over m), and accumulates
//     T^ab_l += s_p [ sum_m A^a_lm A^b_lm - C^ab_l ](p),
// s_p = w_p for data primaries and -S1/N_r for random ones (the DDR^II term
// of Sec. 4.3 estimated with a random catalog).
//
// One warp owns one primary at a time.  Accepted neighbours go to a per-warp
// queue holding r, w_j W, w_j^2 W^2 and the 25 R_lm; the queue is drained with
// one lane per bin edge e, each lane evaluating F_l(r k_e), l = 0..4 (see
// hip_math.cuh) and accumulating w W F_l R_lm into its 25 registers.  The same
// drain forms jbar^a_l from adjacent edges and stages it for the C term.  At
// the end of a primary the edge sums are differenced into A^a_lm and contracted.
#include <cmath>
#include <cstdio>

#include "hip_internal.h"
#include "hip_bispec.h"

static __constant__ HipCoeffs c_coeffs;
// normalisation of the real harmonics: sqrt((l-m)!/(l+m)!) (times sqrt 2 for m > 0)
static __constant__ float c_ylm_norm_f[HIP_LMAX + 1][HIP_LMAX + 1];
static __constant__ double c_ylm_norm_d[HIP_LMAX + 1][HIP_LMAX + 1];

cudaError_t hip_upload_coeffs_bispec()
{
    cudaError_t e = cudaMemcpyToSymbol(c_coeffs, &hip_host_coeffs(), sizeof(HipCoeffs));
    if (e != cudaSuccess) return e;
    float nf[HIP_LMAX + 1][HIP_LMAX + 1];
    double nd[HIP_LMAX + 1][HIP_LMAX + 1];
    for (int l = 0; l <= HIP_LMAX; ++l)
        for (int m = 0; m <= HIP_LMAX; ++m) {
            double v = 0.0;
            if (m <= l) {
                double r = 1.0;
                for (int k = l - m + 1; k <= l + m; ++k) r /= k;
                v = std::sqrt(r) * (m > 0 ? std::sqrt(2.0) : 1.0);
            }
            nd[l][m] = v;
            nf[l][m] = (float)v;
        }
    if ((e = cudaMemcpyToSymbol(c_ylm_norm_f, nf, sizeof(nf))) != cudaSuccess) return e;
    return cudaMemcpyToSymbol(c_ylm_norm_d, nd, sizeof(nd));
}

template <typename T>
__device__ __forceinline__ T ylm_norm(int l, int m);
template <>
__device__ __forceinline__ float ylm_norm<float>(int l, int m) { return c_ylm_norm_f[l][m]; }
template <>
__device__ __forceinline__ double ylm_norm<double>(int l, int m) { return c_ylm_norm_d[l][m]; }

// Real harmonics R_lm(u) for l <= 4 at unit vector (x, y, z), index l*l + l + m:
// R_l0 = P_l(z); R_l,+m = n_lm Ptilde_l^m(z) Re (x + i y)^m; R_l,-m = same with Im,
// Ptilde_l^m(z) = P_l^m(z) / (1 - z^2)^(m/2) by the usual three-term recurrence.
template <typename T>
__device__ __forceinline__ void hip_real_ylm(T x, T y, T z, T *R)
{
    T P[HIP_LMAX + 1][HIP_LMAX + 1];
#pragma unroll
    for (int m = 0; m <= HIP_LMAX; ++m) {
        T pmm = T(1);
#pragma unroll
        for (int k = 1; k <= m; ++k) pmm *= T(2 * k - 1);
        P[m][m] = pmm;
        if (m + 1 <= HIP_LMAX) P[m + 1][m] = T(2 * m + 1) * z * pmm;
#pragma unroll
        for (int l = m + 2; l <= HIP_LMAX; ++l)
            P[l][m] = (T(2 * l - 1) * z * P[l - 1][m] - T(l + m - 1) * P[l - 2][m]) * (T(1) / T(l - m));
    }
    T cm[HIP_LMAX + 1], sm[HIP_LMAX + 1];
    cm[0] = T(1);
    sm[0] = T(0);
#pragma unroll
    for (int m = 1; m <= HIP_LMAX; ++m) {
        cm[m] = cm[m - 1] * x - sm[m - 1] * y;
        sm[m] = sm[m - 1] * x + cm[m - 1] * y;
    }
#pragma unroll
    for (int l = 0; l <= HIP_LMAX; ++l) {
        R[l * l + l] = P[l][0];
#pragma unroll
        for (int m = 1; m <= l; ++m) {
            const T b = ylm_norm<T>(l, m) * P[l][m];
            R[l * l + l + m] = b * cm[m];
            R[l * l + l - m] = b * sm[m];
        }
    }
}

#define HIP_BQ 8                        // neighbours per drain (one K = 8 MMA step)
#define HIP_BPRIM 8                     // primaries per work item
#define HIP_BQCAP (HIP_BQ + 32)         // queue capacity (a ballot adds up to 32)
#define HIP_BWARPS 4
#define HIP_BTHREADS (HIP_BWARPS * 32)
#define HIP_NLM 25
#define HIP_NLMP 28                     // 25 harmonics padded to a multiple of 4

template <typename T, int NKMAX>
struct BWarpSmem {
    T qr[HIP_BQCAP], qw[HIP_BQCAP], qpsi[HIP_BQCAP];
    alignas(16) T qy[HIP_BQCAP][HIP_NLMP];  // R_lm of each queued neighbour (row padded to 16 bytes)
    union {
        // jbar^a_l of each drained neighbour (C term); a fragment load reads
        // J[q = 8 ks + t (+4)][col + g] for t = lane % 4, g = lane / 4, so the bank
        // is (stride t + g) mod 32: a row stride = 8 (mod 32) makes the 32 lanes hit
        // 32 different banks
        T J[HIP_LMAX + 1][HIP_BQ][NKMAX + 8];
        T X[NKMAX + 1][HIP_NLM];           // at the end of a primary: k_e^3 E_e, then A^a_lm
    };
};

__global__ void k_sorted_cells(const int *__restrict__ start, int n_cells, int *__restrict__ scell)
{
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n_cells; c += gridDim.x * blockDim.x)
        for (int i = start[c]; i < start[c + 1]; ++i) scell[i] = c;
}

cudaError_t hip_sorted_cells(const int *cell_start, int n_cells, int *scell, cudaStream_t st)
{
    const int blocks = (n_cells + 255) / 256;
    k_sorted_cells<<<blocks < 1 ? 1 : blocks, 256, 0, st>>>(cell_start, n_cells, scell);
    return cudaGetLastError();
}

__device__ __forceinline__ float hip_sqrt_b(float v) { return sqrtf(v); }
__device__ __forceinline__ double hip_sqrt_b(double v) { return sqrt(v); }

// F_l(u), l = 0..4, as one number per l.
__device__ __forceinline__ void hip_F_all(float u, float *F)
{
    float Fm[5], Fc[5];
    bool series;
    hip_F_f32<31>(u, c_coeffs, Fm, Fc, series);
#pragma unroll
    for (int l = 0; l <= HIP_LMAX; ++l) F[l] = Fm[l] + Fc[l];
    if (series) F[0] += c_coeffs.ser32[0][0];
}
__device__ __forceinline__ void hip_F_all(double u, double *F) { hip_F_f64<31>(u, c_coeffs, F); }

__device__ __forceinline__ float hip_arg(float r, float khi, float klo) { return fmaf(r, khi, r * klo); }
__device__ __forceinline__ double hip_arg(double r, double khi, double) { return r * khi; }

// Drain n queued neighbours of one primary: lanes over edges.  Accumulates the
// edge sums E[t][lm] += w W F_l(r k_e) R_lm and stages jbar^a_l for the C term.
template <typename T, int NCH, int NKMAX>
__device__ __forceinline__ void hip_bdrain(BWarpSmem<T, NKMAX> &sm, int n, const T *kk, const T *kl, const T *k3,
                                           const T *k3n, const T *jfac, int lane, int n_e, T (&E)[NCH][HIP_NLM])
{
    for (int q = 0; q < n; ++q) {
        const T r = sm.qr[q], ww = sm.qw[q];
        T F[NCH][HIP_LMAX + 1];
#pragma unroll
        for (int t = 0; t < NCH; ++t) {
            hip_F_all(hip_arg(r, kk[t], kl[t]), F[t]);
            if (lane + 32 * t < n_e) {
                T y[HIP_NLMP];
#pragma unroll
                for (int i = 0; i < HIP_NLMP; ++i) y[i] = sm.qy[q][i];
#pragma unroll
                for (int l = 0; l <= HIP_LMAX; ++l) {
                    const T f = ww * F[t][l];
#pragma unroll
                    for (int m = -l; m <= l; ++m) E[t][l * l + l + m] += f * y[l * l + l + m];
                }
            }
        }
        // jbar^a_l = jfac_a (k_{a+1}^3 F_l(u_{a+1}) - k_a^3 F_l(u_a)), a = lane + 32 t
#pragma unroll
        for (int t = 0; t < NCH; ++t) {
#pragma unroll
            for (int l = 0; l <= HIP_LMAX; ++l) {
                T nxt = __shfl_down_sync(0xffffffffu, F[t][l], 1);
                const T wrap = __shfl_sync(0xffffffffu, F[(t + 1 < NCH) ? t + 1 : t][l], 0);
                if (lane == 31 && t + 1 < NCH) nxt = wrap;
                const int a = lane + 32 * t;
                if (a < n_e - 1) sm.J[l][q][a] = jfac[t] * (k3n[t] * nxt - k3[t] * F[t][l]);
            }
        }
    }
}

// The CTA accumulator Tc holds, per l, the upper triangle a <= b of the
// symmetric n_k x n_k matrix (both the C term and the contraction are symmetric
// in a, b), row a starting at a nk - a (a - 1) / 2.
__device__ __forceinline__ int hip_tri(int a, int b, int nk) { return a * nk - (a * (a - 1)) / 2 + (b - a); }

// Tc[l][a<=b] -= s_p sum_q psi_q J[l][q][a] J[l][q][b]  (the C term).
template <typename T, int NKMAX>
__device__ __forceinline__ void hip_cterm(const BWarpSmem<T, NKMAX> &sm, int n, int nk, T sp, int lane, T *Tc)
{
    const int per_l = nk * nk, ntri = nk * (nk + 1) / 2;
    for (int i = lane; i < (HIP_LMAX + 1) * per_l; i += 32) {
        const int l = i / per_l, ab = i - l * per_l, a = ab / nk, b = ab - a * nk;
        if (a > b) continue;
        T acc = T(0);
        for (int q = 0; q < n; ++q) acc += sm.qpsi[q] * sm.J[l][q][a] * sm.J[l][q][b];
        atomicAdd(&Tc[l * ntri + hip_tri(a, b, nk)], -sp * acc);
    }
}

// The C term on the tensor cores (FP32 path): for each l, the batch's
// contribution C_l[a][b] = sum_q (psi_q J[l][q][a]) J[l][q][b] is a
// [n_k x 16] x [16 x n_k] product, done with mma.sync m16n8k8 TF32 in three
// products of the split x = hi + lo (hi*hi + hi*lo + lo*hi, FP32 accumulate),
// which keeps ~FP32 accuracy; the 16 x 8 result tiles are added to the CTA
// accumulator.  Fragment layouts of m16n8k8 (g = lane/4, t = lane%4):
// A a0..a3 = (g, t), (g+8, t), (g, t+4), (g+8, t+4); B b0, b1 = (t, g), (t+4, g);
// C c0..c3 = (g, 2t), (g, 2t+1), (g+8, 2t), (g+8, 2t+1).
__device__ __forceinline__ unsigned hip_tf32(float x)
{
    unsigned r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ void hip_mma_tf32(float (&d)[4], const unsigned (&a)[4], const unsigned (&b)[2])
{
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

template <int NKMAX>
__device__ __forceinline__ void hip_cterm_mma(const BWarpSmem<float, NKMAX> &sm, int n, int nk, float sp, int lane,
                                              float *Tc)
{
    constexpr int MT = NKMAX / 16, NT = NKMAX / 8;  // row tiles of 16, column tiles of 8
    const int g = lane >> 2, t = lane & 3;
    float psi[HIP_BQ / 8][2];  // psi of the K columns this lane feeds into A: q = 8 ks + t (+4)
#pragma unroll
    for (int ks = 0; ks < HIP_BQ / 8; ++ks) {
        const int q0 = 8 * ks + t, q1 = q0 + 4;
        psi[ks][0] = q0 < n ? -sp * sm.qpsi[q0] : 0.f;
        psi[ks][1] = q1 < n ? -sp * sm.qpsi[q1] : 0.f;
    }
#pragma unroll 1
    for (int l = 0; l <= HIP_LMAX; ++l) {
#pragma unroll
        for (int mt = 0; mt < MT; ++mt) {
            if (16 * mt >= nk) break;
            float acc[NT][4];
#pragma unroll
            for (int nt = 0; nt < NT; ++nt) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.f;
#pragma unroll
            for (int ks = 0; ks < HIP_BQ / 8; ++ks) {
                const int q0 = 8 * ks + t, q1 = q0 + 4;
                const float x0 = q0 < n ? psi[ks][0] * sm.J[l][q0][16 * mt + g] : 0.f;
                const float x1 = q0 < n ? psi[ks][0] * sm.J[l][q0][16 * mt + g + 8] : 0.f;
                const float x2 = q1 < n ? psi[ks][1] * sm.J[l][q1][16 * mt + g] : 0.f;
                const float x3 = q1 < n ? psi[ks][1] * sm.J[l][q1][16 * mt + g + 8] : 0.f;
                unsigned ah[4] = {hip_tf32(x0), hip_tf32(x1), hip_tf32(x2), hip_tf32(x3)};
                unsigned al[4] = {hip_tf32(x0 - __uint_as_float(ah[0])), hip_tf32(x1 - __uint_as_float(ah[1])),
                                  hip_tf32(x2 - __uint_as_float(ah[2])), hip_tf32(x3 - __uint_as_float(ah[3]))};
#pragma unroll
                for (int nt = 0; nt < NT; ++nt) {
                    if (8 * nt >= nk) break;
                    if (8 * nt + 7 < 16 * mt) continue;  // below the diagonal: not needed
                    const float y0 = q0 < n ? sm.J[l][q0][8 * nt + g] : 0.f;
                    const float y1 = q1 < n ? sm.J[l][q1][8 * nt + g] : 0.f;
                    unsigned bh[2] = {hip_tf32(y0), hip_tf32(y1)};
                    unsigned bl[2] = {hip_tf32(y0 - __uint_as_float(bh[0])), hip_tf32(y1 - __uint_as_float(bh[1]))};
                    hip_mma_tf32(acc[nt], ah, bh);
                    hip_mma_tf32(acc[nt], ah, bl);
                    hip_mma_tf32(acc[nt], al, bh);
                }
            }
#pragma unroll
            for (int nt = 0; nt < NT; ++nt) {
                if (8 * nt >= nk) break;
                if (8 * nt + 7 < 16 * mt) continue;  // tile entirely below the diagonal
                const int r0 = 16 * mt + g, r1 = r0 + 8, c0 = 8 * nt + 2 * t, c1 = c0 + 1;
                float *T = Tc + (size_t)l * (nk * (nk + 1) / 2);
                if (c0 < nk && r0 <= c0) atomicAdd(&T[hip_tri(r0, c0, nk)], acc[nt][0]);
                if (c1 < nk && r0 <= c1) atomicAdd(&T[hip_tri(r0, c1, nk)], acc[nt][1]);
                if (c0 < nk && r1 <= c0) atomicAdd(&T[hip_tri(r1, c0, nk)], acc[nt][2]);
                if (c1 < nk && r1 <= c1) atomicAdd(&T[hip_tri(r1, c1, nk)], acc[nt][3]);
            }
        }
    }
}

template <typename T, int NKMAX>
__device__ __forceinline__ void hip_cterm_any(const BWarpSmem<T, NKMAX> &sm, int n, int nk, T sp, int lane, T *Tc)
{
    if constexpr (sizeof(T) == 4)
        hip_cterm_mma<NKMAX>(sm, n, nk, sp, lane, Tc);
    else
        hip_cterm<T, NKMAX>(sm, n, nk, sp, lane, Tc);
}

// One primary g (data first, then randoms) of the catalog described by a: the
// 27-cell neighbour scan, the queued drains (edge sums, C term) and, at the end,
// the contraction of its A^a_lm into the CTA accumulator Tc (upper triangle).
template <typename T, int NCH, int NKMAX>
__device__ __forceinline__ void hip_bispec_primary(const BispecArgs<T> &a, int g, BWarpSmem<T, NKMAX> &sm, T *Tc,
                                                   const T (&kk)[NCH], const T (&kl)[NCH], const T (&k3)[NCH],
                                                   const T (&k3n)[NCH], const T (&jfac)[NCH], int lane,
                                                   unsigned long long &cnt_d, unsigned long long &cnt_r)
{
    const int n_e = a.n_e, nk = n_e - 1, n_c = a.data.n_c;
    const unsigned lt_mask = (1u << lane) - 1u;
    const T R0sq = a.R0 * a.R0, invR0 = T(1) / a.R0;
    const int ntri = nk * (nk + 1) / 2;
    const bool is_rand = g >= a.n_data;
    const CellList<T> &pl = is_rand ? a.rand : a.data;
    const int p = is_rand ? g - a.n_data : g;
    const int c = is_rand ? a.rcell[p] : a.dcell[p];
    const int cx = c / (n_c * n_c), cy = (c / n_c) % n_c, cz = c % n_c;
    const T px = pl.x[p], py = pl.y[p], pz = pl.z[p];
    const T sp = is_rand ? a.rand_weight : T(pl.w[p]);
    const int self = is_rand ? -1 : p;
    {
        const long long oi = pl.idx[p];
        if (is_rand ? (oi < a.rp0 || oi >= a.rp1) : (oi < a.dp0 || oi >= a.dp1)) return;
    }
    T E[NCH][HIP_NLM];
#pragma unroll
    for (int t = 0; t < NCH; ++t)
#pragma unroll
        for (int i = 0; i < HIP_NLM; ++i) E[t][i] = T(0);
    int qn = 0;
    // cell shifts of this primary: lane 3 axis + d + 1 holds the shift
    // of neighbour offset d along that axis (the shift's low part, below
    // 1e-6 of the cell side, is under the FP32 B budget and dropped)
    T shl = T(0);
    if (lane < 9) {
        const int ax = lane / 3, cc = ax == 0 ? cx : (ax == 1 ? cy : cz);
        T lo;
        hip_cell_shift(a.data, cc, lane % 3 - 1, shl, lo);
    }
    for (int s = 0; s < 27; ++s) {
        const int dx = s / 9 - 1, dy = (s / 3) % 3 - 1, dz = s % 3 - 1;
        const int nb = (((cx + dx + n_c) % n_c) * n_c + (cy + dy + n_c) % n_c) * n_c + (cz + dz + n_c) % n_c;
        const int b0 = a.data.cell_start[nb], b1 = a.data.cell_start[nb + 1];
        const T shx = __shfl_sync(0xffffffffu, shl, dx + 1), shy = __shfl_sync(0xffffffffu, shl, dy + 4),
                shz = __shfl_sync(0xffffffffu, shl, dz + 7);
        const T ox = px - shx, oy = py - shy, oz = pz - shz;
        for (int jb = b0; jb < b1; jb += 32) {
            const int j = jb + lane;
            bool ok = false;
            T ddx = T(0), ddy = T(0), ddz = T(0), r2 = T(0);
            if (j < b1) {
                ddx = ox - a.data.x[j];
                ddy = oy - a.data.y[j];
                ddz = oz - a.data.z[j];
                r2 = ddx * ddx + ddy * ddy + ddz * ddz;
                ok = (r2 < R0sq) && (r2 > T(0)) && (j != self);
            }
            const unsigned m = __ballot_sync(0xffffffffu, ok);
            if (ok) {
                const T r = hip_sqrt_b(r2);
                const T ir = T(1) / r;
                const T W = hip_W<T>(r * invR0);
                const T wj = T(a.data.w[j]);
                const int slot = qn + __popc(m & lt_mask);
                T R[HIP_NLM];
                hip_real_ylm<T>(ddx * ir, ddy * ir, ddz * ir, R);
                sm.qr[slot] = r;
                sm.qw[slot] = wj * W;
                sm.qpsi[slot] = wj * wj * W * W;
#pragma unroll
                for (int i = 0; i < HIP_NLM; ++i) sm.qy[slot][i] = R[i];
            }
            const int nq = __popc(m);
            if (is_rand)
                cnt_r += nq;
            else
                cnt_d += nq;
            qn += nq;
            while (qn >= HIP_BQ) {
                // drain the first HIP_BQ entries, move the rest (< 32) down
                __syncwarp();
                hip_bdrain<T, NCH, NKMAX>(sm, HIP_BQ, kk, kl, k3, k3n, jfac, lane, n_e, E);
                __syncwarp();
                hip_cterm_any<T, NKMAX>(sm, HIP_BQ, nk, sp, lane, Tc);
                const int rest = qn - HIP_BQ;
                T mv[3] = {T(0), T(0), T(0)};
                if (lane < rest) {
                    mv[0] = sm.qr[HIP_BQ + lane];
                    mv[1] = sm.qw[HIP_BQ + lane];
                    mv[2] = sm.qpsi[HIP_BQ + lane];
                }
                T my[HIP_NLM];
#pragma unroll
                for (int i = 0; i < HIP_NLM; ++i) my[i] = lane < rest ? sm.qy[HIP_BQ + lane][i] : T(0);
                __syncwarp();
                if (lane < rest) {
                    sm.qr[lane] = mv[0];
                    sm.qw[lane] = mv[1];
                    sm.qpsi[lane] = mv[2];
#pragma unroll
                    for (int i = 0; i < HIP_NLM; ++i) sm.qy[lane][i] = my[i];
                }
                qn = rest;
                __syncwarp();
            }
        }
    }
    if (qn > 0) {
        __syncwarp();
        hip_bdrain<T, NCH, NKMAX>(sm, qn, kk, kl, k3, k3n, jfac, lane, n_e, E);
        __syncwarp();
        hip_cterm_any<T, NKMAX>(sm, qn, nk, sp, lane, Tc);
        qn = 0;
    }
    // edge sums -> A^a_lm = jfac_a (k_{a+1}^3 E_{a+1} - k_a^3 E_a)
    __syncwarp();
#pragma unroll
    for (int t = 0; t < NCH; ++t) {
        const int e = lane + 32 * t;
        if (e < n_e)
#pragma unroll
            for (int i = 0; i < HIP_NLM; ++i) sm.X[e][i] = k3[t] * E[t][i];
    }
    __syncwarp();
    T Aa[NCH][HIP_NLM];
#pragma unroll
    for (int t = 0; t < NCH; ++t) {
        const int e = lane + 32 * t;
#pragma unroll
        for (int i = 0; i < HIP_NLM; ++i) Aa[t][i] = e < nk ? jfac[t] * (sm.X[e + 1][i] - sm.X[e][i]) : T(0);
    }
    __syncwarp();
#pragma unroll
    for (int t = 0; t < NCH; ++t) {
        const int e = lane + 32 * t;
        if (e < nk)
#pragma unroll
            for (int i = 0; i < HIP_NLM; ++i) sm.X[e][i] = Aa[t][i];
    }
    __syncwarp();
    // contraction: Tc[l][a<=b] += s_p sum_m A^a_lm A^b_lm  (lane owns rows a)
#pragma unroll
    for (int t = 0; t < NCH; ++t) {
        const int aa = lane + 32 * t;
        if (aa < nk) {
            for (int b = aa; b < nk; ++b) {
#pragma unroll
                for (int l = 0; l <= HIP_LMAX; ++l) {
                    T d = T(0);
#pragma unroll
                    for (int mm = -l; mm <= l; ++mm) d += Aa[t][l * l + l + mm] * sm.X[b][l * l + l + mm];
                    atomicAdd(&Tc[l * ntri + hip_tri(aa, b, nk)], sp * d);
                }
            }
        }
    }
    __syncwarp();
}

template <typename T, int NCH, int NKMAX>
__global__ void __launch_bounds__(HIP_BTHREADS) k_bispec(BispecArgs<T> a)
{
    __shared__ BWarpSmem<T, NKMAX> smem[HIP_BWARPS];
    extern __shared__ __align__(16) unsigned char tc_raw[];
    T *Tc = reinterpret_cast<T *>(tc_raw);  // [5][nk][nk] CTA accumulator
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    BWarpSmem<T, NKMAX> &sm = smem[warp];
    const int n_e = a.n_e, nk = n_e - 1;
    const int ntri = nk * (nk + 1) / 2;
    for (int i = threadIdx.x; i < (HIP_LMAX + 1) * ntri; i += HIP_BTHREADS) Tc[i] = T(0);
    __syncthreads();

    T kk[NCH], kl[NCH], k3[NCH], k3n[NCH], jfac[NCH];
#pragma unroll
    for (int t = 0; t < NCH; ++t) {
        const int e = lane + 32 * t;
        kk[t] = e < n_e ? a.k[e] : T(0);
        kl[t] = e < n_e ? a.klo[e] : T(0);
        k3[t] = e < n_e ? a.k3[e] : T(0);
        k3n[t] = e + 1 < n_e ? a.k3[e + 1] : T(0);
        jfac[t] = e + 1 < n_e ? a.jfac[e] : T(0);
    }
    unsigned long long cnt_d = 0, cnt_r = 0;
    const int n_prim = a.n_data + a.n_rand;
    const int n_items = (n_prim + HIP_BPRIM - 1) / HIP_BPRIM;
    for (;;) {
        int item = 0;
        if (lane == 0) item = atomicAdd(a.work_counter, 1);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= n_items) break;
        const int g0 = item * HIP_BPRIM, g1 = min(g0 + HIP_BPRIM, n_prim);
        for (int g = g0; g < g1; ++g)
            hip_bispec_primary<T, NCH, NKMAX>(a, g, sm, Tc, kk, kl, k3, k3n, jfac, lane, cnt_d, cnt_r);
    }
    __syncthreads();
    double *out = a.partials + (size_t)blockIdx.x * (HIP_LMAX + 1) * nk * nk;
    for (int i = threadIdx.x; i < (HIP_LMAX + 1) * nk * nk; i += HIP_BTHREADS) {
        const int l = i / (nk * nk), ab = i - l * nk * nk, x = ab / nk, y = ab - x * nk;
        out[i] = (double)Tc[l * ntri + (x <= y ? hip_tri(x, y, nk) : hip_tri(y, x, nk))];
    }
    // cnt_d, cnt_r are warp-uniform (every lane added each ballot's count)
    if (lane == 0) {
        if (cnt_d) atomicAdd(a.npairs, cnt_d);
        if (cnt_r) atomicAdd(a.npairs + 1, cnt_r);
    }
}

// Many catalogs in one persistent launch: CTA work items of HIP_BCTA_PRIM
// primaries (8 per warp) of one catalog, the catalogs' items laid end to end.
// All warps of a CTA work on the same catalog, so the CTA accumulator Tc serves
// one catalog at a time: when the CTA moves to another catalog it adds Tc to the
// previous catalog's FP64 sums (FP64 atomics), clears it and loads the new
// catalog's edges.
template <typename T, int NCH, int NKMAX>
__global__ void __launch_bounds__(HIP_BTHREADS)
    k_bispec_batched(const BispecCat<T> *__restrict__ cats, int n_cats, int n_items, int *counter)
{
    __shared__ BWarpSmem<T, NKMAX> smem[HIP_BWARPS];
    __shared__ int s_item;
    extern __shared__ __align__(16) unsigned char tc_raw[];
    T *Tc = reinterpret_cast<T *>(tc_raw);  // [5][upper triangle of n_k x n_k]
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    BWarpSmem<T, NKMAX> &sm = smem[warp];
    T kk[NCH], kl[NCH], k3[NCH], k3n[NCH], jfac[NCH];
    unsigned long long cnt_d = 0, cnt_r = 0;
    int cur = -1;
    auto leave = [&](int c) {
        __syncthreads();
        const int nk = cats[c].a.n_e - 1, ntri = nk * (nk + 1) / 2;
        double *acc = cats[c].acc;
        for (int i = threadIdx.x; i < (HIP_LMAX + 1) * nk * nk; i += HIP_BTHREADS) {
            const int l = i / (nk * nk), ab = i - l * nk * nk, x = ab / nk, y = ab - x * nk;
            const T v = Tc[l * ntri + (x <= y ? hip_tri(x, y, nk) : hip_tri(y, x, nk))];
            if (v != T(0)) atomicAdd(&acc[i], (double)v);
        }
        if (lane == 0) {  // cnt_d, cnt_r are warp-uniform
            if (cnt_d) atomicAdd(cats[c].a.npairs, cnt_d);
            if (cnt_r) atomicAdd(cats[c].a.npairs + 1, cnt_r);
        }
        cnt_d = cnt_r = 0;
        __syncthreads();
    };
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
        __syncthreads();
        const int item = s_item;
        __syncthreads();
        if (item >= n_items) break;
        int c = cur < 0 ? 0 : cur;
        while (item >= cats[c].item_end) ++c;
        while (item < cats[c].item_begin) --c;
        if (c != cur) {
            if (cur >= 0) leave(cur);
            cur = c;
            const BispecArgs<T> &a = cats[c].a;
            const int n_e = a.n_e, nk = n_e - 1, ntri = nk * (nk + 1) / 2;
            for (int i = threadIdx.x; i < (HIP_LMAX + 1) * ntri; i += HIP_BTHREADS) Tc[i] = T(0);
#pragma unroll
            for (int t = 0; t < NCH; ++t) {
                const int e = lane + 32 * t;
                kk[t] = e < n_e ? a.k[e] : T(0);
                kl[t] = e < n_e ? a.klo[e] : T(0);
                k3[t] = e < n_e ? a.k3[e] : T(0);
                k3n[t] = e + 1 < n_e ? a.k3[e + 1] : T(0);
                jfac[t] = e + 1 < n_e ? a.jfac[e] : T(0);
            }
            __syncthreads();
        }
        const BispecArgs<T> &a = cats[c].a;
        const int n_prim = a.n_data + a.n_rand;
        const int g0 = (item - cats[c].item_begin) * HIP_BCTA_PRIM + warp * HIP_BPRIM;
        const int g1 = min(g0 + HIP_BPRIM, n_prim);
        for (int g = g0; g < g1; ++g)
            hip_bispec_primary<T, NCH, NKMAX>(a, g, sm, Tc, kk, kl, k3, k3n, jfac, lane, cnt_d, cnt_r);
    }
    if (cur >= 0) leave(cur);
}

template <typename T, int NCH, int NKMAX>
static cudaError_t launch_bispec_batched(const BispecCat<T> *cats, int n_cats, int n_items, int nk_max, int *counter,
                                         int *grid_out, cudaStream_t st)
{
    const size_t dyn = sizeof(T) * (HIP_LMAX + 1) * (nk_max * (nk_max + 1) / 2);
    cudaError_t e = cudaFuncSetAttribute(k_bispec_batched<T, NCH, NKMAX>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)dyn);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, nb = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_bispec_batched<T, NCH, NKMAX>, HIP_BTHREADS, dyn);
    int grid = sms * (nb < 1 ? 1 : nb);
    if (grid > n_items) grid = n_items < 1 ? 1 : n_items;
    *grid_out = grid;
    k_bispec_batched<T, NCH, NKMAX><<<grid, HIP_BTHREADS, dyn, st>>>(cats, n_cats, n_items, counter);
    return cudaGetLastError();
}

template <typename T>
cudaError_t hip_bispec_pairs_batched(const BispecCat<T> *cats, int n_cats, int n_items, int nk_max, int *counter,
                                     int *grid_out, cudaStream_t st)
{
    if (nk_max <= 31) return launch_bispec_batched<T, 1, 32>(cats, n_cats, n_items, nk_max, counter, grid_out, st);
    if constexpr (sizeof(T) == 4) {
        if (nk_max <= 63)
            return launch_bispec_batched<T, 2, 64>(cats, n_cats, n_items, nk_max, counter, grid_out, st);
    }
    return cudaErrorInvalidValue;
}
template cudaError_t hip_bispec_pairs_batched<float>(const BispecCat<float> *, int, int, int, int *, int *,
                                                     cudaStream_t);
template cudaError_t hip_bispec_pairs_batched<double>(const BispecCat<double> *, int, int, int, int *, int *,
                                                      cudaStream_t);

template <typename T, int NCH, int NKMAX>
static cudaError_t launch_bispec(const BispecArgs<T> &a, int max_grid, int *grid_out, cudaStream_t st)
{
    const int nk = a.n_e - 1;
    const size_t dyn = sizeof(T) * (HIP_LMAX + 1) * (nk * (nk + 1) / 2);
    cudaError_t e = cudaFuncSetAttribute(k_bispec<T, NCH, NKMAX>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)dyn);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, nb = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_bispec<T, NCH, NKMAX>, HIP_BTHREADS, dyn);
    int grid = sms * (nb < 1 ? 1 : nb);
    if (grid > max_grid) grid = max_grid;
    *grid_out = grid;
    k_bispec<T, NCH, NKMAX><<<grid, HIP_BTHREADS, dyn, st>>>(a);
    return cudaGetLastError();
}

template <typename T>
cudaError_t hip_bispec_pairs(const BispecArgs<T> &a, int max_grid, int *grid_out, cudaStream_t st)
{
    const int nk = a.n_e - 1;
    if (nk <= 31) return launch_bispec<T, 1, 32>(a, max_grid, grid_out, st);
    if constexpr (sizeof(T) == 4) {
        if (nk <= 63) return launch_bispec<T, 2, 64>(a, max_grid, grid_out, st);
    }
    return cudaErrorInvalidValue;
}
template cudaError_t hip_bispec_pairs<float>(const BispecArgs<float> &, int, int *, cudaStream_t);
template cudaError_t hip_bispec_pairs<double>(const BispecArgs<double> &, int, int *, cudaStream_t);

// B^ab_l = (-1)^l (2l+1) T^ab_l / (V n_w^3)
//          - delta_l0 (W~^a S^b + W~^b S^a) / (V n_w^2) + 2 delta_l0 W~^a W~^b   (Sec. 4.5)
__global__ void k_bispec_final(const double *__restrict__ partials, int nparts, int nk, int lmax, double L,
                               const double *S1, const double *S, const double *Wt, double *B)
{
    const int tot = (lmax + 1) * nk * nk;
    const double V = L * L * L, nw = S1[0] / V;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < tot; i += gridDim.x * blockDim.x) {
        double t = 0.0;
        for (int p = 0; p < nparts; ++p) t += partials[(size_t)p * (HIP_LMAX + 1) * nk * nk + i];
        const int l = i / (nk * nk), ab = i - l * nk * nk, aa = ab / nk, bb = ab - aa * nk;
        double b = ((l & 1) ? -1.0 : 1.0) * (2.0 * l + 1.0) * t / (V * nw * nw * nw);
        if (l == 0) b += -(Wt[aa] * S[bb] + Wt[bb] * S[aa]) / (V * nw * nw) + 2.0 * Wt[aa] * Wt[bb];
        B[i] = b;
    }
}

cudaError_t hip_bispec_finalize(const double *partials, int nparts, int nk, int lmax, double L, const double *S1,
                                const double *S, const double *Wt, double *B, cudaStream_t st)
{
    const int tot = (lmax + 1) * nk * nk;
    k_bispec_final<<<(tot + 255) / 256, 256, 0, st>>>(partials, nparts, nk, lmax, L, S1, S, Wt, B);
    return cudaGetLastError();
}

__global__ void k_bispec_sum(const double *__restrict__ partials, int nparts, int nk, int lmax, double *T)
{
    const int tot = (lmax + 1) * nk * nk;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < tot; i += gridDim.x * blockDim.x) {
        double t = 0.0;
        for (int p = 0; p < nparts; ++p) t += partials[(size_t)p * (HIP_LMAX + 1) * nk * nk + i];
        T[i] = t;
    }
}

cudaError_t hip_bispec_sum(const double *partials, int nparts, int nk, int lmax, double *T, cudaStream_t st)
{
    const int tot = (lmax + 1) * nk * nk;
    k_bispec_sum<<<(tot + 255) / 256, 256, 0, st>>>(partials, nparts, nk, lmax, T);
    return cudaGetLastError();
}

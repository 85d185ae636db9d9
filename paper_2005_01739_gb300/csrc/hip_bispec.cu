// Bispectrum kernels (Sec. 4 of arXiv:2005.01739): the a_lm pass, the FP64
// contraction and the C term.  The tensor-core contraction is in hip_bk_tc.cu.
//
// For every primary p (data particles, then the random catalog) the a_lm pass
// forms, over data neighbours j with 0 < |x_p - x_j| < R0,
//     A^a_lm(p) = sum_j w_j W(r/R0) jbar^a_l(r) R_lm(rhat)        (Eq. AC-def, binned)
// with real spherical harmonics R_lm scaled so that sum_m R_lm(u) R_lm(v) =
// L_l(u.v) (the addition theorem with the 4 pi / (2l+1) absorbed; real and
// complex harmonics give the same sum over m), and writes it to X[p][lm][a].
// The primary sum T^ab_l = sum_p s_p [sum_m A^a_lm A^b_lm - C^ab_l](p) (s_p = w_p
// for data primaries, -S1/N_r for random ones: the DDR^II term of Sec. 4.3 with
// a random catalog) is then the contraction sum_p s_p X_p X_p^T minus
//     sum_p s_p C^ab_l(p) = sum_(p,j) s_p w_j^2 W(r)^2 jbar^a_l(r) jbar^b_l(r),
// a pair sum of a function of r alone.  The a_lm pass accumulates it as 32
// Legendre moments of s_p w_j^2 W^2 per separation interval; the FP64 C-term
// kernels contract them with the products jbar^a_l jbar^b_l.
//
// a_lm pass: one warp owns one primary at a time (8 consecutive sorted primaries
// per work item).  Accepted neighbours are queued as separation vectors; 32 at a
// time they get one lane each for r, W, the 25 R_lm and the C-term moments, and
// are then drained with one lane per bin edge e: each lane evaluates
// F_l(r k_e), l = 0..4 (see hip_math.cuh), and accumulates w W F_l R_lm into its
// 25 registers.  At the end of the primary, adjacent edges give A^a_lm.
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
    if ((e = cudaMemcpyToSymbol(c_ylm_norm_d, nd, sizeof(nd))) != cudaSuccess) return e;
    return cudaSuccess;
}

// blockIdx.y = segment; warp w of block x takes data primaries x * 8 + w, stepping
// by gridDim.x * 8, lane l the bins l and l + 32 (n_k <= 64); the block's sums go
// to S with one FP64 atomic per bin.
template <typename T>
__global__ void __launch_bounds__(256) k_bk_s_sum(const BkSeg *__restrict__ segs)
{
    __shared__ double red[8][64];
    const BkSeg sg = segs[blockIdx.y];
    if (!sg.S) return;  // block-uniform
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nk = sg.n_k;
    const T *X = (const T *)sg.X, *sp = (const T *)sg.sp;
    for (int li = 0; li < sg.n_S; ++li) {  // l = 2 li: harmonic (l, 0) is row l^2 + l, R_l0 = L_l(mu)
        const int hr = (2 * li) * (2 * li) + 2 * li;
        double s0 = 0.0, s1 = 0.0;
        for (int p = blockIdx.x * 8 + warp; p < sg.n_d; p += gridDim.x * 8) {
            const T w = sp[p];  // 0 for an excluded primary, whose row of X is not written
            if (w == T(0)) continue;
            const T *row = X + ((size_t)p * HIP_NLM + hr) * nk;
            if (lane < nk) s0 += (double)w * (double)row[lane];
            if (lane + 32 < nk) s1 += (double)w * (double)row[lane + 32];
        }
        __syncthreads();
        red[warp][lane] = s0;
        red[warp][lane + 32] = s1;
        __syncthreads();
        if (threadIdx.x < 64 && threadIdx.x < nk) {
            double t = 0.0;
#pragma unroll
            for (int q = 0; q < 8; ++q) t += red[q][threadIdx.x];
            if (t != 0.0) atomicAdd(&sg.S[li * nk + threadIdx.x], t);
        }
    }
}

template <typename T>
cudaError_t hip_bk_s_sum(const BkSeg *segs, int n_segs, int, cudaStream_t st)
{
    k_bk_s_sum<T><<<dim3(1216, n_segs), 256, 0, st>>>(segs);
    return cudaGetLastError();
}
template cudaError_t hip_bk_s_sum<float>(const BkSeg *, int, int, cudaStream_t);
template cudaError_t hip_bk_s_sum<double>(const BkSeg *, int, int, cudaStream_t);

int hip_bk_intervals(double R0, double k_max)
{
    const double q = std::ceil(R0 * k_max / 8.0);
    return q < 1.0 ? 1 : (int)q;
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

#define HIP_BK_WARPS 4
#define HIP_BK_THREADS (HIP_BK_WARPS * 32)
#define HIP_NLMP 28  // a drained pair's record: the 25 R_lm, r, w_j W, padding

template <typename T>
struct BkWarpSmem {
    alignas(16) T qa[64][4];            // accepted neighbours: primary minus neighbour, w_j
    alignas(16) T qd[32][HIP_NLMP];     // drained pairs: R_lm (0..24), r (25), w_j W (26)
    T pt[32][HIP_BK_NM + 1];            // C-term weight s_p w_j^2 W^2 times R_m(t), m < 32
    T lq[32][2];                        // L_2, L_4 of each drained pair's mu (n_L = 3)
    int qc[32];                         // C-term interval of each drained pair
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
__device__ __forceinline__ void hip_F_all(float u, float *F) { hip_F_b32(u, c_coeffs, F); }
__device__ __forceinline__ void hip_F_all(double u, double *F) { hip_F_f64<31>(u, c_coeffs, F); }

__device__ __forceinline__ float hip_arg(float r, float khi, float klo) { return fmaf(r, khi, r * klo); }
__device__ __forceinline__ double hip_arg(double r, double khi, double) { return r * khi; }

// The 28 entries of a drained pair's record into registers (vector loads).
__device__ __forceinline__ void bk_load_rec(const float *src, float *dst)
{
#pragma unroll
    for (int i = 0; i < HIP_NLMP / 4; ++i) {
        const float4 v = reinterpret_cast<const float4 *>(src)[i];
        dst[4 * i] = v.x;
        dst[4 * i + 1] = v.y;
        dst[4 * i + 2] = v.z;
        dst[4 * i + 3] = v.w;
    }
}
__device__ __forceinline__ void bk_load_rec(const double *src, double *dst)
{
#pragma unroll
    for (int i = 0; i < HIP_NLMP / 2; ++i) {
        const double2 v = reinterpret_cast<const double2 *>(src)[i];
        dst[2 * i] = v.x;
        dst[2 * i + 1] = v.y;
    }
}

// Edge quantities of lane `lane` for chunk t (edge e = lane + 32 t).
template <typename T, int NCH>
struct BkEdges {
    T kk[NCH], kl[NCH], k3[NCH], k3n[NCH], jfac[NCH];
};

template <typename T, int NCH>
__device__ __forceinline__ void bk_load_edges(const BkCat<T> &a, int lane, BkEdges<T, NCH> &ed)
{
    const int n_e = a.n_e;
#pragma unroll
    for (int t = 0; t < NCH; ++t) {
        const int e = lane + 32 * t;
        ed.kk[t] = e < n_e ? a.k[e] : T(0);
        ed.kl[t] = e < n_e ? a.klo[e] : T(0);
        ed.k3[t] = e < n_e ? a.k3[e] : T(0);
        ed.k3n[t] = e + 1 < n_e ? a.k3[e + 1] : T(0);
        ed.jfac[t] = e + 1 < n_e ? a.jfac[e] : T(0);
    }
}

// Rounding error of s = a + b (Knuth's TwoSum); zero in FP64, where the
// separations are exact enough without it.
__device__ __forceinline__ float bk_low(float a, float b, float s)
{
    const float bv = __fadd_rn(s, -a);
    return __fadd_rn(__fadd_rn(a, -__fadd_rn(s, -bv)), __fadd_rn(b, -bv));
}
__device__ __forceinline__ double bk_low(double, double, double) { return 0.0; }

// Process the first n (<= 32) queued neighbours of the current primary: their
// geometry and harmonics (one per lane), their C-term moments (one lane per
// moment) and their contributions to the edge sums (one lane per bin edge).
template <typename T, int NCH>
__device__ __forceinline__ void bk_flush(BkWarpSmem<T> &sm, T *cm, int n, T s_p, T iR, T iR_lo, T cc_scale, T cc_lo, int n_cc, int n_L,
                                         int n_e, const BkEdges<T, NCH> &ed, int lane, T (&E)[NCH][HIP_NLM])
{
    if (lane < n) {
        const T dx = sm.qa[lane][0], dy = sm.qa[lane][1], dz = sm.qa[lane][2], wj = sm.qa[lane][3];
        const T r = hip_sqrt_b(dx * dx + dy * dy + dz * dz);
        const T ir = T(1) / r;
        const T W = hip_W<T>(fma(r, iR_lo, r * iR));
        T R[HIP_NLM];
        hip_real_ylm<T>(dx * ir, dy * ir, dz * ir, R);
#pragma unroll
        for (int i = 0; i < HIP_NLM; ++i) sm.qd[lane][i] = R[i];
        sm.qd[lane][25] = r;
        sm.qd[lane][26] = wj * W;
        sm.qd[lane][27] = T(0);
        // C term: interval c of width R0 / n_cc, coordinate t in [-1, 1]
        const T x = fma(r, cc_lo, r * cc_scale);
        int c = (int)x;
        if (c > n_cc - 1) c = n_cc - 1;
        T t = T(2) * (x - T(c)) - T(1);
        t = t < T(-1) ? T(-1) : (t > T(1) ? T(1) : t);
        const T wc = s_p * wj * wj * W * W;
        T p0 = wc, p1 = wc * t;
        sm.pt[lane][0] = p0;
        sm.pt[lane][1] = p1;
#pragma unroll
        for (int m = 1; m < HIP_BK_NM - 1; ++m) {
            const T p2 = hip_leg_alpha<T>(m) * t * p1 - hip_leg_beta<T>(m) * p0;  // R_m = d_m P_m
            sm.pt[lane][m + 1] = p2;
            p0 = p1;
            p1 = p2;
        }
        sm.qc[lane] = c;
        if (n_L > 1) {  // mu about the line of sight z (even L: the sign of dz does not matter)
            T l2, l4;
            hip_legendre24<T>(dz * ir, l2, l4);
            sm.lq[lane][0] = l2;
            sm.lq[lane][1] = l4;
        }
    }
    __syncwarp();
    if (n_L > 1) {  // warp-uniform
        for (int q = 0; q < n; ++q) {
            const T v = sm.pt[q][lane];
            const int o = sm.qc[q] * HIP_BK_NM + lane;
            cm[o] += v;
            cm[n_cc * HIP_BK_NM + o] += v * sm.lq[q][0];
            cm[2 * n_cc * HIP_BK_NM + o] += v * sm.lq[q][1];
        }
    } else {
        for (int q = 0; q < n; ++q) cm[sm.qc[q] * HIP_BK_NM + lane] += sm.pt[q][lane];
    }
    for (int q = 0; q < n; ++q) {
        T rec[HIP_NLMP];
        bk_load_rec(sm.qd[q], rec);
        const T r = rec[25], ww = rec[26];
#pragma unroll
        for (int t = 0; t < NCH; ++t) {
            T F[HIP_LMAX + 1];
            hip_F_all(hip_arg(r, ed.kk[t], ed.kl[t]), F);
            if (lane + 32 * t < n_e) {
#pragma unroll
                for (int l = 0; l <= HIP_LMAX; ++l) {
                    const T f = ww * F[l];
#pragma unroll
                    for (int m = -l; m <= l; ++m) E[t][l * l + l + m] += f * rec[l * l + l + m];
                }
            }
        }
    }
    __syncwarp();
}

// One primary g (data first, then randoms) of catalog a: the 27-cell neighbour
// scan and the queued flushes; then A^a_lm = jfac_a (k_{a+1}^3 E_{a+1} - k_a^3 E_a)
// into Xp[lm][a] and s_p into *spp.
template <typename T, int NCH>
__device__ __forceinline__ void bk_primary(const BkCat<T> &a, int g, BkWarpSmem<T> &sm, T *cm,
                                           const BkEdges<T, NCH> &ed, int lane, T *Xp, T *spp,
                                           unsigned long long &cnt_d, unsigned long long &cnt_r)
{
    const int n_e = a.n_e, nk = n_e - 1, n_c = a.data.n_c;
    const unsigned lt_mask = (1u << lane) - 1u;
    const bool is_rand = g >= a.n_data;
    const CellList<T> &pl = is_rand ? a.rand : a.data;
    const int p = is_rand ? g - a.n_data : g;
    const long long oi = pl.idx[p];
    const bool excluded = is_rand ? (oi < a.rp0 || oi >= a.rp1) : (oi < a.dp0 || oi >= a.dp1);
    const T s_p = excluded ? T(0) : (is_rand ? a.rand_weight : T(pl.w[p]));
    if (lane == 0) *spp = s_p;
    if (excluded) return;
    const T R0sq = a.R0 * a.R0, iR = a.iR, iR_lo = a.iR_lo, cc_scale = a.cc_scale, cc_lo = a.cc_lo;
    const int n_cc = a.n_cc;
    const int c = is_rand ? a.rcell[p] : a.dcell[p];
    const int cx = c / (n_c * n_c), cy = (c / n_c) % n_c, cz = c % n_c;
    const T px = pl.x[p], py = pl.y[p], pz = pl.z[p];
    const int self = is_rand ? -1 : p;
    T E[NCH][HIP_NLM];
#pragma unroll
    for (int t = 0; t < NCH; ++t)
#pragma unroll
        for (int i = 0; i < HIP_NLM; ++i) E[t][i] = T(0);
    int qn = 0;
    // cell shifts of this primary: lane 3 axis + d + 1 holds the shift of
    // neighbour offset d along that axis (hi, lo).  The candidate test uses the
    // rounded offset; an accepted neighbour's separation adds the low part (the
    // shift's own and the rounding of p - shift), which is common to all pairs
    // across a periodic face and would otherwise bias them alike.
    T shl = T(0), shll = T(0);
    if (lane < 9) {
        const int ax = lane / 3, cc = ax == 0 ? cx : (ax == 1 ? cy : cz);
        hip_cell_shift(a.data, cc, lane % 3 - 1, shl, shll);
    }
    for (int s = 0; s < 27; ++s) {
        const int dx = s / 9 - 1, dy = (s / 3) % 3 - 1, dz = s % 3 - 1;
        const int nb = (((cx + dx + n_c) % n_c) * n_c + (cy + dy + n_c) % n_c) * n_c + (cz + dz + n_c) % n_c;
        const int b0 = a.data.cell_start[nb], b1 = a.data.cell_start[nb + 1];
        const T shx = __shfl_sync(0xffffffffu, shl, dx + 1), shy = __shfl_sync(0xffffffffu, shl, dy + 4),
                shz = __shfl_sync(0xffffffffu, shl, dz + 7);
        const T ox = px - shx, oy = py - shy, oz = pz - shz;
        const T oxl = bk_low(px, -shx, ox) - __shfl_sync(0xffffffffu, shll, dx + 1),
                oyl = bk_low(py, -shy, oy) - __shfl_sync(0xffffffffu, shll, dy + 4),
                ozl = bk_low(pz, -shz, oz) - __shfl_sync(0xffffffffu, shll, dz + 7);
        for (int jb = b0; jb < b1; jb += 32) {
            const int j = jb + lane;
            bool ok = false;
            T ddx = T(0), ddy = T(0), ddz = T(0);
            if (j < b1) {
                ddx = ox - a.data.x[j];
                ddy = oy - a.data.y[j];
                ddz = oz - a.data.z[j];
                const T r2 = ddx * ddx + ddy * ddy + ddz * ddz;
                ok = (r2 < R0sq) && (r2 > T(0)) && (j != self);
            }
            const unsigned m = __ballot_sync(0xffffffffu, ok);
            if (ok) {
                const int slot = qn + __popc(m & lt_mask);
                sm.qa[slot][0] = ddx + oxl;
                sm.qa[slot][1] = ddy + oyl;
                sm.qa[slot][2] = ddz + ozl;
                sm.qa[slot][3] = T(a.data.w[j]);
            }
            const int nq = __popc(m);
            if (is_rand)
                cnt_r += nq;
            else
                cnt_d += nq;
            qn += nq;
            if (qn >= 32) {
                __syncwarp();
                bk_flush<T, NCH>(sm, cm, 32, s_p, iR, iR_lo, cc_scale, cc_lo, n_cc, a.n_L, n_e, ed, lane, E);
                const int rest = qn - 32;
                T mv[4] = {T(0), T(0), T(0), T(0)};
                if (lane < rest) {
#pragma unroll
                    for (int k = 0; k < 4; ++k) mv[k] = sm.qa[32 + lane][k];
                }
                __syncwarp();
                if (lane < rest) {
#pragma unroll
                    for (int k = 0; k < 4; ++k) sm.qa[lane][k] = mv[k];
                }
                qn = rest;
                __syncwarp();
            }
        }
    }
    if (qn > 0) {
        __syncwarp();
        bk_flush<T, NCH>(sm, cm, qn, s_p, iR, iR_lo, cc_scale, cc_lo, n_cc, a.n_L, n_e, ed, lane, E);
    }
#pragma unroll
    for (int t = 0; t < NCH; ++t) {
        const int aa = lane + 32 * t;
#pragma unroll
        for (int i = 0; i < HIP_NLM; ++i) {
            T nxt = __shfl_down_sync(0xffffffffu, E[t][i], 1);
            const T wrap = __shfl_sync(0xffffffffu, E[(t + 1 < NCH) ? t + 1 : t][i], 0);
            if (lane == 31 && t + 1 < NCH) nxt = wrap;
            if (aa < nk) Xp[i * nk + aa] = ed.jfac[t] * (ed.k3n[t] * nxt - ed.k3[t] * E[t][i]);
        }
    }
}

template <typename T>
size_t hip_bk_alm_smem_bytes(int ncc_max)
{
    return HIP_BK_WARPS * (sizeof(BkWarpSmem<T>) + sizeof(T) * (size_t)ncc_max * HIP_BK_NM);
}

// The a_lm pass: persistent CTAs of 4 warps; each warp takes work items (8
// consecutive primaries of one span) from an atomic counter.  Per warp, the
// C-term moments of the current catalog sit in an FP32 (FP64 on the plain path)
// shared array, added to the warp's FP64 slot after every item and to the
// catalog's moments when the warp leaves the catalog.
template <typename T, int NCH>
__global__ void __launch_bounds__(HIP_BK_THREADS) k_bk_alm(const BkCat<T> *__restrict__ cats,
                                                           const BkSpan *__restrict__ spans, int n_spans, int n_items,
                                                           int ncc_max, T *__restrict__ X, T *__restrict__ sp,
                                                           double *__restrict__ cm_slots, int *counter)
{
    extern __shared__ __align__(16) unsigned char bk_raw[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    BkWarpSmem<T> &sm = reinterpret_cast<BkWarpSmem<T> *>(bk_raw)[warp];
    T *cm = reinterpret_cast<T *>(bk_raw + HIP_BK_WARPS * sizeof(BkWarpSmem<T>)) + (size_t)warp * ncc_max * HIP_BK_NM;
    double *slot = cm_slots + ((size_t)blockIdx.x * HIP_BK_WARPS + warp) * ncc_max * HIP_BK_NM;
    for (int i = lane; i < ncc_max * HIP_BK_NM; i += 32) cm[i] = T(0);
    __syncwarp();
    BkEdges<T, NCH> ed;
    unsigned long long cnt_d = 0, cnt_r = 0;
    int cur = -1, si = 0;
    auto leave = [&](int c) {
        const BkCat<T> &a = cats[c];
        for (int i = lane; i < a.n_L * a.n_cc * HIP_BK_NM; i += 32) {
            const double v = slot[i];
            if (v != 0.0) {
                atomicAdd(&a.cmom[i], v);
                slot[i] = 0.0;
            }
        }
        if (lane == 0) {  // cnt_d, cnt_r are warp-uniform
            if (cnt_d) atomicAdd(a.npairs, cnt_d);
            if (cnt_r) atomicAdd(a.npairs + 1, cnt_r);
        }
        cnt_d = cnt_r = 0;
    };
    for (;;) {
        int item = 0;
        if (lane == 0) item = atomicAdd(counter, 1);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= n_items) break;
        while (si + 1 < n_spans && item >= spans[si].item_end) ++si;
        while (si > 0 && item < spans[si].item_begin) --si;
        const BkSpan sp_ = spans[si];
        if (sp_.cat != cur) {
            if (cur >= 0) leave(cur);
            cur = sp_.cat;
            bk_load_edges<T, NCH>(cats[cur], lane, ed);
        }
        const BkCat<T> &a = cats[cur];
        const int nk = a.n_e - 1;
        const int g0 = sp_.g0 + (item - sp_.item_begin) * HIP_BK_PRIM;
        const int g1 = min(g0 + HIP_BK_PRIM, sp_.g1);
        for (int g = g0; g < g1; ++g) {
            const long long o = g - sp_.g0;
            bk_primary<T, NCH>(a, g, sm, cm, ed, lane, X + sp_.x_off + o * HIP_NLM * nk, sp + sp_.sp_off + o, cnt_d,
                               cnt_r);
        }
        __syncwarp();
        // the item's C-term moments into the warp's FP64 slot
        for (int i = lane; i < a.n_L * a.n_cc * HIP_BK_NM; i += 32) {
            const T v = cm[i];
            if (v != T(0)) {
                slot[i] += (double)v;
                cm[i] = T(0);
            }
        }
        __syncwarp();
    }
    if (cur >= 0) leave(cur);
}

template <typename T>
size_t hip_bk_alm_slot_bytes(int ncc_max)
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // at most 16 CTAs per SM (the shared memory of a CTA is > 14 KB)
    return sizeof(double) * (size_t)sms * 16 * HIP_BK_WARPS * ncc_max * HIP_BK_NM;
}

template <typename T, int NCH>
static cudaError_t launch_bk_alm(const BkCat<T> *cats, const BkSpan *spans, int n_spans, int n_items, int ncc_max,
                                 T *X, T *sp, double *cm_slots, int *counter, cudaStream_t st)
{
    const size_t smem = hip_bk_alm_smem_bytes<T>(ncc_max);
    cudaError_t e = cudaFuncSetAttribute(k_bk_alm<T, NCH>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, nb = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_bk_alm<T, NCH>, HIP_BK_THREADS, smem);
    if (nb < 1) nb = 1;
    if (nb > 16) nb = 16;
    int grid = sms * nb;
    const int need = (n_items + HIP_BK_WARPS - 1) / HIP_BK_WARPS;
    if (grid > need) grid = need < 1 ? 1 : need;
    k_bk_alm<T, NCH><<<grid, HIP_BK_THREADS, smem, st>>>(cats, spans, n_spans, n_items, ncc_max, X, sp, cm_slots,
                                                         counter);
    return cudaGetLastError();
}

template <typename T>
cudaError_t hip_bk_alm(const BkCat<T> *cats, const BkSpan *spans, int n_spans, int n_items, int nk_max, int ncc_max,
                       T *X, T *sp, double *cm_slots, int *counter, cudaStream_t st)
{
    if (nk_max <= 31) return launch_bk_alm<T, 1>(cats, spans, n_spans, n_items, ncc_max, X, sp, cm_slots, counter, st);
    if constexpr (sizeof(T) == 4) {
        if (nk_max <= 63)
            return launch_bk_alm<T, 2>(cats, spans, n_spans, n_items, ncc_max, X, sp, cm_slots, counter, st);
    }
    return cudaErrorInvalidValue;
}
template size_t hip_bk_alm_slot_bytes<float>(int);
template size_t hip_bk_alm_slot_bytes<double>(int);
template cudaError_t hip_bk_alm<float>(const BkCat<float> *, const BkSpan *, int, int, int, int, float *, float *,
                                       double *, int *, cudaStream_t);
template cudaError_t hip_bk_alm<double>(const BkCat<double> *, const BkSpan *, int, int, int, int, double *, double *,
                                        double *, int *, cudaStream_t);

// ------------------------------------------------------- FP64 contraction ----
// sum_p s_p sum_m X_p[lm][a] X_p[lm][b] for a <= b (plain path): CTAs of 256
// threads take contiguous ranges of the segments' primaries (laid end to end),
// stage four primaries' X in shared memory at a time, and keep up to
// HIP_BK64_NE upper-triangle entries (l, a <= b) per thread in FP64 registers;
// on leaving a segment they are added to its accumulator (both triangles).
#define HIP_BK64_THREADS 256
#define HIP_BK64_NE 40    // ceil(5 * 63 * 64 / 2 / 256): every upper-triangle entry up to 63 bins
#define HIP_BK64_STAGE 4  // primaries staged per step

template <typename T>
__global__ void __launch_bounds__(HIP_BK64_THREADS) k_bk_contract_f64(const BkSeg *__restrict__ segs, int n_segs,
                                                                     long long n_total)
{
    extern __shared__ __align__(16) unsigned char c64_raw[];
    double *xs = reinterpret_cast<double *>(c64_raw);  // [HIP_BK64_STAGE][25][n_k]
    __shared__ double s_sp[HIP_BK64_STAGE];
    const long long per = (n_total + gridDim.x - 1) / gridDim.x;
    const long long q0 = blockIdx.x * per, q1 = min(q0 + per, n_total);
    if (q0 >= q1) return;
    // first segment of this CTA
    int sg = 0;
    long long base = 0;
    while (sg < n_segs && base + segs[sg].n_p <= q0) base += segs[sg++].n_p;
    double acc[HIP_BK64_NE];
    int ent[HIP_BK64_NE];  // (l << 16) | (a << 8) | b, or -1
    int cur_nk = -1;
    auto setup = [&](int nk) {
        const int ntri = nk * (nk + 1) / 2;
#pragma unroll
        for (int i = 0; i < HIP_BK64_NE; ++i) {
            acc[i] = 0.0;
            const int e = threadIdx.x + HIP_BK64_THREADS * i;
            ent[i] = -1;
            if (e < (HIP_LMAX + 1) * ntri) {
                const int l = e / ntri;
                int r = e - l * ntri, aa = 0;
                while (r >= nk - aa) {
                    r -= nk - aa;
                    ++aa;
                }
                ent[i] = (l << 16) | (aa << 8) | (aa + r);
            }
        }
        cur_nk = nk;
    };
    auto flush = [&](const BkSeg &s) {
        const int nk = s.n_k;
#pragma unroll
        for (int i = 0; i < HIP_BK64_NE; ++i)
            if (ent[i] >= 0 && acc[i] != 0.0) {
                const int l = ent[i] >> 16, aa = (ent[i] >> 8) & 255, bb = ent[i] & 255;
                atomicAdd(&s.acc[((size_t)l * nk + aa) * nk + bb], acc[i]);
                if (aa != bb) atomicAdd(&s.acc[((size_t)l * nk + bb) * nk + aa], acc[i]);
                acc[i] = 0.0;
            }
    };
    long long q = q0;
    while (q < q1 && sg < n_segs) {
        const BkSeg s = segs[sg];
        const int nk = s.n_k;
        if (nk != cur_nk) setup(nk);
        const long long s_end = min(q1, base + s.n_p);
        const T *Xd = reinterpret_cast<const T *>(s.X);
        const T *spd = reinterpret_cast<const T *>(s.sp);
        while (q < s_end) {
            const int np = (int)min((long long)HIP_BK64_STAGE, s_end - q);
            const long long p0 = q - base;
            __syncthreads();
            for (int i = threadIdx.x; i < np * HIP_NLM * nk; i += HIP_BK64_THREADS)
                xs[i] = (double)Xd[p0 * HIP_NLM * nk + i];
            if (threadIdx.x < HIP_BK64_STAGE)
                s_sp[threadIdx.x] = threadIdx.x < np ? (double)spd[p0 + threadIdx.x] : 0.0;
            __syncthreads();
            for (int pp = 0; pp < np; ++pp) {
                const double spv = s_sp[pp];
                if (spv == 0.0) continue;
                const double *xp = xs + (size_t)pp * HIP_NLM * nk;
#pragma unroll
                for (int i = 0; i < HIP_BK64_NE; ++i) {
                    if (ent[i] < 0) continue;
                    const int l = ent[i] >> 16, aa = (ent[i] >> 8) & 255, bb = ent[i] & 255;
                    double d = 0.0;
                    for (int m = l * l; m <= l * l + 2 * l; ++m) d += xp[m * nk + aa] * xp[m * nk + bb];
                    acc[i] += spv * d;
                }
            }
            q += np;
        }
        flush(s);
        if (q >= base + s.n_p) {
            base += s.n_p;
            ++sg;
        }
    }
}

template <typename T>
cudaError_t hip_bk_contract_f64(const BkSeg *segs, int n_segs, long long n_p_total, int nk_max, cudaStream_t st)
{
    const size_t smem = sizeof(double) * HIP_BK64_STAGE * HIP_NLM * nk_max;
    cudaError_t e =
        cudaFuncSetAttribute(k_bk_contract_f64<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    long long grid = (long long)sms * 4;
    if (grid > n_p_total / 16 + 1) grid = n_p_total / 16 + 1;
    k_bk_contract_f64<T><<<(int)grid, HIP_BK64_THREADS, smem, st>>>(segs, n_segs, n_p_total);
    return cudaGetLastError();
}
template cudaError_t hip_bk_contract_f64<float>(const BkSeg *, int, long long, int, cudaStream_t);
template cudaError_t hip_bk_contract_f64<double>(const BkSeg *, int, long long, int, cudaStream_t);

// ------------------------------------------------------------ the C term ----
// sum_(p,j) s_p w_j^2 W^2 jbar^a_l(r) jbar^b_l(r) from the moments
// M[c][m] = sum over pairs in interval c of s_p w_j^2 W^2 P_m(t): on each interval
// the pair density in t is rho_c(t) = sum_m (2m+1)/2 M[c][m] P_m(t), so the sum is
// sum_c int_{-1}^{1} rho_c(t) f(r_c(t)) dt, taken by 48-point Gauss-Legendre
// (exact for the degree-31 rho times the band-limited f).  All FP64.
#define HIP_BK_CQ 48

static double s_cq_x[HIP_BK_CQ], s_cq_w[HIP_BK_CQ];
static bool s_cq_ready = false;

static void cq_nodes()
{
    if (s_cq_ready) return;
    const int n = HIP_BK_CQ;
    for (int i = 0; i < n; ++i) {
        double x = std::cos(M_PI * (i + 0.75) / (n + 0.5));
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = x;
            for (int k = 2; k <= n; ++k) {
                const double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            const double dp = n * (x * p1 - p0) / (x * x - 1.0);
            const double dx = p1 / dp;
            x -= dx;
            if (std::fabs(dx) < 1e-16) break;
        }
        double p0 = 1.0, p1 = x;
        for (int k = 2; k <= n; ++k) {
            const double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        const double dp = n * (x * p1 - p0) / (x * x - 1.0);
        s_cq_x[i] = x;
        s_cq_w[i] = 2.0 / ((1.0 - x * x) * dp * dp);
    }
    s_cq_ready = true;
}

struct BkCQ {
    double x[HIP_BK_CQ], w[HIP_BK_CQ];
};

size_t hip_bk_cterm_scratch_bytes(int n_cc, int n_k)
{
    const size_t nodes = (size_t)n_cc * HIP_BK_CQ;
    return sizeof(double) * nodes * (1 + (HIP_LMAX + 1) * (size_t)n_k);
}

// Per node: its weight w_q rho_c(t_q) and jbar^a_l(r_q) for every l, a.
__global__ void k_bk_cc_nodes(BkCTerm c, BkCQ q, double *__restrict__ wn, double *__restrict__ J)
{
    const int n_nodes = c.n_cc * HIP_BK_CQ, nk = c.n_e - 1;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_nodes; i += gridDim.x * blockDim.x) {
        const int cc = i / HIP_BK_CQ, iq = i - cc * HIP_BK_CQ;
        const double t = q.x[iq];
        const double r = (cc + 0.5 * (1.0 + t)) * (c.R0 / c.n_cc);
        double rho = 0.0, p0 = 1.0, p1 = t;
        const double *M = c.cmom + (size_t)cc * HIP_BK_NM;
        rho += 0.5 * M[0] * p0 + 1.5 * M[1] * p1;  // M[m] are moments of R_m = d_m P_m
        for (int m = 1; m < HIP_BK_NM - 1; ++m) {
            const double p2 = ((2.0 * m + 1.0) * t * p1 - m * p0) / (m + 1.0);
            rho += (m + 1.5) * (M[m + 1] / hip_leg_scale(m + 1)) * p2;
            p0 = p1;
            p1 = p2;
        }
        wn[i] = q.w[iq] * rho;
        // jbar^a_l(r) = 3 [k_{a+1}^3 F_l(r k_{a+1}) - k_a^3 F_l(r k_a)] / (k_{a+1}^3 - k_a^3)
        double Fp[HIP_LMAX + 1];
        hip_F_f64<31>(r * c.k[0], c_coeffs, Fp);
        double k3p = c.k[0] * c.k[0] * c.k[0];
        for (int a = 0; a < nk; ++a) {
            double Fn[HIP_LMAX + 1];
            hip_F_f64<31>(r * c.k[a + 1], c_coeffs, Fn);
            const double k3n = c.k[a + 1] * c.k[a + 1] * c.k[a + 1];
            const double jf = 3.0 / (k3n - k3p);
            for (int l = 0; l <= HIP_LMAX; ++l) {
                J[((size_t)l * nk + a) * n_nodes + i] = jf * (k3n * Fn[l] - k3p * Fp[l]);
                Fp[l] = Fn[l];
            }
            k3p = k3n;
        }
    }
}

// acc[l][a][b] -= sum_q wn[q] J[l][a][q] J[l][b][q]: one warp per (l, a, b).
__global__ void k_bk_cc_contract(BkCTerm c, const double *__restrict__ wn, const double *__restrict__ J)
{
    const int nk = c.n_e - 1, n_nodes = c.n_cc * HIP_BK_CQ;
    const int lane = threadIdx.x & 31;
    const int n_out = (HIP_LMAX + 1) * nk * nk;
    for (int o = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; o < n_out; o += (gridDim.x * blockDim.x) >> 5) {
        const int l = o / (nk * nk), ab = o - l * nk * nk, a = ab / nk, b = ab - a * nk;
        const double *Ja = J + ((size_t)l * nk + a) * n_nodes, *Jb = J + ((size_t)l * nk + b) * n_nodes;
        double s = 0.0;
        for (int i = lane; i < n_nodes; i += 32) s += wn[i] * Ja[i] * Jb[i];
        for (int d = 16; d > 0; d >>= 1) s += __shfl_xor_sync(0xffffffffu, s, d);
        if (lane == 0) c.acc[o] -= s;
    }
}

cudaError_t hip_bk_cterm(const BkCTerm &c, void *scratch, cudaStream_t st)
{
    cq_nodes();
    BkCQ q;
    for (int i = 0; i < HIP_BK_CQ; ++i) {
        q.x[i] = s_cq_x[i];
        q.w[i] = s_cq_w[i];
    }
    const int n_nodes = c.n_cc * HIP_BK_CQ, nk = c.n_e - 1;
    double *wn = reinterpret_cast<double *>(scratch);
    double *J = wn + n_nodes;
    k_bk_cc_nodes<<<(n_nodes + 127) / 128, 128, 0, st>>>(c, q, wn, J);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int n_out = (HIP_LMAX + 1) * nk * nk;
    k_bk_cc_contract<<<(n_out + 7) / 8, 256, 0, st>>>(c, wn, J);
    return cudaGetLastError();
}

// Anisotropic C term: Tc[c][a][b] -= g_c sum_q wn_{L_c}[q] J[l1_c][a][q] J[l2_c][b][q]
// (g_c = (l1 l2 L; 0 0 0)), one warp per (combination, a, b).
__global__ void k_bk_cc_contract_aniso(BkAnisoCTerm t, int nk, int n_nodes, const double *__restrict__ wn,
                                       const double *__restrict__ J, double *__restrict__ Tc)
{
    const int lane = threadIdx.x & 31;
    const int n_out = t.n_comb * nk * nk;
    for (int o = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; o < n_out; o += (gridDim.x * blockDim.x) >> 5) {
        const int ci = o / (nk * nk), ab = o - ci * nk * nk, a = ab / nk, b = ab - a * nk;
        const double *w = wn + (size_t)t.Lidx[ci] * n_nodes;
        const double *Ja = J + ((size_t)t.l1[ci] * nk + a) * n_nodes, *Jb = J + ((size_t)t.l2[ci] * nk + b) * n_nodes;
        double s = 0.0;
        for (int i = lane; i < n_nodes; i += 32) s += w[i] * Ja[i] * Jb[i];
        for (int d = 16; d > 0; d >>= 1) s += __shfl_xor_sync(0xffffffffu, s, d);
        if (lane == 0) Tc[o] -= t.g[ci] * s;
    }
}

size_t hip_bk_cterm_aniso_scratch_bytes(int n_cc, int n_k)
{
    const size_t nodes = (size_t)n_cc * HIP_BK_CQ;
    return sizeof(double) * nodes * (3 + (HIP_LMAX + 1) * (size_t)n_k);
}

cudaError_t hip_bk_cterm_aniso(const BkCTerm &c, const BkAnisoCTerm &t, void *scratch, double *Tc, cudaStream_t st)
{
    cq_nodes();
    BkCQ q;
    for (int i = 0; i < HIP_BK_CQ; ++i) {
        q.x[i] = s_cq_x[i];
        q.w[i] = s_cq_w[i];
    }
    const int n_nodes = c.n_cc * HIP_BK_CQ, nk = c.n_e - 1;
    double *wn = reinterpret_cast<double *>(scratch);  // [3][n_nodes]: the L = 0, 2, 4 moment sets
    double *J = wn + 3 * (size_t)n_nodes;
    for (int L = 0; L < 3; ++L) {
        BkCTerm cl = c;
        cl.cmom = c.cmom + (size_t)L * c.n_cc * HIP_BK_NM;
        k_bk_cc_nodes<<<(n_nodes + 127) / 128, 128, 0, st>>>(cl, q, wn + (size_t)L * n_nodes, J);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    const int n_out = t.n_comb * nk * nk;
    k_bk_cc_contract_aniso<<<(n_out + 7) / 8, 256, 0, st>>>(t, nk, n_nodes, wn, J, Tc);
    return cudaGetLastError();
}

// ------------------------------------------------------------- finalize -----
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

// Anisotropic bispectrum: the extension the paper's conclusions propose (the sum
// over spherical harmonics of the isotropic estimator becomes a product of two
// harmonics of different order).  The paper fixes no estimator; the reading:
// with the fixed line of sight zhat the triangle is projected onto the tripolar
// functions
//     S_{l1 l2 L}(u, v) = sum_m (l1 l2 L; m, -m, 0) y_{l1 m}(u) y_{l2 -m}(v),
// y_lm = sqrt(4 pi / (2l+1)) Y_lm, for l1 <= l2 <= 4, l1 + l2 and L even,
// |l1 - l2| <= L <= min(l1 + l2, 4) (18 combinations), and
//     T^ab_{l1 l2 L} = sum_p s_p sum_{j != k} w_j w_k W_j W_k jbar^a_l1(r_j) jbar^b_l2(r_k) S(rhat_j, rhat_k).
// In the real harmonics R_lm of the a_lm pass (R_l0 = L_l(mu); R_{l, +-m} =
// sqrt 2 sqrt((l-m)!/(l+m)!) P_l^m cos / sin(m phi), no Condon-Shortley phase)
// the m sum pairs equal real indices:
//     sum_m (...) y_{l1 m} y_{l2 -m} = sum_{m >= 0} kappa_m [R_{l1 m} R_{l2 m} + R_{l1 -m} R_{l2 -m}],
// kappa_0 = (l1 l2 L; 0 0 0) (the m = 0 product counted once), kappa_m = (-1)^m (l1 l2 L; m, -m, 0),
// so T is a combination of the matching-m Gram blocks
//     G_{l1 l2 m}^{ab} = sum_p s_p [X_p(l1 m, a) X_p(l2 m, b) + X_p(l1 -m, a) X_p(l2 -m, b)]
// of the per-primary A^a_lm already written by the a_lm pass (X), minus the
// j = k terms, which are g sum_j w_j^2 W^2 jbar jbar L_L(mu_j), g = (l1 l2 L; 0 0 0).
#include <cmath>
#include <cstring>

#include "hip_internal.h"
#include "hip_bispec.h"

struct AnisoBlk {
    int n;                                   // blocks
    short r1p[HIP_ANISO_NBLK], r1n[HIP_ANISO_NBLK], r2p[HIP_ANISO_NBLK], r2n[HIP_ANISO_NBLK];
    char neg[HIP_ANISO_NBLK];                // m > 0: the -m rows too
};
static __constant__ AnisoBlk c_blk;

// Wigner 3j symbol of integer arguments (Racah's formula), on the host.
static double w3j(int j1, int j2, int j3, int m1, int m2, int m3)
{
    if (m1 + m2 + m3 != 0 || std::abs(m1) > j1 || std::abs(m2) > j2 || std::abs(m3) > j3) return 0.0;
    if (j3 < std::abs(j1 - j2) || j3 > j1 + j2) return 0.0;
    auto f = [](int n) {
        double r = 1.0;
        for (int i = 2; i <= n; ++i) r *= i;
        return r;
    };
    const int t1 = j2 - m1 - j3, t2 = j1 + m2 - j3, t3 = j1 + j2 - j3, t4 = j1 - m1, t5 = j2 + m2;
    double s = 0.0;
    for (int t = std::max(0, std::max(t1, t2)); t <= std::min(t3, std::min(t4, t5)); ++t)
        s += ((t & 1) ? -1.0 : 1.0) / (f(t) * f(t - t1) * f(t - t2) * f(t3 - t) * f(t4 - t) * f(t5 - t));
    const double tri = f(j1 + j2 - j3) * f(j1 - j2 + j3) * f(-j1 + j2 + j3) / f(j1 + j2 + j3 + 1);
    const double sg = ((j1 - j2 - m3) & 1) ? -1.0 : 1.0;
    return sg * std::sqrt(tri * f(j1 + m1) * f(j1 - m1) * f(j2 + m2) * f(j2 - m2) * f(j3 + m3) * f(j3 - m3)) * s;
}

const BkAnisoTables &hip_aniso_tables()
{
    static BkAnisoTables t = [] {
        BkAnisoTables u;
        std::memset(&u, 0, sizeof(u));
        for (int l1 = 0; l1 <= 4; ++l1)
            for (int l2 = l1; l2 <= 4; ++l2) {
                if ((l1 + l2) & 1) continue;
                for (int m = 0; m <= l1; ++m) {
                    const int q = u.n_blk++;
                    u.bl1[q] = l1;
                    u.bl2[q] = l2;
                    u.bm[q] = m;
                }
                for (int L = 0; L <= 4; L += 2) {
                    if (L < l2 - l1 || L > l1 + l2) continue;
                    const int c = u.ct.n_comb++;
                    u.ct.l1[c] = l1;
                    u.ct.l2[c] = l2;
                    u.ct.Lidx[c] = L / 2;
                    u.ct.g[c] = w3j(l1, l2, L, 0, 0, 0);
                    for (int m = 0; m <= l1; ++m)
                        u.kappa[c][m] = (m & 1 ? -1.0 : 1.0) * w3j(l1, l2, L, m, -m, 0);
                }
            }
        return u;
    }();
    return t;
}

cudaError_t hip_upload_aniso_tables()
{
    const BkAnisoTables &t = hip_aniso_tables();
    AnisoBlk b;
    std::memset(&b, 0, sizeof(b));
    b.n = t.n_blk;
    for (int q = 0; q < t.n_blk; ++q) {
        const int l1 = t.bl1[q], l2 = t.bl2[q], m = t.bm[q];
        b.r1p[q] = (short)(l1 * l1 + l1 + m);
        b.r1n[q] = (short)(l1 * l1 + l1 - m);
        b.r2p[q] = (short)(l2 * l2 + l2 + m);
        b.r2n[q] = (short)(l2 * l2 + l2 - m);
        b.neg[q] = m > 0;
    }
    return cudaMemcpyToSymbol(c_blk, &b, sizeof(b));
}

// The matching-m Gram: thread t of blockIdx.y owns tile (blockIdx.y * 256 + t)
// of the output, 4 x 4 entries (a0..a0+3, b0..b0+3) of one block; blockIdx.x
// takes a slice of every segment's primaries.  A CTA stages HIP_AG_PB primaries'
// rows of X (and s_p) in shared memory by asynchronous copies into two buffers
// (the next stage lands while this one is used), each harmonic row padded to a multiple
// of 4 bins (zeros), so a thread reads its 4 a values and 4 b values (and those
// of -m) as two 16-byte loads per primary and forms 16 products from them.  The
// products s_p X X are summed over the stage in FP32, the stage sums added to
// FP32 pairs (TwoSum-compensated), and those to the FP64 G once at the end.
#define HIP_AG_PB 16
#define HIP_AG_T 4
// 4-byte asynchronous copy global -> shared; n = 0 writes a zero (padding)
__device__ __forceinline__ void ag_cp4(float *dst, const float *src, int n)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src), "r"(n)
                 : "memory");
}
__device__ __forceinline__ void ag_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void ag_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

__global__ void __launch_bounds__(256) k_bk_aniso_gram(const BkSeg *__restrict__ segs, int n_segs, int nk_max)
{
    extern __shared__ __align__(16) float ag_raw[];
    const int nkp_max = (nk_max + 3) & ~3;
    const int buf = HIP_AG_PB * HIP_NLM * nkp_max + HIP_AG_PB;  // floats of one stage buffer
    // buffer b: Xs at ag_raw + b buf ([HIP_AG_PB][25][nkp]), then the stage's s_p [HIP_AG_PB]
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int sgi = 0; sgi < n_segs; ++sgi) {
        const BkSeg sg = segs[sgi];
        const int nk = sg.n_k, nkp = (nk + 3) & ~3, nt = nkp / HIP_AG_T, row = HIP_NLM * nkp;
        const float *X = (const float *)sg.X, *sp = (const float *)sg.sp;
        const int tile = blockIdx.y * 256 + threadIdx.x;
        const bool use = tile < c_blk.n * nt * nt;
        const int q = use ? tile / (nt * nt) : 0, tab = use ? tile - q * nt * nt : 0;
        const int a0 = (tab / nt) * HIP_AG_T, b0 = (tab - (tab / nt) * nt) * HIP_AG_T;
        const int o1p = c_blk.r1p[q] * nkp + a0, o1n = c_blk.r1n[q] * nkp + a0;
        const int o2p = c_blk.r2p[q] * nkp + b0, o2n = c_blk.r2n[q] * nkp + b0;
        const bool neg = c_blk.neg[q];
        float hi[HIP_AG_T][HIP_AG_T], lo[HIP_AG_T][HIP_AG_T];
#pragma unroll
        for (int i = 0; i < HIP_AG_T; ++i)
#pragma unroll
            for (int j = 0; j < HIP_AG_T; ++j) hi[i][j] = lo[i][j] = 0.0f;
        const bool any = (blockIdx.y * 256) < c_blk.n * nt * nt;  // block-uniform
        const int per = (sg.n_p + gridDim.x - 1) / gridDim.x;
        const int p0 = blockIdx.x * per, p1 = min(sg.n_p, p0 + per);
        // stage k (primaries p0 + k HIP_AG_PB ...) into buffer k & 1, one harmonic row of nk bins per warp
        auto issue = [&](int pb, int b) {
            const int np = min(HIP_AG_PB, p1 - pb);
            float *Xs = ag_raw + (size_t)b * buf;
            const float *Xb = X + (size_t)pb * HIP_NLM * nk;
            for (int r = warp; r < np * HIP_NLM; r += 8)
                for (int c = lane; c < nkp; c += 32)
                    ag_cp4(Xs + r * nkp + c, Xb + (size_t)r * nk + min(c, nk - 1), c < nk ? 4 : 0);
            if (threadIdx.x < np) ag_cp4(Xs + HIP_AG_PB * row + threadIdx.x, sp + pb + threadIdx.x, 4);
            ag_commit();
        };
        __syncthreads();  // the previous segment's last stage is done with both buffers
        if (any && p0 < p1) issue(p0, 0);
        for (int pb = p0, k = 0; any && pb < p1; pb += HIP_AG_PB, ++k) {
            const int np = min(HIP_AG_PB, p1 - pb);
            __syncthreads();  // every thread is done with stage k - 1, whose buffer the next copy takes
            if (pb + HIP_AG_PB < p1) {
                issue(pb + HIP_AG_PB, (k + 1) & 1);
                ag_wait<1>();  // stage k has landed (k + 1 may be in flight)
            } else {
                ag_wait<0>();
            }
            __syncthreads();  // stage k is in shared memory for all threads
            const float *Xs = ag_raw + (size_t)(k & 1) * buf, *ss = Xs + HIP_AG_PB * row;
            if (!use) continue;
            float st[HIP_AG_T][HIP_AG_T];
#pragma unroll
            for (int i = 0; i < HIP_AG_T; ++i)
#pragma unroll
                for (int j = 0; j < HIP_AG_T; ++j) st[i][j] = 0.0f;
            for (int pi = 0; pi < np; ++pi) {
                const float s = ss[pi];
                if (s == 0.0f) continue;  // excluded primary: its row of X is not written
                const float *x = Xs + pi * row;
                const float4 va = *reinterpret_cast<const float4 *>(x + o1p);
                const float4 vb = *reinterpret_cast<const float4 *>(x + o2p);
                const float ua[4] = {s * va.x, s * va.y, s * va.z, s * va.w}, ub[4] = {vb.x, vb.y, vb.z, vb.w};
#pragma unroll
                for (int i = 0; i < HIP_AG_T; ++i)
#pragma unroll
                    for (int j = 0; j < HIP_AG_T; ++j) st[i][j] = fmaf(ua[i], ub[j], st[i][j]);
                if (neg) {
                    const float4 wa = *reinterpret_cast<const float4 *>(x + o1n);
                    const float4 wb = *reinterpret_cast<const float4 *>(x + o2n);
                    const float za[4] = {s * wa.x, s * wa.y, s * wa.z, s * wa.w}, zb[4] = {wb.x, wb.y, wb.z, wb.w};
#pragma unroll
                    for (int i = 0; i < HIP_AG_T; ++i)
#pragma unroll
                        for (int j = 0; j < HIP_AG_T; ++j) st[i][j] = fmaf(za[i], zb[j], st[i][j]);
                }
            }
#pragma unroll
            for (int i = 0; i < HIP_AG_T; ++i)
#pragma unroll
                for (int j = 0; j < HIP_AG_T; ++j) {  // the stage's sum into hi + lo (TwoSum)
                    const float t = hi[i][j] + st[i][j], bv = t - hi[i][j];
                    lo[i][j] += (hi[i][j] - (t - bv)) + (st[i][j] - bv);
                    hi[i][j] = t;
                }
        }
        if (use)
#pragma unroll
            for (int i = 0; i < HIP_AG_T; ++i)
#pragma unroll
                for (int j = 0; j < HIP_AG_T; ++j) {
                    const double v = (double)hi[i][j] + (double)lo[i][j];
                    if (a0 + i < nk && b0 + j < nk && v != 0.0)
                        atomicAdd(&sg.acc[((size_t)q * nk + a0 + i) * nk + b0 + j], v);
                }
    }
}

cudaError_t hip_bk_aniso_gram(const BkSeg *segs, int n_segs, int nk_max, long long max_prims, cudaStream_t st)
{
    const int nkp = (nk_max + 3) & ~3, nt = nkp / HIP_AG_T;
    const size_t smem = 2 * sizeof(float) * ((size_t)HIP_AG_PB * HIP_NLM * nkp + HIP_AG_PB);  // two stages
    cudaError_t e = cudaFuncSetAttribute(k_bk_aniso_gram, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int chunks = (HIP_ANISO_NBLK * nt * nt + 255) / 256;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // about 2 CTAs per SM in all (the two stage buffers); each slice keeps at least a few stages
    long long slices = std::max(1LL, (long long)2 * sms / chunks);
    slices = std::min(slices, std::max(1LL, max_prims / (4 * HIP_AG_PB)));
    k_bk_aniso_gram<<<dim3((unsigned)slices, chunks), 256, smem, st>>>(segs, n_segs, nk_max);
    return cudaGetLastError();
}

struct AnisoAsm {
    int n_comb, blk0[HIP_ANISO_NCOMB], nm[HIP_ANISO_NCOMB];  // first Gram block of (l1, l2), blocks m = 0..l1
    double kappa[HIP_ANISO_NCOMB][5];
};

// Tc[c][a][b] = sum_{m=0}^{l1} kappa_{c,m} G[blk0_c + m][a][b]
__global__ void k_bk_aniso_assemble(AnisoAsm t, const double *__restrict__ G, int nk, double *__restrict__ Tc)
{
    const int n = t.n_comb * nk * nk;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int c = i / (nk * nk), ab = i - c * nk * nk;
        double s = 0.0;
        for (int m = 0; m < t.nm[c]; ++m) s += t.kappa[c][m] * G[(size_t)(t.blk0[c] + m) * nk * nk + ab];
        Tc[i] = s;
    }
}

cudaError_t hip_bk_aniso_assemble(const double *G, int nk, double *Tc, cudaStream_t st)
{
    const BkAnisoTables &tb = hip_aniso_tables();
    AnisoAsm t;
    std::memset(&t, 0, sizeof(t));
    t.n_comb = tb.ct.n_comb;
    for (int c = 0; c < t.n_comb; ++c) {
        const int l1 = tb.ct.l1[c], l2 = tb.ct.l2[c];
        int q = 0;
        while (q < tb.n_blk && !(tb.bl1[q] == l1 && tb.bl2[q] == l2)) ++q;
        t.blk0[c] = q;
        t.nm[c] = l1 + 1;
        for (int m = 0; m <= l1; ++m) t.kappa[c][m] = tb.kappa[c][m];
    }
    const int n = t.n_comb * nk * nk;
    k_bk_aniso_assemble<<<(n + 255) / 256, 256, 0, st>>>(t, G, nk, Tc);
    return cudaGetLastError();
}

struct AnisoFin {
    int n_comb, l1[HIP_ANISO_NCOMB], l2[HIP_ANISO_NCOMB], L[HIP_ANISO_NCOMB];
};

// B = (2 l1 + 1)(2 l2 + 1)(-1)^((l1 + l2)/2) [ Tc / (V n^3)
//       - d_{l2 0} d_{L l1} k_l1 DD^a_l1 W~^b / (V n^2) - d_{l1 0} d_{L l2} k_l2 W~^a DD^b_l2 / (V n^2)
//       + 2 d_{l1 0} d_{l2 0} W~^a W~^b ],  k_l = (l 0 l; 0 0 0) = (-1)^l / sqrt(2l + 1):
// the random-neighbour terms of N = D - R (the angular average of y_lm on a
// random leg leaves l = 0 there and L_L(mu) on the other leg), the random
// primaries being in Tc through s_p.  (0, 0, 0) is the isotropic summary of Sec. 4.5.
__global__ void k_bk_aniso_final(AnisoFin f, const double *__restrict__ Tc, const double *__restrict__ S,
                                 const double *__restrict__ Wt, const double *S1, int nk, double L,
                                 double *__restrict__ B)
{
    const double V = L * L * L, n = S1[0] / V;
    const int tot = f.n_comb * nk * nk;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < tot; i += gridDim.x * blockDim.x) {
        const int c = i / (nk * nk), ab = i - c * nk * nk, a = ab / nk, b = ab - a * nk;
        const int l1 = f.l1[c], l2 = f.l2[c], Lc = f.L[c];
        double t = Tc[i] / (V * n * n * n);
        if (l2 == 0 && Lc == l1)
            t -= ((l1 & 1) ? -1.0 : 1.0) / sqrt(2.0 * l1 + 1.0) * S[(l1 / 2) * nk + a] * Wt[b] / (V * n * n);
        if (l1 == 0 && Lc == l2)
            t -= ((l2 & 1) ? -1.0 : 1.0) / sqrt(2.0 * l2 + 1.0) * Wt[a] * S[(l2 / 2) * nk + b] / (V * n * n);
        if (l1 == 0 && l2 == 0) t += 2.0 * Wt[a] * Wt[b];
        B[i] = (2.0 * l1 + 1.0) * (2.0 * l2 + 1.0) * ((((l1 + l2) / 2) & 1) ? -1.0 : 1.0) * t;
    }
}

cudaError_t hip_bk_aniso_finalize(const double *Tc, const double *S, const double *Wt, const double *S1, int nk,
                                  double L, double *B, cudaStream_t st)
{
    const BkAnisoTables &tb = hip_aniso_tables();
    AnisoFin f;
    f.n_comb = tb.ct.n_comb;
    for (int c = 0; c < f.n_comb; ++c) {
        f.l1[c] = tb.ct.l1[c];
        f.l2[c] = tb.ct.l2[c];
        f.L[c] = 2 * tb.ct.Lidx[c];
    }
    const int tot = f.n_comb * nk * nk;
    k_bk_aniso_final<<<(tot + 255) / 256, 256, 0, st>>>(f, Tc, S, Wt, S1, nk, L, B);
    return cudaGetLastError();
}

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

// The matching-m Gram: blockIdx.y = a chunk of HIP_AG_EPT * 256 output entries
// (block, a, b), blockIdx.x = a slice of every segment's primaries.  A CTA stages
// HIP_AG_PB primaries' rows of X (and s_p) in shared memory; each thread keeps
// its entries as FP32 pairs (TwoSum-compensated sums of the rounded products
// s_p X X), added to the FP64 G once at the end.
#define HIP_AG_EPT 8
#define HIP_AG_PB 16
__global__ void __launch_bounds__(256) k_bk_aniso_gram(const BkSeg *__restrict__ segs, int n_segs, int nk_max)
{
    extern __shared__ __align__(16) float ag_raw[];
    const int row = HIP_NLM * nk_max;
    float *Xs = ag_raw;                       // [HIP_AG_PB][25 nk]
    float *ss = ag_raw + HIP_AG_PB * row;     // [HIP_AG_PB]
    for (int sgi = 0; sgi < n_segs; ++sgi) {
        const BkSeg sg = segs[sgi];
        const int nk = sg.n_k, n_ent = c_blk.n * nk * nk;
        const float *X = (const float *)sg.X, *sp = (const float *)sg.sp;
        int o1p[HIP_AG_EPT], o1n[HIP_AG_EPT], o2p[HIP_AG_EPT], o2n[HIP_AG_EPT];
        bool neg[HIP_AG_EPT], use[HIP_AG_EPT];
        float hi[HIP_AG_EPT], lo[HIP_AG_EPT];
#pragma unroll
        for (int k = 0; k < HIP_AG_EPT; ++k) {
            const int e = (blockIdx.y * HIP_AG_EPT + k) * 256 + threadIdx.x;
            use[k] = e < n_ent;
            const int q = use[k] ? e / (nk * nk) : 0, ab = use[k] ? e - q * nk * nk : 0;
            const int a = ab / nk, b = ab - a * nk;
            o1p[k] = c_blk.r1p[q] * nk + a;
            o1n[k] = c_blk.r1n[q] * nk + a;
            o2p[k] = c_blk.r2p[q] * nk + b;
            o2n[k] = c_blk.r2n[q] * nk + b;
            neg[k] = c_blk.neg[q];
            hi[k] = lo[k] = 0.0f;
        }
        const bool any = (blockIdx.y * HIP_AG_EPT) * 256 < n_ent;  // block-uniform
        const int per = (sg.n_p + gridDim.x - 1) / gridDim.x;
        const int p0 = blockIdx.x * per, p1 = min(sg.n_p, p0 + per);
        for (int pb = p0; any && pb < p1; pb += HIP_AG_PB) {
            const int np = min(HIP_AG_PB, p1 - pb);
            __syncthreads();
            for (int i = threadIdx.x; i < np * HIP_NLM * nk; i += 256) {
                const int pi = i / (HIP_NLM * nk), j = i - pi * HIP_NLM * nk;
                Xs[pi * row + j] = X[(size_t)(pb + pi) * HIP_NLM * nk + j];
            }
            if (threadIdx.x < np) ss[threadIdx.x] = sp[pb + threadIdx.x];
            __syncthreads();
            for (int pi = 0; pi < np; ++pi) {
                const float s = ss[pi];
                if (s == 0.0f) continue;  // excluded primary: its row of X is not written
                const float *x = Xs + pi * row;
#pragma unroll
                for (int k = 0; k < HIP_AG_EPT; ++k) {
                    float u = x[o1p[k]] * x[o2p[k]];
                    if (neg[k]) u = fmaf(x[o1n[k]], x[o2n[k]], u);
                    const float v = s * u;
                    const float t = hi[k] + v, bv = t - hi[k];
                    lo[k] += (hi[k] - (t - bv)) + (v - bv);
                    hi[k] = t;
                }
            }
        }
#pragma unroll
        for (int k = 0; k < HIP_AG_EPT; ++k) {
            const double v = (double)hi[k] + (double)lo[k];
            if (use[k] && v != 0.0) {
                const int e = (blockIdx.y * HIP_AG_EPT + k) * 256 + threadIdx.x;
                atomicAdd(&sg.acc[e], v);
            }
        }
    }
}

cudaError_t hip_bk_aniso_gram(const BkSeg *segs, int n_segs, int nk_max, long long max_prims, cudaStream_t st)
{
    const size_t smem = sizeof(float) * ((size_t)HIP_AG_PB * HIP_NLM * nk_max + HIP_AG_PB);
    cudaError_t e = cudaFuncSetAttribute(k_bk_aniso_gram, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int n_ent = HIP_ANISO_NBLK * nk_max * nk_max;
    const int chunks = (n_ent + HIP_AG_EPT * 256 - 1) / (HIP_AG_EPT * 256);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // about 4 CTAs per SM in all; each slice keeps at least a few stages of primaries
    long long slices = std::max(1LL, (long long)4 * sms / chunks);
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

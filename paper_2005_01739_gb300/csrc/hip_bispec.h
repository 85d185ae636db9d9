// Internal interface of the bispectrum kernels (hip_bispec.cu, hip_bk_tc.cu).
//
// The primary sum of Sec. 4 (Eq. AC-def binned as in Sec. 4.4, the summary of
// Sec. 4.5),
//     T^ab_l = sum_p s_p [ sum_m A^a_lm(p) A^b_lm(p) - C^ab_l(p) ],
// runs in three steps:
//   1. the a_lm pass (k_bk_alm): per primary the real-harmonic accumulators
//      A^a_lm, written to X[p][lm][a]; per pair the 32 Legendre moments of
//      s_p w_j^2 W^2 in the separation (the C term depends on r alone);
//   2. the contraction sum_p s_p X_p X_p^T (the block-diagonal l blocks), on the
//      tensor cores (hip_bk_tc.cu, tcgen05 kind::f16 on an exact three-slice
//      BF16 split of X) or in FP64; for the anisotropic bispectrum the
//      matching-m Gram blocks instead (hip_bk_aniso.cu);
//   3. the C term from its moments, contracted in FP64 with the products
//      jbar^a_l jbar^b_l, subtracted from the contraction.
#pragma once

#include "hip_internal.h"

#define HIP_BMAXE 65      // bin edges supported by the bispectrum kernels (64 bins)
#define HIP_NLM 25        // real harmonics for l <= 4
#define HIP_BK_NM 32      // Legendre moments of the C term per separation interval
#define HIP_BK_MAXCC 128  // separation intervals of the C term (R0 k_max <= 1024)
#define HIP_BK_PRIM 8     // primaries per warp work item of the a_lm pass

// Intervals of the C-term moments: n_cc = max(1, ceil(R0 k_max / 8)), so that the
// products jbar^a jbar^b (band-limited to 2 k_max) satisfy 2 k_max h <= 8 on
// intervals of half-width h, where 32 Legendre terms reproduce them to ~1e-15.
int hip_bk_intervals(double R0, double k_max);

// One catalog of the a_lm pass (device-resident descriptor).
template <typename T>
struct BkCat {
    CellList<T> data;          // neighbours (and data primaries)
    CellList<T> rand;          // random primaries (same cell grid)
    const int *dcell, *rcell;  // cell of each sorted data / random particle
    int n_data, n_rand;        // primaries: the data (sorted order), then the randoms
    long long dp0, dp1, rp0, rp1;  // primary ranges (input order) of the data and of the randoms
    int n_e;                   // bin edges = n_k + 1
    int n_cc;                  // C-term intervals
    int n_L;                   // C-term moment sets: 1 (L_0), or 3 (L_0, L_2, L_4 of the neighbour's mu, for the
                               // anisotropic bispectrum)
    T R0;
    T rand_weight;             // -S1 / N_r
    T cc_scale, cc_lo;         // n_cc / R0 = cc_scale + cc_lo
    T iR, iR_lo;               // 1 / R0 = iR + iR_lo
    double *cmom;              // [n_L][n_cc][HIP_BK_NM] FP64 C-term moments (atomically added)
    unsigned long long *npairs;  // [0] data-primary pairs, [1] random-primary pairs
    T k[HIP_BMAXE], klo[HIP_BMAXE], k3[HIP_BMAXE], jfac[HIP_BMAXE];
};

// A contiguous range of one catalog's primaries in one a_lm launch.
struct BkSpan {
    int cat;                   // catalog index
    int g0, g1;                // primaries [g0, g1) (data sorted order, then the randoms)
    int item_begin, item_end;  // warp work items [begin, end), HIP_BK_PRIM primaries each
    long long x_off;           // element offset of primary g0's [25][n_k] block in X
    long long sp_off;          // offset of primary g0 in sp
};

// The a_lm pass over the spans' primaries: X and sp (s_p, 0 for a primary
// outside its catalog's ranges) for every primary, C-term moments into the
// catalogs' cmom.  cm_slots: zeroed FP64 scratch of hip_bk_alm_slot_bytes();
// counter: zeroed device int.  nk_max, ncc_max: the largest n_k, n_cc of the
// catalogs.
template <typename T>
size_t hip_bk_alm_slot_bytes(int ncc_max);
template <typename T>
cudaError_t hip_bk_alm(const BkCat<T> *cats, const BkSpan *spans, int n_spans, int n_items, int nk_max, int ncc_max,
                       T *X, T *sp, double *cm_slots, int *counter, cudaStream_t st);

// One catalog's block of X in a contraction launch.
struct BkSeg {
    const void *X;             // [n_p][25][n_k], float (tensor-core path) or double
    const void *sp;            // [n_p] primary weights s_p (0: skip), same type as X
    int n_p, n_k;
    int stage_begin, stage_end;  // tensor-core path: stages of P primaries [begin, end)
    double *acc;               // [5][n_k][n_k] FP64 primary sum (atomically added)
    int n_d;                   // the first n_d primaries are data primaries
    double *S;                 // [n_S][n_k] S^a_l += sum over them of s_p A^a_l0, l = 0, 2, .. (null: not wanted)
    int n_S;                   // 1 (S^a = DD^a_0) or 3 (DD^a_l, l = 0, 2, 4, about zhat: R_l0 = L_l(mu))
};

// Primaries per tensor-core stage for a launch whose largest n_k is nk_max.
int hip_bk_tc_stage_prims(int nk_max);
// Sum_p s_p X_p X_p^T over the segments (device-resident table) on the tensor
// cores (tcgen05.mma kind::f16 on an exact three-slice BF16 split of X, the six
// slice products in three FP32 TMEM accumulators that stay exact, folded into
// float-float rows every fold_prims primaries, 0 = every stage, and into FP64).
// n_stages: total stages of all segments; status: device int, bit 0 set if a
// bounded wait gave up (the results are then invalid).  max_grid caps the CTAs
// (tests).  Supported for n_k <= 42 (hip_bk_tc_supported).
bool hip_bk_tc_supported(int nk_max);
cudaError_t hip_bk_contract_tc(const BkSeg *segs, int n_segs, int n_stages, int nk_max, int *status, int max_grid,
                               int fold_prims, cudaStream_t st);
// The same contraction in FP64 on the CUDA cores (plain path; T = the type of X):
// the segments' primaries (n_total of them) laid end to end.
template <typename T>
cudaError_t hip_bk_contract_f64(const BkSeg *segs, int n_segs, long long n_total, int nk_max, cudaStream_t st);

// S^a = sum over data primaries p of w_p A^a_00(p): the ordered data pair sum
// sum_{p != j} w_p w_j W j^a_0 (R_00 = 1), i.e. the l = 0 power pair sum DD^a_0
// that the summary estimator of Sec. 4.5 subtracts, read from X (FP64 sums).
template <typename T>
cudaError_t hip_bk_s_sum(const BkSeg *segs, int n_segs, int nk_max, cudaStream_t st);

// acc[l][a][b] -= sum over the C-term moments of one catalog (FP64).
struct BkCTerm {
    double k[HIP_BMAXE];
    double R0;
    int n_e, n_cc;
    const double *cmom;        // [n_cc][HIP_BK_NM]
    double *acc;               // [5][n_k][n_k]
};
size_t hip_bk_cterm_scratch_bytes(int n_cc, int n_k);
cudaError_t hip_bk_cterm(const BkCTerm &c, void *scratch, cudaStream_t st);

// ------------------------------------------------ anisotropic bispectrum ----
// Combinations (l1, l2, L) of the anisotropic bispectrum (hip_bispectrum_aniso):
// l1 <= l2 <= 4, l1 + l2 and L even, |l1 - l2| <= L <= min(l1 + l2, 4): 18 of them.
#define HIP_ANISO_NCOMB 18
#define HIP_ANISO_MAXCC 96  // C-term intervals of the anisotropic path (three moment sets per warp: R0 k_max <= 768)
#define HIP_ANISO_NBLK 22  // (l1, l2, |m|) blocks of the matching-m Gram: l1 <= l2, l1 + l2 even, |m| <= l1
struct BkAnisoCTerm {
    int n_comb;
    int l1[HIP_ANISO_NCOMB], l2[HIP_ANISO_NCOMB], Lidx[HIP_ANISO_NCOMB];  // Lidx = L / 2
    double g[HIP_ANISO_NCOMB];                                           // (l1 l2 L; 0 0 0)
};
// The C term of the combinations from the catalog's three C-moment sets
// (c.cmom: [3][n_cc][32], L = 0, 2, 4): Tc [18][n_k][n_k] -= g sum_j w_j^2 W^2
// jbar^a_l1 jbar^b_l2 L_L(mu_j) summed over the primaries with s_p.
// Host tables: the Gram blocks (l1, l2, |m|) in order and, per combination, g and
// kappa_m = (-1)^m (l1 l2 L; m, -m, 0) (m = 0..l1), from Wigner symbols on the host.
struct BkAnisoTables {
    int n_blk;
    int bl1[HIP_ANISO_NBLK], bl2[HIP_ANISO_NBLK], bm[HIP_ANISO_NBLK];
    BkAnisoCTerm ct;
    double kappa[HIP_ANISO_NCOMB][5];
};
const BkAnisoTables &hip_aniso_tables();
cudaError_t hip_upload_aniso_tables();
// G [HIP_ANISO_NBLK][n_k][n_k] (each segment's acc points at its catalog's G,
// zeroed before) += the matching-m Gram blocks of the segments' X.
cudaError_t hip_bk_aniso_gram(const BkSeg *segs, int n_segs, int nk_max, long long max_prims, cudaStream_t st);
// Tc [18][n_k][n_k] = sum_m kappa_m G_{l1 l2 m} (overwrites).
cudaError_t hip_bk_aniso_assemble(const double *G, int nk, double *Tc, cudaStream_t st);
// B [18][n_k][n_k] of the reading from Tc (primary sum with s_p), S [3][n_k]
// (DD^a_l, l = 0, 2, 4 about zhat), W~^a, S1 (device), box side L.
cudaError_t hip_bk_aniso_finalize(const double *Tc, const double *S, const double *Wt, const double *S1, int nk,
                                  double L, double *B, cudaStream_t st);
size_t hip_bk_cterm_aniso_scratch_bytes(int n_cc, int n_k);
cudaError_t hip_bk_cterm_aniso(const BkCTerm &c, const BkAnisoCTerm &t, void *scratch, double *Tc, cudaStream_t st);

// Cell index of every sorted particle from the cell start table.
cudaError_t hip_sorted_cells(const int *cell_start, int n_cells, int *scell, cudaStream_t st);

// T^ab_l = sum of the partial rows (the primary sum before normalisation).
cudaError_t hip_bispec_sum(const double *partials, int nparts, int nk, int lmax, double *T, cudaStream_t st);

// B^ab_l from the summed T partials, S^a (ordered DD_0 sum of the power kernel)
// and W~^a (Sec. 4.5 summary), all in FP64 on the device.
cudaError_t hip_bispec_finalize(const double *partials, int nparts, int nk, int lmax, double L, const double *S1,
                                const double *S, const double *Wt, double *B, cudaStream_t st);

// Internal interface of the moment-based power-spectrum pair pass (hip_moments.cu).
#pragma once

#include "hip_internal.h"

#define HIP_PM_M 16       // Legendre moments per separation interval
#define HIP_PM_NCMAX 256  // most intervals on [0, R0) (n_c = max(8, ceil(R0 k_max / 4)))
#define HIP_PM_REPL 16    // replicas of the FP64 moment totals: CTA b folds into replica b % 16

// Doubles of one catalog's moment totals: HIP_PM_REPL replicas of [3][M][n_c],
// then the sum of |w| (the FP32 fixed-point scales).
__host__ __device__ inline size_t hip_pm_mg_doubles(int n_c) { return (size_t)HIP_PM_REPL * 3 * HIP_PM_M * n_c + 1; }

// Intervals for a given R0 and largest edge, and whether the moment pass applies
// (n_c <= HIP_PM_NCMAX and its shared memory fits); otherwise the direct pass is used.
int hip_pm_intervals(double R0, double k_max);
// Interval width: R0 / n_c rounded up to a 16-bit significand, so that it is exact
// in FP32, the intervals still cover [0, R0), and c dc is exact for c < 256.
double hip_pm_width(double R0, int n_c);
bool hip_pm_applicable(double R0, double k_max, bool fp32);
size_t hip_pm_scratch_bytes(int n_e, int n_c);

// Edge sums S_l(k_e) of the pair pass (the direct kernel's partial rows) written
// as one row [3][n_e] at `row`; scratch holds hip_pm_scratch_bytes(n_e, n_c).
template <typename T>
cudaError_t hip_power_moments(const CellList<T> &cl, const PowerKernelArgs &a, const double *kedges, int n_ell,
                              double R0, void *scratch, double *row, cudaStream_t st);

// Batched moment pass: catalogs' work items laid end to end, one persistent
// launch; the CTA folds its moments into a catalog's totals when it moves on.
template <typename T>
struct PmCat {
    CellList<T> cl;
    long long p0, p1;            // primary range in input order
    int los, n_c;                // line-of-sight axis, intervals
    int item_begin, item_end;    // global work items [begin, end)
    T R0, dc;
    long long n_part;            // particles
    double *Mg;                  // hip_pm_mg_doubles(n_c): FP64 moment totals, sum |w| (zeroed before the launch)
    unsigned long long *npairs;  // ordered pairs counted
};
struct PmContractCat {
    const double *coef, *Mg;     // hip_pm_coeffs output, moment totals (HIP_PM_REPL replicas)
    int n_e, n_c, n_ell;
    double *row;                 // [3][n_e] edge sums written for l < n_ell
};

// Legendre coefficients of the edge functions (n_c intervals for R0, k_max);
// d_kedges and coef are device arrays, coef holds hip_pm_coef_doubles(n_e, n_c).
size_t hip_pm_coef_doubles(int n_e, int n_c);
cudaError_t hip_pm_coeffs(const double *d_kedges, int n_e, int n_ell, double R0, double k_max, double *coef,
                          cudaStream_t st);
template <typename T>
// warps: 4 or 8 per CTA (else chosen from per_cell, the pair-weighted particles
// per cell); fold: pairs between the FP32 sums' folds, 1024..16384 (else 16384).
cudaError_t hip_power_moments_batched(const PmCat<T> *cats, int n_cats, int n_items, int n_c_max, int *counter,
                                      const PmContractCat *cc, int n_e_max, double per_cell, int warps, int fold,
                                      cudaStream_t st);

cudaError_t hip_upload_coeffs_moments();
cudaError_t hip_upload_pm_tables();

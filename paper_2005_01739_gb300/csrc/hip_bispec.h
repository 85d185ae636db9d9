// Internal interface of the bispectrum kernels (hip_bispec.cu).
#pragma once

#include "hip_internal.h"

#define HIP_BMAXE 65  // bin edges supported by the bispectrum kernels (64 bins)

template <typename T>
struct BispecArgs {
    CellList<T> data;        // neighbours (and data primaries)
    CellList<T> rand;        // random primaries (same cell grid)
    int n_cells;             // cells per catalog (n_c^3)
    const int *dcell, *rcell;  // cell of each sorted data / random particle
    int n_data, n_rand;      // primaries: the data, then the randoms
    long long dp0, dp1, rp0, rp1;  // primary ranges (input order) of the data and of the randoms
    int n_e;                 // bin edges = n_k + 1
    T R0;
    T rand_weight;           // -S1 / N_r
    int *work_counter;
    double *partials;        // [gridDim.x][5][n_k][n_k]
    unsigned long long *npairs;  // [0] data-primary pairs, [1] random-primary pairs
    T k[HIP_BMAXE], klo[HIP_BMAXE], k3[HIP_BMAXE], jfac[HIP_BMAXE];
};

// One catalog of a batched bispectrum launch (device-resident descriptor).
template <typename T>
struct BispecCat {
    BispecArgs<T> a;           // the catalog (work_counter and partials unused)
    int item_begin, item_end;  // CTA work items [begin, end): HIP_BCTA_PRIM primaries each
    double *acc;               // [5][n_k][n_k] FP64 primary sums of this catalog (atomically added)
};
#define HIP_BCTA_PRIM 32       // primaries per CTA work item of the batched launch (4 warps x 8)

// Cell index of every sorted particle from the cell start table.
cudaError_t hip_sorted_cells(const int *cell_start, int n_cells, int *scell, cudaStream_t st);

template <typename T>
cudaError_t hip_bispec_pairs(const BispecArgs<T> &a, int max_grid, int *grid_out, cudaStream_t st);

// One persistent launch over the catalogs' work items laid end to end; nk_max
// is the largest n_k (<= 31 for FP64, <= 63 for FP32).
template <typename T>
cudaError_t hip_bispec_pairs_batched(const BispecCat<T> *cats, int n_cats, int n_items, int nk_max, int *counter,
                                     int *grid_out, cudaStream_t st);

// T^ab_l = sum of the partial rows (the primary sum before normalisation).
cudaError_t hip_bispec_sum(const double *partials, int nparts, int nk, int lmax, double *T, cudaStream_t st);

// B^ab_l from the summed T partials, S^a (ordered DD_0 sum of the power kernel)
// and W~^a (Sec. 4.5 summary), all in FP64 on the device.
cudaError_t hip_bispec_finalize(const double *partials, int nparts, int nk, int lmax, double L, const double *S1,
                                const double *S, const double *Wt, double *B, cudaStream_t st);

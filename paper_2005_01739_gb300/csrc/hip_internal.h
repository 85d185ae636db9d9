// Internal declarations shared by the translation units of the CUDA library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/hipster_gb300.h"
#include "hip_math.cuh"

#define HIP_MAX_EDGES (HIP_MAX_BINS + 1)
#define HIP_PAIR_THREADS 128
#define HIP_PAIR_WARPS (HIP_PAIR_THREADS / 32)
#define HIP_NSHIFT 14  // the home cell plus 13 forward neighbours (half shell)

// Sorted cell list of one catalog (device pointers into the workspace).
template <typename T>
struct CellList {
    const T *x, *y, *z;      // cell-local offsets (position minus cell origin)
    const float *w;          // weights (1 for unit)
    const int *idx;          // original index of each sorted particle
    const int *cell_start;   // [n_cells + 1]
    int n_c;                 // cells per side
    T cs;                    // cell side = L / n_c (>= R0)
};

struct PowerKernelArgs {
    int n_e;                 // number of bin edges = n_k + 1
    int los;                 // line-of-sight axis
    long long p0, p1;        // primary range in input order
    int n_items;             // n_cells * HIP_NSHIFT
    int *work_counter;
    double *partials;        // [gridDim.x][3][n_e]
    unsigned long long *npairs;
};

// One catalog of a batched power-spectrum launch (device-resident descriptor).
template <typename T>
struct BatchCat {
    CellList<T> cl;
    long long p0, p1;
    int los, n_e, lin;
    int item_begin, item_end;  // global work items [begin, end)
    T R0, dk32hi, dk32lo;
    T k[HIP_MAX_EDGES], klo[HIP_MAX_EDGES];
    double *acc;                 // [3][n_e] FP64 edge sums (atomically accumulated)
    unsigned long long *npairs;  // ordered pairs counted
};

// Per-catalog inputs of the batched FP64 finalize (device-resident).
struct FinalCat {
    double k[HIP_MAX_EDGES];
    double R0, L;
    int n_e, n_ell;
    const double *acc;  // [3][n_e]
    const double *S1;
    double *Wt;         // [n_k]
    double *DD, *P;     // [n_ell][n_k]
};

template <typename T>
cudaError_t hip_power_pairs_batched(const BatchCat<T> *cats, int n_cats, int n_items, int nch, int *counter,
                                    int grid, cudaStream_t st);
cudaError_t hip_power_finalize_batched(const FinalCat *cats, int n_cats, int nk_max, cudaStream_t st);

// Cell build: returns cudaSuccess or the first error.  `err` (device int) gets
// bit 0 set if a non-finite position or weight is seen; S1 (device double)
// receives sum of weights.
template <typename T>
cudaError_t hip_build_cells(const float *pos, const float *w, int64_t N, double L, int n_c, T *x, T *y, T *z,
                            float *ws, int *idx, int *cid, int *cell_start, int *cell_fill, double *S1, int *err,
                            cudaStream_t st);

cudaError_t hip_upload_coeffs_power();
cudaError_t hip_upload_coeffs_bispec();

// Pair pass of the power spectrum; K = real type (float: mixed, double: plain).
template <typename T>
cudaError_t hip_power_pairs(const CellList<T> &cl, const PowerKernelArgs &a, const double *kedges, int n_ell,
                            double R0, int grid, cudaStream_t st);
template <typename T>
int hip_power_grid();

// W~^a (Eq. wka-def) and the final FP64 reduction/normalisation of P.
cudaError_t hip_power_finalize(const double *partials, int nparts, int n_e, int n_ell, const double *kedges_host,
                               double R0, double L, const double *S1, double *Wt, double *DD, double *P,
                               cudaStream_t st);

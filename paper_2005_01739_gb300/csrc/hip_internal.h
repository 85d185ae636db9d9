// Internal declarations shared by the translation units of the CUDA library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/hipster_gb300.h"
#include "hip_math.cuh"

#define HIP_MAX_CELLS_SIDE 128  // most cells per side of a cell list
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
    double L;                // box side
    double cs;               // cell side = L / n_c (>= R0)
};

#ifdef __CUDACC__
// Origin of cell c along one axis.  For FP32 lists it is the float nearest
// c cs: for c >= 1 that origin is >= cs, so every float coordinate x in the
// cell lies within a factor two of it and x - origin is exact in float
// (Sterbenz's lemma); for c = 0 the offset is x itself.  Cell-local offsets
// therefore carry no rounding, whatever L / n_c is.
template <typename T>
__device__ __forceinline__ double hip_cell_origin(int c, double cs);
template <>
__device__ __forceinline__ double hip_cell_origin<float>(int c, double cs)
{
    return (double)(float)(c * cs);
}
template <>
__device__ __forceinline__ double hip_cell_origin<double>(int c, double cs)
{
    return c * cs;
}

// Offset of the frame of neighbour cell c + d (periodic image included) from
// the frame of home cell c along one axis: unwrapped neighbour origin minus home
// origin, so that a home offset h seen from the neighbour frame is h - shift.
// For FP32 lists the double sum is exact (two floats and L, result ~ cs) and is
// returned as hi + lo.
template <typename T>
__device__ __forceinline__ void hip_cell_shift(const CellList<T> &cl, int c, int d, T &hi, T &lo)
{
    int u = c + d;
    double wrap = 0.0;
    if (u < 0) {
        u += cl.n_c;
        wrap = -cl.L;
    } else if (u >= cl.n_c) {
        u -= cl.n_c;
        wrap = cl.L;
    }
    const double s = (hip_cell_origin<T>(u, cl.cs) - hip_cell_origin<T>(c, cl.cs)) + wrap;
    hi = (T)s;
    lo = (T)(s - (double)hi);
}
#endif

struct PowerKernelArgs {
    int n_e;                 // number of bin edges = n_k + 1
    int los;                 // line-of-sight axis
    long long p0, p1;        // primary range in input order
    int n_items;             // n_cells * HIP_NSHIFT
    long long n_part;        // particles of the catalog (sets the moment pass's CTA size)
    int *work_counter;
    double *partials;        // [gridDim.x][3][n_e]
    unsigned long long *npairs;
};

// Bin edges as seen by the pair kernels.  For FP32 each edge is split into
// khi + klo (two floats) and u = r k is formed as fma(r, khi, r klo): rounding
// the edge itself to a float would shift every pair's argument the same way, a
// systematic error, while the rounding of u then varies from pair to pair.
template <typename T>
struct EdgeTable {
    T k[HIP_MAX_EDGES];
    T klo[HIP_MAX_EDGES];
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
cudaError_t hip_upload_coeffs_pairs_f32_lin();
cudaError_t hip_upload_coeffs_pairs_f32_gen();
cudaError_t hip_upload_coeffs_pairs_f64();
cudaError_t hip_upload_coeffs_pairs_batched();
void hip_pairs_launch_f32_lin(const CellList<float> &cl, const PowerKernelArgs &a, const EdgeTable<float> &ed,
                              int n_ell, float R0, float dhi, float dlo, int grid, cudaStream_t st);
void hip_pairs_launch_f32_gen(const CellList<float> &cl, const PowerKernelArgs &a, const EdgeTable<float> &ed,
                              int n_ell, float R0, float dhi, float dlo, int grid, cudaStream_t st);
void hip_pairs_launch_f64(bool lin, const CellList<double> &cl, const PowerKernelArgs &a,
                          const EdgeTable<double> &ed, int n_ell, double R0, double dhi, double dlo, int grid,
                          cudaStream_t st);
int hip_pairs_blocks_per_sm_f32();
int hip_pairs_blocks_per_sm_f64();

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
// W~^a alone (n_e edges, host array), into Wt [n_e - 1] on the device.
cudaError_t hip_window_transform(int n_e, const double *kedges_host, double R0, double *Wt, cudaStream_t st);
// n_r uniform randoms in [0, L)^3 from SplitMix64 (hip_subsample.cu; the mapping is
// documented at hip_uniform_randoms) into the device array d_out [n_r][3].
cudaError_t hip_launch_uniform_randoms(float *d_out, long long n_r, double L, unsigned long long seed,
                                       cudaStream_t st);
// P [n_ell][n_k] from summed DD [n_ell][n_k] and W~ (device arrays), S1 = sum of all weights.
cudaError_t hip_power_from_dd(const double *DD, int n_k, int n_ell, double L, double S1, const double *Wt, double *P,
                              cudaStream_t st);

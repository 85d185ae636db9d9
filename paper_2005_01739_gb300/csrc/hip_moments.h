// Internal interface of the moment-based power-spectrum pair pass (hip_moments.cu).
#pragma once

#include "hip_internal.h"

#define HIP_PM_M 16       // Legendre moments per separation interval
#define HIP_PM_NCMAX 256  // most intervals on [0, R0) (n_c = max(8, ceil(R0 k_max / 4)))

// Intervals for a given R0 and largest edge, and whether the moment pass applies
// (n_c <= HIP_PM_NCMAX and its shared memory fits); otherwise the direct pass is used.
int hip_pm_intervals(double R0, double k_max);
bool hip_pm_applicable(double R0, double k_max, bool fp32);
size_t hip_pm_scratch_bytes(int n_e, int n_c);

// Edge sums S_l(k_e) of the pair pass (the direct kernel's partial rows) written
// as one row [3][n_e] at `row`; scratch holds hip_pm_scratch_bytes(n_e, n_c).
template <typename T>
cudaError_t hip_power_moments(const CellList<T> &cl, const PowerKernelArgs &a, const double *kedges, int n_ell,
                              double R0, void *scratch, double *row, cudaStream_t st);

cudaError_t hip_upload_coeffs_moments();
cudaError_t hip_upload_pm_tables();

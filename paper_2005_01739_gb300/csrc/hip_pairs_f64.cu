// Pair kernels, FP64 (plain path).
#define HIP_PAIR_UPLOAD hip_upload_coeffs_pairs_f64
#include "hip_pair_kernel.cuh"

void hip_pairs_launch_f64(bool lin, const CellList<double> &cl, const PowerKernelArgs &a,
                          const EdgeTable<double> &ed, int n_ell, double R0, double dhi, double dlo, int grid,
                          cudaStream_t st)
{
    if (lin)
        launch_nch<double, true>(cl, a, ed, n_ell, R0, dhi, dlo, grid, st);
    else
        launch_nch<double, false>(cl, a, ed, n_ell, R0, dhi, dlo, grid, st);
}

int hip_pairs_blocks_per_sm_f64()
{
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_power_pairs<double, 4, 21, true>, HIP_PAIR_THREADS, 0);
    return nb;
}

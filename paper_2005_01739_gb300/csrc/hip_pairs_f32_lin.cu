// Pair kernels, FP32 (mixed path), uniformly spaced edges.
#define HIP_PAIR_UPLOAD hip_upload_coeffs_pairs_f32_lin
#include "hip_pair_kernel.cuh"

void hip_pairs_launch_f32_lin(const CellList<float> &cl, const PowerKernelArgs &a, const EdgeTable<float> &ed,
                              int n_ell, float R0, float dhi, float dlo, int grid, cudaStream_t st)
{
    launch_nch<float, true>(cl, a, ed, n_ell, R0, dhi, dlo, grid, st);
}

int hip_pairs_blocks_per_sm_f32()
{
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_power_pairs<float, 4, 21, true>, HIP_PAIR_THREADS, 0);
    return nb;
}

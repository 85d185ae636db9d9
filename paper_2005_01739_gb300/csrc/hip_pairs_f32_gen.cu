// Pair kernels, FP32 (mixed path), arbitrary edges.
#define HIP_PAIR_UPLOAD hip_upload_coeffs_pairs_f32_gen
#include "hip_pair_kernel.cuh"

void hip_pairs_launch_f32_gen(const CellList<float> &cl, const PowerKernelArgs &a, const EdgeTable<float> &ed,
                              int n_ell, float R0, float dhi, float dlo, int grid, cudaStream_t st)
{
    launch_nch<float, false>(cl, a, ed, n_ell, R0, dhi, dlo, grid, st);
}

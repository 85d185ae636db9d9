// Batched pair kernel: many catalogs in one persistent launch.
#define HIP_PAIR_UPLOAD hip_upload_coeffs_pairs_batched
#include "hip_pair_kernel.cuh"

template <typename T>
cudaError_t hip_power_pairs_batched(const BatchCat<T> *cats, int n_cats, int n_items, int nch, int *counter,
                                    int grid, cudaStream_t st)
{
    if (nch <= 1)
        k_power_pairs_batched<T, 1><<<grid, HIP_PAIR_THREADS, 0, st>>>(cats, n_cats, n_items, counter);
    else if (nch <= 2)
        k_power_pairs_batched<T, 2><<<grid, HIP_PAIR_THREADS, 0, st>>>(cats, n_cats, n_items, counter);
    else if (nch <= 4)
        k_power_pairs_batched<T, 4><<<grid, HIP_PAIR_THREADS, 0, st>>>(cats, n_cats, n_items, counter);
    else
        k_power_pairs_batched<T, 8><<<grid, HIP_PAIR_THREADS, 0, st>>>(cats, n_cats, n_items, counter);
    return cudaGetLastError();
}
template cudaError_t hip_power_pairs_batched<float>(const BatchCat<float> *, int, int, int, int *, int, cudaStream_t);
template cudaError_t hip_power_pairs_batched<double>(const BatchCat<double> *, int, int, int, int *, int,
                                                     cudaStream_t);


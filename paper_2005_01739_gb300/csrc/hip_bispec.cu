// Bispectrum kernels (Sec. 4 of arXiv:2005.01739).
#include "hip_internal.h"

static __constant__ HipCoeffs c_coeffs;

cudaError_t hip_upload_coeffs_bispec()
{
    return cudaMemcpyToSymbol(c_coeffs, &hip_host_coeffs(), sizeof(HipCoeffs));
}

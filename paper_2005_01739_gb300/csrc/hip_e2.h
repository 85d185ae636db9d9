// Internal interface of the random-free DDR^II term (hip_e2.cu, App. A).
#pragma once

#include <vector>

#include "hip_internal.h"

#define HIP_E2_NBIN 16384  // separation bins on [0, 2 R0)

// Quadrature nodes of the E^II integrals: p on [0, k_hi + 120/R0] (panels no
// wider than pi/(2 R0)) and r on the three pieces of W (panels no wider than
// pi/max(p_max, k_hi)), composite 16-point Gauss-Legendre.
struct E2Nodes {
    std::vector<double> p, pw, r, rw;
};

void hip_e2_nodes(const double *k_edges, int n_k, double R0, E2Nodes &nd);
size_t hip_e2_scratch_bytes(const E2Nodes &nd, int n_k);

// Writes row[(l n_k + a) n_k + b] = -(S1/V) sum_{j != k} w_j w_k E^{II,ab}_l(r_jk)
// (zero for l > lmax) from a cell list of cells >= 2 R0 wide.
cudaError_t hip_e2_term(const CellList<float> &cl2, int n_items2, int *counter, double R0, double L,
                        const double *k_edges, int n_k, int lmax, const double *S1, const E2Nodes &nd, void *scratch,
                        double *row, unsigned long long *npairs2, cudaStream_t st);

// omega^a_l(p) (Eq. omega-ell-a-def) for l <= lmax at n_p caller-given p (host):
// out[(l n_k + a) n_p + q] (host, written when the stream reaches it); scratch
// holds hip_omega_scratch_bytes(...) bytes.
size_t hip_omega_scratch_bytes(const double *k_edges, int n_k, double R0, const double *p, int n_p);
cudaError_t hip_omega_eval(const double *k_edges, int n_k, double R0, int lmax, const double *p, int n_p,
                           void *scratch, double *out, cudaStream_t st);

cudaError_t hip_upload_coeffs_e2();

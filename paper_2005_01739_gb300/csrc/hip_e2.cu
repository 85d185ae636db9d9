// The random-free DDR^II term of the bispectrum (App. A of arXiv:2005.01739).
//
// The random catalog enters the estimator only through the sum over random
// primaries of G(x) = sum_{j != k} w_j w_k jbar^a_l(r_j) jbar^b_l(r_k) W W L_l(cos),
// whose expectation is (N_r / V) sum_{j != k} w_j w_k E^{II,ab}_l(r_jk) with the
// kernel E^{II,ab}_l(r) = int p^2 dp/(2 pi^2) j_0(p r) omega^a_l(p) omega^b_l(p) and
// omega^a_l(p) = 4 pi int_0^R0 r^2 j_l(p r) jbar^a_l(r) W(r) dr (Eq. omega-ell-a-def).
// E^II vanishes for r >= 2 R0.  Here the pair sum is taken inside the p integral:
//     sum_{j != k} w_j w_k E(r_jk) = int p^2 dp/(2 pi^2) S(p) omega^a omega^b,
//     S(p) = sum_{j != k} w_j w_k j_0(p r_jk),
// with S(p) from a fine histogram of the pair separations below 2 R0 that keeps
// the first two moments of r inside each bin (so S is exact to third order in
// the bin width), all in FP64:
//   k_pair_hist    ordered-pair weights and moments per separation bin;
//   k_e2_jbar      jbar^a_l W r^2 times the r quadrature weight, at the r nodes;
//   k_e2_omega     omega^a_l(p) at the p nodes;
//   k_e2_S         S(p) at the p nodes from the histogram;
//   k_e2_contract  the p integral, written as one extra FP64 partial row of the
//                  bispectrum primary sum: -(S1/V) sum_{j != k} w_j w_k E^{II}.
#include <algorithm>
#include <cmath>
#include <vector>

#include "hip_e2.h"

static __constant__ HipCoeffs c_coeffs;

cudaError_t hip_upload_coeffs_e2()
{
    return cudaMemcpyToSymbol(c_coeffs, &hip_host_coeffs(), sizeof(HipCoeffs));
}

static __constant__ int c_hshift[14][3] = {{0, 0, 0},  {1, -1, -1}, {1, -1, 0}, {1, -1, 1}, {1, 0, -1},
                                           {1, 0, 0},  {1, 0, 1},   {1, 1, -1}, {1, 1, 0},  {1, 1, 1},
                                           {0, 1, -1}, {0, 1, 0},   {0, 1, 1},  {0, 0, 1}};

// Pair separations below Rmax (= 2 R0), both orders of every pair: per bin b of
// width delta, H0 = sum w w, H1 = sum w w (r - b delta), H2 = sum w w (r - b delta)^2.
// One warp per work item (home cell, half-shell shift), lanes over neighbours.
__global__ void __launch_bounds__(128) k_pair_hist(CellList<float> cl, int n_items, int *counter, float Rmax2,
                                                   double delta, int nbin, double *H0, double *H1, double *H2)
{
    const int lane = threadIdx.x & 31;
    const int n_c = cl.n_c;
    for (;;) {
        int item = 0;
        if (lane == 0) item = atomicAdd(counter, 1);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= n_items) break;
        const int c = item / 14, q = item - c * 14;
        const int cx = c / (n_c * n_c), cy = (c / n_c) % n_c, cz = c % n_c;
        const int dx = c_hshift[q][0], dy = c_hshift[q][1], dz = c_hshift[q][2];
        const int nb = (((cx + dx + n_c) % n_c) * n_c + (cy + dy + n_c) % n_c) * n_c + (cz + dz + n_c) % n_c;
        float sx, sy, sz, lo;
        hip_cell_shift(cl, cx, dx, sx, lo);
        hip_cell_shift(cl, cy, dy, sy, lo);
        hip_cell_shift(cl, cz, dz, sz, lo);
        const int a0 = cl.cell_start[c], a1 = cl.cell_start[c + 1];
        const int b0 = cl.cell_start[nb], b1 = cl.cell_start[nb + 1];
        for (int i = a0; i < a1; ++i) {
            const float xi = cl.x[i] - sx, yi = cl.y[i] - sy, zi = cl.z[i] - sz;
            const double wi = cl.w[i];
            for (int j0 = (q == 0) ? i + 1 : b0; j0 < b1; j0 += 32) {
                const int j = j0 + lane;
                if (j >= b1) continue;
                const float ddx = xi - cl.x[j], ddy = yi - cl.y[j], ddz = zi - cl.z[j];
                const float r2 = ddx * ddx + ddy * ddy + ddz * ddz;
                if (!(r2 < Rmax2) || !(r2 > 0.0f)) continue;
                const double r = sqrt((double)r2);
                int b = (int)(r / delta);
                if (b >= nbin) b = nbin - 1;
                const double t = r - b * delta;
                const double ww = 2.0 * wi * (double)cl.w[j];
                atomicAdd(&H0[b], ww);
                atomicAdd(&H1[b], ww * t);
                atomicAdd(&H2[b], ww * t * t);
            }
        }
    }
}

// G[l][a][i] = rw_i r_i^2 W(r_i/R0) jbar^a_l(r_i): one thread per r node.
__global__ void k_e2_jbar(const double *__restrict__ rn, const double *__restrict__ rw, int nr,
                          const double *__restrict__ kedge, int n_e, double R0, double *G)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nr) return;
    const double r = rn[i];
    const int nk = n_e - 1;
    const double fac = rw[i] * r * r * hip_W<double>(r / R0);
    double Fp[5];
    hip_F_f64<31>(r * kedge[0], c_coeffs, Fp);
    double kp3 = kedge[0] * kedge[0] * kedge[0];
    for (int a = 0; a < nk; ++a) {
        double F[5];
        const double kn = kedge[a + 1], kn3 = kn * kn * kn;
        hip_F_f64<31>(r * kn, c_coeffs, F);
        const double jf = 3.0 / (kn3 - kp3);
        for (int l = 0; l <= HIP_LMAX; ++l) G[((size_t)l * nk + a) * nr + i] = fac * jf * (kn3 * F[l] - kp3 * Fp[l]);
        for (int l = 0; l <= HIP_LMAX; ++l) Fp[l] = F[l];
        kp3 = kn3;
    }
}

// Spherical Bessel j_l(z), l <= 4, in FP64: the power series below z = 2, the
// closed forms in sin z and cos z above (where their cancellation costs at most
// a factor ~500, i.e. ~1e-13).
__device__ double hip_sph_jl(int l, double z)
{
    if (z < 2.0) {
        // j_l(z) = z^l sum_k (-z^2/2)^k / (k! (2l + 2k + 1)!!)
        double df = 1.0;
        for (int q = 3; q <= 2 * l + 1; q += 2) df *= q;
        double term = 1.0 / df, sum = term;
        const double h = -0.5 * z * z;
        for (int k = 1; k < 24; ++k) {
            term *= h / (k * (2.0 * l + 2.0 * k + 1.0));
            sum += term;
        }
        double zl = 1.0;
        for (int q = 0; q < l; ++q) zl *= z;
        return sum * zl;
    }
    double s, c;
    sincos(z, &s, &c);
    const double w = 1.0 / z, w2 = w * w;
    switch (l) {
    case 0: return s * w;
    case 1: return (s * w - c) * w;
    case 2: return ((3.0 * w2 - 1.0) * s - 3.0 * w * c) * w;
    case 3: return ((15.0 * w2 - 6.0) * w * s - (15.0 * w2 - 1.0) * c) * w;
    default: return ((105.0 * w2 * w2 - 45.0 * w2 + 1.0) * s - (105.0 * w2 - 10.0) * w * c) * w;
    }
}

#define HIP_E2_ACH 16  // bins per thread in k_e2_omega

// om[l][a][q] = 4 pi sum_i G[l][a][i] j_l(p_q r_i): one thread per (l, q, 16 bins).
__global__ void k_e2_omega(const double *__restrict__ G, const double *__restrict__ rn, int nr,
                           const double *__restrict__ pn, int nq, int nk, int lmax, double *om)
{
    const int nch = (nk + HIP_E2_ACH - 1) / HIP_E2_ACH;
    const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (tid >= (long long)(lmax + 1) * nq * nch) return;
    const int ch = (int)(tid % nch), q = (int)((tid / nch) % nq), l = (int)(tid / ((long long)nch * nq));
    const double p = pn[q];
    double acc[HIP_E2_ACH];
#pragma unroll
    for (int u = 0; u < HIP_E2_ACH; ++u) acc[u] = 0.0;
    const int a0 = ch * HIP_E2_ACH;
    for (int i = 0; i < nr; ++i) {
        const double j = hip_sph_jl(l, p * rn[i]);
#pragma unroll
        for (int u = 0; u < HIP_E2_ACH; ++u)
            if (a0 + u < nk) acc[u] = fma(G[((size_t)l * nk + a0 + u) * nr + i], j, acc[u]);
    }
#pragma unroll
    for (int u = 0; u < HIP_E2_ACH; ++u)
        if (a0 + u < nk) om[((size_t)l * nk + a0 + u) * nq + q] = 4.0 * M_PI * acc[u];
}

// S[q] = sum_b [H0_b j_0(p x_b) + H1_b d/dx j_0(p x) + H2_b/2 d^2/dx^2 j_0(p x)] at
// x_b = b delta: one block per p node, threads over bins, block reduction.
__global__ void __launch_bounds__(256) k_e2_S(const double *__restrict__ H0, const double *__restrict__ H1,
                                              const double *__restrict__ H2, int nbin, double delta,
                                              const double *__restrict__ pn, double *S)
{
    __shared__ double red[256];
    const int q = blockIdx.x;
    const double p = pn[q];
    double acc = 0.0;
    for (int b = threadIdx.x; b < nbin; b += 256) {
        const double h0 = H0[b], h1 = H1[b], h2 = H2[b];
        if (h0 == 0.0 && h1 == 0.0 && h2 == 0.0) continue;
        const double z = p * b * delta;
        double j0, d1, d2;  // j_0(z), j_0'(z), j_0''(z)
        if (z < 0.05) {
            const double z2 = z * z;
            j0 = 1.0 - z2 / 6.0 + z2 * z2 / 120.0;
            d1 = z * (-1.0 / 3.0 + z2 / 30.0);
            d2 = -1.0 / 3.0 + z2 / 10.0 - z2 * z2 / 168.0;
        } else {
            double s, c;
            sincos(z, &s, &c);
            const double w = 1.0 / z;
            j0 = s * w;
            d1 = (c - s * w) * w;
            d2 = (-s - 2.0 * c * w + 2.0 * s * w * w) * w;
        }
        acc += h0 * j0 + p * h1 * d1 + 0.5 * p * p * h2 * d2;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) S[q] = red[0];
}

// row[(l nk + a) nk + b] = -(S1/V) sum_q pw_q p_q^2 S_q om^a_l om^b_l / (2 pi^2), l <= lmax
// (zero above): the random primaries' term of the bispectrum primary sum.
__global__ void k_e2_contract(const double *__restrict__ om, const double *__restrict__ S,
                              const double *__restrict__ pn, const double *__restrict__ pw, int nq, int nk, int lmax,
                              const double *S1, double V, double *row)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (HIP_LMAX + 1) * nk * nk) return;
    const int l = i / (nk * nk), ab = i - l * nk * nk, a = ab / nk, b = ab - a * nk;
    double acc = 0.0;
    if (l <= lmax) {
        const double *oa = om + ((size_t)l * nk + a) * nq, *ob = om + ((size_t)l * nk + b) * nq;
        for (int q = 0; q < nq; ++q) acc = fma(pw[q] * pn[q] * pn[q] * S[q], oa[q] * ob[q], acc);
        acc *= -(S1[0] / V) / (2.0 * M_PI * M_PI);
    }
    row[i] = acc;
}

// ------------------------------------------------------------------ host ----
static void gl_panels(double a, double b, double hmax, const std::vector<double> &gx, const std::vector<double> &gw,
                      std::vector<double> &x, std::vector<double> &w)
{
    const int n = std::max(1, (int)std::ceil((b - a) / hmax));
    const double h = (b - a) / n;
    for (int i = 0; i < n; ++i) {
        const double lo = a + i * h;
        for (size_t k = 0; k < gx.size(); ++k) {
            x.push_back(lo + 0.5 * h * (gx[k] + 1.0));
            w.push_back(0.5 * h * gw[k]);
        }
    }
}

void hip_gauss_legendre(int n, std::vector<double> &x, std::vector<double> &w);

// 16-point panels: a panel of width pi/(2 R0) covers a quarter period of
// j_0(p r) at r = 2 R0, one of width pi/p_max half a period of j_l(p r) at
// r = R0 -- far finer than 16-point Gauss-Legendre needs for 1e-12.
void hip_e2_nodes(const double *k_edges, int n_k, double R0, E2Nodes &nd)
{
    std::vector<double> gx, gw;
    hip_gauss_legendre(16, gx, gw);
    const double k_hi = k_edges[n_k];
    const double pmax = k_hi + 120.0 / R0;
    nd.p.clear();
    nd.pw.clear();
    gl_panels(0.0, pmax, M_PI / (2.0 * R0), gx, gw, nd.p, nd.pw);
    nd.r.clear();
    nd.rw.clear();
    const double hr = M_PI / std::max(pmax, k_hi);
    gl_panels(0.0, 0.5 * R0, hr, gx, gw, nd.r, nd.rw);
    gl_panels(0.5 * R0, 0.75 * R0, hr, gx, gw, nd.r, nd.rw);
    gl_panels(0.75 * R0, R0, hr, gx, gw, nd.r, nd.rw);
}

size_t hip_e2_scratch_bytes(const E2Nodes &nd, int n_k)
{
    const size_t nr = nd.r.size(), nq = nd.p.size();
    return sizeof(double) * (2 * nr + 2 * nq + (size_t)(n_k + 1) + 3 * (size_t)HIP_E2_NBIN +
                             (size_t)(HIP_LMAX + 1) * n_k * nr + (size_t)(HIP_LMAX + 1) * n_k * nq + nq) +
           64 * 8;
}

cudaError_t hip_e2_term(const CellList<float> &cl2, int n_items2, int *counter, double R0, double L,
                        const double *k_edges, int n_k, int lmax, const double *S1, const E2Nodes &nd, void *scratch,
                        double *row, unsigned long long *npairs2, cudaStream_t st)
{
    (void)npairs2;
    const int nr = (int)nd.r.size(), nq = (int)nd.p.size(), n_e = n_k + 1;
    double *d = (double *)scratch;
    double *rn = d, *rw = rn + nr, *pn = rw + nr, *pw = pn + nq, *ke = pw + nq;
    double *H0 = ke + n_e, *H1 = H0 + HIP_E2_NBIN, *H2 = H1 + HIP_E2_NBIN;
    double *G = H2 + HIP_E2_NBIN, *om = G + (size_t)(HIP_LMAX + 1) * n_k * nr, *S = om + (size_t)(HIP_LMAX + 1) * n_k * nq;
    cudaError_t e;
    if ((e = cudaMemcpyAsync(rn, nd.r.data(), sizeof(double) * nr, cudaMemcpyHostToDevice, st)) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(rw, nd.rw.data(), sizeof(double) * nr, cudaMemcpyHostToDevice, st)) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(pn, nd.p.data(), sizeof(double) * nq, cudaMemcpyHostToDevice, st)) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(pw, nd.pw.data(), sizeof(double) * nq, cudaMemcpyHostToDevice, st)) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(ke, k_edges, sizeof(double) * n_e, cudaMemcpyHostToDevice, st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(H0, 0, sizeof(double) * 3 * HIP_E2_NBIN, st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(counter, 0, sizeof(int), st)) != cudaSuccess) return e;
    const double Rmax = 2.0 * R0, delta = Rmax / HIP_E2_NBIN;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    k_pair_hist<<<sms * 8, 128, 0, st>>>(cl2, n_items2, counter, (float)(Rmax * Rmax), delta, HIP_E2_NBIN, H0, H1, H2);
    k_e2_jbar<<<(nr + 127) / 128, 128, 0, st>>>(rn, rw, nr, ke, n_e, R0, G);
    const long long nth = (long long)(lmax + 1) * nq * ((n_k + HIP_E2_ACH - 1) / HIP_E2_ACH);
    k_e2_omega<<<(unsigned)((nth + 127) / 128), 128, 0, st>>>(G, rn, nr, pn, nq, n_k, lmax, om);
    k_e2_S<<<nq, 256, 0, st>>>(H0, H1, H2, HIP_E2_NBIN, delta, pn, S);
    const int nout = (HIP_LMAX + 1) * n_k * n_k;
    k_e2_contract<<<(nout + 127) / 128, 128, 0, st>>>(om, S, pn, pw, nq, n_k, lmax, S1, L * L * L, row);
    return cudaGetLastError();
}

// r nodes of omega^a_l(p) at caller-given p: composite 16-point Gauss-Legendre on
// the three pieces of W, panels no wider than pi / max(p_max, k_hi), as for the
// DDR^II term.
static void omega_r_nodes(const double *k_edges, int n_k, double R0, const double *p, int n_p, std::vector<double> &rn,
                          std::vector<double> &rw)
{
    std::vector<double> gx, gw;
    hip_gauss_legendre(16, gx, gw);
    double pmax = k_edges[n_k];
    for (int q = 0; q < n_p; ++q) pmax = std::max(pmax, std::fabs(p[q]));
    const double hr = M_PI / pmax;
    rn.clear();
    rw.clear();
    gl_panels(0.0, 0.5 * R0, hr, gx, gw, rn, rw);
    gl_panels(0.5 * R0, 0.75 * R0, hr, gx, gw, rn, rw);
    gl_panels(0.75 * R0, R0, hr, gx, gw, rn, rw);
}

size_t hip_omega_scratch_bytes(const double *k_edges, int n_k, double R0, const double *p, int n_p)
{
    std::vector<double> rn, rw;
    omega_r_nodes(k_edges, n_k, R0, p, n_p, rn, rw);
    const size_t nr = rn.size();
    return sizeof(double) * (2 * nr + (size_t)(n_k + 1) + (size_t)n_p + (size_t)(HIP_LMAX + 1) * n_k * nr +
                             (size_t)(HIP_LMAX + 1) * n_k * n_p) +
           64 * 8;
}

// omega^a_l(p) of Eq. omega-ell-a-def at caller-given p, with the two kernels of
// the DDR^II term.
cudaError_t hip_omega_eval(const double *k_edges, int n_k, double R0, int lmax, const double *p, int n_p,
                           void *scratch, double *out, cudaStream_t st)
{
    std::vector<double> rn, rw;
    omega_r_nodes(k_edges, n_k, R0, p, n_p, rn, rw);
    const int nr = (int)rn.size(), n_e = n_k + 1;
    double *d = (double *)scratch;
    double *drn = d, *drw = drn + nr, *ke = drw + nr, *pn = ke + n_e, *G = pn + n_p;
    double *om = G + (size_t)(HIP_LMAX + 1) * n_k * nr;
    cudaError_t e;
    if ((e = cudaMemcpyAsync(drn, rn.data(), sizeof(double) * nr, cudaMemcpyHostToDevice, st)) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(drw, rw.data(), sizeof(double) * nr, cudaMemcpyHostToDevice, st)) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(ke, k_edges, sizeof(double) * n_e, cudaMemcpyHostToDevice, st)) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(pn, p, sizeof(double) * n_p, cudaMemcpyHostToDevice, st)) != cudaSuccess) return e;
    k_e2_jbar<<<(nr + 127) / 128, 128, 0, st>>>(drn, drw, nr, ke, n_e, R0, G);
    const long long nth = (long long)(lmax + 1) * n_p * ((n_k + HIP_E2_ACH - 1) / HIP_E2_ACH);
    k_e2_omega<<<(unsigned)((nth + 127) / 128), 128, 0, st>>>(G, drn, nr, pn, n_p, n_k, lmax, om);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return cudaMemcpyAsync(out, om, sizeof(double) * (lmax + 1) * n_k * n_p, cudaMemcpyDeviceToHost, st);
}

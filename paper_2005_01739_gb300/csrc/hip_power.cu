// Cell-list build, pair-pass dispatch and FP64 finalize of the power spectrum
// (Sec. 3 of arXiv:2005.01739).  The pair kernels themselves live in
// hip_pair_kernel.cuh, instantiated by the hip_pairs_*.cu units.  The FP64
// finalize sums the CTA partial rows, forms DD^a_l from adjacent edges,
// normalises and subtracts W~^a.
#include <cmath>
#include <cstdio>
#include <cstring>

#include "hip_internal.h"
#include "hip_moments.h"

static __constant__ HipCoeffs c_coeffs;

cudaError_t hip_upload_coeffs_power()
{
    cudaError_t e = cudaMemcpyToSymbol(c_coeffs, &hip_host_coeffs(), sizeof(HipCoeffs));
    if (e == cudaSuccess) e = hip_upload_coeffs_pairs_f32_lin();
    if (e == cudaSuccess) e = hip_upload_coeffs_pairs_f32_gen();
    if (e == cudaSuccess) e = hip_upload_coeffs_pairs_f64();
    if (e == cudaSuccess) e = hip_upload_coeffs_pairs_batched();
    if (e == cudaSuccess) e = hip_upload_coeffs_moments();
    if (e == cudaSuccess) e = hip_upload_pm_tables();
    return e;
}

// ------------------------------------------------------------- cell build ----
__device__ __forceinline__ double hip_wrap(double v, double L)
{
    v -= L * floor(v / L);
    if (v >= L) v -= L;
    if (v < 0.0) v = 0.0;
    return v;
}

// Box and cell geometry of a build: FP64 values and their FP32 companions.
struct CellGeom {
    double L, cs, inv_cs;
    float Lf_lo;     // largest float below L: 0 <= p <= Lf_lo  <=>  p in [0, L)
    float inv_cs_f;  // (float)(1 / cs)
    int n_c;
};

// Cell index along one axis of the FP32 coordinate p, by the FP64 rule
// floor(v / cs) (clamped to n_c - 1) with v = p wrapped into [0, L).  For p
// already in [0, L) (v = p) the index comes from an FP32 product, which is
// within 1.5e-5 of p / cs (p exact, 1/cs and the product rounded, p / cs < 128);
// only when it lies within 4e-5 of an integer does the FP64 product decide, so
// the index is the FP64 rule's at FP32 cost.  Other coordinates take the FP64
// wrap; *wrapped says which way v was formed.
__device__ __forceinline__ int hip_cell_axis(float p, const CellGeom &g, double &v, bool &wrapped)
{
    int ic;
    if (p >= 0.0f && p <= g.Lf_lo) {
        const float y = p * g.inv_cs_f;
        ic = (int)y;
        const float fr = y - (float)ic;
        if (fr < 4e-5f || fr > 0.99996f) ic = (int)((double)p * g.inv_cs);
        wrapped = false;
    } else {
        v = hip_wrap((double)p, g.L);
        ic = (int)(v * g.inv_cs);
        wrapped = true;
    }
    return ic >= g.n_c ? g.n_c - 1 : ic;
}

__global__ void k_cell_count(const float *__restrict__ pos, const float *__restrict__ w, long long N, CellGeom g,
                             int *__restrict__ cid, int *__restrict__ count, double *S1, int *err)
{
    const int n_c = g.n_c;
    double wsum = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        float px = pos[3 * i], py = pos[3 * i + 1], pz = pos[3 * i + 2];
        float wi = w ? w[i] : 1.0f;
        if (!isfinite(px) || !isfinite(py) || !isfinite(pz) || !isfinite(wi)) {
            atomicOr(err, 1);
            cid[i] = 0;
            continue;
        }
        int c3[3];
        float pv[3] = {px, py, pz};
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            double v;
            bool wr;
            c3[k] = hip_cell_axis(pv[k], g, v, wr);
        }
        int id = (c3[0] * n_c + c3[1]) * n_c + c3[2];
        cid[i] = id;
        atomicAdd(&count[id], 1);
        wsum += (double)wi;
    }
    __shared__ double red[32];
    for (int o = 16; o > 0; o >>= 1) wsum += __shfl_xor_sync(0xffffffffu, wsum, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = wsum;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0) atomicAdd(S1, v);
    }
}

// `count` and `fill` may alias: each thread reads its own segment before clearing it.
__global__ void __launch_bounds__(1024) k_cell_scan(const int *count, int n, int *__restrict__ start, int *fill)
{
    __shared__ int s[1024];
    int t = threadIdx.x;
    int per = (n + 1023) / 1024;
    int b = t * per, e = min(b + per, n);
    int sum = 0;
    for (int i = b; i < e; ++i) sum += count[i];
    s[t] = sum;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        int v = t >= off ? s[t - off] : 0;
        __syncthreads();
        s[t] += v;
        __syncthreads();
    }
    int run = s[t] - sum;
    for (int i = b; i < e; ++i) {
        const int ci = count[i];
        start[i] = run;
        fill[i] = 0;
        run += ci;
    }
    if (t == 1023) start[n] = s[1023];
}

template <typename T>
__global__ void k_cell_scatter(const float *__restrict__ pos, const float *__restrict__ w, long long N, CellGeom g,
                               const int *__restrict__ cid, const int *__restrict__ start, int *__restrict__ fill,
                               T *__restrict__ x, T *__restrict__ y, T *__restrict__ z, float *__restrict__ ws,
                               int *__restrict__ idx)
{
    // FP32 lists: the float cell origins, so that the offset of an unwrapped
    // coordinate is one exact FP32 subtraction (Sterbenz)
    __shared__ float s_org[HIP_MAX_CELLS_SIDE];
    for (int c = threadIdx.x; c < g.n_c; c += blockDim.x) s_org[c] = (float)hip_cell_origin<float>(c, g.cs);
    __syncthreads();
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        int id = cid[i];
        int slot = start[id] + atomicAdd(&fill[id], 1);
        float pv[3] = {pos[3 * i], pos[3 * i + 1], pos[3 * i + 2]};
        T loc[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            double v;
            bool wr;
            const int ic = hip_cell_axis(pv[k], g, v, wr);
            if (sizeof(T) == 4 && !wr)
                loc[k] = T(pv[k] - s_org[ic]);
            else
                loc[k] = (T)((wr ? v : (double)pv[k]) - hip_cell_origin<T>(ic, g.cs));
        }
        x[slot] = loc[0];
        y[slot] = loc[1];
        z[slot] = loc[2];
        ws[slot] = w ? w[i] : 1.0f;
        idx[slot] = (int)i;
    }
}

template <typename T>
cudaError_t hip_build_cells(const float *pos, const float *w, int64_t N, double L, int n_c, T *x, T *y, T *z,
                            float *ws, int *idx, int *cid, int *cell_start, int *cell_fill, double *S1, int *err,
                            cudaStream_t st)
{
    int n_cells = n_c * n_c * n_c;
    double cs = L / n_c;
    cudaError_t e;
    if ((e = cudaMemsetAsync(cell_fill, 0, sizeof(int) * n_cells, st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(S1, 0, sizeof(double), st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(err, 0, sizeof(int), st)) != cudaSuccess) return e;
    int blocks = (int)((N + 255) / 256);
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) blocks = 1;
    CellGeom g;
    g.L = L;
    g.cs = cs;
    g.inv_cs = 1.0 / cs;
    g.inv_cs_f = (float)g.inv_cs;
    g.Lf_lo = (float)L;
    if ((double)g.Lf_lo >= L) g.Lf_lo = std::nextafter(g.Lf_lo, 0.0f);
    g.n_c = n_c;
    k_cell_count<<<blocks, 256, 0, st>>>(pos, w, N, g, cid, cell_fill, S1, err);
    k_cell_scan<<<1, 1024, 0, st>>>(cell_fill, n_cells, cell_start, cell_fill);
    k_cell_scatter<T><<<blocks, 256, 0, st>>>(pos, w, N, g, cid, cell_start, cell_fill, x, y, z, ws, idx);
    return cudaGetLastError();
}

template cudaError_t hip_build_cells<float>(const float *, const float *, int64_t, double, int, float *, float *,
                                            float *, float *, int *, int *, int *, int *, double *, int *,
                                            cudaStream_t);
template cudaError_t hip_build_cells<double>(const float *, const float *, int64_t, double, int, double *, double *,
                                             double *, float *, int *, int *, int *, int *, double *, int *,
                                             cudaStream_t);

template <typename T>
int hip_power_grid()
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int nb = sizeof(T) == 4 ? hip_pairs_blocks_per_sm_f32() : hip_pairs_blocks_per_sm_f64();
    return sms * (nb < 1 ? 1 : nb);
}
template int hip_power_grid<float>();
template int hip_power_grid<double>();

static void hip_pairs_launch(bool lin, const CellList<float> &cl, const PowerKernelArgs &a,
                             const EdgeTable<float> &ed, int n_ell, float R0, float dhi, float dlo, int grid,
                             cudaStream_t st)
{
    if (lin)
        hip_pairs_launch_f32_lin(cl, a, ed, n_ell, R0, dhi, dlo, grid, st);
    else
        hip_pairs_launch_f32_gen(cl, a, ed, n_ell, R0, dhi, dlo, grid, st);
}

static void hip_pairs_launch(bool lin, const CellList<double> &cl, const PowerKernelArgs &a,
                             const EdgeTable<double> &ed, int n_ell, double R0, double dhi, double dlo, int grid,
                             cudaStream_t st)
{
    hip_pairs_launch_f64(lin, cl, a, ed, n_ell, R0, dhi, dlo, grid, st);
}

// Are the edges uniformly spaced (to 1e-12 of their magnitude)?
static bool edges_linear(const double *k, int n_e, double *dk)
{
    if (n_e < 2) return false;
    const double d = (k[n_e - 1] - k[0]) / (n_e - 1);
    for (int e = 0; e < n_e; ++e)
        if (std::fabs(k[e] - (k[0] + e * d)) > 1e-12 * (std::fabs(k[n_e - 1]) + std::fabs(k[0]))) return false;
    *dk = d;
    return true;
}

template <typename T>
cudaError_t hip_power_pairs(const CellList<T> &cl, const PowerKernelArgs &a, const double *kedges, int n_ell,
                            double R0, int grid, cudaStream_t st)
{
    EdgeTable<T> ed;
    double dk = 0.0;
    const bool lin = edges_linear(kedges, a.n_e, &dk);
    for (int e = 0; e < HIP_MAX_EDGES; ++e) {
        const double k = e < a.n_e ? kedges[e] : 0.0;
        ed.k[e] = (T)k;
        ed.klo[e] = (T)(k - (double)ed.k[e]);
    }
    const double d32 = 32.0 * dk;
    const T dhi = (T)d32, dlo = (T)(d32 - (double)dhi);
    hip_pairs_launch(lin, cl, a, ed, n_ell, (T)R0, dhi, dlo, grid, st);
    return cudaGetLastError();
}
template cudaError_t hip_power_pairs<float>(const CellList<float> &, const PowerKernelArgs &, const double *, int,
                                            double, int, cudaStream_t);
template cudaError_t hip_power_pairs<double>(const CellList<double> &, const PowerKernelArgs &, const double *, int,
                                             double, int, cudaStream_t);

// --------------------------------------------------------------- finalize ----
struct FinalArgs {
    double k[HIP_MAX_EDGES];
    double glx[16], glw[16];
};

// W~^a = 4 pi int_0^R0 r^2 jbar^a_0(r) W(r/R0) dr (Eq. wka-def), composite
// 16-point Gauss-Legendre on the three polynomial pieces of W, panels no wider
// than pi / (4 k_hi).  One CTA per bin.
__global__ void k_window_transform(FinalArgs f, double R0, double *Wt)
{
    const int a = blockIdx.x;
    const double klo = f.k[a], khi = f.k[a + 1];
    const double k3lo = klo * klo * klo, k3hi = khi * khi * khi;
    const double hmax = 3.14159265358979323846 / (4.0 * khi);
    const double brk[4] = {0.0, 0.5 * R0, 0.75 * R0, R0};
    double acc = 0.0;
    for (int piece = 0; piece < 3; ++piece) {
        const double lo = brk[piece], len = brk[piece + 1] - brk[piece];
        const int np = max(1, (int)ceil(len / hmax));
        const double h = len / np;
        for (int i = threadIdx.x; i < np * 16; i += blockDim.x) {
            const int p = i >> 4, q = i & 15;
            const double r = lo + h * (p + 0.5 * (f.glx[q] + 1.0));
            double Fh[5], Fl[5];
            hip_F_f64<1>(r * khi, c_coeffs, Fh);
            hip_F_f64<1>(r * klo, c_coeffs, Fl);
            const double jb = 3.0 * (k3hi * Fh[0] - k3lo * Fl[0]) / (k3hi - k3lo);
            acc += 0.5 * h * f.glw[q] * r * r * jb * hip_W<double>(r / R0);
        }
    }
    __shared__ double red[32];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0) Wt[a] = 4.0 * 3.14159265358979323846 * v;
    }
}

// Sum of the CTA partials (fixed order), DD^a_l from adjacent edges, and
// P^a_l = (-1)^(l/2) (2l+1) DD^a_l / (n_w^2 V) - delta_l0 W~^a.
__global__ void __launch_bounds__(1024) k_power_final(FinalArgs f, const double *__restrict__ partials, int nparts,
                                                      int n_e, int n_ell, double L, const double *S1,
                                                      const double *__restrict__ Wt, double *DD, double *P)
{
    __shared__ double H[3][HIP_MAX_EDGES];
    for (int i = threadIdx.x; i < n_ell * n_e; i += blockDim.x) {
        double s = 0.0;
        for (int p = 0; p < nparts; ++p) s += partials[(size_t)p * 3 * n_e + i];
        H[i / n_e][i % n_e] = s;
    }
    __syncthreads();
    const int n_k = n_e - 1;
    const double V = L * L * L;
    const double nw = S1[0] / V;
    for (int i = threadIdx.x; i < n_ell * n_k; i += blockDim.x) {
        const int il = i / n_k, a = i - il * n_k;
        const double k3lo = f.k[a] * f.k[a] * f.k[a], k3hi = f.k[a + 1] * f.k[a + 1] * f.k[a + 1];
        const double dd = 3.0 * (H[il][a + 1] - H[il][a]) / (k3hi - k3lo);
        const int l = 2 * il;
        const double sign = (il & 1) ? -1.0 : 1.0;
        double p = sign * (2.0 * l + 1.0) * dd / (nw * nw * V);
        if (il == 0) p -= Wt[a];
        DD[i] = dd;
        P[i] = p;
    }
}

// Batched FP64 finalize: W~^a for every (catalog, bin), then DD and P per catalog.
struct GL16 {
    double x[16], w[16];
};

__global__ void k_window_transform_batched(const FinalCat *__restrict__ cats, GL16 g)
{
    const FinalCat &f = cats[blockIdx.y];
    const int a = blockIdx.x;
    if (a >= f.n_e - 1) return;
    const double klo = f.k[a], khi = f.k[a + 1], R0 = f.R0;
    const double k3lo = klo * klo * klo, k3hi = khi * khi * khi;
    const double hmax = 3.14159265358979323846 / (4.0 * khi);
    const double brk[4] = {0.0, 0.5 * R0, 0.75 * R0, R0};
    double acc = 0.0;
    for (int piece = 0; piece < 3; ++piece) {
        const double lo = brk[piece], len = brk[piece + 1] - brk[piece];
        const int np = max(1, (int)ceil(len / hmax));
        const double h = len / np;
        for (int i = threadIdx.x; i < np * 16; i += blockDim.x) {
            const int p = i >> 4, q = i & 15;
            const double r = lo + h * (p + 0.5 * (g.x[q] + 1.0));
            double Fh[5], Fl[5];
            hip_F_f64<1>(r * khi, c_coeffs, Fh);
            hip_F_f64<1>(r * klo, c_coeffs, Fl);
            const double jb = 3.0 * (k3hi * Fh[0] - k3lo * Fl[0]) / (k3hi - k3lo);
            acc += 0.5 * h * g.w[q] * r * r * jb * hip_W<double>(r / R0);
        }
    }
    __shared__ double red[32];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0) f.Wt[a] = 4.0 * 3.14159265358979323846 * v;
    }
}

__global__ void k_power_final_batched(const FinalCat *__restrict__ cats)
{
    const FinalCat &f = cats[blockIdx.x];
    const int n_e = f.n_e, n_k = n_e - 1;
    const double V = f.L * f.L * f.L, nw = f.S1[0] / V;
    for (int i = threadIdx.x; i < f.n_ell * n_k; i += blockDim.x) {
        const int il = i / n_k, a = i - il * n_k;
        const double k3lo = f.k[a] * f.k[a] * f.k[a], k3hi = f.k[a + 1] * f.k[a + 1] * f.k[a + 1];
        const double dd = 3.0 * (f.acc[il * n_e + a + 1] - f.acc[il * n_e + a]) / (k3hi - k3lo);
        const int l = 2 * il;
        double p = ((il & 1) ? -1.0 : 1.0) * (2.0 * l + 1.0) * dd / (nw * nw * V);
        if (il == 0) p -= f.Wt[a];
        f.DD[i] = dd;
        f.P[i] = p;
    }
}

static void gl16(double *x, double *w);

cudaError_t hip_power_finalize_batched(const FinalCat *cats, int n_cats, int nk_max, cudaStream_t st)
{
    GL16 g;
    gl16(g.x, g.w);
    k_window_transform_batched<<<dim3(nk_max, n_cats), 256, 0, st>>>(cats, g);
    k_power_final_batched<<<n_cats, 256, 0, st>>>(cats);
    return cudaGetLastError();
}

static void gl16(double *x, double *w)
{
    for (int i = 0; i < 16; ++i) {
        double z = cos(3.14159265358979323846 * (i + 0.75) / 16.5), p1 = 0, p0 = 0, dp = 0;
        for (int it = 0; it < 100; ++it) {
            p0 = 1.0;
            p1 = z;
            for (int k = 2; k <= 16; ++k) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = 16.0 * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        p0 = 1.0;
        p1 = z;
        for (int k = 2; k <= 16; ++k) {
            double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        dp = 16.0 * (z * p1 - p0) / (z * z - 1.0);
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

cudaError_t hip_power_finalize(const double *partials, int nparts, int n_e, int n_ell, const double *kedges_host,
                               double R0, double L, const double *S1, double *Wt, double *DD, double *P,
                               cudaStream_t st)
{
    FinalArgs f;
    for (int e = 0; e < HIP_MAX_EDGES; ++e) f.k[e] = e < n_e ? kedges_host[e] : 0.0;
    gl16(f.glx, f.glw);
    k_window_transform<<<n_e - 1, 256, 0, st>>>(f, R0, Wt);
    k_power_final<<<1, 1024, 0, st>>>(f, partials, nparts, n_e, n_ell, L, S1, Wt, DD, P);
    return cudaGetLastError();
}

// P^a_l from summed ordered pair sums DD^a_l (the same normalisation as k_power_final).
__global__ void k_power_from_dd(const double *__restrict__ DD, int n_k, int n_ell, double L, double S1,
                                const double *__restrict__ Wt, double *__restrict__ P)
{
    const double V = L * L * L, nw = S1 / V;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_ell * n_k; i += gridDim.x * blockDim.x) {
        const int il = i / n_k, a = i - il * n_k;
        const double sign = (il & 1) ? -1.0 : 1.0;
        double p = sign * (4.0 * il + 1.0) * DD[i] / (nw * nw * V);
        if (il == 0) p -= Wt[a];
        P[i] = p;
    }
}

cudaError_t hip_power_from_dd(const double *DD, int n_k, int n_ell, double L, double S1, const double *Wt, double *P,
                              cudaStream_t st)
{
    k_power_from_dd<<<1, 256, 0, st>>>(DD, n_k, n_ell, L, S1, Wt, P);
    return cudaGetLastError();
}

cudaError_t hip_window_transform(int n_e, const double *kedges_host, double R0, double *Wt, cudaStream_t st)
{
    FinalArgs f;
    std::memset(&f, 0, sizeof(f));
    for (int e = 0; e < HIP_MAX_EDGES; ++e) f.k[e] = e < n_e ? kedges_host[e] : 0.0;
    gl16(f.glx, f.glw);
    k_window_transform<<<n_e - 1, 256, 0, st>>>(f, R0, Wt);
    return cudaGetLastError();
}

// Power-spectrum pair pass by Legendre moments of the separation.
//
// The pair sum of Sec. 3 asks, for every bin edge k_e and multipole l, for
//     S_l(k_e) = sum_pairs omega L_l(mu) f_e(r),   f_e(r) = k_e^3 F_l(r k_e),
// (omega = w_i w_j W(r/R0); the edge sums the direct kernel accumulates).  f_e is
// an entire function of r, so on a short interval [c dc, (c+1) dc) it is a
// rapidly converging Legendre series f_e(r) = sum_m a^{e}_{c m} P_m(t), t the
// position in the interval mapped to [-1, 1].  Hence
//     S_l(k_e) = sum_c sum_m a^{e l}_{c m} M^l_{c m},  M^l_{c m} = sum_{pairs in c} omega L_l(mu) P_m(t),
// and the pair loop only accumulates the moments M (HIP_PM_M per bin and l)
// instead of evaluating every edge: O(M n_l) per pair instead of O(n_e n_l).
// The coefficients a come from 24-point Gauss-Legendre projection of f_e in FP64
// (once per call), the final contraction is FP64.  With dc = R0 / n_c and
// n_c >= R0 k_max / 2, k dc / 2 <= 1 and the truncation after 16 terms is below
// ~1 / 16! ~ 5e-14 of f, i.e. exact for both precisions; the FP32 path keeps
// FP32 moments per warp in shared memory and folds them into FP64 every
// HIP_PM_FOLD pairs.
#define HIP_PAIR_UPLOAD hip_upload_coeffs_moments
#include "hip_pair_kernel.cuh"

#include <vector>

#include "hip_moments.h"

#define HIP_PM_NG 24
#define HIP_PM_WARPS 4
#define HIP_PM_FOLD 65536  // pairs a warp adds into its FP32 moments before folding them to FP64

__constant__ double c_pm_gw[HIP_PM_NG];           // Gauss-Legendre weights on [-1, 1]
__constant__ double c_pm_gx[HIP_PM_NG];           // and nodes
__constant__ double c_pm_P[HIP_PM_NG][HIP_PM_M];  // P_m at the nodes

cudaError_t hip_upload_pm_tables()
{
    void hip_gauss_legendre(int n, std::vector<double> &x, std::vector<double> &w);
    std::vector<double> x, w;
    hip_gauss_legendre(HIP_PM_NG, x, w);
    double P[HIP_PM_NG][HIP_PM_M];
    for (int g = 0; g < HIP_PM_NG; ++g) {
        P[g][0] = 1.0;
        P[g][1] = x[g];
        for (int m = 1; m + 1 < HIP_PM_M; ++m) P[g][m + 1] = ((2.0 * m + 1.0) * x[g] * P[g][m] - m * P[g][m - 1]) / (m + 1.0);
    }
    cudaError_t e = cudaMemcpyToSymbol(c_pm_gw, w.data(), sizeof(double) * HIP_PM_NG);
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_pm_gx, x.data(), sizeof(double) * HIP_PM_NG);
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_pm_P, P, sizeof(P));
    return e;
}

// a[((il n_e + e) n_c + c) M + m] = (2m+1)/2 int_{-1}^{1} f_e(r(t)) P_m(t) dt, one
// thread per (edge, interval).
__global__ void k_pm_coeffs(const double *__restrict__ kedge, int n_e, int n_c, double dc, int n_ell, double *a)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n_e * n_c) return;
    const int e = idx / n_c, c = idx - e * n_c;
    const double k = kedge[e], k3 = k * k * k;
    double acc[3][HIP_PM_M];
#pragma unroll
    for (int il = 0; il < 3; ++il)
#pragma unroll
        for (int m = 0; m < HIP_PM_M; ++m) acc[il][m] = 0.0;
    for (int g = 0; g < HIP_PM_NG; ++g) {
        const double r = (c + 0.5 * (1.0 + c_pm_gx[g])) * dc;
        double F[5];
        hip_F_f64<21>(r * k, c_coeffs, F);
        const double s = k3 * c_pm_gw[g];
        const double f0 = s * F[0], f2 = s * F[2], f4 = s * F[4];
#pragma unroll
        for (int m = 0; m < HIP_PM_M; ++m) {
            const double p = c_pm_P[g][m];
            acc[0][m] = fma(f0, p, acc[0][m]);
            acc[1][m] = fma(f2, p, acc[1][m]);
            acc[2][m] = fma(f4, p, acc[2][m]);
        }
    }
    for (int il = 0; il < n_ell; ++il)
#pragma unroll
        for (int m = 0; m < HIP_PM_M; ++m)
            a[(((size_t)il * n_e + e) * n_c + c) * HIP_PM_M + m] = 0.5 * (2.0 * m + 1.0) * acc[il][m];
}

// Per-warp staging of the pair kernel: tiles of the two cells and the queue of
// accepted pairs (separation hi + lo, line-of-sight component, weight).
template <typename T>
struct PmWarp {
    T hx[HIP_WTILE], hy[HIP_WTILE], hz[HIP_WTILE];
    float hw[HIP_WTILE];
    int hin[HIP_WTILE];
    T nx[HIP_WTILE], ny[HIP_WTILE], nz[HIP_WTILE];
    float nw[HIP_WTILE];
    int nin[HIP_WTILE];
    T qr[HIP_QCAP], qrl[HIP_QCAP], qdl[HIP_QCAP];
    T qw[HIP_QCAP];  // w_i w_j times the ordered pairs counted (formed in T: FP64 keeps the product exact)
};

__device__ __forceinline__ void hip_pm_add(float *M, float v) { atomicAdd(M, v); }
__device__ __forceinline__ void hip_pm_add(double *M, double v) { atomicAdd(M, v); }

// Moments of the n queued pairs, one pair per lane: M[(il M + m) n_c + c] += omega L_l P_m(t).
template <typename T, int MASK>
__device__ __forceinline__ void hip_pm_drain(const PmWarp<T> &sm, int n, int lane, T *M, int n_c, T dc, T inv_hdc,
                                             T invR0)
{
    for (int i = lane; i < n; i += 32) {
        const T r = sm.qr[i], rl = sm.qrl[i];
        const T mu = sm.qdl[i] / r;
        T l2, l4;
        hip_legendre24<T>(mu, l2, l4);
        const T om = sm.qw[i] * hip_W<T>(r * invR0);
        int c = (int)(r / dc);
        c = c < n_c - 1 ? c : n_c - 1;
        // t in [-1, 1]: r - c dc is exact in FP32 for c >= 1 (Sterbenz), the low part rl added after
        const T t = ((r - T(c) * dc) + rl) * inv_hdc - T(1);
        const T o0 = om, o2 = om * l2, o4 = om * l4;
        T p0 = T(1), p1 = t;
        T *M0 = M + c, *M2 = M + (size_t)HIP_PM_M * n_c + c, *M4 = M + (size_t)2 * HIP_PM_M * n_c + c;
        hip_pm_add(M0, o0);
        if (MASK & 4) hip_pm_add(M2, o2);
        if (MASK & 16) hip_pm_add(M4, o4);
        hip_pm_add(M0 + n_c, o0 * p1);
        if (MASK & 4) hip_pm_add(M2 + n_c, o2 * p1);
        if (MASK & 16) hip_pm_add(M4 + n_c, o4 * p1);
#pragma unroll
        for (int m = 1; m + 1 < HIP_PM_M; ++m) {
            // (m+1) P_{m+1} = (2m+1) t P_m - m P_{m-1}
            const T p2 = (T(2 * m + 1) * t * p1 - T(m) * p0) * T(1.0 / (m + 1));
            p0 = p1;
            p1 = p2;
            hip_pm_add(M0 + (size_t)(m + 1) * n_c, o0 * p2);
            if (MASK & 4) hip_pm_add(M2 + (size_t)(m + 1) * n_c, o2 * p2);
            if (MASK & 16) hip_pm_add(M4 + (size_t)(m + 1) * n_c, o4 * p2);
        }
    }
}

// Fold a moment array into the FP64 totals and clear it (lanes of one warp, or
// the whole CTA when nthreads = blockDim.x).
template <typename T>
__device__ __forceinline__ void hip_pm_fold(T *M, int len, double *Mg, int tid, int nthreads)
{
    for (int i = tid; i < len; i += nthreads) {
        const T v = M[i];
        if (v != T(0)) atomicAdd(&Mg[i], (double)v);
        M[i] = T(0);
    }
}

// The pair pass: warps take work items (home cell, half-shell shift) as in the
// direct kernel, test candidates one per lane, queue accepted pairs (r as hi + lo
// for FP32), and at 32 queued pairs add their moments.  FP32: moments per warp
// (dynamic shared memory [warps][3][M][n_c]), folded every HIP_PM_FOLD pairs.
// FP64: one moment array per CTA, folded at the end.
template <typename T, int MASK>
__global__ void __launch_bounds__(HIP_PM_WARPS * 32)
    k_power_moments(CellList<T> cl, PowerKernelArgs a, T R0, int n_c, T dc, double *Mg)
{
    __shared__ PmWarp<T> smem[HIP_PM_WARPS];
    extern __shared__ __align__(16) unsigned char pm_raw[];
    constexpr bool PERWARP = sizeof(T) == 4;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    PmWarp<T> &sm = smem[warp];
    const int len = 3 * HIP_PM_M * n_c;
    T *M = reinterpret_cast<T *>(pm_raw) + (PERWARP ? (size_t)warp * len : 0);
    for (int i = (PERWARP ? lane : threadIdx.x); i < len; i += (PERWARP ? 32 : blockDim.x)) M[i] = T(0);
    __syncthreads();
    const T R0sq = R0 * R0, invR0 = T(1) / R0, inv_hdc = T(2) / dc;
    const unsigned lt_mask = (1u << lane) - 1u;
    const int n_c3 = cl.n_c;
    unsigned long long cnt = 0;
    int qn = 0;
    long long since_fold = 0;
    for (;;) {
        int item = 0;
        if (lane == 0) item = atomicAdd(a.work_counter, 1);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= a.n_items) break;
        const int c = item / HIP_NSHIFT, q = item - c * HIP_NSHIFT;
        const int cx = c / (n_c3 * n_c3), cy = (c / n_c3) % n_c3, cz = c % n_c3;
        const int dx = c_shift[q][0], dy = c_shift[q][1], dz = c_shift[q][2];
        const int nb = (((cx + dx + n_c3) % n_c3) * n_c3 + (cy + dy + n_c3) % n_c3) * n_c3 + (cz + dz + n_c3) % n_c3;
        T sx, sy, sz, sxl, syl, szl;
        hip_cell_shift(cl, cx, dx, sx, sxl);
        hip_cell_shift(cl, cy, dy, sy, syl);
        hip_cell_shift(cl, cz, dz, sz, szl);
        const int a0 = cl.cell_start[c], a1 = cl.cell_start[c + 1];
        const int b0 = cl.cell_start[nb], b1 = cl.cell_start[nb + 1];
        const bool self = (q == 0);
        for (int hb = a0; hb < a1; hb += HIP_WTILE) {
            const int hn = min(HIP_WTILE, a1 - hb);
            __syncwarp();
            for (int i = lane; i < hn; i += 32) {
                sm.hx[i] = cl.x[hb + i];
                sm.hy[i] = cl.y[hb + i];
                sm.hz[i] = cl.z[hb + i];
                sm.hw[i] = cl.w[hb + i];
                const long long oi = cl.idx[hb + i];
                sm.hin[i] = (oi >= a.p0 && oi < a.p1) ? 1 : 0;
            }
            for (int nbs = self ? hb : b0; nbs < b1; nbs += HIP_WTILE) {
                const int nn = min(HIP_WTILE, b1 - nbs);
                __syncwarp();
                for (int i = lane; i < nn; i += 32) {
                    sm.nx[i] = cl.x[nbs + i];
                    sm.ny[i] = cl.y[nbs + i];
                    sm.nz[i] = cl.z[nbs + i];
                    sm.nw[i] = cl.w[nbs + i];
                    const long long oi = cl.idx[nbs + i];
                    sm.nin[i] = (oi >= a.p0 && oi < a.p1) ? 1 : 0;
                }
                __syncwarp();
                const bool same = self && (nbs == hb);
                for (int il = 0; il < hn; ++il) {
                    const T hx = sm.hx[il], hy = sm.hy[il], hz = sm.hz[il];
                    const T xi = hx - sx, yi = hy - sy, zi = hz - sz;
                    const T xil = hip_low(hx, -sx, xi) - sxl, yil = hip_low(hy, -sy, yi) - syl,
                            zil = hip_low(hz, -sz, zi) - szl;
                    const float wi = sm.hw[il];
                    const int ini = sm.hin[il];
                    for (int jb = same ? il + 1 : 0; jb < nn; jb += 32) {
                        const int jl = jb + lane;
                        bool ok = false;
                        T ddx = T(0), ddy = T(0), ddz = T(0);
                        int mult = 0;
                        if (jl < nn) {
                            ddx = xi - sm.nx[jl];
                            ddy = yi - sm.ny[jl];
                            ddz = zi - sm.nz[jl];
                            const T r2 = ddx * ddx + ddy * ddy + ddz * ddz;
                            mult = ini + sm.nin[jl];
                            ok = (r2 < R0sq) && (r2 > T(0)) && (mult > 0);
                        }
                        const unsigned m = __ballot_sync(0xffffffffu, ok);
                        if (ok) {
                            T r, rl;
                            hip_pair_sep(xi, xil, yi, yil, zi, zil, sm.nx[jl], sm.ny[jl], sm.nz[jl], ddx, ddy, ddz,
                                         &r, &rl);
                            const int slot = qn + __popc(m & lt_mask);
                            sm.qr[slot] = r;
                            sm.qrl[slot] = rl;
                            sm.qdl[slot] = a.los == 0 ? ddx : (a.los == 1 ? ddy : ddz);
                            sm.qw[slot] = T(wi) * T(sm.nw[jl]) * T(mult);
                            cnt += (unsigned long long)mult;
                        }
                        qn += __popc(m);
                        if (qn >= 32) {
                            __syncwarp();
                            hip_pm_drain<T, MASK>(sm, qn, lane, M, n_c, dc, inv_hdc, invR0);
                            since_fold += qn;
                            qn = 0;
                            __syncwarp();
                            if (PERWARP && since_fold >= HIP_PM_FOLD) {
                                hip_pm_fold(M, len, Mg, lane, 32);
                                since_fold = 0;
                                __syncwarp();
                            }
                        }
                    }
                }
            }
        }
    }
    if (qn > 0) {
        __syncwarp();
        hip_pm_drain<T, MASK>(sm, qn, lane, M, n_c, dc, inv_hdc, invR0);
        __syncwarp();
    }
    if (PERWARP) {
        hip_pm_fold(M, len, Mg, lane, 32);
    } else {
        __syncthreads();
        hip_pm_fold(M, len, Mg, threadIdx.x, blockDim.x);
    }
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    if (lane == 0 && cnt) atomicAdd(a.npairs, cnt);
}

// S[il][e] = sum_c sum_m a[il][e][c][m] Mg[il][m][c]: one block per (il, e),
// written as one partial row [3][n_e] of the power finalize.
__global__ void __launch_bounds__(256) k_pm_contract(const double *__restrict__ a, const double *__restrict__ Mg,
                                                     int n_e, int n_c, double *row)
{
    __shared__ double red[256];
    const int il = blockIdx.x / n_e, e = blockIdx.x - il * n_e;
    const double *ae = a + ((size_t)il * n_e + e) * n_c * HIP_PM_M;
    const double *mg = Mg + (size_t)il * HIP_PM_M * n_c;
    double acc = 0.0;
    for (int i = threadIdx.x; i < n_c * HIP_PM_M; i += 256) {
        const int c = i / HIP_PM_M, m = i - c * HIP_PM_M;
        acc = fma(ae[i], mg[(size_t)m * n_c + c], acc);
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) row[il * n_e + e] = red[0];
}

// ------------------------------------------------------------------ host ----
int hip_pm_intervals(double R0, double k_max)
{
    const int n = (int)std::ceil(R0 * k_max / 2.0);
    return n < 8 ? 8 : n;
}

size_t hip_pm_scratch_bytes(int n_e, int n_c)
{
    return sizeof(double) * ((size_t)n_e + (size_t)3 * n_e * n_c * HIP_PM_M + (size_t)3 * HIP_PM_M * n_c) + 256;
}

template <typename T>
static size_t pm_dyn_smem(int n_c)
{
    return sizeof(T) * 3 * HIP_PM_M * (size_t)n_c * (sizeof(T) == 4 ? HIP_PM_WARPS : 1);
}

bool hip_pm_applicable(double R0, double k_max, bool fp32)
{
    const int n_c = hip_pm_intervals(R0, k_max);
    if (n_c > HIP_PM_NCMAX) return false;
    const size_t dyn = fp32 ? pm_dyn_smem<float>(n_c) : pm_dyn_smem<double>(n_c);
    return dyn + sizeof(PmWarp<double>) * HIP_PM_WARPS <= 220 * 1024;
}

template <typename T, int MASK>
static cudaError_t pm_launch(const CellList<T> &cl, const PowerKernelArgs &a, T R0, int n_c, T dc, double *Mg,
                             cudaStream_t st)
{
    const size_t dyn = pm_dyn_smem<T>(n_c);
    cudaError_t e = cudaFuncSetAttribute(k_power_moments<T, MASK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)dyn);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, nb = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_power_moments<T, MASK>, HIP_PM_WARPS * 32, dyn);
    const int grid = sms * (nb < 1 ? 1 : nb);
    k_power_moments<T, MASK><<<grid, HIP_PM_WARPS * 32, dyn, st>>>(cl, a, R0, n_c, dc, Mg);
    return cudaGetLastError();
}

template <typename T>
cudaError_t hip_power_moments(const CellList<T> &cl, const PowerKernelArgs &a, const double *kedges, int n_ell,
                              double R0, void *scratch, double *row, cudaStream_t st)
{
    const int n_e = a.n_e;
    const int n_c = hip_pm_intervals(R0, kedges[n_e - 1]);
    const double dc = R0 / n_c;
    double *ke = (double *)scratch;
    double *coef = ke + n_e;
    double *Mg = coef + (size_t)3 * n_e * n_c * HIP_PM_M;
    cudaError_t e;
    if ((e = cudaMemcpyAsync(ke, kedges, sizeof(double) * n_e, cudaMemcpyHostToDevice, st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(Mg, 0, sizeof(double) * 3 * HIP_PM_M * n_c, st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(row, 0, sizeof(double) * 3 * n_e, st)) != cudaSuccess) return e;
    k_pm_coeffs<<<(n_e * n_c + 127) / 128, 128, 0, st>>>(ke, n_e, n_c, dc, n_ell, coef);
    if (n_ell == 3)
        e = pm_launch<T, 21>(cl, a, (T)R0, n_c, (T)dc, Mg, st);
    else if (n_ell == 2)
        e = pm_launch<T, 5>(cl, a, (T)R0, n_c, (T)dc, Mg, st);
    else
        e = pm_launch<T, 1>(cl, a, (T)R0, n_c, (T)dc, Mg, st);
    if (e != cudaSuccess) return e;
    k_pm_contract<<<n_ell * n_e, 256, 0, st>>>(coef, Mg, n_e, n_c, row);
    return cudaGetLastError();
}
template cudaError_t hip_power_moments<float>(const CellList<float> &, const PowerKernelArgs &, const double *, int,
                                              double, void *, double *, cudaStream_t);
template cudaError_t hip_power_moments<double>(const CellList<double> &, const PowerKernelArgs &, const double *,
                                               int, double, void *, double *, cudaStream_t);

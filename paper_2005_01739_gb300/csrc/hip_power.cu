// Cell-list build and power-spectrum pair kernels (Sec. 3 of arXiv:2005.01739).
//
// Pair pass: persistent CTAs pull work items (home cell, one of 14 half-shell
// shifts) from an atomic counter.  A CTA stages a tile of the home cell and a
// tile of the shifted neighbour cell in shared memory (positions as cell-local
// offsets, so separations keep full precision whatever the box size), each warp
// tests candidate pairs with one lane per candidate and appends accepted pairs to
// a per-warp queue.  The queue is drained with one lane per bin EDGE: for every
// queued pair each lane evaluates F_l(r k_e) at its own edges and accumulates
// omega_l F_l into registers.  No lane ever writes another lane's edge, so there
// is no atomic and no divergence on the bin loop.  Per work item the FP32
// register sums are folded into FP64 registers; at the end each CTA reduces its
// warps in shared memory and writes one FP64 partial row.  The FP64 finalize sums
// the partials, forms DD^a_l from adjacent edges, normalises and subtracts W~^a.
#include <cmath>
#include <cstdio>

#include "hip_internal.h"

static __constant__ HipCoeffs c_coeffs;

cudaError_t hip_upload_coeffs_power()
{
    return cudaMemcpyToSymbol(c_coeffs, &hip_host_coeffs(), sizeof(HipCoeffs));
}

// ------------------------------------------------------------- cell build ----
__device__ __forceinline__ double hip_wrap(double v, double L)
{
    v -= L * floor(v / L);
    if (v >= L) v -= L;
    if (v < 0.0) v = 0.0;
    return v;
}

__global__ void k_cell_count(const float *__restrict__ pos, const float *__restrict__ w, long long N, double L,
                             int n_c, double inv_cs, int *__restrict__ cid, int *__restrict__ count, double *S1,
                             int *err)
{
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
            double v = hip_wrap((double)pv[k], L);
            int ic = (int)(v * inv_cs);
            c3[k] = ic >= n_c ? n_c - 1 : ic;
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
__global__ void k_cell_scatter(const float *__restrict__ pos, const float *__restrict__ w, long long N, double L,
                               int n_c, double cs, double inv_cs, const int *__restrict__ cid,
                               const int *__restrict__ start, int *__restrict__ fill, T *__restrict__ x,
                               T *__restrict__ y, T *__restrict__ z, float *__restrict__ ws, int *__restrict__ idx)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        int id = cid[i];
        int slot = start[id] + atomicAdd(&fill[id], 1);
        float pv[3] = {pos[3 * i], pos[3 * i + 1], pos[3 * i + 2]};
        double loc[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            double v = hip_wrap((double)pv[k], L);
            int ic = (int)(v * inv_cs);
            ic = ic >= n_c ? n_c - 1 : ic;
            loc[k] = v - ic * cs;
        }
        x[slot] = (T)loc[0];
        y[slot] = (T)loc[1];
        z[slot] = (T)loc[2];
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
    k_cell_count<<<blocks, 256, 0, st>>>(pos, w, N, L, n_c, 1.0 / cs, cid, cell_fill, S1, err);
    k_cell_scan<<<1, 1024, 0, st>>>(cell_fill, n_cells, cell_start, cell_fill);
    k_cell_scatter<T><<<blocks, 256, 0, st>>>(pos, w, N, L, n_c, cs, 1.0 / cs, cid, cell_start, cell_fill, x, y, z,
                                              ws, idx);
    return cudaGetLastError();
}

template cudaError_t hip_build_cells<float>(const float *, const float *, int64_t, double, int, float *, float *,
                                            float *, float *, int *, int *, int *, int *, double *, int *,
                                            cudaStream_t);
template cudaError_t hip_build_cells<double>(const float *, const float *, int64_t, double, int, double *, double *,
                                             double *, float *, int *, int *, int *, int *, double *, int *,
                                             cudaStream_t);

// ------------------------------------------------------------- pair pass -----
// Bin edges as seen by the pair kernels.  For FP32 each edge is split into
// khi + klo (two floats) and u = r k is formed as fma(r, khi, r klo): rounding
// the edge itself to a float would shift every pair's argument the same way, a
// systematic error, while the rounding of u then varies from pair to pair.
template <typename T>
struct EdgeTable {
    T k[HIP_MAX_EDGES];
    T klo[HIP_MAX_EDGES];
};

template <typename T>
__device__ __forceinline__ T hip_sqrt(T v);
template <>
__device__ __forceinline__ float hip_sqrt<float>(float v) { return sqrtf(v); }
template <>
__device__ __forceinline__ double hip_sqrt<double>(double v) { return sqrt(v); }

#define HIP_WTILE 64
#define HIP_QCAP 64

// Shared memory of one warp: a tile of the home cell, a tile of the shifted
// neighbour cell, and the queue of accepted pairs awaiting the bin pass.
template <typename T>
struct WarpSmem {
    T hx[HIP_WTILE], hy[HIP_WTILE], hz[HIP_WTILE];
    float hw[HIP_WTILE];
    int hin[HIP_WTILE];
    T nx[HIP_WTILE], ny[HIP_WTILE], nz[HIP_WTILE];
    float nw[HIP_WTILE];
    int nin[HIP_WTILE];
    T qr[HIP_QCAP];                // separation r
    T qo[3][HIP_QCAP];             // omega L_l(mu), l = 0, 2, 4
    T qc[HIP_QCAP], qs[HIP_QCAP];  // cos, sin of 32 r dk: rotation between 32-edge chunks
};

__constant__ int c_shift[HIP_NSHIFT][3] = {{0, 0, 0},  {1, -1, -1}, {1, -1, 0}, {1, -1, 1}, {1, 0, -1},
                                           {1, 0, 0},  {1, 0, 1},   {1, 1, -1}, {1, 1, 0},  {1, 1, 1},
                                           {0, 1, -1}, {0, 1, 0},   {0, 1, 1},  {0, 0, 1}};

__device__ __forceinline__ void hip_sincos(float u, float *s, float *c) { sincosf(u, s, c); }
__device__ __forceinline__ void hip_sincos(double u, double *s, double *c) { sincos(u, s, c); }

// Bin pass over the n queued pairs of a warp: lanes over bin edges (edge
// lane + 32 t in chunk t), pairs broadcast.  sin/cos of u = r k_e come from one
// accurate sincos in chunk 0 and, for uniformly spaced edges, a rotation by the
// pair's 32 r dk for every later chunk.  When the last used chunk (index tl)
// holds tw <= 16 edges it is "packed": lane l handles edge 32 tl + l % tw of
// pair q0 + l / tw, so 32 / tw pairs share one pass instead of leaving most
// lanes idle.
__device__ __forceinline__ void hip_edge_acc(float u, float s, float c, bool need_sc, float o0, float o2, float o4,
                                             int mask, float &H0, float &H2, float &H4, float &C0, float &C2,
                                             float &C4)
{
    float Fm[5], Fc[5];
    if (u < HIP_F32_USMALL) {
        if (mask & 16)
            hip_F_f32_series<21>(u, c_coeffs, Fm, Fc);
        else if (mask & 4)
            hip_F_f32_series<5>(u, c_coeffs, Fm, Fc);
        else
            hip_F_f32_series<1>(u, c_coeffs, Fm, Fc);
        H0 = fmaf(o0, c_coeffs.ser32[0][0], H0);
        C0 = fmaf(o0, Fc[0], C0);
        if (mask & 4) C2 = fmaf(o2, Fc[2], C2);
        if (mask & 16) C4 = fmaf(o4, Fc[4], C4);
    } else {
        if (need_sc) sincosf(u, &s, &c);
        if (mask & 16)
            hip_F_f32_closed<21>(u, s, c, c_coeffs, Fm);
        else if (mask & 4)
            hip_F_f32_closed<5>(u, s, c, c_coeffs, Fm);
        else
            hip_F_f32_closed<1>(u, s, c, c_coeffs, Fm);
    }
    H0 = fmaf(o0, Fm[0], H0);
    if (mask & 4) H2 = fmaf(o2, Fm[2], H2);
    if (mask & 16) H4 = fmaf(o4, Fm[4], H4);
}

__device__ __forceinline__ void hip_edge_acc(double u, double s, double c, bool need_sc, double o0, double o2,
                                             double o4, int mask, double &H0, double &H2, double &H4, double &,
                                             double &, double &)
{
    double F[5];
    if (u < HIP_F64_USMALL) {
        if (mask & 16)
            hip_F_f64_series<21>(u, c_coeffs, F);
        else if (mask & 4)
            hip_F_f64_series<5>(u, c_coeffs, F);
        else
            hip_F_f64_series<1>(u, c_coeffs, F);
    } else {
        if (need_sc) sincos(u, &s, &c);
        if (mask & 16)
            hip_F_f64_closed<21>(u, s, c, c_coeffs, F);
        else if (mask & 4)
            hip_F_f64_closed<5>(u, s, c, c_coeffs, F);
        else
            hip_F_f64_closed<1>(u, s, c, c_coeffs, F);
    }
    H0 = fma(o0, F[0], H0);
    if (mask & 4) H2 = fma(o2, F[2], H2);
    if (mask & 16) H4 = fma(o4, F[4], H4);
}

__device__ __forceinline__ float hip_arg(float r, float khi, float klo) { return fmaf(r, khi, r * klo); }
__device__ __forceinline__ double hip_arg(double r, double khi, double) { return r * khi; }

// Edge handled by `lane` in chunk t (or -1), given the tail chunk tl and the
// packed tail width tw (0 when the tail is not packed).
__device__ __forceinline__ int hip_lane_edge(int lane, int t, int n_e, int tl, int tw)
{
    if (t == tl && tw > 0) return lane < (32 / tw) * tw ? 32 * tl + lane % tw : -1;
    const int e = lane + 32 * t;
    return (t <= tl && e < n_e) ? e : -1;
}

template <typename T, int NCH, int MASK>
__device__ __forceinline__ void hip_drain(const WarpSmem<T> &sm, int n, const T *kk, const T *kl, int lane, int n_e,
                                          bool LIN, int tl, int tw, T (&H)[3][NCH], T (&Hc)[3][NCH])
{
    for (int q = 0; q < n; ++q) {
        const T r = sm.qr[q];
        const T o0 = sm.qo[0][q], o2 = sm.qo[1][q], o4 = sm.qo[2][q];
        const T rc = sm.qc[q], rs = sm.qs[q];
        T s = T(0), c = T(1);
#pragma unroll
        for (int t = 0; t < NCH; ++t) {
            if (t < tl || (t == tl && tw == 0)) {
                const T u = hip_arg(r, kk[t], kl[t]);
                if (LIN) {
                    if (t == 0) {
                        hip_sincos(u, &s, &c);
                    } else {
                        const T s2 = fma(s, rc, c * rs);
                        c = fma(c, rc, -s * rs);
                        s = s2;
                    }
                }
                if (lane + 32 * t < n_e)
                    hip_edge_acc(u, s, c, !LIN, o0, o2, o4, MASK, H[0][t], H[1][t], H[2][t], Hc[0][t], Hc[1][t],
                                 Hc[2][t]);
            }
        }
    }
    if (tw > 0) {
        const int per = 32 / tw, sub = lane / tw;
#pragma unroll
        for (int t = 0; t < NCH; ++t) {
            if (t != tl) continue;
            for (int q0 = 0; q0 < n; q0 += per) {
                const int q = q0 + sub;
                if (sub < per && q < n) {
                    const T r = sm.qr[q];
                    hip_edge_acc(hip_arg(r, kk[t], kl[t]), T(0), T(1), true, sm.qo[0][q], sm.qo[1][q], sm.qo[2][q],
                                 MASK, H[0][t], H[1][t], H[2][t], Hc[0][t], Hc[1][t], Hc[2][t]);
                }
            }
        }
    }
}

__device__ __forceinline__ float hip_rot_angle(float r, float dhi, float dlo) { return fmaf(r, dhi, r * dlo); }

__device__ __forceinline__ double hip_rot_angle(double r, double dhi, double) { return r * dhi; }

// Drain a warp's queue and fold the FP32 register sums into the FP64 ones.
template <typename T, int NCH, int MASK>
__device__ __forceinline__ void hip_drain_fold(const WarpSmem<T> &sm, int &qn, const T *kk, const T *kl, int lane,
                                               int n_e, bool lin, int tl, int tw, T (&H)[3][NCH], T (&Hc)[3][NCH],
                                               double (&R)[3][NCH])
{
    __syncwarp();
    hip_drain<T, NCH, MASK>(sm, qn, kk, kl, lane, n_e, lin, tl, tw, H, Hc);
#pragma unroll
    for (int l = 0; l < 3; ++l)
#pragma unroll
        for (int t = 0; t < NCH; ++t) {
            R[l][t] += (double)H[l][t] + (double)Hc[l][t];
            H[l][t] = T(0);
            Hc[l][t] = T(0);
        }
    qn = 0;
    __syncwarp();
}

// One work item (home cell, half-shell shift) of one catalog, processed by one
// warp: stage 64-particle tiles of both cells in the warp's shared memory, test
// candidates one per lane, queue accepted pairs, drain the queue at 32 pairs.
template <typename T, int NCH, int MASK>
__device__ __forceinline__ void hip_pair_item(const CellList<T> &cl, int item, long long p0, long long p1, int los,
                                              T R0sq, T invR0, bool lin, T dk32hi, T dk32lo, WarpSmem<T> &sm,
                                              int lane, const T *kk, const T *kl, int n_e, int tl, int tw,
                                              T (&H)[3][NCH],
                                              T (&Hc)[3][NCH], double (&R)[3][NCH], int &qn,
                                              unsigned long long &cnt)
{
    const unsigned lt_mask = (1u << lane) - 1u;
    const int n_c = cl.n_c;
    const int c = item / HIP_NSHIFT, q = item - c * HIP_NSHIFT;
    const int cx = c / (n_c * n_c), cy = (c / n_c) % n_c, cz = c % n_c;
    const int dx = c_shift[q][0], dy = c_shift[q][1], dz = c_shift[q][2];
    const int nb = (((cx + dx + n_c) % n_c) * n_c + (cy + dy + n_c) % n_c) * n_c + (cz + dz + n_c) % n_c;
    const T sx = T(dx) * cl.cs, sy = T(dy) * cl.cs, sz = T(dz) * cl.cs;
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
            sm.hin[i] = (oi >= p0 && oi < p1) ? 1 : 0;
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
                sm.nin[i] = (oi >= p0 && oi < p1) ? 1 : 0;
            }
            __syncwarp();
            const bool same = self && (nbs == hb);
            for (int il = 0; il < hn; ++il) {
                const T xi = sm.hx[il] - sx, yi = sm.hy[il] - sy, zi = sm.hz[il] - sz;
                const float wi = sm.hw[il];
                const int ini = sm.hin[il];
                for (int jb = same ? il + 1 : 0; jb < nn; jb += 32) {
                    const int jl = jb + lane;
                    bool ok = false;
                    T ddx = T(0), ddy = T(0), ddz = T(0), r2 = T(0);
                    int mult = 0;
                    if (jl < nn) {
                        ddx = xi - sm.nx[jl];
                        ddy = yi - sm.ny[jl];
                        ddz = zi - sm.nz[jl];
                        r2 = ddx * ddx + ddy * ddy + ddz * ddz;
                        mult = ini + sm.nin[jl];
                        ok = (r2 < R0sq) && (r2 > T(0)) && (mult > 0);
                    }
                    const unsigned m = __ballot_sync(0xffffffffu, ok);
                    if (ok) {
                        const T r = hip_sqrt<T>(r2);
                        const T dl = los == 0 ? ddx : (los == 1 ? ddy : ddz);
                        const T mu = dl / r;
                        T l2, l4;
                        hip_legendre24<T>(mu, l2, l4);
                        const T om = T(wi) * T(sm.nw[jl]) * hip_W<T>(r * invR0) * T(mult);
                        const int slot = qn + __popc(m & lt_mask);
                        sm.qr[slot] = r;
                        sm.qo[0][slot] = om;
                        sm.qo[1][slot] = om * l2;
                        sm.qo[2][slot] = om * l4;
                        if (lin) {
                            T rs, rc;
                            hip_sincos(hip_rot_angle(r, dk32hi, dk32lo), &rs, &rc);
                            sm.qc[slot] = rc;
                            sm.qs[slot] = rs;
                        }
                        cnt += (unsigned long long)mult;
                    }
                    qn += __popc(m);
                    if (qn >= 32) hip_drain_fold<T, NCH, MASK>(sm, qn, kk, kl, lane, n_e, lin, tl, tw, H, Hc, R);
                }
            }
        }
    }
}

// Pair pass of one catalog.  Each warp works on its own: it takes work items
// from the global counter and processes them with hip_pair_item; the queue
// persists across items.  After each drain the FP32 register sums are folded
// into FP64 registers, so an FP32 sum never spans more than 64 pairs.  At the
// end each CTA reduces its warps in shared memory into one FP64 partial row.
template <typename T, int NCH, int MASK, bool LIN>
__global__ void __launch_bounds__(HIP_PAIR_THREADS, 6)
    k_power_pairs(CellList<T> cl, PowerKernelArgs a, EdgeTable<T> ed, T R0, T dk32hi, T dk32lo)
{
    __shared__ WarpSmem<T> smem[HIP_PAIR_WARPS];
    __shared__ double red[3][HIP_MAX_EDGES];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    WarpSmem<T> &sm = smem[warp];
    const T R0sq = R0 * R0, invR0 = T(1) / R0;
    const int n_e = a.n_e;
    const int n_ell = (MASK & 16) ? 3 : ((MASK & 4) ? 2 : 1);
    const int tl = (n_e - 1) / 32, tw = (n_e - 32 * tl <= 16) ? n_e - 32 * tl : 0;

    T kk[NCH], kl[NCH];
#pragma unroll
    for (int t = 0; t < NCH; ++t) {
        const int e = hip_lane_edge(lane, t, n_e, tl, tw);
        kk[t] = e >= 0 ? ed.k[e] : T(0);
        kl[t] = e >= 0 ? ed.klo[e] : T(0);
    }
    T H[3][NCH], Hc[3][NCH];
    double R[3][NCH];
#pragma unroll
    for (int l = 0; l < 3; ++l)
#pragma unroll
        for (int t = 0; t < NCH; ++t) {
            H[l][t] = T(0);
            Hc[l][t] = T(0);
            R[l][t] = 0.0;
        }
    unsigned long long cnt = 0;
    int qn = 0;
    for (;;) {
        int item = 0;
        if (lane == 0) item = atomicAdd(a.work_counter, 1);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= a.n_items) break;
        hip_pair_item<T, NCH, MASK>(cl, item, a.p0, a.p1, a.los, R0sq, invR0, LIN, dk32hi, dk32lo, sm, lane, kk, kl,
                                    n_e, tl, tw, H, Hc, R, qn, cnt);
    }
    if (qn > 0) hip_drain_fold<T, NCH, MASK>(sm, qn, kk, kl, lane, n_e, LIN, tl, tw, H, Hc, R);
    // CTA reduction of the per-lane FP64 sums into one partial row.
    for (int i = threadIdx.x; i < 3 * HIP_MAX_EDGES; i += HIP_PAIR_THREADS) (&red[0][0])[i] = 0.0;
    __syncthreads();
    for (int wv = 0; wv < HIP_PAIR_WARPS; ++wv) {
        if (warp == wv) {
#pragma unroll
            for (int l = 0; l < 3; ++l)
#pragma unroll
                for (int t = 0; t < NCH; ++t) {
                    const int e = hip_lane_edge(lane, t, n_e, tl, tw);
                    if (e >= 0) atomicAdd(&red[l][e], R[l][t]);  // packed-tail lanes share edges
                }
        }
        __syncthreads();
    }
    double *out = a.partials + (size_t)blockIdx.x * 3 * n_e;
    for (int i = threadIdx.x; i < n_ell * n_e; i += HIP_PAIR_THREADS) {
        const int l = i / n_e, e = i - l * n_e;
        out[l * n_e + e] = red[l][e];
    }
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    if (lane == 0 && cnt) atomicAdd(a.npairs, cnt);
}

// Pair pass over many catalogs in one launch.  Global work items are the
// catalogs' items laid end to end (catalog c owns [item_begin, item_end));
// a warp that moves to another catalog first drains its queue and adds its FP64
// sums to the previous catalog's accumulator (FP64 atomics), then loads the new
// catalog's edges.  All catalogs share the kernel's NCH (the largest needed).
template <typename T, int NCH>
__global__ void __launch_bounds__(HIP_PAIR_THREADS)
    k_power_pairs_batched(const BatchCat<T> *__restrict__ cats, int n_cats, int n_items, int *work_counter)
{
    __shared__ WarpSmem<T> smem[HIP_PAIR_WARPS];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    WarpSmem<T> &sm = smem[warp];
    T kk[NCH], kl[NCH];
    T H[3][NCH], Hc[3][NCH];
    double R[3][NCH];
#pragma unroll
    for (int l = 0; l < 3; ++l)
#pragma unroll
        for (int t = 0; t < NCH; ++t) {
            H[l][t] = T(0);
            Hc[l][t] = T(0);
            R[l][t] = 0.0;
        }
    unsigned long long cnt = 0;
    int qn = 0, cur = -1, tl = 0, tw = 0;
    auto leave = [&](int c) {
        if (qn > 0)
            hip_drain_fold<T, NCH, 21>(sm, qn, kk, kl, lane, cats[c].n_e, cats[c].lin != 0, tl, tw, H, Hc, R);
        const int ne = cats[c].n_e;
#pragma unroll
        for (int l = 0; l < 3; ++l)
#pragma unroll
            for (int t = 0; t < NCH; ++t) {
                const int e = hip_lane_edge(lane, t, ne, tl, tw);
                if (e >= 0 && R[l][t] != 0.0) atomicAdd(&cats[c].acc[l * ne + e], R[l][t]);
                R[l][t] = 0.0;
            }
        for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
        if (lane == 0 && cnt) atomicAdd(cats[c].npairs, cnt);
        cnt = 0;
    };
    for (;;) {
        int item = 0;
        if (lane == 0) item = atomicAdd(work_counter, 1);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= n_items) break;
        int c = cur < 0 ? 0 : cur;
        while (item >= cats[c].item_end) ++c;
        while (item < cats[c].item_begin) --c;
        if (c != cur) {
            if (cur >= 0) leave(cur);
            cur = c;
            const int ne = cats[c].n_e;
            tl = (ne - 1) / 32;
            tw = (ne - 32 * tl <= 16) ? ne - 32 * tl : 0;
#pragma unroll
            for (int t = 0; t < NCH; ++t) {
                const int e = hip_lane_edge(lane, t, ne, tl, tw);
                kk[t] = e >= 0 ? cats[c].k[e] : T(0);
                kl[t] = e >= 0 ? cats[c].klo[e] : T(0);
            }
        }
        const BatchCat<T> &bc = cats[c];
        hip_pair_item<T, NCH, 21>(bc.cl, item - bc.item_begin, bc.p0, bc.p1, bc.los, bc.R0 * bc.R0, T(1) / bc.R0,
                                  bc.lin != 0, bc.dk32hi, bc.dk32lo, sm, lane, kk, kl, bc.n_e, tl, tw, H, Hc, R, qn,
                                  cnt);
    }
    if (cur >= 0) leave(cur);
}

template <typename T>
int hip_power_grid()
{
    int dev = 0, sms = 0, nb = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_power_pairs<T, 4, 21, true>, HIP_PAIR_THREADS, 0);
    return sms * (nb < 1 ? 1 : nb);
}
template int hip_power_grid<float>();
template int hip_power_grid<double>();

template <typename T, int NCH, bool LIN>
static void launch_mask(const CellList<T> &cl, const PowerKernelArgs &a, const EdgeTable<T> &ed, int n_ell, T R0,
                        T dhi, T dlo, int grid, cudaStream_t st)
{
    if (n_ell == 3)
        k_power_pairs<T, NCH, 21, LIN><<<grid, HIP_PAIR_THREADS, 0, st>>>(cl, a, ed, R0, dhi, dlo);
    else if (n_ell == 2)
        k_power_pairs<T, NCH, 5, LIN><<<grid, HIP_PAIR_THREADS, 0, st>>>(cl, a, ed, R0, dhi, dlo);
    else
        k_power_pairs<T, NCH, 1, LIN><<<grid, HIP_PAIR_THREADS, 0, st>>>(cl, a, ed, R0, dhi, dlo);
}

template <typename T, bool LIN>
static void launch_nch(const CellList<T> &cl, const PowerKernelArgs &a, const EdgeTable<T> &ed, int n_ell, T R0,
                       T dhi, T dlo, int grid, cudaStream_t st)
{
    const int nch = (a.n_e + 31) / 32;
    if (nch <= 1)
        launch_mask<T, 1, LIN>(cl, a, ed, n_ell, R0, dhi, dlo, grid, st);
    else if (nch <= 2)
        launch_mask<T, 2, LIN>(cl, a, ed, n_ell, R0, dhi, dlo, grid, st);
    else if (nch <= 4)
        launch_mask<T, 4, LIN>(cl, a, ed, n_ell, R0, dhi, dlo, grid, st);
    else
        launch_mask<T, 8, LIN>(cl, a, ed, n_ell, R0, dhi, dlo, grid, st);
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
    if (lin)
        launch_nch<T, true>(cl, a, ed, n_ell, (T)R0, dhi, dlo, grid, st);
    else
        launch_nch<T, false>(cl, a, ed, n_ell, (T)R0, dhi, dlo, grid, st);
    return cudaGetLastError();
}
template cudaError_t hip_power_pairs<float>(const CellList<float> &, const PowerKernelArgs &, const double *, int,
                                            double, int, cudaStream_t);
template cudaError_t hip_power_pairs<double>(const CellList<double> &, const PowerKernelArgs &, const double *, int,
                                             double, int, cudaStream_t);

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
        const double dd = 3.0 * (k3hi * H[il][a + 1] - k3lo * H[il][a]) / (k3hi - k3lo);
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
        const double dd = 3.0 * (k3hi * f.acc[il * n_e + a + 1] - k3lo * f.acc[il * n_e + a]) / (k3hi - k3lo);
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

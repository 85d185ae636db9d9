// Pair-pass kernels of the power spectrum (Sec. 3 of arXiv:2005.01739), included
// by the translation units that instantiate them (one per precision / edge
// layout, so that the library builds in parallel).  Each including unit gets
// its own copy of the constant-memory tables and defines HIP_PAIR_UPLOAD, the
// function that fills its copy of the series and fit coefficients.
//
// Pair pass: persistent CTAs pull work items (home cell, one of 14 half-shell
// shifts) from an atomic counter.  A warp stages a tile of the home cell and a
// tile of the shifted neighbour cell in shared memory (positions as cell-local
// offsets, so separations keep full precision whatever the box size), tests
// candidate pairs with one lane per candidate and appends accepted pairs to its
// queue.  The queue is drained with one lane per bin EDGE: for every queued pair
// each lane evaluates F_l(r k_e) at its own edges and accumulates omega_l F_l
// into registers.  No lane ever writes another lane's edge, so there is no
// atomic and no divergence on the bin loop.  After each drain the FP32 register
// sums are folded into FP64 registers; at the end each CTA reduces its warps in
// shared memory and writes one FP64 partial row.
#pragma once
#include <cmath>

#include "hip_internal.h"

#ifndef HIP_PAIR_UPLOAD
#error "define HIP_PAIR_UPLOAD before including hip_pair_kernel.cuh"
#endif

static __constant__ HipCoeffs c_coeffs;

cudaError_t HIP_PAIR_UPLOAD()
{
    return cudaMemcpyToSymbol(c_coeffs, &hip_host_coeffs(), sizeof(HipCoeffs));
}

// ------------------------------------------------------------- pair pass -----
#define HIP_WTILE 64
#define HIP_QCAP 64
#define HIP_SQCAP 64

// Series queue of the FP32 pass (empty for FP64): (u, pair slot, edge) of the
// lanes whose argument is below HIP_F32_USMALL, evaluated 32 at a time one per
// lane, and the per-edge FP32 sums they feed (folded to FP64 with each drain).
template <typename T, int NCH>
struct SeriesQueue {
};
template <int NCH>
struct SeriesQueue<float, NCH> {
    float u[HIP_SQCAP];
    unsigned char q[HIP_SQCAP], e[HIP_SQCAP];
    float acc[3][HIP_MAX_EDGES];
};

// Shared memory of one warp: a tile of the home cell, a tile of the shifted
// neighbour cell, and the queue of accepted pairs awaiting the bin pass.
template <typename T, int NCH>
struct WarpSmem {
    T hx[HIP_WTILE], hy[HIP_WTILE], hz[HIP_WTILE];
    float hw[HIP_WTILE];
    int hin[HIP_WTILE];
    T nx[HIP_WTILE], ny[HIP_WTILE], nz[HIP_WTILE];
    float nw[HIP_WTILE];
    int nin[HIP_WTILE];
    T qr[HIP_QCAP], qrl[HIP_QCAP];  // separation r = qr + qrl (qrl: FP32 low part, 0 for FP64)
    T qo[3][HIP_QCAP];             // omega L_l(mu), l = 0, 2, 4 (FP32: divided by r^3)
    T qc[HIP_QCAP], qs[HIP_QCAP];  // cos, sin of 32 r dk: rotation between 32-edge chunks
    SeriesQueue<T, NCH> sq;
};

static __constant__ int c_shift[HIP_NSHIFT][3] = {{0, 0, 0},  {1, -1, -1}, {1, -1, 0}, {1, -1, 1}, {1, 0, -1},
                                           {1, 0, 0},  {1, 0, 1},   {1, 1, -1}, {1, 1, 0},  {1, 1, 1},
                                           {0, 1, -1}, {0, 1, 0},   {0, 1, 1},  {0, 0, 1}};


__device__ __forceinline__ float hip_arg(float r, float khi, float klo) { return fmaf(r, khi, r * klo); }
__device__ __forceinline__ double hip_arg(double r, double khi, double) { return r * khi; }

// u = (rh + rl)(khi + klo) as uh + ul, for the arguments whose sin and cos are
// evaluated directly (the phase of every later chunk is derived from them).
// ul holds the rounding of uh and the low-order products; products of two low
// parts are dropped.
__device__ __forceinline__ void hip_arg2(float rh, float rl, float khi, float klo, float &uh, float &ul)
{
    const float m = fmaf(rl, khi, rh * klo);
    uh = fmaf(rh, khi, m);
    ul = fmaf(rh, khi, -uh) + m;
}
__device__ __forceinline__ void hip_arg2(double rh, double, double khi, double, double &uh, double &ul)
{
    uh = rh * khi;
    ul = 0.0;
}

__device__ __forceinline__ void hip_sincos2(float u, float ul, float *s, float *c)
{
    float s0, c0;
    sincosf(u, &s0, &c0);
    *s = fmaf(c0, ul, s0);
    *c = fmaf(-s0, ul, c0);
}
__device__ __forceinline__ void hip_sincos2(double u, double, double *s, double *c) { sincos(u, s, c); }

// Edge handled by `lane` in chunk t (or -1), given the tail chunk tl and the
// packed tail width tw (0 when the tail is not packed).
__device__ __forceinline__ int hip_lane_edge(int lane, int t, int n_e, int tl, int tw)
{
    if (t == tl && tw > 0) return lane < (32 / tw) * tw ? 32 * tl + lane % tw : -1;
    const int e = lane + 32 * t;
    return (t <= tl && e < n_e) ? e : -1;
}

// Bin pass over the n queued pairs of a warp: lanes over bin edges (edge
// lane + 32 t in chunk t), pairs broadcast.  sin/cos of u = r k_e come from one
// accurate sincos in chunk 0 and, for uniformly spaced edges, a rotation by the
// pair's 32 r dk for every later chunk.  When the last used chunk (index tl)
// holds tw <= 16 edges it is "packed": lane l handles edge 32 tl + l % tw of
// pair q0 + l / tw, so 32 / tw pairs share one pass instead of leaving most
// lanes idle.
//
// FP32: every lane accumulates omega_l D_l(u) / r^3 (the weights in the queue
// are already divided by r^3).  Lanes whose u is below HIP_F32_USMALL do not
// branch into the series: they append (u, pair, edge) to the series queue, which
// is evaluated 32 entries at a time, one entry per lane.  The closed forms take
// the asymptotic Si auxiliaries when every closed-form lane of the warp has
// u >= HIP_F32_UASYM (a warp-uniform choice) and the fitted ones otherwise.
template <int NCH, int MASK>
__device__ __forceinline__ void hip_series_eval(WarpSmem<float, NCH> &sm, int n, int lane)
{
    if (lane < n) {
        const float u = sm.sq.u[lane];
        const int q = sm.sq.q[lane], e = sm.sq.e[lane];
        float D[5];
        hip_D_f32_series<MASK>(u, c_coeffs, D);
        atomicAdd(&sm.sq.acc[0][e], sm.qo[0][q] * D[0]);
        if (MASK & 4) atomicAdd(&sm.sq.acc[1][e], sm.qo[1][q] * D[2]);
        if (MASK & 16) atomicAdd(&sm.sq.acc[2][e], sm.qo[2][q] * D[4]);
    }
}

template <int NCH, int MASK>
__device__ __forceinline__ void hip_series_push(WarpSmem<float, NCH> &sm, int &sn, bool need, float u, int q, int e,
                                                int lane)
{
    const unsigned m = __ballot_sync(0xffffffffu, need);
    if (m == 0u) return;
    if (need) {
        const int slot = sn + __popc(m & ((1u << lane) - 1u));
        sm.sq.u[slot] = u;
        sm.sq.q[slot] = (unsigned char)q;
        sm.sq.e[slot] = (unsigned char)e;
    }
    sn += __popc(m);  // < HIP_SQCAP: sn was < 32 before this push
    if (sn >= 32) {
        __syncwarp();
        hip_series_eval<NCH, MASK>(sm, 32, lane);
        const int rest = sn - 32;
        float mu = 0.0f;
        int mq = 0, me = 0;
        if (lane < rest) {
            mu = sm.sq.u[32 + lane];
            mq = sm.sq.q[32 + lane];
            me = sm.sq.e[32 + lane];
        }
        __syncwarp();
        if (lane < rest) {
            sm.sq.u[lane] = mu;
            sm.sq.q[lane] = (unsigned char)mq;
            sm.sq.e[lane] = (unsigned char)me;
        }
        sn = rest;
        __syncwarp();
    }
}

template <int MASK>
__device__ __forceinline__ void hip_closed_acc(float u, float w, float s, float c, bool asym, float o0, float o2,
                                               float o4, float &H0, float &H2, float &H4)
{
    float D[5];
    if (asym)
        hip_D_f32_closed<MASK, true>(u, w, s, c, c_coeffs, D);
    else
        hip_D_f32_closed<MASK, false>(u, w, s, c, c_coeffs, D);
    H0 = fmaf(o0, D[0], H0);
    if (MASK & 4) H2 = fmaf(o2, D[2], H2);
    if (MASK & 16) H4 = fmaf(o4, D[4], H4);
}

template <int NCH, int MASK>
__device__ __forceinline__ void hip_drain(WarpSmem<float, NCH> &sm, int n, const float *kk, const float *kl,
                                          const float *, int lane, int n_e, bool LIN, int tl, int tw,
                                          float (&H)[3][NCH])
{
    int sn = 0;
    for (int q = 0; q < n; ++q) {
        const float r = sm.qr[q], rl = sm.qrl[q];
        const float o0 = sm.qo[0][q], o2 = sm.qo[1][q], o4 = sm.qo[2][q];
        const float rc = sm.qc[q], rs = sm.qs[q];
        float s = 0.0f, c = 1.0f;
#pragma unroll
        for (int t = 0; t < NCH; ++t) {
            if (t < tl || (t == tl && tw == 0)) {
                const int e = lane + 32 * t;
                const bool act = e < n_e;
                float u, ul = 0.0f;
                if (t == 0 || !LIN) {
                    hip_arg2(r, rl, kk[t], kl[t], u, ul);
                } else {
                    u = hip_arg(r, kk[t], kl[t]);  // sin, cos come from the rotation
                }
                if (LIN) {
                    if (t == 0) {
                        hip_sincos2(u, ul, &s, &c);
                    } else {
                        const float s2 = fmaf(s, rc, c * rs);
                        c = fmaf(c, rc, -s * rs);
                        s = s2;
                    }
                }
                const bool ser = act && u < HIP_F32_USMALL;
                hip_series_push<NCH, MASK>(sm, sn, ser, u, q, e, lane);
                const bool clo = act && !ser;
                const bool asym = __all_sync(0xffffffffu, !clo || u >= HIP_F32_UASYM);
                if (clo) {
                    if (!LIN) hip_sincos2(u, ul, &s, &c);
                    hip_closed_acc<MASK>(u, __fdividef(1.0f, u), s, c, asym, o0, o2, o4, H[0][t], H[1][t], H[2][t]);
                }
            }
        }
    }
    if (tw > 0) {
        const int per = 32 / tw, sub = lane / tw;
#pragma unroll
        for (int t = 0; t < NCH; ++t) {
            if (t != tl) continue;
            const int e = 32 * tl + lane % tw;
            for (int q0 = 0; q0 < n; q0 += per) {
                const int q = q0 + sub;
                const bool act = sub < per && q < n;
                float u = 0.0f, ul = 0.0f;
                if (act) hip_arg2(sm.qr[q], sm.qrl[q], kk[t], kl[t], u, ul);
                const bool ser = act && u < HIP_F32_USMALL;
                hip_series_push<NCH, MASK>(sm, sn, ser, u, q, e, lane);
                const bool clo = act && !ser;
                const bool asym = __all_sync(0xffffffffu, !clo || u >= HIP_F32_UASYM);
                if (clo) {
                    float s, c;
                    hip_sincos2(u, ul, &s, &c);
                    hip_closed_acc<MASK>(u, __fdividef(1.0f, u), s, c, asym, sm.qo[0][q], sm.qo[1][q], sm.qo[2][q],
                                         H[0][t], H[1][t], H[2][t]);
                }
            }
        }
    }
    if (sn > 0) {
        __syncwarp();
        hip_series_eval<NCH, MASK>(sm, sn, lane);
    }
}

// FP64: the series / closed-form branch is taken per lane; every lane
// accumulates omega_l k_e^3 F_l(u).
__device__ __forceinline__ void hip_edge_acc64(double u, double k3, double s, double c, bool need_sc, double o0,
                                               double o2, double o4, int mask, double &H0, double &H2, double &H4)
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
    H0 = fma(o0 * k3, F[0], H0);
    if (mask & 4) H2 = fma(o2 * k3, F[2], H2);
    if (mask & 16) H4 = fma(o4 * k3, F[4], H4);
}

template <int NCH, int MASK>
__device__ __forceinline__ void hip_drain(WarpSmem<double, NCH> &sm, int n, const double *kk, const double *,
                                          const double *k3, int lane, int n_e, bool LIN, int tl, int tw,
                                          double (&H)[3][NCH])
{
    for (int q = 0; q < n; ++q) {
        const double r = sm.qr[q];
        const double o0 = sm.qo[0][q], o2 = sm.qo[1][q], o4 = sm.qo[2][q];
        const double rc = sm.qc[q], rs = sm.qs[q];
        double s = 0.0, c = 1.0;
#pragma unroll
        for (int t = 0; t < NCH; ++t) {
            if (t < tl || (t == tl && tw == 0)) {
                const double u = r * kk[t];
                if (LIN) {
                    if (t == 0) {
                        sincos(u, &s, &c);
                    } else {
                        const double s2 = fma(s, rc, c * rs);
                        c = fma(c, rc, -s * rs);
                        s = s2;
                    }
                }
                if (lane + 32 * t < n_e)
                    hip_edge_acc64(u, k3[t], s, c, !LIN, o0, o2, o4, MASK, H[0][t], H[1][t], H[2][t]);
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
                if (sub < per && q < n)
                    hip_edge_acc64(sm.qr[q] * kk[t], k3[t], 0.0, 1.0, true, sm.qo[0][q], sm.qo[1][q], sm.qo[2][q],
                                   MASK, H[0][t], H[1][t], H[2][t]);
            }
        }
    }
}

// sin and cos of the rotation angle 32 (rh + rl) dk between 32-edge chunks.
__device__ __forceinline__ void hip_rotation(float rh, float rl, float dhi, float dlo, float *rs, float *rc)
{
    float th, tl;
    hip_arg2(rh, rl, dhi, dlo, th, tl);
    hip_sincos2(th, tl, rs, rc);
}
__device__ __forceinline__ void hip_rotation(double rh, double, double dhi, double, double *rs, double *rc)
{
    sincos(rh * dhi, rs, rc);
}

// Separation of an accepted pair as rh + rl.  The caller's rounded components
// d = xi - xj (xi = home offset minus shift, rounded, with low part xil) are
// made exact by the TwoSum error of xi - xj; r^2 is summed with exact products
// (FMA residuals) and TwoSums; r = sqrt(r^2) takes one Newton correction from
// the FMA residual of the rounded root.  With FP32 positions this keeps the
// argument r k of the oscillating kernels at ~1e-7 absolute even at r k ~ 1e3,
// where the plain FP32 separation is off by up to a few 1e-6 of r.
__device__ __forceinline__ float hip_two_sum_err(float a, float b, float s)
{
    const float bb = s - a;
    return (a - (s - bb)) + (b - bb);
}

__device__ __forceinline__ void hip_pair_sep(float xi, float xil, float yi, float yil, float zi, float zil, float xj,
                                             float yj, float zj, float dx, float dy, float dz, int los, float *rh,
                                             float *rl, float *dlo)
{
    const float lx = hip_two_sum_err(xi, -xj, dx) + xil;
    const float ly = hip_two_sum_err(yi, -yj, dy) + yil;
    const float lz = hip_two_sum_err(zi, -zj, dz) + zil;
    // __fmul_rn / __fadd_rn: the products must stay rounded (no FMA contraction)
    // for the TwoSum errors below to be exact
    const float px = __fmul_rn(dx, dx), py = __fmul_rn(dy, dy), pz = __fmul_rn(dz, dz);
    const float ex = fmaf(dx, dx, -px), ey = fmaf(dy, dy, -py), ez = fmaf(dz, dz, -pz);
    const float s1 = __fadd_rn(px, py), e1 = hip_two_sum_err(px, py, s1);
    const float s2 = __fadd_rn(s1, pz), e2 = hip_two_sum_err(s1, pz, s2);
    const float cross = 2.0f * fmaf(dx, lx, fmaf(dy, ly, dz * lz));
    const float low = ((e1 + e2) + (ex + ey + ez)) + cross;
    const float r = sqrtf(s2);
    *rh = r;
    *rl = (fmaf(-r, r, s2) + low) * (0.5f / r);
    *dlo = los == 0 ? lx : (los == 1 ? ly : lz);  // low part of the line-of-sight component
}
__device__ __forceinline__ float hip_low(float a, float b, float s) { return hip_two_sum_err(a, b, s); }
__device__ __forceinline__ double hip_low(double, double, double) { return 0.0; }

__device__ __forceinline__ void hip_pair_sep(double, double, double, double, double, double, double, double, double,
                                             double dx, double dy, double dz, int, double *rh, double *rl,
                                             double *dlo)
{
    *rh = sqrt(dx * dx + dy * dy + dz * dz);
    *rl = 0.0;
    *dlo = 0.0;
}

// Drain a warp's queue and fold the register sums (and, for FP32, the series
// sums in shared memory) into the FP64 registers.
template <int NCH>
__device__ __forceinline__ void hip_fold_series(WarpSmem<float, NCH> &sm, int lane, int n_e, int tl, double (&R)[3][NCH])
{
#pragma unroll
    for (int t = 0; t < NCH; ++t) {
        const int e = lane + 32 * t;
        if (t <= tl && e < n_e) {
#pragma unroll
            for (int l = 0; l < 3; ++l) {
                R[l][t] += (double)sm.sq.acc[l][e];
                sm.sq.acc[l][e] = 0.0f;
            }
        }
    }
}
template <int NCH>
__device__ __forceinline__ void hip_fold_series(WarpSmem<double, NCH> &, int, int, int, double (&)[3][NCH])
{
}

// kx: per-lane k_e^3 (FP64 path; unused by the FP32 path).
template <typename T, int NCH, int MASK>
__device__ __forceinline__ void hip_drain_fold(WarpSmem<T, NCH> &sm, int &qn, const T *kk, const T *kl, const T *kx,
                                               int lane, int n_e, bool lin, int tl, int tw, T (&H)[3][NCH],
                                               double (&R)[3][NCH])
{
    __syncwarp();
    hip_drain<NCH, MASK>(sm, qn, kk, kl, kx, lane, n_e, lin, tl, tw, H);
    __syncwarp();
#pragma unroll
    for (int l = 0; l < 3; ++l)
#pragma unroll
        for (int t = 0; t < NCH; ++t) {
            R[l][t] += (double)H[l][t];
            H[l][t] = T(0);
        }
    hip_fold_series<NCH>(sm, lane, n_e, tl, R);
    qn = 0;
    __syncwarp();
}

// Per-lane edge constants: the edge as khi + klo and kx = k_e^3 (FP64 path).
__device__ __forceinline__ float hip_kx(float, float) { return 0.0f; }
__device__ __forceinline__ double hip_kx(double k, double) { return k * k * k; }

template <typename T, int NCH>
__device__ __forceinline__ void hip_lane_edges(const T *k, const T *klo, int lane, int n_e, int tl, int tw, T (&kk)[NCH],
                                               T (&kl)[NCH], T (&kx)[NCH])
{
#pragma unroll
    for (int t = 0; t < NCH; ++t) {
        const int e = hip_lane_edge(lane, t, n_e, tl, tw);
        kk[t] = e >= 0 ? k[e] : T(0);
        kl[t] = e >= 0 ? klo[e] : T(0);
        kx[t] = hip_kx(kk[t], kl[t]);
    }
}

// Zero the series sums of a warp (FP32) before its first item.
template <int NCH>
__device__ __forceinline__ void hip_series_clear(WarpSmem<float, NCH> &sm, int lane)
{
    for (int i = lane; i < 3 * HIP_MAX_EDGES; i += 32) (&sm.sq.acc[0][0])[i] = 0.0f;
    __syncwarp();
}
template <int NCH>
__device__ __forceinline__ void hip_series_clear(WarpSmem<double, NCH> &, int)
{
}

// Weight of a queued pair: omega L_l(mu), divided by r^3 on the FP32 path
// (which accumulates D_l(r k) / r^3 = k^3 F_l(r k)).
__device__ __forceinline__ float hip_qscale(float r)
{
    const float ir = 1.0f / r;
    return ir * ir * ir;
}
__device__ __forceinline__ double hip_qscale(double) { return 1.0; }

// One work item (home cell, half-shell shift) of one catalog, processed by one
// warp: stage 64-particle tiles of both cells in the warp's shared memory, test
// candidates one per lane, queue accepted pairs, drain the queue at 32 pairs.
template <typename T, int NCH, int MASK>
__device__ __forceinline__ void hip_pair_item(const CellList<T> &cl, int item, long long p0, long long p1, int los,
                                              T R0sq, T invR0, T invR0lo, bool lin, T dk32hi, T dk32lo, WarpSmem<T, NCH> &sm,
                                              int lane, const T *kk, const T *kl, const T *kx, int n_e, int tl,
                                              int tw, T (&H)[3][NCH], double (&R)[3][NCH], int &qn,
                                              unsigned long long &cnt)
{
    const unsigned lt_mask = (1u << lane) - 1u;
    const int n_c = cl.n_c;
    const int c = item / HIP_NSHIFT, q = item - c * HIP_NSHIFT;
    const int cx = c / (n_c * n_c), cy = (c / n_c) % n_c, cz = c % n_c;
    const int dx = c_shift[q][0], dy = c_shift[q][1], dz = c_shift[q][2];
    const int nb = (((cx + dx + n_c) % n_c) * n_c + (cy + dy + n_c) % n_c) * n_c + (cz + dz + n_c) % n_c;
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
                const T hx = sm.hx[il], hy = sm.hy[il], hz = sm.hz[il];
                const T xi = hx - sx, yi = hy - sy, zi = hz - sz;
                // low parts of xi, yi, zi: rounding of the subtraction and the shift's low part
                const T xil = hip_low(hx, -sx, xi) - sxl, yil = hip_low(hy, -sy, yi) - syl,
                        zil = hip_low(hz, -sz, zi) - szl;
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
                        T r, rl, dlo;
                        hip_pair_sep(xi, xil, yi, yil, zi, zil, sm.nx[jl], sm.ny[jl], sm.nz[jl], ddx, ddy, ddz, los,
                                     &r, &rl, &dlo);
                        // mu and W from the full separation (hi + lo): the low parts carry the
                        // cell shift's rounding, common to all pairs across a periodic face
                        const T rr = r + rl;
                        const T mu = ((los == 0 ? ddx : (los == 1 ? ddy : ddz)) + dlo) / rr;
                        T l2, l4;
                        hip_legendre24<T>(mu, l2, l4);
                        const T om = T(wi) * T(sm.nw[jl]) * hip_W<T>(fma(rr, invR0lo, rr * invR0)) * T(mult) * hip_qscale(rr);
                        const int slot = qn + __popc(m & lt_mask);
                        sm.qr[slot] = r;
                        sm.qrl[slot] = rl;
                        sm.qo[0][slot] = om;
                        sm.qo[1][slot] = om * l2;
                        sm.qo[2][slot] = om * l4;
                        if (lin) {
                            T rs, rc;
                            hip_rotation(r, rl, dk32hi, dk32lo, &rs, &rc);
                            sm.qc[slot] = rc;
                            sm.qs[slot] = rs;
                        }
                        cnt += (unsigned long long)mult;
                    }
                    qn += __popc(m);
                    if (qn >= 32)
                        hip_drain_fold<T, NCH, MASK>(sm, qn, kk, kl, kx, lane, n_e, lin, tl, tw, H, R);
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
__global__ void __launch_bounds__(HIP_PAIR_THREADS)
    k_power_pairs(CellList<T> cl, PowerKernelArgs a, EdgeTable<T> ed, T R0, T dk32hi, T dk32lo)
{
    __shared__ WarpSmem<T, NCH> smem[HIP_PAIR_WARPS];
    __shared__ double red[3][HIP_MAX_EDGES];
    __shared__ int done;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    WarpSmem<T, NCH> &sm = smem[warp];
    for (int i = threadIdx.x; i < 3 * HIP_MAX_EDGES; i += HIP_PAIR_THREADS) (&red[0][0])[i] = 0.0;
    if (threadIdx.x == 0) done = 0;
    __syncthreads();
    const T R0sq = R0 * R0, invR0 = T(1) / R0, invR0lo = fma(-R0, invR0, T(1)) / R0;  // 1/R0 = invR0 + invR0lo
    const int n_e = a.n_e;
    const int n_ell = (MASK & 16) ? 3 : ((MASK & 4) ? 2 : 1);
    const int tl = (n_e - 1) / 32, tw = (n_e - 32 * tl <= 16) ? n_e - 32 * tl : 0;

    T kk[NCH], kl[NCH], kx[NCH];
    hip_lane_edges<T, NCH>(ed.k, ed.klo, lane, n_e, tl, tw, kk, kl, kx);
    T H[3][NCH];
    double R[3][NCH];
#pragma unroll
    for (int l = 0; l < 3; ++l)
#pragma unroll
        for (int t = 0; t < NCH; ++t) {
            H[l][t] = T(0);
            R[l][t] = 0.0;
        }
    hip_series_clear(sm, lane);
    unsigned long long cnt = 0;
    int qn = 0;
    for (;;) {
        int item = 0;
        if (lane == 0) item = atomicAdd(a.work_counter, 1);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= a.n_items) break;
        hip_pair_item<T, NCH, MASK>(cl, item, a.p0, a.p1, a.los, R0sq, invR0, invR0lo, LIN, dk32hi, dk32lo, sm, lane, kk, kl,
                                    kx, n_e, tl, tw, H, R, qn, cnt);
    }
    if (qn > 0) hip_drain_fold<T, NCH, MASK>(sm, qn, kk, kl, kx, lane, n_e, LIN, tl, tw, H, R);
    __syncthreads();
    for (int wv = 0; wv < HIP_PAIR_WARPS; ++wv) {
        if (warp == wv) {
#pragma unroll
            for (int l = 0; l < 3; ++l)
#pragma unroll
                for (int t = 0; t < NCH; ++t) {
                    const int e = hip_lane_edge(lane, t, n_e, tl, tw);
                    if (e >= 0) atomicAdd(&red[l][e], R[l][t]);
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
// (5 CTAs per SM: measured faster than the compiler's own register choice)
__global__ void __launch_bounds__(HIP_PAIR_THREADS, 5)
    k_power_pairs_batched(const BatchCat<T> *__restrict__ cats, int n_cats, int n_items, int *work_counter)
{
    __shared__ WarpSmem<T, NCH> smem[HIP_PAIR_WARPS];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    WarpSmem<T, NCH> &sm = smem[warp];
    T kk[NCH], kl[NCH], kx[NCH];
    T H[3][NCH];
    double R[3][NCH];
#pragma unroll
    for (int l = 0; l < 3; ++l)
#pragma unroll
        for (int t = 0; t < NCH; ++t) {
            H[l][t] = T(0);
            R[l][t] = 0.0;
        }
    hip_series_clear(sm, lane);
    unsigned long long cnt = 0;
    int qn = 0, cur = -1, tl = 0, tw = 0;
    auto leave = [&](int c) {
        if (qn > 0)
            hip_drain_fold<T, NCH, 21>(sm, qn, kk, kl, kx, lane, cats[c].n_e, cats[c].lin != 0, tl, tw, H, R);
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
            hip_lane_edges<T, NCH>(cats[c].k, cats[c].klo, lane, ne, tl, tw, kk, kl, kx);
        }
        const BatchCat<T> &bc = cats[c];
        hip_pair_item<T, NCH, 21>(bc.cl, item - bc.item_begin, bc.p0, bc.p1, bc.los, bc.R0 * bc.R0, T(1) / bc.R0,
                                  fma(-bc.R0, T(1) / bc.R0, T(1)) / bc.R0, bc.lin != 0, bc.dk32hi, bc.dk32lo, sm, lane, kk, kl, kx, bc.n_e, tl, tw, H, R,
                                  qn, cnt);
    }
    if (cur >= 0) leave(cur);
}

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


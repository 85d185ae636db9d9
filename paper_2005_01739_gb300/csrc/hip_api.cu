// C ABI of the library: argument validation, the per-device workspace, and the
// sequencing of the kernels for hip_power (Sec. 3 of arXiv:2005.01739).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include "hip_bispec.h"
#include "hip_e2.h"
#include "hip_moments.h"
#include "hip_internal.h"
#include "hip_workspace.h"

static thread_local char g_errbuf[512];

static void set_err(const char *what, cudaError_t e)
{
    std::snprintf(g_errbuf, sizeof(g_errbuf), "%s: %s", what, cudaGetErrorString(e));
}

extern "C" const char *hip_last_error(void) { return g_errbuf; }
void hip_clear_error() { g_errbuf[0] = 0; }
void hip_set_error(const char *what, cudaError_t e) { set_err(what, e); }

extern "C" const char *hip_status_string(hip_status s)
{
    switch (s) {
    case HIP_OK: return "ok";
    case HIP_ERR_ARG: return "invalid argument";
    case HIP_ERR_RANGE: return "argument out of range";
    case HIP_ERR_NONFINITE: return "non-finite position or weight";
    case HIP_ERR_CUDA: return "CUDA error";
    case HIP_ERR_NOMEM: return "out of device memory";
    case HIP_ERR_TIMEOUT: return "device wait timed out";
    }
    return "unknown status";
}

std::mutex &hip_api_mutex()
{
    static std::mutex m;
    return m;
}

// ------------------------------------------------------------- workspace ----
static Workspace g_ws[64];
static bool g_coeffs_ready[64];

hip_status hip_device_setup(int *dev_out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        set_err("cudaGetDevice", e);
        return HIP_ERR_CUDA;
    }
    if (dev < 0 || dev >= 64) return HIP_ERR_ARG;
    if (!g_coeffs_ready[dev]) {
        if ((e = hip_upload_coeffs_power()) != cudaSuccess || (e = hip_upload_coeffs_bispec()) != cudaSuccess ||
            (e = hip_upload_coeffs_e2()) != cudaSuccess) {
            set_err("coefficient upload", e);
            return HIP_ERR_CUDA;
        }
        g_coeffs_ready[dev] = true;
    }
    *dev_out = dev;
    return HIP_OK;
}

Workspace &hip_workspace(int dev) { return g_ws[dev]; }

hip_status Workspace::reserve(size_t bytes, cudaStream_t st)
{
    if (bytes <= cap) return HIP_OK;
    if (base) {
        cudaStreamSynchronize(st);
        cudaFree(base);
        base = nullptr;
        cap = 0;
    }
    size_t want = bytes + bytes / 4 + (1 << 20);
    cudaError_t e = cudaMalloc(&base, want);
    if (e != cudaSuccess) {
        cudaGetLastError();
        base = nullptr;
        set_err("cudaMalloc(workspace)", e);
        return HIP_ERR_NOMEM;
    }
    cap = want;
    return HIP_OK;
}

// Does `p` point to device-accessible memory of the current device?
bool hip_is_device_ptr(const void *p)
{
    if (!p) return false;
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

int hip_cells_per_side(double L, double R0)
{
    double q = std::floor(L / R0);
    int n = (int)q;
    if (n < 1) n = 1;
    if (n > 128) n = 128;
    return n;
}

hip_status hip_check_edges(const double *k_edges, int n_k)
{
    if (!k_edges) return HIP_ERR_ARG;
    if (n_k < 1 || n_k > HIP_MAX_BINS) return HIP_ERR_RANGE;
    for (int a = 0; a <= n_k; ++a)
        if (!std::isfinite(k_edges[a])) return HIP_ERR_RANGE;
    if (k_edges[0] < 0.0) return HIP_ERR_RANGE;
    for (int a = 0; a < n_k; ++a)
        if (!(k_edges[a + 1] > k_edges[a])) return HIP_ERR_RANGE;
    return HIP_OK;
}

// ------------------------------------------------------------- profiling -----
#define HIP_NSTAGE 5
static bool g_prof = false;
static bool g_prof_valid = false;
static double g_stage_ms[HIP_NSTAGE];

// Events: 0 start, 1 inputs uploaded, 2 cells built, 3 pair kernel begins,
// 4 pair kernel ends, 5 finalize ends, 6 results downloaded.
struct StageTimer {
    static const int NEV = 7;
    cudaEvent_t ev[NEV];
    bool on = false;
    cudaStream_t st;
    explicit StageTimer(cudaStream_t s) : st(s)
    {
        on = g_prof;
        g_prof_valid = false;
        if (on)
            for (auto &e : ev) cudaEventCreate(&e);
    }
    void mark(int i)
    {
        if (on) cudaEventRecord(ev[i], st);
    }
    void finish()
    {
        if (!on) return;
        cudaEventSynchronize(ev[NEV - 1]);
        const int a[HIP_NSTAGE] = {0, 1, 3, 4, 5}, b[HIP_NSTAGE] = {1, 2, 4, 5, 6};
        for (int i = 0; i < HIP_NSTAGE; ++i) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, ev[a[i]], ev[b[i]]);
            g_stage_ms[i] = ms;
        }
        g_prof_valid = true;
    }
    ~StageTimer()
    {
        if (on)
            for (auto &e : ev) cudaEventDestroy(e);
    }
};

extern "C" void hip_set_profiling(int on) { g_prof = on != 0; }

extern "C" int hip_power_pair_pass(double R0, double k_max, hip_precision prec)
{
    if (!(R0 > 0.0) || !(k_max > 0.0) || (prec != HIP_PREC_FP64 && prec != HIP_PREC_MIXED)) return -1;
    return hip_pm_applicable(R0, k_max, prec == HIP_PREC_MIXED) ? 1 : 0;
}

extern "C" int hip_stage_times(double *ms, int n)
{
    if (!g_prof_valid || !ms) return 0;
    int m = n < HIP_NSTAGE ? n : HIP_NSTAGE;
    for (int i = 0; i < m; ++i) ms[i] = g_stage_ms[i];
    return m;
}

// ------------------------------------------------------------- hip_power -----
template <typename T>
static hip_status power_impl(const float *pos, const float *w, int64_t N, double L, double R0,
                             const double *k_edges, int n_k, int ell_max, int los, int64_t p0, int64_t p1,
                             double *P_out, double *DD_out, int64_t *npairs_out, cudaStream_t st, int dev)
{
    Workspace &ws = hip_workspace(dev);
    const int n_c = hip_cells_per_side(L, R0);
    const int n_cells = n_c * n_c * n_c;
    const int n_e = n_k + 1, n_ell = ell_max / 2 + 1;
    const int grid = hip_power_grid<T>();
    const bool dpos = hip_is_device_ptr(pos);
    const bool dw = w && hip_is_device_ptr(w);

    Carve cv;
    size_t o_pos = dpos ? 0 : cv.take(sizeof(float) * 3 * N);
    size_t o_w = (w && !dw) ? cv.take(sizeof(float) * N) : 0;
    size_t o_x = cv.take(sizeof(T) * N), o_y = cv.take(sizeof(T) * N), o_z = cv.take(sizeof(T) * N);
    size_t o_ws = cv.take(sizeof(float) * N), o_idx = cv.take(sizeof(int) * N), o_cid = cv.take(sizeof(int) * N);
    size_t o_start = cv.take(sizeof(int) * (n_cells + 1)), o_fill = cv.take(sizeof(int) * n_cells);
    size_t o_part = cv.take(sizeof(double) * (size_t)grid * 3 * n_e);
    size_t o_small = cv.take(sizeof(double) * 8);
    size_t o_wt = cv.take(sizeof(double) * n_k);
    size_t o_dd = cv.take(sizeof(double) * 3 * n_k), o_p = cv.take(sizeof(double) * 3 * n_k);
    // the moment pass (Legendre moments of the separation) where it applies, else the direct one
    const bool moments = hip_pm_applicable(R0, k_edges[n_k], sizeof(T) == 4);
    const size_t o_pm = moments ? cv.take(hip_pm_scratch_bytes(n_e, hip_pm_intervals(R0, k_edges[n_k]))) : 0;
    hip_status hs = ws.reserve(cv.total, st);
    if (hs != HIP_OK) return hs;
    char *b = (char *)ws.base;
    cudaError_t e;
#define HIP_CK(call, what)                                                                                           \
    do {                                                                                                             \
        if ((e = (call)) != cudaSuccess) {                                                                           \
            set_err(what, e);                                                                                        \
            return HIP_ERR_CUDA;                                                                                     \
        }                                                                                                            \
    } while (0)
    const float *dposp = pos;
    const float *dwp = w;
    StageTimer tm(st);
    tm.mark(0);
    if (!dpos) {
        HIP_CK(cudaMemcpyAsync(b + o_pos, pos, sizeof(float) * 3 * N, cudaMemcpyHostToDevice, st), "H2D positions");
        dposp = (const float *)(b + o_pos);
    }
    if (w && !dw) {
        HIP_CK(cudaMemcpyAsync(b + o_w, w, sizeof(float) * N, cudaMemcpyHostToDevice, st), "H2D weights");
        dwp = (const float *)(b + o_w);
    }
    T *x = (T *)(b + o_x), *y = (T *)(b + o_y), *z = (T *)(b + o_z);
    float *wsrt = (float *)(b + o_ws);
    int *idx = (int *)(b + o_idx), *cid = (int *)(b + o_cid);
    int *cstart = (int *)(b + o_start), *cfill = (int *)(b + o_fill);
    double *partials = (double *)(b + o_part);
    double *small = (double *)(b + o_small);  // [0] S1, [1] npairs (u64), [2] err|counter (ints)
    double *S1 = small;
    unsigned long long *npairs = (unsigned long long *)(small + 1);
    int *err = (int *)(small + 2);
    int *counter = err + 1;
    double *Wt = (double *)(b + o_wt), *DD = (double *)(b + o_dd), *P = (double *)(b + o_p);

    tm.mark(1);
    HIP_CK(hip_build_cells<T>(dposp, dwp, N, L, n_c, x, y, z, wsrt, idx, cid, cstart, cfill, S1, err, st),
           "cell build");
    tm.mark(2);
    int herr = 0;
    HIP_CK(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st), "D2H error word");
    HIP_CK(cudaStreamSynchronize(st), "cell build sync");
    if (herr) return HIP_ERR_NONFINITE;

    HIP_CK(cudaMemsetAsync(npairs, 0, sizeof(unsigned long long), st), "memset");
    HIP_CK(cudaMemsetAsync(counter, 0, sizeof(int), st), "memset");
    CellList<T> cl{x, y, z, wsrt, idx, cstart, n_c, L, L / n_c};
    PowerKernelArgs ka;
    ka.n_e = n_e;
    ka.los = los;
    ka.p0 = p0;
    ka.p1 = p1;
    ka.n_items = n_cells * HIP_NSHIFT;
    ka.work_counter = counter;
    ka.partials = partials;
    ka.npairs = npairs;
    tm.mark(3);
    if (moments)
        HIP_CK(hip_power_moments<T>(cl, ka, k_edges, n_ell, R0, b + o_pm, partials, st), "moment pair pass");
    else
        HIP_CK(hip_power_pairs<T>(cl, ka, k_edges, n_ell, R0, grid, st), "pair kernel");
    tm.mark(4);
    HIP_CK(hip_power_finalize(partials, moments ? 1 : grid, n_e, n_ell, k_edges, R0, L, S1, Wt, DD, P, st),
           "finalize");
    tm.mark(5);
    std::vector<double> hP(n_ell * n_k), hDD(n_ell * n_k);
    unsigned long long hn = 0;
    HIP_CK(cudaMemcpyAsync(hP.data(), P, sizeof(double) * n_ell * n_k, cudaMemcpyDeviceToHost, st), "D2H P");
    HIP_CK(cudaMemcpyAsync(hDD.data(), DD, sizeof(double) * n_ell * n_k, cudaMemcpyDeviceToHost, st), "D2H DD");
    HIP_CK(cudaMemcpyAsync(&hn, npairs, sizeof(hn), cudaMemcpyDeviceToHost, st), "D2H npairs");
    tm.mark(6);
    HIP_CK(cudaStreamSynchronize(st), "stream sync");
    tm.finish();
#undef HIP_CK
    std::memcpy(P_out, hP.data(), sizeof(double) * n_ell * n_k);
    if (DD_out) std::memcpy(DD_out, hDD.data(), sizeof(double) * n_ell * n_k);
    if (npairs_out) *npairs_out = (int64_t)hn;
    return HIP_OK;
}

extern "C" hip_status hip_power(const float *pos, const float *w, int64_t N, double L, double R0, hip_window window,
                                const double *k_edges, int n_k, int ell_max, int los_axis, hip_precision prec,
                                int64_t prim_begin, int64_t prim_end, double *P_out, double *DD_out,
                                int64_t *npairs_out, void *cuda_stream)
{
    g_errbuf[0] = 0;
    if (!pos || !P_out) return HIP_ERR_ARG;
    if (N < 1 || N > 2000000000LL) return HIP_ERR_ARG;
    if (window != HIP_WINDOW_PHILCOX) return HIP_ERR_ARG;
    if (prec != HIP_PREC_FP64 && prec != HIP_PREC_MIXED) return HIP_ERR_ARG;
    if (ell_max != 0 && ell_max != 2 && ell_max != 4) return HIP_ERR_ARG;
    if (los_axis < 0 || los_axis > 2) return HIP_ERR_ARG;
    if (!(L > 0.0) || !std::isfinite(L) || !(R0 > 0.0) || !(R0 < 0.5 * L)) return HIP_ERR_RANGE;
    if (prim_begin < 0 || prim_end > N || prim_begin > prim_end) return HIP_ERR_RANGE;
    hip_status hs = hip_check_edges(k_edges, n_k);
    if (hs != HIP_OK) return hs;
    std::lock_guard<std::mutex> lk(hip_api_mutex());
    int dev = 0;
    if ((hs = hip_device_setup(&dev)) != HIP_OK) return hs;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if (prec == HIP_PREC_MIXED)
        return power_impl<float>(pos, w, N, L, R0, k_edges, n_k, ell_max, los_axis, prim_begin, prim_end, P_out,
                                 DD_out, npairs_out, st, dev);
    return power_impl<double>(pos, w, N, L, R0, k_edges, n_k, ell_max, los_axis, prim_begin, prim_end, P_out,
                              DD_out, npairs_out, st, dev);
}

// --------------------------------------------------------- hip_bispectrum ----
// S^a of the bispectrum estimator (Sec. 4.5): the l = 0 pair sum of the power
// pass over all data, finalized into DD; the Legendre-moment pass where it
// applies (pm_scratch then holds s_pass_scratch bytes), else the direct pass.
static size_t s_pass_scratch(double R0, const double *k_edges, int n_k, bool fp32)
{
    if (!hip_pm_applicable(R0, k_edges[n_k], fp32)) return 256;
    return hip_pm_scratch_bytes(n_k + 1, hip_pm_intervals(R0, k_edges[n_k]));
}
template <typename T>
static cudaError_t s_pass(const CellList<T> &cl, const PowerKernelArgs &ka, const double *k_edges, int n_k, double R0,
                          double L, const double *S1, double *Wt, double *DD, double *P, void *pm_scratch, int pgrid,
                          cudaStream_t st)
{
    const bool pm = hip_pm_applicable(R0, k_edges[n_k], sizeof(T) == 4);
    const cudaError_t e = pm ? hip_power_moments<T>(cl, ka, k_edges, 1, R0, pm_scratch, ka.partials, st)
                             : hip_power_pairs<T>(cl, ka, k_edges, 1, R0, pgrid, st);
    if (e != cudaSuccess) return e;
    return hip_power_finalize(ka.partials, pm ? 1 : pgrid, n_k + 1, 1, k_edges, R0, L, S1, Wt, DD, P, st);
}

template <typename T>
static hip_status bispec_impl(const float *pos, const float *w, int64_t N, const float *rpos, int64_t N_r, double L,
                              double R0, const double *k_edges, int n_k, int lmax, double *B_out,
                              int64_t *npairs_out, cudaStream_t st, int dev, const int64_t *ranges, bool partial)
{
    Workspace &ws = hip_workspace(dev);
    const int n_c = hip_cells_per_side(L, R0);
    const int n_cells = n_c * n_c * n_c;
    const int n_e = n_k + 1;
    const int pgrid = hip_power_grid<T>();
    const bool dpos = hip_is_device_ptr(pos), dw = w && hip_is_device_ptr(w), drp = hip_is_device_ptr(rpos);
    const int bparts_max = 152 * 8;  // upper bound on the bispectrum grid
    const size_t tsz = (size_t)(HIP_LMAX + 1) * n_k * n_k;

    Carve cv;
    const size_t o_pos = dpos ? 0 : cv.take(sizeof(float) * 3 * N);
    const size_t o_w = (w && !dw) ? cv.take(sizeof(float) * N) : 0;
    const size_t o_rp = drp ? 0 : cv.take(sizeof(float) * 3 * N_r);
    const size_t o_dx = cv.take(sizeof(T) * N), o_dy = cv.take(sizeof(T) * N), o_dz = cv.take(sizeof(T) * N);
    const size_t o_dw = cv.take(sizeof(float) * N), o_didx = cv.take(sizeof(int) * N), o_dcid = cv.take(sizeof(int) * N);
    const size_t o_rx = cv.take(sizeof(T) * N_r), o_ry = cv.take(sizeof(T) * N_r), o_rz = cv.take(sizeof(T) * N_r);
    const size_t o_rw = cv.take(sizeof(float) * N_r), o_ridx = cv.take(sizeof(int) * N_r);
    const size_t o_rcid = cv.take(sizeof(int) * N_r);
    const size_t o_ds = cv.take(sizeof(int) * (n_cells + 1)), o_df = cv.take(sizeof(int) * n_cells);
    const size_t o_dsc = cv.take(sizeof(int) * N), o_rsc = cv.take(sizeof(int) * N_r);
    const size_t o_rs = cv.take(sizeof(int) * (n_cells + 1)), o_rf = cv.take(sizeof(int) * n_cells);
    const size_t o_pp = cv.take(sizeof(double) * (size_t)pgrid * 3 * n_e);
    const size_t o_bp = cv.take(sizeof(double) * bparts_max * tsz);
    const size_t o_small = cv.take(sizeof(double) * 16);
    const size_t o_wt = cv.take(sizeof(double) * n_k), o_dd = cv.take(sizeof(double) * 3 * n_k);
    const size_t o_p = cv.take(sizeof(double) * 3 * n_k), o_b = cv.take(sizeof(double) * tsz);
    const size_t o_pm = cv.take(s_pass_scratch(R0, k_edges, n_k, sizeof(T) == 4));
    hip_status hs = ws.reserve(cv.total, st);
    if (hs != HIP_OK) return hs;
    char *b = (char *)ws.base;
    cudaError_t e;
#define HIP_CK(call, what)                                                                                           \
    do {                                                                                                             \
        if ((e = (call)) != cudaSuccess) {                                                                           \
            set_err(what, e);                                                                                        \
            return HIP_ERR_CUDA;                                                                                     \
        }                                                                                                            \
    } while (0)
    const float *dposp = pos, *dwp = w, *drpp = rpos;
    if (!dpos) {
        HIP_CK(cudaMemcpyAsync(b + o_pos, pos, sizeof(float) * 3 * N, cudaMemcpyHostToDevice, st), "H2D positions");
        dposp = (const float *)(b + o_pos);
    }
    if (w && !dw) {
        HIP_CK(cudaMemcpyAsync(b + o_w, w, sizeof(float) * N, cudaMemcpyHostToDevice, st), "H2D weights");
        dwp = (const float *)(b + o_w);
    }
    if (!drp) {
        HIP_CK(cudaMemcpyAsync(b + o_rp, rpos, sizeof(float) * 3 * N_r, cudaMemcpyHostToDevice, st), "H2D randoms");
        drpp = (const float *)(b + o_rp);
    }
    double *small = (double *)(b + o_small);
    double *S1 = small, *S1r = small + 1;
    unsigned long long *npairs = (unsigned long long *)(small + 2);  // [2]: P pass; [3], [4]: B pass
    int *err = (int *)(small + 5), *errr = err + 1;
    int *counter = (int *)(small + 6), *bcounter = counter + 1;
    T *dx = (T *)(b + o_dx), *dy = (T *)(b + o_dy), *dz = (T *)(b + o_dz);
    T *rx = (T *)(b + o_rx), *ry = (T *)(b + o_ry), *rz = (T *)(b + o_rz);
    int *dstart = (int *)(b + o_ds), *rstart = (int *)(b + o_rs);
    HIP_CK(hip_build_cells<T>(dposp, dwp, N, L, n_c, dx, dy, dz, (float *)(b + o_dw), (int *)(b + o_didx),
                              (int *)(b + o_dcid), dstart, (int *)(b + o_df), S1, err, st),
           "cell build (data)");
    HIP_CK(hip_build_cells<T>(drpp, nullptr, N_r, L, n_c, rx, ry, rz, (float *)(b + o_rw), (int *)(b + o_ridx),
                              (int *)(b + o_rcid), rstart, (int *)(b + o_rf), S1r, errr, st),
           "cell build (randoms)");
    HIP_CK(hip_sorted_cells(dstart, n_cells, (int *)(b + o_dsc), st), "sorted cells (data)");
    HIP_CK(hip_sorted_cells(rstart, n_cells, (int *)(b + o_rsc), st), "sorted cells (randoms)");
    int herr[2] = {0, 0};
    double hS1 = 0.0;
    HIP_CK(cudaMemcpyAsync(herr, err, 2 * sizeof(int), cudaMemcpyDeviceToHost, st), "D2H error word");
    HIP_CK(cudaMemcpyAsync(&hS1, S1, sizeof(double), cudaMemcpyDeviceToHost, st), "D2H S1");
    HIP_CK(cudaStreamSynchronize(st), "cell build sync");
    if (herr[0] || herr[1]) return HIP_ERR_NONFINITE;

    // S^a: ordered DD_0 pair sum over all data (the power pass with l = 0 only)
    CellList<T> dcl{dx, dy, dz, (const float *)(b + o_dw), (const int *)(b + o_didx), dstart, n_c, L, L / n_c};
    CellList<T> rcl{rx, ry, rz, (const float *)(b + o_rw), (const int *)(b + o_ridx), rstart, n_c, L, L / n_c};
    HIP_CK(cudaMemsetAsync(npairs, 0, 3 * sizeof(unsigned long long), st), "memset");
    HIP_CK(cudaMemsetAsync(counter, 0, 2 * sizeof(int), st), "memset");
    PowerKernelArgs ka;
    ka.n_e = n_e;
    ka.los = 2;
    ka.p0 = 0;
    ka.p1 = N;
    ka.n_items = n_cells * HIP_NSHIFT;
    ka.work_counter = counter;
    ka.partials = (double *)(b + o_pp);
    ka.npairs = npairs;
    double *Wt = (double *)(b + o_wt), *DD = (double *)(b + o_dd), *P = (double *)(b + o_p);
    HIP_CK(s_pass<T>(dcl, ka, k_edges, n_k, R0, L, S1, Wt, DD, P, b + o_pm, pgrid, st), "pair pass (S)");

    BispecArgs<T> ba;
    ba.data = dcl;
    ba.rand = rcl;
    ba.n_cells = n_cells;
    ba.dcell = (const int *)(b + o_dsc);
    ba.rcell = (const int *)(b + o_rsc);
    ba.n_data = (int)N;
    ba.n_rand = (int)N_r;
    ba.n_e = n_e;
    ba.R0 = (T)R0;
    ba.rand_weight = (T)(-hS1 / (double)N_r);
    ba.work_counter = bcounter;
    ba.partials = (double *)(b + o_bp);
    ba.npairs = npairs + 1;
    ba.dp0 = ranges ? ranges[0] : 0;
    ba.dp1 = ranges ? ranges[1] : N;
    ba.rp0 = ranges ? ranges[2] : 0;
    ba.rp1 = ranges ? ranges[3] : N_r;
    for (int q = 0; q < HIP_BMAXE; ++q) {
        const double k = q < n_e ? k_edges[q] : 0.0;
        ba.k[q] = (T)k;
        ba.klo[q] = (T)(k - (double)ba.k[q]);
        ba.k3[q] = (T)(k * k * k);
        ba.jfac[q] = q + 1 < n_e ? (T)(3.0 / (k_edges[q + 1] * k_edges[q + 1] * k_edges[q + 1] - k * k * k)) : T(0);
    }
    int bgrid = 0;
    HIP_CK(hip_bispec_pairs<T>(ba, bparts_max, &bgrid, st), "bispectrum kernel");
    double *B = (double *)(b + o_b);
    if (partial)
        HIP_CK(hip_bispec_sum(ba.partials, bgrid, n_k, lmax, B, st), "bispectrum sum");
    else
        HIP_CK(hip_bispec_finalize(ba.partials, bgrid, n_k, lmax, L, S1, DD, Wt, B, st), "bispectrum finalize");
    const size_t nout = (size_t)(lmax + 1) * n_k * n_k;
    std::vector<double> hB(nout);
    unsigned long long hn[3] = {0, 0, 0};
    HIP_CK(cudaMemcpyAsync(hB.data(), B, sizeof(double) * nout, cudaMemcpyDeviceToHost, st), "D2H B");
    HIP_CK(cudaMemcpyAsync(hn, npairs, sizeof(hn), cudaMemcpyDeviceToHost, st), "D2H npairs");
    HIP_CK(cudaStreamSynchronize(st), "stream sync");
#undef HIP_CK
    std::memcpy(B_out, hB.data(), sizeof(double) * nout);
    if (npairs_out) {
        npairs_out[0] = (int64_t)hn[1];
        npairs_out[1] = (int64_t)hn[2];
    }
    return HIP_OK;
}

extern "C" hip_status hip_bispectrum(const float *pos, const float *w, int64_t N, const float *rand_pos, int64_t N_r,
                                     double L, double R0, hip_window window, const double *k_edges, int n_k,
                                     int lmax, hip_precision prec, double *B_out, int64_t *npairs_out,
                                     void *cuda_stream)
{
    g_errbuf[0] = 0;
    if (!pos || !rand_pos || !B_out) return HIP_ERR_ARG;
    if (N < 1 || N > 2000000000LL || N_r < 1 || N_r > 2000000000LL) return HIP_ERR_ARG;
    if (window != HIP_WINDOW_PHILCOX) return HIP_ERR_ARG;
    if (prec != HIP_PREC_FP64 && prec != HIP_PREC_MIXED) return HIP_ERR_ARG;
    if (lmax < 0 || lmax > HIP_LMAX) return HIP_ERR_ARG;
    if (!(L > 0.0) || !std::isfinite(L) || !(R0 > 0.0) || !(R0 < 0.5 * L)) return HIP_ERR_RANGE;
    hip_status hs = hip_check_edges(k_edges, n_k);
    if (hs != HIP_OK) return hs;
    if (n_k > (prec == HIP_PREC_MIXED ? HIP_BMAXE - 2 : 31)) return HIP_ERR_RANGE;
    std::lock_guard<std::mutex> lk(hip_api_mutex());
    int dev = 0;
    if ((hs = hip_device_setup(&dev)) != HIP_OK) return hs;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if (prec == HIP_PREC_MIXED)
        return bispec_impl<float>(pos, w, N, rand_pos, N_r, L, R0, k_edges, n_k, lmax, B_out, npairs_out, st, dev,
                                  nullptr, false);
    return bispec_impl<double>(pos, w, N, rand_pos, N_r, L, R0, k_edges, n_k, lmax, B_out, npairs_out, st, dev,
                               nullptr, false);
}

// Batched bispectra: per catalog the buffers of bispec_impl (one workspace
// carve for all), one persistent bispectrum launch over every catalog's
// primaries, FP64 finalize per catalog.
template <typename T>
static hip_status bispec_batched_impl(const hip_bcatalog *cats, int nc, cudaStream_t st, int dev)
{
    Workspace &ws = hip_workspace(dev);
    const int pgrid = hip_power_grid<T>();
    struct Lay {
        int n_c, n_cells, n_k, n_e;
        bool dpos, dw, drp;
        size_t o_pos, o_w, o_rp, o_dx, o_dy, o_dz, o_dw, o_didx, o_dcid, o_rx, o_ry, o_rz, o_rw, o_ridx, o_rcid;
        size_t o_ds, o_df, o_dsc, o_rsc, o_rs, o_rf, o_small, o_wt, o_dd, o_p, o_b, o_acc;
    };
    std::vector<Lay> lay(nc);
    Carve cv;
    int nk_max = 0, ne_max = 0;
    for (int i = 0; i < nc; ++i) {
        const hip_bcatalog &c = cats[i];
        Lay &y = lay[i];
        y.n_c = hip_cells_per_side(c.L, c.R0);
        y.n_cells = y.n_c * y.n_c * y.n_c;
        y.n_k = c.n_k;
        y.n_e = c.n_k + 1;
        nk_max = std::max(nk_max, y.n_k);
        ne_max = std::max(ne_max, y.n_e);
        y.dpos = hip_is_device_ptr(c.pos);
        y.dw = c.w && hip_is_device_ptr(c.w);
        y.drp = hip_is_device_ptr(c.rand_pos);
        const int64_t N = c.N, Nr = c.N_r;
        const size_t tsz = (size_t)(HIP_LMAX + 1) * c.n_k * c.n_k;
        y.o_pos = y.dpos ? 0 : cv.take(sizeof(float) * 3 * N);
        y.o_w = (c.w && !y.dw) ? cv.take(sizeof(float) * N) : 0;
        y.o_rp = y.drp ? 0 : cv.take(sizeof(float) * 3 * Nr);
        y.o_dx = cv.take(sizeof(T) * N), y.o_dy = cv.take(sizeof(T) * N), y.o_dz = cv.take(sizeof(T) * N);
        y.o_dw = cv.take(sizeof(float) * N), y.o_didx = cv.take(sizeof(int) * N), y.o_dcid = cv.take(sizeof(int) * N);
        y.o_rx = cv.take(sizeof(T) * Nr), y.o_ry = cv.take(sizeof(T) * Nr), y.o_rz = cv.take(sizeof(T) * Nr);
        y.o_rw = cv.take(sizeof(float) * Nr), y.o_ridx = cv.take(sizeof(int) * Nr);
        y.o_rcid = cv.take(sizeof(int) * Nr);
        y.o_ds = cv.take(sizeof(int) * (y.n_cells + 1)), y.o_df = cv.take(sizeof(int) * y.n_cells);
        y.o_dsc = cv.take(sizeof(int) * N), y.o_rsc = cv.take(sizeof(int) * Nr);
        y.o_rs = cv.take(sizeof(int) * (y.n_cells + 1)), y.o_rf = cv.take(sizeof(int) * y.n_cells);
        y.o_small = cv.take(sizeof(double) * 16);
        y.o_wt = cv.take(sizeof(double) * c.n_k), y.o_dd = cv.take(sizeof(double) * 3 * c.n_k);
        y.o_p = cv.take(sizeof(double) * 3 * c.n_k), y.o_b = cv.take(sizeof(double) * tsz);
        y.o_acc = cv.take(sizeof(double) * tsz);
    }
    const size_t o_pp = cv.take(sizeof(double) * (size_t)pgrid * 3 * ne_max);
    size_t pm_bytes = 256;  // the S passes run one after another in stream order and share this scratch
    for (int i = 0; i < nc; ++i)
        pm_bytes = std::max(pm_bytes, s_pass_scratch(cats[i].R0, cats[i].k_edges, cats[i].n_k, sizeof(T) == 4));
    const size_t o_pm = cv.take(pm_bytes);
    const size_t o_desc = cv.take(sizeof(BispecCat<T>) * nc);
    const size_t o_cnt = cv.take(sizeof(int) * 4);
    hip_status hs = ws.reserve(cv.total, st);
    if (hs != HIP_OK) return hs;
    char *b = (char *)ws.base;
    cudaError_t e;
#define HIP_CK(call, what)                                                                                           \
    do {                                                                                                             \
        if ((e = (call)) != cudaSuccess) {                                                                           \
            set_err(what, e);                                                                                        \
            return HIP_ERR_CUDA;                                                                                     \
        }                                                                                                            \
    } while (0)
    std::vector<CellList<T>> dcl(nc), rcl(nc);
    for (int i = 0; i < nc; ++i) {
        const hip_bcatalog &c = cats[i];
        const Lay &y = lay[i];
        const float *dposp = c.pos, *dwp = c.w, *drpp = c.rand_pos;
        if (!y.dpos) {
            HIP_CK(cudaMemcpyAsync(b + y.o_pos, c.pos, sizeof(float) * 3 * c.N, cudaMemcpyHostToDevice, st),
                   "H2D positions");
            dposp = (const float *)(b + y.o_pos);
        }
        if (c.w && !y.dw) {
            HIP_CK(cudaMemcpyAsync(b + y.o_w, c.w, sizeof(float) * c.N, cudaMemcpyHostToDevice, st), "H2D weights");
            dwp = (const float *)(b + y.o_w);
        }
        if (!y.drp) {
            HIP_CK(cudaMemcpyAsync(b + y.o_rp, c.rand_pos, sizeof(float) * 3 * c.N_r, cudaMemcpyHostToDevice, st),
                   "H2D randoms");
            drpp = (const float *)(b + y.o_rp);
        }
        double *small = (double *)(b + y.o_small);
        int *err = (int *)(small + 5);
        T *dx = (T *)(b + y.o_dx), *dy = (T *)(b + y.o_dy), *dz = (T *)(b + y.o_dz);
        T *rx = (T *)(b + y.o_rx), *ry = (T *)(b + y.o_ry), *rz = (T *)(b + y.o_rz);
        int *dstart = (int *)(b + y.o_ds), *rstart = (int *)(b + y.o_rs);
        HIP_CK(hip_build_cells<T>(dposp, dwp, c.N, c.L, y.n_c, dx, dy, dz, (float *)(b + y.o_dw), (int *)(b + y.o_didx),
                                  (int *)(b + y.o_dcid), dstart, (int *)(b + y.o_df), small, err, st),
               "cell build (data)");
        HIP_CK(hip_build_cells<T>(drpp, nullptr, c.N_r, c.L, y.n_c, rx, ry, rz, (float *)(b + y.o_rw),
                                  (int *)(b + y.o_ridx), (int *)(b + y.o_rcid), rstart, (int *)(b + y.o_rf), small + 1,
                                  err + 1, st),
               "cell build (randoms)");
        HIP_CK(hip_sorted_cells(dstart, y.n_cells, (int *)(b + y.o_dsc), st), "sorted cells (data)");
        HIP_CK(hip_sorted_cells(rstart, y.n_cells, (int *)(b + y.o_rsc), st), "sorted cells (randoms)");
        dcl[i] = CellList<T>{dx, dy, dz, (const float *)(b + y.o_dw), (const int *)(b + y.o_didx), dstart, y.n_c, c.L,
                             c.L / y.n_c};
        rcl[i] = CellList<T>{rx, ry, rz, (const float *)(b + y.o_rw), (const int *)(b + y.o_ridx), rstart, y.n_c, c.L,
                             c.L / y.n_c};
    }
    // S1 of every catalog (for the random primaries' weight) and the error words
    std::vector<double> hsm((size_t)nc * 6);
    for (int i = 0; i < nc; ++i)
        HIP_CK(cudaMemcpyAsync(&hsm[(size_t)i * 6], b + lay[i].o_small, sizeof(double) * 6, cudaMemcpyDeviceToHost,
                               st),
               "D2H S1");
    HIP_CK(cudaStreamSynchronize(st), "cell build sync");
    for (int i = 0; i < nc; ++i) {
        int herr[2];
        std::memcpy(herr, &hsm[(size_t)i * 6 + 5], sizeof(herr));
        if (herr[0] || herr[1]) return HIP_ERR_NONFINITE;
    }
    // S^a of every catalog: the l = 0 power pair sum (one launch each; the
    // partial rows are reused in stream order)
    std::vector<BispecCat<T>> desc(nc);
    int items = 0;
    for (int i = 0; i < nc; ++i) {
        const hip_bcatalog &c = cats[i];
        const Lay &y = lay[i];
        double *small = (double *)(b + y.o_small);
        unsigned long long *npairs = (unsigned long long *)(small + 2);
        int *counter = (int *)(small + 6);
        HIP_CK(cudaMemsetAsync(npairs, 0, 3 * sizeof(unsigned long long), st), "memset");
        HIP_CK(cudaMemsetAsync(counter, 0, sizeof(int), st), "memset");
        HIP_CK(cudaMemsetAsync(b + y.o_acc, 0, sizeof(double) * (HIP_LMAX + 1) * c.n_k * c.n_k, st), "memset");
        PowerKernelArgs ka;
        ka.n_e = y.n_e;
        ka.los = 2;
        ka.p0 = 0;
        ka.p1 = c.N;
        ka.n_items = y.n_cells * HIP_NSHIFT;
        ka.work_counter = counter;
        ka.partials = (double *)(b + o_pp);
        ka.npairs = npairs;
        HIP_CK(s_pass<T>(dcl[i], ka, c.k_edges, c.n_k, c.R0, c.L, small, (double *)(b + y.o_wt),
                         (double *)(b + y.o_dd), (double *)(b + y.o_p), b + o_pm, pgrid, st),
               "pair pass (S)");
        BispecCat<T> &d = desc[i];
        std::memset(&d, 0, sizeof(d));
        BispecArgs<T> &ba = d.a;
        ba.data = dcl[i];
        ba.rand = rcl[i];
        ba.n_cells = y.n_cells;
        ba.dcell = (const int *)(b + y.o_dsc);
        ba.rcell = (const int *)(b + y.o_rsc);
        ba.n_data = (int)c.N;
        ba.n_rand = (int)c.N_r;
        ba.n_e = y.n_e;
        ba.R0 = (T)c.R0;
        ba.rand_weight = (T)(-hsm[(size_t)i * 6] / (double)c.N_r);
        ba.npairs = npairs + 1;
        ba.dp0 = 0;
        ba.dp1 = c.N;
        ba.rp0 = 0;
        ba.rp1 = c.N_r;
        for (int q = 0; q < HIP_BMAXE; ++q) {
            const double k = q < y.n_e ? c.k_edges[q] : 0.0;
            ba.k[q] = (T)k;
            ba.klo[q] = (T)(k - (double)ba.k[q]);
            ba.k3[q] = (T)(k * k * k);
            ba.jfac[q] = q + 1 < y.n_e
                             ? (T)(3.0 / (c.k_edges[q + 1] * c.k_edges[q + 1] * c.k_edges[q + 1] - k * k * k))
                             : T(0);
        }
        const int64_t n_prim = c.N + c.N_r;
        d.item_begin = items;
        items += (int)((n_prim + HIP_BCTA_PRIM - 1) / HIP_BCTA_PRIM);
        d.item_end = items;
        d.acc = (double *)(b + y.o_acc);
    }
    BispecCat<T> *ddesc = (BispecCat<T> *)(b + o_desc);
    int *bcounter = (int *)(b + o_cnt);
    HIP_CK(cudaMemcpyAsync(ddesc, desc.data(), sizeof(BispecCat<T>) * nc, cudaMemcpyHostToDevice, st),
           "H2D descriptors");
    HIP_CK(cudaMemsetAsync(bcounter, 0, sizeof(int), st), "memset");
    int bgrid = 0;
    HIP_CK(hip_bispec_pairs_batched<T>(ddesc, nc, items, nk_max, bcounter, &bgrid, st), "batched bispectrum kernel");
    std::vector<std::vector<double>> hB(nc);
    std::vector<unsigned long long> hn((size_t)nc * 3);
    for (int i = 0; i < nc; ++i) {
        const hip_bcatalog &c = cats[i];
        const Lay &y = lay[i];
        double *small = (double *)(b + y.o_small);
        double *B = (double *)(b + y.o_b);
        HIP_CK(hip_bispec_finalize((double *)(b + y.o_acc), 1, c.n_k, c.lmax, c.L, small, (double *)(b + y.o_dd),
                                   (double *)(b + y.o_wt), B, st),
               "bispectrum finalize");
        hB[i].resize((size_t)(c.lmax + 1) * c.n_k * c.n_k);
        HIP_CK(cudaMemcpyAsync(hB[i].data(), B, sizeof(double) * hB[i].size(), cudaMemcpyDeviceToHost, st), "D2H B");
        HIP_CK(cudaMemcpyAsync(&hn[(size_t)i * 3], small + 2, 3 * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                               st),
               "D2H npairs");
    }
    HIP_CK(cudaStreamSynchronize(st), "stream sync");
#undef HIP_CK
    for (int i = 0; i < nc; ++i) {
        std::memcpy(cats[i].B_out, hB[i].data(), sizeof(double) * hB[i].size());
        if (cats[i].npairs_out) {
            cats[i].npairs_out[0] = (int64_t)hn[(size_t)i * 3 + 1];
            cats[i].npairs_out[1] = (int64_t)hn[(size_t)i * 3 + 2];
        }
    }
    return HIP_OK;
}

extern "C" hip_status hip_bispectrum_batched(const hip_bcatalog *cats, int n_cats, hip_precision prec,
                                             void *cuda_stream)
{
    g_errbuf[0] = 0;
    if (!cats || n_cats < 1 || n_cats > 4096) return HIP_ERR_ARG;
    if (prec != HIP_PREC_FP64 && prec != HIP_PREC_MIXED) return HIP_ERR_ARG;
    for (int i = 0; i < n_cats; ++i) {
        const hip_bcatalog &c = cats[i];
        if (!c.pos || !c.rand_pos || !c.B_out) return HIP_ERR_ARG;
        if (c.N < 1 || c.N > 2000000000LL || c.N_r < 1 || c.N_r > 2000000000LL) return HIP_ERR_ARG;
        if (c.lmax < 0 || c.lmax > HIP_LMAX) return HIP_ERR_ARG;
        if (!(c.L > 0.0) || !std::isfinite(c.L) || !(c.R0 > 0.0) || !(c.R0 < 0.5 * c.L)) return HIP_ERR_RANGE;
        hip_status hs = hip_check_edges(c.k_edges, c.n_k);
        if (hs != HIP_OK) return hs;
        if (c.n_k > (prec == HIP_PREC_MIXED ? HIP_BMAXE - 2 : 31)) return HIP_ERR_RANGE;
    }
    std::lock_guard<std::mutex> lk(hip_api_mutex());
    int dev = 0;
    hip_status hs;
    if ((hs = hip_device_setup(&dev)) != HIP_OK) return hs;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if (prec == HIP_PREC_MIXED) return bispec_batched_impl<float>(cats, n_cats, st, dev);
    return bispec_batched_impl<double>(cats, n_cats, st, dev);
}

// Bispectrum with the random-free DDR^II term (App. A): data primaries only,
// plus one FP64 partial row -(S1/V) sum_{j != k} w_j w_k E^{II}(r_jk) from
// hip_e2_term (pairs to 2 R0 on a second cell list of cells >= 2 R0 wide).
template <typename T>
static hip_status bispec_analytic_impl(const float *pos, const float *w, int64_t N, double L, double R0,
                                       const double *k_edges, int n_k, int lmax, double *B_out, int64_t *npairs_out,
                                       cudaStream_t st, int dev)
{
    Workspace &ws = hip_workspace(dev);
    const int n_c = hip_cells_per_side(L, R0), n_cells = n_c * n_c * n_c;
    const int n_c2 = hip_cells_per_side(L, 2.0 * R0), n_cells2 = n_c2 * n_c2 * n_c2;
    const int n_e = n_k + 1;
    const int pgrid = hip_power_grid<T>();
    const bool dpos = hip_is_device_ptr(pos), dw = w && hip_is_device_ptr(w);
    const int bparts_max = 152 * 8;
    const size_t tsz = (size_t)(HIP_LMAX + 1) * n_k * n_k;
    E2Nodes nodes;
    hip_e2_nodes(k_edges, n_k, R0, nodes);

    Carve cv;
    const size_t o_pos = dpos ? 0 : cv.take(sizeof(float) * 3 * N);
    const size_t o_w = (w && !dw) ? cv.take(sizeof(float) * N) : 0;
    const size_t o_dx = cv.take(sizeof(T) * N), o_dy = cv.take(sizeof(T) * N), o_dz = cv.take(sizeof(T) * N);
    const size_t o_dw = cv.take(sizeof(float) * N), o_didx = cv.take(sizeof(int) * N), o_dcid = cv.take(sizeof(int) * N);
    const size_t o_ds = cv.take(sizeof(int) * (n_cells + 1)), o_df = cv.take(sizeof(int) * n_cells);
    const size_t o_dsc = cv.take(sizeof(int) * N);
    const size_t o_x2 = cv.take(sizeof(float) * N), o_y2 = cv.take(sizeof(float) * N), o_z2 = cv.take(sizeof(float) * N);
    const size_t o_w2 = cv.take(sizeof(float) * N), o_i2 = cv.take(sizeof(int) * N), o_c2 = cv.take(sizeof(int) * N);
    const size_t o_s2 = cv.take(sizeof(int) * (n_cells2 + 1)), o_f2 = cv.take(sizeof(int) * n_cells2);
    const size_t o_pp = cv.take(sizeof(double) * (size_t)pgrid * 3 * n_e);
    const size_t o_bp = cv.take(sizeof(double) * (bparts_max + 1) * tsz);
    const size_t o_small = cv.take(sizeof(double) * 16);
    const size_t o_wt = cv.take(sizeof(double) * n_k), o_dd = cv.take(sizeof(double) * 3 * n_k);
    const size_t o_p = cv.take(sizeof(double) * 3 * n_k), o_b = cv.take(sizeof(double) * tsz);
    const size_t o_e2 = cv.take(hip_e2_scratch_bytes(nodes, n_k));
    const size_t o_pm = cv.take(s_pass_scratch(R0, k_edges, n_k, sizeof(T) == 4));
    hip_status hs = ws.reserve(cv.total, st);
    if (hs != HIP_OK) return hs;
    char *b = (char *)ws.base;
    cudaError_t e;
#define HIP_CK(call, what)                                                                                           \
    do {                                                                                                             \
        if ((e = (call)) != cudaSuccess) {                                                                           \
            set_err(what, e);                                                                                        \
            return HIP_ERR_CUDA;                                                                                     \
        }                                                                                                            \
    } while (0)
    const float *dposp = pos, *dwp = w;
    if (!dpos) {
        HIP_CK(cudaMemcpyAsync(b + o_pos, pos, sizeof(float) * 3 * N, cudaMemcpyHostToDevice, st), "H2D positions");
        dposp = (const float *)(b + o_pos);
    }
    if (w && !dw) {
        HIP_CK(cudaMemcpyAsync(b + o_w, w, sizeof(float) * N, cudaMemcpyHostToDevice, st), "H2D weights");
        dwp = (const float *)(b + o_w);
    }
    double *small = (double *)(b + o_small);
    double *S1 = small, *S1b = small + 1;
    unsigned long long *npairs = (unsigned long long *)(small + 2);  // [0]: P pass; [1], [2]: B pass
    int *err = (int *)(small + 5), *err2 = err + 1;
    int *counter = (int *)(small + 6), *bcounter = counter + 1, *hcounter = counter + 2;
    T *dx = (T *)(b + o_dx), *dy = (T *)(b + o_dy), *dz = (T *)(b + o_dz);
    int *dstart = (int *)(b + o_ds);
    HIP_CK(hip_build_cells<T>(dposp, dwp, N, L, n_c, dx, dy, dz, (float *)(b + o_dw), (int *)(b + o_didx),
                              (int *)(b + o_dcid), dstart, (int *)(b + o_df), S1, err, st),
           "cell build (R0)");
    HIP_CK(hip_build_cells<float>(dposp, dwp, N, L, n_c2, (float *)(b + o_x2), (float *)(b + o_y2),
                                  (float *)(b + o_z2), (float *)(b + o_w2), (int *)(b + o_i2), (int *)(b + o_c2),
                                  (int *)(b + o_s2), (int *)(b + o_f2), S1b, err2, st),
           "cell build (2 R0)");
    HIP_CK(hip_sorted_cells(dstart, n_cells, (int *)(b + o_dsc), st), "sorted cells");
    int herr[2] = {0, 0};
    HIP_CK(cudaMemcpyAsync(herr, err, 2 * sizeof(int), cudaMemcpyDeviceToHost, st), "D2H error word");
    HIP_CK(cudaStreamSynchronize(st), "cell build sync");
    if (herr[0] || herr[1]) return HIP_ERR_NONFINITE;

    CellList<T> dcl{dx, dy, dz, (const float *)(b + o_dw), (const int *)(b + o_didx), dstart, n_c, L, L / n_c};
    HIP_CK(cudaMemsetAsync(npairs, 0, 3 * sizeof(unsigned long long), st), "memset");
    HIP_CK(cudaMemsetAsync(counter, 0, 3 * sizeof(int), st), "memset");
    PowerKernelArgs ka;
    ka.n_e = n_e;
    ka.los = 2;
    ka.p0 = 0;
    ka.p1 = N;
    ka.n_items = n_cells * HIP_NSHIFT;
    ka.work_counter = counter;
    ka.partials = (double *)(b + o_pp);
    ka.npairs = npairs;
    double *Wt = (double *)(b + o_wt), *DD = (double *)(b + o_dd), *P = (double *)(b + o_p);
    HIP_CK(s_pass<T>(dcl, ka, k_edges, n_k, R0, L, S1, Wt, DD, P, b + o_pm, pgrid, st), "pair pass (S)");

    BispecArgs<T> ba;
    std::memset(&ba, 0, sizeof(ba));
    ba.data = dcl;
    ba.rand = dcl;  // no random primaries
    ba.n_cells = n_cells;
    ba.dcell = (const int *)(b + o_dsc);
    ba.rcell = (const int *)(b + o_dsc);
    ba.n_data = (int)N;
    ba.n_rand = 0;
    ba.n_e = n_e;
    ba.R0 = (T)R0;
    ba.rand_weight = T(0);
    ba.work_counter = bcounter;
    ba.partials = (double *)(b + o_bp);
    ba.npairs = npairs + 1;
    ba.dp0 = 0;
    ba.dp1 = N;
    ba.rp0 = 0;
    ba.rp1 = 0;
    for (int q = 0; q < HIP_BMAXE; ++q) {
        const double k = q < n_e ? k_edges[q] : 0.0;
        ba.k[q] = (T)k;
        ba.klo[q] = (T)(k - (double)ba.k[q]);
        ba.k3[q] = (T)(k * k * k);
        ba.jfac[q] = q + 1 < n_e ? (T)(3.0 / (k_edges[q + 1] * k_edges[q + 1] * k_edges[q + 1] - k * k * k)) : T(0);
    }
    int bgrid = 0;
    HIP_CK(hip_bispec_pairs<T>(ba, bparts_max, &bgrid, st), "bispectrum kernel");
    CellList<float> cl2{(const float *)(b + o_x2), (const float *)(b + o_y2), (const float *)(b + o_z2),
                        (const float *)(b + o_w2), (const int *)(b + o_i2), (const int *)(b + o_s2), n_c2, L,
                        L / n_c2};
    HIP_CK(hip_e2_term(cl2, n_cells2 * HIP_NSHIFT, hcounter, R0, L, k_edges, n_k, lmax, S1, nodes, b + o_e2,
                       ba.partials + (size_t)bgrid * tsz, nullptr, st),
           "DDR^II term");
    double *B = (double *)(b + o_b);
    HIP_CK(hip_bispec_finalize(ba.partials, bgrid + 1, n_k, lmax, L, S1, DD, Wt, B, st), "bispectrum finalize");
    const size_t nout = (size_t)(lmax + 1) * n_k * n_k;
    std::vector<double> hB(nout);
    unsigned long long hn[3] = {0, 0, 0};
    HIP_CK(cudaMemcpyAsync(hB.data(), B, sizeof(double) * nout, cudaMemcpyDeviceToHost, st), "D2H B");
    HIP_CK(cudaMemcpyAsync(hn, npairs, sizeof(hn), cudaMemcpyDeviceToHost, st), "D2H npairs");
    HIP_CK(cudaStreamSynchronize(st), "stream sync");
#undef HIP_CK
    std::memcpy(B_out, hB.data(), sizeof(double) * nout);
    if (npairs_out) npairs_out[0] = (int64_t)hn[1];
    return HIP_OK;
}

extern "C" hip_status hip_bispectrum_analytic(const float *pos, const float *w, int64_t N, double L, double R0,
                                              hip_window window, const double *k_edges, int n_k, int lmax,
                                              hip_precision prec, double *B_out, int64_t *npairs_out,
                                              void *cuda_stream)
{
    g_errbuf[0] = 0;
    if (!pos || !B_out) return HIP_ERR_ARG;
    if (N < 2 || N > 2000000000LL) return HIP_ERR_ARG;
    if (window != HIP_WINDOW_PHILCOX) return HIP_ERR_ARG;
    if (prec != HIP_PREC_FP64 && prec != HIP_PREC_MIXED) return HIP_ERR_ARG;
    if (lmax < 0 || lmax > HIP_LMAX) return HIP_ERR_ARG;
    if (!(L > 0.0) || !std::isfinite(L) || !(R0 > 0.0) || !(R0 < 0.25 * L)) return HIP_ERR_RANGE;
    hip_status hs = hip_check_edges(k_edges, n_k);
    if (hs != HIP_OK) return hs;
    if (n_k > (prec == HIP_PREC_MIXED ? HIP_BMAXE - 2 : 31)) return HIP_ERR_RANGE;
    std::lock_guard<std::mutex> lk(hip_api_mutex());
    int dev = 0;
    if ((hs = hip_device_setup(&dev)) != HIP_OK) return hs;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if (prec == HIP_PREC_MIXED)
        return bispec_analytic_impl<float>(pos, w, N, L, R0, k_edges, n_k, lmax, B_out, npairs_out, st, dev);
    return bispec_analytic_impl<double>(pos, w, N, L, R0, k_edges, n_k, lmax, B_out, npairs_out, st, dev);
}

extern "C" hip_status hip_bispectrum_partial(const float *pos, const float *w, int64_t N, const float *rand_pos,
                                             int64_t N_r, double L, double R0, hip_window window,
                                             const double *k_edges, int n_k, int lmax, hip_precision prec,
                                             const int64_t *prim_ranges, double *T_out, int64_t *npairs_out,
                                             void *cuda_stream)
{
    g_errbuf[0] = 0;
    if (!pos || !rand_pos || !T_out || !prim_ranges) return HIP_ERR_ARG;
    if (N < 1 || N > 2000000000LL || N_r < 1 || N_r > 2000000000LL) return HIP_ERR_ARG;
    if (window != HIP_WINDOW_PHILCOX) return HIP_ERR_ARG;
    if (prec != HIP_PREC_FP64 && prec != HIP_PREC_MIXED) return HIP_ERR_ARG;
    if (lmax < 0 || lmax > HIP_LMAX) return HIP_ERR_ARG;
    if (!(L > 0.0) || !std::isfinite(L) || !(R0 > 0.0) || !(R0 < 0.5 * L)) return HIP_ERR_RANGE;
    if (prim_ranges[0] < 0 || prim_ranges[1] > N || prim_ranges[0] > prim_ranges[1] || prim_ranges[2] < 0 ||
        prim_ranges[3] > N_r || prim_ranges[2] > prim_ranges[3])
        return HIP_ERR_RANGE;
    hip_status hs = hip_check_edges(k_edges, n_k);
    if (hs != HIP_OK) return hs;
    if (n_k > (prec == HIP_PREC_MIXED ? HIP_BMAXE - 2 : 31)) return HIP_ERR_RANGE;
    std::lock_guard<std::mutex> lk(hip_api_mutex());
    int dev = 0;
    if ((hs = hip_device_setup(&dev)) != HIP_OK) return hs;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if (prec == HIP_PREC_MIXED)
        return bispec_impl<float>(pos, w, N, rand_pos, N_r, L, R0, k_edges, n_k, lmax, T_out, npairs_out, st, dev,
                                  prim_ranges, true);
    return bispec_impl<double>(pos, w, N, rand_pos, N_r, L, R0, k_edges, n_k, lmax, T_out, npairs_out, st, dev,
                               prim_ranges, true);
}

// ------------------------------------------------------ host self-checks -----
// Evaluate the pair kernels' F_l(u) = D_l(u)/u^3 on the host with the same source
// and coefficient tables (FP32 path when prec == HIP_PREC_MIXED).  For tests.
extern "C" hip_status hip_window_omega(const double *k_edges, int n_k, double R0, int lmax, const double *p, int n_p,
                                       double *omega_out, void *cuda_stream)
{
    g_errbuf[0] = 0;
    if (!k_edges || !p || !omega_out || n_p < 1 || n_p > (1 << 20) || lmax < 0 || lmax > HIP_LMAX) return HIP_ERR_ARG;
    if (!(R0 > 0.0) || !std::isfinite(R0)) return HIP_ERR_RANGE;
    hip_status hs = hip_check_edges(k_edges, n_k);
    if (hs != HIP_OK) return hs;
    for (int q = 0; q < n_p; ++q)
        if (!(p[q] >= 0.0) || !std::isfinite(p[q])) return HIP_ERR_RANGE;
    std::lock_guard<std::mutex> lk(hip_api_mutex());
    int dev = 0;
    if ((hs = hip_device_setup(&dev)) != HIP_OK) return hs;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    Workspace &ws = g_ws[dev];
    if ((hs = ws.reserve(hip_omega_scratch_bytes(k_edges, n_k, R0, p, n_p), st)) != HIP_OK) return hs;
    cudaError_t e = hip_omega_eval(k_edges, n_k, R0, lmax, p, n_p, ws.base, omega_out, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        set_err("window omega", e);
        return HIP_ERR_CUDA;
    }
    return HIP_OK;
}

extern "C" double hip_debug_F(int prec, int l, double u)
{
    if (l < 0 || l > HIP_LMAX) return NAN;
    const HipCoeffs &C = hip_host_coeffs();
    if (prec == HIP_PREC_MIXED) {
        double F[5] = {0, 0, 0, 0, 0};
        hip_F_f32_total<31>((float)u, C, F);
        return F[l];
    }
    double F[5] = {0, 0, 0, 0, 0};
    hip_F_f64<31>(u, C, F);
    return F[l];
}

// D_l(u) = u^3 F_l(u) as the FP32 pair kernels evaluate it (host build of the
// same code): variant 0 = series, 1 = closed form with fitted Si auxiliaries,
// 2 = closed form with asymptotic auxiliaries.
extern "C" double hip_debug_D(int variant, int l, double u)
{
    if (l < 0 || l > HIP_LMAX || variant < 0 || variant > 2) return NAN;
    const HipCoeffs &C = hip_host_coeffs();
    const float uf = (float)u;
    float D[5] = {0, 0, 0, 0, 0};
    if (variant == 0) {
        hip_D_f32_series<31>(uf, C, D);
    } else {
        const float s = (float)std::sin((double)uf), c = (float)std::cos((double)uf);
        if (variant == 1)
            hip_D_f32_closed<31, false>(uf, 1.0f / uf, s, c, C, D);
        else
            hip_D_f32_closed<31, true>(uf, 1.0f / uf, s, c, C, D);
    }
    return (double)D[l];
}

// Vector form of hip_debug_F: out[i] = F_l(u[i]).
extern "C" void hip_debug_F_array(int prec, int l, const double *u, double *out, int64_t n)
{
    for (int64_t i = 0; i < n; ++i) out[i] = hip_debug_F(prec, l, u[i]);
}

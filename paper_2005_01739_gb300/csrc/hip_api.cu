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
            (e = hip_upload_coeffs_e2()) != cudaSuccess || (e = hip_upload_aniso_tables()) != cudaSuccess) {
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
    if (n > HIP_MAX_CELLS_SIDE) n = HIP_MAX_CELLS_SIDE;
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
    ka.n_part = N;
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

// ------------------------------------------------ hip_power_from_pairs ----
extern "C" hip_status hip_power_from_pairs(const double *DD, int n_k, int ell_max, double L, double R0,
                                           hip_window window, const double *k_edges, double S1, double *P_out,
                                           void *cuda_stream)
{
    g_errbuf[0] = 0;
    if (!DD || !P_out) return HIP_ERR_ARG;
    if (window != HIP_WINDOW_PHILCOX) return HIP_ERR_ARG;
    if (ell_max != 0 && ell_max != 2 && ell_max != 4) return HIP_ERR_ARG;
    if (!(L > 0.0) || !std::isfinite(L) || !(R0 > 0.0) || !(R0 < 0.5 * L)) return HIP_ERR_RANGE;
    if (!std::isfinite(S1) || S1 == 0.0) return HIP_ERR_RANGE;
    hip_status hs = hip_check_edges(k_edges, n_k);
    if (hs != HIP_OK) return hs;
    const int n_ell = ell_max / 2 + 1;
    for (int i = 0; i < n_ell * n_k; ++i)
        if (!std::isfinite(DD[i])) return HIP_ERR_NONFINITE;
    std::lock_guard<std::mutex> lk(hip_api_mutex());
    int dev = 0;
    if ((hs = hip_device_setup(&dev)) != HIP_OK) return hs;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    Workspace &ws = hip_workspace(dev);
    Carve cv;
    const size_t o_dd = cv.take(sizeof(double) * n_ell * n_k), o_wt = cv.take(sizeof(double) * n_k);
    const size_t o_p = cv.take(sizeof(double) * n_ell * n_k);
    if ((hs = ws.reserve(cv.total, st)) != HIP_OK) return hs;
    char *b = (char *)ws.base;
    cudaError_t e;
#define HIP_CK(call, what)                                                                                           \
    do {                                                                                                             \
        if ((e = (call)) != cudaSuccess) {                                                                           \
            set_err(what, e);                                                                                        \
            return HIP_ERR_CUDA;                                                                                     \
        }                                                                                                            \
    } while (0)
    HIP_CK(cudaMemcpyAsync(b + o_dd, DD, sizeof(double) * n_ell * n_k, cudaMemcpyHostToDevice, st), "H2D DD");
    HIP_CK(hip_window_transform(n_k + 1, k_edges, R0, (double *)(b + o_wt), st), "window transform");
    HIP_CK(hip_power_from_dd((const double *)(b + o_dd), n_k, n_ell, L, S1, (const double *)(b + o_wt),
                             (double *)(b + o_p), st),
           "finalize");
    HIP_CK(cudaMemcpyAsync(P_out, b + o_p, sizeof(double) * n_ell * n_k, cudaMemcpyDeviceToHost, st), "D2H P");
    HIP_CK(cudaStreamSynchronize(st), "stream sync");
#undef HIP_CK
    return HIP_OK;
}

// ------------------------------------------------ the bispectrum primary sum ----
// Scratch plan of the B pass for catalogs whose largest n_k, n_cc are nk_max,
// ncc_max and whose primaries (data then randoms, catalogs end to end) number
// `total`.  Primaries go through the a_lm pass and the contraction in chunks of
// at most `chunk` primaries, so X stays within HIP_BK_XBUDGET bytes.
#define HIP_BK_XBUDGET ((size_t)8 << 30)  // a few percent of the 288 GB of HBM
static int g_bk_tc_grid_cap = 0;  // tests: caps the contraction's CTAs (0 = one per SM)
static int g_bk_chunk_cap = 0;    // tests: caps the primaries per chunk (0 = by the X budget)
static int g_bk_fold = 0;         // tests: primaries between the contraction's FP64 folds (0 = default)
static int g_bk_cores = 0;        // tests: contract FP32 accumulators on the CUDA cores in FP64

// Stage timing of the last bispectrum primary sum (when profiling is on): the
// a_lm passes, the contractions and the C terms, summed over chunks, in ms, and
// the number of chunks.
static double g_bk_ms[4];
static bool g_bk_ms_valid = false;

extern "C" int hip_bispectrum_stage_times(double *ms, int n)
{
    if (!g_bk_ms_valid || !ms) return 0;
    const int m = n < 4 ? n : 4;
    for (int i = 0; i < m; ++i) ms[i] = g_bk_ms[i];
    return m;
}

struct BkPlan {
    int nc = 0, nk_max = 0, ncc_max = 0;
    long long chunk = 0;
    size_t o_cats = 0, o_spans = 0, o_segs = 0, o_X = 0, o_sp = 0, o_slots = 0, o_cc = 0, o_cnt = 0;
    size_t slots_bytes = 0;
    bool tc = false;  // contraction on the tensor cores
};

template <typename T>
static BkPlan bk_plan(Carve &cv, int nc, int nk_max, int ncc_max, long long total, size_t cc_bytes)
{
    BkPlan pl;
    pl.nc = nc;
    pl.nk_max = nk_max;
    pl.ncc_max = ncc_max;
    const size_t per = sizeof(T) * HIP_NLM * (size_t)nk_max;
    long long ch = (long long)(HIP_BK_XBUDGET / per);
    if (g_bk_chunk_cap > 0 && ch > g_bk_chunk_cap) ch = g_bk_chunk_cap;
    ch = (ch / 8) * 8;
    if (ch < 8) ch = 8;
    const long long tot8 = ((total + 7) / 8) * 8;
    pl.chunk = ch < tot8 ? ch : tot8;
    pl.o_cats = cv.take(sizeof(BkCat<T>) * nc);
    pl.o_spans = cv.take(sizeof(BkSpan) * (nc + 1));
    pl.o_segs = cv.take(sizeof(BkSeg) * (nc + 1));
    pl.o_X = cv.take(per * (size_t)pl.chunk + sizeof(T) * 64 * (size_t)(nc + 1));
    pl.o_sp = cv.take(sizeof(T) * ((size_t)pl.chunk + 8 * (size_t)(nc + 1)));
    pl.slots_bytes = hip_bk_alm_slot_bytes<T>(ncc_max);
    pl.o_slots = cv.take(pl.slots_bytes);
    pl.tc = sizeof(T) == 4 && hip_bk_tc_supported(nk_max);
    pl.o_cc = cv.take(cc_bytes);
    pl.o_cnt = cv.take(sizeof(int) * 4);
    return pl;
}

// Per catalog of the B pass (host side).
struct BkHostCat {
    long long n_prim;      // data + random primaries
    int n_k, n_cc;
    double R0;
    const double *k_edges;  // host
    double *cmom;           // device [n_cc][32]
    double *acc;            // device [5][n_k][n_k], zeroed by bk_run
    long long n_data;       // the data primaries (first in the primary order)
    double *S;              // device [n_S][n_k]: S^a_l from the data primaries' A^a_l0 (zeroed by bk_run), or null
    int n_S = 1;            // 1 (l = 0) or 3 (l = 0, 2, 4)
    double *G = nullptr;    // anisotropic: device [HIP_ANISO_NBLK][n_k][n_k] Gram blocks (zeroed by bk_run)
    double *Tc = nullptr;   // anisotropic: device [18][n_k][n_k] primary sums (written by bk_run)
};

// The primary sum T of every catalog into its acc: the a_lm pass and the
// contraction chunk by chunk, then the C term of each catalog.  `cats` holds the
// device descriptors' host copies (complete but for cmom, which bk_run fills).
template <typename T>
static hip_status bk_run(std::vector<BkCat<T>> &cats, const std::vector<BkHostCat> &hc, const BkPlan &pl, char *b,
                         cudaStream_t st)
{
    cudaError_t e;
#define HIP_CK(call, what)                                                                                           \
    do {                                                                                                             \
        if ((e = (call)) != cudaSuccess) {                                                                           \
            set_err(what, e);                                                                                        \
            return HIP_ERR_CUDA;                                                                                     \
        }                                                                                                            \
    } while (0)
    const int nc = pl.nc;
    BkCat<T> *dcats = (BkCat<T> *)(b + pl.o_cats);
    BkSpan *dspans = (BkSpan *)(b + pl.o_spans);
    BkSeg *dsegs = (BkSeg *)(b + pl.o_segs);
    T *X = (T *)(b + pl.o_X);
    T *sp = (T *)(b + pl.o_sp);
    double *slots = (double *)(b + pl.o_slots);
    int *cnt = (int *)(b + pl.o_cnt);  // [0] work counter, [1] status
    bool want_s = false;
    for (int i = 0; i < nc; ++i) {
        const int nL = hc[i].G ? 3 : 1;
        HIP_CK(cudaMemsetAsync(hc[i].cmom, 0, sizeof(double) * nL * hc[i].n_cc * HIP_BK_NM, st), "memset");
        if (hc[i].G)
            HIP_CK(cudaMemsetAsync(hc[i].G, 0, sizeof(double) * HIP_ANISO_NBLK * hc[i].n_k * hc[i].n_k, st),
                   "memset");
        else
            HIP_CK(cudaMemsetAsync(hc[i].acc, 0, sizeof(double) * (HIP_LMAX + 1) * hc[i].n_k * hc[i].n_k, st),
                   "memset");
        if (hc[i].S) {
            HIP_CK(cudaMemsetAsync(hc[i].S, 0, sizeof(double) * hc[i].n_S * hc[i].n_k, st), "memset");
            want_s = true;
        }
    }
    HIP_CK(cudaMemsetAsync(slots, 0, pl.slots_bytes, st), "memset");
    HIP_CK(cudaMemsetAsync(cnt, 0, sizeof(int) * 4, st), "memset");
    HIP_CK(cudaMemcpyAsync(dcats, cats.data(), sizeof(BkCat<T>) * nc, cudaMemcpyHostToDevice, st), "H2D catalogs");
    const int P = hip_bk_tc_stage_prims(pl.nk_max);
    // optional event pairs around the stages: [chunk][a_lm, contraction], then the C terms
    std::vector<cudaEvent_t> evs;
    auto mark = [&]() {
        if (!g_prof) return;
        cudaEvent_t ev;
        cudaEventCreate(&ev);
        cudaEventRecord(ev, st);
        evs.push_back(ev);
    };
    g_bk_ms_valid = false;
    int n_chunks = 0;
    // walk the catalogs' primaries end to end, one chunk at a time
    int ci = 0;
    long long gi = 0;  // next primary of catalog ci
    while (ci < nc) {
        std::vector<BkSpan> spans;
        std::vector<BkSeg> segs;
        long long used = 0, x_off = 0, sp_off = 0;
        int items = 0, stages = 0;
        while (ci < nc && used < pl.chunk) {
            const long long take = std::min(hc[ci].n_prim - gi, pl.chunk - used);
            if (take > 0) {
                BkSpan s;
                s.cat = ci;
                s.g0 = (int)gi;
                s.g1 = (int)(gi + take);
                s.item_begin = items;
                items += (int)((take + HIP_BK_PRIM - 1) / HIP_BK_PRIM);
                s.item_end = items;
                s.x_off = x_off;
                s.sp_off = sp_off;
                spans.push_back(s);
                BkSeg g;
                g.X = X + x_off;
                g.sp = sp + sp_off;
                g.n_p = (int)take;
                g.n_k = hc[ci].n_k;
                g.stage_begin = stages;
                stages += (int)((take + P - 1) / P);
                g.stage_end = stages;
                g.acc = hc[ci].G ? hc[ci].G : hc[ci].acc;
                g.n_d = (int)std::max(0LL, std::min(hc[ci].n_data - gi, take));
                g.S = hc[ci].S;
                g.n_S = hc[ci].n_S;
                segs.push_back(g);
                x_off += ((take * HIP_NLM * hc[ci].n_k + 63) / 64) * 64;
                sp_off += ((take + 7) / 8) * 8;
                used += take;
                gi += take;
            }
            if (gi >= hc[ci].n_prim) {
                ++ci;
                gi = 0;
            }
        }
        if (spans.empty()) break;
        HIP_CK(cudaMemcpyAsync(dspans, spans.data(), sizeof(BkSpan) * spans.size(), cudaMemcpyHostToDevice, st),
               "H2D spans");
        HIP_CK(cudaMemcpyAsync(dsegs, segs.data(), sizeof(BkSeg) * segs.size(), cudaMemcpyHostToDevice, st),
               "H2D segments");
        HIP_CK(cudaMemsetAsync(cnt, 0, sizeof(int), st), "memset");
        ++n_chunks;
        mark();
        HIP_CK(hip_bk_alm<T>(dcats, dspans, (int)spans.size(), items, pl.nk_max, pl.ncc_max, X, sp, slots, cnt, st),
               "bispectrum a_lm pass");
        mark();
        if (hc[0].G)  // anisotropic: the matching-m Gram blocks (every catalog of the call is anisotropic)
            HIP_CK(hip_bk_aniso_gram(dsegs, (int)segs.size(), pl.nk_max, used, st), "anisotropic Gram");
        else if (pl.tc && !g_bk_cores)
            HIP_CK(hip_bk_contract_tc(dsegs, (int)segs.size(), stages, pl.nk_max, cnt + 1, g_bk_tc_grid_cap, g_bk_fold,
                                      st),
                   "bispectrum contraction (tensor cores)");
        else
            HIP_CK(hip_bk_contract_f64<T>(dsegs, (int)segs.size(), used, pl.nk_max, st), "bispectrum contraction");
        if (want_s) HIP_CK(hip_bk_s_sum<T>(dsegs, (int)segs.size(), pl.nk_max, st), "bispectrum S sum");
        mark();
    }
    mark();
    for (int i = 0; i < nc; ++i) {
        BkCTerm c;
        std::memset(&c, 0, sizeof(c));
        for (int q = 0; q <= hc[i].n_k; ++q) c.k[q] = hc[i].k_edges[q];
        c.R0 = hc[i].R0;
        c.n_e = hc[i].n_k + 1;
        c.n_cc = hc[i].n_cc;
        c.cmom = hc[i].cmom;
        c.acc = hc[i].acc;
        if (hc[i].G) {
            HIP_CK(hip_bk_aniso_assemble(hc[i].G, hc[i].n_k, hc[i].Tc, st), "anisotropic assembly");
            HIP_CK(hip_bk_cterm_aniso(c, hip_aniso_tables().ct, b + pl.o_cc, hc[i].Tc, st), "anisotropic C term");
        } else {
            HIP_CK(hip_bk_cterm(c, b + pl.o_cc, st), "bispectrum C term");
        }
    }
    int status = 0;
    HIP_CK(cudaMemcpyAsync(&status, cnt + 1, sizeof(int), cudaMemcpyDeviceToHost, st), "D2H status");
    mark();
    HIP_CK(cudaStreamSynchronize(st), "bispectrum sync");
#undef HIP_CK
    if (g_prof && (int)evs.size() == 3 * n_chunks + 2) {
        for (double &v : g_bk_ms) v = 0.0;
        for (int c = 0; c < n_chunks; ++c) {
            float a = 0.f, k = 0.f;
            cudaEventElapsedTime(&a, evs[3 * c], evs[3 * c + 1]);
            cudaEventElapsedTime(&k, evs[3 * c + 1], evs[3 * c + 2]);
            g_bk_ms[0] += a;
            g_bk_ms[1] += k;
        }
        float ct = 0.f;
        cudaEventElapsedTime(&ct, evs[3 * n_chunks], evs[3 * n_chunks + 1]);
        g_bk_ms[2] = ct;
        g_bk_ms[3] = n_chunks;
        g_bk_ms_valid = true;
    }
    for (cudaEvent_t ev : evs) cudaEventDestroy(ev);
    if (status) {
        std::snprintf(g_errbuf, sizeof(g_errbuf), "bispectrum contraction: a bounded device wait gave up");
        return HIP_ERR_TIMEOUT;
    }
    return HIP_OK;
}

// Host copy of one catalog's a_lm-pass descriptor.
template <typename T>
static BkCat<T> bk_cat(const CellList<T> &dcl, const CellList<T> &rcl, const int *dcell, const int *rcell,
                       int64_t N, int64_t N_r, const int64_t *ranges, const double *k_edges, int n_k, double R0,
                       double rand_weight, unsigned long long *npairs, double *cmom)
{
    BkCat<T> a;
    std::memset(&a, 0, sizeof(a));
    a.data = dcl;
    a.rand = rcl;
    a.dcell = dcell;
    a.rcell = rcell;
    a.n_data = (int)N;
    a.n_rand = (int)N_r;
    a.dp0 = ranges ? ranges[0] : 0;
    a.dp1 = ranges ? ranges[1] : N;
    a.rp0 = ranges ? ranges[2] : 0;
    a.rp1 = ranges ? ranges[3] : N_r;
    a.n_e = n_k + 1;
    a.n_cc = hip_bk_intervals(R0, k_edges[n_k]);
    a.n_L = 1;
    a.R0 = (T)R0;
    a.rand_weight = (T)rand_weight;
    a.cc_scale = (T)(a.n_cc / R0);
    a.cc_lo = (T)(a.n_cc / R0 - (double)a.cc_scale);
    a.iR = (T)(1.0 / R0);
    a.iR_lo = (T)(1.0 / R0 - (double)a.iR);
    a.cmom = cmom;
    a.npairs = npairs;
    for (int q = 0; q < HIP_BMAXE; ++q) {
        const double k = q <= n_k ? k_edges[q] : 0.0;
        a.k[q] = (T)k;
        a.klo[q] = (T)(k - (double)a.k[q]);
        a.k3[q] = (T)(k * k * k);
        a.jfac[q] = q < n_k ? (T)(3.0 / (k_edges[q + 1] * k_edges[q + 1] * k_edges[q + 1] - k * k * k)) : T(0);
    }
    return a;
}

extern "C" void hip_debug_bk_caps(int tc_grid_cap, int chunk_cap)
{
    g_bk_tc_grid_cap = tc_grid_cap > 0 ? tc_grid_cap : 0;
    g_bk_chunk_cap = chunk_cap > 0 ? chunk_cap : 0;
}

extern "C" void hip_debug_bk_mode(int contract_on_cores, int fold_prims)
{
    g_bk_cores = contract_on_cores != 0;
    g_bk_fold = fold_prims > 0 ? fold_prims : 0;
}

template <typename T>
static hip_status bispec_impl(const float *pos, const float *w, int64_t N, const float *rpos, int64_t N_r, double L,
                              double R0, const double *k_edges, int n_k, int lmax, double *B_out,
                              int64_t *npairs_out, cudaStream_t st, int dev, const int64_t *ranges, bool partial,
                              bool aniso = false)
{
    Workspace &ws = hip_workspace(dev);
    const int n_c = hip_cells_per_side(L, R0);
    const int n_cells = n_c * n_c * n_c;
    const int n_e = n_k + 1;
    const bool dpos = hip_is_device_ptr(pos), dw = w && hip_is_device_ptr(w), drp = hip_is_device_ptr(rpos);
    const size_t tsz = (size_t)(aniso ? HIP_ANISO_NCOMB : HIP_LMAX + 1) * n_k * n_k;
    const int n_cc = hip_bk_intervals(R0, k_edges[n_k]);
    const int n_L = aniso ? 3 : 1;  // C-moment sets (L_0, L_2, L_4 of mu for the anisotropic bispectrum)

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
    const size_t o_acc = cv.take(sizeof(double) * tsz);
    const size_t o_cmom = cv.take(sizeof(double) * n_L * n_cc * HIP_BK_NM);
    const size_t o_small = cv.take(sizeof(double) * 16);
    const size_t o_wt = cv.take(sizeof(double) * n_k), o_dd = cv.take(sizeof(double) * 3 * n_k);
    const size_t o_p = cv.take(sizeof(double) * 3 * n_k), o_b = cv.take(sizeof(double) * tsz);
    const size_t o_G = aniso ? cv.take(sizeof(double) * HIP_ANISO_NBLK * n_k * n_k) : 0;
    const BkPlan pl = bk_plan<T>(cv, 1, n_k, n_L * n_cc, N + N_r,
                                 aniso ? hip_bk_cterm_aniso_scratch_bytes(n_cc, n_k)
                                       : hip_bk_cterm_scratch_bytes(n_cc, n_k));
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
    int *counter = (int *)(small + 6);
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
    double *Wt = (double *)(b + o_wt), *DD = (double *)(b + o_dd), *P = (double *)(b + o_p);
    (void)P;
    // S^a (the l = 0 data pair sum) comes from the a_lm pass (hip_bk_s_sum); W~^a here
    if (!partial) HIP_CK(hip_window_transform(n_e, k_edges, R0, Wt, st), "window transform");
    std::vector<BkCat<T>> cats(1, bk_cat<T>(dcl, rcl, (const int *)(b + o_dsc), (const int *)(b + o_rsc), N, N_r,
                                            ranges, k_edges, n_k, R0, -hS1 / (double)N_r, npairs + 1,
                                            (double *)(b + o_cmom)));
    cats[0].n_L = n_L;
    std::vector<BkHostCat> hc(1);
    hc[0] = BkHostCat{N + N_r, n_k, n_cc, R0, k_edges, (double *)(b + o_cmom), (double *)(b + o_acc), N,
                      partial ? nullptr : DD};
    if (aniso) {
        hc[0].n_S = 3;  // DD^a_l, l = 0, 2, 4, about zhat
        hc[0].G = (double *)(b + o_G);
        hc[0].Tc = (double *)(b + o_acc);
    }
    if ((hs = bk_run<T>(cats, hc, pl, b, st)) != HIP_OK) return hs;
    double *acc = (double *)(b + o_acc);
    double *B = (double *)(b + o_b);
    if (aniso)
        HIP_CK(hip_bk_aniso_finalize(acc, DD, Wt, S1, n_k, L, B, st), "anisotropic finalize");
    else if (partial)
        HIP_CK(hip_bispec_sum(acc, 1, n_k, lmax, B, st), "bispectrum sum");
    else
        HIP_CK(hip_bispec_finalize(acc, 1, n_k, lmax, L, S1, DD, Wt, B, st), "bispectrum finalize");
    const size_t nout = aniso ? tsz : (size_t)(lmax + 1) * n_k * n_k;
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

// hip_bispectrum with its random catalog generated on the device from a seed
// (hip_uniform_randoms' mapping) into a buffer the library keeps per device and
// grows on demand; calls through this entry point are serialised on the host.
extern "C" hip_status hip_bispectrum_seeded(const float *pos, const float *w, int64_t N, int64_t N_r,
                                            uint64_t rand_seed, double L, double R0, hip_window window,
                                            const double *k_edges, int n_k, int lmax, hip_precision prec,
                                            double *B_out, int64_t *npairs_out, void *cuda_stream)
{
    g_errbuf[0] = 0;
    if (N_r < 1 || N_r > 2000000000LL) return HIP_ERR_ARG;
    if (!(L > 0.0) || !std::isfinite(L)) return HIP_ERR_RANGE;
    static std::mutex mu;
    static float *buf[64] = {nullptr};
    static size_t cap[64] = {0};
    std::lock_guard<std::mutex> lk(mu);
    int dev = 0;
    {
        std::lock_guard<std::mutex> lk2(hip_api_mutex());
        hip_status hs = hip_device_setup(&dev);
        if (hs != HIP_OK) return hs;
    }
    if (dev < 0 || dev >= 64) return HIP_ERR_ARG;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const size_t need = sizeof(float) * 3 * (size_t)N_r;
    cudaError_t e = cudaSuccess;
    if (cap[dev] < need) {
        if (buf[dev]) {
            e = cudaStreamSynchronize(st);  // the previous call's launches have finished with the buffer
            if (e == cudaSuccess) e = cudaFree(buf[dev]);
            buf[dev] = nullptr;
            cap[dev] = 0;
        }
        if (e == cudaSuccess) e = cudaMalloc((void **)&buf[dev], need);
        if (e != cudaSuccess) {
            buf[dev] = nullptr;
            set_err("random catalog buffer", e);
            cudaGetLastError();
            return HIP_ERR_CUDA;
        }
        cap[dev] = need;
    }
    if ((e = hip_launch_uniform_randoms(buf[dev], N_r, L, rand_seed, st)) != cudaSuccess) {
        set_err("uniform randoms", e);
        cudaGetLastError();
        return HIP_ERR_CUDA;
    }
    return hip_bispectrum(pos, w, N, buf[dev], N_r, L, R0, window, k_edges, n_k, lmax, prec, B_out, npairs_out,
                          cuda_stream);
}

extern "C" hip_status hip_bispectrum_aniso(const float *pos, const float *w, int64_t N, const float *rand_pos,
                                           int64_t N_r, double L, double R0, hip_window window,
                                           const double *k_edges, int n_k, double *B_out, int64_t *npairs_out,
                                           void *cuda_stream)
{
    g_errbuf[0] = 0;
    if (!pos || !rand_pos || !B_out) return HIP_ERR_ARG;
    if (N < 1 || N > 2000000000LL || N_r < 1 || N_r > 2000000000LL) return HIP_ERR_ARG;
    if (window != HIP_WINDOW_PHILCOX) return HIP_ERR_ARG;
    if (!(L > 0.0) || !std::isfinite(L) || !(R0 > 0.0) || !(R0 < 0.5 * L)) return HIP_ERR_RANGE;
    hip_status hs = hip_check_edges(k_edges, n_k);
    if (hs != HIP_OK) return hs;
    if (n_k > HIP_BMAXE - 2 || hip_bk_intervals(R0, k_edges[n_k]) > HIP_ANISO_MAXCC) return HIP_ERR_RANGE;
    std::lock_guard<std::mutex> lk(hip_api_mutex());
    int dev = 0;
    if ((hs = hip_device_setup(&dev)) != HIP_OK) return hs;
    return bispec_impl<float>(pos, w, N, rand_pos, N_r, L, R0, k_edges, n_k, HIP_LMAX, B_out, npairs_out,
                              (cudaStream_t)cuda_stream, dev, nullptr, false, true);
}

// Batched bispectra: per catalog the buffers of bispec_impl (one workspace
// carve for all), one persistent bispectrum launch over every catalog's
// primaries, FP64 finalize per catalog.
template <typename T>
static hip_status bispec_batched_impl(const hip_bcatalog *cats, int nc, cudaStream_t st, int dev)
{
    Workspace &ws = hip_workspace(dev);
    struct Lay {
        int n_c, n_cells, n_k, n_e;
        bool dpos, dw, drp;
        size_t o_pos, o_w, o_rp, o_dx, o_dy, o_dz, o_dw, o_didx, o_dcid, o_rx, o_ry, o_rz, o_rw, o_ridx, o_rcid;
        size_t o_ds, o_df, o_dsc, o_rsc, o_rs, o_rf, o_small, o_wt, o_dd, o_p, o_b, o_acc, o_cmom;
        int n_cc;
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
        y.n_cc = hip_bk_intervals(c.R0, c.k_edges[c.n_k]);
        y.o_cmom = cv.take(sizeof(double) * y.n_cc * HIP_BK_NM);
    }
    int ncc_max = 1;
    size_t cc_bytes = 256;
    long long total = 0;
    for (int i = 0; i < nc; ++i) {
        ncc_max = std::max(ncc_max, lay[i].n_cc);
        cc_bytes = std::max(cc_bytes, hip_bk_cterm_scratch_bytes(lay[i].n_cc, lay[i].n_k));
        total += cats[i].N + cats[i].N_r;
    }
    const BkPlan pl = bk_plan<T>(cv, nc, nk_max, ncc_max, total, cc_bytes);
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
    // per catalog: W~^a, the a_lm-pass descriptor (S^a comes from the a_lm pass)
    std::vector<BkCat<T>> bcats(nc);
    std::vector<BkHostCat> hcs(nc);
    for (int i = 0; i < nc; ++i) {
        const hip_bcatalog &c = cats[i];
        const Lay &y = lay[i];
        double *small = (double *)(b + y.o_small);
        unsigned long long *npairs = (unsigned long long *)(small + 2);
        int *counter = (int *)(small + 6);
        HIP_CK(cudaMemsetAsync(npairs, 0, 3 * sizeof(unsigned long long), st), "memset");
        HIP_CK(cudaMemsetAsync(counter, 0, sizeof(int), st), "memset");
        // S^a comes from the a_lm pass (hip_bk_s_sum); W~^a here
        HIP_CK(hip_window_transform(y.n_e, c.k_edges, c.R0, (double *)(b + y.o_wt), st), "window transform");
        bcats[i] = bk_cat<T>(dcl[i], rcl[i], (const int *)(b + y.o_dsc), (const int *)(b + y.o_rsc), c.N, c.N_r,
                             nullptr, c.k_edges, c.n_k, c.R0, -hsm[(size_t)i * 6] / (double)c.N_r, npairs + 1,
                             (double *)(b + y.o_cmom));
        hcs[i] = BkHostCat{c.N + c.N_r, c.n_k, y.n_cc, c.R0, c.k_edges, (double *)(b + y.o_cmom),
                           (double *)(b + y.o_acc), c.N, (double *)(b + y.o_dd)};
    }
    if ((hs = bk_run<T>(bcats, hcs, pl, b, st)) != HIP_OK) return hs;
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
    const bool dpos = hip_is_device_ptr(pos), dw = w && hip_is_device_ptr(w);
    const size_t tsz = (size_t)(HIP_LMAX + 1) * n_k * n_k;
    const int n_cc = hip_bk_intervals(R0, k_edges[n_k]);
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
    const size_t o_acc = cv.take(sizeof(double) * 2 * tsz);  // [0] primary sum, [1] the E^II row
    const size_t o_cmom = cv.take(sizeof(double) * n_cc * HIP_BK_NM);
    const size_t o_small = cv.take(sizeof(double) * 16);
    const size_t o_wt = cv.take(sizeof(double) * n_k), o_dd = cv.take(sizeof(double) * 3 * n_k);
    const size_t o_p = cv.take(sizeof(double) * 3 * n_k), o_b = cv.take(sizeof(double) * tsz);
    const size_t o_e2 = cv.take(hip_e2_scratch_bytes(nodes, n_k));
    const BkPlan pl = bk_plan<T>(cv, 1, n_k, n_cc, N, hip_bk_cterm_scratch_bytes(n_cc, n_k));
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
    int *counter = (int *)(small + 6), *hcounter = counter + 2;
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
    double *Wt = (double *)(b + o_wt), *DD = (double *)(b + o_dd);
    // S^a comes from the a_lm pass (hip_bk_s_sum); W~^a here
    HIP_CK(hip_window_transform(n_e, k_edges, R0, Wt, st), "window transform");

    // the data primaries' sum (no random primaries)
    std::vector<BkCat<T>> cats(1, bk_cat<T>(dcl, dcl, (const int *)(b + o_dsc), (const int *)(b + o_dsc), N, 0,
                                            nullptr, k_edges, n_k, R0, 0.0, npairs + 1, (double *)(b + o_cmom)));
    std::vector<BkHostCat> hc(1);
    double *acc = (double *)(b + o_acc);
    hc[0] = BkHostCat{N, n_k, n_cc, R0, k_edges, (double *)(b + o_cmom), acc, N, DD};
    if ((hs = bk_run<T>(cats, hc, pl, b, st)) != HIP_OK) return hs;
    CellList<float> cl2{(const float *)(b + o_x2), (const float *)(b + o_y2), (const float *)(b + o_z2),
                        (const float *)(b + o_w2), (const int *)(b + o_i2), (const int *)(b + o_s2), n_c2, L,
                        L / n_c2};
    HIP_CK(hip_e2_term(cl2, n_cells2 * HIP_NSHIFT, hcounter, R0, L, k_edges, n_k, lmax, S1, nodes, b + o_e2,
                       acc + tsz, nullptr, st),
           "DDR^II term");
    double *B = (double *)(b + o_b);
    HIP_CK(hip_bispec_finalize(acc, 2, n_k, lmax, L, S1, DD, Wt, B, st), "bispectrum finalize");
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

// F_l(u) as the bispectrum's FP32 a_lm pass evaluates it (host build of the same code).
extern "C" double hip_debug_Fb(int l, double u)
{
    if (l < 0 || l > HIP_LMAX) return NAN;
    float F[5] = {0, 0, 0, 0, 0};
    hip_F_b32((float)u, hip_host_coeffs(), F);
    return (double)F[l];
}

// Vector form of hip_debug_F: out[i] = F_l(u[i]).
extern "C" void hip_debug_F_array(int prec, int l, const double *u, double *out, int64_t n)
{
    for (int64_t i = 0; i < n; ++i) out[i] = hip_debug_F(prec, l, u[i]);
}

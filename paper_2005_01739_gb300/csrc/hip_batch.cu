// Batched power spectra: many catalogs (each with its own N, L, R0, bins) in one
// persistent pair-kernel launch, with the cell builds, the pair pass and the
// FP64 finalize recorded once into a CUDA graph and replayed per run.  The pair
// pass is the Legendre-moment pass (hip_moments.cu) when every catalog has
// R0 k_max <= 1024, with the edge functions' coefficients computed once when
// the plan is built; otherwise the direct pass.
//
// A plan owns its device memory (sized for its catalogs at creation); the graph
// refers to fixed addresses in it.  Host-resident inputs are copied into the
// plan's staging area before each replay; device-resident inputs are read in
// place, so their current contents are used on every run.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <numeric>
#include <vector>

#include "hip_internal.h"
#include "hip_moments.h"
#include "hip_workspace.h"

std::mutex &hip_api_mutex();

namespace {

thread_local char g_batch_msg[256];

struct CatLayout {
    bool dev_pos = false, dev_w = false;
    int n_c = 1, n_cells = 1, n_e = 2, n_ell = 1, items = 0;
    size_t o_pos = 0, o_w = 0, o_x = 0, o_y = 0, o_z = 0, o_ws = 0, o_idx = 0, o_cid = 0, o_start = 0, o_fill = 0;
    size_t o_acc = 0, o_s1 = 0, o_np = 0, o_wt = 0, o_dd = 0, o_p = 0;
    int pm_nc = 0;  // moment intervals (moment pass)
    size_t o_ke = 0, o_coef = 0, o_mg = 0;
};

// Cells per side for a batched catalog: at least R0 wide, and no more cells
// than about one per `occ` particles (sparse catalogs otherwise spend their time
// on empty work items; occ = 0: cells R0 wide whatever the occupancy).  occ is
// the plan's tunable (hip_batch_plan_tune).
int batch_cells_per_side(const hip_catalog &c, int occ)
{
    int n = hip_cells_per_side(c.L, c.R0);
    if (occ <= 0) return n;
    const int by_occ = std::max(1, (int)std::floor(std::cbrt((double)c.N / (double)occ)));
    return std::max(1, std::min(n, by_occ));
}

hip_status check_catalog(const hip_catalog &c)
{
    if (!c.pos || !c.P_out) return HIP_ERR_ARG;
    if (c.N < 1 || c.N > 2000000000LL) return HIP_ERR_ARG;
    if (c.ell_max != 0 && c.ell_max != 2 && c.ell_max != 4) return HIP_ERR_ARG;
    if (c.los_axis < 0 || c.los_axis > 2) return HIP_ERR_ARG;
    if (!(c.L > 0.0) || !std::isfinite(c.L) || !(c.R0 > 0.0) || !(c.R0 < 0.5 * c.L)) return HIP_ERR_RANGE;
    if (c.prim_begin < 0 || c.prim_end > c.N || c.prim_begin > c.prim_end) return HIP_ERR_RANGE;
    return hip_check_edges(c.k_edges, c.n_k);
}

}  // namespace

struct hip_batch_plan {
    int dev = 0;
    hip_precision prec = HIP_PREC_MIXED;
    std::vector<hip_catalog> cats;
    std::vector<CatLayout> lay;
    void *buf = nullptr;
    double *h_out = nullptr;  // pinned: per catalog P, DD, npairs; then the error word
    size_t out_bytes = 0;
    std::vector<size_t> out_off;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t cap_stream = nullptr;
    int launches = 0;
    int occ = 64;   // target particles per cell (see batch_cells_per_side)
    int warps = 0;  // moment pass: warps per CTA (4 or 8; 0 = by the cell occupancy)
    int fold = 0;   // moment pass: pairs between folds of the FP32 sums (0 = the largest, 16384)
};

extern "C" const char *hip_batch_message(void) { return g_batch_msg; }

template <typename T>
static hip_status plan_build(hip_batch_plan *pl, cudaStream_t st)
{
    const int nc = (int)pl->cats.size();
    pl->lay.assign(nc, CatLayout());
    Carve cv;
    int nch = 1, nk_max = 1, items = 0;
    bool pm = true;  // every catalog within the moment pass's range
    for (int i = 0; i < nc; ++i)
        pm = pm && hip_pm_applicable(pl->cats[i].R0, pl->cats[i].k_edges[pl->cats[i].n_k], sizeof(T) == 4);
    // process the most expensive catalogs first (their items come first in the work list); the
    // direct pass costs per pair and edge, the moment pass per pair
    std::vector<int> order(nc);
    std::iota(order.begin(), order.end(), 0);
    std::vector<double> cost(nc);
    for (int i = 0; i < nc; ++i) {
        const hip_catalog &c = pl->cats[i];
        cost[i] = (double)c.N * (double)c.N / (c.L * c.L * c.L) * c.R0 * c.R0 * c.R0 * (pm ? 1.0 : c.n_k + 1.0);
    }
    int nc_max = 1, ne_max = 1;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
    for (int i = 0; i < nc; ++i) {
        const hip_catalog &c = pl->cats[i];
        CatLayout &L = pl->lay[i];
        L.dev_pos = hip_is_device_ptr(c.pos);
        L.dev_w = c.w && hip_is_device_ptr(c.w);
        L.n_c = batch_cells_per_side(c, pl->occ);
        L.n_cells = L.n_c * L.n_c * L.n_c;
        L.n_e = c.n_k + 1;
        L.n_ell = c.ell_max / 2 + 1;
        L.items = L.n_cells * HIP_NSHIFT;
        nch = std::max(nch, (L.n_e + 31) / 32);
        nk_max = std::max(nk_max, c.n_k);
        const size_t N = (size_t)c.N;
        if (!L.dev_pos) L.o_pos = cv.take(sizeof(float) * 3 * N);
        if (c.w && !L.dev_w) L.o_w = cv.take(sizeof(float) * N);
        L.o_x = cv.take(sizeof(T) * N);
        L.o_y = cv.take(sizeof(T) * N);
        L.o_z = cv.take(sizeof(T) * N);
        L.o_ws = cv.take(sizeof(float) * N);
        L.o_idx = cv.take(sizeof(int) * N);
        L.o_cid = cv.take(sizeof(int) * N);
        L.o_start = cv.take(sizeof(int) * (L.n_cells + 1));
        L.o_fill = cv.take(sizeof(int) * L.n_cells);
        L.o_acc = cv.take(sizeof(double) * 3 * L.n_e);
        L.o_s1 = cv.take(sizeof(double) * 2);
        L.o_np = cv.take(sizeof(unsigned long long));
        L.o_wt = cv.take(sizeof(double) * c.n_k);
        L.o_dd = cv.take(sizeof(double) * 3 * c.n_k);
        L.o_p = cv.take(sizeof(double) * 3 * c.n_k);
        if (pm) {
            L.pm_nc = hip_pm_intervals(c.R0, c.k_edges[c.n_k]);
            nc_max = std::max(nc_max, L.pm_nc);
            ne_max = std::max(ne_max, L.n_e);
            L.o_ke = cv.take(sizeof(double) * L.n_e);
            L.o_coef = cv.take(sizeof(double) * hip_pm_coef_doubles(L.n_e, L.pm_nc));
            L.o_mg = cv.take(sizeof(double) * hip_pm_mg_doubles(L.pm_nc));
        }
    }
    const size_t o_bc = cv.take(sizeof(BatchCat<T>) * nc), o_fc = cv.take(sizeof(FinalCat) * nc);
    const size_t o_pc = cv.take(sizeof(PmCat<T>) * nc), o_cc = cv.take(sizeof(PmContractCat) * nc);
    const size_t o_misc = cv.take(sizeof(int) * 4);
    cudaError_t e = cudaMalloc(&pl->buf, cv.total);
    if (e != cudaSuccess) {
        cudaGetLastError();
        std::snprintf(g_batch_msg, sizeof(g_batch_msg), "cudaMalloc(%zu): %s", cv.total, cudaGetErrorString(e));
        return HIP_ERR_NOMEM;
    }
    char *b = (char *)pl->buf;
    int *err = (int *)(b + o_misc), *counter = err + 1;
    // descriptors
    std::vector<BatchCat<T>> bc(nc);
    std::vector<FinalCat> fc(nc);
    std::vector<PmCat<T>> pc(nc);
    std::vector<PmContractCat> cc(nc);
    for (int oi = 0; oi < nc; ++oi) {
        const int i = order[oi];
        const hip_catalog &c = pl->cats[i];
        const CatLayout &L = pl->lay[i];
        BatchCat<T> &d = bc[oi];
        std::memset(&d, 0, sizeof(d));
        d.cl = CellList<T>{(T *)(b + L.o_x), (T *)(b + L.o_y), (T *)(b + L.o_z), (float *)(b + L.o_ws),
                           (int *)(b + L.o_idx), (int *)(b + L.o_start), L.n_c, c.L, c.L / L.n_c};
        d.p0 = c.prim_begin;
        d.p1 = c.prim_end;
        d.los = c.los_axis;
        d.n_e = L.n_e;
        d.R0 = (T)c.R0;
        const double dk = (c.k_edges[c.n_k] - c.k_edges[0]) / c.n_k;
        bool lin = true;
        for (int q = 0; q <= c.n_k; ++q)
            if (std::fabs(c.k_edges[q] - (c.k_edges[0] + q * dk)) >
                1e-12 * (std::fabs(c.k_edges[c.n_k]) + std::fabs(c.k_edges[0])))
                lin = false;
        d.lin = lin ? 1 : 0;
        const double d32 = 32.0 * dk;
        d.dk32hi = (T)d32;
        d.dk32lo = (T)(d32 - (double)d.dk32hi);
        for (int q = 0; q < HIP_MAX_EDGES; ++q) {
            const double k = q < L.n_e ? c.k_edges[q] : 0.0;
            d.k[q] = (T)k;
            d.klo[q] = (T)(k - (double)d.k[q]);
        }
        d.item_begin = items;
        items += L.items;
        d.item_end = items;
        d.acc = (double *)(b + L.o_acc);
        d.npairs = (unsigned long long *)(b + L.o_np);
        FinalCat &f = fc[oi];
        std::memset(&f, 0, sizeof(f));
        for (int q = 0; q < HIP_MAX_EDGES; ++q) f.k[q] = q < L.n_e ? c.k_edges[q] : 0.0;
        f.R0 = c.R0;
        f.L = c.L;
        f.n_e = L.n_e;
        f.n_ell = L.n_ell;
        f.acc = (double *)(b + L.o_acc);
        f.S1 = (double *)(b + L.o_s1);
        f.Wt = (double *)(b + L.o_wt);
        f.DD = (double *)(b + L.o_dd);
        f.P = (double *)(b + L.o_p);
        if (pm) {
            PmCat<T> &m = pc[oi];
            std::memset(&m, 0, sizeof(m));
            m.cl = d.cl;
            m.p0 = d.p0;
            m.p1 = d.p1;
            m.los = d.los;
            m.n_c = L.pm_nc;
            m.item_begin = d.item_begin;
            m.item_end = d.item_end;
            m.R0 = (T)c.R0;
            m.dc = (T)hip_pm_width(c.R0, L.pm_nc);
            m.n_part = c.N;
            m.Mg = (double *)(b + L.o_mg);
            m.npairs = d.npairs;
            PmContractCat &k = cc[oi];
            k.coef = (const double *)(b + L.o_coef);
            k.Mg = (const double *)(b + L.o_mg);
            k.n_e = L.n_e;
            k.n_c = L.pm_nc;
            k.n_ell = L.n_ell;
            k.row = d.acc;
        }
    }
    if ((e = cudaMemcpy(b + o_bc, bc.data(), sizeof(BatchCat<T>) * nc, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(b + o_fc, fc.data(), sizeof(FinalCat) * nc, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (pm && (e = cudaMemcpy(b + o_pc, pc.data(), sizeof(PmCat<T>) * nc, cudaMemcpyHostToDevice)) != cudaSuccess) ||
        (pm && (e = cudaMemcpy(b + o_cc, cc.data(), sizeof(PmContractCat) * nc, cudaMemcpyHostToDevice)) !=
                   cudaSuccess)) {
        std::snprintf(g_batch_msg, sizeof(g_batch_msg), "descriptor upload: %s", cudaGetErrorString(e));
        return HIP_ERR_CUDA;
    }
    // the moment pass's edge-function coefficients depend only on the bins and R0: once per plan
    for (int i = 0; pm && i < nc; ++i) {
        const hip_catalog &c = pl->cats[i];
        const CatLayout &L = pl->lay[i];
        if ((e = cudaMemcpy(b + L.o_ke, c.k_edges, sizeof(double) * L.n_e, cudaMemcpyHostToDevice)) != cudaSuccess ||
            (e = hip_pm_coeffs((const double *)(b + L.o_ke), L.n_e, L.n_ell, c.R0, c.k_edges[c.n_k],
                               (double *)(b + L.o_coef), nullptr)) != cudaSuccess ||
            (e = cudaDeviceSynchronize()) != cudaSuccess) {
            std::snprintf(g_batch_msg, sizeof(g_batch_msg), "moment coefficients: %s", cudaGetErrorString(e));
            return HIP_ERR_CUDA;
        }
    }
    // pinned host mirror of the outputs
    pl->out_off.assign(nc, 0);
    size_t ob = 0;
    for (int i = 0; i < nc; ++i) {
        pl->out_off[i] = ob;
        ob += 2 * (size_t)pl->lay[i].n_ell * pl->cats[i].n_k + 2;  // P, DD, npairs bits, error word
    }
    pl->out_bytes = sizeof(double) * ob;
    if ((e = cudaMallocHost((void **)&pl->h_out, pl->out_bytes)) != cudaSuccess) {
        cudaGetLastError();
        std::snprintf(g_batch_msg, sizeof(g_batch_msg), "cudaMallocHost: %s", cudaGetErrorString(e));
        return HIP_ERR_NOMEM;
    }
    const int grid = hip_power_grid<T>();

    // ---- record the graph, on a stream of our own (the legacy default stream,
    // which callers may pass, cannot be captured); runs replay it on the caller's.
    (void)st;
    cudaStream_t cst = nullptr;
    if ((e = cudaStreamCreateWithFlags(&cst, cudaStreamNonBlocking)) != cudaSuccess) {
        std::snprintf(g_batch_msg, sizeof(g_batch_msg), "stream: %s", cudaGetErrorString(e));
        return HIP_ERR_CUDA;
    }
    pl->cap_stream = cst;
    st = cst;
    if ((e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) {
        std::snprintf(g_batch_msg, sizeof(g_batch_msg), "begin capture: %s", cudaGetErrorString(e));
        return HIP_ERR_CUDA;
    }
    int launches = 0;
    cudaError_t ce = cudaMemsetAsync(err, 0, sizeof(int) * 4, st);  // the work counter
    for (int i = 0; i < nc && ce == cudaSuccess; ++i) {
        const hip_catalog &c = pl->cats[i];
        const CatLayout &L = pl->lay[i];
        const float *pos = L.dev_pos ? c.pos : (const float *)(b + L.o_pos);
        const float *w = c.w ? (L.dev_w ? c.w : (const float *)(b + L.o_w)) : nullptr;
        if ((ce = cudaMemsetAsync(b + L.o_acc, 0, sizeof(double) * 3 * L.n_e, st)) != cudaSuccess) break;
        if ((ce = cudaMemsetAsync(b + L.o_np, 0, sizeof(unsigned long long), st)) != cudaSuccess) break;
        if (pm && (ce = cudaMemsetAsync(b + L.o_mg, 0, sizeof(double) * hip_pm_mg_doubles(L.pm_nc), st)) !=
                      cudaSuccess)
            break;
        // each catalog has its own S1 and error word (the cell build clears both)
        ce = hip_build_cells<T>(pos, w, c.N, c.L, L.n_c, (T *)(b + L.o_x), (T *)(b + L.o_y), (T *)(b + L.o_z),
                                (float *)(b + L.o_ws), (int *)(b + L.o_idx), (int *)(b + L.o_cid),
                                (int *)(b + L.o_start), (int *)(b + L.o_fill), (double *)(b + L.o_s1),
                                (int *)(b + L.o_s1 + sizeof(double)), st);
        launches += 3;
    }
    if (pm) {
        // particles per cell, weighted by each catalog's share of the pairs
        double wsum = 0.0, psum = 0.0;
        for (int i = 0; i < nc; ++i) {
            const hip_catalog &c = pl->cats[i];
            const double cells = (double)pl->lay[i].n_c * pl->lay[i].n_c * pl->lay[i].n_c;
            const double pairs = (double)c.N * (double)c.N / (c.L * c.L * c.L) * c.R0 * c.R0 * c.R0;
            wsum += pairs;
            psum += pairs * (double)c.N / cells;
        }
        if (ce == cudaSuccess)
            ce = hip_power_moments_batched<T>((const PmCat<T> *)(b + o_pc), nc, items, nc_max, counter,
                                              (const PmContractCat *)(b + o_cc), ne_max,
                                              wsum > 0.0 ? psum / wsum : 0.0, pl->warps, pl->fold, st);
        launches += sizeof(T) == 4 ? 3 : 2;  // (sum |w|,) moments, contraction
    } else {
        if (ce == cudaSuccess)
            ce = hip_power_pairs_batched<T>((const BatchCat<T> *)(b + o_bc), nc, items, nch, counter, grid, st);
        launches += 1;
    }
    if (ce == cudaSuccess) ce = hip_power_finalize_batched((const FinalCat *)(b + o_fc), nc, nk_max, st);
    launches += 2;
    // copy the outputs and error words into the pinned host mirror
    for (int i = 0; i < nc && ce == cudaSuccess; ++i) {
        const CatLayout &L = pl->lay[i];
        const size_t n = (size_t)L.n_ell * pl->cats[i].n_k;
        double *dst = pl->h_out + pl->out_off[i];
        if ((ce = cudaMemcpyAsync(dst, b + L.o_p, sizeof(double) * n, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
            break;
        if ((ce = cudaMemcpyAsync(dst + n, b + L.o_dd, sizeof(double) * n, cudaMemcpyDeviceToHost, st)) !=
            cudaSuccess)
            break;
        if ((ce = cudaMemcpyAsync(dst + 2 * n, b + L.o_np, sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                                  st)) != cudaSuccess)
            break;
        ce = cudaMemcpyAsync(dst + 2 * n + 1, b + L.o_s1 + sizeof(double), sizeof(int), cudaMemcpyDeviceToHost, st);
    }
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(st, &g);
    if (ce != cudaSuccess || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        std::snprintf(g_batch_msg, sizeof(g_batch_msg), "capture: %s / %s", cudaGetErrorString(ce),
                      cudaGetErrorString(e));
        cudaGetLastError();
        return HIP_ERR_CUDA;
    }
    pl->graph = g;
    if ((e = cudaGraphInstantiate(&pl->exec, g, 0)) != cudaSuccess) {
        std::snprintf(g_batch_msg, sizeof(g_batch_msg), "instantiate: %s", cudaGetErrorString(e));
        return HIP_ERR_CUDA;
    }
    pl->launches = launches;
    return HIP_OK;
}

// Release what plan_build made (graph, buffers, capture stream); the catalogs stay.
static void plan_release(hip_batch_plan *pl)
{
    if (pl->exec) cudaGraphExecDestroy(pl->exec);
    if (pl->graph) cudaGraphDestroy(pl->graph);
    if (pl->buf) cudaFree(pl->buf);
    if (pl->h_out) cudaFreeHost(pl->h_out);
    if (pl->cap_stream) cudaStreamDestroy(pl->cap_stream);
    pl->exec = nullptr;
    pl->graph = nullptr;
    pl->buf = nullptr;
    pl->h_out = nullptr;
    pl->cap_stream = nullptr;
    pl->out_off.clear();
    pl->launches = 0;
}

static void plan_free(hip_batch_plan *pl)
{
    if (!pl) return;
    plan_release(pl);
    delete pl;
}

extern "C" hip_status hip_batch_plan_create(const hip_catalog *cats, int n_cats, hip_precision prec,
                                            hip_batch_plan **plan_out, void *cuda_stream)
{
    g_batch_msg[0] = 0;
    if (!cats || n_cats < 1 || n_cats > 4096 || !plan_out) return HIP_ERR_ARG;
    if (prec != HIP_PREC_FP64 && prec != HIP_PREC_MIXED) return HIP_ERR_ARG;
    for (int i = 0; i < n_cats; ++i) {
        hip_status s = check_catalog(cats[i]);
        if (s != HIP_OK) {
            std::snprintf(g_batch_msg, sizeof(g_batch_msg), "catalog %d rejected", i);
            return s;
        }
    }
    std::lock_guard<std::mutex> lk(hip_api_mutex());
    int dev = 0;
    hip_status hs = hip_device_setup(&dev);
    if (hs != HIP_OK) return hs;
    hip_batch_plan *pl = new hip_batch_plan();
    pl->dev = dev;
    pl->prec = prec;
    pl->cats.assign(cats, cats + n_cats);
    cudaStream_t st = (cudaStream_t)cuda_stream;
    hs = prec == HIP_PREC_MIXED ? plan_build<float>(pl, st) : plan_build<double>(pl, st);
    if (hs != HIP_OK) {
        plan_free(pl);
        return hs;
    }
    *plan_out = pl;
    return HIP_OK;
}

extern "C" int hip_batch_plan_launches(const hip_batch_plan *plan) { return plan ? plan->launches : 0; }

// Copy host inputs, replay the graph, check and unpack (caller holds the API lock).
// If ms is given, the graph replay alone is timed with events on st.
static hip_status plan_run_locked(hip_batch_plan *pl, cudaStream_t st, float *ms)
{
    cudaError_t e;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    char *b = (char *)pl->buf;
    const int nc = (int)pl->cats.size();
    for (int i = 0; i < nc; ++i) {
        const hip_catalog &c = pl->cats[i];
        const CatLayout &L = pl->lay[i];
        if (!L.dev_pos && (e = cudaMemcpyAsync(b + L.o_pos, c.pos, sizeof(float) * 3 * c.N, cudaMemcpyHostToDevice,
                                               st)) != cudaSuccess)
            goto fail;
        if (c.w && !L.dev_w &&
            (e = cudaMemcpyAsync(b + L.o_w, c.w, sizeof(float) * c.N, cudaMemcpyHostToDevice, st)) != cudaSuccess)
            goto fail;
    }
    if (ms) {
        if ((e = cudaEventCreate(&ev0)) != cudaSuccess || (e = cudaEventCreate(&ev1)) != cudaSuccess ||
            (e = cudaEventRecord(ev0, st)) != cudaSuccess)
            goto fail;
    }
    if ((e = cudaGraphLaunch(pl->exec, st)) != cudaSuccess) goto fail;
    if (ms && (e = cudaEventRecord(ev1, st)) != cudaSuccess) goto fail;
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) goto fail;
    if (ms) {
        if ((e = cudaEventElapsedTime(ms, ev0, ev1)) != cudaSuccess) goto fail;
        cudaEventDestroy(ev0);
        cudaEventDestroy(ev1);
        ev0 = ev1 = nullptr;
    }
    for (int i = 0; i < nc; ++i) {
        const size_t n = (size_t)pl->lay[i].n_ell * pl->cats[i].n_k;
        int errw;
        std::memcpy(&errw, pl->h_out + pl->out_off[i] + 2 * n + 1, sizeof(int));
        if (errw) {
            std::snprintf(g_batch_msg, sizeof(g_batch_msg), "catalog %d has a non-finite position or weight", i);
            return HIP_ERR_NONFINITE;
        }
    }
    for (int i = 0; i < nc; ++i) {
        const hip_catalog &c = pl->cats[i];
        const size_t n = (size_t)pl->lay[i].n_ell * c.n_k;
        const double *src = pl->h_out + pl->out_off[i];
        std::memcpy(c.P_out, src, sizeof(double) * n);
        if (c.DD_out) std::memcpy(c.DD_out, src + n, sizeof(double) * n);
        unsigned long long np;
        std::memcpy(&np, src + 2 * n, sizeof(np));
        if (c.npairs_out) *c.npairs_out = (int64_t)np;
    }
    return HIP_OK;
fail:
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
    std::snprintf(g_batch_msg, sizeof(g_batch_msg), "run: %s", cudaGetErrorString(e));
    return HIP_ERR_CUDA;
}

extern "C" hip_status hip_batch_plan_run(hip_batch_plan *pl, void *cuda_stream)
{
    g_batch_msg[0] = 0;
    if (!pl) return HIP_ERR_ARG;
    std::lock_guard<std::mutex> lk(hip_api_mutex());
    return plan_run_locked(pl, (cudaStream_t)cuda_stream, nullptr);
}

// Candidate target occupancies of the autotuner (particles per cell; 0 = cells
// exactly R0 wide).
static const int k_tune_occ[] = {4, 8, 16, 32, 64, 128, 256, 0};

extern "C" hip_status hip_batch_plan_tune(hip_batch_plan *pl, void *cuda_stream, int *chosen_out, float *ms_out)
{
    g_batch_msg[0] = 0;
    if (!pl) return HIP_ERR_ARG;
    std::lock_guard<std::mutex> lk(hip_api_mutex());
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const int nt = (int)(sizeof(k_tune_occ) / sizeof(k_tune_occ[0]));
    int best = -1;
    float best_ms = 0.0f;
    for (int i = 0; i < nt; ++i) {
        plan_release(pl);
        pl->occ = k_tune_occ[i];
        hip_status hs = pl->prec == HIP_PREC_MIXED ? plan_build<float>(pl, st) : plan_build<double>(pl, st);
        if (hs == HIP_OK) hs = plan_run_locked(pl, st, nullptr);  // warm-up
        float ms = 0.0f;
        if (hs == HIP_OK) hs = plan_run_locked(pl, st, &ms);
        if (hs != HIP_OK) return hs;
        if (ms_out) ms_out[i] = ms;
        if (best < 0 || ms < best_ms) {
            best = i;
            best_ms = ms;
        }
    }
    plan_release(pl);
    pl->occ = k_tune_occ[best];
    hip_status hs = pl->prec == HIP_PREC_MIXED ? plan_build<float>(pl, st) : plan_build<double>(pl, st);
    if (hs != HIP_OK) return hs;
    if (chosen_out) *chosen_out = pl->occ;
    return HIP_OK;
}

// The in-kernel shapes of the moment pass at the plan's cell occupancy: warps per
// CTA x fold period, each candidate timed on one replay after a warm-up.
static const int k_tune_warps[] = {4, 8};
static const int k_tune_fold[] = {4096, 8192, 16384};

extern "C" hip_status hip_batch_plan_tune_kernel(hip_batch_plan *pl, void *cuda_stream, int *warps_out, int *fold_out,
                                                 float *ms_out)
{
    g_batch_msg[0] = 0;
    if (!pl) return HIP_ERR_ARG;
    std::lock_guard<std::mutex> lk(hip_api_mutex());
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int best_w = 0, best_f = 0, i = 0;
    float best_ms = 0.0f;
    for (int w : k_tune_warps)
        for (int f : k_tune_fold) {
            plan_release(pl);
            pl->warps = w;
            pl->fold = f;
            hip_status hs = pl->prec == HIP_PREC_MIXED ? plan_build<float>(pl, st) : plan_build<double>(pl, st);
            if (hs == HIP_OK) hs = plan_run_locked(pl, st, nullptr);  // warm-up
            float ms = 0.0f;
            if (hs == HIP_OK) hs = plan_run_locked(pl, st, &ms);
            if (hs != HIP_OK) return hs;
            if (ms_out) ms_out[i] = ms;
            ++i;
            if (best_w == 0 || ms < best_ms) {
                best_w = w;
                best_f = f;
                best_ms = ms;
            }
        }
    plan_release(pl);
    pl->warps = best_w;
    pl->fold = best_f;
    hip_status hs = pl->prec == HIP_PREC_MIXED ? plan_build<float>(pl, st) : plan_build<double>(pl, st);
    if (hs != HIP_OK) return hs;
    if (warps_out) *warps_out = pl->warps;
    if (fold_out) *fold_out = pl->fold;
    return HIP_OK;
}

extern "C" void hip_batch_plan_shape(const hip_batch_plan *pl, int *occ, int *warps, int *fold)
{
    if (!pl) return;
    if (occ) *occ = pl->occ;
    if (warps) *warps = pl->warps;
    if (fold) *fold = pl->fold;
}

extern "C" void hip_batch_plan_destroy(hip_batch_plan *plan)
{
    std::lock_guard<std::mutex> lk(hip_api_mutex());
    plan_free(plan);
}

extern "C" hip_status hip_power_batched(const hip_catalog *cats, int n_cats, hip_precision prec, void *cuda_stream)
{
    hip_batch_plan *pl = nullptr;
    hip_status s = hip_batch_plan_create(cats, n_cats, prec, &pl, cuda_stream);
    if (s != HIP_OK) return s;
    s = hip_batch_plan_run(pl, cuda_stream);
    hip_batch_plan_destroy(pl);
    return s;
}

// hip_power_noalloc: the power-spectrum pass of hip_power (mixed precision) with
// all of its scratch in one fixed, statically sized device array instead of the
// library's growable workspace.
//
// Who needs this: callers that cannot allocate device memory while they run --
// a host application whose own memory pool has already reserved the device's
// memory (a cudaMalloc from a library would fail, or take memory the pool
// counts on), and services that must know their peak device footprint before
// they start, so that no call may grow it.
//
// The call is eager and synchronising: it reads the cell build's error word back
// to the host in the middle of the call and synchronises `cuda_stream` before it
// returns, like hip_power.
//
// The array below is reserved on every device that loads this library, for the
// lifetime of the process.  Its device address is looked up once per device
// (cudaGetSymbolAddress) on the first call made with that device current.
// Every call reuses the same array
// and it keeps the previous call's contents, so each call clears the counters
// and accumulators it needs.  Calls must not overlap on the GPU: two calls whose
// kernels ran at the same time would race on the array.  This entry point
// serialises its calls on the host and synchronises the caller's stream before
// returning, also when a step fails, so calls made through it never overlap one
// another.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "hip_internal.h"
#include "hip_moments.h"
#include "hip_workspace.h"

#define HIP_NOALLOC_BYTES ((size_t)64 << 20)  // 64 MiB

static __device__ __align__(256) unsigned char g_noalloc_scratch[HIP_NOALLOC_BYTES];
static void *g_noalloc_ptr[64];
static char g_noalloc_msg[256];

std::mutex &hip_api_mutex();

extern "C" size_t hip_noalloc_capacity(void) { return HIP_NOALLOC_BYTES; }

extern "C" const char *hip_noalloc_message(void) { return g_noalloc_msg; }

extern "C" hip_status hip_power_noalloc(const float *pos, const float *w, int64_t N, double L, double R0,
                                        hip_window window, const double *k_edges, int n_k, int ell_max, int los_axis,
                                        int64_t prim_begin, int64_t prim_end, double *P_out, double *DD_out,
                                        int64_t *npairs_out, void *cuda_stream)
{
    if (!pos || !P_out) return HIP_ERR_ARG;
    if (N < 1 || N > 2000000000LL) return HIP_ERR_ARG;
    if (window != HIP_WINDOW_PHILCOX) return HIP_ERR_ARG;
    if (ell_max != 0 && ell_max != 2 && ell_max != 4) return HIP_ERR_ARG;
    if (los_axis < 0 || los_axis > 2) return HIP_ERR_ARG;
    if (!(L > 0.0) || !std::isfinite(L) || !(R0 > 0.0) || !(R0 < 0.5 * L)) return HIP_ERR_RANGE;
    if (prim_begin < 0 || prim_end > N || prim_begin > prim_end) return HIP_ERR_RANGE;
    hip_status hs = hip_check_edges(k_edges, n_k);
    if (hs != HIP_OK) return hs;

    std::lock_guard<std::mutex> lk(hip_api_mutex());
    g_noalloc_msg[0] = 0;
    int dev = 0;
    if ((hs = hip_device_setup(&dev)) != HIP_OK) {
        std::snprintf(g_noalloc_msg, sizeof(g_noalloc_msg), "device set-up: %s", hip_last_error());
        return hs;
    }
    cudaError_t e;
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        if ((e = cudaGetSymbolAddress(&p, g_noalloc_scratch)) != cudaSuccess || !p) {
            std::snprintf(g_noalloc_msg, sizeof(g_noalloc_msg), "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
            return HIP_ERR_CUDA;
        }
        g_noalloc_ptr[dev] = p;
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const int n_c = hip_cells_per_side(L, R0);
    const int n_cells = n_c * n_c * n_c;
    const int n_e = n_k + 1, n_ell = ell_max / 2 + 1;
    const int grid = hip_power_grid<float>();
    const bool dpos = hip_is_device_ptr(pos);
    const bool dw = w && hip_is_device_ptr(w);

    Carve cv;
    const size_t o_pos = dpos ? 0 : cv.take(sizeof(float) * 3 * N);
    const size_t o_w = (w && !dw) ? cv.take(sizeof(float) * N) : 0;
    const size_t o_x = cv.take(sizeof(float) * N), o_y = cv.take(sizeof(float) * N), o_z = cv.take(sizeof(float) * N);
    const size_t o_ws = cv.take(sizeof(float) * N), o_idx = cv.take(sizeof(int) * N), o_cid = cv.take(sizeof(int) * N);
    const size_t o_start = cv.take(sizeof(int) * (n_cells + 1)), o_fill = cv.take(sizeof(int) * n_cells);
    const size_t o_part = cv.take(sizeof(double) * (size_t)grid * 3 * n_e);
    const size_t o_small = cv.take(sizeof(double) * 8);
    const size_t o_wt = cv.take(sizeof(double) * n_k);
    const size_t o_dd = cv.take(sizeof(double) * 3 * n_k), o_p = cv.take(sizeof(double) * 3 * n_k);
    // the Legendre-moment pass where it applies (as hip_power), else the direct pass
    const bool moments = hip_pm_applicable(R0, k_edges[n_k], true);
    const size_t o_pm = moments ? cv.take(hip_pm_scratch_bytes(n_e, hip_pm_intervals(R0, k_edges[n_k]))) : 0;
    if (cv.total > HIP_NOALLOC_BYTES) {
        std::snprintf(g_noalloc_msg, sizeof(g_noalloc_msg),
                      "hip_power_noalloc: this call needs %zu bytes of scratch, the static array holds %zu "
                      "(about 24 bytes per particle for device inputs, 36 for host positions, 40 with host weights)",
                      cv.total, (size_t)HIP_NOALLOC_BYTES);
        return HIP_ERR_RANGE;
    }
    char *b = (char *)g_noalloc_ptr[dev];
    // a failed step returns only after the work already queued on the array has
    // finished, so that the next call cannot race with it
#define HIP_NA_CK(call, what)                                                                                        \
    do {                                                                                                             \
        if ((e = (call)) != cudaSuccess) {                                                                           \
            std::snprintf(g_noalloc_msg, sizeof(g_noalloc_msg), "%s: %s", what, cudaGetErrorString(e));              \
            cudaStreamSynchronize(st);                                                                               \
            cudaGetLastError();                                                                                      \
            return HIP_ERR_CUDA;                                                                                     \
        }                                                                                                            \
    } while (0)
    const float *dposp = pos, *dwp = w;
    if (!dpos) {
        HIP_NA_CK(cudaMemcpyAsync(b + o_pos, pos, sizeof(float) * 3 * N, cudaMemcpyHostToDevice, st), "H2D positions");
        dposp = (const float *)(b + o_pos);
    }
    if (w && !dw) {
        HIP_NA_CK(cudaMemcpyAsync(b + o_w, w, sizeof(float) * N, cudaMemcpyHostToDevice, st), "H2D weights");
        dwp = (const float *)(b + o_w);
    }
    float *x = (float *)(b + o_x), *y = (float *)(b + o_y), *z = (float *)(b + o_z);
    int *idx = (int *)(b + o_idx), *cid = (int *)(b + o_cid);
    int *cstart = (int *)(b + o_start), *cfill = (int *)(b + o_fill);
    double *partials = (double *)(b + o_part);
    double *small = (double *)(b + o_small);
    double *S1 = small;
    unsigned long long *npairs = (unsigned long long *)(small + 1);
    int *err = (int *)(small + 2);
    int *counter = err + 1;
    double *Wt = (double *)(b + o_wt), *DD = (double *)(b + o_dd), *P = (double *)(b + o_p);
    // the cell build clears the cell counts, S1 and the error word it uses
    HIP_NA_CK(hip_build_cells<float>(dposp, dwp, N, L, n_c, x, y, z, (float *)(b + o_ws), idx, cid, cstart, cfill, S1,
                                     err, st),
              "cell build");
    int herr = 0;
    HIP_NA_CK(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st), "D2H error word");
    HIP_NA_CK(cudaStreamSynchronize(st), "cell build sync");
    if (herr) return HIP_ERR_NONFINITE;
    // the pair counter and the work counter start at zero on every call
    HIP_NA_CK(cudaMemsetAsync(npairs, 0, sizeof(unsigned long long), st), "clear pair count");
    HIP_NA_CK(cudaMemsetAsync(counter, 0, sizeof(int), st), "clear work counter");
    CellList<float> cl{x, y, z, (const float *)(b + o_ws), idx, cstart, n_c, L, L / n_c};
    PowerKernelArgs ka;
    ka.n_e = n_e;
    ka.los = los_axis;
    ka.p0 = prim_begin;
    ka.p1 = prim_end;
    ka.n_items = n_cells * HIP_NSHIFT;
    ka.n_part = N;
    ka.work_counter = counter;
    ka.partials = partials;  // every CTA overwrites its own row
    ka.npairs = npairs;
    if (moments)
        HIP_NA_CK(hip_power_moments<float>(cl, ka, k_edges, n_ell, R0, b + o_pm, partials, st), "moment pass");
    else
        HIP_NA_CK(hip_power_pairs<float>(cl, ka, k_edges, n_ell, R0, grid, st), "pair kernel");
    HIP_NA_CK(hip_power_finalize(partials, moments ? 1 : grid, n_e, n_ell, k_edges, R0, L, S1, Wt, DD, P, st),
              "finalize");
    unsigned long long hn = 0;
    HIP_NA_CK(cudaMemcpyAsync(P_out, P, sizeof(double) * n_ell * n_k, cudaMemcpyDeviceToHost, st), "D2H P");
    if (DD_out)
        HIP_NA_CK(cudaMemcpyAsync(DD_out, DD, sizeof(double) * n_ell * n_k, cudaMemcpyDeviceToHost, st), "D2H DD");
    HIP_NA_CK(cudaMemcpyAsync(&hn, npairs, sizeof(hn), cudaMemcpyDeviceToHost, st), "D2H npairs");
    HIP_NA_CK(cudaStreamSynchronize(st), "stream sync");
#undef HIP_NA_CK
    if (npairs_out) *npairs_out = (int64_t)hn;
    return HIP_OK;
}

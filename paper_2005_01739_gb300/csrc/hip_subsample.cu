// Random subsampling of a catalog: keep a random fraction of the tracers before
// the pair count (Sec. 9: the estimators scale as N^2 at fixed R0, so matter
// catalogs are counted on a subsample of 1/f_sub of their particles; the
// estimator itself is unchanged and takes the subsample's own n_w).
//
// Particle i is kept iff its uniform variate u_i < fraction, with u_i the top 53
// bits of the i-th output of SplitMix64 seeded with `seed` (Steele, Lea & Flood
// 2014): z = seed + (i + 1) * 0x9E3779B97F4A7C15, then the two xor-shift-multiply
// rounds and a final xor-shift.  In integers: keep iff (z_i >> 11) < floor(fraction
// 2^53), so the selection is exact and the same on every machine.  Kept particles
// keep their input order.
//
// Three launches: per-block counts, one exclusive scan of the block counts, and
// the ordered scatter (each block re-derives its flags and ranks them with warp
// ballots).  All are HBM-bound: 12 (16 with weights) bytes read per particle and
// as many written per kept particle.
#include <algorithm>
#include <cmath>
#include <mutex>

#include "hip_internal.h"
#include "hip_workspace.h"

std::mutex &hip_api_mutex();

#define HIP_SUB_THREADS 256
#define HIP_SUB_ITEMS 16  // particles per thread per block pass
#define HIP_SUB_CHUNK (HIP_SUB_THREADS * HIP_SUB_ITEMS)

// Output i + 1 of SplitMix64 seeded with `seed` (i = 0, 1, ...).
__device__ __forceinline__ unsigned long long hip_sm64(unsigned long long seed, unsigned long long i)
{
    unsigned long long z = seed + (i + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ bool hip_sub_keep(unsigned long long seed, unsigned long long i, unsigned long long thr)
{
    return (hip_sm64(seed, i) >> 11) < thr;
}

// Uniform random catalog (the random catalog of the DDR^II term, Sec. 4.3):
// coordinate d of random j is out[3 j + d] = u L with u = (z_i >> 40) 2^-24, z_i
// output i + 1 of SplitMix64 for i = 3 j + d, and the product rounded once to
// float (u is exact in float, L is taken as a float).  Grid-stride, HBM-bound
// (12 bytes written per random).
__global__ void __launch_bounds__(HIP_SUB_THREADS) k_uniform_randoms(float *out, long long n3,
                                                                     unsigned long long seed, float Lf)
{
    const long long stride = (long long)gridDim.x * HIP_SUB_THREADS;
    for (long long i = (long long)blockIdx.x * HIP_SUB_THREADS + threadIdx.x; i < n3; i += stride) {
        const float u = (float)(unsigned)(hip_sm64(seed, (unsigned long long)i) >> 40) * 5.9604644775390625e-08f;
        out[i] = __fmul_rn(u, Lf);
    }
}

cudaError_t hip_launch_uniform_randoms(float *d_out, long long n_r, double L, unsigned long long seed,
                                       cudaStream_t st)
{
    if (n_r <= 0) return cudaSuccess;
    const long long n3 = 3 * n_r;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long want = (n3 + HIP_SUB_THREADS - 1) / HIP_SUB_THREADS;
    const unsigned blocks = (unsigned)std::min<long long>(want, (long long)sms * 16);
    k_uniform_randoms<<<blocks, HIP_SUB_THREADS, 0, st>>>(d_out, n3, seed, (float)L);
    return cudaGetLastError();
}

// counts[b] = kept particles of chunk b (HIP_SUB_CHUNK particles per block)
__global__ void __launch_bounds__(HIP_SUB_THREADS) k_sub_count(long long N, unsigned long long seed,
                                                               unsigned long long thr, int *counts)
{
    __shared__ int red[HIP_SUB_THREADS / 32];
    const long long base = (long long)blockIdx.x * HIP_SUB_CHUNK;
    int n = 0;
#pragma unroll 4
    for (int k = 0; k < HIP_SUB_ITEMS; ++k) {
        const long long i = base + (long long)k * HIP_SUB_THREADS + threadIdx.x;
        if (i < N && hip_sub_keep(seed, (unsigned long long)i, thr)) ++n;
    }
    for (int o = 16; o > 0; o >>= 1) n += __shfl_xor_sync(0xffffffffu, n, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = n;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int w = 0; w < HIP_SUB_THREADS / 32; ++w) t += red[w];
        counts[blockIdx.x] = t;
    }
}

// offsets[b] = sum of counts before b; offsets[nb] = total (one block)
__global__ void __launch_bounds__(1024) k_sub_scan(const int *counts, int nb, long long *offsets)
{
    __shared__ long long part[1024];
    const int per = (nb + 1023) / 1024;
    const int b0 = threadIdx.x * per, b1 = min(nb, b0 + per);
    long long s = 0;
    for (int b = b0; b < b1; ++b) s += counts[b];
    part[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long run = 0;
        for (int t = 0; t < 1024; ++t) {
            const long long v = part[t];
            part[t] = run;
            run += v;
        }
        offsets[nb] = run;
    }
    __syncthreads();
    long long run = part[threadIdx.x];
    for (int b = b0; b < b1; ++b) {
        offsets[b] = run;
        run += counts[b];
    }
}

// kept particles of chunk b written in input order from offsets[b] on
__global__ void __launch_bounds__(HIP_SUB_THREADS) k_sub_scatter(const float *__restrict__ pos,
                                                                 const float *__restrict__ w, long long N,
                                                                 unsigned long long seed, unsigned long long thr,
                                                                 const long long *__restrict__ offsets,
                                                                 float *__restrict__ pos_out, float *__restrict__ w_out)
{
    __shared__ int wsum[HIP_SUB_THREADS / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long base = (long long)blockIdx.x * HIP_SUB_CHUNK;
    long long out = offsets[blockIdx.x];
    for (int k = 0; k < HIP_SUB_ITEMS; ++k) {  // one block-wide pass of HIP_SUB_THREADS particles
        const long long i = base + (long long)k * HIP_SUB_THREADS + threadIdx.x;
        const bool keep = i < N && hip_sub_keep(seed, (unsigned long long)i, thr);
        const unsigned bal = __ballot_sync(0xffffffffu, keep);
        if (lane == 0) wsum[warp] = __popc(bal);
        __syncthreads();
        int before = 0, total = 0;
#pragma unroll
        for (int v = 0; v < HIP_SUB_THREADS / 32; ++v) {
            const int c = wsum[v];
            before += v < warp ? c : 0;
            total += c;
        }
        if (keep) {
            const long long j = out + before + __popc(bal & ((1u << lane) - 1u));
            pos_out[3 * j] = pos[3 * i];
            pos_out[3 * j + 1] = pos[3 * i + 1];
            pos_out[3 * j + 2] = pos[3 * i + 2];
            if (w_out) w_out[j] = w[i];
        }
        out += total;
        __syncthreads();
    }
}

extern "C" hip_status hip_subsample(const float *pos, const float *w, int64_t N, double fraction, uint64_t seed,
                                    float *pos_out, float *w_out, int64_t *n_out, void *cuda_stream)
{
    hip_clear_error();
    if (!pos || !pos_out || !n_out || N < 0 || N > 2000000000LL) return HIP_ERR_ARG;
    if (!(fraction >= 0.0 && fraction <= 1.0)) return HIP_ERR_RANGE;
    std::lock_guard<std::mutex> lk(hip_api_mutex());
    int dev = 0;
    hip_status hs = hip_device_setup(&dev);
    if (hs != HIP_OK) return hs;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const bool use_w = w && w_out;
    const bool dpos = hip_is_device_ptr(pos), dw = use_w && hip_is_device_ptr(w);
    const bool dpo = hip_is_device_ptr(pos_out), dwo = use_w && hip_is_device_ptr(w_out);
    const long long nb = (N + HIP_SUB_CHUNK - 1) / HIP_SUB_CHUNK;
    const unsigned long long thr = (unsigned long long)std::floor(std::ldexp(fraction, 53));
    Carve cv;
    const size_t o_pos = dpos ? 0 : cv.take(sizeof(float) * 3 * (size_t)N);
    const size_t o_w = (use_w && !dw) ? cv.take(sizeof(float) * (size_t)N) : 0;
    const size_t o_po = dpo ? 0 : cv.take(sizeof(float) * 3 * (size_t)N);
    const size_t o_wo = (use_w && !dwo) ? cv.take(sizeof(float) * (size_t)N) : 0;
    const size_t o_cnt = cv.take(sizeof(int) * (size_t)(nb + 1));
    const size_t o_off = cv.take(sizeof(long long) * (size_t)(nb + 1));
    Workspace &ws = hip_workspace(dev);
    if ((hs = ws.reserve(cv.total, st)) != HIP_OK) return hs;
    char *b = (char *)ws.base;
    cudaError_t e = cudaSuccess;
    const float *dp = pos, *dwp = use_w ? w : nullptr;
    float *po = dpo ? pos_out : (float *)(b + o_po);
    float *wo = use_w ? (dwo ? w_out : (float *)(b + o_wo)) : nullptr;
    long long total = 0;
    if (N > 0) {
        if (!dpos) {
            e = cudaMemcpyAsync(b + o_pos, pos, sizeof(float) * 3 * (size_t)N, cudaMemcpyHostToDevice, st);
            dp = (const float *)(b + o_pos);
        }
        if (e == cudaSuccess && use_w && !dw) {
            e = cudaMemcpyAsync(b + o_w, w, sizeof(float) * (size_t)N, cudaMemcpyHostToDevice, st);
            dwp = (const float *)(b + o_w);
        }
        int *counts = (int *)(b + o_cnt);
        long long *offsets = (long long *)(b + o_off);
        if (e == cudaSuccess) {
            k_sub_count<<<(unsigned)nb, HIP_SUB_THREADS, 0, st>>>(N, seed, thr, counts);
            k_sub_scan<<<1, 1024, 0, st>>>(counts, (int)nb, offsets);
            k_sub_scatter<<<(unsigned)nb, HIP_SUB_THREADS, 0, st>>>(dp, dwp, N, seed, thr, offsets, po, wo);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaMemcpyAsync(&total, offsets + nb, sizeof(long long), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e == cudaSuccess && total > 0 && !dpo)
            e = cudaMemcpyAsync(pos_out, po, sizeof(float) * 3 * (size_t)total, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess && total > 0 && use_w && !dwo)
            e = cudaMemcpyAsync(w_out, wo, sizeof(float) * (size_t)total, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    if (e != cudaSuccess) {
        hip_set_error("subsample", e);
        cudaGetLastError();
        return HIP_ERR_CUDA;
    }
    *n_out = total;
    return HIP_OK;
}

extern "C" hip_status hip_uniform_randoms(float *out, int64_t N_r, double L, uint64_t seed, void *cuda_stream)
{
    hip_clear_error();
    if (!out || N_r < 0 || N_r > 2000000000LL) return HIP_ERR_ARG;
    if (!(L > 0.0) || !std::isfinite(L) || !((float)L < 3.0e38f)) return HIP_ERR_RANGE;
    std::lock_guard<std::mutex> lk(hip_api_mutex());
    int dev = 0;
    hip_status hs = hip_device_setup(&dev);
    if (hs != HIP_OK) return hs;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const bool dout = hip_is_device_ptr(out);
    float *d = out;
    if (!dout && N_r > 0) {
        Workspace &ws = hip_workspace(dev);
        if ((hs = ws.reserve(sizeof(float) * 3 * (size_t)N_r, st)) != HIP_OK) return hs;
        d = (float *)ws.base;
    }
    cudaError_t e = hip_launch_uniform_randoms(d, N_r, L, seed, st);
    if (e == cudaSuccess && !dout && N_r > 0)
        e = cudaMemcpyAsync(out, d, sizeof(float) * 3 * (size_t)N_r, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        hip_set_error("uniform randoms", e);
        cudaGetLastError();
        return HIP_ERR_CUDA;
    }
    return HIP_OK;
}

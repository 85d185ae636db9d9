// The bispectrum contraction on the Blackwell tensor cores (Sec. 4.4 / 4.5 of
// arXiv:2005.01739):
//
//     T^ab_l += sum_p s_p sum_m A^a_lm(p) A^b_lm(p),
//
// i.e. for each l the Gram-type product X_l diag(s) X_l^T of the per-primary
// accumulators (rows: bins a; columns: primaries p and orders m).
//
// Layout.  The rows (l, a) of all multipoles are stacked: a tile of 128 rows
// holds floor(128 / n_k) whole l blocks (all five for n_k <= 25, two tiles up to
// n_k = 42), so one M = 128 MMA per tile computes every diagonal block (l, l) it
// needs (the off-diagonal blocks come for free and are ignored).  The K dimension
// runs over (p, slot): each primary has 9 slots, slot m + l of row (l, a) holding
// A^a_lm and slots beyond 2l zero, so the diagonal blocks contract exactly over m.
// Slots 0..7 of primary p fill K group p (8 BF16 values, 16 bytes); slot 8 (only
// l = 4 uses it) of primaries 8g .. 8g + 7 fills K group P + g.  A stage of P
// primaries (8 for one tile, 4 for two) is K = 9P rounded up to 16.
//
// Precision: an error-free split in the manner of Ozaki et al.  The tensor core
// rounds its FP32 accumulator at the accumulator's magnitude, and a plain hi/lo
// TF32 split loses about 1e-6 of each stage's sum that way (measured), too much
// for the cancelling data and random primary sums.  Instead each row r of a stage
// is scaled by a power of two 2^e_r above its largest |value| and cut into three
// slices of 8 significant bits, x = (h + m + l) 2^e_r with h, m, l integer
// multiples of 2^-8, 2^-16, 2^-24 (|h| <= 1, |m|, |l| <= 2^-9): x to 2^-25 of the
// row's largest value.  Every slice is exact in BF16, every product of two
// slices is an exact integer multiple of its unit, and a stage's sums of at most
// 72 products stay below 2^24 units, so the three accumulators
//     A0 = h h^T,  A1 = h m^T + m h^T,  A2 = h l^T + l h^T + m m^T
// (separate tensor-memory columns; the dropped terms are below 2^-32 of A0) are
// exact whatever the accumulator's rounding (kind::f16, BF16 operands, FP32
// accumulation); they are added in FP64 into the CTA's rows in shared memory
// after every unit of work.  Primary weights enter as sqrt|s_p| before the split
// and the sign through the MMA's negate-A bit, so a unit holds primaries of one
// sign (a stage with both signs is issued twice, once per sign, with the other
// primaries zeroed).
//
// Pipeline (one CTA of 16 warps per SM, persistent over a contiguous range of
// stages; a unit is one (stage, sign, tile)): a bulk copy (cp.async.bulk,
// mbarrier completion) brings the next stage's X block into shared memory; four
// threads share row r of the tile (its scale and its slices, written as 16-byte K
// groups in the canonical K-major layout without swizzle: 8-row x 16-byte core
// matrices, 8-row groups 128 bytes apart, K groups 2048 bytes apart) and split
// unit u + 1 into the second slice buffer while the MMAs of unit u run; one
// thread issues the MMAs and commits them to an mbarrier; the warps read the
// accumulators back with tcgen05.ld (warp w owns lanes 32 (w mod 4)..+31, the
// four warps of a lane group split the columns) and add them to the CTA's FP64
// rows, which go to the catalog's FP64 sums (atomics) when the CTA leaves the
// catalog.  Every wait is bounded (about two seconds); a wait that gives up sets
// bit 0 of *status, stops the CTA's work, and the CTA still waits (bounded) for
// its own MMAs before it frees its tensor memory.
#include <cstdint>
#include <cstdio>

#include "hip_internal.h"
#include "hip_bispec.h"

#define TC_THREADS 512
#define TC_ROWB 2048        // bytes of one K group (8 bf16) of a 128-row operand
#define TC_WAIT_CYCLES 4000000000LL
#define TC_SEGS 32          // segments cached in shared memory

__device__ __forceinline__ uint32_t tc_smem(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t tc_desc(uint32_t addr)
{
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
    d |= (uint64_t)(TC_ROWB >> 4) << 16;  // leading dimension (K) byte offset between core matrices
    d |= (uint64_t)(128 >> 4) << 32;      // stride dimension (M/N) byte offset between 8-row groups
    d |= (uint64_t)1 << 46;               // descriptor version of tcgen05
    return d;                             // base offset 0, relative offsets, no swizzle
}

// instruction descriptor: D f32, A and B bf16, both K-major, M = 128, N = n
__device__ __forceinline__ uint32_t tc_idesc(int n, bool negate_a)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((negate_a ? 1u : 0u) << 13) | ((uint32_t)(n >> 3) << 17) |
           ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t tmem_d, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem_d),
        "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void tc_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(tc_smem(bar))
                 : "memory");
}

__device__ __forceinline__ bool tc_try(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(tc_smem(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait on one phase of an mbarrier; false if it gave up.
__device__ __forceinline__ bool tc_wait(uint64_t *bar, uint32_t parity)
{
    if (tc_try(bar, parity)) return true;
    const long long t0 = clock64();
    while (!tc_try(bar, parity))
        if (clock64() - t0 > TC_WAIT_CYCLES) return false;
    return true;
}

// two floats that are exact in BF16 as one packed pair (lo in the low half)
__device__ __forceinline__ uint32_t tc_bf16x2(float lo, float hi)
{
    uint32_t r;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
    return r;
}

struct TcGeom {
    int nk, lpt, G;  // bins, l blocks per 128-row tile, tiles
    int rows[3];     // valid rows of each tile
    int ncol[3];     // N of each tile's MMA (rows rounded up to 16)
};

__device__ __forceinline__ void tc_geom(int nk, TcGeom &g)
{
    g.nk = nk;
    g.lpt = 128 / nk;
    if (g.lpt > HIP_LMAX + 1) g.lpt = HIP_LMAX + 1;
    g.G = (HIP_LMAX + 1 + g.lpt - 1) / g.lpt;
#pragma unroll
    for (int t = 0; t < 3; ++t) {
        int nl = HIP_LMAX + 1 - t * g.lpt;
        if (nl > g.lpt) nl = g.lpt;
        if (nl < 0) nl = 0;
        g.rows[t] = nl * nk;
        g.ncol[t] = ((g.rows[t] + 15) / 16) * 16;
    }
}

int hip_bk_tc_stage_prims(int nk_max) { return (128 / nk_max >= HIP_LMAX + 1) ? 8 : 4; }

static int tc_tiles(int nk)
{
    int lpt = 128 / nk;
    if (lpt > HIP_LMAX + 1) lpt = HIP_LMAX + 1;
    return (HIP_LMAX + 1 + lpt - 1) / lpt;
}

// Byte offsets of the dynamic shared memory (from the 1024-byte aligned base):
// two buffers of the three slices of one tile, two staging buffers of a stage's
// X block, the rows as two float arrays, three mbarriers.  The same function
// lays out the kernel and sizes (and checks) the launch.
struct TcLayout {
    size_t slice;     // bytes of one slice operand (128 rows x K bf16)
    size_t stg;       // offset of staging buffer 0 (buffer 1 follows after stg_bytes)
    size_t stg_bytes; // bytes of one staging buffer
    size_t rows;      // offset of the row sums: hi [nrow] floats, then lo [nrow]
    int nrow;         // 5 n_k^2
    size_t bars;      // offset of the three mbarriers (8-byte aligned)
    size_t total;     // bytes used from the aligned base
};

__host__ __device__ __forceinline__ TcLayout tc_layout(int nk_max, int P)
{
    TcLayout t;
    const int K = ((9 * P + 15) / 16) * 16;
    t.slice = (size_t)128 * K * 2;
    t.stg = 6 * t.slice;
    t.stg_bytes = (size_t)P * HIP_NLM * nk_max * 4;
    t.rows = t.stg + 2 * t.stg_bytes;
    t.nrow = (HIP_LMAX + 1) * nk_max * nk_max;
    t.bars = (t.rows + (size_t)2 * t.nrow * 4 + 7) & ~(size_t)7;
    t.total = t.bars + 3 * 8;
    return t;
}

static size_t tc_smem_bytes(int nk_max, int P) { return tc_layout(nk_max, P).total + 1024; }

bool hip_bk_tc_supported(int nk_max) { return tc_tiles(nk_max) <= 2; }

// One unit of work: a stage's primaries of one sign, one tile of rows.
struct TcUnit {
    int s, sgn, t;      // stage, sign (+1 / -1), tile
    int si, nk, nv;     // segment, its n_k, valid primaries of the stage
};

template <int P>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_bk_contract_tc(const BkSeg *__restrict__ segs, int n_segs, int n_stages, int nk_max, int *status)
{
    extern __shared__ __align__(1024) unsigned char tc_dyn[];
    // operands start on a 1024-byte boundary whatever the toolchain aligns the
    // dynamic shared memory to (the launch asks for 1024 bytes of slack)
    unsigned char *tc_raw = tc_dyn + ((1024u - (tc_smem(tc_dyn) & 1023u)) & 1023u);
    constexpr int K = ((9 * P + 15) / 16) * 16, KG = K / 8;  // K groups of 8 bf16
    constexpr int GPT = (KG + 3) / 4;                          // K groups per thread
    const TcLayout lay = tc_layout(nk_max, P);
    const size_t slice = lay.slice;                            // bytes of one slice operand
    unsigned char *slices = tc_raw;                            // [2 buffers][h, m, l]
    float *stg0 = reinterpret_cast<float *>(tc_raw + lay.stg);
    const int stg_elems = P * HIP_NLM * nk_max;
    // the CTA's rows of the current catalog, [5][n_k][n_k], as unevaluated sums
    // hi + lo of two floats (FP64 arithmetic is slow on this part; two floats
    // carry ~48 bits, more than the folds need)
    const int nrow = lay.nrow;
    float *rowhi = reinterpret_cast<float *>(tc_raw + lay.rows), *rowlo = rowhi + nrow;
    uint64_t *bars = reinterpret_cast<uint64_t *>(tc_raw + lay.bars);  // copies 0, 1; MMA
    __shared__ uint32_t s_tmem;
    __shared__ float s_scale[8];
    __shared__ int s_sign[8];
    __shared__ BkSeg s_segs[TC_SEGS];  // the first segments of the table, read often
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int i = tid; i < n_segs && i < TC_SEGS; i += TC_THREADS) s_segs[i] = segs[i];
    auto SEG = [&](int i) -> const BkSeg & { return i < TC_SEGS ? s_segs[i] : segs[i]; };

    const int per = (n_stages + gridDim.x - 1) / gridDim.x;
    const int s_lo = blockIdx.x * per, s_hi = min(s_lo + per, n_stages);
    const uint32_t ncols = 512u;  // A0, A1, A2 at columns 0, 128, 256
    for (int i = tid; i < nrow; i += TC_THREADS) rowhi[i] = rowlo[i] = 0.f;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc_smem(&s_tmem)),
                     "r"(ncols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        for (int i = 0; i < 3; ++i) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc_smem(&bars[i])));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = s_tmem;
    bool ok = true;
    int n_commit = 0;

    auto seg_of = [&](int s) {
        int i = 0;
        while (i + 1 < n_segs && s >= SEG(i).stage_end) ++i;
        return i;
    };
    // thread 0: bulk copy of stage s's X block into staging buffer b
    auto prefetch = [&](int s, int b) {
        const BkSeg &sg = SEG(seg_of(s));
        const int j = s - sg.stage_begin;
        const int nv = min(P, sg.n_p - j * P);
        // a bulk copy moves a multiple of 16 bytes: the last stage of a segment may
        // read up to 12 bytes past its last primary (the X buffer has slack there)
        const uint32_t bytes = ((uint32_t)nv * HIP_NLM * sg.n_k * 4 + 15u) & ~15u;
        const float *src = reinterpret_cast<const float *>(sg.X) + (size_t)j * P * HIP_NLM * sg.n_k;
        float *dst = stg0 + (size_t)b * stg_elems;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(tc_smem(&bars[b])), "r"(bytes)
                     : "memory");
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                tc_smem(dst)),
            "l"(src), "r"(bytes), "r"(tc_smem(&bars[b]))
            : "memory");
    };
    int has_pos = 0, has_neg = 0;
    // make stage s current: the next stage's copy is started, this one's awaited,
    // its primaries' weights read (all threads; CTA-uniform outcome)
    auto prepare = [&](int s) {
        if (s + 1 < s_hi && tid == 0) prefetch(s + 1, (s + 1 - s_lo) & 1);
        const BkSeg &sg = SEG(seg_of(s));
        const int jst = s - sg.stage_begin, nv = min(P, sg.n_p - jst * P);
        if (tid < P) {
            const float v = tid < nv ? reinterpret_cast<const float *>(sg.sp)[(size_t)jst * P + tid] : 0.f;
            s_scale[tid] = sqrtf(fabsf(v));
            s_sign[tid] = v > 0.f ? 1 : (v < 0.f ? -1 : 0);
        }
        const uint32_t use = (uint32_t)((s - s_lo) >> 1);
        if (!__syncthreads_and(tc_wait(&bars[(s - s_lo) & 1], use & 1u))) {
            if (tid == 0) atomicOr(status, 1);
            ok = false;
        }
        has_pos = has_neg = 0;
        for (int p = 0; p < P; ++p) {
            has_pos |= s_sign[p] > 0;
            has_neg |= s_sign[p] < 0;
        }
    };
    // the unit after u (u.s < 0: none yet); false when the CTA's stages are done
    auto advance = [&](TcUnit &u) -> bool {
        int s = u.s, pass = u.s < 0 ? -1 : (u.sgn > 0 ? 0 : 1), t = u.t;
        TcGeom g;
        if (s >= 0) tc_geom(u.nk, g);
        for (;;) {
            if (s >= 0 && t + 1 < g.G) {
                ++t;
            } else {
                // next sign of this stage, or the next stage
                t = 0;
                bool found = false;
                while (!found) {
                    if (s >= 0 && pass == 0 && has_neg) {
                        pass = 1;
                        found = true;
                    } else {
                        s = s < 0 ? s_lo : s + 1;
                        if (s >= s_hi) return false;
                        prepare(s);
                        if (!ok) return false;
                        pass = -1;
                        if (has_pos) {
                            pass = 0;
                            found = true;
                        } else if (has_neg) {
                            pass = 1;
                            found = true;
                        }
                    }
                }
                const int si = seg_of(s);
                const BkSeg &sg = SEG(si);
                u.si = si;
                u.nk = sg.n_k;
                u.nv = min(P, sg.n_p - (s - sg.stage_begin) * P);
                tc_geom(u.nk, g);
            }
            u.s = s;
            u.sgn = pass == 0 ? 1 : -1;
            u.t = t;
            return true;
        }
    };
    // split unit u into slice buffer sb: four threads per row, K groups q, q + 4, ...
    // K group p < P holds slots 0..7 of primary p, group P + g slot 8 (m = 4 of
    // l = 4) of primaries 8g .. 8g + 7; the rest is zero padding
    auto transform = [&](const TcUnit &u, int sb) {
        TcGeom g;
        tc_geom(u.nk, g);
        const int nk = u.nk, R = g.rows[u.t];
        const int row = tid >> 2, q = tid & 3;
        int l = -1, a = 0;
        if (row < R) {
            const int ll = row / nk;
            l = u.t * g.lpt + ll;
            a = row - ll * nk;
        }
        const float *stg = stg0 + (size_t)((u.s - s_lo) & 1) * stg_elems;
        const float *col = stg + (size_t)(l > 0 ? l * l : 0) * nk + a;  // slot 0 of primary 0
        const size_t pstride = (size_t)HIP_NLM * nk;
        float v[GPT * 8];
        float vmax = 0.f;
#pragma unroll
        for (int j = 0; j < GPT; ++j) {
            const int kg = q + 4 * j;
#pragma unroll
            for (int i = 0; i < 8; ++i) v[8 * j + i] = 0.f;
            if (kg < P) {
                const int p = kg;
                const float w = (p < u.nv && s_sign[p] == u.sgn) ? s_scale[p] : 0.f;
                if (w != 0.f && l >= 0) {
                    const float *src = col + p * pstride;
#pragma unroll
                    for (int i = 0; i < 8; ++i)
                        if (i <= 2 * l) v[8 * j + i] = src[(size_t)i * nk] * w;
                }
            } else if (kg < P + (P + 7) / 8 && l == HIP_LMAX) {
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int p = 8 * (kg - P) + i;
                    if (p < P && p < u.nv && s_sign[p] == u.sgn) v[8 * j + i] = col[p * pstride + 8 * nk] * s_scale[p];
                }
            }
#pragma unroll
            for (int i = 0; i < 8; ++i) vmax = fmaxf(vmax, fabsf(v[8 * j + i]));
        }
        vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, 1));
        vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, 2));
        // 2^e > vmax, from the exponent field (vmax = f 2^e with f in [0.5, 1)):
        // x 2^-e in (-1, 1); e is clamped so that both powers of two are normal
        int e = vmax > 0.f ? (int)((__float_as_uint(vmax) >> 23) & 0xFFu) - 126 : 0;
        e = e < -100 ? -100 : (e > 118 ? 118 : e);
        // 2^(8-e), 2^(e-8), 2^(e-16), 2^(e-24)
        const float down8 = __uint_as_float((uint32_t)(135 - e) << 23);
        const float up8 = __uint_as_float((uint32_t)(119 + e) << 23), up16 = __uint_as_float((uint32_t)(111 + e) << 23),
                    up24 = __uint_as_float((uint32_t)(103 + e) << 23);
        unsigned char *buf = slices + (size_t)sb * 3 * slice;
#pragma unroll
        for (int j = 0; j < GPT; ++j) {
            const int kg = q + 4 * j;
            if (kg >= KG) break;
            uint32_t h[4], m[4], lo[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                float hh[2], mm[2], ll2[2];
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    // in units of 2^(e-8): h = round(x), then the next 8 bits twice
                    const float x = v[8 * j + 2 * i + c] * down8;
                    const float ih = rintf(x);
                    const float r1 = (x - ih) * 256.f;
                    const float im = rintf(r1);
                    const float il = rintf((r1 - im) * 256.f);
                    hh[c] = ih * up8;
                    mm[c] = im * up16;
                    ll2[c] = il * up24;
                }
                h[i] = tc_bf16x2(hh[0], hh[1]);
                m[i] = tc_bf16x2(mm[0], mm[1]);
                lo[i] = tc_bf16x2(ll2[0], ll2[1]);
            }
            const size_t off = (size_t)kg * TC_ROWB + (size_t)row * 16;
            *reinterpret_cast<uint4 *>(buf + off) = make_uint4(h[0], h[1], h[2], h[3]);
            *reinterpret_cast<uint4 *>(buf + slice + off) = make_uint4(m[0], m[1], m[2], m[3]);
            *reinterpret_cast<uint4 *>(buf + 2 * slice + off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
        }
        asm volatile("fence.proxy.async.shared::cta;");
    };
    // thread 0: the MMAs of unit u from slice buffer sb, committed to the MMA barrier
    auto issue = [&](const TcUnit &u, int sb) {
        if (tid == 0) {
            TcGeom g;
            tc_geom(u.nk, g);
            const unsigned char *buf = slices + (size_t)sb * 3 * slice;
            const uint32_t ah = tc_smem(buf), am = tc_smem(buf + slice), al = tc_smem(buf + 2 * slice);
            const uint32_t idesc = tc_idesc(g.ncol[u.t], u.sgn < 0);
            // the descriptors' start-address field is addr >> 4 in the low bits:
            // a K step adds 2 TC_ROWB >> 4 to it (no carry: addresses < 256 KB)
            const uint64_t dh0 = tc_desc(ah), dm0 = tc_desc(am), dl0 = tc_desc(al);
#pragma unroll
            for (int ks = 0; ks < K / 16; ++ks) {
                const uint64_t off = (uint64_t)ks * (2 * TC_ROWB >> 4);
                const uint32_t acc = ks == 0 ? 0u : 1u;
                const uint64_t dh = dh0 + off, dm = dm0 + off, dl = dl0 + off;
                tc_mma(tmem, dh, dh, idesc, acc);
                tc_mma(tmem + 128u, dh, dm, idesc, acc);
                tc_mma(tmem + 128u, dm, dh, idesc, 1u);
                tc_mma(tmem + 256u, dh, dl, idesc, acc);
                tc_mma(tmem + 256u, dl, dh, idesc, 1u);
                tc_mma(tmem + 256u, dm, dm, idesc, 1u);
            }
            tc_commit(&bars[2]);
        }
        ++n_commit;
    };
    auto wait_mma = [&]() {
        const bool good = tc_wait(&bars[2], (uint32_t)((n_commit - 1) & 1));
        if (!__syncthreads_and(good)) {
            if (tid == 0) atomicOr(status, 1);
            ok = false;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
    };
    // A0 + A1 + A2 of unit u -> the CTA's FP64 rows (the unit's MMAs are done)
    auto fold = [&](const TcUnit &u) {
        TcGeom g;
        tc_geom(u.nk, g);
        const int nk = u.nk, R = g.rows[u.t];
        const int r0 = 32 * (warp & 3), gq = warp >> 2;
        if (r0 < R) {  // warp-uniform
            const int row = r0 + lane;
            const bool valid = row < R;
            const int ll = row / nk, a = row - ll * nk, l = u.t * g.lpt + ll;
            const int ll_lo = r0 / nk, ll_hi = min(R - 1, r0 + 31) / nk;
            const int c0 = (ll_lo * nk) & ~7, c1 = min(g.ncol[u.t], (ll_hi + 1) * nk);
            for (int c = c0 + 8 * gq; c < c1; c += 32) {
                uint32_t v0[8], v1[8], v2[8];
                const uint32_t ta = tmem + ((uint32_t)r0 << 16) + (uint32_t)c;
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                    : "=r"(v0[0]), "=r"(v0[1]), "=r"(v0[2]), "=r"(v0[3]), "=r"(v0[4]), "=r"(v0[5]), "=r"(v0[6]),
                      "=r"(v0[7])
                    : "r"(ta));
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                    : "=r"(v1[0]), "=r"(v1[1]), "=r"(v1[2]), "=r"(v1[3]), "=r"(v1[4]), "=r"(v1[5]), "=r"(v1[6]),
                      "=r"(v1[7])
                    : "r"(ta + 128u));
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                    : "=r"(v2[0]), "=r"(v2[1]), "=r"(v2[2]), "=r"(v2[3]), "=r"(v2[4]), "=r"(v2[5]), "=r"(v2[6]),
                      "=r"(v2[7])
                    : "r"(ta + 256u));
                asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int b = c + j - ll * nk;
                    if (valid && b >= 0 && b < nk) {
                        // (hi, lo) += A0 + A1 + A2: A0 by an exact two-sum, the small rest into lo
                        const size_t i = ((size_t)l * nk + a) * nk + b;
                        const float x0 = __uint_as_float(v0[j]), hi = rowhi[i];
                        const float sum = hi + x0, bb = sum - hi;
                        const float err = (hi - (sum - bb)) + (x0 - bb);
                        const float rest = rowlo[i] + err + (__uint_as_float(v1[j]) + __uint_as_float(v2[j]));
                        const float nh = sum + rest;
                        rowhi[i] = nh;
                        rowlo[i] = rest - (nh - sum);
                    }
                }
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;");
    };
    // this CTA's rows -> the segment's FP64 accumulator
    auto flush = [&](int si) {
        __syncthreads();
        const BkSeg &sg = SEG(si);
        const int n = (HIP_LMAX + 1) * sg.n_k * sg.n_k;
        for (int i = tid; i < n; i += TC_THREADS) {
            const double v = (double)rowhi[i] + (double)rowlo[i];
            if (v != 0.0) atomicAdd(&sg.acc[i], v);
            rowhi[i] = rowlo[i] = 0.f;
        }
        __syncthreads();
    };

    if (s_lo < s_hi && tid == 0) prefetch(s_lo, 0);
    TcUnit cur;
    cur.s = -1;
    cur.t = 0;
    cur.sgn = 1;
    cur.si = -1;
    cur.nk = nk_max;
    cur.nv = 0;
    int sb = 0;
    bool have = advance(cur);
    if (have) {
        transform(cur, sb);
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;");
        issue(cur, sb);
    }
    while (have && ok) {
        TcUnit nxt = cur;
        const bool more = advance(nxt);
        if (more) transform(nxt, sb ^ 1);  // overlaps the MMAs of cur
        wait_mma();
        if (!ok) break;
        fold(cur);
        if (!more || nxt.si != cur.si) flush(cur.si);
        if (!more) break;
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;");
        sb ^= 1;
        cur = nxt;
        issue(cur, sb);
    }
    // wait (bounded) for this CTA's MMAs before freeing tensor memory
    if (n_commit > 0) tc_wait(&bars[2], (uint32_t)((n_commit - 1) & 1));
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols));
}

cudaError_t hip_bk_contract_tc(const BkSeg *segs, int n_segs, int n_stages, int nk_max, int *status, int max_grid,
                               int fold_prims, cudaStream_t st)
{
    (void)fold_prims;  // the exact split folds after every unit
    if (!hip_bk_tc_supported(nk_max)) return cudaErrorInvalidValue;
    if (n_stages < 1) return cudaSuccess;
    const int P = hip_bk_tc_stage_prims(nk_max);
    // the layout's alignment requirements, checked before any launch: operands
    // on 1024 bytes (descriptors), bulk-copy destinations and sizes on 16 bytes,
    // mbarriers on 8 bytes, all inside the opt-in shared memory
    const TcLayout lay = tc_layout(nk_max, P);
    int optin = 0, dev0 = 0;
    cudaGetDevice(&dev0);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev0);
    if (lay.slice % 1024 != 0 || lay.stg % 16 != 0 || lay.stg_bytes % 16 != 0 || lay.rows % 8 != 0 ||
        lay.bars % 8 != 0 || tc_smem_bytes(nk_max, P) + 2048 > (size_t)optin)
        return cudaErrorInvalidValue;
    const size_t smem = tc_smem_bytes(nk_max, P);
    cudaError_t e = cudaFuncSetAttribute(P == 8 ? k_bk_contract_tc<8> : k_bk_contract_tc<4>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int grid = sms;
    if (max_grid > 0 && grid > max_grid) grid = max_grid;
    if (grid > n_stages) grid = n_stages;
    const int per = (n_stages + grid - 1) / grid;
    grid = (n_stages + per - 1) / per;  // no CTA without stages
    if (P == 8)
        k_bk_contract_tc<8><<<grid, TC_THREADS, smem, st>>>(segs, n_segs, n_stages, nk_max, status);
    else
        k_bk_contract_tc<4><<<grid, TC_THREADS, smem, st>>>(segs, n_segs, n_stages, nk_max, status);
    return cudaGetLastError();
}

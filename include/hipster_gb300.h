/*
 * hipster_gb300 -- C ABI of the GB300 (sm_103a) small-scale spectrum estimators of
 * Philcox, "A Faster Fourier Transform? Computing Small-Scale Power Spectra and
 * Bispectra for Cosmological Simulations in O(N^2) Time" (arXiv:2005.01739).
 *
 * Every entry point takes plain pointers and sizes.  Positions and weights may
 * live in host memory or in device memory of the current CUDA device (detected
 * per pointer); results are always written to HOST memory, in float64.  The
 * library owns its scratch (cell lists, tables, partial sums) in a per-device
 * workspace that grows on demand and is reused across calls; calls are
 * serialised by a process-wide lock and are synchronous with respect to their
 * host outputs (they synchronise `cuda_stream` before returning).  Outputs are
 * written only when the call returns HIP_OK.
 *
 * Units: positions, L and R0 in Mpc/h; k-bin edges in h/Mpc.  Positions outside
 * [0, L) are wrapped periodically.
 */
#ifndef HIPSTER_GB300_H
#define HIPSTER_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    HIP_OK = 0,
    HIP_ERR_ARG = -1,       /* null pointer, bad size, unknown enum, odd ell_max for P */
    HIP_ERR_RANGE = -2,     /* L <= 0, R0 <= 0, R0 >= L/2, edges not strictly increasing or < 0, too many bins */
    HIP_ERR_NONFINITE = -3, /* a position or weight is NaN/Inf */
    HIP_ERR_CUDA = -4,      /* a CUDA runtime call failed (message via hip_last_error) */
    HIP_ERR_NOMEM = -5,     /* device workspace allocation failed */
    HIP_ERR_TIMEOUT = -6    /* a bounded device-side wait gave up */
} hip_status;

/* Pair-separation window W(r; R0).  The only window of the paper: Eq. window_defn
 * (Sec. 2), piecewise quartic, C^1, support r < R0. */
typedef enum { HIP_WINDOW_PHILCOX = 0 } hip_window;

/* Arithmetic of the pair kernels.  FP64: every per-pair and per-bin quantity in
 * double precision (the plain baseline).  MIXED: pair geometry, bin-averaged
 * Bessel functions and per-warp (moment pass: per-CTA) accumulation in FP32,
 * folded into FP64 every few ten thousand pairs; cross-warp reduction,
 * normalisation and the analytic random-pair terms in FP64. */
typedef enum { HIP_PREC_FP64 = 0, HIP_PREC_MIXED = 1 } hip_precision;

#define HIP_MAX_BINS 255

/* Power-spectrum multipoles of a periodic box, Sec. 3 of the paper:
 *
 *   P^a_l = (-i)^l (2l+1) / (n_w^2 V) * DD^a_l  -  delta_l0 W~^a(R0),
 *   DD^a_l = sum_{i in S} sum_{j != i, 0 < r_ij < R0} w_i w_j W(r_ij/R0) jbar^a_l(r_ij) L_l(mu_ij),
 *
 * (binned estimator following Eq. pk-binned; jbar from Eq. jla-def; W~^a from
 * Eq. wka-def; (-i)^l = (-1)^(l/2) for the even l computed here).  r_ij is the
 * minimum-image separation x_i - x_j, mu_ij its cosine to the `los_axis` axis,
 * n_w = (sum_i w_i) / L^3 over ALL particles, V = L^3.
 *
 *   pos        [N][3] float32, xyz interleaved (host or device)
 *   w          [N] float32 weights, or NULL for unit weights (host or device)
 *   N          number of particles, >= 1
 *   L, R0      box side and truncation radius, 0 < R0 < L/2
 *   window     HIP_WINDOW_PHILCOX
 *   k_edges    [n_k+1] float64 host, strictly increasing, k_edges[0] >= 0
 *   n_k        number of k bins, 1..HIP_MAX_BINS
 *   ell_max    0, 2 or 4; multipoles l = 0, 2, ..., ell_max are returned
 *   los_axis   0, 1 or 2 (line of sight; the paper uses a fixed axis for boxes)
 *   prec       HIP_PREC_FP64 or HIP_PREC_MIXED
 *   prim_begin, prim_end   primary range S = [prim_begin, prim_end) in input
 *              order (0, N for all).  Partial results over disjoint ranges add
 *              up to the full DD (for sharding over devices or processes).
 *   P_out      [(ell_max/2+1) * n_k] float64 host, row-major (l, a)
 *   DD_out     same shape, the unnormalised DD^a_l; may be NULL
 *   npairs_out number of ordered pairs (i in S, j) with 0 < r < R0; may be NULL
 *   cuda_stream  cudaStream_t to run on (NULL = legacy default stream)
 */
hip_status hip_power(const float *pos, const float *w, int64_t N, double L, double R0, hip_window window,
                     const double *k_edges, int n_k, int ell_max, int los_axis, hip_precision prec,
                     int64_t prim_begin, int64_t prim_end, double *P_out, double *DD_out, int64_t *npairs_out,
                     void *cuda_stream);

/* P^a_l from ordered pair sums DD^a_l that the caller has added up, e.g. the
 * DD_out of hip_power calls over disjoint primary ranges of one catalog run on
 * several devices or processes (their sum is the full DD of Sec. 3):
 *
 *   P^a_l = (-i)^l (2l+1) / (n_w^2 V) * DD^a_l  -  delta_l0 W~^a(R0),  n_w = S1 / L^3,
 *
 * the normalisation and W~^a (Eq. wka-def) of hip_power, in FP64 on the device.
 *
 *   DD         [(ell_max/2+1) * n_k] float64 host, row-major (l, a)
 *   n_k, ell_max, L, R0, window, k_edges   as for hip_power (the same values)
 *   S1         sum of the weights of the WHOLE catalog (N for unit weights), != 0
 *   P_out      [(ell_max/2+1) * n_k] float64 host
 *   cuda_stream  cudaStream_t to run on (NULL = legacy default stream)
 *
 * Returns HIP_ERR_ARG / HIP_ERR_RANGE for invalid arguments, HIP_ERR_NONFINITE
 * if DD holds a non-finite value; synchronises the stream. */
hip_status hip_power_from_pairs(const double *DD, int n_k, int ell_max, double L, double R0, hip_window window,
                                const double *k_edges, double S1, double *P_out, void *cuda_stream);

/* Isotropic bispectrum multipoles of a periodic box, Sec. 4 of the paper (the
 * summary estimator of Sec. 4.5):
 *
 *   B^ab_l = (-1)^l (2l+1) / (V n_w^3) * T^ab_l
 *            - delta_l0 (W~^a S^b + W~^b S^a) / (V n_w^2) + 2 delta_l0 W~^a W~^b,
 *   T^ab_l = sum_{i data} w_i G^ab_l(x_i) - (S1/N_r) sum_{r random} G^ab_l(x_r),
 *   G^ab_l(x) = 4pi/(2l+1) sum_m A^a_lm(x) A^b*_lm(x) - C^ab_l(x),
 *   A^a_lm(x) = sum_j w_j jbar^a_l(r) W(r/R0) Y_lm(rhat),  C^ab_l(x) = sum_j w_j^2 jbar^a_l jbar^b_l W^2,
 *
 * over data j with 0 < r = |x - x_j| < R0 (minimum image; j != i for a data
 * primary), Eq. AC-def binned as in Sec. 4.4; S^a = the ordered DD_0 pair sum of
 * hip_power (the DDR^I term, Sec. 4.3); the DDR^II term uses the random
 * catalog (f_rand = N_r / N); S1 = sum of data weights, n_w = S1 / L^3.
 *
 *   pos, w, N        data as in hip_power (w NULL = unit weights)
 *   rand_pos, N_r    [N_r][3] float32 uniform random positions (host or device), N_r >= 1
 *   L, R0, window    as in hip_power
 *   k_edges, n_k     as in hip_power, n_k <= 63 (MIXED) or <= 31 (FP64)
 *   lmax             0..4; multipoles l = 0..lmax are returned
 *   prec             HIP_PREC_FP64 or HIP_PREC_MIXED
 *   B_out            [(lmax+1) * n_k * n_k] float64 host, row-major (l, a, b); symmetric in a, b
 *   npairs_out       [2] or NULL: ordered (primary, data) pairs counted for data and
 *                    for random primaries
 *   cuda_stream      as in hip_power
 */
hip_status hip_bispectrum(const float *pos, const float *w, int64_t N, const float *rand_pos, int64_t N_r, double L,
                          double R0, hip_window window, const double *k_edges, int n_k, int lmax, hip_precision prec,
                          double *B_out, int64_t *npairs_out, void *cuda_stream);

/* A uniform random catalog in the box, for the DDR^II term's random catalog
 * (Sec. 4.3; the paper uses f_rand = N_r / N = 3, Sec. 9).  Coordinate d of
 * random j is out[3j + d] = fl(u * fl(L)), u = (z >> 40) * 2^-24 in [0, 1) with z
 * output 3j + d + 1 of SplitMix64 seeded with `seed` (the generator and
 * constants of hip_subsample); u is exact in float32 and the product is rounded
 * once (round to nearest), so the catalog is the same on every machine.  Every
 * value lies in [0, fl(L)): u fl(L) <= fl(L) - fl(L) 2^-24, more than half a
 * unit in the last place below fl(L) unless fl(L) is a power of two, where it
 * is a float.
 *
 *   out         [N_r][3] float32, host or device, caller-owned
 *   N_r         number of randoms, 0 .. 2e9 (0 writes nothing)
 *   L           box side (> 0, finite, below the float32 range)
 *   seed        generator seed
 *   cuda_stream stream to run on; the call returns after `out` is written
 * Errors: HIP_ERR_ARG (NULL out, N_r out of range), HIP_ERR_RANGE (L), HIP_ERR_CUDA. */
hip_status hip_uniform_randoms(float *out, int64_t N_r, double L, uint64_t seed, void *cuda_stream);

/* hip_bispectrum with a seeded random catalog instead of a caller-supplied one:
 * the N_r randoms are those hip_uniform_randoms(., N_r, L, rand_seed) writes,
 * generated on the device into a buffer the library keeps per device (grown on
 * demand, never freed before exit), then the same computation as hip_bispectrum
 * (identical results for the same randoms).  Calls through this entry point are
 * serialised on the host.  Arguments and errors as in hip_bispectrum, with
 * N_r >= 1 and rand_seed in place of rand_pos. */
hip_status hip_bispectrum_seeded(const float *pos, const float *w, int64_t N, int64_t N_r, uint64_t rand_seed,
                                 double L, double R0, hip_window window, const double *k_edges, int n_k, int lmax,
                                 hip_precision prec, double *B_out, int64_t *npairs_out, void *cuda_stream);

/* Anisotropic bispectrum multipoles about the line of sight zhat: the extension
 * proposed in the paper's conclusions (the sum over spherical harmonics of the
 * isotropic estimator replaced by a product of two harmonics of different
 * order).  The paper fixes no estimator; this one projects the triangle onto
 *
 *   S_{l1 l2 L}(u, v) = sum_m (l1 l2 L; m, -m, 0) y_{l1 m}(u) y_{l2 -m}(v),   y_lm = sqrt(4pi/(2l+1)) Y_lm,
 *
 * for the 18 combinations l1 <= l2 <= 4, l1 + l2 and L even, |l1 - l2| <= L <=
 * min(l1 + l2, 4), in this order: (0,0,0) (0,2,2) (0,4,4) (1,1,0) (1,1,2)
 * (1,3,2) (1,3,4) (2,2,0) (2,2,2) (2,2,4) (2,4,2) (2,4,4) (3,3,0) (3,3,2)
 * (3,3,4) (4,4,0) (4,4,2) (4,4,4); B^ba_{l2 l1 L} = B^ab_{l1 l2 L} gives the rest.
 *
 *   B^ab_{l1 l2 L} = (2l1+1)(2l2+1)(-1)^((l1+l2)/2) [ T / (V n_w^3)
 *        - d_{l2 0} d_{L l1} k_{l1} DD^a_{l1} W~^b / (V n_w^2) - d_{l1 0} d_{L l2} k_{l2} W~^a DD^b_{l2} / (V n_w^2)
 *        + 2 d_{l1 0} d_{l2 0} W~^a W~^b ],   k_l = (-1)^l / sqrt(2l+1),
 *   T = sum_{i data} w_i G(x_i) - (S1/N_r) sum_{r random} G(x_r),
 *   G(x) = sum_{j != k} w_j w_k W_j W_k jbar^a_{l1}(r_j) jbar^b_{l2}(r_k) S_{l1 l2 L}(rhat_j, rhat_k),
 *
 * DD^a_l the ordered power pair sum of hip_power about zhat.  (l, l, 0) equals
 * (-1)^l sqrt(2l+1) times hip_bispectrum's B_l.  Mixed precision only (the a_lm
 * pass of hip_bispectrum, the matching-m Gram of its per-primary A_lm with
 * compensated FP32 sums folded in FP64, FP64 C term and finalize).
 *
 *   arguments as for hip_bispectrum (no lmax, no precision); R0 k_max <= 768
 *   B_out      [18 * n_k * n_k] float64 host, row-major (combination, a, b)
 *   npairs_out [2] or NULL: data-primary and random-primary pairs
 * Errors as for hip_bispectrum. */
hip_status hip_bispectrum_aniso(const float *pos, const float *w, int64_t N, const float *rand_pos, int64_t N_r,
                                double L, double R0, hip_window window, const double *k_edges, int n_k, double *B_out,
                                int64_t *npairs_out, void *cuda_stream);

/* Isotropic bispectrum multipoles without a random catalog (App. A of the paper):
 * as hip_bispectrum, but the random primaries' term (S1/N_r) sum_r G(x_r) is
 * replaced by its expectation (S1/V) sum_{j != k} w_j w_k E^{II,ab}_l(r_jk), with
 * the kernel E^{II,ab}_l(r) = int p^2 dp/(2 pi^2) j_0(p r) omega^a_l(p) omega^b_l(p)
 * (omega^a_l of Eq. omega-ell-a-def), which vanishes beyond 2 R0.  The pair sum is
 * taken inside the p integral from a 16384-bin histogram of the separations below
 * 2 R0 that keeps the first two moments of r in each bin (FP64), so the result is
 * exact to third order in the bin width 2 R0 / 16384.
 *   pos, w, N, L, R0, window, k_edges, n_k, lmax, prec, B_out, cuda_stream  as in
 *                    hip_bispectrum (no randoms), except R0 < L/4 (HIP_ERR_RANGE)
 *   npairs_out       [1] or NULL: ordered (primary, data) pairs within R0
 */
hip_status hip_bispectrum_analytic(const float *pos, const float *w, int64_t N, double L, double R0,
                                   hip_window window, const double *k_edges, int n_k, int lmax, hip_precision prec,
                                   double *B_out, int64_t *npairs_out, void *cuda_stream);

/* The bispectrum's primary sum over chosen primaries, for sharding and sampled
 * checks: T_out = sum_{i in data range} w_i G^ab_l(x_i) - (S1/N_r) sum_{r in random
 * range} G^ab_l(x_r), with G as in hip_bispectrum (before the normalisation and
 * the analytic terms of Sec. 4.5).  prim_ranges = {d0, d1, r0, r1}: data
 * primaries [d0, d1) and random primaries [r0, r1) in input order (neighbours
 * are always all the data).  Partial sums over disjoint ranges add up to the
 * full T.  Other arguments, errors and npairs_out as in hip_bispectrum;
 * T_out is [(lmax+1) * n_k * n_k] float64 host. */
hip_status hip_bispectrum_partial(const float *pos, const float *w, int64_t N, const float *rand_pos, int64_t N_r,
                                  double L, double R0, hip_window window, const double *k_edges, int n_k, int lmax,
                                  hip_precision prec, const int64_t *prim_ranges, double *T_out, int64_t *npairs_out,
                                  void *cuda_stream);

/* One catalog of a batched bispectrum computation: the arguments of
 * hip_bispectrum for that catalog (host or device inputs; host outputs). */
typedef struct {
    const float *pos;      /* [N][3] float32 */
    const float *w;        /* [N] float32 or NULL */
    int64_t N;
    const float *rand_pos; /* [N_r][3] float32 */
    int64_t N_r;
    double L, R0;
    const double *k_edges; /* [n_k+1] host */
    int n_k, lmax;
    double *B_out;         /* [(lmax+1) * n_k * n_k] host */
    int64_t *npairs_out;   /* [2] or NULL */
} hip_bcatalog;

/* Batched bispectra (the estimator of hip_bispectrum, Sec. 4, for many
 * catalogs of uneven N, L, R0 and bins).  Every catalog's cell lists and its
 * l = 0 pair sum S^a are built first; then ONE persistent kernel launch runs the
 * primaries of all catalogs (work items of 32 primaries, the catalogs' items laid
 * end to end), accumulating each catalog's primary sums in FP64; a FP64 finalize
 * per catalog follows.  Per catalog the result equals hip_bispectrum's up to the
 * order of the FP32 / FP64 sums.  All catalogs must satisfy hip_bispectrum's
 * argument rules (n_k <= 63 MIXED, <= 31 FP64); errors as in hip_bispectrum (the
 * first failing catalog decides).  The call synchronises cuda_stream once after
 * the cell builds and once at the end.  1 <= n_cats <= 4096. */
hip_status hip_bispectrum_batched(const hip_bcatalog *cats, int n_cats, hip_precision prec, void *cuda_stream);

/* One catalog of a batched power-spectrum computation: the arguments of
 * hip_power for that catalog (host or device inputs; host outputs). */
typedef struct {
    const float *pos;    /* [N][3] float32 */
    const float *w;      /* [N] float32 or NULL */
    int64_t N;
    double L, R0;
    const double *k_edges; /* [n_k+1] host */
    int n_k;
    int ell_max, los_axis;
    int64_t prim_begin, prim_end;
    double *P_out;       /* [(ell_max/2+1) * n_k] host */
    double *DD_out;      /* same shape or NULL */
    int64_t *npairs_out; /* or NULL */
} hip_catalog;

typedef struct hip_batch_plan hip_batch_plan;

/* Batched power spectra (the estimator of hip_power, Sec. 3, for many catalogs):
 * the catalogs' cell builds, ONE persistent pair-pass launch over all of their
 * work items (the Legendre-moment pass, with one batched FP64 contraction, when
 * every catalog has R0 k_max <= 1024; else the direct pass), and the FP64
 * finalize are recorded into a CUDA graph at plan creation and replayed by
 * hip_batch_plan_run.  Catalogs may differ in N, L, R0, bins, ell_max and line
 * of sight.
 *
 * hip_batch_plan_create: validates every catalog (HIP_ERR_ARG/RANGE as in
 *   hip_power; hip_batch_message() names the catalog), allocates the plan's
 *   device memory and pinned output mirror, records and instantiates the graph
 *   (capturing on `cuda_stream`).  The hip_catalog array is copied; the data and
 *   output pointers it holds must stay valid for the plan's lifetime.
 * hip_batch_plan_run: copies host-resident inputs into the plan, replays the
 *   graph, synchronises `cuda_stream` and writes every catalog's outputs;
 *   device-resident inputs are read in place (their current contents).
 *   HIP_ERR_NONFINITE if a catalog has a non-finite position or weight.
 * hip_power_batched: create + run + destroy in one call.
 * hip_batch_plan_launches: number of kernel launches recorded in the graph. */
hip_status hip_batch_plan_create(const hip_catalog *cats, int n_cats, hip_precision prec, hip_batch_plan **plan,
                                 void *cuda_stream);
hip_status hip_batch_plan_run(hip_batch_plan *plan, void *cuda_stream);

/* Autotuner of a plan's cell shape (no counterpart in the paper, whose CPU code
 * picks cells by hand): a batched catalog uses cells at least R0 wide and, when
 * it is sparse, fewer of them, about one per `occ` particles (more particles per
 * work item, fewer empty items).  hip_batch_plan_tune rebuilds the plan for occ
 * in {4, 8, 16, 32, 64, 128, 256} and for cells exactly R0 wide (reported as
 * 0), replays each once after a warm-up (the catalogs' inputs must be valid;
 * their outputs are overwritten), and keeps the fastest.  chosen_out (or NULL)
 * receives the chosen occ; ms_out (or NULL) receives the eight replay times in
 * that order, in ms.  A new plan starts at occ = 64.  Errors as in
 * hip_batch_plan_run. */
hip_status hip_batch_plan_tune(hip_batch_plan *plan, void *cuda_stream, int *chosen_out, float *ms_out);
/* The second stage of the autotuner, at the plan's current cell occupancy: the
 * moment pass's warps per CTA (4, 8) and the number of pairs a CTA adds to its
 * FP32 moment sums between folds into FP64 (4096, 8192, 16384), each of the six
 * shapes timed on one replay after a warm-up, in that order (warps outer) into
 * ms_out[6] (or NULL); the fastest is kept and reported through warps_out and
 * fold_out (or NULL).  A new plan starts with warps chosen from its cells'
 * occupancy and folds every 16384 pairs.  The tile of 128 particles per cell
 * and the 32-pair drains are fixed.  Errors as in hip_batch_plan_run.
 * hip_batch_plan_shape reports the plan's current occ, warps (0 = by
 * occupancy) and fold (0 = 16384). */
hip_status hip_batch_plan_tune_kernel(hip_batch_plan *plan, void *cuda_stream, int *warps_out, int *fold_out,
                                      float *ms_out);
void hip_batch_plan_shape(const hip_batch_plan *plan, int *occ, int *warps, int *fold);
void hip_batch_plan_destroy(hip_batch_plan *plan);
int hip_batch_plan_launches(const hip_batch_plan *plan);
hip_status hip_power_batched(const hip_catalog *cats, int n_cats, hip_precision prec, void *cuda_stream);
const char *hip_batch_message(void);

/* hip_power without any device allocation (no counterpart in the paper: this is
 * a property of the library, not of the estimator).
 *
 * Same arguments, results and errors as hip_power with prec = HIP_PREC_MIXED,
 * but all scratch lives in one statically sized device array of
 * hip_noalloc_capacity() bytes (64 MiB) that every device loading the library
 * reserves until the process exits; no cudaMalloc/cudaFree or other allocating
 * routine is called.  It is for callers that cannot allocate device memory
 * while they run: a host application whose own memory pool has already
 * reserved the device's memory (a library cudaMalloc would fail or take memory
 * the pool counts on), or a service that must know its peak device footprint
 * before it starts.  The call is eager and synchronising, like hip_power: it
 * reads an error word back to the host after the cell build and synchronises
 * `cuda_stream` before returning.
 *
 * Limit: the call needs about 24 bytes per particle for device-resident inputs
 * (36 for host positions, 40 with host weights), plus cell tables and per-CTA partial sums; a call that
 * would not fit returns HIP_ERR_RANGE and hip_noalloc_message() says how many
 * bytes it needed.  The array's device address is looked up on the first call
 * made with each device current.  Every call shares the array (it keeps the previous call's
 * contents; each call clears what must start at zero); calls that overlapped
 * on the GPU would race on it, so this entry point serialises its calls and
 * synchronises `cuda_stream` before returning, on success and on failure.
 * hip_noalloc_message() holds the reason for the last failing call (empty after
 * a successful one). */
hip_status hip_power_noalloc(const float *pos, const float *w, int64_t N, double L, double R0, hip_window window,
                             const double *k_edges, int n_k, int ell_max, int los_axis, int64_t prim_begin,
                             int64_t prim_end, double *P_out, double *DD_out, int64_t *npairs_out, void *cuda_stream);
size_t hip_noalloc_capacity(void);
const char *hip_noalloc_message(void);

/* The binned window kernel of the pair-separation window (Eq. omega-ell-a-def):
 *
 *   omega^a_l(p) = 4 pi int_0^R0 r^2 j_l(p r) jbar^a_l(r) W(r/R0) dr,
 *
 * which carries the window convolution and the Poisson/Gaussian covariance of
 * the estimators (Sec. 6) and the random-free DDR^II term (App. A), in FP64:
 * composite 16-point Gauss-Legendre in r on the three polynomial pieces of W,
 * panels no wider than pi / max(p_max, k_hi).
 *
 *   k_edges, n_k   bins as in hip_power (host)
 *   R0             truncation radius, > 0
 *   lmax           0..4: l = 0 .. lmax are returned
 *   p, n_p         [n_p] wavenumbers >= 0 (host), 1 <= n_p <= 2^20
 *   omega_out      [(lmax+1)][n_k][n_p] float64 host, row-major (l, a, q)
 *   cuda_stream    stream to run on; the call returns after omega_out is written
 * Errors: HIP_ERR_ARG (NULL arrays, n_p or lmax out of range), HIP_ERR_RANGE
 * (R0, edges or p invalid), HIP_ERR_NOMEM, HIP_ERR_CUDA. */
hip_status hip_window_omega(const double *k_edges, int n_k, double R0, int lmax, const double *p, int n_p,
                            double *omega_out, void *cuda_stream);

/* Random subsample of a catalog (Sec. 9: at fixed R0 the estimators cost N^2,
 * so large catalogs, matter particles in the paper, are counted on a random
 * fraction 1/f_sub of their tracers; the estimators then apply unchanged, with
 * the subsample's own n_w).  Particle i is kept iff (z_i >> 11) <
 * floor(fraction 2^53), z_i the i-th output of SplitMix64 seeded with `seed`
 * (z = seed + (i+1) 0x9E3779B97F4A7C15, z ^= z >> 30, z *= 0xBF58476D1CE4E5B9,
 * z ^= z >> 27, z *= 0x94D049BB133111EB, z ^= z >> 31); kept particles keep
 * their input order.  Exact: the same selection on every machine.
 *
 *   pos, w      inputs as in hip_power (w NULL: no weights are written)
 *   N           number of particles, 0 .. 2e9
 *   fraction    kept fraction, 0 <= fraction <= 1 (1 keeps all)
 *   seed        generator seed
 *   pos_out     [N][3] float32, host or device, caller-owned (room for N)
 *   w_out       [N] float32 or NULL (ignored when w is NULL)
 *   n_out       number of particles kept (host)
 *   cuda_stream stream to run on; the call returns after the outputs are written
 * Errors: HIP_ERR_ARG (NULL pos, pos_out or n_out, N out of range),
 * HIP_ERR_RANGE (fraction outside [0, 1] or not finite), HIP_ERR_CUDA. */
hip_status hip_subsample(const float *pos, const float *w, int64_t N, double fraction, uint64_t seed, float *pos_out,
                         float *w_out, int64_t *n_out, void *cuda_stream);

/* Stage timing of the most recent hip_power call on this process, for
 * measurement.  When enabled (on != 0), each call records CUDA events on its
 * stream around its stages; hip_stage_times then writes, in milliseconds,
 *   ms[0] input upload (0 for device-resident inputs),  ms[1] cell-list build,
 *   ms[2] pair pass (the pair kernel; for the moment pass also its FP64
 *         coefficient and contraction kernels),  ms[3] FP64 finalize (W~,
 *         reduction, normalisation),
 *   ms[4] result download,
 * for the first min(n, 5) entries.  Returns the number of entries written
 * (0 if profiling was off during the last call).  Not thread-safe with
 * respect to concurrent calls (calls are serialised anyway). */
void hip_set_profiling(int on);
int hip_stage_times(double *ms, int n);

/* Stage timing of the most recent bispectrum primary sum (hip_bispectrum,
 * hip_bispectrum_partial, hip_bispectrum_analytic, hip_bispectrum_batched) with
 * profiling on: ms[0] the a_lm pass (per-primary A^a_lm and the C-term moments
 * of Eq. AC-def), ms[1] the contraction sum_p s_p sum_m A^a_lm A^b_lm (tensor
 * cores on the mixed path), both summed over the call's chunks of primaries,
 * ms[2] the C terms, ms[3] the number of chunks.  Writes min(n, 4) entries and
 * returns that number (0 if profiling was off during the last such call). */
int hip_bispectrum_stage_times(double *ms, int n);

/* The pair pass hip_power uses for these arguments (k_max = k_edges[n_k]):
 *   0  direct: every bin edge's function k^3 F_l(r k) (App. C) evaluated per pair;
 *   1  Legendre moments: per separation interval of width R0/n_c,
 *      n_c = max(8, ceil(R0 k_max / 4)), the pair loop sums omega L_l P_m(t)
 *      for m < 16 (t the position in the interval), and the edge sums are the
 *      FP64 contraction of those moments with the edge functions' Legendre
 *      coefficients (truncation below 1e-12 relative: the same edge sums).
 * The moment pass is taken while n_c <= 256 and its shared-memory array fits
 * (R0 k_max <= 1024).  Returns -1 for invalid arguments (R0 <= 0, k_max <= 0,
 * unknown prec). */
int hip_power_pair_pass(double R0, double k_max, hip_precision prec);

/* Human-readable name of a status code (static string). */
const char *hip_status_string(hip_status s);

/* Text of the last CUDA error seen by this thread's most recent failing call
 * (static thread-local buffer; empty if none). */
const char *hip_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* HIPSTER_GB300_H */

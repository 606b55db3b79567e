/*
 * bv.h -- C ABI of the GB300-native block-Vecchia Gaussian-process library.
 *
 * The library evaluates the block-Vecchia approximation of the Gaussian log-likelihood
 * (Pan, Abdulah, Genton, Sun, "Block Vecchia Approximation for Scalable and Efficient
 * Gaussian Process Computations", arXiv 2410.04477):
 *
 *   ell(theta) = sum_i log p(y_{B_i} | y_{NN_i})                      (Eq. 4)
 *
 * over K-means blocks B_i taken in a random block order, each conditioned on the m_i
 * nearest points of earlier blocks, with the Matern covariance of Eq. 5 plus a nugget.
 * The per-block steps are those of Algorithm 1; the library computes them fused on the
 * GPU (sm_103a).
 *
 * Conventions (all entry points):
 *   - Return value: a bv_status code (BV_OK = 0).  bv_strerror() describes it.
 *   - Pointers are host pointers unless an argument says "device".  The caller owns
 *     every buffer it passes; the library copies inputs in and writes outputs to the
 *     caller's buffers.  The context owns all device memory it allocates and frees it
 *     in bv_destroy().
 *   - Work is issued on the context's stream (the one given to bv_create, or a stream
 *     the context creates).  Calls marked "synchronous" return after the stream drains.
 *   - A context is not thread-safe: calls on one context must not overlap.
 *   - Indices are 0-based.  Point indices refer to the rows of the location array.
 */
#ifndef BV_H
#define BV_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bv_ctx bv_ctx;

/* Covariance parameters theta = (sigma^2, beta, nu) of Eq. 5, plus an absolute nugget
 * tau^2 added to the diagonal (the same observation with itself).  With aniso = 0 the
 * range is range[0] and distances are Euclidean (Eq. 5); with aniso = 1 the scaled
 * distance is sqrt(sum_k ((s_ik - s_jk) / range[k])^2).  Supported smoothness: nu in
 * {0.5, 1.5, 2.5} (the paper's low / medium / high smoothness, Sec. 3.1). */
typedef struct bv_theta {
    double sigma2;
    double range[3];
    double nu;
    double nugget;
    int32_t aniso;
    int32_t reserved;
} bv_theta;

typedef enum bv_status {
    BV_OK = 0,
    BV_EINVAL = 1,    /* invalid argument (size, pointer, theta outside its domain)      */
    BV_ENOMEM = 2,    /* device or host allocation failed                                 */
    BV_ECUDA = 3,     /* a CUDA runtime call failed (bv_last_cuda_error has the text)     */
    BV_ENOTPD = 4,    /* a block's covariance was not positive definite; ell = -inf       */
    BV_ETIMEOUT = 5,  /* reserved: no entry point waits on the device with a time limit,
                         so none returns it; the value stays assigned so that codes keep
                         their meaning                                                    */
    BV_ESTATE = 6,    /* call out of order (e.g. no data, no blocks, no neighbours yet)   */
    BV_EINTERNAL = 7  /* internal consistency check failed                                */
} bv_status;

typedef enum bv_precision {
    BV_FP64 = 0,  /* every step in FP64                                                    */
    BV_MIXED = 1  /* covariance generation, triangular solves and Schur-complement updates
                     in FP32; log-determinant and quadratic form accumulated in FP64; an
                     FP64 check keeps every dataset's relative error within a stated
                     bound by recomputing its worst-conditioned blocks in FP64
                     (bv_mixed_check_info, bv_set_mixed_tolerance)                       */
} bv_precision;

/* ---- context -------------------------------------------------------------------- */

/* Create a context on CUDA device `device`.  `cuda_stream` is a cudaStream_t to issue
 * work on, or NULL for a stream owned by the context. */
int bv_create(bv_ctx** out, int device, void* cuda_stream);
void bv_destroy(bv_ctx* ctx);
const char* bv_strerror(int status);
/* Text of the last failing CUDA call in this process (empty if none). */
const char* bv_last_cuda_error(void);

/* ---- data ----------------------------------------------------------------------- */

/* One dataset: n locations s_1..s_n in R^d (row-major n x d, d in 1..3) and the
 * observations y (length n, zero-mean model, Sec. 1; may be NULL and set later).
 * Synchronous.  Replaces any previous data and drops blocks and neighbours. */
int bv_set_data(bv_ctx* ctx, const double* locs, const double* y, int64_t n, int32_t d);

/* Several independent datasets evaluated together (one batched launch).  Dataset k has
 * n_per[k] points; `locs` (sum n_per x d, row-major) and `y` (sum n_per, may be NULL)
 * hold the datasets one after another.  Point indices in all later calls are global
 * (into the concatenation). */
int bv_set_datasets(bv_ctx* ctx, int32_t ndatasets, const int64_t* n_per,
                    const double* locs, const double* y, int32_t d);

/* Replace the observations (all datasets, concatenated).  `y` is a host pointer, or a
 * device pointer when y_on_device != 0 (then the copy is asynchronous on the stream).
 * A host y with a NaN or infinite entry returns BV_EINVAL and leaves the observations
 * unchanged (bv_set_data / bv_set_datasets check y and the locations the same way); a
 * device y is not inspected, and a non-finite entry there makes the evaluation's ell
 * -inf with BV_ENOTPD. */
int bv_set_observations(bv_ctx* ctx, const double* y, int32_t y_on_device);

/* ---- preprocessing (one-time; excluded from the timed evaluation, Sec. 3.1) ------ */

/* K-means blocks (Sec. 2.1; Algorithm 1 "Clustering" and "Block permutation"):
 * k-means++ seeding and `lloyd_iters` Lloyd iterations into bc clusters, empty clusters
 * dropped, then a random block order zeta.  Deterministic in (locations, bc, seed,
 * lloyd_iters); bit-identical to the reference definition (exact-integer centroid sums,
 * squared distances without fused multiply-add, lowest-index ties).  Outputs (may be
 * NULL): block_ptr[bc_eff+1] and point_idx[n] in block order (block p holds
 * point_idx[block_ptr[p] .. block_ptr[p+1]), ascending point index inside a block);
 * *bc_eff the number of non-empty blocks.  Synchronous. */
int bv_build_blocks(bv_ctx* ctx, int64_t bc, uint64_t seed, int32_t lloyd_iters,
                    int64_t* block_ptr, int32_t* point_idx, int64_t* bc_eff);

/* Multi-dataset form: dataset k gets bc_per[k] clusters (seeded with seed + k).
 * bc_eff_per[k] (may be NULL) receives its number of blocks.  Blocks are stored dataset
 * after dataset. */
int bv_build_blocks_multi(bv_ctx* ctx, const int64_t* bc_per, uint64_t seed,
                          int32_t lloyd_iters, int64_t* bc_eff_per);

/* Block orderings (Sec. 2.1; compared by KL divergence in Sec. 3.1). */
enum { BV_ORDER_RANDOM = 0, BV_ORDER_MAXMIN = 1, BV_ORDER_MORTON = 2, BV_ORDER_KDTREE = 3,
       BV_ORDER_HILBERT = 4 };

/* Place the context's blocks (one dataset) in a new order chosen from their centroids,
 * ties to the lower current position; neighbour sets must be selected again.
 *   RANDOM   Fisher-Yates over the current positions, block-permutation stream of seed
 *   MAXMIN   first the block whose centroid is nearest the mean centroid, then repeatedly
 *            the block farthest (largest smallest squared distance) from those placed
 *   MORTON   Z-order of the centroids scaled to 21-bit integers over their bounding box
 *            (q = min(2^21-1, floor((c - lo) / (hi - lo) 2^21)); bit b of axis k at b d + k)
 *   KDTREE   recursive median split, axis = depth mod d, sorted by (coordinate, position),
 *            the first floor(|S|/2) first
 *   HILBERT  Hilbert index of the same integers (Skilling's transform; levels from the
 *            most significant, axis 0 first)
 * Outputs (may be NULL): block_ptr[bc+1], point_idx[n] in the new order. */
int bv_order_blocks(bv_ctx* ctx, int32_t order, uint64_t seed, int64_t* block_ptr, int32_t* point_idx);

/* Classic Vecchia (Sec. 1: the special case of blocks of size 1): every point its own
 * block, the blocks in a random order (Fisher-Yates over the n points with the stream of
 * bv_build_blocks' block permutation), each singleton's query point for
 * bv_select_neighbors the point itself.  Outputs as bv_build_blocks (n + 1 and n
 * entries; may be NULL).  One dataset. */
int bv_build_singletons(bv_ctx* ctx, uint64_t seed, int64_t* block_ptr, int32_t* point_idx);

/* Caller-supplied partition (Algorithm 1 input g and zeta) for the single-dataset case:
 * bc blocks in the order to evaluate, block_ptr[bc+1], point_idx[n] (a permutation of
 * 0..n-1), centroids[bc x d] (the query points of the neighbour search; NULL = member
 * means). */
int bv_set_blocks(bv_ctx* ctx, int64_t bc, const int64_t* block_ptr, const int32_t* point_idx,
                  const double* centroids);

/* Block nearest neighbours (Sec. 2.2; Algorithm 1 "Nearest neighbors"): for the block at
 * position i, the m_i points of blocks 0..i-1 nearest to its centroid, keyed by
 * (squared distance, point index), m_i = min(m or m_per_block[i], available points).
 * Bit-identical to the reference definition.  Outputs (may be NULL): nn_ptr[bc_eff+1]
 * and nn_idx[nn_ptr[bc_eff]] (ascending key order inside a block).  Synchronous. */
int bv_select_neighbors(bv_ctx* ctx, int32_t m, const int32_t* m_per_block,
                        int64_t* nn_ptr, int32_t* nn_idx);

/* Caller-supplied conditioning sets (Algorithm 1 input m_1..m_bc with the sets). */
int bv_set_neighbors(bv_ctx* ctx, const int64_t* nn_ptr, const int32_t* nn_idx);

/* Sizes of the current structure: number of blocks and total conditioning entries. */
int bv_get_sizes(bv_ctx* ctx, int64_t* n_blocks, int64_t* n_nn_entries);

/* Copy the current structure out (any pointer may be NULL). */
int bv_get_blocks(bv_ctx* ctx, int64_t* block_ptr, int32_t* point_idx, double* centroids);
int bv_get_neighbors(bv_ctx* ctx, int64_t* nn_ptr, int32_t* nn_idx);

/* ---- evaluation (the hot path) -------------------------------------------------- */

/* Block-Vecchia log-likelihood (Eq. 4 by Algorithm 1) of dataset 0 at theta.
 * out_loglik: the scalar ell.  out_per_block (may be NULL): the bc_eff per-block
 * conditional log-likelihoods.  On a non-positive-definite block returns BV_ENOTPD and
 * sets *out_loglik = -INFINITY.  Synchronous. */
int bv_loglik(bv_ctx* ctx, const bv_theta* theta, int32_t precision, double* out_loglik,
              double* out_per_block);

/* The two terms of ell for dataset 0: ell = -(quad + logdet + n log 2 pi) / 2, with
 * quad = y^T Sigma~^{-1} y = sum_i u_i and logdet = log |Sigma~| = sum_i d_i (Algorithm 1's
 * u_i and d_i summed over blocks).  Because every block's conditional covariance scales
 * with sigma^2 while its kriging weights do not, quad at sigma^2 = 1 gives the profile
 * estimate sigma^2 = quad / n for a fixed range and nugget-to-sigma^2 ratio (used by
 * bv_mle).  Any output pointer but out_loglik may be NULL.  Synchronous. */
int bv_loglik_terms(bv_ctx* ctx, const bv_theta* theta, int32_t precision, double* out_loglik,
                    double* out_quad, double* out_logdet);

/* The exact Gaussian log-likelihood, Eq. 1, of dataset 0 (n <= 65536) by a dense tiled
 * FP64 Cholesky factorisation on the device (memory: about 4 (n+1)^2 bytes, freed on
 * return).  use_y = 0 evaluates at y = 0 (as the KL divergence of Sec. 3.1 needs); else
 * the context's observations.  Outputs (any but none required): ell, quad = y^T Sigma^-1 y,
 * logdet = log|Sigma|.  BV_ENOTPD if Sigma is not positive definite.  Synchronous. */
int bv_exact_loglik(bv_ctx* ctx, const bv_theta* theta, int32_t use_y, double* out_loglik,
                    double* out_quad, double* out_logdet);

/* Leading-term flops of one bv_exact_loglik on n points ((n+1)^3/3 + (n+1)^2). */
int bv_exact_flops(int64_t n, double* flops);

/* KL divergence of the block-Vecchia approximation from the exact GP (Eq. 7, Sec. 3.1):
 * KL = ell_0(theta; 0) - ell_a(theta; 0) = (log|Sigma_a| - log|Sigma_0|) / 2, with the
 * exact log-determinant from bv_exact_loglik and the approximate one from the context's
 * blocks and neighbour sets (bv_loglik_terms in `precision`).  Without observations the
 * context's y is set to zeros.  Outputs: kl, and (may be NULL) both log-determinants. */
int bv_kl_divergence(bv_ctx* ctx, const bv_theta* theta, int32_t precision, double* out_kl,
                     double* out_logdet_exact, double* out_logdet_approx);

/* ell and the quadratic form of every dataset (host arrays of ndatasets; out_quad may be
 * NULL); as bv_loglik_multi otherwise. */
int bv_loglik_terms_multi(bv_ctx* ctx, const bv_theta* thetas, int32_t precision, double* out_loglik,
                          double* out_quad);

/* All datasets at once: thetas[ndatasets] (host), out_loglik[ndatasets] (host).
 * Synchronous. */
int bv_loglik_multi(bv_ctx* ctx, const bv_theta* thetas, int32_t precision,
                    double* out_loglik);

/* Asynchronous form for callers that keep the result on the device: enqueues one
 * evaluation of every dataset on the context's stream and writes ell to
 * d_out_loglik[ndatasets] (device).  No host synchronisation; status is checked by the
 * next synchronous call or bv_sync().  The enqueued sequence is a CUDA graph captured
 * on first use for each precision. */
int bv_loglik_async(bv_ctx* ctx, const bv_theta* thetas, int32_t precision,
                    double* d_out_loglik);

/* Blocks of the last mixed-precision evaluation whose FP32 factorisation broke down (a
 * non-positive pivot) and that were recomputed in FP64 within the same evaluation; only
 * a block that also fails in FP64 makes ell -inf. */
int bv_mixed_fallbacks(bv_ctx* ctx, int64_t* count);

/* The error check of the last mixed-precision evaluation.  The FP32 error of a block's
 * term is modelled as r_i eps B_i: eps = 2^-24, B_i the block's error weight
 * (bv_mixed_block_indicator) and r_i independent, zero-mean, of a scale rho that depends
 * on the dataset.  Every dataset recomputes a fixed sample of its blocks in FP64 (all
 * blocks of a dataset with fewer than 64; else max(64, ceil(B/256)) of its B blocks at
 * evenly spaced positions of the random block order); the sample gives rho (the RMS of
 * delta_i / (eps B_i), delta_i the FP32 minus FP64 term), a test for a systematic bias
 * (|mean| over 4 standard errors: the whole dataset is recomputed in FP64); L is the sum
 * of the dataset's terms (FP32 and sampled FP64).  The bound on the dataset's relative
 * error is 3 x 2.5 rho eps sqrt(sum B_i^2) / |L| over the blocks still in FP32 (three
 * standard deviations of their summed noise; the margin of 2.5 on the sampled rho covers
 * its sampling error and a small conditioning-dependent mean of the errors that cancels
 * over a dataset but not over its well-conditioned blocks); while it exceeds the
 * tolerance (bv_set_mixed_tolerance, default 1e-6) the blocks with the largest B_i are
 * recomputed in FP64 in the same evaluation.  The sampled blocks always keep their FP64
 * terms.  Outputs: *blocks_fp64 = blocks whose terms came from FP64 (sampled and
 * recomputed; not counting the FP32-breakdown fallback of bv_mixed_fallbacks);
 * *datasets_touched (may be NULL) = datasets with any block recomputed beyond the
 * sample; est_rel[ndatasets] (may be NULL) = each dataset's final bound (0 when every
 * block was sampled, +inf when a sampled block failed in FP64 or a bias was found).
 * Synchronous.  BV_ESTATE before the first mixed evaluation; all zero with the check off. */
int bv_mixed_check_info(bv_ctx* ctx, int64_t* blocks_fp64, int32_t* datasets_touched, double* est_rel);

/* The bound the mixed-precision check enforces (default 1e-6); 0 switches the check off
 * (FP32 throughout, only blocks whose FP32 factorisation breaks down are recomputed in
 * FP64).  Takes effect at the next evaluation.  BV_EINVAL unless 0 <= tol < 1. */
int bv_set_mixed_tolerance(bv_ctx* ctx, double tol);

/* Per-block error weight of the last mixed-precision evaluation (nblocks floats): the
 * block's conditioning indicator -- the sum over the N = m_i + b_i pivots of its FP32
 * factorisation of (sigma^2 + tau^2) / pivot, i.e. of each point's variance over its
 * conditional variance given the points before it -- times 1 + u_i / b_i (u_i the
 * block's quadratic form).  The FP32 rounding error of the block's term grows with it;
 * 0 for a block recomputed in FP64 after an FP32 breakdown.  Synchronous.  BV_ESTATE
 * before the first mixed evaluation. */
int bv_mixed_block_indicator(bv_ctx* ctx, float* out);

/* First failing block (not positive definite) of the last synchronous evaluation, or -1. */
int bv_last_error_block(bv_ctx* ctx, int64_t* block);

/* Wait for the context's stream; report any device-side failure since the last check
 * (BV_ENOTPD with the first failing block in *failed_block, may be NULL). */
int bv_sync(bv_ctx* ctx, int64_t* failed_block);

/* FP64 log-likelihood for callers that cannot allocate device memory.  The paper has no
 * counterpart: this is a deployment form of bv_loglik.  Some callers may not call
 * cudaMalloc at all: code running inside a host callback or another library's
 * stream-ordered section, under a memory manager that owns every device allocation, or
 * in a latency-bound loop that cannot afford an allocation's implicit synchronisation.
 * This entry point allocates nothing: the caller passes every input and output as a
 * device pointer, and the per-block partial results live in a static device array of
 * BV_NOALLOC_MAX_BLOCKS + 32 doubles (about 8 MiB) that each GPU loading the library
 * keeps until the process exits.
 *   d_locs: SoA coordinates, d_locs[k * n + j] = coordinate k of point j (d in 1..3);
 *   d_y[n]; d_block_ptr[bc+1], d_point_idx[n], d_nn_ptr[bc+1], d_nn_idx[d_nn_ptr[bc]]:
 *   the block and conditioning structure as produced by bv_build_blocks /
 *   bv_select_neighbors; d_out_loglik[1] receives ell; d_out_per_block[bc] (may be NULL)
 *   the per-block terms.  cuda_stream: the stream to use (NULL = legacy default stream).
 * Limits: bc <= BV_NOALLOC_MAX_BLOCKS, and every block's m_i + b_i at most 235 (d = 1),
 * 234 (d = 2) or 233 (d = 3).  A first small kernel reads the two pointer arrays to find
 * the largest m_i + b_i and to check them (both start at 0, neither decreases,
 * d_block_ptr[bc] <= n); a size beyond the limit or a malformed structure returns
 * BV_EINVAL before the likelihood kernel runs.  A point or neighbour index outside
 * [0, n) is recorded by the likelihood kernel without being read and also returns
 * BV_EINVAL.  Every call waits for its stream to drain (it reads these checks and the
 * failure word back to the host) and returns BV_ENOTPD as bv_loglik does.
 * The first call made with a device current looks up the array's device address for
 * that device: make that first call outside any stream capture.  Every call reuses the
 * same array (its status words are reset at the start of each call, its per-block
 * entries are rewritten), so calls whose work overlaps on the GPU -- different streams
 * or host threads without synchronisation -- race and must be serialised by the caller. */
#define BV_NOALLOC_MAX_BLOCKS 1048576
int bv_loglik_noalloc(const bv_theta* theta, const double* d_locs, const double* d_y, int64_t n,
                      int32_t d, int64_t bc, const int64_t* d_block_ptr, const int32_t* d_point_idx,
                      const int64_t* d_nn_ptr, const int32_t* d_nn_idx, double* d_out_loglik,
                      double* d_out_per_block, void* cuda_stream);

/* Run the launch-shape autotuner for `precision` now (otherwise it runs on first use).
 * Times each candidate of every size bin on the current structure and the current
 * parameters -- the theta of the last evaluation, or sigma^2 = 1, range 0.1, nu = 1/2,
 * tau^2 = 1e-3 if none has run; the kernels' cost depends on the Matern form, so an
 * evaluation at representative parameters first (which tunes on first use) gives the
 * better plan.  Candidates: one CTA per block with 96, 160, 288 or 544 threads (FP64 with
 * one- or two-column factorisation steps, and 1024 threads for N >= 128), one warp per
 * block with 2, 4 or 8 warps per CTA for small blocks (FP64 N <= 64, mixed N <= 128), the
 * tensor-core form for mixed N >= 64; then the whole evaluation with the size bins as
 * parallel branches or in sequence.  The graph of an evaluation is timed against the
 * same launches issued directly on first use, and the faster is kept.  The environment
 * variable BV_KERNEL_FORM=cta, cta2, warp or tc restricts the candidates to one form.
 * Every form does the same per-block arithmetic, so the choice changes speed only (the
 * FP64 result is bit-identical across re-tuned plans).  Errors: BV_EINVAL (precision),
 * BV_ESTATE (no neighbours selected yet), BV_ECUDA. */
int bv_autotune(bv_ctx* ctx, int32_t precision);

/* Launch plan of one evaluation at `precision` (built on demand): number of kernel
 * launches per evaluation, number of size bins, and the algorithmic work of one
 * evaluation, sum over blocks of (N^3/3 + N^2) flops with N = m_i + b_i (the Cholesky of
 * the augmented matrix plus its forward solve), and the number of covariance entries
 * generated, sum of N(N+1)/2.  Any output pointer may be NULL. */
int bv_plan_info(bv_ctx* ctx, int32_t precision, int32_t* launches_per_eval, int32_t* n_bins,
                 double* flops_per_eval, double* cov_entries_per_eval);

/* Test support: the device's Matern correlation rho(x) of Eq. 5 (sigma^2 = 1, beta = 1)
 * at n scaled distances x (host arrays), for 0 < nu <= 20; the half-integers use their
 * closed forms, any other nu the library's K_nu (Temme's series / continued fraction) or,
 * with tabulated != 0, the per-evaluation octave table the log-likelihood kernels use. */
int bv_matern_check(double nu, int32_t tabulated, int64_t n, const double* x, double* out);

/* Diagnostic: the tensor-core tile update of the mixed-precision kernel for large blocks,
 * out = C - XI XJ^T for 16 x 16 FP32 tiles (host arrays, row-major): every operand split
 * exactly into three BF16 parts, the six products of combined order <= 2 accumulated in
 * FP32 by mma.sync m16n8k16 (one warp on the GPU). */
int bv_tc_update_check(const float* C, const float* XI, const float* XJ, float* out);

/* Diagnostic: the library's device FP64 exponential e^{-x} (x >= 0; Tang's table-driven
 * method, used for the Matern kernel in the FP64 path) evaluated on the GPU for host
 * inputs x[n] into host out[n]. */
int bv_exp_neg_check(int64_t n, const double* x, double* out);

/* Diagnostic: the mixed-precision kernels' FP32 e^{-x} (own[i]) and CUDA's expf(-x)
 * (lib[i]) on the device for host x[n] >= 0 (host arrays).  Synchronous. */
int bv_exp_neg32_check(int64_t n, const float* x, float* own, float* lib);

/* ---- block-Vecchia sampler (Eq. 4 read generatively) ------------------------------ */

/* Draw y from the block-Vecchia model of dataset 0 at theta with the current blocks and
 * neighbours: blocks in order, y_{B_i} = mu_i(y_{NN_i}) + chol(Sigma^new_i) z_{B_i}.
 * z[n] (host) holds standard normals indexed by point; y_out[n] (host, may be NULL)
 * receives the draw, which also becomes the context's observations.  Synchronous. */
int bv_simulate(bv_ctx* ctx, const bv_theta* theta, const double* z, double* y_out);

/* ---- maximum likelihood --------------------------------------------------------- */

/* Bits of bv_mle's free_mask: which parameters the optimizer moves (others stay at
 * theta0).  Ranges move together (anisotropic ranges keep their ratios).  A free
 * smoothness nu (the paper estimates it, Sec. 3.2) is searched in log nu inside
 * [lo.nu, hi.nu], hi.nu <= 20; any value other than 1/2, 3/2, 5/2 goes through K_nu. */
enum { BV_FREE_SIGMA2 = 1, BV_FREE_RANGE = 2, BV_FREE_NUGGET = 4, BV_FREE_NU = 8 };

typedef struct bv_mle_opts {
    int32_t precision;   /* bv_precision of every evaluation                         */
    int32_t max_evals;   /* hard cap on log-likelihood evaluations (e.g. 2000)         */
    double ftol_rel;     /* stop when the simplex's ell spread < ftol_rel * |ell|      */
    double xtol;         /* ... and its log-parameter spread < xtol                     */
    double init_step;    /* initial simplex step in log-parameter units (e.g. 0.5)     */
    double init_step_nugget; /* initial step of the nugget's coordinate, log tau^2 or,
                                with sigma^2 profiled, log(tau^2 / sigma^2) (0: same as
                                init_step); the nugget is the least identified parameter,
                                so a start point can be much surer of sigma^2 and beta */
    int32_t newton_first;  /* 1 (recommended): trust-region Newton iterations on a
                              central-difference quadratic model from theta0 (radius 0.5
                              in log units to start, up to 40 iterations; in FP64 to
                              ftol_rel / xtol, in mixed precision to the coarse stage's
                              tolerances and then an FP64 polish), the Nelder-Mead search
                              only if they fail (no step lowers ell's negative, the
                              iterations run out).  A start near the optimum, such as the
                              learned warm start, converges in a few iterations.
                              0: Nelder-Mead first, then the FP64 Newton polish          */
    int32_t reserved;
} bv_mle_opts;

/* Maximise ell over log(sigma^2), log(beta), log(nu), log(tau^2) (free_mask selects) inside the
 * box [lo, hi] by a bounded Nelder-Mead search (derivative-free, as the paper's BOBYQA,
 * Sec. 3.2).  When sigma^2 is free and the nugget is free or zero, sigma^2 is profiled
 * out: the search runs over log beta and log(tau^2 / sigma^2) and sigma^2 takes its
 * closed-form maximiser Q / n (bv_loglik_terms) clamped to the box.  theta0: start
 * point, or NULL for the learned warm start (bv_warmstart_load first; it is applied to
 * the geometric centre of [lo, hi], whose smoothness and range ratios it keeps).  Outputs: theta_hat, loglik_hat (the FP64 ell at theta_hat), n_evals.
 * Synchronous (one device evaluation per optimizer step). */
int bv_mle(bv_ctx* ctx, const bv_theta* theta0, const bv_theta* lo, const bv_theta* hi,
           uint32_t free_mask, const bv_mle_opts* opts, bv_theta* theta_hat,
           double* loglik_hat, int32_t* n_evals);

/* Test support (host only, no device): bv_mle's search -- the same stages, options and
 * box handling -- on a synthetic likelihood instead of the block-Vecchia one, so that the
 * optimizer's logic can be checked on a CPU.  model[8] = (n, beta0, eta0, c_q, a, b, c_uv,
 * k); with u = log(beta / beta0), v = log(eta / eta0), eta = tau^2 / sigma^2,
 * Q = n exp(c_q u), D = n (a u^2 + b v^2 + c_uv u v + k (u^4 + v^4)) and
 * ell = -(Q / sigma^2 + D + n log sigma^2 + n log 2 pi) / 2; BV_MIXED evaluations add
 * n 1e-7 sin(1e3 (u + 2 v)).  Other arguments and outputs as bv_mle. */
int bv_mle_check(const double* model, const bv_theta* theta0, const bv_theta* lo, const bv_theta* hi,
                 uint32_t free_mask, const bv_mle_opts* opts, bv_theta* theta_hat, double* loglik_hat,
                 int32_t* n_evals);


/* ---- prediction (Sec. 2.4, Algorithm 2) ----------------------------------------- */

/* New locations S* (n_star x d, row-major, host; d as set by bv_set_data) and optionally
 * the held-out values there (host, n_star, may be NULL), against which bv_cond_sim
 * counts coverage.  Copied in; replaces any earlier prediction set.  Needs one dataset. */
int bv_set_pred_locations(bv_ctx* ctx, const double* locs_star, const double* y_true, int64_t n_star);

/* Algorithm 2 "Clustering": K-means blocks of S* with the conventions of
 * bv_build_blocks (seeding, iterations, exact-integer centroids), empty clusters dropped,
 * blocks in cluster-index order (no permutation: prediction blocks do not condition on
 * one another), members ascending.  Outputs as bv_build_blocks (indices into S*). */
int bv_build_pred_blocks(bv_ctx* ctx, int64_t bc, uint64_t seed, int32_t lloyd_iters,
                         int64_t* block_ptr, int32_t* point_idx, int64_t* bc_eff);

/* Algorithm 2 "Nearest neighbors": for each prediction block the min(m, n) observations
 * nearest to its centroid, key (squared distance, index) as bv_select_neighbors, from ALL
 * n observations.  min(m, n) <= 4000.  Outputs (may be NULL): nn_ptr[nb+1], nn_idx. */
int bv_select_pred_neighbors(bv_ctx* ctx, int32_t m, int64_t* nn_ptr, int32_t* nn_idx);

/* n_star, prediction blocks, conditioning entries, packed covariance entries
 * (sum_i b_i (b_i + 1) / 2); any pointer may be NULL. */
int bv_get_pred_sizes(bv_ctx* ctx, int64_t* n_star, int64_t* nblk, int64_t* n_nn, int64_t* n_cov);

/* Conditional means mu = Sigma^cross (Sigma^con)^-1 y_NN and covariances Sigma_B =
 * Sigma^lk - Sigma^cross (Sigma^con)^-1 Sigma^cross^T of every prediction block, in FP64
 * (Algorithm 2), with the observations of bv_set_data and the nugget on the diagonal of
 * Sigma^lk (a new location is its own point).  Host outputs, each may be NULL (results
 * stay on the device for bv_cond_sim): mean[n_star] and var[n_star] (diag Sigma_B) by
 * new-location index; cov_packed[n_cov]: each block's Sigma_B lower triangle row by row,
 * blocks in order.  BV_ENOTPD if a Sigma^con is not positive definite (its block's
 * outputs are NaN).  Synchronous. */
int bv_predict(bv_ctx* ctx, const bv_theta* theta, double* mean, double* var, double* cov_packed);

/* Univariate conditional simulation from the last bv_predict (Sec. 2.4): for each new
 * location j `rounds` draws mean + sqrt(var) z, z standard normal by Box-Muller, two per
 * pair of SplitMix64 uniforms (stream seed ^ 0x636f6e6473696d5f; pair k of location j uses
 * draws 2c and 2c+1, c = j * ceil(rounds/2) + k: u1 = 1 - (x_2c >> 11) 2^-53,
 * u2 = (x_2c+1 >> 11) 2^-53, z_2k = sqrt(-2 ln u1) cos(2 pi u2), z_2k+1 = the same with
 * sin); the interval is sample mean -/+ z_crit * sample sd (divisor rounds - 1).  Outputs
 * (host, may be NULL): lower[n_star], upper[n_star], covered = number of held-out values
 * inside their interval (PICP = covered / n_star; -1 without held-out values).
 * rounds >= 2.  Synchronous. */
int bv_cond_sim(bv_ctx* ctx, int32_t rounds, uint64_t seed, double z_crit, double* lower,
                double* upper, int64_t* covered);

/* Algorithmic work of one bv_predict: flops of the partial factorisations and covariance
 * evaluations. */
int bv_pred_plan_info(bv_ctx* ctx, double* flops, double* cov_evals);

/* Maximum likelihood for every dataset of a multi-dataset context at once (e.g. the
 * paper's study of 50 simulated datasets, Sec. 3.2): each dataset runs bv_mle's search;
 * their log-likelihood evaluations are gathered and issued as batched evaluations of all
 * datasets (one graph launch per precision requested).  theta0[ndatasets] (or NULL for
 * the learned warm start of every dataset); lo, hi, free_mask, opts shared.  Outputs
 * (ndatasets each, any but theta_hat may be NULL): theta_hat, loglik_hat, n_evals, status
 * (bv_mle's status per dataset); n_batches: batched evaluations issued.  Returns BV_OK
 * unless a dataset hit an error other than BV_ENOTPD. */
int bv_mle_multi(bv_ctx* ctx, const bv_theta* theta0, const bv_theta* lo, const bv_theta* hi,
                 uint32_t free_mask, const bv_mle_opts* opts, bv_theta* theta_hat,
                 double* loglik_hat, int32_t* n_evals, int32_t* status, int32_t* n_batches);

/* ---- learned warm start --------------------------------------------------------- */

/* The paper suggests warm-starting the estimation from a cheaper fit (Sec. 2.3: estimate
 * at small bc/m, reuse as the starting value).  The library adds a learned warm start: a
 * small MLP maps per-dataset summary features to a starting theta.  The search is the
 * same from either start; a cold start (an explicit theta0) needs no network, and its
 * estimate is the standard the warm-started one must reproduce. */

/* Features per dataset (BV_NFEAT floats):
 *   [0..31]  empirical semivariogram gamma_k / var(y) in 32 equal bins of the distance h on
 *            (0, 0.5]: bin k = min(31, floor(64 h)); gamma_k = mean over pairs in the bin of
 *            (y_i - y_j)^2 / 2 (0 if the bin is empty), over a seeded subsample of
 *            min(n, max_points) points (point j kept when floor(r_j n / 2^64) < max_points,
 *            r_j = SplitMix64 draw j of stream seed);
 *   [32] log var(y); [33..37] block-size histogram: the fractions of the blocks with
 *   b_i in 1-4, 5-8, 9-12, 13-16 and >= 17 points (the same at any n for a given n / bc);
 *   [38] nearest-neighbour semivariance: mean over subsample points i of
 *   (y_i - y_nn(i))^2 / 2, divided by var(y), nn(i) the nearest other subsample point
 *   (squared distance without fused multiply-add, lowest index on ties); [39] 64 x the
 *   mean nearest-neighbour distance (in semivariogram-bin units).
 * Blocks and neighbours must exist.  out[ndatasets x BV_NFEAT] (host).  Synchronous. */
#define BV_NFEAT 40
int bv_features(bv_ctx* ctx, int32_t max_points, uint64_t seed, float* out);

/* MLP: BV_NFEAT inputs (standardised) -> 3 x 128 GELU (exact erf form) -> 6 outputs:
 * standardised (log sigma^2, log beta, log tau^2) and 3 logits for nu in {0.5, 1.5, 2.5}.
 * A weights blob is BV_MLP_BLOB floats: BV_NFEAT input means, BV_NFEAT input scales,
 * 3 target means, 3 target scales, then the BV_MLP_NPARAM parameters
 * (W1[40x128], b1, W2[128x128], b2, W3[128x128], b3, W4[128x6], b4; row-major [in][out]). */
#define BV_MLP_NPARAM 39046
#define BV_MLP_BLOB (BV_MLP_NPARAM + 2 * BV_NFEAT + 6)

/* Train on the GPU with the library's own forward, backward and Adam kernels (FP32):
 * X[n x BV_NFEAT], T[n x 4] = (log sigma^2, log beta, log tau^2, nu) (host).  Loss = mean
 * squared error of the standardised regression outputs / 3 + cross-entropy of the nu
 * class.  Mini-batches of `batch` from a seeded shuffle, `epochs` passes, Adam(lr, 0.9,
 * 0.999, 1e-8) with its step count running across epochs.  blob_out[BV_MLP_BLOB] receives
 * the trained weights and standardisation; loss_out[epochs] (may be NULL) the mean
 * training loss per epoch.
 *   Standardisation: per input column the mean and population standard deviation of X
 *   (FP64 sums in row order, stored as float); a column whose deviation is at most
 *   1e-6 (|mean| + 1) gets the scale 1e30.  The same for the three regression targets
 *   (scale 1 below 1e-12).
 *   Initial parameters: biases 0; every weight, in blob order, (2u - 1) a with
 *   a = 1 / sqrtf(fan_in) (float) and u = (x_c >> 11) 2^-53, x_c = SplitMix64 draw c =
 *   0, 1, 2, ... of the stream seed ^ 0x6d6c7077 ("mlpw"), rounded to float.
 *   Shuffle: the row order starts as 0 .. n-1 and is carried from epoch to epoch; epoch e
 *   (from 0) applies Fisher-Yates, for i = n-1 down to 1 swapping positions i and
 *   j = floor(x_i (i + 1) / 2^64) with x_i = SplitMix64 draw i of the stream
 *   seed + 1000003 (e + 1) (mod 2^64); the mini-batches are consecutive runs of `batch`
 *   rows of that order, and a final partial run is skipped. */
int bv_mlp_train(const float* X, const float* T, int64_t n, int32_t epochs, int32_t batch, float lr,
                 uint64_t seed, float* blob_out, float* loss_out);

/* Forward pass on the GPU: out[n x 6] = raw outputs (standardised regression outputs,
 * nu logits) for inputs X[n x BV_NFEAT]. */
int bv_mlp_forward(const float* blob, const float* X, int64_t n, float* out);

/* Loss and its gradient with respect to the BV_MLP_NPARAM parameters for one batch
 * (the backward kernels used by training): loss_out[1], grad_out[BV_MLP_NPARAM]. */
int bv_mlp_loss_grad(const float* blob, const float* X, const float* T, int64_t n, float* loss_out,
                     float* grad_out);

/* Warm start for dataset 0: load a weights blob from a file (raw floats, BV_MLP_BLOB of
 * them after a 16-byte header "BVWS", version, count), then predict theta from the
 * current data's features (max_points 10000, seed 0).  theta_in supplies nu and aniso;
 * sigma^2, the range (all axes scaled together) and the nugget come from the network. */
int bv_warmstart_load(bv_ctx* ctx, const char* weights_path);
/* theta_in with nu = 0 asks for the network's smoothness class too (1/2, 3/2 or 5/2,
 * the arg-max of its three-way head); otherwise nu is kept. */
int bv_warmstart_predict(bv_ctx* ctx, const bv_theta* theta_in, bv_theta* theta_out);
/* The same for every dataset of a multi-dataset context (theta_in/theta_out[ndatasets]). */
int bv_warmstart_predict_multi(bv_ctx* ctx, const bv_theta* theta_in, bv_theta* theta_out);

#ifdef __cplusplus
}
#endif

#endif /* BV_H */

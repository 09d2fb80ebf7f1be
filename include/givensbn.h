/*
 * givensbn.h -- C ABI of the GB300 library that scores every family of a
 * Gaussian Bayesian network by the Givens-rotation walk of arXiv 1901.07643.
 *
 * A family is a child variable c and a parent set S of the other variables;
 * m variables give m * 2^(m-1) families (Sec. 1).  For each family the
 * library computes the residual sum of squares RSS(c|S) of the least-squares
 * regression of the centred column c on the centred columns S, exactly up to
 * rounding (Sec. 1 and Sec. 2), and stores the BIC-style local score
 *
 *     score(c|S) = n * ln(RSS / n) + |S| * ln(n)          (lower is better)
 *
 * at table slot idx(c,S) = c * 2^(m-1) + compress(S, c), where compress
 * deletes bit c from the m-bit parent mask (child-major table, one
 * (m-1)-bit parent mask per child).  RSS == 0 (exact collinearity) gives -inf;
 * in the FP32 walk so does an RSS below 2^-126 (the logarithm flushes
 * subnormal inputs), and with opts.fixup_tau > 0 such families are listed
 * and re-scored in FP64 (GBN_STATUS_FIXUP_OVERFLOW if the list overflows).
 *
 * How: one FP64 QR R0 of the centred n x m data (CholeskyQR2), then the
 * greedy sequence of adjacent column transpositions of Algorithm 1, each
 * re-triangularised by one Givens rotation (the GRC operator of Sec. 1.3);
 * every R on the walk yields the RSS of the families whose parents are a
 * prefix of its column ordering (Sec. 2).  The sequence is split into
 * independent sub-walks as in Sec. 6 (Algorithm 2, corrected reading), one
 * per GPU lane.
 *
 * Conventions for every entry point:
 *  - Pointers marked "device" are CUDA device pointers on the current device;
 *    pointers marked "host" are ordinary host memory.  The caller owns all
 *    buffers; the library allocates nothing.  Scratch memory is the caller's
 *    workspace, sized by givensbn_workspace_size().
 *  - Work is enqueued on opts->stream (NULL = legacy default stream) and the
 *    call returns without synchronising.  Device-side conditions (a
 *    rank-deficient Gram matrix) are recorded in the workspace and read with
 *    givensbn_status(), which synchronises the stream.
 *  - Return value: 0 on success, a negative GBN_ERR_* code otherwise; no work
 *    has been enqueued when an argument error is returned.
 *  - X is row-major n x m FP64 (row t, column j at X[t*m + j]), raw (the
 *    library centres the columns unless opts->center == 0).
 */
#ifndef GIVENSBN_H
#define GIVENSBN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* error codes */
#define GBN_OK 0
#define GBN_ERR_M (-1)          /* m outside [GBN_MIN_M, GBN_MAX_M] */
#define GBN_ERR_N (-2)          /* n < m + 1 */
#define GBN_ERR_NULL (-3)       /* a required pointer is NULL */
#define GBN_ERR_ALIGN (-4)      /* a pointer is not 16-byte aligned */
#define GBN_ERR_WORKSPACE (-5)  /* workspace missing or smaller than required */
#define GBN_ERR_CUDA (-6)       /* a CUDA launch or runtime call failed */
#define GBN_ERR_Q (-7)          /* opts->q outside the supported range for m */
#define GBN_ERR_PRECISION (-8)  /* opts->precision not 0 or 1 */
#define GBN_ERR_BATCH (-9)      /* batched arguments inconsistent */
#define GBN_ERR_STATIC_SCRATCH (-10) /* input needs more than the no-alloc entry point's scratch */
#define GBN_ERR_OPTS (-11)      /* an option outside its range (score, shard, consumer warps) */
#define GBN_ERR_TUNE (-12)      /* the autotuner could not time or record a candidate */

/* device status bits (givensbn_status) */
#define GBN_STATUS_RANK_DEFICIENT 1 /* a Cholesky pivot was <= 0: RSS 0 for some families */
#define GBN_STATUS_WATCHDOG 2       /* a bounded wait inside a kernel expired: output incomplete */
#define GBN_STATUS_FIXUP_OVERFLOW 4 /* more ill-conditioned families than the fix-up list holds;
                                       the rest keep their FP32 scores */
#define GBN_STATUS_BAD_FAMILY 8     /* givensbn_family_coefficients: a listed family was invalid
                                       (child out of range, or parents holding the child or
                                       variables >= m); its outputs are NaN */

#define GBN_MIN_M 2
#define GBN_MAX_M 30

typedef struct givensbn_opts {
    int32_t precision;      /* 0: FP32 rotations and fp32 scores; 1: FP64 throughout, fp64 scores */
    int32_t center;         /* 1 (default): centre the columns of X first */
    int32_t q;              /* variables per sub-walk (0 = automatic choice) */
    int32_t debug_coverage; /* 1: instead of scores, add 1 to a uint32 counter per table slot */
    void* stream;           /* cudaStream_t, NULL for the default stream */
    void* workspace;        /* device scratch, >= givensbn_workspace_size() bytes, 256-byte aligned */
    size_t workspace_bytes;
    void* stage_events;     /* NULL, or host array of 4 cudaEvent_t recorded on the stream before
                               the R0 stage, after it, after the sub-walk roots and after the walk
                               (before the FP64 fix-up pass) */
    double fixup_tau;       /* FP32 walk only: a family whose RSS falls below fixup_tau times
                               the child's centred sum of squares is recomputed in FP64 from R0
                               (QR of its columns) and scored in FP64; 0 disables.  Default 1e-6 */
    int64_t watchdog_ns;    /* bound, in nanoseconds, on every wait between the warps of a walk
                               block; on expiry the kernel sets GBN_STATUS_WATCHDOG and returns
                               (the table is then incomplete).  0 = the default, 2 s */
    int32_t max_parents;    /* bounded in-degree K: only families with |S| <= K are written (the
                               other slots of the table are left untouched); -1 = no bound
                               (default) */
    int32_t score;          /* GBN_SCORE_BIC (default), GBN_SCORE_AIC, GBN_SCORE_PENALTY or
                               GBN_SCORE_BGE */
    double penalty;         /* GBN_SCORE_PENALTY: score = n ln(RSS/n) + penalty * |S| */
    int32_t shard_index;    /* score only shard shard_index of shard_count shards of the table */
    int32_t shard_count;    /* (see givensbn_shard_range); 0 or 1 = the whole table (default) */
    int32_t consumer_warps; /* consumer warps per walk block, 1..8; 0 = automatic */
    int32_t reserved0;
    const char* tune_cache; /* host path of an autotuner cache file (givensbn_autotune), or NULL.
                               With q == 0 and consumer_warps == 0 the plan takes the cached
                               choice for this device and size class, else the automatic one */
    double bge_alpha_mu;    /* GBN_SCORE_BGE: prior precision scale of the mean, > 0; 0 = 1 */
    double bge_alpha_w;     /* GBN_SCORE_BGE: prior Wishart degrees of freedom, > m + 1;
                               0 = m + 2 */
} givensbn_opts;

/* Score of a family from its residual sum of squares (opts->score). */
#define GBN_SCORE_BIC 0     /* n ln(RSS/n) + |S| ln n */
#define GBN_SCORE_AIC 1     /* n ln(RSS/n) + 2 |S| */
#define GBN_SCORE_PENALTY 2 /* n ln(RSS/n) + opts->penalty * |S| */
/* BGe: the log marginal likelihood ratio ln p(d_{S u c}) - ln p(d_S) under the normal-Wishart
 * prior (Geiger and Heckerman 2002, corrected by Kuipers, Moffa and Heckerman 2014) with prior
 * mean the sample mean and T0 = t I, t = alpha_mu (alpha_w - m - 1) / (alpha_mu + 1).  The walk
 * runs over a factor of the posterior matrix t I + S_n (S_n the centred scatter matrix), so its
 * residuals are the Schur complements rho(c | S); a pass then forms ln det of every parent
 * block by the recursion L[S] = L[S - h] + ln rho(h | S - h) (h the highest variable of S) and
 * writes K(|S|) - ((n + alpha_w - m + |S| + 1) / 2) ln rho(c | S) - L[S] / 2.  Higher is
 * better (a log likelihood), unlike the other kinds: negate the table before
 * givensbn_structure_search, which minimises.  Single-dataset calls without shards only; the
 * workspace grows by 2^m table elements. */
#define GBN_SCORE_BGE 3

/* Default options: FP32, centring on, automatic q, no workspace, fixup_tau 1e-6, BIC score, no
 * in-degree bound, the whole table, the default watchdog, no tuning cache. */
void givensbn_default_opts(givensbn_opts* opts);

/*
 * Bytes of device workspace score_all_families needs for (n, m) with these
 * options (precision and q matter).  Writes *bytes; returns 0 or GBN_ERR_*.
 */
int givensbn_workspace_size(int64_t n, int32_t m, const givensbn_opts* opts, size_t* bytes);

/*
 * Scores of every family of the n x m data X (the problem of Sec. 1;
 * method of Sec. 1.3, Sec. 3 and Sec. 6).
 *   X          device, n x m FP64 row-major, read only
 *   out_scores device-accessible, m * 2^(m-1) elements: float (precision 0)
 *              or double (precision 1), or uint32 counters if
 *              opts->debug_coverage; every element is written exactly once
 *              (the FP64 fix-up may write a listed element a second time).
 *              Device memory, or pinned host memory (unified addressing): the
 *              kernels then store the table straight into host memory.
 *   opts       host; workspace required
 */
int score_all_families(const double* X, int64_t n, int32_t m, void* out_scores,
                       const givensbn_opts* opts);

/* Device status word recorded by the last call that used this workspace
 * (GBN_STATUS_* bits).  Synchronises opts->stream.  Returns 0 or GBN_ERR_*. */
int givensbn_status(const givensbn_opts* opts, int32_t* status);

/* Human-readable text for a GBN_ERR_* code (static storage). */
const char* givensbn_strerror(int code);

/* The q the automatic choice picks for (m, precision). */
int32_t givensbn_auto_q(int32_t m, int32_t precision);

/* The sub-walk size q and consumer warps per walk block that a call with these arguments
 * would use (opts->q / opts->consumer_warps, else the tuning cache, else the automatic
 * choice).  Host only; no device work.  Returns 0 or GBN_ERR_*. */
int givensbn_plan_choice(int64_t n, int32_t m, const givensbn_opts* opts, int32_t* q,
                         int32_t* consumer_warps);

/*
 * Sharding one table (the parallel split of Sec. 6, Algorithm 2, across calls).
 * The walk runs 2^k sub-walks, k = m - q, one per front set F of the fixed variables
 * H = {0 .. k-1}; sub-walk F writes exactly the families (c, S) with S n H = F.  The
 * sub-walks are grouped 2^W to a CTA (W = min(5, k), lanes over the lowest W fixed
 * variables), CTA g holding the front sets with F >> W == g.  With
 * opts->shard_count = N > 1, the call with shard_index = i walks only CTAs
 * [cta_begin, cta_end) (contiguous ranges of CTA pairs, one per shard, covering all
 * 2^(k-W) CTAs once), i.e. it writes exactly the families with
 * ((S & (2^k - 1)) >> W) in [cta_begin, cta_end) and leaves every other slot of
 * out_scores untouched.  Shards need no communication; every shard computes R0 itself.
 * This call reports k, W and the range for (n, m, opts).  Host only.  Returns 0 or
 * GBN_ERR_*. */
int givensbn_shard_range(int64_t n, int32_t m, const givensbn_opts* opts, int32_t* fixed_k,
                         int32_t* lane_bits, int64_t* cta_begin, int64_t* cta_end);

/*
 * Scores of B datasets of uneven size in one set of launches (the same
 * computation as score_all_families for each dataset; batching is an
 * engineering addition, the paper scores one dataset).
 *   Xs          host array of B device pointers, each n_b x m_b FP64 row-major
 *   ns, ms      host arrays of B sizes (each as for score_all_families)
 *   out         device; table b occupies out_offsets[b] .. + m_b * 2^(m_b-1)
 *               elements (float, or double for precision 1, or uint32 counters
 *               with debug_coverage); tables must not overlap and each must
 *               start 16-byte aligned
 *   out_offsets host array of B element offsets into out
 *   opts        host; opts->q is the common sub-walk size (0 = the smallest
 *               automatic choice over the batch); workspace >=
 *               givensbn_batched_workspace_size()
 * The call plans every dataset on the host, writes a device table into the
 * head of the workspace with kernel launches (no runtime memcpy, allocation or
 * synchronisation), then runs each stage as one launch over all datasets,
 * largest datasets first.  The whole call may be captured into a CUDA graph;
 * replaying the graph re-runs it with the same pointers.  Status words are
 * per dataset and are not read by givensbn_status.  Returns 0 or GBN_ERR_*.
 */
int score_all_families_batched(const double* const* Xs, const int64_t* ns, const int32_t* ms,
                               int32_t B, void* out, const int64_t* out_offsets,
                               const givensbn_opts* opts);

/* Workspace bytes score_all_families_batched needs for these sizes and options. */
int givensbn_batched_workspace_size(const int64_t* ns, const int32_t* ms, int32_t B,
                                    const givensbn_opts* opts, size_t* bytes);

/*
 * Gradient of L = sum_f w_f * score_f with respect to X (the adjoint of the
 * scoring path; the paper has no gradient, the derivative follows from the
 * least-squares problem of Sec. 1 and the walk of Sec. 1.3 / Algorithm 1).
 * Every score depends on X only through the centred Gram G = Xc^T Xc, and
 *     grad_X = Xc (Gbar + Gbar^T),   Gbar = sum_f (w_f n / RSS_f) v_f v_f^T,
 * v_f = e_c - beta_f with beta_f the family's least-squares coefficients.
 * Gbar is accumulated along the Givens walk, one sub-walk per warp, each
 * sub-walk re-formed from R0 by GRC steps (the R0 checkpoint).
 *   X       device, n x m FP64 row-major (raw; centred as in the forward pass)
 *   w       device, m * 2^(m-1) weights in table layout: float (precision 0,
 *           FP32 walk state) or double (precision 1), 16-byte aligned
 *   grad_X  device, n x m FP64 row-major, written (not accumulated)
 *   opts    host; workspace >= givensbn_backward_workspace_size(); opts->q is
 *           the sub-walk size of the backward walk (0 = automatic, m - 9)
 * Families with RSS == 0 contribute nothing (their score is -inf); a singular
 * sub-walk factor sets GBN_STATUS_RANK_DEFICIENT and is skipped.
 * Deterministic: sums are formed in a fixed order.  Returns 0 or GBN_ERR_*.
 */
int score_all_families_backward(const double* X, int64_t n, int32_t m, const void* w,
                                double* grad_X, const givensbn_opts* opts);

/* Workspace bytes score_all_families_backward needs for (n, m, opts). */
int givensbn_backward_workspace_size(int64_t n, int32_t m, const givensbn_opts* opts,
                                     size_t* bytes);

/*
 * score_all_families_backward for B datasets of uneven size in four launch groups: the R0
 * stage of every dataset (as in score_all_families_batched), one launch of the adjoint walk
 * over all datasets' sub-walks, one reduction and one gradient launch.  Each gradient is
 * bit-identical to the single-dataset call's (the same sub-walks on the same warps, sums in
 * the same order).  Batching is an engineering addition; the paper has no gradient.
 *   Xs, ns, ms  as for score_all_families_batched
 *   weights     host array of B device pointers, weights of dataset b in its table layout
 *               (m_b 2^(m_b-1) entries; float for precision 0, double for 1), 16-byte aligned
 *   grads       host array of B device pointers, n_b x m_b FP64 outputs
 *   opts        host; opts->q is the backward sub-walk size (0 = m - 9 per dataset);
 *               workspace >= givensbn_backward_batched_workspace_size()
 * Returns 0 or GBN_ERR_*; per-dataset status words are not read by givensbn_status.
 */
int score_all_families_backward_batched(const double* const* Xs, const int64_t* ns,
                                        const int32_t* ms, int32_t B, const void* const* weights,
                                        double* const* grads, const givensbn_opts* opts);
int givensbn_backward_batched_workspace_size(const int64_t* ns, const int32_t* ms, int32_t B,
                                             const givensbn_opts* opts, size_t* bytes);

/*
 * score_all_families without a workspace and without any allocation.  The
 * paper has no counterpart: this is an engineering variant for callers that
 * cannot allocate device memory when they call (a host runtime whose pool
 * owns all free device memory; loops where cudaMalloc/cudaFree would
 * synchronise the device).  Same computation as score_all_families with the
 * default options: FP32 walk, fp32 scores, centring, automatic q.
 *   X          device, n x m FP64 row-major, read only
 *   out_scores device, m * 2^(m-1) floats, every element written once
 *   stream     cudaStream_t (NULL = legacy default stream); asynchronous
 * Scratch: a 16 MiB array in the library's device image (enough for every n
 * at m <= 20); larger inputs return GBN_ERR_STATIC_SCRATCH with nothing
 * enqueued.  Its 256-byte status block is cleared by every call on `stream`.
 * All calls on a device share that scratch, so calls must not overlap: a
 * call may start only after the previous call's kernels have completed.  The
 * first call on each device looks up the scratch address (with that device
 * current); make it before any stream capture.  The address is kept for the
 * life of the process, so after cudaDeviceReset of a device this entry point
 * must not be called on that device again.  Device status words are not
 * reported by this entry point.  Returns 0 or GBN_ERR_*.
 */
int score_all_families_noalloc(const double* X, int64_t n, int32_t m, float* out_scores,
                               void* stream);

/*
 * Autotuner (the split size of Sec. 6 / Algorithm 2 and the walk block's consumer warps,
 * measured on the device).  Times whole scoring calls for the candidates q in
 * {a-1, a, a+1} (a = the automatic choice; within the compiled range and <= m) times
 * consumer warps in {4, 6, 8}: one untimed call, then the median of three calls timed with
 * CUDA events on opts->stream (the call synchronises that stream).  The fastest candidate
 * is returned and, when opts->tune_cache is set, appended to that file as one line
 *   gbn-tune-v1 device=<name> kind=single precision=<p> m=<m> mmin=<m> count=1
 *               nlog2=<floor(log2 n)> q=<q> cw=<warps> ms=<median ms>
 * Later calls with q == 0, consumer_warps == 0 and the same tune_cache take the last line
 * matching their device (or device=*), kind, precision, m, mmin, count and nlog2.
 *   X, out_scores  as for score_all_families (out_scores is overwritten by the trials)
 *   opts           host; workspace >= givensbn_autotune_workspace_size(); opts->q and
 *                  opts->consumer_warps are ignored (they are what is tuned)
 *   q_out, cw_out, ms_out   host, may be NULL: the winner and its median time
 *   results        host array of max_results entries, may be NULL: every candidate's time
 *   n_results      host, may be NULL: the number of candidates timed
 * Returns 0, GBN_ERR_* of a trial call, or GBN_ERR_TUNE if the cache file cannot be
 * written (the winner is still returned).
 */
typedef struct givensbn_tune_result {
    int32_t q;
    int32_t consumer_warps;
    double ms;
} givensbn_tune_result;

int givensbn_autotune_workspace_size(int64_t n, int32_t m, const givensbn_opts* opts,
                                     size_t* bytes);
int givensbn_autotune(const double* X, int64_t n, int32_t m, void* out_scores,
                      const givensbn_opts* opts, int32_t* q_out, int32_t* cw_out, double* ms_out,
                      givensbn_tune_result* results, int32_t max_results, int32_t* n_results);

/* The same for score_all_families_batched: one common q for the batch (candidates around
 * the smallest automatic choice, q <= the smallest m), cached as kind=batch with m = the
 * largest m, mmin = the smallest, count = B and nlog2 = floor(log2(sum of n)). */
int givensbn_autotune_batched_workspace_size(const int64_t* ns, const int32_t* ms, int32_t B,
                                             const givensbn_opts* opts, size_t* bytes);
int givensbn_autotune_batched(const double* const* Xs, const int64_t* ns, const int32_t* ms,
                              int32_t B, void* out, const int64_t* out_offsets,
                              const givensbn_opts* opts, int32_t* q_out, int32_t* cw_out,
                              double* ms_out, givensbn_tune_result* results, int32_t max_results,
                              int32_t* n_results);

/*
 * Least-squares coefficients of listed families (the regression of Sec. 1.1, solved on the
 * initial QR decomposition R0 of Sec. 2 instead of the n x m data: Xc = Q R0 gives the same
 * problem with m rows).  FP64 throughout: R0 by CholeskyQR2, then per family Householder QR
 * of R0's columns for S and c, the residual sum of squares and back substitution.
 *   X        device, n x m FP64 row-major (centred by the call unless opts->center == 0)
 *   child    device, count int32 child variables
 *   parents  device, count uint64 parent bitmasks (bit v = variable v; must not hold the
 *            child or bits >= m)
 *   beta     device, count x (m + 1) doubles, written: row f holds b_v for v in S at index
 *            v, 0 for the other variables, and at index m the intercept
 *            mean_c - sum_v b_v mean_v (0 when opts->center == 0)
 *   rss      device, count doubles (RSS of each family), or NULL
 *   opts     host; precision and q are ignored; workspace >=
 *            givensbn_coefficients_workspace_size()
 * An invalid family gets NaN outputs and sets GBN_STATUS_BAD_FAMILY; a family whose parent
 * columns are linearly dependent gets NaN coefficients (its RSS is still written) and sets
 * GBN_STATUS_RANK_DEFICIENT (givensbn_status).  Returns 0 or GBN_ERR_*.
 */
int givensbn_coefficients_workspace_size(int64_t n, int32_t m, const givensbn_opts* opts,
                                         size_t* bytes);
int givensbn_family_coefficients(const double* X, int64_t n, int32_t m, const int32_t* child,
                                 const uint64_t* parents, int64_t count, double* beta,
                                 double* rss, const givensbn_opts* opts);

/*
 * Exact structure search over a local-score table (the use of the all-family scores that the
 * method serves, Sec. 1: learning a Bayesian network structure from every child / parent-set
 * score).  Lower scores are better; a slot holding +inf is a family that may not be chosen
 * (e.g. |S| > K after a bounded-in-degree call, if the caller filled the table with +inf
 * first).  The search finds a DAG minimising sum_c score(c, parents(c)):
 *   1. best parents: B[c][U] = min over S subset of U of score(c, S) and its argmin, for every
 *      child c and candidate set U of the other variables (a subset-minimum transform);
 *   2. F[W] = min over c in W of F[W \ c] + B[c][W \ c], F[{}] = 0, over all 2^m subsets
 *      W in order of size (FP64 sums); c is the sink of W;
 *   3. backtracking from W = all variables through the sinks.
 * Ties go to the smaller parent set in step 1 and to the smallest sink in step 2.
 *
 * givensbn_best_parents: step 1 alone.
 *   scores    device, m * 2^(m-1) floats in table layout (see score_all_families)
 *   best      device, m * 2^(m-1) floats, written: best[c 2^(m-1) + u] = B[c][U] for the
 *             compressed candidate mask u of U (the table's own slot indexing)
 *   best_set  device, m * 2^(m-1) uint32, written: the compressed mask of the argmin S
 *   opts      host, may be NULL (stream only)
 * givensbn_structure_search: all three steps.
 *   scores    as above
 *   parents   device, m uint32, written: the parent bitmask (bit v = variable v) of each
 *             variable in an optimal DAG
 *   order     device, m int32, or NULL: an optimal variable ordering (parents come first)
 *   total     device, one double: the optimal network score (the FP64 sum of the chosen
 *             table entries)
 *   opts      host; workspace >= givensbn_structure_search_workspace_size(m) (8 bytes per
 *             table slot plus 9 bytes per variable subset and 8.4 KB; 7.3 GB at m = 26)
 * Both are asynchronous on opts->stream and return 0 or GBN_ERR_*.
 */
int givensbn_best_parents(const float* scores, int32_t m, float* best, uint32_t* best_set,
                          const givensbn_opts* opts);

/*
 * Measured arithmetic-pipe peaks of the current device (a measurement helper, not part of
 * the paper's method): FP32 and FP64 fused multiply-add throughput in TFLOP/s (2 flops per
 * FMA), each the best of three timed launches of independent FMA chains on every SM.
 *   scratch  device, 8 bytes, 8-byte aligned (never written for these inputs)
 *   stream   cudaStream_t (synchronised)
 * Returns 0 or GBN_ERR_*.
 */
int givensbn_pipe_peaks(void* scratch, void* stream, double* fp32_tflops, double* fp64_tflops);
/*
 * Measured FP64 tensor-core throughput of the current device (a measurement helper, not part
 * of the paper's method): independent chains of mma.sync m8n8k4 f64 on every SM, 512 flops
 * per warp instruction, TFLOP/s, best of three timed launches.  It is the rate an FP64 Gram
 * on the matrix units could reach, beside the FMA rate of givensbn_pipe_peaks.
 *   scratch  device, 8 bytes, 8-byte aligned (never written for these inputs)
 *   stream   cudaStream_t (synchronised)
 * Returns 0 or GBN_ERR_*.
 */
int givensbn_dmma_peak(void* scratch, void* stream, double* tflops);
int givensbn_structure_search_workspace_size(int32_t m, size_t* bytes);
int givensbn_structure_search(const float* scores, int32_t m, uint32_t* parents, int32_t* order,
                              double* total, const givensbn_opts* opts);

#ifdef __cplusplus
}
#endif

#endif /* GIVENSBN_H */

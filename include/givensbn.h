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

/* device status bits (givensbn_status) */
#define GBN_STATUS_RANK_DEFICIENT 1 /* a Cholesky pivot was <= 0: RSS 0 for some families */
#define GBN_STATUS_WATCHDOG 2       /* a bounded wait inside a kernel expired: output incomplete */
#define GBN_STATUS_FIXUP_OVERFLOW 4 /* more ill-conditioned families than the fix-up list holds;
                                       the rest keep their FP32 scores */

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
} givensbn_opts;

/* Default options: FP32, centring on, automatic q, no workspace, fixup_tau 1e-6. */
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
 *           the sub-walk size of the backward walk (0 = automatic, m - 10)
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
 * current); make it before any stream capture.  Device status words are not
 * reported by this entry point.  Returns 0 or GBN_ERR_*.
 */
int score_all_families_noalloc(const double* X, int64_t n, int32_t m, float* out_scores,
                               void* stream);

#ifdef __cplusplus
}
#endif

#endif /* GIVENSBN_H */

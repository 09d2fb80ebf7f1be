// C ABI of libgivensbn: argument checks, the execution plan and the stage launches.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include "gbn_internal.cuh"

namespace gbn {

static size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

static int max_q(int precision) { return precision ? kMaxQFp64 : kMaxQ; }

int auto_q(int m, int precision) {
    // Small sub-walks keep the walk's unrolled code small (its instruction
    // fetch bounds it), large ones need fewer roots; the tape of one sub-walk
    // (2^Q - Q - 1 steps) stays in shared memory.  This rule is the fallback;
    // givensbn_autotune measures the candidates on the device.
    int q = m - 19;
    if (q < 6) q = 6;
    if (q > 8) q = 8;
    if (q > max_q(precision)) q = max_q(precision);
    if (q > m) q = m;
    return q;
}

void shard_range(int64_t n_cta_total, int index, int count, int64_t* begin, int64_t* end) {
    if (count <= 1) {
        *begin = 0;
        *end = n_cta_total;
        return;
    }
    if (n_cta_total % 2 != 0) {  // a single CTA: shard 0 takes it
        *begin = index == 0 ? 0 : n_cta_total;
        *end = n_cta_total;
        return;
    }
    const int64_t pairs = n_cta_total / 2;
    *begin = 2 * (pairs * index / count);
    *end = 2 * (pairs * (index + 1) / count);
}

// Consumer warps of the walk when the caller and the tuner leave it open:
// enough that the largest CTA gives each a few columns to replay.
static int auto_consumer_warps(const Plan& p) {
    const int g = p.W >= 1 ? (p.lanes >> 1) : 1;
    const int n5 = p.W >= 1 ? (p.W + (32 / g) - 1) / (32 / g) : 0;
    const int items = p.Q + (p.k - p.W) + n5;
    int nw = (items + kItemsPerWarp - 1) / kItemsPerWarp;
    if (nw > 8) nw = 8;
    return nw < 1 ? 1 : nw;
}

int make_plan(int64_t n, int32_t m, const givensbn_opts* opts, Plan* p) {
    if (m < GBN_MIN_M || m > GBN_MAX_M) return GBN_ERR_M;
    if (n < (int64_t)m + 1) return GBN_ERR_N;
    const int precision = opts ? opts->precision : 0;
    if (precision != 0 && precision != 1) return GBN_ERR_PRECISION;
    const int cw_req = opts ? opts->consumer_warps : 0;
    if (cw_req < 0 || cw_req > 8) return GBN_ERR_OPTS;
    int Q = (opts && opts->q > 0) ? opts->q : 0;
    int cw = cw_req;
    if (Q == 0 && cw == 0 && opts && opts->tune_cache && !opts->debug_coverage) {
        int tq = 0, tcw = 0;
        if (tune_lookup(opts->tune_cache, 0, precision, m, m, 1, n, &tq, &tcw) && tq >= kMinQ &&
            tq <= max_q(precision) && tq <= m && tcw >= 1 && tcw <= 8) {
            Q = tq;
            cw = tcw;
        }
    }
    if (Q == 0) Q = auto_q(m, precision);
    if (Q < kMinQ || Q > max_q(precision) || Q > m) return GBN_ERR_Q;
    const int score = opts ? opts->score : GBN_SCORE_BIC;
    double lam;
    double bge_am = 0.0, bge_aw = 0.0;
    switch (score) {
        case GBN_SCORE_BIC: lam = log((double)n); break;
        case GBN_SCORE_AIC: lam = 2.0; break;
        case GBN_SCORE_PENALTY:
            lam = opts->penalty;
            if (!(lam == lam) || lam > 1e300 || lam < -1e300) return GBN_ERR_OPTS;
            break;
        case GBN_SCORE_BGE:  // the walk stores n ln(rho / n); the BGe pass does the rest
            lam = 0.0;
            bge_am = opts->bge_alpha_mu == 0.0 ? 1.0 : opts->bge_alpha_mu;
            bge_aw = opts->bge_alpha_w == 0.0 ? (double)m + 2.0 : opts->bge_alpha_w;
            if (!(bge_am > 0.0 && bge_am < 1e300 && bge_aw > (double)m + 1.0 && bge_aw < 1e300))
                return GBN_ERR_OPTS;
            if (opts->debug_coverage) return GBN_ERR_OPTS;
            break;
        default: return GBN_ERR_OPTS;
    }
    const int shard_count = opts ? opts->shard_count : 0;
    const int shard_index = opts ? opts->shard_index : 0;
    if (shard_count < 0 || shard_index < 0 || (shard_count <= 1 ? shard_index != 0
                                                                  : shard_index >= shard_count))
        return GBN_ERR_OPTS;
    if (score == GBN_SCORE_BGE && shard_count > 1) return GBN_ERR_OPTS;  // needs every family
    const long long wd = opts ? (long long)opts->watchdog_ns : 0;
    if (wd < 0) return GBN_ERR_OPTS;
    *p = Plan();
    p->m = m;
    p->n = n;
    p->precision = precision;
    p->Q = Q;
    p->k = m - Q;
    p->W = p->k < kLaneBits ? p->k : kLaneBits;
    p->lanes = 1 << p->W;
    p->n_cta_total = (int64_t)1 << (p->k - p->W);
    int64_t cb = 0, ce = 0;
    shard_range(p->n_cta_total, shard_index, shard_count, &cb, &ce);
    p->cta_begin = cb;
    p->n_cta = ce - cb;
    p->lam = lam;
    if (score == GBN_SCORE_BGE) {
        p->bge = 1;
        p->bge_alpha_mu = bge_am;
        p->bge_alpha_w = bge_aw;
        p->bge_t = bge_am * (bge_aw - m - 1.0) / (bge_am + 1.0);
    }
    const int mp = opts ? opts->max_parents : -1;
    p->kmax = (mp < 0 || mp > m - 1) ? m - 1 : mp;
    p->watchdog_ns = wd > 0 ? wd : kWatchdogNs;
    int pos = 0;
    for (int v = p->W; v < p->k; ++v) p->order[pos++] = v;
    for (int v = p->W - 1; v >= 0; --v) p->order[pos++] = v;
    for (int v = p->k; v < m; ++v) p->order[pos++] = v;
    int panels = (int)(n / 32);
    if (panels < 1) panels = 1;
    if (panels > kMaxPanels) panels = kMaxPanels;
    p->rows_per_panel = (int)((n + panels - 1) / panels);
    p->panels = (int)((n + p->rows_per_panel - 1) / p->rows_per_panel);
    p->center = opts ? (opts->center != 0) : 1;
    p->coverage = opts ? (opts->debug_coverage != 0) : 0;
    const size_t es = precision ? sizeof(double) : sizeof(float);
    p->leaf_stride = leaf_stride_elems(Q, p->k);
    p->n_bwarps = cw > 0 ? cw : auto_consumer_warps(*p);
    size_t off = 0;
    p->off_status = off;
    off = align_up(off + 256, 256);
    p->off_colsum = off;  // per-panel column sums, then per-panel exponent maxima of |x|
    off = align_up(off + sizeof(double) * 2 * (size_t)p->panels * m, 256);
    p->off_mu = off;  // 32 means, then 32 column scale exponents
    off = align_up(off + sizeof(double) * 64, 256);
    p->off_gram = off;
    off = align_up(off + sizeof(double) * (size_t)p->panels * (m * (m + 1) / 2), 256);
    p->off_gsum = off;
    off = align_up(off + sizeof(double) * (size_t)(m * (m + 1) / 2), 256);
    p->off_r1 = off;
    off = align_up(off + sizeof(double) * (size_t)m * m, 256);
    p->off_r1inv = off;
    off = align_up(off + sizeof(double) * (size_t)m * m, 256);
    p->off_r0 = off;
    off = align_up(off + sizeof(double) * (size_t)m * m, 256);
    p->off_leaves = off;
    off = align_up(off + es * p->leaf_stride * (size_t)p->n_cta, 256);
    p->off_top = off;
    off = align_up(off + top_node_bytes(*p), 256);
    const double tau = opts ? opts->fixup_tau : 1e-6;
    if (precision == 0 && !p->coverage && tau > 0.0) {
        p->fix_cap = kFixCap;
        p->fix_tau = tau;
        p->off_fix = off;
        off = align_up(off + 256 + sizeof(long long) * (size_t)kFixCap, 256);
    }
    if (p->bge) {
        p->off_bge = off;
        off = align_up(off + es * ((size_t)1 << m), 256);
    }
    if (precision == 0 && !p->coverage) {
        p->scale = 1;
        p->off_scale = off;
        off = align_up(off + sizeof(int) * 33, 256);
    }
    p->total_bytes = off;
    return GBN_OK;
}

}  // namespace gbn

using namespace gbn;

// Checked builds synchronise after every stage and report the CUDA error and
// the first out-of-bounds index the kernels caught; ordinary builds pass rc on.
static int checked_stage(const char* name, int rc, const Plan& p, char* ws, cudaStream_t stream) {
#ifdef GBN_CHECKED
    cudaError_t e = cudaGetLastError();
    cudaError_t s = cudaStreamSynchronize(stream);
    unsigned long long rec[4] = {0, 0, 0, 0};
    cudaError_t c = cudaMemcpy(rec, ws + p.off_status + kCheckOffset, sizeof(rec),
                               cudaMemcpyDeviceToHost);
    fprintf(stderr,
            "[givensbn checked] stage %s: rc=%d launch=%s sync=%s copy=%s violations=%llu "
            "site=%llu index=%llu bound=%llu\n",
            name, rc, cudaGetErrorString(e), cudaGetErrorString(s), cudaGetErrorString(c), rec[0],
            rec[1], rec[2], rec[3]);
    if (rc == GBN_OK && (e != cudaSuccess || s != cudaSuccess || rec[0] != 0)) rc = GBN_ERR_CUDA;
#else
    (void)name;
    (void)p;
    (void)ws;
    (void)stream;
#endif
    return rc;
}

namespace gbn {

int run_pipeline(const Plan& p, const double* X, char* ws, void* out, cudaStream_t stream,
                 void* stage_events) {
    cudaEvent_t* ev = static_cast<cudaEvent_t*>(stage_events);
    if (ev && cudaEventRecord(ev[0], stream) != cudaSuccess) return GBN_ERR_CUDA;
    int rc = launch_r0(p, X, ws, stream);
    if (rc == GBN_OK && p.bge) rc = launch_bge_prior(p, ws, stream);
    if (rc == GBN_OK && p.scale) rc = launch_scale_r0(p, ws, stream);
    if (rc == GBN_OK && p.fix_cap) rc = launch_fix_flags(p, ws, stream);
    if ((rc = checked_stage("r0", rc, p, ws, stream))) return rc;
    if (ev && cudaEventRecord(ev[1], stream) != cudaSuccess) return GBN_ERR_CUDA;
    rc = launch_roots(p, ws, stream);
    if ((rc = checked_stage("roots", rc, p, ws, stream))) return rc;
    if (ev && cudaEventRecord(ev[2], stream) != cudaSuccess) return GBN_ERR_CUDA;
    rc = launch_walk(p, ws, out, stream);
    if ((rc = checked_stage("walk", rc, p, ws, stream))) return rc;
    if (ev && cudaEventRecord(ev[3], stream) != cudaSuccess) return GBN_ERR_CUDA;
    if (p.fix_cap) {
        rc = launch_fixup(p, ws, out, stream);
        if ((rc = checked_stage("fixup", rc, p, ws, stream))) return rc;
    }
    if (p.scale) {
        rc = launch_unscale(p, ws, out, stream);
        if ((rc = checked_stage("unscale", rc, p, ws, stream))) return rc;
    }
    if (p.bge) {
        rc = launch_bge_finalize(p, ws, out, stream);
        if ((rc = checked_stage("bge", rc, p, ws, stream))) return rc;
    }
    return GBN_OK;
}

}  // namespace gbn

extern "C" {

void givensbn_default_opts(givensbn_opts* opts) {
    if (!opts) return;
    memset(opts, 0, sizeof(*opts));
    opts->center = 1;
    opts->fixup_tau = 1e-6;
    opts->max_parents = -1;
    opts->score = GBN_SCORE_BIC;
}

int givensbn_plan_choice(int64_t n, int32_t m, const givensbn_opts* opts, int32_t* q,
                         int32_t* consumer_warps) {
    if (!q || !consumer_warps) return GBN_ERR_NULL;
    Plan p;
    const int rc = make_plan(n, m, opts, &p);
    if (rc) return rc;
    *q = p.Q;
    *consumer_warps = p.n_bwarps;
    return GBN_OK;
}

int givensbn_shard_range(int64_t n, int32_t m, const givensbn_opts* opts, int32_t* fixed_k,
                         int32_t* lane_bits, int64_t* cta_begin, int64_t* cta_end) {
    if (!fixed_k || !lane_bits || !cta_begin || !cta_end) return GBN_ERR_NULL;
    Plan p;
    const int rc = make_plan(n, m, opts, &p);
    if (rc) return rc;
    *fixed_k = p.k;
    *lane_bits = p.W;
    *cta_begin = p.cta_begin;
    *cta_end = p.cta_begin + p.n_cta;
    return GBN_OK;
}

int32_t givensbn_auto_q(int32_t m, int32_t precision) { return auto_q(m, precision); }

int givensbn_workspace_size(int64_t n, int32_t m, const givensbn_opts* opts, size_t* bytes) {
    if (!bytes) return GBN_ERR_NULL;
    Plan p;
    const int rc = make_plan(n, m, opts, &p);
    if (rc) return rc;
    *bytes = p.total_bytes;
    return GBN_OK;
}

int score_all_families(const double* X, int64_t n, int32_t m, void* out_scores,
                       const givensbn_opts* opts) {
    if (!opts) return GBN_ERR_NULL;
    Plan p;
    int rc = make_plan(n, m, opts, &p);
    if (rc) return rc;
    if (!X || !out_scores) return GBN_ERR_NULL;
    if (((uintptr_t)X & 7u) || ((uintptr_t)out_scores & 15u)) return GBN_ERR_ALIGN;
    if (!opts->workspace || opts->workspace_bytes < p.total_bytes) return GBN_ERR_WORKSPACE;
    if ((uintptr_t)opts->workspace & 255u) return GBN_ERR_ALIGN;
    char* ws = static_cast<char*>(opts->workspace);
    return run_pipeline(p, X, ws, out_scores, static_cast<cudaStream_t>(opts->stream),
                        opts->stage_events);
}

int givensbn_status(const givensbn_opts* opts, int32_t* status) {
    if (!opts || !status || !opts->workspace) return GBN_ERR_NULL;
    cudaStream_t stream = static_cast<cudaStream_t>(opts->stream);
    int32_t v = 0;
    if (cudaMemcpyAsync(&v, opts->workspace, sizeof(v), cudaMemcpyDeviceToHost, stream) !=
        cudaSuccess)
        return GBN_ERR_CUDA;
    if (cudaStreamSynchronize(stream) != cudaSuccess) return GBN_ERR_CUDA;
    *status = v;
    return GBN_OK;
}

const char* givensbn_strerror(int code) {
    switch (code) {
        case GBN_OK: return "success";
        case GBN_ERR_M: return "m outside the supported range [2, 30]";
        case GBN_ERR_N: return "n must be at least m + 1";
        case GBN_ERR_NULL: return "a required pointer is NULL";
        case GBN_ERR_ALIGN: return "a pointer is misaligned";
        case GBN_ERR_WORKSPACE: return "workspace missing or too small";
        case GBN_ERR_CUDA: return "CUDA launch or runtime error";
        case GBN_ERR_Q: return "q outside the supported range";
        case GBN_ERR_PRECISION: return "precision must be 0 (FP32) or 1 (FP64)";
        case GBN_ERR_BATCH: return "inconsistent batched arguments";
        case GBN_ERR_STATIC_SCRATCH:
            return "input too large for the 16 MiB static scratch of score_all_families_noalloc "
                   "(m <= 20 with the automatic q)";
        case GBN_ERR_OPTS:
            return "an option is outside its range (score, penalty, shard, consumer warps, "
                   "watchdog) or not supported by this entry point";
        case GBN_ERR_TUNE: return "the autotuner could not time or record a candidate";
        default: return "unknown error";
    }
}

}  // extern "C"

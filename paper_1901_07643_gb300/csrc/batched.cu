// Batched scoring: many datasets of uneven (n, m) in one set of launches.
//
// The host plans every dataset (one common sub-walk size Q), orders the
// datasets largest first, lays out one workspace region per dataset and
// writes a device-side table (plans, pointers, walk arguments, block
// prefixes) into the head of the workspace with small upload kernels whose
// payload travels as kernel parameters.  Every stage is then one launch over
// all datasets; a block finds its dataset by binary search in the prefix of
// block counts.  Nothing here allocates, copies through the runtime's memcpy
// or synchronises, so a whole call can be captured into a CUDA graph.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "walk3.cuh"

namespace gbn {
namespace {

constexpr int kUploadBytes = 30 * 1024;  // payload per upload launch (kernel parameter)

struct UploadChunk {
    unsigned char* dst;
    int bytes;
    unsigned char data[kUploadBytes];
};

__global__ void upload_kernel(const __grid_constant__ UploadChunk c) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < c.bytes; i += gridDim.x * blockDim.x)
        c.dst[i] = c.data[i];
}

size_t up256(size_t x) { return (x + 255) / 256 * 256; }

struct BatchLayout {
    std::vector<Plan> plans;
    std::vector<int32_t> launch_order;  // launch position -> dataset
    std::vector<size_t> ws_off;         // per dataset, from the workspace base
    size_t table_bytes = 0;             // device table at the workspace head
    size_t total = 0;
    int Q = 0, maxW = 0, n_cwarps = 1;
    size_t max_stride = 0;
    int64_t total_cta = 0, total_panels = 0;
    // table offsets (from the workspace base)
    size_t off_cta_prefix = 0, off_panel_prefix = 0, off_dataset_of = 0, off_plans = 0,
           off_X = 0, off_ws = 0, off_out = 0, off_args = 0;
    size_t off_panel_pos = 0, off_cta_pos = 0;  // position maps, filled on the device
    size_t off_pass2 = 0;                       // pass-2 panel prefix, filled on the device
};

int plan_batch(const int64_t* ns, const int32_t* ms, int32_t B, const givensbn_opts* opts,
               BatchLayout* L) {
    if (B < 1 || !ns || !ms) return B < 1 ? GBN_ERR_BATCH : GBN_ERR_NULL;
    givensbn_opts o;
    givensbn_default_opts(&o);
    if (opts) o = *opts;
    int precision = o.precision;
    if (precision != 0 && precision != 1) return GBN_ERR_PRECISION;
    if (o.shard_count > 1) return GBN_ERR_OPTS;  // sharding splits one table, not a batch
    int mmin = GBN_MAX_M, mmax = GBN_MIN_M;
    int64_t nsum = 0;
    for (int b = 0; b < B; ++b) {
        if (ms[b] < GBN_MIN_M || ms[b] > GBN_MAX_M) return GBN_ERR_M;
        mmin = std::min(mmin, (int)ms[b]);
        mmax = std::max(mmax, (int)ms[b]);
        nsum += ns[b];
    }
    // one Q for the whole batch: the requested one, else the autotuner's cached
    // choice for this batch's size class, else the smallest automatic choice
    int Q = o.q;
    if (Q <= 0 && o.consumer_warps == 0 && o.tune_cache && !o.debug_coverage) {
        int tq = 0, tcw = 0;
        if (tune_lookup(o.tune_cache, 1, precision, mmax, mmin, B, nsum, &tq, &tcw) &&
            tq >= kMinQ && tq <= mmin && tq <= (precision ? kMaxQFp64 : kMaxQ) && tcw >= 1 &&
            tcw <= 8) {
            Q = tq;
            o.consumer_warps = tcw;
        }
    }
    if (Q <= 0) {
        Q = 1 << 30;
        for (int b = 0; b < B; ++b) Q = std::min(Q, auto_q(ms[b], precision));
    }
    o.q = Q;
    o.fixup_tau = 0.0;  // the FP64 fix-up pass belongs to the single-dataset entry point
    if (o.score == GBN_SCORE_BGE) return GBN_ERR_OPTS;  // the BGe pass: single datasets only
    L->plans.resize(B);
    for (int b = 0; b < B; ++b) {
        const int rc = make_plan(ns[b], ms[b], &o, &L->plans[b]);
        if (rc) return rc;
    }
    L->Q = Q;
    L->maxW = 0;
    L->n_cwarps = 1;
    for (const Plan& p : L->plans) {
        L->maxW = std::max(L->maxW, p.W);
        L->max_stride = std::max(L->max_stride, p.leaf_stride);
        L->n_cwarps = std::max(L->n_cwarps, p.n_bwarps);
    }
    // largest first: walk CTAs x families per CTA
    L->launch_order.resize(B);
    for (int b = 0; b < B; ++b) L->launch_order[b] = b;
    std::stable_sort(L->launch_order.begin(), L->launch_order.end(), [&](int a, int c) {
        return ((int64_t)L->plans[a].m << L->plans[a].m) > ((int64_t)L->plans[c].m << L->plans[c].m);
    });
    size_t off = 0;
    L->off_cta_prefix = off;
    off = up256(off + sizeof(int64_t) * (B + 1));
    L->off_panel_prefix = off;
    off = up256(off + sizeof(int64_t) * (B + 1));
    L->off_dataset_of = off;
    off = up256(off + sizeof(int32_t) * B);
    L->off_plans = off;
    off = up256(off + sizeof(Plan) * B);
    L->off_X = off;
    off = up256(off + sizeof(void*) * B);
    L->off_ws = off;
    off = up256(off + sizeof(void*) * B);
    L->off_out = off;
    off = up256(off + sizeof(void*) * B);
    L->off_args = off;
    off = up256(off + std::max(sizeof(WalkArgs<float>), sizeof(WalkArgs<double>)) * B);
    L->table_bytes = off;
    L->total_cta = 0;
    L->total_panels = 0;
    for (int b = 0; b < B; ++b) {
        L->total_cta += L->plans[b].n_cta;
        L->total_panels += L->plans[b].panels;
    }
    if (L->total_cta > 0x7fffffff || L->total_panels > 0x7fffffff) return GBN_ERR_BATCH;
    L->off_panel_pos = off;
    off = up256(off + sizeof(int32_t) * (size_t)L->total_panels);
    L->off_cta_pos = off;
    off = up256(off + sizeof(int32_t) * (size_t)(L->total_cta > 0 ? L->total_cta : 1));
    L->off_pass2 = off;
    off = up256(off + sizeof(int64_t) * (size_t)(B + 1));
    L->ws_off.resize(B);
    for (int b = 0; b < B; ++b) {
        L->ws_off[b] = off;
        off = up256(off + L->plans[b].total_bytes);
    }
    L->total = off;
    return GBN_OK;
}

template <typename T>
WalkArgs<T> walk_args_for(const Plan& p, char* ws, void* out, int n_cwarps) {
    WalkArgs<T> a = make_walk_args<T>(p, ws, out);
    a.n_cwarps = n_cwarps;
    return a;
}

int upload(const std::vector<unsigned char>& host, char* dst, cudaStream_t stream) {
    static thread_local UploadChunk chunk;  // host staging for the kernel parameter
    for (size_t pos = 0; pos < host.size(); pos += kUploadBytes) {
        const size_t nb = std::min(host.size() - pos, (size_t)kUploadBytes);
        chunk.dst = reinterpret_cast<unsigned char*>(dst + pos);
        chunk.bytes = (int)nb;
        memcpy(chunk.data, host.data() + pos, nb);
        if (launch_plain(upload_kernel, dim3(32), dim3(256), 0, stream, chunk) != cudaSuccess)
            return GBN_ERR_CUDA;
    }
    return GBN_OK;
}

}  // namespace
}  // namespace gbn

using namespace gbn;

extern "C" int givensbn_batched_workspace_size(const int64_t* ns, const int32_t* ms, int32_t B,
                                               const givensbn_opts* opts, size_t* bytes) {
    if (!bytes) return GBN_ERR_NULL;
    BatchLayout L;
    const int rc = plan_batch(ns, ms, B, opts, &L);
    if (rc) return rc;
    *bytes = L.total;
    return GBN_OK;
}

extern "C" int score_all_families_batched(const double* const* Xs, const int64_t* ns,
                                          const int32_t* ms, int32_t B, void* out,
                                          const int64_t* out_offsets, const givensbn_opts* opts) {
    if (!opts || !Xs || !out || !out_offsets) return GBN_ERR_NULL;
    BatchLayout L;
    int rc = plan_batch(ns, ms, B, opts, &L);
    if (rc) return rc;
    if (!opts->workspace || opts->workspace_bytes < L.total) return GBN_ERR_WORKSPACE;
    if ((uintptr_t)opts->workspace & 255u) return GBN_ERR_ALIGN;
    const int precision = opts->precision;
    const size_t es = precision ? sizeof(double) : sizeof(float);
    char* base = static_cast<char*>(opts->workspace);
    cudaStream_t stream = static_cast<cudaStream_t>(opts->stream);
    // per-dataset pointers and checks
    std::vector<const double*> X(B);
    std::vector<char*> ws(B);
    std::vector<void*> outp(B);
    for (int b = 0; b < B; ++b) {
        if (!Xs[b]) return GBN_ERR_NULL;
        if ((uintptr_t)Xs[b] & 7u) return GBN_ERR_ALIGN;
        if (out_offsets[b] < 0) return GBN_ERR_BATCH;
        X[b] = Xs[b];
        ws[b] = base + L.ws_off[b];
        outp[b] = static_cast<char*>(out) + (size_t)out_offsets[b] * es;
        if ((uintptr_t)outp[b] & 15u) return GBN_ERR_ALIGN;
    }
    for (int b = 0; b < B; ++b)  // tables must not overlap
        for (int c = b + 1; c < B; ++c) {
            const int64_t sb = (int64_t)ms[b] << (ms[b] - 1), sc = (int64_t)ms[c] << (ms[c] - 1);
            if (out_offsets[b] < out_offsets[c] + sc && out_offsets[c] < out_offsets[b] + sb)
                return GBN_ERR_BATCH;
        }
    // device table
    std::vector<unsigned char> host(L.table_bytes, 0);
    int64_t* cta_prefix = reinterpret_cast<int64_t*>(host.data() + L.off_cta_prefix);
    int64_t* panel_prefix = reinterpret_cast<int64_t*>(host.data() + L.off_panel_prefix);
    int32_t* dataset_of = reinterpret_cast<int32_t*>(host.data() + L.off_dataset_of);
    cta_prefix[0] = panel_prefix[0] = 0;
    for (int i = 0; i < B; ++i) {
        const int b = L.launch_order[i];
        dataset_of[i] = b;
        cta_prefix[i + 1] = cta_prefix[i] + L.plans[b].n_cta;
        panel_prefix[i + 1] = panel_prefix[i] + L.plans[b].panels;
    }
    memcpy(host.data() + L.off_plans, L.plans.data(), sizeof(Plan) * B);
    memcpy(host.data() + L.off_X, X.data(), sizeof(void*) * B);
    memcpy(host.data() + L.off_ws, ws.data(), sizeof(void*) * B);
    memcpy(host.data() + L.off_out, outp.data(), sizeof(void*) * B);
    for (int b = 0; b < B; ++b) {
        if (precision) {
            const WalkArgs<double> a = walk_args_for<double>(L.plans[b], ws[b], outp[b], L.n_cwarps);
            memcpy(host.data() + L.off_args + sizeof(a) * b, &a, sizeof(a));
        } else {
            const WalkArgs<float> a = walk_args_for<float>(L.plans[b], ws[b], outp[b], L.n_cwarps);
            memcpy(host.data() + L.off_args + sizeof(a) * b, &a, sizeof(a));
        }
    }
    if ((rc = upload(host, base, stream))) return rc;
    BatchView v;
    v.B = B;
    v.cta_prefix = reinterpret_cast<const int64_t*>(base + L.off_cta_prefix);
    v.panel_prefix = reinterpret_cast<const int64_t*>(base + L.off_panel_prefix);
    v.dataset_of = reinterpret_cast<const int32_t*>(base + L.off_dataset_of);
    v.panel_pos = reinterpret_cast<int32_t*>(base + L.off_panel_pos);
    v.cta_pos = reinterpret_cast<int32_t*>(base + L.off_cta_pos);
    v.pass2_prefix = reinterpret_cast<int64_t*>(base + L.off_pass2);
    v.plans = reinterpret_cast<const Plan*>(base + L.off_plans);
    v.X = reinterpret_cast<const double* const*>(base + L.off_X);
    v.ws = reinterpret_cast<char* const*>(base + L.off_ws);
    v.out = reinterpret_cast<void* const*>(base + L.off_out);
    v.walk_args = base + L.off_args;
    v.pairs = (precision == 0 && opts->debug_coverage == 0) ? 1 : 0;
    for (int b = 0; b < B && v.pairs; ++b) {  // the paired walk's conditions, for every dataset
        const Plan& pb = L.plans[b];
        if (pb.W != 5 || pb.lanes != 32 || pb.n_cta % 2 != 0 || pb.kmax < pb.m - 1) v.pairs = 0;
    }
    int max_m = 1;
    for (int b = 0; b < B; ++b) max_m = std::max(max_m, L.plans[b].m);
    if ((rc = launch_r0_batched(v, L.total_panels, max_m, stream))) return rc;
    int64_t dfs_cta = 0;  // the launch-order prefix of datasets with at least 4 walk CTAs
    for (int i = 0; i < B && L.plans[L.launch_order[i]].n_cta >= 4; ++i)
        dfs_cta += L.plans[L.launch_order[i]].n_cta;
    if ((rc = launch_roots_batched(v, L.total_cta, dfs_cta, L.Q, L.maxW, L.max_stride, precision,
                                   stream)))
        return rc;
    return launch_walk_batched(v, L.total_cta, L.Q, precision, opts->debug_coverage != 0,
                               L.n_cwarps, stream);
}

// ---------------------------------------------------------------- the adjoint of a batch
// score_all_families_backward_batched: the R0 stage of every dataset as in a
// scoring batch (the same kernels, so each R0 is bit-identical to a single
// call's), then one launch of the adjoint walk over all datasets' sub-walks
// (warp w of the launch belongs to the dataset whose warp range holds it),
// one reduction launch and one gradient launch over (block, dataset).

namespace {

struct BwdBatchLayout {
    BatchLayout L;
    std::vector<int> Qb;
    std::vector<int64_t> n_sub, warps;
    std::vector<size_t> off_partials, off_gsym, off_muv;
    size_t off_args = 0, off_prefix = 0, total = 0;
};

int plan_bwd_batch(const int64_t* ns, const int32_t* ms, int32_t B, const givensbn_opts* opts,
                   BwdBatchLayout* K) {
    givensbn_opts o;
    givensbn_default_opts(&o);
    if (opts) o = *opts;
    if (o.shard_count > 1) return GBN_ERR_OPTS;
    const int qreq = o.q;
    o.q = 0;
    o.consumer_warps = 0;
    o.tune_cache = nullptr;
    o.debug_coverage = 0;
    int rc = plan_batch(ns, ms, B, &o, &K->L);
    if (rc) return rc;
    K->Qb.resize(B);
    K->n_sub.resize(B);
    K->warps.resize(B);
    K->off_partials.resize(B);
    K->off_gsym.resize(B);
    K->off_muv.resize(B);
    size_t off = K->L.total;
    for (int b = 0; b < B; ++b) {
        if ((rc = bwd_subwalk_plan(ms[b], qreq, &K->Qb[b], &K->n_sub[b], &K->warps[b]))) return rc;
        const size_t m = (size_t)ms[b];
        K->off_partials[b] = off;
        off = up256(off + sizeof(double) * (size_t)K->warps[b] * m * m);
        K->off_gsym[b] = off;
        off = up256(off + sizeof(double) * m * m);
        K->off_muv[b] = off;
        off = up256(off + sizeof(double) * 32);
    }
    K->off_args = off;
    off = up256(off + sizeof(BwdArgs) * B);
    K->off_prefix = off;
    off = up256(off + sizeof(int64_t) * (B + 2));  // one warp prefix per width group
    K->total = off;
    return GBN_OK;
}

}  // namespace

extern "C" int givensbn_backward_batched_workspace_size(const int64_t* ns, const int32_t* ms,
                                                        int32_t B, const givensbn_opts* opts,
                                                        size_t* bytes) {
    if (!bytes) return GBN_ERR_NULL;
    BwdBatchLayout K;
    const int rc = plan_bwd_batch(ns, ms, B, opts, &K);
    if (rc) return rc;
    *bytes = K.total;
    return GBN_OK;
}

extern "C" int score_all_families_backward_batched(const double* const* Xs, const int64_t* ns,
                                                   const int32_t* ms, int32_t B,
                                                   const void* const* weights,
                                                   double* const* grads,
                                                   const givensbn_opts* opts) {
    if (!opts || !Xs || !weights || !grads) return GBN_ERR_NULL;
    BwdBatchLayout K;
    int rc = plan_bwd_batch(ns, ms, B, opts, &K);
    if (rc) return rc;
    const BatchLayout& L = K.L;
    if (!opts->workspace || opts->workspace_bytes < K.total) return GBN_ERR_WORKSPACE;
    if ((uintptr_t)opts->workspace & 255u) return GBN_ERR_ALIGN;
    const int precision = opts->precision;
    char* base = static_cast<char*>(opts->workspace);
    cudaStream_t stream = static_cast<cudaStream_t>(opts->stream);
    std::vector<const double*> X(B);
    std::vector<char*> ws(B);
    std::vector<void*> outp(B, nullptr);
    for (int b = 0; b < B; ++b) {
        if (!Xs[b] || !weights[b] || !grads[b]) return GBN_ERR_NULL;
        if (((uintptr_t)Xs[b] & 7u) || ((uintptr_t)weights[b] & 15u) || ((uintptr_t)grads[b] & 7u))
            return GBN_ERR_ALIGN;
        X[b] = Xs[b];
        ws[b] = base + L.ws_off[b];
    }
    // the scoring batch's device table (prefixes, plans, pointers) ...
    std::vector<unsigned char> host(L.table_bytes, 0);
    int64_t* cta_prefix = reinterpret_cast<int64_t*>(host.data() + L.off_cta_prefix);
    int64_t* panel_prefix = reinterpret_cast<int64_t*>(host.data() + L.off_panel_prefix);
    int32_t* dataset_of = reinterpret_cast<int32_t*>(host.data() + L.off_dataset_of);
    cta_prefix[0] = panel_prefix[0] = 0;
    for (int i = 0; i < B; ++i) {
        const int b = L.launch_order[i];
        dataset_of[i] = b;
        cta_prefix[i + 1] = cta_prefix[i] + L.plans[b].n_cta;
        panel_prefix[i + 1] = panel_prefix[i] + L.plans[b].panels;
    }
    memcpy(host.data() + L.off_plans, L.plans.data(), sizeof(Plan) * B);
    memcpy(host.data() + L.off_X, X.data(), sizeof(void*) * B);
    memcpy(host.data() + L.off_ws, ws.data(), sizeof(void*) * B);
    memcpy(host.data() + L.off_out, outp.data(), sizeof(void*) * B);
    if ((rc = upload(host, base, stream))) return rc;
    // ... and the adjoint's: per-dataset arguments, datasets with m <= 16 first (the
    // 16-column kernel), each width group with its own prefix of warps
    std::vector<unsigned char> tail(K.total - K.off_args, 0);
    BwdArgs* args = reinterpret_cast<BwdArgs*>(tail.data());
    int64_t* prefix = reinterpret_cast<int64_t*>(tail.data() + (K.off_prefix - K.off_args));
    int B_narrow = 0;
    for (int b = 0; b < B; ++b) B_narrow += ms[b] <= 16;
    int64_t warps_group[2] = {0, 0};
    int slot[2] = {0, B_narrow};
    prefix[0] = 0;
    prefix[B_narrow + 1] = 0;
    for (int b = 0; b < B; ++b) {
        const int grp = ms[b] <= 16 ? 0 : 1;
        const int i = slot[grp]++;
        args[i] = bwd_args(L.plans[b], ws[b], X[b], weights[b], grads[b], K.Qb[b], K.n_sub[b],
                           K.warps[b], reinterpret_cast<double*>(base + K.off_partials[b]),
                           reinterpret_cast<double*>(base + K.off_gsym[b]),
                           reinterpret_cast<double*>(base + K.off_muv[b]));
        warps_group[grp] += K.warps[b];
        prefix[i + grp + 1] = prefix[i + grp] + K.warps[b];
    }
    if ((rc = upload(tail, base + K.off_args, stream))) return rc;
    BatchView v;
    v.B = B;
    v.cta_prefix = reinterpret_cast<const int64_t*>(base + L.off_cta_prefix);
    v.panel_prefix = reinterpret_cast<const int64_t*>(base + L.off_panel_prefix);
    v.dataset_of = reinterpret_cast<const int32_t*>(base + L.off_dataset_of);
    v.panel_pos = reinterpret_cast<int32_t*>(base + L.off_panel_pos);
    v.cta_pos = reinterpret_cast<int32_t*>(base + L.off_cta_pos);
    v.pass2_prefix = reinterpret_cast<int64_t*>(base + L.off_pass2);
    v.plans = reinterpret_cast<const Plan*>(base + L.off_plans);
    v.X = reinterpret_cast<const double* const*>(base + L.off_X);
    v.ws = reinterpret_cast<char* const*>(base + L.off_ws);
    v.out = reinterpret_cast<void* const*>(base + L.off_out);
    v.walk_args = nullptr;
    v.pairs = 0;
    int max_m = 1;
    for (int b = 0; b < B; ++b) max_m = std::max(max_m, L.plans[b].m);
    if ((rc = launch_r0_batched(v, L.total_panels, max_m, stream))) return rc;
    return launch_bwd_batched(reinterpret_cast<const BwdArgs*>(base + K.off_args),
                              reinterpret_cast<const int64_t*>(base + K.off_prefix), B, B_narrow,
                              warps_group[0], warps_group[1], precision, stream);
}

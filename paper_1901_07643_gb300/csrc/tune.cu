// Autotuner of the walk's launch shape: the sub-walk size q and the number of
// consumer warps per walk block, measured on the device.
//
// q is the free parameter of the parallel split (Sec. 6, Algorithm 2): the
// table is walked as 2^(m-q) sub-walks of the greedy sequence Upsilon(q) of
// Algorithm 1.  Small q means many sub-walk roots to build, large q a long
// unrolled replay and a large tape in shared memory; where the balance lies
// depends on m, n, the precision and the device, so it is measured.  Each
// candidate (q, consumer warps) runs the whole scoring call (one untimed call,
// then kTuneReps timed ones with CUDA events on the caller's stream); the
// fastest median wins.  The result can be appended to a cache file, one line
// per measurement:
//
//   gbn-tune-v1 device=<name> kind=<single|batch> precision=<0|1> m=<m> mmin=<m>
//               count=<datasets> nlog2=<floor(log2 n)> q=<q> cw=<warps> ms=<time>
//
// (one line in the file; for a batch m and mmin are the largest and smallest
// m, count the number of datasets and n the total of their rows).  A plan with
// q == 0 and consumer_warps == 0 and a cache path takes the last line that
// matches this device (or device=*) and the size class; lines that do not
// parse or do not match are ignored, so a missing or foreign file falls back
// to the automatic choice.
#include <math.h>
#include <stdio.h>
#include <string.h>
#include <sys/stat.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#include "gbn_internal.cuh"

namespace gbn {
namespace {

constexpr int kTuneReps = 3;
constexpr int kMaxDevices = 64;

struct TuneEntry {
    std::string device;
    int batched = 0, precision = 0, m = 0, mmin = 0, nlog2 = 0, q = 0, cw = 0;
    long long count = 0;
    double ms = 0.0;
};

struct CacheFile {
    std::string path;
    long long mtime_ns = -1;
    long long size = -1;
    std::vector<TuneEntry> entries;
};

std::mutex g_tune_mu;
std::vector<CacheFile> g_files;
std::string g_dev_name[kMaxDevices];
bool g_dev_known[kMaxDevices] = {};

int floor_log2(int64_t n) {
    int l = 0;
    while (n > 1) {
        n >>= 1;
        ++l;
    }
    return l;
}

// Name of the current device with blanks replaced, "" without a device.
std::string device_name() {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();  // no device: clear the error this query just raised
        return std::string();
    }
    if (!g_dev_known[dev]) {
        cudaDeviceProp prop;
        std::string s;
        if (cudaGetDeviceProperties(&prop, dev) == cudaSuccess) {
            s = prop.name;
            for (char& c : s)
                if (c == ' ' || c == '\t' || c == '=') c = '_';
        }
        g_dev_name[dev] = s;
        g_dev_known[dev] = true;
    }
    return g_dev_name[dev];
}

bool parse_line(const char* line, TuneEntry* e) {
    char buf[512];
    strncpy(buf, line, sizeof(buf) - 1);
    buf[sizeof(buf) - 1] = '\0';
    char* save = nullptr;
    char* tok = strtok_r(buf, " \t\r\n", &save);
    if (!tok || strcmp(tok, "gbn-tune-v1") != 0) return false;
    int seen = 0;
    while ((tok = strtok_r(nullptr, " \t\r\n", &save))) {
        char* eq = strchr(tok, '=');
        if (!eq) return false;
        *eq = '\0';
        const char* key = tok;
        const char* val = eq + 1;
        char* end = nullptr;
        if (!strcmp(key, "device")) {
            e->device = val;
            seen |= 1;
        } else if (!strcmp(key, "kind")) {
            if (!strcmp(val, "single")) e->batched = 0;
            else if (!strcmp(val, "batch")) e->batched = 1;
            else return false;
            seen |= 2;
        } else if (!strcmp(key, "ms")) {
            e->ms = strtod(val, &end);
            if (end == val) return false;
        } else {
            const long long v = strtoll(val, &end, 10);
            if (end == val || *end != '\0') return false;
            if (!strcmp(key, "precision")) e->precision = (int)v, seen |= 4;
            else if (!strcmp(key, "m")) e->m = (int)v, seen |= 8;
            else if (!strcmp(key, "mmin")) e->mmin = (int)v, seen |= 16;
            else if (!strcmp(key, "count")) e->count = v, seen |= 32;
            else if (!strcmp(key, "nlog2")) e->nlog2 = (int)v, seen |= 64;
            else if (!strcmp(key, "q")) e->q = (int)v, seen |= 128;
            else if (!strcmp(key, "cw")) e->cw = (int)v, seen |= 256;
        }
    }
    return seen == 511;
}

// The parsed cache file at `path`, re-read when its size or time changes
// (the caller holds g_tune_mu).  nullptr when it cannot be read.
const CacheFile* cache_for(const char* path) {
    struct stat st;
    if (stat(path, &st) != 0) return nullptr;
    const long long mt = (long long)st.st_mtim.tv_sec * 1000000000ll + st.st_mtim.tv_nsec;
    CacheFile* f = nullptr;
    for (CacheFile& c : g_files)
        if (c.path == path) f = &c;
    if (!f) {
        g_files.emplace_back();
        f = &g_files.back();
        f->path = path;
    }
    if (f->mtime_ns == mt && f->size == (long long)st.st_size) return f;
    f->entries.clear();
    f->mtime_ns = mt;
    f->size = (long long)st.st_size;
    FILE* fp = fopen(path, "r");
    if (!fp) return nullptr;
    char line[512];
    while (fgets(line, sizeof(line), fp)) {
        TuneEntry e;
        if (parse_line(line, &e)) f->entries.push_back(e);
    }
    fclose(fp);
    return f;
}

int append_entry(const char* path, const TuneEntry& e) {
    FILE* fp = fopen(path, "a");
    if (!fp) return GBN_ERR_TUNE;
    const int w = fprintf(fp,
                          "gbn-tune-v1 device=%s kind=%s precision=%d m=%d mmin=%d count=%lld "
                          "nlog2=%d q=%d cw=%d ms=%.6f\n",
                          e.device.empty() ? "*" : e.device.c_str(), e.batched ? "batch" : "single",
                          e.precision, e.m, e.mmin, e.count, e.nlog2, e.q, e.cw, e.ms);
    const int c = fclose(fp);
    return (w > 0 && c == 0) ? GBN_OK : GBN_ERR_TUNE;
}

// Candidate q values around a centre choice, within [lo, hi].
std::vector<int> q_candidates(int centre, int lo, int hi) {
    std::vector<int> v;
    for (int q = centre - 1; q <= centre + 1; ++q)
        if (q >= lo && q <= hi) v.push_back(q);
    if (v.empty() && lo <= hi) v.push_back(std::min(std::max(centre, lo), hi));
    return v;
}
constexpr int kCwCandidates[] = {4, 6, 8};

int max_q_for(int precision) { return precision ? kMaxQFp64 : kMaxQ; }

// Median of kTuneReps timed runs of fn (after one untimed run), in ms.
template <class F>
int time_call(F&& fn, cudaStream_t stream, double* ms) {
    cudaEvent_t a = nullptr, b = nullptr;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
        if (a) cudaEventDestroy(a);
        return GBN_ERR_CUDA;
    }
    int rc = fn();
    std::vector<double> t;
    for (int r = 0; r < kTuneReps && rc == GBN_OK; ++r) {
        if (cudaEventRecord(a, stream) != cudaSuccess) rc = GBN_ERR_CUDA;
        if (rc == GBN_OK) rc = fn();
        if (rc == GBN_OK && cudaEventRecord(b, stream) != cudaSuccess) rc = GBN_ERR_CUDA;
        float e = 0.f;
        if (rc == GBN_OK && (cudaEventSynchronize(b) != cudaSuccess ||
                             cudaEventElapsedTime(&e, a, b) != cudaSuccess))
            rc = GBN_ERR_CUDA;
        t.push_back(e);
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (rc) return rc;
    std::sort(t.begin(), t.end());
    *ms = t[t.size() / 2];
    return GBN_OK;
}

}  // namespace

bool tune_lookup(const char* path, int batched, int precision, int m, int mmin, int64_t count,
                 int64_t n, int* q, int* cw) {
    if (!path || !*path) return false;
    std::lock_guard<std::mutex> lock(g_tune_mu);
    const CacheFile* f = cache_for(path);
    if (!f) return false;
    const std::string dev = device_name();
    const int nl = floor_log2(n);
    for (auto it = f->entries.rbegin(); it != f->entries.rend(); ++it) {
        const TuneEntry& e = *it;
        if (e.batched != batched || e.precision != precision || e.m != m || e.mmin != mmin ||
            e.count != count || e.nlog2 != nl)
            continue;
        if (e.device != "*" && (dev.empty() || e.device != dev)) continue;
        *q = e.q;
        *cw = e.cw;
        return true;
    }
    return false;
}

}  // namespace gbn

using namespace gbn;

namespace {

// The candidate plans' options for one dataset (or a batch: centre q = the
// batch's automatic choice, q at most the smallest m).
std::vector<givensbn_opts> single_candidates(int32_t m, const givensbn_opts& base) {
    std::vector<givensbn_opts> c;
    const int prec = base.precision;
    for (int q : q_candidates(auto_q(m, prec), kMinQ, std::min(max_q_for(prec), (int)m)))
        for (int cw : kCwCandidates) {
            givensbn_opts o = base;
            o.q = q;
            o.consumer_warps = cw;
            o.tune_cache = nullptr;
            o.debug_coverage = 0;
            c.push_back(o);
        }
    return c;
}

std::vector<givensbn_opts> batch_candidates(const int32_t* ms, int32_t B,
                                            const givensbn_opts& base) {
    std::vector<givensbn_opts> c;
    const int prec = base.precision;
    int centre = 1 << 30, mmin = GBN_MAX_M;
    for (int b = 0; b < B; ++b) {
        centre = std::min(centre, auto_q(ms[b], prec));
        mmin = std::min(mmin, (int)ms[b]);
    }
    for (int q : q_candidates(centre, kMinQ, std::min(max_q_for(prec), mmin)))
        for (int cw : kCwCandidates) {
            givensbn_opts o = base;
            o.q = q;
            o.consumer_warps = cw;
            o.tune_cache = nullptr;
            o.debug_coverage = 0;
            c.push_back(o);
        }
    return c;
}

int finish(const givensbn_opts* opts, TuneEntry best, const std::vector<givensbn_tune_result>& all,
           int32_t* q_out, int32_t* cw_out, double* ms_out, givensbn_tune_result* results,
           int32_t max_results, int32_t* n_results) {
    if (q_out) *q_out = best.q;
    if (cw_out) *cw_out = best.cw;
    if (ms_out) *ms_out = best.ms;
    if (n_results) *n_results = (int32_t)all.size();
    if (results)
        for (int i = 0; i < (int)all.size() && i < max_results; ++i) results[i] = all[i];
    if (opts->tune_cache && *opts->tune_cache) {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        best.device = device_name();
        return append_entry(opts->tune_cache, best);
    }
    return GBN_OK;
}

}  // namespace

extern "C" int givensbn_autotune_workspace_size(int64_t n, int32_t m, const givensbn_opts* opts,
                                                size_t* bytes) {
    if (!bytes || !opts) return GBN_ERR_NULL;
    size_t mx = 0;
    for (const givensbn_opts& o : single_candidates(m, *opts)) {
        size_t b = 0;
        const int rc = givensbn_workspace_size(n, m, &o, &b);
        if (rc) return rc;
        mx = std::max(mx, b);
    }
    *bytes = mx;
    return GBN_OK;
}

extern "C" int givensbn_autotune(const double* X, int64_t n, int32_t m, void* out_scores,
                                 const givensbn_opts* opts, int32_t* q_out, int32_t* cw_out,
                                 double* ms_out, givensbn_tune_result* results,
                                 int32_t max_results, int32_t* n_results) {
    if (!opts) return GBN_ERR_NULL;
    if (opts->debug_coverage) return GBN_ERR_OPTS;
    const std::vector<givensbn_opts> cands = single_candidates(m, *opts);
    if (cands.empty()) return GBN_ERR_Q;
    cudaStream_t stream = static_cast<cudaStream_t>(opts->stream);
    TuneEntry best;
    best.ms = 1e300;
    std::vector<givensbn_tune_result> all;
    for (const givensbn_opts& o : cands) {
        givensbn_opts oc = o;
        oc.stage_events = nullptr;
        double ms = 0.0;
        const int rc = time_call([&] { return score_all_families(X, n, m, out_scores, &oc); },
                                 stream, &ms);
        if (rc) return rc;
        all.push_back(givensbn_tune_result{oc.q, oc.consumer_warps, ms});
        if (ms < best.ms) {
            best.ms = ms;
            best.q = oc.q;
            best.cw = oc.consumer_warps;
        }
    }
    best.batched = 0;
    best.precision = opts->precision;
    best.m = m;
    best.mmin = m;
    best.count = 1;
    best.nlog2 = floor_log2(n);
    return finish(opts, best, all, q_out, cw_out, ms_out, results, max_results, n_results);
}

extern "C" int givensbn_autotune_batched_workspace_size(const int64_t* ns, const int32_t* ms,
                                                        int32_t B, const givensbn_opts* opts,
                                                        size_t* bytes) {
    if (!bytes || !opts || !ns || !ms) return GBN_ERR_NULL;
    if (B < 1) return GBN_ERR_BATCH;
    for (int b = 0; b < B; ++b)
        if (ms[b] < GBN_MIN_M || ms[b] > GBN_MAX_M) return GBN_ERR_M;
    size_t mx = 0;
    for (const givensbn_opts& o : batch_candidates(ms, B, *opts)) {
        size_t b = 0;
        const int rc = givensbn_batched_workspace_size(ns, ms, B, &o, &b);
        if (rc) return rc;
        mx = std::max(mx, b);
    }
    *bytes = mx;
    return GBN_OK;
}

extern "C" int givensbn_autotune_batched(const double* const* Xs, const int64_t* ns,
                                         const int32_t* ms, int32_t B, void* out,
                                         const int64_t* out_offsets, const givensbn_opts* opts,
                                         int32_t* q_out, int32_t* cw_out, double* ms_out,
                                         givensbn_tune_result* results, int32_t max_results,
                                         int32_t* n_results) {
    if (!opts || !ns || !ms) return GBN_ERR_NULL;
    if (opts->debug_coverage) return GBN_ERR_OPTS;
    if (B < 1) return GBN_ERR_BATCH;
    for (int b = 0; b < B; ++b)
        if (ms[b] < GBN_MIN_M || ms[b] > GBN_MAX_M) return GBN_ERR_M;
    const std::vector<givensbn_opts> cands = batch_candidates(ms, B, *opts);
    if (cands.empty()) return GBN_ERR_Q;
    cudaStream_t stream = static_cast<cudaStream_t>(opts->stream);
    TuneEntry best;
    best.ms = 1e300;
    std::vector<givensbn_tune_result> all;
    for (const givensbn_opts& o : cands) {
        givensbn_opts oc = o;
        double t = 0.0;
        const int rc = time_call(
            [&] { return score_all_families_batched(Xs, ns, ms, B, out, out_offsets, &oc); },
            stream, &t);
        if (rc) return rc;
        all.push_back(givensbn_tune_result{oc.q, oc.consumer_warps, t});
        if (t < best.ms) {
            best.ms = t;
            best.q = oc.q;
            best.cw = oc.consumer_warps;
        }
    }
    int mmin = GBN_MAX_M, mmax = GBN_MIN_M;
    int64_t nsum = 0;
    for (int b = 0; b < B; ++b) {
        mmin = std::min(mmin, (int)ms[b]);
        mmax = std::max(mmax, (int)ms[b]);
        nsum += ns[b];
    }
    best.batched = 1;
    best.precision = opts->precision;
    best.m = mmax;
    best.mmin = mmin;
    best.count = B;
    best.nlog2 = floor_log2(nsum);
    return finish(opts, best, all, q_out, cw_out, ms_out, results, max_results, n_results);
}

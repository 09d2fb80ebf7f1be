// Internal declarations shared by the CUDA translation units of libgivensbn.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/givensbn.h"

// Checked builds (-DGBN_CHECKED) test every computed global or shared-memory
// index against its bound before the access; a violation skips the access and
// records (count, site, index, bound) in four 64-bit words of the workspace
// status block.  Ordinary builds compile the checks away.
#ifdef GBN_CHECKED
__device__ __forceinline__ bool gbn_in_bounds(unsigned long long* rec, int site, long long idx,
                                              long long bound) {
    if (idx >= 0 && idx < bound) return true;
    if (atomicAdd(rec, 1ull) == 0ull) {
        rec[1] = (unsigned long long)site;
        rec[2] = (unsigned long long)idx;
        rec[3] = (unsigned long long)bound;
    }
    return false;
}
#define GBN_IN(rec, site, idx, bound) \
    gbn_in_bounds((rec), (site), (long long)(idx), (long long)(bound))
#else
#define GBN_IN(rec, site, idx, bound) true
#endif

namespace gbn {

constexpr int kCheckOffset = 64;    // byte offset of the check record in the status block
constexpr int kTimingOffset = 128;  // byte offset of the timing counters (timing builds)
constexpr int kFixCountOffset = 16; // byte offset of the fix-up list length (unsigned)
constexpr int kR0OnePassOffset = 32; // byte offset of the R0 stage's one-pass flag (int)
constexpr int kFixCap = 1 << 18;    // fix-up list capacity (families)

constexpr int kMaxQ = 9;     // largest sub-walk size compiled (FP32; the tape lives in shared memory)
constexpr int kMaxQFp64 = 8; // FP64: the register-resident block is twice as large
constexpr int kMinQ = 2;
constexpr int kItemsPerWarp = 3;  // columns each consumer warp replays, for the largest CTA
constexpr int kLaneBits = 5; // sub-walks per warp = 2^kLaneBits (one per lane)

// Row-panel count for the tall-skinny passes over X.
constexpr int kMaxPanels = 304;

// Execution plan of one scoring call (host side, passed to kernels by value).
struct Plan {
    int m = 0;        // variables
    int64_t n = 0;    // samples
    int precision = 0;
    int Q = 0;        // variables per sub-walk (the free block, walked by Algorithm 1)
    int k = 0;        // fixed variables = m - Q (the bits of Algorithm 2's processor code)
    int W = 0;        // fixed variables that vary across the lanes of a warp, min(5, k)
    int lanes = 0;    // 2^W sub-walks per CTA
    int64_t n_cta = 0;        // sub-walk CTAs of this call (all 2^(k-W) unless sharded)
    int64_t n_cta_total = 0;  // 2^(k-W): sub-walk CTAs of the whole table
    int64_t cta_begin = 0;    // global index of this call's first CTA (even when n_cta is)
    int order[32] = {}; // column order of R0: [W..k-1, W-1..0, k..m-1]
    int panels = 0;
    int rows_per_panel = 0;
    int center = 1;
    int coverage = 0;
    // workspace layout (byte offsets)
    size_t off_status = 0, off_colsum = 0, off_mu = 0, off_gram = 0, off_gsum = 0, off_r1 = 0;
    size_t off_r1inv = 0;
    size_t off_r0 = 0;
    size_t off_leaves = 0;
    size_t off_top = 0;      // the CTA roots of the sub-walk tree (nodes at depth k - W)
    size_t off_fix = 0;      // fix-up: [mask (u32) | pad | thr float[32]] then the slot list
    int fix_cap = 0;         // 0: no fix-up (FP64 walk, coverage mode or fixup_tau == 0)
    double fix_tau = 0.0;
    size_t total_bytes = 0;
    size_t leaf_stride = 0;  // elements per CTA leaf record
    int n_bwarps = 1;        // consumer warps per walk CTA (they loop over the CTA's columns)
    double lam = 0.0;        // score penalty per parent (ln n: BIC, 2: AIC, or the caller's)
    int kmax = 0;            // in-degree bound: families with more parents are not written (m-1: none)
    long long watchdog_ns = 0;  // bound on every wait between the warps of a walk block
    // BGe score: the walk runs over a factor of t I + S_n and stores n ln(rho / n); a
    // pass over the table then forms the BGe scores (L: 2^m elements at off_bge)
    int bge = 0;
    double bge_t = 0.0, bge_alpha_mu = 0.0, bge_alpha_w = 0.0;
    size_t off_bge = 0;
    // FP32 walk: R0's columns scaled by powers of two into a safe range before the
    // FP32 stages, the scores of scaled children corrected after the walk
    // (exponents by variable and an any-scaled word at off_scale)
    int scale = 0;
    size_t off_scale = 0;
    __host__ __device__ bool sharded() const { return cta_begin != 0 || n_cta != n_cta_total; }
};

// Whether this call wrote slot s (compressed parent mask) of child c: the
// family's parent count is within the bound, and with sharding its sub-walk
// CTA, (S & H) >> W with H the fixed variables 0..k-1, is in the call's range.
__device__ __forceinline__ bool slot_written(const Plan& p, int c, int64_t s) {
    const uint64_t cs = (uint64_t)s;
    if (__popcll(cs) > p.kmax) return false;
    if (!p.sharded()) return true;
    const uint64_t S = (cs & ((1ull << c) - 1ull)) | ((cs >> c) << (c + 1));
    const int64_t g = (int64_t)((S & ((1ull << p.k) - 1ull)) >> p.W);
    return g >= p.cta_begin && g < p.cta_begin + p.n_cta;
}

// A wait inside the walk that lasts this long means the schedule is broken.
constexpr long long kWatchdogNs = 2000000000ll;

// Sub-walk CTAs [*begin, *end) of shard `index` of `count` (the table split
// into contiguous ranges of CTA pairs, so that every range starts even).
void shard_range(int64_t n_cta_total, int index, int count, int64_t* begin, int64_t* end);
// The autotuner's cached (q, consumer warps) for this device and size class;
// false when the cache has no usable entry.
bool tune_lookup(const char* path, int batched, int precision, int m, int mmin, int64_t count,
                 int64_t n, int* q, int* cw);

int make_plan(int64_t n, int32_t m, const givensbn_opts* opts, Plan* plan);
int auto_q(int m, int precision);

// Stages (each enqueues kernels on `stream`; return GBN_OK or GBN_ERR_CUDA).
int launch_r0(const Plan& p, const double* X, char* ws, cudaStream_t stream);
int launch_roots(const Plan& p, char* ws, cudaStream_t stream);
size_t top_node_bytes(const Plan& p);
int launch_walk(const Plan& p, char* ws, void* out, cudaStream_t stream);
// Ill-conditioned families (FP32 walk): flag the variables whose smallest
// possible RSS is tiny before the walk, recompute the listed families after it.
int launch_fix_flags(const Plan& p, char* ws, cudaStream_t stream);
int launch_fixup(const Plan& p, char* ws, void* out, cudaStream_t stream);
// BGe: R0 <- the factor of R0^T R0 + t I (before the flags and roots), and the
// pass that turns the walk's table into BGe scores (after the fix-up).
int launch_bge_prior(const Plan& p, char* ws, cudaStream_t stream);
int launch_bge_finalize(const Plan& p, char* ws, void* out, cudaStream_t stream);
// FP32 walk: equilibrate R0's columns (after the R0 stage) and correct the
// scaled children's scores (after the fix-up).
int launch_scale_r0(const Plan& p, char* ws, cudaStream_t stream);
int launch_unscale(const Plan& p, char* ws, void* out, cudaStream_t stream);
// The whole single-dataset pipeline (R0, flags, roots, walk, fix-up).
int run_pipeline(const Plan& p, const double* X, char* ws, void* out, cudaStream_t stream,
                 void* stage_events);

// The t-th swap (0-based t, 1-based swap index in [1, Q-1]) of the greedy
// sequence Upsilon(Q) of Algorithm 1, read as
//     Upsilon(q) = Upsilon(q-1) : [q-1 .. 1] : (Upsilon(q-1) + 1),
// evaluated by descending the recursion (O(Q) per call).  Returns 0 when t is
// outside [0, 2^Q - Q - 1).
__host__ __device__ inline int upsilon_at(int Q, int64_t t) {
    int shift = 0, q = Q;
    while (q >= 2 && t >= 0) {
        const int64_t len = ((int64_t)1 << (q - 1)) - (q - 1) - 1;  // |Upsilon(q-1)|
        if (t < len) {
            --q;
            continue;
        }
        t -= len;
        if (t < q - 1) return shift + (q - 1) - (int)t;
        t -= q - 1;
        ++shift;
        --q;
    }
    return 0;
}

// Device view of a batch (see batched.cu): per-dataset plans and pointers, and
// the running block counts of the stages in launch order (largest dataset
// first).  Kernels map a block to (dataset, local block) with batch_locate.
struct BatchView {
    int B = 0;
    const int64_t* cta_prefix = nullptr;    // B+1: sub-walk CTAs (roots, walk)
    const int64_t* panel_prefix = nullptr;  // B+1: row panels (R0 passes)
    const int32_t* dataset_of = nullptr;    // launch position -> dataset index
    int32_t* panel_pos = nullptr;           // global row panel -> launch position
    int32_t* cta_pos = nullptr;             // global sub-walk CTA -> launch position
    int64_t* pass2_prefix = nullptr;        // B+1: row panels of the datasets that need
                                            // CholeskyQR's second pass (filled on the device)
    const Plan* plans = nullptr;
    const double* const* X = nullptr;
    char* const* ws = nullptr;              // per-dataset workspace region
    void* const* out = nullptr;             // per-dataset score table
    const void* walk_args = nullptr;        // WalkArgs<T>[B]
    int pairs = 0;                          // every dataset takes the paired FP32 walk
};

// Programmatic dependent launch.  A kernel launched with launch_dep may be
// dispatched while the previous kernel on the stream finishes; every such
// kernel calls grid_dep_wait() before anything else, which returns once the
// previous kernel has completed and its writes are visible, so results are
// those of plain stream order (without such a launch the wait is a no-op).
// grid_dep_launch() lets the next kernel be dispatched before this one ends.
__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_dep_launch() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
template <typename... KArgs, typename... Args>
inline cudaError_t launch_dep(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                              cudaStream_t stream, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// A plain launch whose own error is returned (cudaLaunchKernelEx reports the
// launch's error without reading or clearing the thread's sticky error state,
// which may hold an error of the caller's unrelated work).
template <typename... KArgs, typename... Args>
inline cudaError_t launch_plain(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                                cudaStream_t stream, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cfg.attrs = nullptr;
    cfg.numAttrs = 0;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}
inline int launch_rc(cudaError_t e) { return e == cudaSuccess ? GBN_OK : GBN_ERR_CUDA; }

__device__ __forceinline__ int batch_locate(const BatchView& v, const int64_t* prefix,
                                            const int32_t* pos, int64_t bx, int64_t& local) {
    const int l = pos[bx];  // filled from the prefix once per call (launch_r0_batched)
    local = bx - prefix[l];
    return v.dataset_of[l];
}

// Dataset index for global block bx: the launch position l with
// prefix[l] <= bx < prefix[l+1] (read from the position map pos, which the
// first kernel of launch_r0_batched fills for panels and CTAs); local = bx - prefix[l].
int launch_r0_batched(const BatchView& v, int64_t total_panels, int max_m, cudaStream_t stream);

// The adjoint walk of one dataset (backward.cu): its R0, weights, per-warp
// FP64 partial sums of Gbar and the outputs.
struct BwdArgs {
    const double* R0;      // m x m, plan column order
    const void* w;         // weights, table layout (float or double)
    double* partials;      // [warps][m*m], one slot per warp of this dataset
    int* status;
    unsigned long long* chk;
    int m, k, Q;
    int64_t n_sub;         // 2^k sub-walks
    int64_t warps;         // warps given to this dataset
    double n;              // samples
    int order[32];         // plan order: position -> variable of R0's columns
    const double* X;       // the data (n x m), for grad_X = Xc (Gbar + Gbar^T)
    int64_t rows;
    const double* mu_plan; // column means, plan order
    double* gsym;          // m x m: Gbar + Gbar^T
    double* mu_var;        // the means by variable
    double* grad;          // n x m output
};
int bwd_subwalk_plan(int m, int q_requested, int* Qb, int64_t* n_sub, int64_t* warps);
BwdArgs bwd_args(const Plan& p, char* ws, const double* X, const void* w, double* grad, int Qb,
                 int64_t n_sub, int64_t warps, double* partials, double* gsym, double* mu_var);
// The adjoint walk of a batch: args[0, B_narrow) hold datasets with m <= 16
// (the 16-column kernel; warp prefix at prefix[0, B_narrow]), args[B_narrow, B)
// the rest (warp prefix at prefix[B_narrow + 1, B + 1]); then the reduction and
// the gradient of every dataset.
int launch_bwd_batched(const BwdArgs* args, const int64_t* prefix, int B, int B_narrow,
                       int64_t warps_narrow, int64_t warps_wide, int precision,
                       cudaStream_t stream);
// dfs_cta: the walk CTAs of the launch-order prefix of datasets with at least 4
// CTAs each (their top nodes depth first, four CTAs per warp).
int launch_roots_batched(const BatchView& v, int64_t total_cta, int64_t dfs_cta, int Q, int max_w,
                         size_t max_stride, int precision, cudaStream_t stream);
int launch_walk_batched(const BatchView& v, int64_t total_cta, int Q, int precision, bool coverage,
                        int n_cwarps, cudaStream_t stream);

// Leaf record of one CTA (2^W sub-walk roots), elements of the scalar type,
// lane-interleaved so that lane l of a warp reads element e at [e*32 + l]:
//   [0, LQ*32)                 L block, packed upper triangle, e = p(p+1)/2 + r
//   [LQ*32, LQ*32 + k(Q+1)*32) per fixed variable v: rows 0..Q-1 of its column
//                              in the sub-walk basis, then its residual C
inline size_t leaf_stride_elems(int Q, int k) {
    return (size_t)32 * ((size_t)Q * (Q + 1) / 2 + (size_t)k * (Q + 1));
}

}  // namespace gbn

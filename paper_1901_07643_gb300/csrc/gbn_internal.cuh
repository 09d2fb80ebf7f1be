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
    int64_t n_cta = 0;  // 2^(k-W) CTAs
    int order[32] = {}; // column order of R0: [W..k-1, 0..W-1, k..m-1]
    int panels = 0;
    int rows_per_panel = 0;
    int center = 1;
    int coverage = 0;
    // workspace layout (byte offsets)
    size_t off_status = 0, off_colsum = 0, off_gram = 0, off_r1 = 0, off_r0 = 0, off_leaves = 0;
    size_t total_bytes = 0;
    size_t leaf_stride = 0;  // elements per CTA leaf record
    int n_bwarps = 1;        // consumer warps per walk CTA (they loop over the CTA's columns)
};

int make_plan(int64_t n, int32_t m, const givensbn_opts* opts, Plan* plan);

// Stages (each enqueues kernels on `stream`; return GBN_OK or GBN_ERR_CUDA).
int launch_r0(const Plan& p, const double* X, char* ws, cudaStream_t stream);
int launch_roots(const Plan& p, char* ws, cudaStream_t stream);
int launch_walk(const Plan& p, char* ws, void* out, cudaStream_t stream);

// Leaf record of one CTA (2^W sub-walk roots), elements of the scalar type,
// lane-interleaved so that lane l of a warp reads element e at [e*32 + l]:
//   [0, LQ*32)                 L block, packed upper triangle, e = p(p+1)/2 + r
//   [LQ*32, LQ*32 + k(Q+1)*32) per fixed variable v: rows 0..Q-1 of its column
//                              in the sub-walk basis, then its residual C
inline size_t leaf_stride_elems(int Q, int k) {
    return (size_t)32 * ((size_t)Q * (Q + 1) / 2 + (size_t)k * (Q + 1));
}

}  // namespace gbn

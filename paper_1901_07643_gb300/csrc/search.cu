// Exact structure search over the local-score table: the use of the
// all-family scores that motivates the method (Sec. 1: structure learning of
// a Bayesian network from every child / parent-set score).
//
// With scores where lower is better and no constraint but acyclicity, an
// optimal DAG is found by dynamic programming over variable subsets:
//   1. best parents: B[c][U] = min over S subset of U of score(c, S), for every
//      child c and candidate set U of the other variables, with its argmin;
//   2. sinks: F[W] = min over c in W of F[W \ c] + B[c][W \ c], F[empty] = 0,
//      the score of the best network on the variables W (c is W's sink, the
//      last variable of an optimal ordering of W);
//   3. backtracking from W = V through the recorded sinks gives an optimal
//      ordering and, with the argmins of step 1, the parent set of each
//      variable.
// Step 1 is a subset-minimum transform of each child's 2^(m-1) block (one bit
// of the compressed parent mask at a time; a block of bits per pass through a
// shared-memory tile, so HBM is read and written once per pass: 12 bits in
// the first, 7 in each later one, 3 passes at m = 26); step 2 runs one launch per subset size, threads over the subsets of
// that size (unranked in the combinatorial number system), in FP64.
// Ties: the smaller candidate set (the subset) in step 1, the smallest sink in
// step 2, so the result is deterministic.
#include <math.h>

#include "gbn_internal.cuh"

namespace gbn {
namespace {

constexpr int kFirstBits = 12;  // bits of the first (contiguous) pass: 4096-entry tiles
constexpr int kPassBits = 7;    // bits of each later pass: 128 rows x 32 columns
constexpr int kCols = 32;       // consecutive entries per row of a strided tile (128 bytes:
                                // a whole cache line, where 32-byte rows left DRAM at 1/8)
constexpr int kTileThreads = 512;

// One tile in shared memory: R rows (stride `rs` apart in the child block)
// of C consecutive entries; the transform runs over the row bits.
__device__ __forceinline__ void tile_transform(float* v, uint32_t* s, int rbits, int C) {
    const int rows = 1 << rbits;
    for (int b = 0; b < rbits; ++b) {
        const int half = rows >> 1;
        for (int e = threadIdx.x; e < half * C; e += blockDim.x) {
            const int pr = e / C, col = e % C;
            // pair (lo, hi) of rows differing in bit b: lo has it clear
            const int lo = ((pr >> b) << (b + 1)) | (pr & ((1 << b) - 1));
            const int hi = lo | (1 << b);
            const float a = v[lo * C + col], x = v[hi * C + col];
            if (a <= x) {  // the subset wins ties
                v[hi * C + col] = a;
                s[hi * C + col] = s[lo * C + col];
            }
        }
        __syncthreads();
    }
}

// Pass over bits [b0, b0 + rbits) of every child block.  Tile t of a block:
// its column group (bits below b0, kCols entries at a time) and its high bits.
// First pass (b0 = 0): rows of one entry, and the sets start as the slots'
// own compressed masks.
__global__ void __launch_bounds__(kTileThreads)
    bps_pass_kernel(const float* __restrict__ src, float* __restrict__ best,
                    uint32_t* __restrict__ bset, int m, int b0, int rbits, int first) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int C = first ? 1 : kCols;
    const int rows = 1 << rbits;
    float* v = reinterpret_cast<float*>(smem);
    uint32_t* s = reinterpret_cast<uint32_t*>(smem + sizeof(float) * rows * C);
    const int64_t block = (int64_t)1 << (m - 1);
    const int64_t groups_lo = first ? 1 : ((int64_t)1 << b0) / kCols;  // column groups
    const int64_t tiles_per_child = block / ((int64_t)rows * C);
    const int64_t t = blockIdx.x;
    const int64_t child = t / tiles_per_child;
    const int64_t r = t % tiles_per_child;
    const int64_t lo = r % groups_lo, hi = r / groups_lo;
    const int64_t base = child * block + (hi << (b0 + rbits)) + lo * C;
    for (int e = threadIdx.x; e < rows * C; e += blockDim.x) {
        const int row = e / C, col = e % C;
        const int64_t idx = base + ((int64_t)row << b0) + col;
        v[e] = (first ? src : best)[idx];
        s[e] = first ? (uint32_t)(idx - child * block) : bset[idx];
    }
    __syncthreads();
    tile_transform(v, s, rbits, C);
    for (int e = threadIdx.x; e < rows * C; e += blockDim.x) {
        const int row = e / C, col = e % C;
        const int64_t idx = base + ((int64_t)row << b0) + col;
        best[idx] = v[e];
        bset[idx] = s[e];
    }
}

// The same passes with the levels spread over registers, lanes and warps, so
// that most of them need no barrier; the levels still run in ascending bit order
// with the subset winning ties, so every minimum and argmin equals
// tile_transform's.
//
// First pass, 12 bits: a tile is 4096 consecutive entries of a child block;
// thread t holds entries t + 512 k (k < 8): mask bits 0-4 are its lane (levels
// by shuffles), 5-8 its warp (through shared memory, one barrier per level), 9-11
// its register index.
__global__ void __launch_bounds__(kTileThreads)
    bps_first12_kernel(const float* __restrict__ src, float* __restrict__ best,
                       uint32_t* __restrict__ bset, int m) {
    __shared__ float sv[4096];
    __shared__ uint32_t ss[4096];
    const int t = threadIdx.x, lane = t & 31;
    const int64_t block = (int64_t)1 << (m - 1);
    const int64_t tiles_per_child = block >> 12;
    const int64_t child = blockIdx.x / tiles_per_child;
    const int64_t r = blockIdx.x % tiles_per_child;
    const int64_t base = child * block + (r << 12);
    float v[8];
    uint32_t s[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        v[k] = src[base + t + 512 * k];
        s[k] = (uint32_t)((r << 12) + t + 512 * k);  // the compressed mask itself
    }
#pragma unroll
    for (int b = 0; b < 5; ++b) {
        const bool hi = (lane >> b) & 1;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const float a = __shfl_xor_sync(0xffffffffu, v[k], 1 << b);
            const uint32_t sa = __shfl_xor_sync(0xffffffffu, s[k], 1 << b);
            if (hi && a <= v[k]) {
                v[k] = a;
                s[k] = sa;
            }
        }
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        sv[t + 512 * k] = v[k];
        ss[t + 512 * k] = s[k];
    }
    __syncthreads();
#pragma unroll
    for (int b = 5; b < 9; ++b) {  // reads are of entries with bit b clear, writes with it set
        if ((t >> b) & 1) {
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int lo = (t + 512 * k) ^ (1 << b);
                const float a = sv[lo];
                if (a <= v[k]) {
                    v[k] = a;
                    s[k] = ss[lo];
                    sv[t + 512 * k] = a;
                    ss[t + 512 * k] = s[k];
                }
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int b = 0; b < 3; ++b) {
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            if ((k >> b) & 1) {
                const int lo = k ^ (1 << b);
                if (v[lo] <= v[k]) {
                    v[k] = v[lo];
                    s[k] = s[lo];
                }
            }
        }
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        best[base + t + 512 * k] = v[k];
        bset[base + t + 512 * k] = s[k];
    }
}

// A later pass over rbits (4..7) bits from b0: a tile is 2^rbits rows (stride
// 2^b0) of kCols consecutive entries; lane = column, warp w holds rows w + 16 j
// (j < 2^(rbits-4)): row bits 0-3 are the warp (through shared memory), the rest
// registers.
__global__ void __launch_bounds__(kTileThreads)
    bps_strided_kernel(float* __restrict__ best, uint32_t* __restrict__ bset, int m, int b0,
                       int rbits) {
    __shared__ float sv[128 * kCols];
    __shared__ uint32_t ss[128 * kCols];
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const int nr = 1 << (rbits - 4);  // rows per thread
    const int rows = 1 << rbits;
    const int64_t block = (int64_t)1 << (m - 1);
    const int64_t groups_lo = ((int64_t)1 << b0) / kCols;
    const int64_t tiles_per_child = block / ((int64_t)rows * kCols);
    const int64_t child = blockIdx.x / tiles_per_child;
    const int64_t r = blockIdx.x % tiles_per_child;
    const int64_t lo_g = r % groups_lo, hi_g = r / groups_lo;
    const int64_t base = child * block + (hi_g << (b0 + rbits)) + lo_g * kCols + lane;
    float v[8];
    uint32_t s[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        if (j < nr) {
            const int64_t idx = base + ((int64_t)(w + 16 * j) << b0);
            v[j] = best[idx];
            s[j] = bset[idx];
            sv[(w + 16 * j) * kCols + lane] = v[j];
            ss[(w + 16 * j) * kCols + lane] = s[j];
        }
    }
    __syncthreads();
#pragma unroll
    for (int b = 0; b < 4; ++b) {  // reads are of rows with bit b clear, writes with it set
        if ((w >> b) & 1) {
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                if (j < nr) {
                    const int row = w + 16 * j;
                    const int lo = (row ^ (1 << b)) * kCols + lane;
                    const float a = sv[lo];
                    if (a <= v[j]) {
                        v[j] = a;
                        s[j] = ss[lo];
                        sv[row * kCols + lane] = a;
                        ss[row * kCols + lane] = s[j];
                    }
                }
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        if (b < rbits - 4) {
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                if (j < nr && ((j >> b) & 1)) {
                    const int lo = j ^ (1 << b);
                    if (v[lo] <= v[j]) {
                        v[j] = v[lo];
                        s[j] = s[lo];
                    }
                }
            }
        }
    }
    (void)rows;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        if (j < nr) {
            const int64_t idx = base + ((int64_t)(w + 16 * j) << b0);
            best[idx] = v[j];
            bset[idx] = s[j];
        }
    }
}

// The rank-th p-subset of {0..m-1} (combinatorial number system, largest
// element first) as a bitmask; binom[x * 33 + k] = C(x, k).
__device__ __forceinline__ uint32_t unrank(long long rank, int p, int m, const long long* binom) {
    uint32_t w = 0;
    int x = m - 1;
    for (int k = p; k >= 1; --k) {
        while (binom[x * 33 + k] > rank) --x;  // the largest x with C(x, k) <= rank
        rank -= binom[x * 33 + k];
        w |= 1u << x;
        --x;
    }
    return w;
}

__device__ __forceinline__ uint32_t compress_mask(uint32_t U, int c) {
    return (U & ((1u << c) - 1u)) | ((U >> (c + 1)) << c);
}

// Subsets W of size p: F[W] and its sink.
// C(x, k) for x < 32, k <= 32 by Pascal's rule (additions only, exact), once per
// search, into g[x * 33 + k]; one block of 33 threads, thread = k.
__global__ void binom_kernel(long long* __restrict__ g) {
    __shared__ long long row[2][33];
    const int k = threadIdx.x;
    for (int x = 0; x < 32; ++x) {
        const long long* prev = row[(x + 1) & 1];
        const long long v = k == 0 ? 1 : (x == 0 ? 0 : prev[k - 1] + prev[k]);
        row[x & 1][k] = v;
        g[x * 33 + k] = v;
        __syncthreads();
    }
}

__global__ void dp_layer_kernel(const float* __restrict__ best, double* __restrict__ F,
                                uint8_t* __restrict__ sink, int m, int p, long long count,
                                const long long* __restrict__ gbinom) {
    __shared__ long long binom[32 * 33];
    for (int e = threadIdx.x; e < m * 33; e += blockDim.x) binom[e] = gbinom[e];  // C(x, k)
    __syncthreads();
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= count) return;
    const uint32_t W = unrank(r, p, m, binom);
    const int64_t block = (int64_t)1 << (m - 1);
    double fbest = INFINITY;
    int cbest = 0;
    for (uint32_t rest = W; rest; rest &= rest - 1) {
        const int c = __ffs(rest) - 1;
        const uint32_t U = W & ~(1u << c);
        const double val = F[U] + (double)best[(int64_t)c * block + compress_mask(U, c)];
        if (val < fbest) {  // strict: the smallest sink wins ties
            fbest = val;
            cbest = c;
        }
    }
    F[W] = fbest;
    sink[W] = (uint8_t)cbest;
}

__global__ void dp_init_kernel(double* F) { F[0] = 0.0; }

// Backtracking from the full set: one thread, m steps.
__global__ void backtrack_kernel(const double* __restrict__ F, const uint8_t* __restrict__ sink,
                                 const uint32_t* __restrict__ bset, int m,
                                 uint32_t* __restrict__ parents, int32_t* __restrict__ order,
                                 double* __restrict__ total) {
    const int64_t block = (int64_t)1 << (m - 1);
    uint32_t W = (m == 32) ? 0xffffffffu : ((1u << m) - 1u);
    total[0] = F[W];
    for (int step = m - 1; step >= 0; --step) {
        const int c = sink[W];
        const uint32_t U = W & ~(1u << c);
        const uint32_t cs = bset[(int64_t)c * block + compress_mask(U, c)];
        parents[c] = (cs & ((1u << c) - 1u)) | ((cs >> c) << (c + 1));  // expand: re-insert bit c
        if (order) order[step] = c;
        W = U;
    }
}

struct SearchLayout {
    size_t off_best = 0, off_set = 0, off_F = 0, off_sink = 0, off_binom = 0, total = 0;
};

SearchLayout search_layout(int m) {
    auto up = [](size_t x) { return (x + 255) / 256 * 256; };
    const size_t table = (size_t)m << (m - 1);
    SearchLayout L;
    size_t off = 0;
    L.off_best = off;
    off = up(off + sizeof(float) * table);
    L.off_set = off;
    off = up(off + sizeof(uint32_t) * table);
    L.off_F = off;
    off = up(off + sizeof(double) * ((size_t)1 << m));
    L.off_sink = off;
    off = up(off + ((size_t)1 << m));
    L.off_binom = off;
    off = up(off + sizeof(long long) * 32 * 33);
    L.total = off;
    return L;
}

int run_bps(const float* scores, int m, float* best, uint32_t* bset, cudaStream_t stream) {
    const int bits = m - 1;
    const int64_t table = (int64_t)m << (m - 1);
    int b0 = 0;
    bool first = true;
    while (first || b0 < bits) {
        int rb, C;
        if (first) {
            rb = bits < kFirstBits ? bits : kFirstBits;
            C = 1;
        } else {
            rb = bits - b0 < kPassBits ? bits - b0 : kPassBits;
            C = kCols;
        }
        const int64_t tiles = table / ((int64_t)C << rb);
        if (first && rb == kFirstBits) {
            if (launch_plain(bps_first12_kernel, dim3((unsigned)tiles), dim3(kTileThreads), 0,
                             stream, scores, best, bset, m) != cudaSuccess)
                return GBN_ERR_CUDA;
        } else if (!first && rb >= 4) {
            if (launch_plain(bps_strided_kernel, dim3((unsigned)tiles), dim3(kTileThreads), 0,
                             stream, best, bset, m, b0, rb) != cudaSuccess)
                return GBN_ERR_CUDA;
        } else {  // small tables and short last passes
            const size_t smem = (size_t)(8 << rb) * C;
            if (cudaFuncSetAttribute(bps_pass_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem) != cudaSuccess)
                return GBN_ERR_CUDA;
            if (launch_plain(bps_pass_kernel, dim3((unsigned)tiles), dim3(kTileThreads), smem,
                             stream, scores, best, bset, m, b0, rb, first ? 1 : 0) != cudaSuccess)
                return GBN_ERR_CUDA;
        }
        b0 += rb;
        first = false;
    }
    return GBN_OK;
}

}  // namespace
}  // namespace gbn

using namespace gbn;

extern "C" int givensbn_best_parents(const float* scores, int32_t m, float* best,
                                     uint32_t* best_set, const givensbn_opts* opts) {
    if (m < GBN_MIN_M || m > GBN_MAX_M) return GBN_ERR_M;
    if (!scores || !best || !best_set) return GBN_ERR_NULL;
    if (((uintptr_t)scores & 15u) || ((uintptr_t)best & 15u) || ((uintptr_t)best_set & 15u))
        return GBN_ERR_ALIGN;
    return run_bps(scores, m, best, best_set, static_cast<cudaStream_t>(opts ? opts->stream : nullptr));
}

extern "C" int givensbn_structure_search_workspace_size(int32_t m, size_t* bytes) {
    if (!bytes) return GBN_ERR_NULL;
    if (m < GBN_MIN_M || m > GBN_MAX_M) return GBN_ERR_M;
    *bytes = search_layout(m).total;
    return GBN_OK;
}

extern "C" int givensbn_structure_search(const float* scores, int32_t m, uint32_t* parents,
                                         int32_t* order, double* total,
                                         const givensbn_opts* opts) {
    if (!opts) return GBN_ERR_NULL;
    if (m < GBN_MIN_M || m > GBN_MAX_M) return GBN_ERR_M;
    if (!scores || !parents || !total) return GBN_ERR_NULL;
    if (((uintptr_t)scores & 15u) || ((uintptr_t)parents & 3u) || ((uintptr_t)order & 3u) ||
        ((uintptr_t)total & 7u))
        return GBN_ERR_ALIGN;
    const SearchLayout L = search_layout(m);
    if (!opts->workspace || opts->workspace_bytes < L.total) return GBN_ERR_WORKSPACE;
    if ((uintptr_t)opts->workspace & 255u) return GBN_ERR_ALIGN;
    char* ws = static_cast<char*>(opts->workspace);
    cudaStream_t stream = static_cast<cudaStream_t>(opts->stream);
    int rc;
    float* best = reinterpret_cast<float*>(ws + L.off_best);
    uint32_t* bset = reinterpret_cast<uint32_t*>(ws + L.off_set);
    double* F = reinterpret_cast<double*>(ws + L.off_F);
    uint8_t* sink = reinterpret_cast<uint8_t*>(ws + L.off_sink);
    if ((rc = run_bps(scores, m, best, bset, stream))) return rc;
    long long* gbinom = reinterpret_cast<long long*>(ws + L.off_binom);
    if (launch_plain(dp_init_kernel, dim3(1), dim3(1), 0, stream, F) != cudaSuccess ||
        launch_plain(binom_kernel, dim3(1), dim3(33), 0, stream, gbinom) != cudaSuccess)
        return GBN_ERR_CUDA;
    long long cnt = 1;  // C(m, p)
    for (int p = 1; p <= m; ++p) {
        cnt = cnt * (m - p + 1) / p;
        const unsigned blocks = (unsigned)((cnt + 255) / 256);
        if (launch_plain(dp_layer_kernel, dim3(blocks), dim3(256), 0, stream,
                         (const float*)best, F, sink, (int)m, p, cnt,
                         (const long long*)gbinom) != cudaSuccess)
            return GBN_ERR_CUDA;
    }
    return launch_rc(launch_plain(backtrack_kernel, dim3(1), dim3(1), 0, stream, (const double*)F,
                                  (const uint8_t*)sink, (const uint32_t*)bset, (int)m, parents,
                                  order, total));
}

// The Givens walk (Sec. 1.3, Sec. 2, Algorithm 1) over the sub-walks of one CTA.
//
// Each CTA owns 2^W sub-walks that share their front variables above the
// lowest W fixed variables and differ in those W (lane l of a warp <-> the
// sub-walk whose front set contains fixed variable b iff bit b of l is set).
// Every sub-walk runs the same local swap sequence Upsilon(Q), so the sequence
// is a compile-time table and the whole walk is unrolled with static register
// indices: no lane ever diverges.
//
// Warp 0 ("L warp") holds, per lane, the Q x Q block of R over the free
// variables with registers named by column POSITION, so a column transposition
// is a renaming done by the compiler.  Per swap at index i it computes the
// rotation (c, s) from the two entries of the column at position i+1 (the
// GRC_i rotation of Sec. 1.3, with s = r_{i+1,i+1}/rho), rotates rows i, i+1,
// updates one tail sum per column, writes (c, s) to the shared-memory tape and
// emits the scores of the free variables behind the new prefix.
//
// All warps then replay the tape over the fixed variables outside the front
// set ("B columns"): each such column is a Q-vector in the free block's basis
// plus the residual below it, rotated by the same (c, s) sequence; it is a
// child of every prefix of the walk.
//
// Tail sums: for a column with entries z in the free rows and residual C
// below them, w[r] = sum_{t>=r} z_t^2 + C is the RSS of that column on the
// variables in positions < r.  A swap at i leaves every w[r] with r <= i
// unchanged (rotations preserve the norm of rows i, i+1) and only w[i+1]
// changes: w[i+1] = w[i+2] + z_{i+1}^2.  The families a swap adds are exactly
// those whose parent set is the new prefix of length i (Sec. 4).
//
// Scores: score = n ln(RSS/n) + |S| ln n = (n ln 2) log2(RSS) + (|S| ln n - n ln n),
// written to idx(c,S) = c 2^(m-1) + compress(S, c).  With the free variables
// the highest-numbered ones and the lanes differing in the lowest fixed
// variables, the 32 lanes of a warp write 32 consecutive table slots per
// emission (one 128-byte line) for every child outside those W variables.
#pragma once

#include <utility>

#include "gbn_internal.cuh"

namespace gbn {

template <typename T>
struct Vec2T;
template <>
struct Vec2T<float> {
    using type = float2;
};
template <>
struct Vec2T<double> {
    using type = double2;
};

template <typename T>
struct WalkArgs {
    void* out;
    const T* leaves;
    size_t leaf_stride;
    int m, k, W, lanes;
    T alpha;  // n ln 2
    T lnn;    // ln n
    T nlnn;   // n ln n
    unsigned long long* chk;  // check record (checked builds)
    size_t out_size;          // table elements
};

__device__ __forceinline__ float wk_rsqrt(float x) { return rsqrtf(x); }
__device__ __forceinline__ double wk_rsqrt(double x) { return rsqrt(x); }
__device__ __forceinline__ float wk_log2(float x) { return __log2f(x); }
__device__ __forceinline__ double wk_log2(double x) { return log2(x); }
__device__ __forceinline__ float2 wk_pair(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ double2 wk_pair(double a, double b) { return make_double2(a, b); }

constexpr unsigned compress_bit(unsigned mask, int j) {
    return (mask & ((1u << j) - 1u)) | ((mask >> (j + 1)) << j);
}

template <size_t... Ts, class F>
__device__ __forceinline__ void for_steps(std::index_sequence<Ts...>, F&& f) {
    (f(std::integral_constant<int, (int)Ts>{}), ...);
}

template <typename T, bool COV>
__device__ __forceinline__ void emit(const WalkArgs<T>& a, size_t idx, T rss, T pen) {
    if (!GBN_IN(a.chk, 301, idx, a.out_size)) return;
    void* out = a.out;
    const T alpha = a.alpha;
    if constexpr (COV) {
        atomicAdd(reinterpret_cast<unsigned*>(out) + idx, 1u);
    } else {
        reinterpret_cast<T*>(out)[idx] = fma(alpha, wk_log2(rss), pen);
    }
}

// ---------------------------------------------------------------------------
// L warp: one sub-walk per lane over its free block.
template <typename T, int Q, bool COV>
__device__ __forceinline__ void l_walk(const WalkArgs<T>& a, const T* __restrict__ rec,
                                       typename Vec2T<T>::type* tape, int lane, uint64_t F) {
    constexpr int N = WalkSeq<Q>::N;
    // Register arrays, flat and indexed only by compile-time constants:
    // R[row * Q + position] (rows <= position) and
    // Wt[r * Q + p] = sum_{t=r..p} R[(t) * Q + (p)]^2.
    T R[Q * Q];
    T Wt[(Q + 1) * Q];
#pragma unroll
    for (int pc = 0; pc < Q; ++pc)
#pragma unroll
        for (int r = 0; r <= pc; ++r)
            R[(r) * Q + (pc)] = GBN_IN(a.chk, 302, (size_t)(pc * (pc + 1) / 2 + r) * 32 + lane, a.leaf_stride)
                           ? rec[(size_t)(pc * (pc + 1) / 2 + r) * 32 + lane]
                           : T(0);
#pragma unroll
    for (int pc = 0; pc < Q; ++pc) {
        T acc = T(0);
#pragma unroll
        for (int r = pc; r >= 0; --r) {
            acc = fma(R[(r) * Q + (pc)], R[(r) * Q + (pc)], acc);
            Wt[(r) * Q + (pc)] = acc;
        }
    }
    const int dF = __popcll(F);
    T pen[Q + 1];
#pragma unroll
    for (int s = 0; s <= Q; ++s) pen[s] = fma(T(dF + s), a.lnn, -a.nlnn);
    const size_t cstride = (size_t)1 << (a.m - 1);
    const size_t base = ((size_t)a.k << (a.m - 1)) + F;
    const int ksh = a.k;
    // families of the root: parents = first s free variables (initial order)
#pragma unroll
    for (int s = 0; s < Q; ++s)
#pragma unroll
        for (int pc = s; pc < Q; ++pc)
            emit<T, COV>(a, base + (size_t)pc * cstride + ((size_t)((1u << s) - 1u) << ksh),
                         Wt[(s) * Q + (pc)], pen[s]);
    for_steps(std::make_index_sequence<N>{}, [&](auto tc) {
        constexpr int t = decltype(tc)::value;
        constexpr int i = kWalkSeq<Q>.idx[t] - 1;  // rows i, i+1 (0-based)
        const T x0 = R[(i) * Q + (i + 1)], y0 = R[(i + 1) * Q + (i + 1)];
        const T rho2 = fma(x0, x0, y0 * y0);
        const T inv = wk_rsqrt(rho2);
        const bool ok = rho2 > T(0);
        const T c = ok ? x0 * inv : T(1);
        const T s = ok ? y0 * inv : T(0);
        const T rho = ok ? rho2 * inv : T(0);
        const T rii = R[(i) * Q + (i)];
        // transpose positions i, i+1 (renaming of the rows above i)
#pragma unroll
        for (int r = 0; r < i; ++r) {
            const T tmp = R[(r) * Q + (i)];
            R[(r) * Q + (i)] = R[(r) * Q + (i + 1)];
            R[(r) * Q + (i + 1)] = tmp;
        }
#pragma unroll
        for (int r = 0; r <= i; ++r) {
            const T tmp = Wt[(r) * Q + (i)];
            Wt[(r) * Q + (i)] = Wt[(r) * Q + (i + 1)];
            Wt[(r) * Q + (i + 1)] = tmp;
        }
        R[(i) * Q + (i)] = rho;
        R[(i) * Q + (i + 1)] = c * rii;
        R[(i + 1) * Q + (i + 1)] = -s * rii;
        Wt[(i + 1) * Q + (i + 1)] = R[(i + 1) * Q + (i + 1)] * R[(i + 1) * Q + (i + 1)];
#pragma unroll
        for (int pc = i + 2; pc < Q; ++pc) {
            const T x = R[(i) * Q + (pc)], y = R[(i + 1) * Q + (pc)];
            R[(i) * Q + (pc)] = fma(c, x, s * y);
            R[(i + 1) * Q + (pc)] = fma(c, y, -s * x);
            Wt[(i + 1) * Q + (pc)] = fma(R[(i + 1) * Q + (pc)], R[(i + 1) * Q + (pc)], Wt[(i + 2) * Q + (pc)]);
        }
        if (GBN_IN(a.chk, 303, t * 32 + lane, N * 32)) tape[t * 32 + lane] = wk_pair(c, s);
        constexpr unsigned pre = kWalkSeq<Q>.prefix[t];
        for_steps(std::make_index_sequence<Q>{}, [&](auto pcc) {
            constexpr int pc = decltype(pcc)::value;
            if constexpr (pc > i) {
                constexpr int j = kWalkSeq<Q>.var_at[t][pc];
                constexpr unsigned cT = compress_bit(pre, j);
                emit<T, COV>(a, base + (size_t)j * cstride + ((size_t)cT << ksh),
                             Wt[(i + 1) * Q + (pc)], pen[i + 1]);
            }
        });
    });
}

// ---------------------------------------------------------------------------
// One fixed variable v outside the front set of sub-walk ell, replayed from the tape.
template <typename T, int Q, bool COV>
__device__ __forceinline__ void b_walk(const WalkArgs<T>& a, const T* __restrict__ rec,
                                       const typename Vec2T<T>::type* tape, int v, int ell,
                                       uint64_t F) {
    constexpr int N = WalkSeq<Q>::N;
    constexpr int LQ = Q * (Q + 1) / 2;
    const T* bv = rec + (size_t)32 * (LQ + v * (Q + 1));
    T z[Q];
    T w[Q + 1];
#pragma unroll
    for (int e = 0; e < Q; ++e)
        z[e] = GBN_IN(a.chk, 304, (size_t)32 * (LQ + v * (Q + 1)) + e * 32 + ell, a.leaf_stride)
                   ? bv[(size_t)e * 32 + ell]
                   : T(0);
    w[Q] = GBN_IN(a.chk, 305, (size_t)32 * (LQ + v * (Q + 1)) + Q * 32 + ell, a.leaf_stride)
               ? bv[(size_t)Q * 32 + ell]
               : T(0);
#pragma unroll
    for (int r = Q - 1; r >= 0; --r) w[r] = fma(z[r], z[r], w[r + 1]);
    const int dF = __popcll(F);
    T pen[Q + 1];
#pragma unroll
    for (int s = 0; s <= Q; ++s) pen[s] = fma(T(dF + s), a.lnn, -a.nlnn);
    const uint64_t lowmask = (1ull << v) - 1ull;
    const size_t base =
        ((size_t)v << (a.m - 1)) + (size_t)((F & lowmask) | ((F >> (v + 1)) << v));
    const int ksh = a.k - 1;
#pragma unroll
    for (int s = 0; s <= Q; ++s)
        emit<T, COV>(a, base + ((size_t)((1u << s) - 1u) << ksh), w[s], pen[s]);
    for_steps(std::make_index_sequence<N>{}, [&](auto tc) {
        constexpr int t = decltype(tc)::value;
        constexpr int i = kWalkSeq<Q>.idx[t] - 1;
        typename Vec2T<T>::type cs{};
        if (GBN_IN(a.chk, 306, t * 32 + ell, N * 32)) cs = tape[t * 32 + ell];
        const T x = z[i], y = z[i + 1];
        z[i] = fma(cs.x, x, cs.y * y);
        z[i + 1] = fma(cs.x, y, -cs.y * x);
        w[i + 1] = fma(z[i + 1], z[i + 1], w[i + 2]);
        constexpr unsigned pre = kWalkSeq<Q>.prefix[t];
        emit<T, COV>(a, base + ((size_t)pre << ksh), w[i + 1], pen[i + 1]);
    });
}

__device__ __forceinline__ int nth_zero_bit(uint64_t x, int nth) {
    for (int b = 0;; ++b) {
        if (!((x >> b) & 1ull)) {
            if (nth == 0) return b;
            --nth;
        }
    }
}

template <typename T, int Q, bool COV>
__global__ void __launch_bounds__(128) walk_kernel(WalkArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    using T2 = typename Vec2T<T>::type;
    T2* tape = reinterpret_cast<T2*>(smem_raw);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const uint64_t cta = blockIdx.x;
    const uint64_t Fhi = cta << a.W;
    const T* rec = a.leaves + (size_t)blockIdx.x * a.leaf_stride;
    if (warp == 0 && lane < a.lanes) l_walk<T, Q, COV>(a, rec, tape, lane, Fhi | (uint64_t)lane);
    __syncthreads();
    const int nhi = a.k - a.W;
    const int nu = nhi - __popcll(cta);
    const int g = a.W >= 1 ? (a.lanes >> 1) : 1;
    const int vpi = 32 / g;
    const int n5 = a.W >= 1 ? (a.W + vpi - 1) / vpi : 0;
    const int nitems = nu + n5;
    for (int it = warp; it < nitems; it += nwarps) {
        int v, ell;
        bool active;
        if (it < nu) {
            v = a.W + nth_zero_bit(cta, it);
            ell = lane;
            active = lane < a.lanes;
        } else {
            const int j = it - nu;
            const int u = lane / g, sub = lane % g;
            v = j * vpi + u;
            active = v < a.W;
            ell = (sub & ((1 << v) - 1)) | ((sub >> v) << (v + 1));
        }
        if (active) b_walk<T, Q, COV>(a, rec, tape, v, ell, Fhi | (uint64_t)ell);
    }
}

template <typename T, int Q, bool COV>
int launch_walk_q(const WalkArgs<T>& a, int64_t n_cta, cudaStream_t stream) {
    constexpr int N = WalkSeq<Q>::N;
    const size_t smem = (size_t)(N > 0 ? N : 1) * 32 * sizeof(typename Vec2T<T>::type);
    if (cudaFuncSetAttribute(walk_kernel<T, Q, COV>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess)
        return GBN_ERR_CUDA;
    walk_kernel<T, Q, COV><<<(unsigned)n_cta, 128, smem, stream>>>(a);
    return cudaGetLastError() == cudaSuccess ? GBN_OK : GBN_ERR_CUDA;
}

}  // namespace gbn

// One instantiation per (scalar type, Q, coverage); each is compiled as its
// own object from walk_inst.cu so that the build runs in parallel.
#define GBN_WALK_INST_NAME(T, Q, COV) gbn_launch_walk_##T##_q##Q##_c##COV
#define GBN_WALK_DECL(T, Q, COV) \
    int GBN_WALK_INST_NAME(T, Q, COV)(const gbn::WalkArgs<T>& a, int64_t n_cta, cudaStream_t s)

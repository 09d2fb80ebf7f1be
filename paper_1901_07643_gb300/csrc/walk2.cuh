// The Givens walk (Sec. 1.3, Sec. 2, Algorithm 1) over the sub-walks of one CTA,
// compact form: a runtime loop over the swap sequence, so the code size does
// not grow with the 2^Q - Q - 1 steps of Upsilon(Q).
//
// Each CTA owns 2^W sub-walks that share their front variables above the
// lowest W fixed variables and differ in those W (lane l of a warp <-> the
// sub-walk whose front set holds fixed variable b iff bit b of l is set).  All
// sub-walks run the same local sequence Upsilon(Q), so the swap row i of step
// t and the prefix set after it are per-step constants shared by every lane;
// they come from a table in constant memory built at compile time.
//
// Warp 0 (producer) holds, per lane, the Q x Q block of R over the free
// variables in shared memory, one private column per variable.  Per step it
// forms the rotation of the GRC operator from rows i, i+1 of the column at
// position i+1 (cos = r_{i,i+1}/rho, sin = r_{i+1,i+1}/rho: the paper prints
// the same numerator twice; this is the rotation that zeroes the
// sub-diagonal), rotates rows i, i+1 of the columns behind it, updates one
// tail sum per column and emits the scores of the free variables behind the
// new prefix.  It writes (cos, sin) to a ring of tape chunks in shared memory.
//
// Warps 1.. (consumers) each carry up to NI fixed variables outside the front
// set ("B columns") in registers: a Q-vector in the free block's basis plus
// the residual C below it.  They replay the tape chunk by chunk and, per
// step, rotate rows i, i+1 of each vector, update its tail sum and emit its
// score; a B column is a child of every prefix.
//
// Tail sums: w[r] = sum_{t>=r} z_t^2 + C is the RSS of the column on the
// variables in positions < r.  A swap at i leaves every w[r] with r <= i
// unchanged (rotations keep the norm of rows i, i+1) and only w[i+1] changes:
// w[i+1] = w[i+2] + z_{i+1}^2.  The families a swap adds are exactly those
// whose parent set is the new prefix of length i+1 (Sec. 4).
//
// Producer and consumers synchronise through mbarriers, one "full" and one
// "empty" barrier per ring slot.  Every wait is bounded by a wall-clock
// watchdog: when it expires the warp records GBN_STATUS_WATCHDOG in the status
// word and returns, so a broken schedule ends the kernel instead of hanging.
//
// Scores: score = n ln(RSS/n) + |S| ln n = (n ln 2) log2(RSS) + (|S| ln n - n ln n),
// stored at idx(c,S) = c 2^(m-1) + compress(S, c).  The lanes of a warp write
// consecutive table slots (the lowest W parent bits vary across lanes).
#pragma once

#include <type_traits>
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
    unsigned long long* timing;  // role cycle counters (timing builds)
    int* status;              // status word (watchdog bit)
    size_t out_size;          // table elements
    int n_bwarps;             // consumer warps per CTA
    int ni;                   // fixed-variable slots per consumer thread
    long long watchdog_ns;    // bound on every wait
};

constexpr int kChunk = 32;  // steps per tape chunk
constexpr int kRing = 4;    // tape chunks in flight

// Per-step table: bits 0..3 = swap row i (0-based; the paper's GRC_{i+1}),
// bits 4.. = mask of the local free variables at positions 0..i after the swap.
template <int Q>
struct StepTab {
    static constexpr int N = (1 << Q) - Q - 1;  // |Upsilon(Q)|, Sec. 3
    uint32_t e[N > 0 ? N : 1];
};

template <int Q>
constexpr StepTab<Q> make_step_tab() {
    StepTab<Q> tab{};
    int buf[(1 << Q) + 1] = {};
    int len = 0;
    if (Q >= 2) {
        buf[0] = 1;  // Upsilon(2) = [1]
        len = 1;
    }
    // Upsilon(j+1) = Upsilon(j) : [j .. 1] : (Upsilon(j) + 1)   (Sec. 3, Sec. 5)
    for (int j = 2; j < Q; ++j) {
        const int old = len;
        for (int i = j; i >= 1; --i) buf[len++] = i;
        for (int t = 0; t < old; ++t) buf[len++] = buf[t] + 1;
    }
    int pos[Q > 0 ? Q : 1] = {};
    for (int p = 0; p < Q; ++p) pos[p] = p;
    for (int t = 0; t < len; ++t) {
        const int i = buf[t];
        const int tmp = pos[i - 1];
        pos[i - 1] = pos[i];
        pos[i] = tmp;
        uint32_t mask = 0;
        for (int p = 0; p < i; ++p) mask |= 1u << pos[p];
        tab.e[t] = (uint32_t)(i - 1) | (mask << 4);
    }
    return tab;
}

__device__ __forceinline__ float wk_rsqrt(float x) { return rsqrtf(x); }
__device__ __forceinline__ double wk_rsqrt(double x) { return rsqrt(x); }
__device__ __forceinline__ float wk_log2(float x) { return __log2f(x); }
__device__ __forceinline__ double wk_log2(double x) { return log2(x); }
__device__ __forceinline__ float2 wk_pair(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ double2 wk_pair(double a, double b) { return make_double2(a, b); }

__device__ __forceinline__ unsigned compress_bit_rt(unsigned mask, int j) {
    return (mask & ((1u << j) - 1u)) | ((mask >> (j + 1)) << j);
}


// Element type of the output table: scores, or 32-bit counters in coverage mode.
template <typename T, bool COV>
using OutT = typename std::conditional<COV, unsigned, T>::type;

// Store at p + off (p: a per-thread pointer into the table, off < 2^32) when
// `on`.  The score is computed unconditionally and only the store is
// predicated, so no per-lane branch is taken around the arithmetic.
template <typename T, bool COV>
__device__ __forceinline__ void emit_ptr(const WalkArgs<T>& a, OutT<T, COV>* p, uint32_t off,
                                         T rss, T pen, bool on = true) {
    if constexpr (COV) {
        if (on && GBN_IN(a.chk, 302,
                         (size_t)(p - reinterpret_cast<OutT<T, COV>*>(a.out)) + off, a.out_size))
            atomicAdd(p + off, 1u);
    } else {
        const T v = fma(a.alpha, wk_log2(rss), pen);
        if (on && GBN_IN(a.chk, 302,
                         (size_t)(p - reinterpret_cast<OutT<T, COV>*>(a.out)) + off, a.out_size))
            p[off] = v;
    }
}

// ---------------------------------------------------------------- mbarriers
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile(
        "{\n\t.reg .b64 st;\n\tmbarrier.arrive.release.cta.shared::cta.b64 st, [%0];\n\t}" ::"r"(
            smem_addr(bar))
        : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ long long global_ns() {
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Bounded wait for the phase with the given parity; false = watchdog expired.
// try_wait suspends the thread for a short hardware-defined time when the
// phase is not complete; the clock is read only every 64 polls.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, long long limit_ns,
                                          int* status) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = global_ns();
    for (unsigned n = 1;; ++n) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((n & 63u) == 0) {
            if (global_ns() - t0 > limit_ns) {
                atomicOr(status, GBN_STATUS_WATCHDOG);
                return false;
            }
            __nanosleep(128);
        }
    }
}

// Timing builds (-DGBN_TIMING) add the cycles each role spends waiting on the
// tape barriers and in total to counters in the workspace status block:
// [0] producer total, [1] producer waiting, [2] consumer total, [3] consumer
// waiting (summed over warps, lane 0 only).  Ordinary builds compile them away.
#ifdef GBN_TIMING
#define GBN_TIMER_DECL long long gbn_t_wait = 0, gbn_t_start = clock64();
#define GBN_TIMED_WAIT(expr)                      \
    ({                                            \
        const long long gbn_t0 = clock64();       \
        const bool gbn_ok = (expr);               \
        gbn_t_wait += clock64() - gbn_t0;         \
        gbn_ok;                                   \
    })
#define GBN_TIMER_FLUSH(ctr, slot)                                                       \
    if ((threadIdx.x & 31) == 0) {                                                       \
        atomicAdd((unsigned long long*)(ctr) + 2 * (slot), (unsigned long long)(clock64() - gbn_t_start)); \
        atomicAdd((unsigned long long*)(ctr) + 2 * (slot) + 1, (unsigned long long)gbn_t_wait); \
    }
#else
#define GBN_TIMER_DECL
#define GBN_TIMED_WAIT(expr) (expr)
#define GBN_TIMER_FLUSH(ctr, slot)
#endif

// Warp-uniform form: lane 0 polls, every lane gets the same answer, and the
// __syncwarp orders lane 0's acquire before the other lanes' later reads.
__device__ __forceinline__ bool warp_wait(uint64_t* bar, unsigned parity, long long limit_ns,
                                          int* status) {
    int ok = 1;
    if ((threadIdx.x & 31) == 0) ok = mbar_wait(bar, parity, limit_ns, status) ? 1 : 0;
    ok = __shfl_sync(0xffffffffu, ok, 0);
    __syncwarp();
    return ok != 0;
}

__device__ __forceinline__ int nth_zero_bit(uint64_t x, int nth) {
    for (int b = 0; b < 64; ++b) {
        if (!((x >> b) & 1ull)) {
            if (nth == 0) return b;
            --nth;
        }
    }
    return 63;
}

// Shared-memory layout of one CTA: the tape ring, the producer's tail sums
// (named by variable, lane-private) and the barriers.
template <typename T, int Q>
struct Smem {
    static constexpr size_t tape_elems = (size_t)kRing * kChunk * 32;  // (cos, sin) pairs
    static constexpr size_t w_elems = (size_t)Q * Q * 32;             // [(row*Q + var)*32 + lane]
    static constexpr size_t off_tape = 0;
    static constexpr size_t off_w = tape_elems * 2 * sizeof(T);
    static constexpr size_t off_bar = (off_w + w_elems * sizeof(T) + 15) / 16 * 16;
    static constexpr size_t bytes = off_bar + 2 * kRing * sizeof(uint64_t);
};

template <int... Is, class F>
__device__ __forceinline__ void static_for(std::integer_sequence<int, Is...>, F&& f) {
    (f(std::integral_constant<int, Is>{}), ...);
}

// One swap of the producer at compile-time row I.  R is named by position:
// R[r * Q + p] (r <= p) is row r of the column at position p, and vp[p] is
// the free variable there.  Tail sums live in shared memory named by
// variable, Ws[(r * Q + var) * 32] (lane offset already applied), so a
// transposition moves none of them.  Emits the scores of the free variables
// behind the new prefix.
template <typename T, int Q, int I, bool COV>
__device__ __forceinline__ void produce_step(T (&R)[Q * Q], int (&vp)[Q], T* Ws, T& c_out,
                                             T& s_out, const WalkArgs<T>& a, unsigned pre,
                                             OutT<T, COV>* lane_out, size_t cstride, T pen,
                                             bool active) {
    T wnext[Q];
#pragma unroll
    for (int p = I + 2; p < Q; ++p) wnext[p] = Ws[((I + 2) * Q + vp[p]) * 32];
    const T x0 = R[I * Q + I + 1], y0 = R[(I + 1) * Q + I + 1];
    const T rho2 = fma(x0, x0, y0 * y0);
    const T inv = wk_rsqrt(rho2);
    const bool ok = rho2 > T(0);
    const T c = ok ? x0 * inv : T(1);
    const T s = ok ? y0 * inv : T(0);
    const T rii = R[I * Q + I];
#pragma unroll
    for (int r = 0; r < I; ++r) {
        const T tr = R[r * Q + I];
        R[r * Q + I] = R[r * Q + I + 1];
        R[r * Q + I + 1] = tr;
    }
    const int u = vp[I];
    vp[I] = vp[I + 1];
    vp[I + 1] = u;
    R[I * Q + I] = ok ? rho2 * inv : T(0);
    const T yu = -s * rii;
    R[I * Q + I + 1] = c * rii;
    R[(I + 1) * Q + I + 1] = yu;
    const T wu = yu * yu;
    Ws[((I + 1) * Q + u) * 32] = wu;
    const int ksh = a.k;
    const unsigned pre1 = pre >> 1;
    {  // block of child u: lane_out + u 2^(m-1); offset within it < 2^(m-1)
        const unsigned lm = (1u << u) - 1u;
        emit_ptr<T, COV>(a, lane_out + (size_t)u * cstride, ((pre & lm) | (pre1 & ~lm)) << ksh,
                         wu, pen, active);
    }
#pragma unroll
    for (int p = I + 2; p < Q; ++p) {
        const T x = R[I * Q + p], y = R[(I + 1) * Q + p];
        R[I * Q + p] = fma(c, x, s * y);
        const T yn = fma(c, y, -s * x);
        R[(I + 1) * Q + p] = yn;
        const T ww = fma(yn, yn, wnext[p]);
        const int j = vp[p];
        Ws[((I + 1) * Q + j) * 32] = ww;
        {
            const unsigned lm = (1u << j) - 1u;
            emit_ptr<T, COV>(a, lane_out + (size_t)j * cstride,
                             ((pre & lm) | (pre1 & ~lm)) << ksh, ww, pen, active);
        }
    }
    c_out = c;
    s_out = s;
}

// ---------------------------------------------------------------------------
// Producer: one sub-walk per lane over its free block; publishes the
// (cos, sin) of every step and emits the free variables' scores.
template <typename T, int Q, bool COV>
__device__ __forceinline__ void produce(const WalkArgs<T>& a, const StepTab<Q>& tab,
                                        const T* __restrict__ rec, unsigned char* smem, int lane,
                                        uint64_t F, bool active, bool has_consumers) {
    using S = Smem<T, Q>;
    using T2 = typename Vec2T<T>::type;
    constexpr int N = StepTab<Q>::N;
    T2* tape = reinterpret_cast<T2*>(smem + S::off_tape);
    T* Ws = reinterpret_cast<T*>(smem + S::off_w) + lane;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + S::off_bar);
    uint64_t* empty = full + kRing;
    T R[Q * Q];
    int vp[Q];
    static_for(std::make_integer_sequence<int, Q>{}, [&](auto pc) {
        constexpr int p = decltype(pc)::value;
        vp[p] = p;
        T acc = T(0);
        static_for(std::make_integer_sequence<int, p + 1>{}, [&](auto rc) {
            constexpr int r = p - decltype(rc)::value;  // r = p .. 0
            const size_t e = (size_t)(p * (p + 1) / 2 + r) * 32 + lane;
            const T v = (active && GBN_IN(a.chk, 311, e, a.leaf_stride)) ? rec[e] : T(0);
            R[r * Q + p] = v;
            acc = fma(v, v, acc);
            Ws[(r * Q + p) * 32] = acc;
        });
    });
    const T pen0 = fma(T(__popcll(F)), a.lnn, -a.nlnn);
    const size_t cstride = (size_t)1 << (a.m - 1);
    OutT<T, COV>* lane_out =
        reinterpret_cast<OutT<T, COV>*>(a.out) + (((size_t)a.k << (a.m - 1)) + F);
    if (active) {  // families of the root: parents = first s free variables
        for (int s = 0; s < Q; ++s) {
            const T pen = fma(T(s), a.lnn, pen0);
            for (int p = s; p < Q; ++p)
                emit_ptr<T, COV>(a, lane_out + (size_t)p * cstride, ((1u << s) - 1u) << a.k,
                                 Ws[(s * Q + p) * 32], pen);
        }
    }
    // The swap rows of Upsilon(Q) start at 0 and move by exactly one per step
    // (Algorithm 1: each concatenation joins rows that differ by one), so the
    // walk is a state machine over rows: every row has its own straight-line
    // block that ends in a direct branch to the row above or below.
    static_assert(N >= 1, "Upsilon(Q) has at least one swap for Q >= 2");
    GBN_TIMER_DECL
    int t = 0;
    T c = T(1), s = T(0);
#define GBN_PSTEP(r, UP, DOWN)                                                         \
    if (r < Q - 1) {                                                                   \
        produce_step<T, Q, (r < Q - 1 ? r : 0), COV>(R, vp, Ws, c, s, a, tab.e[t] >> 4,  \
                                                     lane_out, cstride,                \
                                                     fma(T(r + 1), a.lnn, pen0), active); \
        tape[((t / kChunk) % kRing * kChunk + t % kChunk) * 32 + lane] = wk_pair(c, s); \
        if (++t == N) goto p_done;                                                     \
        if (t % kChunk == 0) {                                                         \
            __syncwarp();                                                              \
            if (lane == 0) mbar_arrive(&full[(t / kChunk - 1) % kRing]);               \
            const int use = (t / kChunk) / kRing;                                      \
            if (use > 0 && has_consumers &&                                            \
                !GBN_TIMED_WAIT(warp_wait(&empty[(t / kChunk) % kRing], (use - 1) & 1, \
                                          a.watchdog_ns, a.status)))                   \
                return;                                                                \
        }                                                                              \
        if ((int)(tab.e[t] & 15u) > r) goto UP;                                        \
        goto DOWN;                                                                     \
    }
p_r0: GBN_PSTEP(0, p_r1, p_r0)
p_r1: GBN_PSTEP(1, p_r2, p_r0)
p_r2: GBN_PSTEP(2, p_r3, p_r1)
p_r3: GBN_PSTEP(3, p_r4, p_r2)
p_r4: GBN_PSTEP(4, p_r5, p_r3)
p_r5: GBN_PSTEP(5, p_r6, p_r4)
p_r6: GBN_PSTEP(6, p_r7, p_r5)
p_r7: GBN_PSTEP(7, p_r8, p_r6)
p_r8: GBN_PSTEP(8, p_r9, p_r7)
p_r9: GBN_PSTEP(9, p_r10, p_r8)
p_r10: GBN_PSTEP(10, p_r10, p_r9)
#undef GBN_PSTEP
p_done:
    __syncwarp();
    if (lane == 0) mbar_arrive(&full[((N - 1) / kChunk) % kRing]);
    GBN_TIMER_FLUSH(a.timing, 0)
}

// Fixed-variable items of a CTA: the variables above the lowest W outside
// F_hi (each covers all lanes), then the lowest W variables packed 32/g per
// item, g = 2^(W-1) lanes each (only sub-walks without that variable in F).
__device__ __forceinline__ int count_b_items(int k, int W, int lanes, uint64_t cta) {
    const int nu = (k - W) - __popcll(cta);
    const int g = W >= 1 ? (lanes >> 1) : 1;
    const int n5 = W >= 1 ? (W + (32 / g) - 1) / (32 / g) : 0;
    return nu + n5;
}

// ---------------------------------------------------------------------------
// Consumers: NI fixed variables outside the front set per thread, replayed
// from the tape.  A column is a Q-vector z in the free block's basis plus the
// residual C below it, with tail sums w; every step rotates rows i, i+1 and
// updates w[i+1].  It is a child of every prefix: its score goes to
// v 2^(m-1) + compress(F, v) + (T << (k-1)).
// SHARED: every slot belongs to the lane's own sub-walk (one tape load per
// step); otherwise each slot has its own sub-walk ell (the lowest W variables).
template <typename T, int Q, bool COV, int NI, bool SHARED>
__device__ __forceinline__ void consume(const WalkArgs<T>& a, const StepTab<Q>& tab,
                                        const T* __restrict__ rec, unsigned char* smem, int lane,
                                        int first_item, uint64_t cta, uint64_t Fhi) {
    using S = Smem<T, Q>;
    using T2 = typename Vec2T<T>::type;
    constexpr int N = StepTab<Q>::N;
    constexpr int LQ = Q * (Q + 1) / 2;
    const T2* tape = reinterpret_cast<const T2*>(smem + S::off_tape);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + S::off_bar);
    uint64_t* empty = full + kRing;
    const int nu = (a.k - a.W) - __popcll(cta);
    const int g = a.W >= 1 ? (a.lanes >> 1) : 1;
    const int vpi = 32 / g;
    const int n5 = a.W >= 1 ? (a.W + vpi - 1) / vpi : 0;
    T z[NI][Q];
    T w[NI][Q + 1];
    T penb[NI];
    OutT<T, COV>* dst[NI];
    int ell[NI];
    bool act[NI];
#pragma unroll
    for (int k = 0; k < NI; ++k) {
        const int it = first_item + k;
        int v = 0, el = lane;
        bool on = false;
        if constexpr (SHARED) {
            if (it < nu) {
                v = a.W + nth_zero_bit(cta, it);
                on = lane < a.lanes;
            }
        } else if (it < n5) {
            const int uu = lane / g, sub = lane % g;
            v = it * vpi + uu;
            on = v < a.W;
            el = on ? ((sub & ((1 << v) - 1)) | ((sub >> v) << (v + 1))) : 0;
        }
        act[k] = on;
        ell[k] = el;
        const uint64_t F = Fhi | (uint64_t)el;
        penb[k] = fma(T(__popcll(F)), a.lnn, -a.nlnn);
        const T* bv = rec + (size_t)32 * (LQ + v * (Q + 1));
#pragma unroll
        for (int e = 0; e < Q; ++e) {
            const size_t ix = (size_t)32 * (LQ + v * (Q + 1)) + e * 32 + el;
            z[k][e] = (on && GBN_IN(a.chk, 321, ix, a.leaf_stride)) ? bv[(size_t)e * 32 + el] : T(0);
        }
        const size_t ix = (size_t)32 * (LQ + v * (Q + 1)) + Q * 32 + el;
        w[k][Q] = (on && GBN_IN(a.chk, 322, ix, a.leaf_stride)) ? bv[(size_t)Q * 32 + el] : T(0);
#pragma unroll
        for (int r = Q - 1; r >= 0; --r) w[k][r] = fma(z[k][r], z[k][r], w[k][r + 1]);
        const uint64_t lowmask = (1ull << v) - 1ull;
        dst[k] = reinterpret_cast<OutT<T, COV>*>(a.out) + ((size_t)v << (a.m - 1)) +
                 (size_t)((F & lowmask) | ((F >> (v + 1)) << v));
        if (on) {  // families of the root: parents = first s free variables
#pragma unroll
            for (int s = 0; s <= Q; ++s)
                emit_ptr<T, COV>(a, dst[k], ((1u << s) - 1u) << (a.k - 1), w[k][s],
                                 fma(T(s), a.lnn, penb[k]));
        }
    }
    const int ksh = a.k - 1;
    auto step = [&](auto rc, uint32_t e, const T2* row) {
        constexpr int r = decltype(rc)::value;
        const uint32_t off = (e >> 4) << ksh;
        const T apen = T(r + 1) * a.lnn;
        T2 cs0;
        if constexpr (SHARED) cs0 = row[lane];
#pragma unroll
        for (int k = 0; k < NI; ++k) {
            T2 cs;
            if constexpr (SHARED)
                cs = cs0;
            else
                cs = row[ell[k]];
            const T x = z[k][r], y = z[k][r + 1];
            z[k][r] = fma(cs.x, x, cs.y * y);
            const T yn = fma(cs.x, y, -cs.y * x);
            z[k][r + 1] = yn;
            const T wn = fma(yn, yn, w[k][r + 2]);
            w[k][r + 1] = wn;
            emit_ptr<T, COV>(a, dst[k], off, wn, penb[k] + apen, act[k]);
        }
    };
    // state machine over rows, as in the producer
    GBN_TIMER_DECL
    int t = 0;
    if (!GBN_TIMED_WAIT(warp_wait(&full[0], 0, a.watchdog_ns, a.status))) return;
    uint32_t e = tab.e[0];
    const T2* row = tape;
#define GBN_CSTEP(r, UP, DOWN)                                                          \
    if (r < Q - 1) {                                                                    \
        step(std::integral_constant<int, (r < Q - 1 ? r : 0)>{}, e, row);               \
        if (++t == N) goto c_done;                                                      \
        if (t % kChunk == 0) {                                                          \
            __syncwarp();                                                               \
            if (lane == 0) mbar_arrive(&empty[(t / kChunk - 1) % kRing]);               \
            if (!GBN_TIMED_WAIT(warp_wait(&full[(t / kChunk) % kRing],                  \
                                          ((t / kChunk) / kRing) & 1, a.watchdog_ns,    \
                                          a.status)))                                   \
                return;                                                                 \
        }                                                                               \
        e = tab.e[t];                                                                   \
        row = tape + ((t / kChunk) % kRing * kChunk + t % kChunk) * 32;                 \
        if ((int)(e & 15u) > r) goto UP;                                                \
        goto DOWN;                                                                      \
    }
c_r0: GBN_CSTEP(0, c_r1, c_r0)
c_r1: GBN_CSTEP(1, c_r2, c_r0)
c_r2: GBN_CSTEP(2, c_r3, c_r1)
c_r3: GBN_CSTEP(3, c_r4, c_r2)
c_r4: GBN_CSTEP(4, c_r5, c_r3)
c_r5: GBN_CSTEP(5, c_r6, c_r4)
c_r6: GBN_CSTEP(6, c_r7, c_r5)
c_r7: GBN_CSTEP(7, c_r8, c_r6)
c_r8: GBN_CSTEP(8, c_r9, c_r7)
c_r9: GBN_CSTEP(9, c_r10, c_r8)
c_r10: GBN_CSTEP(10, c_r10, c_r9)
#undef GBN_CSTEP
c_done:
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[((N - 1) / kChunk) % kRing]);
    GBN_TIMER_FLUSH(a.timing, 1)
}

}  // namespace gbn

// The kernel and its step table exist only in the translation unit compiled
// for one Q (walk_inst.cu with -DGBN_Q=...).
#ifdef GBN_Q
namespace gbn {

__constant__ StepTab<GBN_Q> c_steps = make_step_tab<GBN_Q>();

constexpr int kMaxConsumerWarps = 8;

// Block: warp 0 produces; then warps for the fixed variables above the
// lowest W (NI per thread, all of the lane's own sub-walk); then warps for
// the lowest W variables.
template <typename T, int Q, bool COV, int NI>
__global__ void __launch_bounds__(32 * (1 + kMaxConsumerWarps)) walk_kernel(WalkArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem[];
    using S = Smem<T, Q>;
    static_assert(Q == GBN_Q, "one Q per translation unit");
    static_assert(Q <= 12, "the step table packs the swap row in 4 bits");
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + S::off_bar);
    uint64_t* empty = full + kRing;
    const uint64_t cta = blockIdx.x;
    const int nu = (a.k - a.W) - __popcll(cta);
    const int g = a.W >= 1 ? (a.lanes >> 1) : 1;
    const int n5 = a.W >= 1 ? (a.W + (32 / g) - 1) / (32 / g) : 0;
    const int uw_max = (a.k - a.W + NI - 1) / NI;  // uniform warps launched
    const int uw = (nu + NI - 1) / NI;             // uniform warps with items
    const int lw = (n5 + NI - 1) / NI;             // lowest-W warps
    const int consumers = uw + lw;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kRing; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], consumers > 0 ? consumers : 1);
        }
    }
    __syncthreads();
    const uint64_t Fhi = cta << a.W;
    const T* rec = a.leaves + (size_t)blockIdx.x * a.leaf_stride;
    if (warp == 0) {
        produce<T, Q, COV>(a, c_steps, rec, smem, lane, Fhi | (uint64_t)lane, lane < a.lanes,
                           consumers > 0);
    } else if (warp - 1 < uw_max) {
        if (warp - 1 < uw)
            consume<T, Q, COV, NI, true>(a, c_steps, rec, smem, lane, (warp - 1) * NI, cta, Fhi);
    } else if (warp - 1 - uw_max < lw) {
        consume<T, Q, COV, NI, false>(a, c_steps, rec, smem, lane, (warp - 1 - uw_max) * NI, cta,
                                      Fhi);
    }
}

template <typename T, int Q, bool COV, int NI>
int launch_walk_q(const WalkArgs<T>& a, int64_t n_cta, cudaStream_t stream) {
    const size_t smem = Smem<T, Q>::bytes;
    if (a.n_bwarps < 1 || a.n_bwarps > kMaxConsumerWarps || a.ni != NI) return GBN_ERR_Q;
    if (cudaFuncSetAttribute(walk_kernel<T, Q, COV, NI>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return GBN_ERR_CUDA;
    walk_kernel<T, Q, COV, NI><<<(unsigned)n_cta, 32 * (1 + a.n_bwarps), smem, stream>>>(a);
    return cudaGetLastError() == cudaSuccess ? GBN_OK : GBN_ERR_CUDA;
}

}  // namespace gbn
#endif

// One instantiation per (scalar type, Q, coverage), each compiled as its own
// object from walk_inst.cu so that the build runs in parallel.
#define GBN_WALK_INST_NAME(T, Q, COV) gbn_launch_walk_##T##_q##Q##_c##COV
#define GBN_WALK_DECL(T, Q, COV) \
    int GBN_WALK_INST_NAME(T, Q, COV)(const gbn::WalkArgs<T>& a, int64_t n_cta, cudaStream_t s)

// The Givens walk (Sec. 1.3, Sec. 2, Algorithm 1) over the sub-walks of one CTA.
//
// Each CTA owns 2^W sub-walks that share their front variables above the
// lowest W fixed variables and differ in those W (lane l of a warp <-> the
// sub-walk whose front set holds fixed variable b iff bit b of l is set).  All
// sub-walks run the same local sequence Upsilon(Q), so the swap row of every
// step and the prefix set after it are compile-time constants.
//
// Warp 0 (producer) walks, per lane, the Q x Q block of R over the free
// variables with registers named by column position and writes the rotation
// of every step to a tape in shared memory: cos = r_{i,i+1}/rho and
// sin = r_{i+1,i+1}/rho, the rotation of the GRC operator that zeroes the
// sub-diagonal (the paper prints the same numerator for both).  The swap rows
// move by exactly one per step (Algorithm 1 joins its parts at rows that
// differ by one), so the producer is a state machine with one straight-line
// block per row and a direct branch to the row above or below: its code size
// is O(Q^2), whatever the 2^Q - Q - 1 steps.
//
// The other warps (consumers) take the CTA's columns one at a time and replay
// the whole tape over each with straight-line code unrolled over the steps:
//   * free variable j: its column of the root block;  it is a child whenever
//     j is behind the prefix;
//   * fixed variable v outside the front set: its Q entries in the free
//     block's rows plus the residual C below them; a child of every prefix.
// A column is a Q-vector z with tail sums w[r] = sum_{t>=r} z_t^2 + C, the RSS
// of the column on the variables in positions < r.  A swap at row i rotates
// rows i, i+1 of z (rows ahead of the column's position are zero and stay
// zero) and changes only w[i+1] = w[i+2] + z_{i+1}^2; the families it adds are
// those whose parent set is the new prefix of length i+1 (Sec. 4).
//
// The tape is written in chunks; each chunk has an mbarrier the producer
// arrives on, so consumers start on the first chunk while the producer walks
// on.  Every wait is bounded by a wall-clock watchdog that records
// GBN_STATUS_WATCHDOG and returns.
//
// Scores: score = n ln(RSS/n) + |S| ln n = (n ln 2) log2(RSS) + (|S| ln n - n ln n),
// stored at idx(c,S) = c 2^(m-1) + compress(S, c); the lanes of a warp write
// consecutive table slots.
//
// FP32 scores with full warps of sub-walks take one of two refinements:
//   * the paired walk: one block runs the 64 sub-walks of two neighbouring
//     roots CTAs, and a consumer lane carries two of them whose front sets
//     differ in fixed variable 0 only.  Two producer warps write one tape of
//     (c_x, c_y, s_x, s_y) per step and lane; the lane holds its column of
//     both sub-walks in float2 registers and rotates, sums and scores them
//     with packed FP32 instructions, and both scores leave in one 8-byte
//     store (the slots are adjacent);
//   * the paired ring (Q <= 6): the same pairs in persistent blocks with two
//     tapes in shared memory, so one pair's tape is written while the
//     consumers replay the previous one.
#pragma once

#include <mutex>
#include <type_traits>
#include <utility>
#include <vector>

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
    T alpha;                     // n ln 2
    T lam;                       // penalty per parent (ln n for BIC, 2 for AIC)
    T nlnn;                      // n ln n
    unsigned long long* chk;     // check record (checked builds)
    unsigned long long* timing;  // role cycle counters (timing builds)
    int* status;                 // status word (watchdog bit)
    size_t out_size;             // table elements
    int n_cwarps;                // consumer warps per CTA
    long long watchdog_ns;       // bound on every wait
    int kmax;                    // families with more parents are not stored (m - 1: no bound)
    int64_t cta0;                // global index of this launch's first sub-walk CTA (sharding)
};


// Walk arguments of one dataset (host side).
template <typename T>
inline WalkArgs<T> make_walk_args(const Plan& p, char* ws, void* out) {
    WalkArgs<T> a;
    a.out = out;
    a.leaves = reinterpret_cast<const T*>(ws + p.off_leaves);
    a.leaf_stride = p.leaf_stride;
    a.m = p.m;
    a.k = p.k;
    a.W = p.W;
    a.lanes = p.lanes;
    const double n = (double)p.n;
    a.alpha = (T)(n * 0.69314718055994530942);
    a.lam = (T)p.lam;
    a.nlnn = (T)(n * log(n));
    a.chk = reinterpret_cast<unsigned long long*>(ws + p.off_status + kCheckOffset);
    a.timing = reinterpret_cast<unsigned long long*>(ws + p.off_status + kTimingOffset);
    a.status = reinterpret_cast<int*>(ws + p.off_status);
    a.out_size = (size_t)p.m << (p.m - 1);
    a.n_cwarps = p.n_bwarps;
    a.watchdog_ns = p.watchdog_ns;
    a.kmax = p.kmax;
    a.cta0 = p.cta_begin;
    return a;
}

constexpr int kChunk = 16;  // tape steps per barrier
// Levels of code sharing in the consumers' replay: blocks of at most
// kSplitBase variables (|Upsilon(kSplitBase)| steps of unrolled code).
constexpr int kSplitBase = 6;
constexpr int split_levels(int Q) { return Q <= kSplitBase ? 0 : Q - kSplitBase; }

// The swap sequence of Algorithm 1 with, per step, the 0-based swap row i
// (the paper's GRC_{i+1}) and the mask of the local free variables at
// positions 0..i after the swap.
template <int Q>
struct StepTab {
    static constexpr int N = (1 << Q) - Q - 1;  // |Upsilon(Q)|, Sec. 3
    uint8_t row[N > 0 ? N : 1];
    uint16_t pre[N > 0 ? N : 1];
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
        unsigned mask = 0;
        for (int p = 0; p < i; ++p) mask |= 1u << pos[p];
        tab.row[t] = (uint8_t)(i - 1);
        tab.pre[t] = (uint16_t)mask;
    }
    return tab;
}

template <int Q>
inline constexpr StepTab<Q> kSteps = make_step_tab<Q>();

// Per step t and column bit jj (0..Q-1 a free variable, Q a fixed one): the
// prefix mask compressed for that column's child block, or kNotChild when
// the column's variable is itself in the prefix.
constexpr uint16_t kNotChild = 0xffff;
template <int Q>
struct SlotTab {
    static constexpr int N = StepTab<Q>::N;
    uint16_t v[(N > 0 ? N : 1) * (Q + 1)];
};
template <int Q>
constexpr SlotTab<Q> make_slot_tab() {
    SlotTab<Q> tab{};
    const StepTab<Q> st = make_step_tab<Q>();
    for (int t = 0; t < StepTab<Q>::N; ++t)
        for (int jj = 0; jj <= Q; ++jj) {
            const unsigned pre = st.pre[t], lm = (1u << jj) - 1u;
            tab.v[t * (Q + 1) + jj] = ((pre >> jj) & 1u)
                                          ? kNotChild
                                          : (uint16_t)((pre & lm) | ((pre >> 1) & ~lm));
        }
    return tab;
}

#ifdef GBN_Q
// The step table of this translation unit's Q in constant memory (the
// producer's rows), and the consumers' compressed slot table.
__constant__ StepTab<GBN_Q> c_steps = make_step_tab<GBN_Q>();
__constant__ SlotTab<GBN_Q> c_slots = make_slot_tab<GBN_Q>();
#endif

__device__ __forceinline__ float wk_rsqrt(float x) { return rsqrtf(x); }
__device__ __forceinline__ double wk_rsqrt(double x) { return rsqrt(x); }
// FP32: the hardware base-2 logarithm with subnormal inputs flushed to zero
// (an RSS below 2^-126 scores -inf; the FP64 fix-up re-scores such families).
__device__ __forceinline__ float wk_log2(float x) {
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
// FP64: the library's base-2 logarithm.
__device__ __forceinline__ double wk_log2(double x) { return log2(x); }
__device__ __forceinline__ float2 wk_pair(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ double2 wk_pair(double a, double b) { return make_double2(a, b); }

// Element type of the output table: scores, or 32-bit counters in coverage mode.
template <typename T, bool COV>
using OutT = typename std::conditional<COV, unsigned, T>::type;

__device__ __forceinline__ void st_pred(float* addr, float v, bool on) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %2, 0;\n\t@p st.global.f32 [%0], %1;\n\t}"
        :
        : "l"(addr), "f"(v), "r"((unsigned)on));
}
__device__ __forceinline__ void st_pred(double* addr, double v, bool on) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %2, 0;\n\t@p st.global.f64 [%0], %1;\n\t}"
        :
        : "l"(addr), "d"(v), "r"((unsigned)on));
}

// Store at p + off (p: a per-thread pointer into the table, off < 2^32) when
// `on`.  The score is computed unconditionally; only the store is predicated.
template <typename T, bool COV>
__device__ __forceinline__ void emit_ptr(const WalkArgs<T>& a, OutT<T, COV>* p, uint32_t off,
                                         T rss, T pen, bool on) {
    if constexpr (COV) {
        if (on && GBN_IN(a.chk, 302,
                         (size_t)(p - reinterpret_cast<OutT<T, COV>*>(a.out)) + off, a.out_size))
            atomicAdd(p + off, 1u);
    } else {
        const T v = fma(a.alpha, wk_log2(rss), pen);
#ifdef GBN_CHECKED
        if (on && GBN_IN(a.chk, 302,
                         (size_t)(p - reinterpret_cast<OutT<T, COV>*>(a.out)) + off, a.out_size))
            p[off] = v;
#else
        st_pred(p + off, v, on);  // a predicated store, never a branch around it
#endif
    }
}

// Store the score of the family at byte address base + cT * stride when
// cT is a slot (not kNotChild) and `on` is set: one wide multiply-add forms
// the address, and the predicate is built inside the store's own asm.
__device__ __forceinline__ void st_slot(char* base, unsigned stride, unsigned cT, float v,
                                        unsigned on) {
    char* addr = base + (size_t)cT * stride;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 q, %3, 0;\n\t"
        "setp.ne.and.u32 p, %2, 65535, q;\n\t@p st.global.cs.f32 [%0], %1;\n\t}"
        :
        : "l"(addr), "f"(v), "r"(cT), "r"(on));
}
__device__ __forceinline__ void st_slot(char* base, unsigned stride, unsigned cT, double v,
                                        unsigned on) {
    char* addr = base + (size_t)cT * stride;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 q, %3, 0;\n\t"
        "setp.ne.and.u32 p, %2, 65535, q;\n\t@p st.global.cs.f64 [%0], %1;\n\t}"
        :
        : "l"(addr), "d"(v), "r"(cT), "r"(on));
}

// Prefetch [p, p + bytes) into L2, one 128-byte line per thread and pass: a
// paired-walk block's leaf records are read at the start of each consumer item,
// and most of them are no longer in L2 when the walk reaches them (the leaf
// kernel wrote them all before); fetching them when the block starts turns the
// later items' record loads into L2 hits (m = 26: walk 0.712 -> 0.692 ms).  The
// ring walk's producers, one unit ahead of its consumers, measured slower with
// the same prefetch (q = 6: 0.777 -> 0.828 ms) and do without it.
__device__ __forceinline__ void prefetch_l2(const void* p, size_t bytes, unsigned t, unsigned nt) {
    const char* b = static_cast<const char*>(p);
    for (size_t o = (size_t)t * 128; o < bytes; o += (size_t)nt * 128)
        asm volatile("prefetch.global.L2 [%0];" ::"l"(b + o));
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
// One poll that suspends: a thread whose phase is not complete is suspended
// until it completes or about kSuspendNs pass, so a waiting warp issues
// almost nothing.
constexpr unsigned kSuspendNs = 20000;
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2, "
        "%3;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity), "r"(kSuspendNs)
        : "memory");
    return ok != 0;
}
// One poll that returns at once.
__device__ __forceinline__ bool mbar_test_wait(uint64_t* bar, unsigned parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.acquire.cta.shared::cta.b64 p, [%1], "
        "%2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
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
// Bounded wait for the phase with the given parity (false = the watchdog
// expired).  The first poll returns at once; after it fails, the clock
// starts and every later poll suspends (up to about kSuspendNs) and is
// followed by a clock check, so a wait that is not complete within limit_ns
// ends after about that long.  A bound below kSuspendNs cannot be resolved by
// suspending polls: such a bound expires a wait whose phase is not complete
// at its first poll (so a bound shorter than the producer's time for one tape
// chunk makes a consumer's first wait expire).  Warp-uniform: every lane
// polls (one instruction for the warp, the same phase seen by all lanes, each
// lane's own acquire), so the loop has no divergent branch and no broadcast;
// only the watchdog's status write is made by lane 0.
__device__ __forceinline__ bool warp_wait(uint64_t* bar, unsigned parity, long long limit_ns,
                                          int* status) {
    if (mbar_test_wait(bar, parity)) return true;
    if (limit_ns >= (long long)kSuspendNs) {
        const long long t0 = global_ns();
        for (;;) {
            if (mbar_try_wait(bar, parity)) return true;
            if (global_ns() - t0 > limit_ns) break;
        }
    }
    if ((threadIdx.x & 31) == 0) atomicOr(status, GBN_STATUS_WATCHDOG);
    return false;
}

// Timing builds (-DGBN_TIMING) add the cycles each role spends in total and
// waiting on the tape barriers to counters in the workspace status block:
// [0] producer total, [1] producer waiting, [2] consumer total, [3] consumer
// waiting (summed over warps, lane 0 only).  Ordinary builds compile them away.
#ifdef GBN_TIMING
#define GBN_TIMER_DECL long long gbn_t_wait = 0, gbn_t_start = clock64();
#define GBN_TIMED_WAIT(expr)                \
    ({                                      \
        const long long gbn_t0 = clock64(); \
        const bool gbn_ok = (expr);         \
        gbn_t_wait += clock64() - gbn_t0;   \
        gbn_ok;                             \
    })
#define GBN_TIMER_FLUSH(ctr, slot)                                                              \
    if ((threadIdx.x & 31) == 0) {                                                              \
        atomicAdd((unsigned long long*)(ctr) + 2 * (slot),                                      \
                  (unsigned long long)(clock64() - gbn_t_start));                               \
        atomicAdd((unsigned long long*)(ctr) + 2 * (slot) + 1, (unsigned long long)gbn_t_wait); \
    }
#else
#define GBN_TIMER_DECL
#define GBN_TIMED_WAIT(expr) (expr)
#define GBN_TIMER_FLUSH(ctr, slot)
#endif

template <int... Is, class F>
__device__ __forceinline__ void static_for(std::integer_sequence<int, Is...>, F&& f) {
    (f(std::integral_constant<int, Is>{}), ...);
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

// Shared-memory layout of one CTA: the whole tape and one barrier per chunk.
template <typename T, int Q>
struct Smem {
    static constexpr int N = StepTab<Q>::N;
    static constexpr int chunks = (N + kChunk - 1) / kChunk;
    static constexpr size_t off_tape = 0;
    static constexpr size_t off_bar = ((size_t)N * 32 * 2 * sizeof(T) + 15) / 16 * 16;
    static constexpr size_t bytes = off_bar + (size_t)chunks * sizeof(uint64_t);
};

// Shared memory of the paired walk: a tape of (c_x, c_y, s_x, s_y) per step and
// lane (FP32), then the chunk barriers (two producer arrivals each).
template <int Q>
struct SmemP {
    static constexpr int N = StepTab<Q>::N;
    static constexpr int chunks = (N + kChunk - 1) / kChunk;
    static constexpr size_t off_tape = 0;
    static constexpr size_t off_bar = (size_t)N * 32 * 4 * sizeof(float);
    static constexpr size_t bytes = off_bar + (size_t)chunks * sizeof(uint64_t);
};

// One swap of the producer at compile-time row I.  R is named by position:
// R[r * Q + p] (r <= p) is row r of the column at position p.
template <typename T, int Q, int I>
__device__ __forceinline__ void produce_step(T (&R)[Q * Q], T& c_out, T& s_out) {
    const T x0 = R[I * Q + I + 1], y0 = R[(I + 1) * Q + I + 1];
    const T rho2 = fma(x0, x0, y0 * y0);
    const T inv = wk_rsqrt(rho2);
    const bool ok = rho2 > T(0);
    const T c = ok ? x0 * inv : T(1);
    const T s = ok ? y0 * inv : T(0);
    const T rii = R[I * Q + I];
    // transpose positions I and I+1: the rows above I move with their columns
#pragma unroll
    for (int r = 0; r < I; ++r) {
        const T tr = R[r * Q + I];
        R[r * Q + I] = R[r * Q + I + 1];
        R[r * Q + I + 1] = tr;
    }
    R[I * Q + I] = ok ? rho2 * inv : T(0);
    R[I * Q + I + 1] = c * rii;
    R[(I + 1) * Q + I + 1] = -s * rii;
#pragma unroll
    for (int p = I + 2; p < Q; ++p) {
        const T x = R[I * Q + p], y = R[(I + 1) * Q + p];
        R[I * Q + p] = fma(c, x, s * y);
        R[(I + 1) * Q + p] = fma(c, y, -s * x);
    }
    c_out = c;
    s_out = s;
}

// Producer: one sub-walk per lane over its free block, rotations only.  It
// stays a state machine: a version unrolled over all 2^Q - Q - 1 steps (swaps
// as register renames, no row table) measured 20-30 % slower at Q = 6, 7 --
// its code does not stay in the instruction cache beside the consumers'.
// PAIR false: the tape holds (c, s) per step and lane.  PAIR true (the
// paired walk): the tape holds four words per step and consumer lane,
// (c_x, c_y, s_x, s_y), and this lane writes its c to word tl and its s to
// word tl + 2 of each step's 128.
template <typename T, int Q, bool PAIR = false>
__device__ __forceinline__ void produce(const WalkArgs<T>& a, const StepTab<Q>& tab,
                                        const T* __restrict__ rec, unsigned char* tape_base,
                                        uint64_t* full, int lane, bool active, int tl = 0) {
    using T2 = typename Vec2T<T>::type;
    constexpr int N = StepTab<Q>::N;
    T2* tape = reinterpret_cast<T2*>(tape_base);
    T* tape4 = reinterpret_cast<T*>(tape_base);
    T R[Q * Q];
    static_for(std::make_integer_sequence<int, Q>{}, [&](auto pc) {
        constexpr int p = decltype(pc)::value;
        static_for(std::make_integer_sequence<int, p + 1>{}, [&](auto rc) {
            constexpr int r = decltype(rc)::value;
            const size_t e = (size_t)(p * (p + 1) / 2 + r) * 32 + lane;
            R[r * Q + p] = (active && GBN_IN(a.chk, 311, e, a.leaf_stride)) ? rec[e] : T(0);
        });
    });
    GBN_TIMER_DECL
    int t = 0;
    T c = T(1), s = T(0);
#define GBN_PSTEP(r, UP, DOWN)                                                     \
    if (r < Q - 1) {                                                               \
        produce_step<T, Q, (r < Q - 1 ? r : 0)>(R, c, s);                          \
        if constexpr (!PAIR) {                                                     \
            tape[t * 32 + lane] = wk_pair(c, s);                                   \
        } else {                                                                   \
            tape4[t * 128 + tl] = c;                                               \
            tape4[t * 128 + tl + 2] = s;                                           \
        }                                                                          \
        if (++t == N) goto p_done;                                                 \
        if (t % kChunk == 0) {                                                     \
            __syncwarp();                                                          \
            if (lane == 0) mbar_arrive(&full[t / kChunk - 1]);                     \
        }                                                                          \
        if ((int)tab.row[t] > r) goto UP;                                          \
        goto DOWN;                                                                 \
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
    if (lane == 0) mbar_arrive(&full[(N - 1) / kChunk]);
    GBN_TIMER_FLUSH(a.timing, 0)
}

// One column replayed from the tape with straight-line code.  jj is the bit
// of the column's free variable in the prefix masks (Q for a fixed variable:
// never in a prefix), sh the shift that places the compressed prefix mask in
// the table slot, kr the largest prefix length whose families are stored
// (the in-degree bound less the lane's front-set size).  Returns false if a
// wait expired.
template <typename T, int Q, bool COV>
__device__ __forceinline__ bool replay(const WalkArgs<T>& a, const typename Vec2T<T>::type* tape,
                                       uint64_t* full, unsigned par, T (&z)[Q], T cres, int ell,
                                       int jj, int sh,
                                       OutT<T, COV>* base, T penb, bool on, int kr) {
    constexpr int N = StepTab<Q>::N;
    T w[Q + 1];
    w[Q] = cres;
#pragma unroll
    for (int r = Q - 1; r >= 0; --r) w[r] = fma(z[r], z[r], w[r + 1]);
    const unsigned lm = (1u << jj) - 1u;
    // families of the root: parents = the first s free variables
    static_for(std::make_integer_sequence<int, Q + 1>{}, [&](auto sc) {
        constexpr int s = decltype(sc)::value;
        constexpr unsigned pre = (1u << s) - 1u;
        const bool child = !((pre >> jj) & 1u);
        const unsigned cT = (pre & lm) | ((pre >> 1) & ~lm);
        emit_ptr<T, COV>(a, base, cT << sh, w[s], fma(T(s), a.lam, penb), on && child && s <= kr);
    });
    bool ok = true;
    static_for(std::make_integer_sequence<int, N>{}, [&](auto tc) {
        constexpr int t = decltype(tc)::value;
        if constexpr (t % kChunk == 0) {
            if (ok) ok = warp_wait(&full[t / kChunk], par, a.watchdog_ns, a.status);
        }
        constexpr int i = kSteps<Q>.row[t];
        constexpr unsigned pre = kSteps<Q>.pre[t];
        const auto cs = tape[t * 32 + ell];
        const T x = z[i], y = z[i + 1];
        z[i] = fma(cs.x, x, cs.y * y);
        const T yn = fma(cs.x, y, -cs.y * x);
        z[i + 1] = yn;
        const T wn = fma(yn, yn, w[i + 2]);
        w[i + 1] = wn;
#ifdef GBN_Q
        (void)pre;
        const unsigned cT = c_slots.v[t * (Q + 1) + jj];
        emit_ptr<T, COV>(a, base, cT << sh, wn, fma(T(i + 1), a.lam, penb),
                         on && cT != kNotChild && i + 1 <= kr);
#else
        const bool child = !((pre >> jj) & 1u);
        const unsigned cT = (pre & lm) | ((pre >> 1) & ~lm);
        emit_ptr<T, COV>(a, base, cT << sh, wn, fma(T(i + 1), a.lam, penb),
                         on && child && ok && i + 1 <= kr);
#endif
    });
    return ok;
}

#ifdef GBN_Q
// The same replay with 2^-H of the code, using the recursion of Algorithm 1,
// Upsilon(q) = Upsilon(q-1) : [q-1 .. 1] : (Upsilon(q-1) + 1), H times:
// Upsilon(Q) is 2^H blocks of Upsilon(Q-H), block b acting on rows shifted
// by popcount(b), each followed (except the last) by the chain of level L =
// trailing ones of b -- [Q-H+L .. 1] shifted by popcount(b >> (L+1)).  One
// unrolled copy of the block's steps runs 2^H times through a shifted
// register view; each (chain length, shift) pair has one unrolled copy; the
// prefix masks come from the constant step table at run time.  The walk is
// bound by instruction fetch, so shrinking its code pays for the table load.
// Calls f(integral_constant<OO>) for exactly one OO in 0 .. NB: OO = x, or NB
// when x >= NB.  Every path takes one branch, so a value written in all of
// them is known to be overwritten (a plain "if (x == OO)" per OO leaves a
// path with none taken and keeps the old values alive in registers).
template <int OO, int NB, class F>
__device__ __forceinline__ void pick_from(int x, F&& f) {
    if constexpr (OO == NB) {
        f(std::integral_constant<int, OO>{});
    } else {
        if (x == OO)
            f(std::integral_constant<int, OO>{});
        else
            pick_from<OO + 1, NB>(x, f);
    }
}
template <int NB, class F>
__device__ __forceinline__ void pick(int x, F&& f) {
    pick_from<0, NB>(x, f);
}

template <int Q1, int NB>
struct ViewCopy {  // zv/wv <-> z/w rows o .. o + Q1 (o a run-time shift 0 .. NB)
    template <typename T, int Q>
    __device__ static __forceinline__ void in(T (&zv)[Q1], T (&wv)[Q1 + 1], const T (&z)[Q],
                                              const T (&w)[Q + 1], int o) {
        pick<NB>(o, [&](auto oc) {
            constexpr int oo = decltype(oc)::value;
            static_for(std::make_integer_sequence<int, Q1>{}, [&](auto rc) {
                constexpr int r = decltype(rc)::value;
                zv[r] = z[r + oo];
                wv[r] = w[r + oo];
            });
            wv[Q1] = w[Q1 + oo];
        });
    }
    template <typename T, int Q>
    __device__ static __forceinline__ void out(const T (&zv)[Q1], const T (&wv)[Q1 + 1], T (&z)[Q],
                                               T (&w)[Q + 1], int o) {
        pick<NB>(o, [&](auto oc) {
            constexpr int oo = decltype(oc)::value;
            static_for(std::make_integer_sequence<int, Q1>{}, [&](auto rc) {
                constexpr int r = decltype(rc)::value;
                z[r + oo] = zv[r];
                w[r + oo] = wv[r];
            });
        });
    }
};

template <typename T, int Q, int H, bool COV>
__device__ __forceinline__ bool replay_split(const WalkArgs<T>& a,
                                             const typename Vec2T<T>::type* tape, uint64_t* full,
                                             unsigned par, T (&z)[Q], T cres, int ell, int jj, int sh,
                                             OutT<T, COV>* base, T penb, bool on, int kr) {
    static_assert(Q == GBN_Q, "the step table in constant memory is this unit's");
    static_assert(H >= 1 && Q - H >= 2, "blocks of at least two variables");
    constexpr int N = StepTab<Q>::N;
    constexpr int last_chunk = (N - 1) / kChunk;
    constexpr int QB = Q - H;              // variables of a block
    constexpr int NBLK = StepTab<QB>::N;   // steps of a block
    T w[Q + 1];
    w[Q] = cres;
#pragma unroll
    for (int r = Q - 1; r >= 0; --r) w[r] = fma(z[r], z[r], w[r + 1]);
    const unsigned lm = (1u << jj) - 1u;
    static_for(std::make_integer_sequence<int, Q + 1>{}, [&](auto sc) {  // the root's families
        constexpr int s = decltype(sc)::value;
        constexpr unsigned pre = (1u << s) - 1u;
        const bool child = !((pre >> jj) & 1u);
        const unsigned cT = (pre & lm) | ((pre >> 1) & ~lm);
        emit_ptr<T, COV>(a, base, cT << sh, w[s], fma(T(s), a.lam, penb), on && child && s <= kr);
    });
    // one step at row i (of the view), tape step t; the compressed slot from
    // the table; kv the largest stored prefix length within the view.  After
    // an expired wait the remaining stores may hold stale scores; the status
    // word reports it.
    const uint16_t* slots = c_slots.v + jj;
    char* const base_b = reinterpret_cast<char*>(base);
    const unsigned stride = (unsigned)sizeof(OutT<T, COV>) << sh;
    const unsigned on_u = on ? 1u : 0u;
    auto step = [&](auto& zz, auto& ww, int kv, auto ic, int t, T pen_base, bool& ok) {
        constexpr int i = decltype(ic)::value;
        (void)ok;
        const unsigned cT = slots[t * (Q + 1)];
        const auto cs = tape[(size_t)t * 32 + ell];
        const T x = zz[i], y = zz[i + 1];
        zz[i] = fma(cs.x, x, cs.y * y);
        const T yn = fma(cs.x, y, -cs.y * x);
        zz[i + 1] = yn;
        const T wn = fma(yn, yn, ww[i + 2]);
        ww[i + 1] = wn;
        if constexpr (COV) {
            emit_ptr<T, COV>(a, base, cT << sh, wn, fma(T(i + 1), a.lam, pen_base),
                             on && cT != kNotChild && i + 1 <= kv);
        } else {
#ifdef GBN_CHECKED
            emit_ptr<T, COV>(a, base, cT << sh, wn, fma(T(i + 1), a.lam, pen_base),
                             on && cT != kNotChild && i + 1 <= kv);
#else
            (void)base_b;
            st_slot(base_b, stride, cT, fma(a.alpha, wk_log2(wn), fma(T(i + 1), a.lam, pen_base)),
                    on_u & (unsigned)(i + 1 <= kv));
#endif
        }
    };
    auto wait_for = [&](int t, bool& ok) {  // tape steps t .. t + kChunk - 1 are written
        int c = (t + kChunk - 1) / kChunk;
        if (c > last_chunk) c = last_chunk;
        if (ok) ok = warp_wait(&full[c], par, a.watchdog_ns, a.status);
    };
    bool ok = true;
    int t0 = 0;  // tape step of the current block's first step
#pragma unroll 1
    for (int b = 0; b < (1 << H); ++b) {
        const int o = __popc(b);  // row shift of this block
        T zv[QB], wv[QB + 1];
        ViewCopy<QB, H>::template in<T, Q>(zv, wv, z, w, o);
        const T penv = fma(T(o), a.lam, penb);  // the o moved variables are parents throughout
        static_for(std::make_integer_sequence<int, NBLK>{}, [&](auto tc) {
            constexpr int t = decltype(tc)::value;
            if constexpr (t % kChunk == 0) wait_for(t0 + t, ok);
            step(zv, wv, kr - o, std::integral_constant<int, kSteps<QB>.row[t]>{}, t0 + t, penv,
                 ok);
        });
        ViewCopy<QB, H>::template out<T, Q>(zv, wv, z, w, o);
        t0 += NBLK;
        if (b + 1 == (1 << H)) break;
        // the chain after block b: level L = trailing ones of b, variables QB + 1 + L,
        // rows shifted by popcount(b >> (L + 1))
        const int L = __ffs(~b) - 1;
        const int oc = __popc(b >> (L + 1));
        wait_for(t0, ok);
        static_for(std::make_integer_sequence<int, H>{}, [&](auto lc) {
            constexpr int LL = decltype(lc)::value;
            constexpr int len = QB + LL;  // chain [QB+LL .. 1]
            if (L == LL) {
                static_for(std::make_integer_sequence<int, H - LL>{}, [&](auto occ) {
                    constexpr int OO = decltype(occ)::value;
                    if (oc == OO) {
                        static_for(std::make_integer_sequence<int, len>{}, [&](auto uc) {
                            constexpr int u = decltype(uc)::value;
                            constexpr int i = OO + len - 1 - u;  // absolute swap row
                            step(z, w, kr, std::integral_constant<int, i>{}, t0 + u, penb, ok);
                        });
                    }
                });
                t0 += len;
            }
        });
    }
    return ok;
}
#endif

#ifdef GBN_Q
// ---------------------------------------------------------------- paired walk
// A block takes the 64 sub-walks of roots CTAs 2c and 2c+1 (W = 5: fixed
// variables 0..4 vary over a CTA's lanes, variable 5 tells the two CTAs
// apart).  Consumer lane l (the "pair lane") carries two sub-walks, x and y,
// whose front sets differ in fixed variable 0 only:
//     F_x = (c << 6) | (l << 1),  F_y = F_x | 1,
// that is roots CTA 2c + (l >> 4), CTA lanes 2 (l & 15) and 2 (l & 15) + 1.
// A column's entries of both sit in one float2 and every rotation, tail sum
// and score is one packed FP32 operation for the two families.  Because
// variable 0 is the lowest, the two scores of every column but variable 0's
// land in adjacent table slots (one 8-byte store); variable 0 is a child of
// x only (one 4-byte store).  The tape holds (c_x, c_y, s_x, s_y) per step
// and pair lane.  Same block/chain structure as replay_split.
__device__ __forceinline__ float2 f2(float x) { return make_float2(x, x); }

// Tape word (of a step's 128) of producer warp h's lane: its sub-walk is
// pair lane (h << 4) | (lane >> 1), component x (even lane) or y (odd lane).
__device__ __forceinline__ int pair_tape_word(int h, int lane) {
    return (((h << 4) | (lane >> 1)) << 2) | (lane & 1);
}

// Store both scores (8 bytes at base + cT * stride) when on_xy, or only x's
// (4 bytes) when on_x, if cT is a slot; the address is one wide multiply-add
// and the predicates are formed inside the store's own asm.  The table is
// written once and not read back here: streaming stores (.cs) measured 2 %
// faster than default ones.
__device__ __forceinline__ void st_pair(char* base, unsigned stride, unsigned cT, float2 v,
                                        unsigned on_xy, unsigned on_x) {
    char* addr = base + (size_t)cT * stride;
    asm volatile(
        "{\n\t.reg .pred q, r, a, b;\n\tsetp.ne.u32 q, %4, 0;\n\tsetp.ne.u32 r, %5, 0;\n\t"
        "setp.ne.and.u32 a, %3, 65535, q;\n\tsetp.ne.and.u32 b, %3, 65535, r;\n\t"
        "@a st.global.cs.v2.f32 [%0], {%1, %2};\n\t@b st.global.cs.f32 [%0], %1;\n\t}"
        :
        : "l"(addr), "f"(v.x), "f"(v.y), "r"(cT), "r"(on_xy), "r"(on_x));
}

// KB: the bounded in-degree form.  kx is the largest prefix length whose
// family of sub-walk x is stored (the bound less |F_x|); y's families have
// one parent more, so at a prefix length where only x's family is within
// the bound the 8-byte store becomes x's 4-byte store.
template <int Q, int H, bool KB>
__device__ __forceinline__ bool replay_pair(const WalkArgs<float>& a, const float4* tape,
                                            uint64_t* full, unsigned par, float2 (&z)[Q], float2 cres,
                                            int ell, int jj, int sh, char* base, float2 penb,
                                            unsigned on_xy, unsigned on_x, int kx) {
    static_assert(Q == GBN_Q, "the step tables in constant memory are this unit's");
    constexpr int N = StepTab<Q>::N;
    constexpr int last_chunk = (N - 1) / kChunk;
    constexpr int QB = Q - H;
    constexpr int NBLK = StepTab<QB>::N;
    float2 w[Q + 1];
    w[Q] = cres;
#pragma unroll
    for (int r = Q - 1; r >= 0; --r) w[r] = __ffma2_rn(z[r], z[r], w[r + 1]);
    const float2 alpha2 = f2(a.alpha), lnn2 = f2(a.lam);
    const unsigned stride = 4u << sh;
    const unsigned lm = (1u << jj) - 1u;
    (void)kx;
    // pl: the family's prefix length within the view, kv: the largest one stored for x
    auto emit2 = [&](unsigned cT, float2 rss, float2 pen, int pl, int kv) {
        unsigned oxy = on_xy, ox = on_x;
        if constexpr (KB) {  // y has one parent more than x (fixed variable 0)
            const unsigned y_in = (unsigned)(pl + 1 <= kv), x_in = (unsigned)(pl <= kv);
            ox = (on_x | (on_xy & (y_in ^ 1u))) & x_in;
            oxy = on_xy & y_in;
        }
        (void)pl;
        (void)kv;
        const float2 lg = make_float2(wk_log2(rss.x), wk_log2(rss.y));
        const float2 sc = __ffma2_rn(alpha2, lg, pen);
#ifdef GBN_CHECKED
        if (cT != kNotChild) {
            const size_t e0 = (size_t)(base - reinterpret_cast<char*>(a.out)) / 4 +
                              (size_t)cT * (stride / 4);
            float* p = reinterpret_cast<float*>(base + (size_t)cT * stride);
            if ((oxy || ox) && GBN_IN(a.chk, 332, e0, a.out_size)) p[0] = sc.x;
            if (oxy && GBN_IN(a.chk, 333, e0 + 1, a.out_size)) p[1] = sc.y;
            if (oxy && (e0 & 1)) GBN_IN(a.chk, 334, e0, 0);  // an 8-byte store must be aligned
        }
#else
        st_pair(base, stride, cT, sc, oxy, ox);
#endif
    };
    static_for(std::make_integer_sequence<int, Q + 1>{}, [&](auto sc) {  // the roots' families
        constexpr int s = decltype(sc)::value;
        constexpr unsigned pre = (1u << s) - 1u;
        const unsigned cT = ((pre >> jj) & 1u) ? kNotChild : ((pre & lm) | ((pre >> 1) & ~lm));
        emit2(cT, w[s], __ffma2_rn(f2(float(s)), lnn2, penb), s, kx);
    });
    const uint16_t* slots = c_slots.v + jj;
    auto step = [&](auto& zz, auto& ww, auto ic, int t, float2 pen_base, int kv) {
        constexpr int i = decltype(ic)::value;
        const unsigned cT = slots[t * (Q + 1)];
        const float4 cs = tape[(size_t)t * 32 + ell];
        const float2 c2 = make_float2(cs.x, cs.y), s2 = make_float2(cs.z, cs.w);
        const float2 x = zz[i], y = zz[i + 1];
        zz[i] = __ffma2_rn(c2, x, __fmul2_rn(s2, y));
        // -(s x) as one packed multiply by -1 (exact), not two scalar negations
        const float2 nsx = __fmul2_rn(__fmul2_rn(s2, x), f2(-1.f));
        const float2 yn = __ffma2_rn(c2, y, nsx);
        zz[i + 1] = yn;
        const float2 wn = __ffma2_rn(yn, yn, ww[i + 2]);
        ww[i + 1] = wn;
        emit2(cT, wn, __ffma2_rn(f2(float(i + 1)), lnn2, pen_base), i + 1, kv);
    };
    auto wait_for = [&](int t, bool& ok) {
        int c = (t + kChunk - 1) / kChunk;
        if (c > last_chunk) c = last_chunk;
        if (ok) ok = warp_wait(&full[c], par, a.watchdog_ns, a.status);
    };
    bool ok = true;
    int t0 = 0;
#pragma unroll 1
    for (int b = 0; b < (1 << H); ++b) {
        const int o = __popc(b);
        float2 zv[QB], wv[QB + 1];
        ViewCopy<QB, H>::template in<float2, Q>(zv, wv, z, w, o);
        const float2 penv = __ffma2_rn(f2(float(o)), lnn2, penb);
        static_for(std::make_integer_sequence<int, NBLK>{}, [&](auto tc) {
            constexpr int t = decltype(tc)::value;
            if constexpr (t % kChunk == 0) wait_for(t0 + t, ok);
            step(zv, wv, std::integral_constant<int, kSteps<QB>.row[t]>{}, t0 + t, penv, kx - o);
        });
        ViewCopy<QB, H>::template out<float2, Q>(zv, wv, z, w, o);
        t0 += NBLK;
        if (b + 1 == (1 << H)) break;
        const int L = __ffs(~b) - 1;
        const int oc = __popc(b >> (L + 1));
        wait_for(t0, ok);
        static_for(std::make_integer_sequence<int, (H > 0 ? H : 1)>{}, [&](auto lc) {
            constexpr int LL = decltype(lc)::value;
            constexpr int len = QB + LL;
            if (L == LL) {
                static_for(std::make_integer_sequence<int, (H > LL ? H - LL : 1)>{}, [&](auto occ) {
                    constexpr int OO = decltype(occ)::value;
                    if (oc == OO) {
                        static_for(std::make_integer_sequence<int, len>{}, [&](auto uc) {
                            constexpr int u = decltype(uc)::value;
                            constexpr int i = OO + len - 1 - u;
                            if constexpr (i + 1 < Q)
                                step(z, w, std::integral_constant<int, i>{}, t0 + u, penb, kx);
                        });
                    }
                });
                t0 += len;
            }
        });
    }
    return ok;
}

// Consumers of the paired walk.  Items: the Q free variables; the fixed
// variables above 5 outside the pair's front sets; variables 1..5 in groups
// of 16 pair lanes (those without the variable in F); variable 0 (x only).
// Pair lane l reads its column from record 2c + (l >> 4) at CTA lanes
// 2 (l & 15) and 2 (l & 15) + 1 (one 8-byte load).  The warp takes items
// first, first + stride, ...; returns the number of items of the pair, or -1
// when a wait expired.
template <int Q, bool KB>
__device__ __forceinline__ int consume_pair(const WalkArgs<float>& a, const float* __restrict__ rec0,
                                            const float* __restrict__ rec1, const float4* tape,
                                            uint64_t* full, unsigned par, int lane, int first,
                                            int stride, uint64_t pc) {
    constexpr int LQ = Q * (Q + 1) / 2;
    constexpr int H = split_levels(Q);
    const int nu = (a.k - 6) - __popcll(pc);  // fixed variables above 5 outside F
    const int nitems = Q + nu + 3 + 1;
    char* out = reinterpret_cast<char*>(a.out);
    const float lnn = a.lam;
    // penalty bases of the two sub-walks, rounded as the single walk rounds them
    auto pen2 = [&](uint64_t Fx) {
        const float c0 = float(__popcll(Fx));
        return make_float2(fmaf(c0, lnn, -a.nlnn), fmaf(c0 + 1.f, lnn, -a.nlnn));
    };
    // entry ix (of a record's per-lane layout, CTA lane 0) of pair lane pl: x and y
    auto ld2 = [&](size_t ix, int pl, bool on, int site) {
        const float* r = (pl >> 4) ? rec1 : rec0;
        const size_t e = ix + 2 * (size_t)(pl & 15);
        return (on && GBN_IN(a.chk, site, e + 1, a.leaf_stride))
                   ? *reinterpret_cast<const float2*>(r + e)
                   : make_float2(0.f, 0.f);
    };
    for (int it = first; it < nitems; it += stride) {
        // the item's column, then one replay call site (its code is the walk's size)
        float2 z[Q], cres = make_float2(0.f, 0.f);
        int pl = lane, jj = Q, sh = a.k - 1;
        unsigned on_xy = 1u, on_x = 0u;
        size_t slot;  // table element of x's prefix-0 family
        if (it < Q) {  // free variable j
            const int j = it;
#pragma unroll
            for (int e = 0; e < Q; ++e) z[e] = ld2((size_t)(j * (j + 1) / 2 + e) * 32, pl, e <= j, 330);
            jj = j;
            sh = a.k;
            slot = ((size_t)(a.k + j) << (a.m - 1)) + ((pc << 6) | ((uint64_t)pl << 1));
        } else {  // a fixed variable v outside the front sets
            int v, rs;  // rs: the variable's slot in the (compact) leaf record
            bool on = true;
            if (it < Q + nu) {  // above 5: record 0 (variable 5 outside F) holds it one slot up
                v = 6 + nth_zero_bit(pc, it - Q);
                rs = 6 - (pl >> 4) + (it - Q);
            } else if (it < Q + nu + 3) {  // 1..5, 16 pair lanes each (bit v-1 of pl clear)
                const int j = it - Q - nu;
                const int uu = lane >> 4, sub = lane & 15;
                v = 1 + 2 * j + uu;
                on = v <= 5;
                const int b = on ? v - 1 : 0;
                pl = (sub & ((1 << b) - 1)) | ((sub >> b) << (b + 1));
                if (!on) v = 1;
                on_xy = on ? 1u : 0u;
                rs = v;
            } else {  // variable 0: a child of x only
                v = 0;
                rs = 0;
                on_xy = 0u;
                on_x = 1u;
            }
            const size_t b0 = (size_t)32 * (LQ + rs * (Q + 1));
#pragma unroll
            for (int e = 0; e < Q; ++e) z[e] = ld2(b0 + (size_t)e * 32, pl, on, 331);
            cres = ld2(b0 + (size_t)Q * 32, pl, on, 331);
            const uint64_t Fx = (pc << 6) | ((uint64_t)pl << 1);
            const uint64_t lowmask = (1ull << v) - 1ull;
            slot = ((size_t)v << (a.m - 1)) + ((Fx & lowmask) | ((Fx >> (v + 1)) << v));
        }
        const uint64_t Fx = (pc << 6) | ((uint64_t)pl << 1);
        const bool ok = replay_pair<Q, H, KB>(a, tape, full, par, z, cres, pl, jj, sh,
                                              out + slot * 4, pen2(Fx), on_xy, on_x,
                                              KB ? a.kmax - __popcll(Fx) : 0);
        if (!ok) return -1;
    }
    return nitems;
}
#endif

// Consumers: the CTA's columns; the warp takes items first, first + stride, ...
// and returns the CTA's item count (-1 when a wait expired).
//   items [0, Q)             free variable j = it, every lane;
//   items [Q, Q + nu)        the fixed variables above the lowest W outside F_hi;
//   items [Q + nu, + n5)     the lowest W variables, 32/g per item, g = 2^(W-1)
//                            lanes each (only sub-walks without it in F).
template <typename T, int Q, bool COV>
__device__ __forceinline__ int consume(const WalkArgs<T>& a, const T* __restrict__ rec,
                                       const typename Vec2T<T>::type* tape, uint64_t* full,
                                       unsigned par, int lane, int first, int stride, uint64_t cta,
                                       uint64_t Fhi) {
    constexpr int LQ = Q * (Q + 1) / 2;
    const int nu = (a.k - a.W) - __popcll(cta);
    const int g = a.W >= 1 ? (a.lanes >> 1) : 1;
    const int vpi = 32 / g;
    const int n5 = a.W >= 1 ? (a.W + vpi - 1) / vpi : 0;
    const int nitems = Q + nu + n5;
    GBN_TIMER_DECL
    for (int it = first; it < nitems; it += stride) {
        T z[Q];
        int ell = lane, jj, sh;
        bool on;
        OutT<T, COV>* base;
        T cres = T(0);
        if (it < Q) {  // free variable j: column j of the root block
            const int j = it;
            on = lane < a.lanes;
#pragma unroll
            for (int e = 0; e < Q; ++e) {
                const size_t ix = (size_t)(j * (j + 1) / 2 + e) * 32 + lane;
                z[e] = (on && e <= j && GBN_IN(a.chk, 323, ix, a.leaf_stride)) ? rec[ix] : T(0);
            }
            jj = j;
            sh = a.k;
            base = reinterpret_cast<OutT<T, COV>*>(a.out) + ((size_t)(a.k + j) << (a.m - 1)) +
                   (Fhi | (uint64_t)lane);
        } else {  // fixed variable v outside the front set
            int v, rs;  // rs: the variable's slot in the (compact) leaf record
            if (it < Q + nu) {
                v = a.W + nth_zero_bit(cta, it - Q);
                rs = a.W + (it - Q);
                on = lane < a.lanes;
            } else {
                const int j = it - Q - nu;
                const int uu = lane / g, sub = lane % g;
                v = j * vpi + uu;
                on = v < a.W;
                ell = on ? ((sub & ((1 << v) - 1)) | ((sub >> v) << (v + 1))) : 0;
                if (!on) v = 0;
                rs = v;
            }
            const size_t b0 = (size_t)32 * (LQ + rs * (Q + 1));
#pragma unroll
            for (int e = 0; e < Q; ++e) {
                const size_t ix = b0 + e * 32 + ell;
                z[e] = (on && GBN_IN(a.chk, 321, ix, a.leaf_stride)) ? rec[ix] : T(0);
            }
            {
                const size_t ix = b0 + Q * 32 + ell;
                cres = (on && GBN_IN(a.chk, 322, ix, a.leaf_stride)) ? rec[ix] : T(0);
            }
            const uint64_t F = Fhi | (uint64_t)ell;
            const uint64_t lowmask = (1ull << v) - 1ull;
            jj = Q;
            sh = a.k - 1;
            base = reinterpret_cast<OutT<T, COV>*>(a.out) + ((size_t)v << (a.m - 1)) +
                   (size_t)((F & lowmask) | ((F >> (v + 1)) << v));
        }
        const int nF = __popcll(Fhi | (uint64_t)ell);
        const T penb = fma(T(nF), a.lam, -a.nlnn);
        const int kr = a.kmax - nF;
        bool ok;
#ifdef GBN_Q
        if constexpr (split_levels(Q) > 0)
            ok = replay_split<T, Q, split_levels(Q), COV>(a, tape, full, par, z, cres, ell, jj, sh,
                                                        base, penb, on, kr);
        else
#endif
            ok = replay<T, Q, COV>(a, tape, full, par, z, cres, ell, jj, sh, base, penb, on, kr);
        if (!ok) return -1;
    }
    GBN_TIMER_FLUSH(a.timing, 1)
    return nitems;
}

}  // namespace gbn

// The kernel exists only in the translation unit compiled for one Q
// (walk_inst.cu with -DGBN_Q=...).
#ifdef GBN_Q
namespace gbn {

constexpr int kMaxConsumerWarps = 8;
// Resident CTAs per SM the FP32 walk's register allocation must allow at 288
// threads: five up to Q = 7 (40 registers), three at Q = 8 (the tape's shared
// memory allows no more); the FP64 walk is not bounded.
template <typename T, int Q>
constexpr int walk_min_blocks() {
    return std::is_same<T, float>::value ? (Q <= 7 ? 5 : (Q == 8 ? 3 : 1)) : 1;
}

template <typename T, int Q, bool COV>
__device__ __forceinline__ void walk_body(const WalkArgs<T>& a, uint64_t cta) {
    extern __shared__ __align__(16) unsigned char smem[];
    using S = Smem<T, Q>;
    static_assert(Q == GBN_Q, "one Q per translation unit");
    static_assert(Q <= 9, "the whole tape is kept in shared memory");
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + S::off_bar);
    if (threadIdx.x < S::chunks) mbar_init(&full[threadIdx.x], 1);
    for (int c = threadIdx.x + blockDim.x; c < S::chunks; c += blockDim.x) mbar_init(&full[c], 1);
    __syncthreads();
    // cta: this launch's CTA (leaf record); g: its global index (front set bits)
    const uint64_t g = cta + (uint64_t)a.cta0;
    if (__popcll(g) > a.kmax) return;  // every family of these sub-walks has too many parents
    const uint64_t Fhi = g << a.W;
    const T* rec = a.leaves + (size_t)cta * a.leaf_stride;
    if (warp == 0)
        produce<T, Q>(a, c_steps, rec, smem + S::off_tape, full, lane, lane < a.lanes);
    else
        consume<T, Q, COV>(a, rec, reinterpret_cast<const typename Vec2T<T>::type*>(smem + S::off_tape),
                           full, 0u, lane, warp - 1, a.n_cwarps, g, Fhi);
}

template <typename T, int Q, bool COV>
__global__ void __launch_bounds__(32 * (1 + kMaxConsumerWarps), walk_min_blocks<T, Q>())
    walk_kernel(const WalkArgs<T> a) {
    walk_body<T, Q, COV>(a, blockIdx.x);
}

// A batch: the block finds its dataset through the prefix of sub-walk CTAs
// and copies that dataset's arguments.
template <typename T, int Q, bool COV>
__global__ void __launch_bounds__(32 * (1 + kMaxConsumerWarps)) walk_kernel_b(const BatchView v) {
    int64_t local;
    const int d = batch_locate(v, v.cta_prefix, v.cta_pos, blockIdx.x, local);
    const WalkArgs<T> a = static_cast<const WalkArgs<T>*>(v.walk_args)[d];
    walk_body<T, Q, COV>(a, (uint64_t)local);
}

// The paired FP32 walk: block c runs the sub-walks of roots CTAs 2c and 2c+1
// (W = 5).  Warps 0 and 1 produce the two halves of the tape, the others
// consume both sub-walks at once.
constexpr int kPairConsumerWarps = 8;
constexpr int kPairThreads = 32 * (2 + kPairConsumerWarps);
constexpr size_t kPairMaxSmem = 160 * 1024;  // the tape of Q = 9 does not fit
// pc: the pair of this launch (leaf records 2 pc, 2 pc + 1).  GEN, the
// general form, serves a bounded in-degree (KB stores) and shards: the pair's
// global index (its front set bits) is pc + cta0 / 2, cta0 being even.  The
// plain form (the whole table, no bound) takes pc itself, which the compiler
// can re-read from the block index instead of keeping it in a register.
template <int Q, bool GEN>
__device__ __forceinline__ void walk_pair_body(const WalkArgs<float>& a, uint64_t pc) {
    extern __shared__ __align__(16) unsigned char smem[];
    using S = SmemP<Q>;
    static_assert(Q == GBN_Q, "one Q per translation unit");
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + S::off_bar);
    for (int c = threadIdx.x; c < S::chunks; c += blockDim.x) mbar_init(&full[c], 2);
    uint64_t gpc = pc;
    if constexpr (GEN) gpc += (uint64_t)a.cta0 >> 1;
    {  // the elements in use of the two compact records (CTA 2 gpc + h: nu_h slots above 5)
        constexpr int LQ = Q * (Q + 1) / 2;
        const int nu0 = (a.k - 5) - __popcll(2 * gpc);
        const float* r0 = a.leaves + (size_t)(2 * pc) * a.leaf_stride;
        prefetch_l2(r0, (size_t)(LQ + (5 + nu0) * (Q + 1)) * 32 * sizeof(float), threadIdx.x,
                    blockDim.x);
        prefetch_l2(r0 + a.leaf_stride, (size_t)(LQ + (4 + nu0) * (Q + 1)) * 32 * sizeof(float),
                    threadIdx.x, blockDim.x);
    }
    __syncthreads();
    if constexpr (GEN) {
        if (__popcll(gpc) > a.kmax) return;  // every family here has too many parents
    }
    const float* rec0 = a.leaves + (size_t)(2 * pc) * a.leaf_stride;
    const float* rec1 = rec0 + a.leaf_stride;
    if (warp < 2)
        produce<float, Q, true>(a, c_steps, warp ? rec1 : rec0, smem + S::off_tape, full, lane,
                                true, pair_tape_word(warp, lane));
    else
        consume_pair<Q, GEN>(a, rec0, rec1, reinterpret_cast<const float4*>(smem + S::off_tape),
                             full, 0u, lane, warp - 2, (int)(blockDim.x >> 5) - 2, gpc);
}

template <int Q, bool GEN>
__global__ void __launch_bounds__(kPairThreads, Q >= 8 ? 1 : 3) walk_kernel_pair(const WalkArgs<float> a) {
    walk_pair_body<Q, GEN>(a, blockIdx.x);
}

// A batch in which every dataset takes the paired walk (every CTA count is
// even, so pair g of the batch is walk CTA 2g): the block finds its dataset
// through the prefix of walk CTAs and copies that dataset's arguments.
template <int Q>
__global__ void __launch_bounds__(kPairThreads, Q >= 8 ? 1 : 3) walk_kernel_pair_b(const BatchView v) {
    int64_t local;
    const int d = batch_locate(v, v.cta_prefix, v.cta_pos, 2 * (int64_t)blockIdx.x, local);
    const WalkArgs<float> a = static_cast<const WalkArgs<float>*>(v.walk_args)[d];
    walk_pair_body<Q, false>(a, (uint64_t)local >> 1);
}

// Whether a launch takes the paired walk: FP32 scores, full warps of
// sub-walks (W = 5) and an even number of roots CTAs.
template <typename T, int Q, bool COV>
constexpr bool pair_walk_compiled() {
    return std::is_same<T, float>::value && !COV && SmemP<Q>::bytes <= kPairMaxSmem;
}

// ------------------------------------------------- resident blocks (cached)
// SMs x resident blocks per SM of a persistent kernel at a launch shape, found
// once per (kernel, device, threads, shared memory): the occupancy query costs
// more host time than a launch, and a small call's kernels are short enough for
// host time to show.  The first query for a kernel on a device also sets its
// dynamic shared-memory limit to smem_max (at least any launch's).
struct ResidentEntry {
    const void* fn;
    int dev, threads;
    size_t smem;
    int blocks;
};

template <typename K>
int resident_blocks(K* kernel, int threads, size_t smem, size_t smem_max, int* blocks) {
    static std::mutex mu;
    static std::vector<ResidentEntry> cache;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return GBN_ERR_CUDA;
    const void* fn = reinterpret_cast<const void*>(kernel);
    std::lock_guard<std::mutex> lock(mu);
    bool limit_set = false;
    for (const ResidentEntry& e : cache) {
        if (e.fn != fn || e.dev != dev) continue;
        limit_set = true;
        if (e.threads == threads && e.smem == smem) {
            *blocks = e.blocks;
            return GBN_OK;
        }
    }
    int sms = 0, per_sm = 0;
    if ((!limit_set && cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)smem_max) != cudaSuccess) ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) !=
            cudaSuccess)
        return GBN_ERR_CUDA;
    if (per_sm < 1) return GBN_ERR_CUDA;
    cache.push_back(ResidentEntry{fn, dev, threads, smem, sms * per_sm});
    *blocks = sms * per_sm;
    return GBN_OK;
}

// ---------------------------------------------------------------- ring walk
// A persistent form of the FP32 walk.  A unit is one roots CTA's 32
// sub-walks (PAIR: two neighbouring ones, as in the paired walk); block b takes
// units b, b + gridDim.x, ... and keeps a ring of two tapes in shared memory.
// The producer warp(s) write the tape of the block's j-th unit into slot j mod 2
// as soon as the consumers have released unit j - 2, so while the consumers
// replay one unit the next unit's tape is being written: they do not wait for
// a producer that starts when they do.  The consumer warps take the items of
// successive units as one round-robin stream, so no warp idles at a unit's end
// while another finishes a third item.
template <int Q, bool PAIR>
struct RingSmem {
    static constexpr int N = StepTab<Q>::N;
    static constexpr int chunks = (N + kChunk - 1) / kChunk;
    static constexpr size_t tape_bytes = (size_t)N * 32 * (PAIR ? 16 : 8);
    static constexpr size_t off_full = 2 * tape_bytes;                       // [2][chunks]
    static constexpr size_t off_empty = off_full + 2 * (size_t)chunks * 8;   // [2]
    static constexpr size_t bytes = off_empty + 2 * 8;
    // resident blocks per SM: what the shared memory allows (228 KB per SM,
    // 1 KB reserved per block), at most five (three for the paired form, whose
    // consumers hold two families per register pair)
    static constexpr int cap = PAIR ? 3 : 5;
    static constexpr int per_sm =
        (233472 / (bytes + 1024)) < cap ? (int)(233472 / (bytes + 1024)) : cap;
};
constexpr int kRingConsumerWarps = 8;
template <int Q, bool PAIR>
constexpr int ring_threads() { return 32 * ((PAIR ? 2 : 1) + kRingConsumerWarps); }
// compiled where at least two blocks fit on an SM
template <int Q, bool PAIR>
constexpr bool ring_walk_compiled() { return RingSmem<Q, PAIR>::per_sm >= 2; }

template <int Q, bool PAIR>
__global__ void __launch_bounds__(ring_threads<Q, PAIR>(),
                                  RingSmem<Q, PAIR>::per_sm < 1 ? 1 : RingSmem<Q, PAIR>::per_sm)
    walk_ring_kernel(const WalkArgs<float> a, int64_t n_units) {
    extern __shared__ __align__(16) unsigned char smem[];
    using S = RingSmem<Q, PAIR>;
    static_assert(Q == GBN_Q, "one Q per translation unit");
    constexpr int NP = PAIR ? 2 : 1;  // producer warps
    constexpr int NC = kRingConsumerWarps;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + S::off_full);
    uint64_t* empty = reinterpret_cast<uint64_t*>(smem + S::off_empty);
    for (int c = threadIdx.x; c < 2 * S::chunks; c += blockDim.x) mbar_init(&full[c], NP);
    if (threadIdx.x < 2) mbar_init(&empty[threadIdx.x], NC);
    __syncthreads();
    if (warp < NP) {
        int j = 0;
        for (int64_t u = blockIdx.x; u < n_units; u += gridDim.x, ++j) {
            const int s = j & 1;
            if (j >= 2 && !warp_wait(&empty[s], ((j - 2) >> 1) & 1, a.watchdog_ns, a.status))
                return;
            unsigned char* tb = smem + s * S::tape_bytes;
            uint64_t* fb = full + s * S::chunks;
            if constexpr (PAIR) {
                const float* rec = a.leaves + (size_t)(2 * u + warp) * a.leaf_stride;
                produce<float, Q, true>(a, c_steps, rec, tb, fb, lane, true,
                                        pair_tape_word(warp, lane));
            } else {
                const float* rec = a.leaves + (size_t)u * a.leaf_stride;
                produce<float, Q>(a, c_steps, rec, tb, fb, lane, lane < a.lanes);
            }
        }
    } else {
        const int cw = warp - NP;
        int off = 0, j = 0;  // off: items handed out so far, mod NC
        for (int64_t u = blockIdx.x; u < n_units; u += gridDim.x, ++j) {
            const int s = j & 1;
            const unsigned par = (unsigned)(j >> 1) & 1u;
            const int first = ((cw - off) % NC + NC) % NC;
            const unsigned char* tb = smem + s * S::tape_bytes;
            uint64_t* fb = full + s * S::chunks;
            int n;
            if constexpr (PAIR) {
                const float* rec0 = a.leaves + (size_t)(2 * u) * a.leaf_stride;
                n = consume_pair<Q, false>(a, rec0, rec0 + a.leaf_stride,
                                           reinterpret_cast<const float4*>(tb), fb, par, lane,
                                           first, NC, (uint64_t)u);
            } else {
                const float* rec = a.leaves + (size_t)u * a.leaf_stride;
                n = consume<float, Q, false>(a, rec, reinterpret_cast<const float2*>(tb), fb, par,
                                             lane, first, NC, (uint64_t)u, (uint64_t)u << a.W);
            }
            if (n < 0) return;
            off = (off + n) % NC;
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[s]);  // this warp is done with the slot
        }
    }
}

template <int Q, bool PAIR>
int launch_walk_ring(const WalkArgs<float>& a, int64_t n_units, cudaStream_t stream) {
    const size_t smem = RingSmem<Q, PAIR>::bytes;
    const int threads = ring_threads<Q, PAIR>();
    int resident = 0;
    const int rc = resident_blocks(walk_ring_kernel<Q, PAIR>, threads, smem, smem, &resident);
    if (rc != GBN_OK) return rc;
    const int64_t blocks = std::min<int64_t>(n_units, (int64_t)resident);
    return launch_rc(launch_plain(walk_ring_kernel<Q, PAIR>, dim3((unsigned)blocks), dim3(threads),
                                  smem, stream, a, n_units));
}

// Which FP32 score walk a launch takes (full warps of sub-walks, W = 5):
// 0 the per-CTA walk, 1 the paired walk, 2 the ring walk, 3 the paired ring.
// Measured at m = 26: the paired ring is the fastest at Q = 6; at Q = 7 its
// two tapes leave room for one block per SM and the paired walk is faster.
template <int Q>
constexpr int fp32_walk_form() {
    return (Q <= 6 && ring_walk_compiled<Q, true>()) ? 3 : 1;
}

template <int Q, bool GEN>
int launch_walk_pair(const WalkArgs<float>& a, int64_t n_cta, cudaStream_t stream) {
    const size_t smem_p = SmemP<Q>::bytes;
    if (cudaFuncSetAttribute(walk_kernel_pair<Q, GEN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem_p) != cudaSuccess)
        return GBN_ERR_CUDA;
    const int ncw = a.n_cwarps < kPairConsumerWarps ? a.n_cwarps : kPairConsumerWarps;
    return launch_rc(launch_plain(walk_kernel_pair<Q, GEN>, dim3((unsigned)(n_cta / 2)),
                                  dim3(32 * (2 + ncw)), smem_p, stream, a));
}

// n_cta: the sub-walk CTAs of this launch (a.cta0 is the global index of the
// first; even whenever n_cta is).
template <typename T, int Q, bool COV>
int launch_walk_q(const WalkArgs<T>& a, int64_t n_cta, cudaStream_t stream) {
    const size_t smem = Smem<T, Q>::bytes;
    if (a.n_cwarps < 1 || a.n_cwarps > kMaxConsumerWarps) return GBN_ERR_Q;
    if (n_cta < 1) return GBN_OK;
    // the general forms for a bounded in-degree or a shard of the table
    const bool general = a.kmax < a.m - 1 || a.cta0 != 0;
    if constexpr (std::is_same<T, float>::value && !COV) {
        constexpr int form = fp32_walk_form<Q>();
        const bool full_warps = a.W == 5 && a.lanes == 32;
        const bool pairs = full_warps && n_cta >= 2 && n_cta % 2 == 0 && a.cta0 % 2 == 0;
        if constexpr (form == 3) {
            if (pairs && !general) return launch_walk_ring<Q, true>(a, n_cta / 2, stream);
        }
        if constexpr (form >= 2) {
            if (full_warps && !general) return launch_walk_ring<Q, false>(a, n_cta, stream);
        }
        if constexpr (pair_walk_compiled<T, Q, COV>()) {
            if (pairs) {
                if (general) return launch_walk_pair<Q, true>(a, n_cta, stream);
                if (form == 1) return launch_walk_pair<Q, false>(a, n_cta, stream);
            }
        }
    }
    if (cudaFuncSetAttribute(walk_kernel<T, Q, COV>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess)
        return GBN_ERR_CUDA;
    return launch_rc(launch_plain(walk_kernel<T, Q, COV>, dim3((unsigned)n_cta),
                                  dim3(32 * (1 + a.n_cwarps)), smem, stream, a));
}

template <typename T, int Q, bool COV>
int launch_walk_batched_q(const BatchView& v, int64_t total_cta, int n_cwarps, cudaStream_t stream) {
    const size_t smem = Smem<T, Q>::bytes;
    if (n_cwarps < 1 || n_cwarps > kMaxConsumerWarps) return GBN_ERR_Q;
    if constexpr (pair_walk_compiled<T, Q, COV>()) {
        if (v.pairs && total_cta % 2 == 0) {
            const size_t smem_p = SmemP<Q>::bytes;
            if (cudaFuncSetAttribute(walk_kernel_pair_b<Q>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem_p) != cudaSuccess)
                return GBN_ERR_CUDA;
            const int ncw = n_cwarps < kPairConsumerWarps ? n_cwarps : kPairConsumerWarps;
            return launch_rc(launch_plain(walk_kernel_pair_b<Q>, dim3((unsigned)(total_cta / 2)),
                                          dim3(32 * (2 + ncw)), smem_p, stream, v));
        }
    }
    if (cudaFuncSetAttribute(walk_kernel_b<T, Q, COV>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess)
        return GBN_ERR_CUDA;
    return launch_rc(launch_plain(walk_kernel_b<T, Q, COV>, dim3((unsigned)total_cta),
                                  dim3(32 * (1 + n_cwarps)), smem, stream, v));
}

}  // namespace gbn
#endif

// One instantiation per (scalar type, Q, coverage), each compiled as its own
// object from walk_inst.cu so that the build runs in parallel.
#define GBN_WALK_INST_NAME(T, Q, COV) gbn_launch_walk_##T##_q##Q##_c##COV
#define GBN_WALK_DECL(T, Q, COV) \
    int GBN_WALK_INST_NAME(T, Q, COV)(const gbn::WalkArgs<T>& a, int64_t n_cta, cudaStream_t s)
#define GBN_WALK_B_INST_NAME(T, Q, COV) gbn_launch_walk_b_##T##_q##Q##_c##COV
#define GBN_WALK_B_DECL(T, Q, COV)                                                          \
    int GBN_WALK_B_INST_NAME(T, Q, COV)(const gbn::BatchView& v, int64_t total_cta, int nw, \
                                        cudaStream_t s)

// Roots of the sub-walks: the parallel split of Sec. 6 (Algorithm 2).
//
// A sub-walk is fixed by its front set F, a subset of the k fixed variables:
// its ordering is [F, L, B] with L the Q free variables and B the fixed
// variables outside F, and it runs Upsilon(Q) shifted by |F|.  The walk only
// rotates rows |F|+1 .. |F|+Q, so a root is fully described by
//   * the Q x Q block of R for L after projecting out F (the "L block"), and
//   * for every v in B: the Q entries of v's column in those rows and the
//     residual C_v = RSS(v | F u L) below them.
//
// The roots are built as a binary tree over the fixed variables (the same
// recursion as Algorithm 2, one level per fixed variable), starting from R0
// whose column order puts the fixed variables first.  At each level the first
// undecided variable either joins F -- drop the first row, since the rest of
// R is already the factor of the remaining columns after projecting it out --
// or joins B -- its column leaves the triangle, the remaining upper-Hessenberg
// block is re-triangularised with one Givens rotation per row pair, the
// deleted column is carried along (rotated with the rest) and the row that
// falls off the bottom is added to its residual.  Lane l owns column l of R0
// (plan order) throughout: columns never move, a decision only changes the
// lane's role (undecided / in F / carried in B) and drops one row.
//
// Two kernels, each with a small instruction footprint:
//   * top: one warp per 4 walk CTAs follows their shared path through the
//     top levels and enumerates their last 2 top levels depth first, on a
//     node kept in shared memory (rows addressed through a moving first-row
//     offset, a compact loop per rotation), storing each CTA's node: the Q + W
//     live rows of every column, the residuals and the carried-column mask
//     (the batched form takes one CTA per warp);
//   * leaves: one warp per walk CTA loads that node into registers (at most
//     16 rows) and enumerates the 2^W leaves of the last W levels depth first,
//     saving each level's node in shared memory to restart from it, and
//     writes every leaf, lane-interleaved, into the record the walk reads.
#include <math.h>

#include <type_traits>
#include <utility>

#include "gbn_internal.cuh"

namespace gbn {
namespace {

constexpr int kDfsRows = 16;  // register rows of the depth-first nodes (Q + W <= 16)
constexpr int kTopWarps = 4;  // warps per block of the batched top kernel (one CTA root each)
constexpr int kDfsWarps = 4;  // warps per block of the leaf kernel (one walk CTA each)

// Compile-time loop: f(integral_constant<int, i>) for i in the sequence, so
// that register arrays are only ever indexed by constants.
template <int... Is, typename F>
__device__ __forceinline__ void sfor(std::integer_sequence<int, Is...>, F&& f) {
    (f(std::integral_constant<int, Is>{}), ...);
}

__device__ __forceinline__ float rsqrt_t(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsqrt_t(double x) { return rsqrt(x); }

template <typename T>
__device__ __forceinline__ void givens_cs(T a, T b, T& c, T& s) {
    const T r2 = fma(a, a, b * b);  // explicit fma: every instance rounds alike
    c = T(1);
    s = T(0);
    if (r2 > T(0)) {
        const T inv = rsqrt_t(r2);
        c = a * inv;
        s = b * inv;
    }
}

// Size of a stored node with `rows` rows: the rows, the residuals, the
// carried mask (one element of T, read as a word), all lane-interleaved.
__host__ __device__ __forceinline__ size_t node_elems(int rows) { return (size_t)(rows + 2) * 32; }

template <typename T>
__device__ __forceinline__ unsigned* mask_of(T* node, int rows) {
    return reinterpret_cast<unsigned*>(node + (size_t)(rows + 1) * 32);
}

// The variable of R0 column (lane) `lane`: the plan order is
// [W..k-1, W-1..0, free variables].
__device__ __forceinline__ int var_of_lane(const Plan& p, int lane) {
    const int kw = p.k - p.W;
    return lane < kw ? lane + p.W : (lane < p.k ? p.W - 1 - (lane - kw) : lane);
}

// Compact leaf records: the fixed variables above the lowest W that are in the
// CTA's front set (the same for all its leaves) are never read by the walk, so
// they get no slot.  Slot of fixed variable lane `lane` in a leaf whose carried
// mask is `carried`: the lowest W variables keep slots 0 .. W-1; a variable
// above them outside the front set takes slot W + the number of such variables
// below it (the order in which the walk's items take them).
__device__ __forceinline__ int rec_slot(const Plan& p, int lane, unsigned carried) {
    const int kw = p.k - p.W;
    return lane < kw ? p.W + __popc(carried & ((1u << lane) - 1u)) : var_of_lane(p, lane);
}
// Record elements (per lane) in use: the L block and W + nu slots of Q + 1.
__device__ __forceinline__ int rec_rows(const Plan& p, unsigned carried) {
    const int kw = p.k - p.W;
    const int nu = __popc(carried & ((1u << kw) - 1u));
    return p.Q * (p.Q + 1) / 2 + (p.W + nu) * (p.Q + 1);
}

// ------------------------------------------------------------- top levels

// A node in shared memory: live rows r0 .. r0 + rows - 1 of S (row r of the
// lane's column at S[r * 32 + lane]), the carried residuals and mask.
template <typename T>
struct TopNode {
    int r0, rows;
    T C;
    unsigned carried;
};

template <typename T>
__device__ __forceinline__ void top_load(const double* __restrict__ R0, const Plan& p,
                                         unsigned long long* chk, T* S, TopNode<T>& nd) {
    const int lane = threadIdx.x & 31, m = p.m;
    for (int r = 0; r < 32; ++r)
        S[r * 32 + lane] = (r < m && lane < m && GBN_IN(chk, 231, r * m + lane, m * m))
                               ? (T)R0[r * m + lane]
                               : T(0);
    __syncwarp();
    nd.r0 = 0;
    nd.rows = m;
    nd.C = T(0);
    nd.carried = 0u;
}

// Decide fixed variable f (the node's first live column): include drops the
// first live row; exclude carries column f and re-triangularises the rest.
template <typename T>
__device__ __forceinline__ void top_decide(T* S, TopNode<T>& nd, int f, bool include) {
    const int lane = threadIdx.x & 31;
    if (include) {
        ++nd.r0;
        --nd.rows;
        return;
    }
    nd.carried |= 1u << f;
    for (int j = 0; j + 1 < nd.rows; ++j) {
        const int ra = nd.r0 + j, piv = f + 1 + j;
        const T a = S[ra * 32 + piv], b = S[(ra + 1) * 32 + piv];
        const T x = S[ra * 32 + lane], y = S[(ra + 1) * 32 + lane];
        T c, s;
        givens_cs(a, b, c, s);
        __syncwarp();
        S[ra * 32 + lane] = fma(c, x, s * y);
        S[(ra + 1) * 32 + lane] = fma(c, y, -s * x);
        __syncwarp();
    }
    const T yb = S[(nd.r0 + nd.rows - 1) * 32 + lane];  // the bottom row falls off
    if ((nd.carried >> lane) & 1u) nd.C = fma(yb, yb, nd.C);
    --nd.rows;
}

// rows == Q + W: store the node as walk CTA cta's root
template <typename T>
__device__ __forceinline__ void top_store(const T* S, const TopNode<T>& nd, T* __restrict__ top,
                                          uint64_t cta) {
    const int lane = threadIdx.x & 31;
    T* out = top + (size_t)cta * node_elems(nd.rows);
    for (int r = 0; r < nd.rows; ++r) out[(size_t)r * 32 + lane] = S[(nd.r0 + r) * 32 + lane];
    out[(size_t)nd.rows * 32 + lane] = nd.C;
    if (lane == 0) *mask_of(out, nd.rows) = nd.carried;
}

// One walk CTA's root: its path through the k - W top levels (the bits of
// its global index g), stored at slot `local` of this call's nodes.
template <typename T>
__device__ __forceinline__ void top_body(const double* __restrict__ R0, const Plan& p,
                                         T* __restrict__ top, unsigned long long* chk,
                                         uint64_t g, uint64_t local,
                                         T* S /* 32 x 32, [row * 32 + lane] */) {
    TopNode<T> nd;
    top_load(R0, p, chk, S, nd);
    for (int f = 0; f < p.k - p.W; ++f) top_decide(S, nd, f, ((g >> f) & 1ull) != 0);
    top_store(S, nd, top, local);
}

// The roots of 2^d walk CTAs at once: they share the path through the first
// P = k - W - d top levels (the low P bits of the CTA index) and differ in
// the last d, which one warp enumerates depth first, so every node of the
// subtree is built once (a path per CTA builds the shared part 2^d times).
// Level t's node is saved in its stack slot before the include branch and
// restored for the exclude branch; the results are bit-identical to top_body.
// The chains of rotations are latency-bound, so d trades work for parallel
// warps: at m = 26 the kernel took 85.5 us with d = 0, 43.7 us with d = 2 and
// 72.7 us with d = 4.
constexpr int kTopDfsLevels = 2;
constexpr int kTopDfsWarps = 2;

template <typename T, int L>
struct TopDfs {
    __device__ static __forceinline__ void run(T* S, T* stack, const TopNode<T>& nd, int f,
                                               int nlev, uint64_t cta, T* __restrict__ top) {
        if constexpr (L < kTopDfsLevels) {
            if (L < nlev) {
                const int lane = threadIdx.x & 31;
                T* slot = stack;  // this level's slot; deeper levels follow it
                for (int r = 0; r < nd.rows; ++r) slot[r * 32 + lane] = S[(nd.r0 + r) * 32 + lane];
                __syncwarp();
                T* deeper = stack + (size_t)nd.rows * 32;
                TopNode<T> c = nd;
                top_decide(S, c, f, true);
                TopDfs<T, L + 1>::run(S, deeper, c, f + 1, nlev, cta | (1ull << f), top);
                __syncwarp();
                for (int r = 0; r < nd.rows; ++r) S[(nd.r0 + r) * 32 + lane] = slot[r * 32 + lane];
                __syncwarp();
                c = nd;
                top_decide(S, c, f, false);
                TopDfs<T, L + 1>::run(S, deeper, c, f + 1, nlev, cta, top);
                return;
            }
        }
        top_store(S, nd, top, cta);
        __syncwarp();
    }
};

// Levels enumerated depth first by one top warp, and the stack it needs
// (elements: each level's saved rows).
__host__ __device__ __forceinline__ int top_dfs_levels(const Plan& p) {
    const int D = p.k - p.W;
    return D < kTopDfsLevels ? D : kTopDfsLevels;
}
__host__ __device__ __forceinline__ size_t top_dfs_stack_elems(const Plan& p) {
    const int nlev = top_dfs_levels(p);
    const int rows0 = p.m - (p.k - p.W - nlev);  // live rows when the subtree starts
    size_t e = 0;
    for (int t = 0; t < nlev; ++t) e += (size_t)(rows0 - t) * 32;
    return e;
}

template <typename T>
__device__ __forceinline__ void top_dfs_body(const double* __restrict__ R0, const Plan& p,
                                             T* __restrict__ top, unsigned long long* chk,
                                             uint64_t g, T* S, T* stack) {
    const int nlev = top_dfs_levels(p);
    const int P = p.k - p.W - nlev;
    TopNode<T> nd;
    top_load(R0, p, chk, S, nd);
    for (int f = 0; f < P; ++f) top_decide(S, nd, f, ((g >> f) & 1ull) != 0);
    TopDfs<T, 0>::run(S, stack, nd, P, nlev, g, top);
}

// ------------------------------------------------------------- last W levels

// Include: the front variable joins F.  Drop row 0 (all lanes shift their rows).
template <typename T>
__device__ __forceinline__ void drop_first_row(T (&M)[kDfsRows]) {
    sfor(std::make_integer_sequence<int, kDfsRows - 1>{}, [&](auto rc) {
        constexpr int r = decltype(rc)::value;
        M[r] = M[r + 1];
    });
    M[kDfsRows - 1] = T(0);
}

// Exclude: the column at lane `front` leaves the triangle (carried from now
// on); rows 0 .. p-1 of the live columns front+1 .. front+p-1 are
// re-triangularised, every lane applying the same rotations to its column;
// carried lanes add the dropped bottom row p-1 to their residual.
template <typename T>
__device__ __forceinline__ void exclude_front(T (&M)[kDfsRows], T& C, int front, int p,
                                              bool carried) {
    sfor(std::make_integer_sequence<int, kDfsRows - 1>{}, [&](auto jc) {
        constexpr int j = decltype(jc)::value;
        if (j + 1 < p) {
            const int piv = front + 1 + j;
            const T a = __shfl_sync(0xffffffffu, M[j], piv);
            const T b = __shfl_sync(0xffffffffu, M[j + 1], piv);
            T c, s;
            givens_cs(a, b, c, s);
            const T x = M[j], y = M[j + 1];
            M[j] = fma(c, x, s * y);
            M[j + 1] = fma(c, y, -s * x);
        }
    });
    sfor(std::make_integer_sequence<int, kDfsRows>{}, [&](auto rc) {
        constexpr int r = decltype(rc)::value;
        if (r == p - 1) {
            if (carried) C = fma(M[r], M[r], C);
            M[r] = T(0);
        }
    });
}

template <typename T>
__device__ __forceinline__ void decide(T (&M)[kDfsRows], T& C, unsigned& carried_mask, int lane,
                                       int front, int p, bool include) {
    if (include) {
        drop_first_row(M);
    } else {
        carried_mask |= 1u << front;
        exclude_front(M, C, front, p, (carried_mask >> lane) & 1u);
    }
}

template <typename T>
__device__ __forceinline__ void save_node(T* st, const T (&M)[kDfsRows], T C, unsigned carried,
                                          int lane, int rows) {
    sfor(std::make_integer_sequence<int, kDfsRows>{}, [&](auto rc) {
        constexpr int r = decltype(rc)::value;
        if (r < rows) st[r * 32 + lane] = M[r];
    });
    st[rows * 32 + lane] = C;
    if (lane == 0) *mask_of(st, rows) = carried;
    __syncwarp();
}

template <typename T>
__device__ __forceinline__ void load_node(const T* st, T (&M)[kDfsRows], T& C, unsigned& carried,
                                          int lane, int rows) {
    sfor(std::make_integer_sequence<int, kDfsRows>{}, [&](auto rc) {
        constexpr int r = decltype(rc)::value;
        M[r] = (r < rows) ? st[r * 32 + lane] : T(0);
    });
    C = st[rows * 32 + lane];
    carried = *mask_of(const_cast<T*>(st), rows);
}

// Write leaf ell's record straight to the CTA's record (lane-interleaved).
template <typename T>
__device__ __forceinline__ void write_leaf(const T (&M)[kDfsRows], T C, const Plan& p, int lane,
                                           unsigned carried_mask, int ell, T* rec,
                                           unsigned long long* chk) {
    const int Q = p.Q, k = p.k, LQ = Q * (Q + 1) / 2;
    if (lane >= k && lane < p.m) {  // L column i: rows 0 .. i of the L block
        const int i = lane - k;
        sfor(std::make_integer_sequence<int, kDfsRows>{}, [&](auto rc) {
            constexpr int r = decltype(rc)::value;
            if (r <= i) {
                const size_t ix = (size_t)(i * (i + 1) / 2 + r) * 32 + ell;
                if (GBN_IN(chk, 221, ix, p.leaf_stride)) rec[ix] = M[r];
            }
        });
    } else if (lane < k && ((carried_mask >> lane) & 1u)) {  // fixed variable in B
        const size_t b0 = (size_t)(LQ + rec_slot(p, lane, carried_mask) * (Q + 1)) * 32 + ell;
        sfor(std::make_integer_sequence<int, kDfsRows>{}, [&](auto rc) {
            constexpr int r = decltype(rc)::value;
            if (r < Q) {
                const size_t ix = b0 + (size_t)r * 32;
                if (GBN_IN(chk, 224, ix, p.leaf_stride)) rec[ix] = M[r];
            }
        });
        const size_t ix = b0 + (size_t)Q * 32;
        if (GBN_IN(chk, 225, ix, p.leaf_stride)) rec[ix] = C;
    }
}

// Shared-memory elements of one warp's depth-first stack: level t holds a
// node of Q + W - t rows.
__host__ __device__ __forceinline__ size_t dfs_stack_elems(int Q, int W) {
    size_t e = 0;
    for (int t = 0; t < W; ++t) e += node_elems(Q + W - t);
    return e > 0 ? e : 32;
}

// One warp's shared memory in the leaf kernel: the stack, then 8 staged
// leaf records.
// The staging of eight leaf records: element e of leaf j (0..7) at
// 8 e + j + skew(e), the skew 0 in the L block (e < Q(Q+1)/2) and 1 + v in
// the block of fixed variable v.  Without it the lanes of one store (one
// column each, the fixed variables' entries a multiple of Q + 1 apart) hit
// few banks (one when Q + 1 = 8); with it a lane's entries are 8 apart from
// a per-lane base, so its stores take immediate offsets.
template <int Q>
__device__ __forceinline__ int stage_skew(int e) {
    constexpr int LQ = Q * (Q + 1) / 2;
    return e < LQ ? 0 : 1 + (e - LQ) / (Q + 1);
}
__host__ __device__ __forceinline__ size_t stage_elems(size_t leaf_stride) {
    return (leaf_stride / 32) * 8 + 33;  // skews up to 1 + (k - 1) <= 32
}

__host__ __device__ __forceinline__ size_t warp_smem_elems(int Q, int W, size_t leaf_stride) {
    return dfs_stack_elems(Q, W) + stage_elems(leaf_stride);
}

template <typename T>
__device__ __forceinline__ void leaves_body(const T* __restrict__ top, const Plan& p,
                                            T* __restrict__ leaves, unsigned long long* chk,
                                            uint64_t cta, T* stack) {
    const int lane = threadIdx.x & 31;
    const int W = p.W, rows_top = p.Q + W, topk = p.k - W;
    T M[kDfsRows];
    T C;
    unsigned carried;
    load_node(top + (size_t)cta * node_elems(rows_top), M, C, carried, lane, rows_top);
    T* rec = leaves + (size_t)cta * p.leaf_stride;
    int prev = 0;
    for (int ell = 0; ell < p.lanes; ++ell) {
        // level t decides the fixed variable W-1-t with bit W-1-t of ell, so
        // consecutive leaves differ in the deepest levels first
        const int t0 = (ell == 0) ? 0 : W - 1 - (31 - __clz(ell ^ prev));
        size_t off = 0;
        for (int t = 0; t < t0; ++t) off += node_elems(rows_top - t);
        if (ell > 0) load_node(stack + off, M, C, carried, lane, rows_top - t0);
        for (int t = t0; t < W; ++t) {
            const int rows = rows_top - t;
            save_node(stack + off, M, C, carried, lane, rows);
            off += node_elems(rows);
            decide(M, C, carried, lane, topk + t, rows, ((ell >> (W - 1 - t)) & 1) != 0);
        }
        write_leaf(M, C, p, lane, carried, ell, rec, chk);
        prev = ell;
    }
}

// ---- the depth-first part for W = 5 with Q known at compile time: every
// level's row count is a constant, so each level's code does exactly its
// rotations and row moves, with no guards.
template <int RT, int L>
constexpr size_t stack_off() {
    size_t e = 0;
    for (int u = 0; u < L; ++u) e += (size_t)(RT - u + 2) * 32;
    return e;
}

// `node` is the saved copy of M: row j+1 of step j's pivot column is not yet
// touched by the earlier rotations, so it is read from shared memory off the
// critical path and only row j travels by shuffle.
template <typename T, int RT, int rows>
__device__ __forceinline__ void exclude_n(T (&M)[RT], T& C, int front, bool carried,
                                          const T* node) {
    sfor(std::make_integer_sequence<int, rows - 1>{}, [&](auto jc) {
        constexpr int j = decltype(jc)::value;
        const int piv = front + 1 + j;
        const T a = __shfl_sync(0xffffffffu, M[j], piv);
        const T b = node[(j + 1) * 32 + piv];
        T c, s;
        givens_cs(a, b, c, s);
        const T x = M[j], y = M[j + 1];
        M[j] = fma(c, x, s * y);
        M[j + 1] = fma(c, y, -s * x);
    });
    if (carried) C = fma(M[rows - 1], M[rows - 1], C);
    M[rows - 1] = T(0);
}

template <typename T, int RT, int rows>
__device__ __forceinline__ void include_n(T (&M)[RT]) {
    sfor(std::make_integer_sequence<int, rows - 1>{}, [&](auto rc) {
        constexpr int r = decltype(rc)::value;
        M[r] = M[r + 1];
    });
    M[rows - 1] = T(0);
}

template <typename T, int RT, int rows>
__device__ __forceinline__ void save_n(T* st, const T (&M)[RT], T C, unsigned carried, int lane) {
    sfor(std::make_integer_sequence<int, rows>{}, [&](auto rc) {
        constexpr int r = decltype(rc)::value;
        st[r * 32 + lane] = M[r];
    });
    st[rows * 32 + lane] = C;
    if (lane == 0) *mask_of(st, rows) = carried;
    __syncwarp();
}

template <typename T, int RT, int rows>
__device__ __forceinline__ void load_n(const T* st, T (&M)[RT], T& C, unsigned& carried, int lane) {
    sfor(std::make_integer_sequence<int, rows>{}, [&](auto rc) {
        constexpr int r = decltype(rc)::value;
        M[r] = st[r * 32 + lane];
    });
    C = st[rows * 32 + lane];
    carried = *mask_of(const_cast<T*>(st), rows);
}

// Stage leaf ell's record in shared memory, stg[8 e + (ell & 7) + skew(e)]; after
// the eighth leaf of a group (the enumeration runs ell = 31 down to 0) write
// the group out as 8-element runs, one full 32-byte sector per record element
// (FP32: two 16-byte stores).
template <typename T, int Q, int RT>
__device__ __forceinline__ void stage_leaf_q(const T (&M)[RT], T C, const Plan& p, int lane,
                                             unsigned carried_mask, int ell, T* stg, T* rec,
                                             unsigned long long* chk) {
    constexpr int LQ = Q * (Q + 1) / 2;
    const int k = p.k, j = ell & 7;
    if (lane >= k && lane < p.m) {  // L column i: rows 0 .. i of the L block
        const int i = lane - k;
        T* sb = stg + 8 * (i * (i + 1) / 2) + j;  // skew 0
        sfor(std::make_integer_sequence<int, Q>{}, [&](auto rc) {
            constexpr int r = decltype(rc)::value;
            if (r <= i) sb[8 * r] = M[r];
        });
    } else if (lane < k && ((carried_mask >> lane) & 1u)) {  // fixed variable in B
        const int v = rec_slot(p, lane, carried_mask);
        T* sb = stg + 8 * (LQ + v * (Q + 1)) + j + 1 + v;
        sfor(std::make_integer_sequence<int, Q>{}, [&](auto rc) {
            constexpr int r = decltype(rc)::value;
            sb[8 * r] = M[r];
        });
        sb[8 * Q] = C;
    }
    if (j == 0) {  // the group ell .. ell + 7 is complete
        __syncwarp();
        const int R = rec_rows(p, carried_mask);  // the record's elements in use
        if constexpr (std::is_same<T, float>::value) {
            // four leaves of one element per lane: one 16-byte store (ell is a
            // multiple of 8 here and records start 128-byte aligned)
            for (int u = lane; u < R * 2; u += 32) {
                const int e = u >> 1, h4 = (u & 1) * 4;
                const float* src = stg + 8 * e + h4 + stage_skew<Q>(e);
                const size_t ix = (size_t)e * 32 + ell + h4;
                if (GBN_IN(chk, 227, ix + 3, p.leaf_stride))
                    *reinterpret_cast<float4*>(rec + ix) = make_float4(src[0], src[1], src[2], src[3]);
            }
        } else {
            for (int idx = lane; idx < R * 8; idx += 32) {
                const size_t ix = (size_t)(idx >> 3) * 32 + ell + (idx & 7);
                if (GBN_IN(chk, 227, ix, p.leaf_stride))
                    rec[ix] = stg[idx + stage_skew<Q>(idx >> 3)];
            }
        }
        __syncwarp();
    }
}

// Level L of the depth-first enumeration: save the node, then for each
// choice of the level's variable (join F first, then join B) build the child
// and descend.  One copy of each level's code.
template <typename T, int Q, int L>
struct Dfs5 {
    static constexpr int W = 5, RT = Q + W, rows = RT - L;
    __device__ static __forceinline__ void run(T (&M)[RT], T& C, unsigned& carried, int lane,
                                               int topk, int ell, T* stack, const Plan& p, T* rec,
                                               unsigned long long* chk) {
        if constexpr (L == W) {
            (void)rows;  // a leaf: no node below it
            stage_leaf_q<T, Q, RT>(M, C, p, lane, carried, ell, stack + stack_off<RT, W>(), rec,
                                   chk);
        } else {
            T* slot = stack + stack_off<RT, L>();
            save_n<T, RT, rows>(slot, M, C, carried, lane);
#pragma unroll 1
            for (int b = 1; b >= 0; --b) {
                if (b) {
                    include_n<T, RT, rows>(M);
                } else {
                    load_n<T, RT, rows>(slot, M, C, carried, lane);
                    carried |= 1u << (topk + L);
                    exclude_n<T, RT, rows>(M, C, topk + L, (carried >> lane) & 1u, slot);
                }
                Dfs5<T, Q, L + 1>::run(M, C, carried, lane, topk, ell | (b << (W - 1 - L)), stack,
                                       p, rec, chk);
            }
        }
    }
};

// FP32 form of the same enumeration with the saved nodes in registers (one
// array per level, constant indices): a level's node is copied before the
// include branch and copied back for the exclude branch, with no shared
// memory traffic, and shared memory holds only the leaf staging.  In the
// exclude, the pivot lane forms each rotation from its own column (row j as
// rotated so far, row j+1 untouched) and broadcasts it: the same (c, s) every
// lane formed from the shuffled and the saved entry before.
template <typename T, int RT, int rows>
__device__ __forceinline__ void exclude_r(T (&M)[RT], T& C, int front, bool carried) {
    sfor(std::make_integer_sequence<int, rows - 1>{}, [&](auto jc) {
        constexpr int j = decltype(jc)::value;
        const int piv = front + 1 + j;
        T c, s;
        givens_cs(M[j], M[j + 1], c, s);
        c = __shfl_sync(0xffffffffu, c, piv);
        s = __shfl_sync(0xffffffffu, s, piv);
        const T x = M[j], y = M[j + 1];
        M[j] = fma(c, x, s * y);
        M[j + 1] = fma(c, y, -s * x);
    });
    if (carried) C = fma(M[rows - 1], M[rows - 1], C);
    M[rows - 1] = T(0);
}

template <typename T, int Q, int L>
struct Dfs5R {
    static constexpr int W = 5, RT = Q + W, rows = RT - L;
    __device__ static __forceinline__ void run(T (&M)[RT], T& C, unsigned& carried, int lane,
                                               int topk, int ell, T* stg, const Plan& p, T* rec,
                                               unsigned long long* chk) {
        if constexpr (L == W) {
            (void)rows;  // a leaf: no node below it
            stage_leaf_q<T, Q, RT>(M, C, p, lane, carried, ell, stg, rec, chk);
        } else {
            T sv[rows];
            sfor(std::make_integer_sequence<int, rows>{}, [&](auto rc) {
                constexpr int r = decltype(rc)::value;
                sv[r] = M[r];
            });
            const T svC = C;
            const unsigned svK = carried;
#pragma unroll 1
            for (int b = 1; b >= 0; --b) {
                if (b) {
                    include_n<T, RT, rows>(M);
                } else {
                    sfor(std::make_integer_sequence<int, rows>{}, [&](auto rc) {
                        constexpr int r = decltype(rc)::value;
                        M[r] = sv[r];
                    });
                    C = svC;
                    carried = svK | (1u << (topk + L));
                    exclude_r<T, RT, rows>(M, C, topk + L, (carried >> lane) & 1u);
                }
                Dfs5R<T, Q, L + 1>::run(M, C, carried, lane, topk, ell | (b << (W - 1 - L)), stg,
                                        p, rec, chk);
            }
        }
    }
};

// Whether the leaf kernel keeps its depth-first stack in registers (FP32,
// W = 5, a compiled Q): its shared memory is then the leaf staging alone.
template <typename T>
__host__ __device__ __forceinline__ bool leaves_in_registers(int Q, int W) {
    return std::is_same<T, float>::value && W == 5 && Q >= 4 && Q <= 9;
}
template <typename T>
__host__ __device__ __forceinline__ size_t leaf_warp_elems(const Plan& p) {
    return leaves_in_registers<T>(p.Q, p.W) ? stage_elems(p.leaf_stride)
                                              : warp_smem_elems(p.Q, p.W, p.leaf_stride);
}

// The FP32 form (REG) gives a walk CTA four warps: quarter qd takes the
// choices of bits 1 and 0 of qd (1: join F) at the first two leaf levels and
// enumerates the 8 leaves below them, so that four times as many warps share
// the chains of rotations and each keeps three levels' nodes in registers.
// The FP64 form (shared-memory stack) enumerates all 32 leaves in one warp.
template <typename T, int Q, bool REG>
__device__ __forceinline__ void leaves_w5(const T* __restrict__ top, const Plan& p,
                                          T* __restrict__ leaves, unsigned long long* chk,
                                          uint64_t cta, T* stack, int qd = -1) {
    constexpr int RT = Q + 5;
    const int lane = threadIdx.x & 31;
    T M[RT];
    T C;
    unsigned carried;
    load_n<T, RT, RT>(top + (size_t)cta * node_elems(RT), M, C, carried, lane);
    if constexpr (REG) {  // staging at the start of the warp's shared memory
        T* rec = leaves + (size_t)cta * p.leaf_stride;
        const int topk = p.k - 5;
        const int b0 = (qd >> 1) & 1, b1 = qd & 1;
        if (b0) {
            include_n<T, RT, RT>(M);
        } else {
            carried |= 1u << topk;
            exclude_r<T, RT, RT>(M, C, topk, (carried >> lane) & 1u);
        }
        if (b1) {
            include_n<T, RT, RT - 1>(M);
        } else {
            carried |= 1u << (topk + 1);
            exclude_r<T, RT, RT - 1>(M, C, topk + 1, (carried >> lane) & 1u);
        }
        Dfs5R<T, Q, 2>::run(M, C, carried, lane, topk, (b0 << 4) | (b1 << 3), stack, p, rec, chk);
    } else
        Dfs5<T, Q, 0>::run(M, C, carried, lane, p.k - 5, 0, stack, p,
                           leaves + (size_t)cta * p.leaf_stride, chk);
}

// The specialised enumeration (shared-memory stack) when W = 5 and Q is one
// of the compiled sizes; the batched leaf kernel's dispatch.
template <typename T>
__device__ __forceinline__ bool leaves_fast(const T* __restrict__ top, const Plan& p,
                                            T* __restrict__ leaves, unsigned long long* chk,
                                            uint64_t cta, T* stack) {
    if (p.W != 5) return false;
    switch (p.Q) {
        case 4: leaves_w5<T, 4, false>(top, p, leaves, chk, cta, stack); return true;
        case 5: leaves_w5<T, 5, false>(top, p, leaves, chk, cta, stack); return true;
        case 6: leaves_w5<T, 6, false>(top, p, leaves, chk, cta, stack); return true;
        case 7: leaves_w5<T, 7, false>(top, p, leaves, chk, cta, stack); return true;
        case 8: leaves_w5<T, 8, false>(top, p, leaves, chk, cta, stack); return true;
        case 9: leaves_w5<T, 9, false>(top, p, leaves, chk, cta, stack); return true;
        default: return false;
    }
}

template <typename T>
__device__ __forceinline__ T* top_nodes(const Plan& p, char* ws) {
    return reinterpret_cast<T*>(ws + p.off_top);
}


// One warp per group of 2^d walk CTAs (the low P bits of the CTA index).
template <typename T>
__global__ void __launch_bounds__(32 * kTopDfsWarps) roots_top_dfs_kernel(const Plan p, char* ws) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    grid_dep_wait();
    const int warp = threadIdx.x >> 5;
    const uint64_t g = (uint64_t)blockIdx.x * kTopDfsWarps + warp;
    const uint64_t groups = (uint64_t)p.n_cta >> top_dfs_levels(p);
    if (g >= groups) return;
    T* base = reinterpret_cast<T*>(smem_raw) + (size_t)warp * (32 * 32 + top_dfs_stack_elems(p));
    top_dfs_body<T>(reinterpret_cast<const double*>(ws + p.off_r0), p, top_nodes<T>(p, ws),
                    reinterpret_cast<unsigned long long*>(ws + p.off_status + kCheckOffset), g, base,
                    base + 32 * 32);
}

// One dataset: QF = the compiled Q of the specialised enumeration (FP32
// with the stack in registers, FP64 in shared memory), or 0 for the generic
// one; each instance gets the registers its own Q needs.
template <typename T, int QF>
__global__ void __launch_bounds__(32 * kDfsWarps, (std::is_same<T, float>::value && QF > 0) ? 8 : 1)
    roots_leaves_kernel(const Plan p, char* ws) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    grid_dep_wait();
    const int warp = threadIdx.x >> 5;
    constexpr bool kReg = std::is_same<T, float>::value && QF > 0;
    constexpr int kWarpsPerCta = kReg ? 4 : 1;
    const uint64_t gw = (uint64_t)blockIdx.x * kDfsWarps + warp;
    const uint64_t cta = gw / kWarpsPerCta;
    if (cta >= (uint64_t)p.n_cta) return;
    // a walk CTA whose front sets all exceed the in-degree bound is not walked
    if (__popcll(cta + (uint64_t)p.cta_begin) > p.kmax) return;
    T* stack = reinterpret_cast<T*>(smem_raw) + warp * leaf_warp_elems<T>(p);
    T* leaves = reinterpret_cast<T*>(ws + p.off_leaves);
    unsigned long long* chk = reinterpret_cast<unsigned long long*>(ws + p.off_status + kCheckOffset);
    if constexpr (QF > 0)
        leaves_w5<T, QF, kReg>(top_nodes<T>(p, ws), p, leaves, chk, cta, stack,
                               kReg ? (int)(gw & 3) : -1);
    else
        leaves_body<T>(top_nodes<T>(p, ws), p, leaves, chk, cta, stack);
}

// A batch: warps find their dataset through the prefix of walk CTAs.  Warp w
// follows the path of global CTA c0 + w (c0: the first CTA of the datasets too
// small for the depth-first form below).
template <typename T>
__global__ void __launch_bounds__(32 * kTopWarps) roots_top_kernel_b(const BatchView v, int64_t c0) {
    __shared__ T S[kTopWarps * 32 * 32];
    const int warp = threadIdx.x >> 5;
    const int64_t g = c0 + (int64_t)blockIdx.x * kTopWarps + warp;
    if (g >= v.cta_prefix[v.B]) return;
    int64_t local;
    const int d = batch_locate(v, v.cta_prefix, v.cta_pos, g, local);
    const Plan& p = v.plans[d];
    char* ws = v.ws[d];
    top_body<T>(reinterpret_cast<const double*>(ws + p.off_r0), p, top_nodes<T>(p, ws),
                reinterpret_cast<unsigned long long*>(ws + p.off_status + kCheckOffset),
                (uint64_t)local, (uint64_t)local, S + warp * 32 * 32);
}

// One dataset, a shard of the table: one warp per walk CTA of the shard, each
// following its own path (global index cta_begin + local).
template <typename T>
__global__ void __launch_bounds__(32 * kTopWarps) roots_top_kernel(const Plan p, char* ws) {
    __shared__ T S[kTopWarps * 32 * 32];
    grid_dep_wait();
    const int warp = threadIdx.x >> 5;
    const int64_t local = (int64_t)blockIdx.x * kTopWarps + warp;
    if (local >= p.n_cta) return;
    top_body<T>(reinterpret_cast<const double*>(ws + p.off_r0), p, top_nodes<T>(p, ws),
                reinterpret_cast<unsigned long long*>(ws + p.off_status + kCheckOffset),
                (uint64_t)(p.cta_begin + local), (uint64_t)local, S + warp * 32 * 32);
}

template <typename T>
__global__ void __launch_bounds__(32 * kDfsWarps) roots_leaves_kernel_b(const BatchView v,
                                                                         int Q, int max_w,
                                                                         size_t max_stride) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5;
    const int64_t g = (int64_t)blockIdx.x * kDfsWarps + warp;
    if (g >= v.cta_prefix[v.B]) return;
    int64_t local;
    const int d = batch_locate(v, v.cta_prefix, v.cta_pos, g, local);
    const Plan& p = v.plans[d];
    char* ws = v.ws[d];
    T* stack = reinterpret_cast<T*>(smem_raw) + warp * warp_smem_elems(Q, max_w, max_stride);
    T* leaves = reinterpret_cast<T*>(ws + p.off_leaves);
    unsigned long long* chk = reinterpret_cast<unsigned long long*>(ws + p.off_status + kCheckOffset);
    if (!leaves_fast<T>(top_nodes<T>(p, ws), p, leaves, chk, (uint64_t)local, stack))
        leaves_body<T>(top_nodes<T>(p, ws), p, leaves, chk, (uint64_t)local, stack);
}

template <typename T, int QF>
int launch_leaves_q(const Plan& p, char* ws, size_t smem, cudaStream_t stream) {
    if (cudaFuncSetAttribute(roots_leaves_kernel<T, QF>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess)
        return GBN_ERR_CUDA;
    const int warps_per_cta = (std::is_same<T, float>::value && QF > 0) ? 4 : 1;
    const unsigned nb = (unsigned)((p.n_cta * warps_per_cta + kDfsWarps - 1) / kDfsWarps);
    if (launch_dep(roots_leaves_kernel<T, QF>, dim3(nb), dim3(32 * kDfsWarps), smem, stream, p, ws) !=
        cudaSuccess)
        return GBN_ERR_CUDA;
    return GBN_OK;
}

template <typename T>
int launch_roots_t(const Plan& p, char* ws, cudaStream_t stream) {
    if (p.Q + p.W > kDfsRows) return GBN_ERR_Q;
    const size_t smem = sizeof(T) * leaf_warp_elems<T>(p) * kDfsWarps;
    if (smem > 227 * 1024) return GBN_ERR_Q;
    if (p.n_cta < 1) return GBN_OK;  // an empty shard
    if (p.sharded()) {  // one path per CTA of the shard
        const unsigned nb = (unsigned)((p.n_cta + kTopWarps - 1) / kTopWarps);
        if (launch_dep(roots_top_kernel<T>, dim3(nb), dim3(32 * kTopWarps), 0, stream, p, ws) !=
            cudaSuccess)
            return GBN_ERR_CUDA;
    } else {  // subtrees of 2^d CTAs enumerated depth first
        const uint64_t groups = (uint64_t)p.n_cta >> top_dfs_levels(p);
        const unsigned nb_top = (unsigned)((groups + kTopDfsWarps - 1) / kTopDfsWarps);
        const size_t smem_top = sizeof(T) * (32 * 32 + top_dfs_stack_elems(p)) * kTopDfsWarps;
        if (cudaFuncSetAttribute(roots_top_dfs_kernel<T>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem_top) != cudaSuccess)
            return GBN_ERR_CUDA;
        if (launch_dep(roots_top_dfs_kernel<T>, dim3(nb_top), dim3(32 * kTopDfsWarps), smem_top,
                       stream, p, ws) != cudaSuccess)
            return GBN_ERR_CUDA;
    }
    int rc;
    switch (p.W == 5 ? p.Q : 0) {
        case 4: rc = launch_leaves_q<T, 4>(p, ws, smem, stream); break;
        case 5: rc = launch_leaves_q<T, 5>(p, ws, smem, stream); break;
        case 6: rc = launch_leaves_q<T, 6>(p, ws, smem, stream); break;
        case 7: rc = launch_leaves_q<T, 7>(p, ws, smem, stream); break;
        case 8: rc = launch_leaves_q<T, 8>(p, ws, smem, stream); break;
        case 9: rc = launch_leaves_q<T, 9>(p, ws, smem, stream); break;
        default: rc = launch_leaves_q<T, 0>(p, ws, smem, stream); break;
    }
    return rc;
}

// A batch whose datasets all have W = 5 (FP32, a compiled Q): the four-warp
// register-stack leaf enumeration of the single-dataset kernel, warps finding
// their dataset through the prefix of walk CTAs.
template <typename T, int QF>
__global__ void __launch_bounds__(32 * kDfsWarps, 8)
    roots_leaves_kernel_bq(const BatchView v, size_t max_stride) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5;
    const int64_t gw = (int64_t)blockIdx.x * kDfsWarps + warp;
    const int64_t g = gw >> 2;
    if (g >= v.cta_prefix[v.B]) return;
    int64_t local;
    const int d = batch_locate(v, v.cta_prefix, v.cta_pos, g, local);
    const Plan& p = v.plans[d];
    char* ws = v.ws[d];
    T* stg = reinterpret_cast<T*>(smem_raw) + warp * stage_elems(max_stride);
    unsigned long long* chk = reinterpret_cast<unsigned long long*>(ws + p.off_status + kCheckOffset);
    leaves_w5<T, QF, true>(top_nodes<T>(p, ws), p, reinterpret_cast<T*>(ws + p.off_leaves), chk,
                           (uint64_t)local, stg, (int)(gw & 3));
}

template <typename T, int QF>
int launch_leaves_bq(const BatchView& v, int64_t total_cta, size_t max_stride,
                     cudaStream_t stream) {
    const size_t smem = sizeof(T) * stage_elems(max_stride) * kDfsWarps;
    if (cudaFuncSetAttribute(roots_leaves_kernel_bq<T, QF>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return GBN_ERR_CUDA;
    const unsigned nb = (unsigned)((4 * total_cta + kDfsWarps - 1) / kDfsWarps);
    return launch_rc(launch_plain(roots_leaves_kernel_bq<T, QF>, dim3(nb), dim3(32 * kDfsWarps),
                                  smem, stream, v, max_stride));
}

// A batch, the datasets with at least 4 walk CTAs (a prefix of the launch order,
// which is largest first, so every such dataset's first CTA is a multiple of 4):
// warp w takes the depth-first group w - (that dataset's first CTA) / 4 of the
// dataset, as the single-dataset kernel does, so the nodes are the same.
constexpr int kTopDfsStackMax = 2 * 32 * 32;  // two saved levels of at most 32 rows
template <typename T>
__global__ void __launch_bounds__(32 * kTopDfsWarps) roots_top_dfs_kernel_b(const BatchView v,
                                                                            int64_t n_warps) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5;
    const int64_t gw = (int64_t)blockIdx.x * kTopDfsWarps + warp;
    if (gw >= n_warps) return;
    int64_t local;
    const int d = batch_locate(v, v.cta_prefix, v.cta_pos, 4 * gw, local);
    const Plan& p = v.plans[d];
    char* ws = v.ws[d];
    T* base = reinterpret_cast<T*>(smem_raw) + (size_t)warp * (32 * 32 + kTopDfsStackMax);
    top_dfs_body<T>(reinterpret_cast<const double*>(ws + p.off_r0), p, top_nodes<T>(p, ws),
                    reinterpret_cast<unsigned long long*>(ws + p.off_status + kCheckOffset),
                    (uint64_t)(local >> 2), base, base + 32 * 32);
}

template <typename T>
int launch_roots_batched_t(const BatchView& v, int64_t total_cta, int64_t dfs_cta, int Q,
                           int max_w, size_t max_stride, cudaStream_t stream) {
    if (Q + max_w > kDfsRows) return GBN_ERR_Q;
    const size_t smem = sizeof(T) * warp_smem_elems(Q, max_w, max_stride) * kDfsWarps;
    if (smem > 227 * 1024) return GBN_ERR_Q;
    if (cudaFuncSetAttribute(roots_leaves_kernel_b<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess)
        return GBN_ERR_CUDA;
    const unsigned nb_dfs = (unsigned)((total_cta + kDfsWarps - 1) / kDfsWarps);
    if (dfs_cta > 0) {  // top nodes of the larger datasets, depth first
        const int64_t n_warps = dfs_cta / 4;
        const size_t smem_top = sizeof(T) * (32 * 32 + kTopDfsStackMax) * kTopDfsWarps;
        if (cudaFuncSetAttribute(roots_top_dfs_kernel_b<T>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem_top) != cudaSuccess)
            return GBN_ERR_CUDA;
        const unsigned nb = (unsigned)((n_warps + kTopDfsWarps - 1) / kTopDfsWarps);
        if (launch_plain(roots_top_dfs_kernel_b<T>, dim3(nb), dim3(32 * kTopDfsWarps), smem_top,
                         stream, v, n_warps) != cudaSuccess)
            return GBN_ERR_CUDA;
    }
    if (total_cta > dfs_cta) {  // the rest, one path per CTA
        const unsigned nb_top = (unsigned)((total_cta - dfs_cta + kTopWarps - 1) / kTopWarps);
        if (launch_plain(roots_top_kernel_b<T>, dim3(nb_top), dim3(32 * kTopWarps), 0, stream, v,
                         dfs_cta) != cudaSuccess)
            return GBN_ERR_CUDA;
    }
    bool reg = false;
    if constexpr (std::is_same<T, float>::value) reg = v.pairs && leaves_in_registers<T>(Q, 5);
    if (reg) {
        int rc = GBN_OK;
        if constexpr (std::is_same<T, float>::value) {
            switch (Q) {
                case 4: rc = launch_leaves_bq<T, 4>(v, total_cta, max_stride, stream); break;
                case 5: rc = launch_leaves_bq<T, 5>(v, total_cta, max_stride, stream); break;
                case 6: rc = launch_leaves_bq<T, 6>(v, total_cta, max_stride, stream); break;
                case 7: rc = launch_leaves_bq<T, 7>(v, total_cta, max_stride, stream); break;
                case 8: rc = launch_leaves_bq<T, 8>(v, total_cta, max_stride, stream); break;
                default: rc = launch_leaves_bq<T, 9>(v, total_cta, max_stride, stream); break;
            }
        }
        return rc;
    }
    return launch_rc(launch_plain(roots_leaves_kernel_b<T>, dim3(nb_dfs), dim3(32 * kDfsWarps), smem,
                                  stream, v, Q, max_w, max_stride));
}

}  // namespace

size_t top_node_bytes(const Plan& p) {
    const size_t es = p.precision ? sizeof(double) : sizeof(float);
    return es * node_elems(p.Q + p.W) * (size_t)p.n_cta;
}

int launch_roots(const Plan& p, char* ws, cudaStream_t stream) {
    return p.precision ? launch_roots_t<double>(p, ws, stream)
                       : launch_roots_t<float>(p, ws, stream);
}

int launch_roots_batched(const BatchView& v, int64_t total_cta, int64_t dfs_cta, int Q, int max_w,
                         size_t max_stride, int precision, cudaStream_t stream) {
    return precision ? launch_roots_batched_t<double>(v, total_cta, dfs_cta, Q, max_w, max_stride,
                                                      stream)
                     : launch_roots_batched_t<float>(v, total_cta, dfs_cta, Q, max_w, max_stride,
                                                     stream);
}

}  // namespace gbn

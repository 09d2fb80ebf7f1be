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
// falls off the bottom is added to its residual.
//
// One warp per CTA of the walk; lane l owns column l of R0 (plan order) for
// the whole tree and keeps it in registers: columns never move, deciding a
// variable only changes the lane's role (undecided / in F / carried in B)
// and drops one row.  The warp follows its CTA's path through the k - W top
// levels, then enumerates the 2^W leaves of the last W levels depth first,
// saving each level's node in shared memory to restart from it, and writes
// every leaf, lane-interleaved, into the leaf record the walk reads.
#include <math.h>

#include "gbn_internal.cuh"

namespace gbn {
namespace {

constexpr int kMaxRows = 32;

__device__ __forceinline__ float rsqrt_t(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsqrt_t(double x) { return rsqrt(x); }

// Include: the front variable joins F.  Drop row 0 (all lanes shift their rows).
template <typename T>
__device__ __forceinline__ void drop_first_row(T (&M)[kMaxRows]) {
#pragma unroll
    for (int r = 0; r + 1 < kMaxRows; ++r) M[r] = M[r + 1];
    M[kMaxRows - 1] = T(0);
}

// Exclude: the column at lane `front` leaves the triangle (it is carried from
// now on); rows 0 .. p-1 of the live columns front+1 .. front+p-1 are
// re-triangularised, every lane applying the same rotations to its column;
// carried lanes add the dropped bottom row p-1 to their residual.
template <typename T>
__device__ __forceinline__ void exclude_front(T (&M)[kMaxRows], T& C, int lane, int front, int p,
                                              bool carried) {
#pragma unroll
    for (int j = 0; j + 1 < kMaxRows; ++j) {
        if (j + 1 < p) {
            const int piv = front + 1 + j;
            const T a = __shfl_sync(0xffffffffu, M[j], piv);
            const T b = __shfl_sync(0xffffffffu, M[j + 1], piv);
            const T r2 = a * a + b * b;
            T c = T(1), s = T(0), rho = T(0);
            if (r2 > T(0)) {
                const T inv = rsqrt_t(r2);
                c = a * inv;
                s = b * inv;
                rho = r2 * inv;
            }
            const T x = M[j], y = M[j + 1];
            M[j] = (lane == piv) ? rho : c * x + s * y;
            M[j + 1] = (lane == piv) ? T(0) : c * y - s * x;
        }
    }
    // the bottom row p-1 falls off: into the residual of carried columns
#pragma unroll
    for (int r = 0; r < kMaxRows; ++r) {
        if (r == p - 1) {
            if (carried) C = fma(M[r], M[r], C);
            M[r] = T(0);
        }
    }
}

template <typename T>
__device__ __forceinline__ void decide(T (&M)[kMaxRows], T& C, unsigned& carried_mask, int lane,
                                       int front, int p, bool include) {
    if (include) {
        drop_first_row(M);
    } else {
        carried_mask |= 1u << front;
        exclude_front(M, C, lane, front, p, (carried_mask >> lane) & 1u);
    }
}

// Save / restore the lane's rows 0 .. rows-1 and residual (shared memory,
// [slot][row][lane], conflict-free).
// A slot holds `rows` rows and then the residual: (rows + 1) x 32 elements.
template <typename T>
__device__ __forceinline__ void save_node(T* st, const T (&M)[kMaxRows], T C, int lane, int rows) {
#pragma unroll
    for (int r = 0; r < kMaxRows; ++r)
        if (r < rows) st[r * 32 + lane] = M[r];
    st[rows * 32 + lane] = C;
}
template <typename T>
__device__ __forceinline__ void load_node(const T* st, T (&M)[kMaxRows], T& C, int lane, int rows) {
#pragma unroll
    for (int r = 0; r < kMaxRows; ++r) M[r] = (r < rows) ? st[r * 32 + lane] : T(0);
    C = st[rows * 32 + lane];
}

// Leaf record of sub-walk ell (lane-interleaved, see gbn_internal.cuh).
template <typename T>
__device__ __forceinline__ void write_leaf(const T (&M)[kMaxRows], T C, const Plan& p, int lane,
                                           unsigned carried_mask, int ell, T* rec,
                                           unsigned long long* chk) {
    const int Q = p.Q, k = p.k, LQ = Q * (Q + 1) / 2;
    if (lane >= k && lane < p.m) {  // L column i: rows 0 .. i of the L block
        const int i = lane - k;
#pragma unroll
        for (int r = 0; r < kMaxRows; ++r) {
            if (r <= i) {
                const size_t ix = (size_t)(i * (i + 1) / 2 + r) * 32 + ell;
                if (GBN_IN(chk, 221, ix, p.leaf_stride)) rec[ix] = M[r];
            }
        }
    } else if (lane < k && ((carried_mask >> lane) & 1u)) {  // fixed variable in B
        const int v = p.order[lane];
        const size_t b0 = (size_t)(LQ + v * (Q + 1)) * 32 + ell;
#pragma unroll
        for (int r = 0; r < kMaxRows; ++r) {
            if (r < Q) {
                const size_t ix = b0 + (size_t)r * 32;
                if (GBN_IN(chk, 224, ix, p.leaf_stride)) rec[ix] = M[r];
            }
        }
        const size_t ix = b0 + (size_t)Q * 32;
        if (GBN_IN(chk, 225, ix, p.leaf_stride)) rec[ix] = C;
    }
}

template <typename T>
__device__ __forceinline__ void roots_body(const double* __restrict__ R0, const Plan& p,
                                           T* __restrict__ leaves, unsigned long long* chk,
                                           uint64_t cta) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* stack = reinterpret_cast<T*>(smem_raw);  // W slots of (Q + W + 1) x 32
    const int lane = threadIdx.x & 31;
    const int m = p.m;
    T M[kMaxRows];
#pragma unroll
    for (int r = 0; r < kMaxRows; ++r)
        M[r] = (r < m && lane < m && GBN_IN(chk, 231, r * m + lane, m * m)) ? (T)R0[r * m + lane]
                                                                         : T(0);
    T C = T(0);
    unsigned carried = 0u;
    int front = 0;
    for (; front < p.k - p.W; ++front)
        decide(M, C, carried, lane, front, m - front, ((cta >> front) & 1ull) != 0ull);
    T* rec = leaves + (size_t)cta * p.leaf_stride;
    const int top = front;
    const unsigned carried_top = carried;
    const size_t slot = (size_t)(p.Q + p.W + 1) * 32;  // rows at level t: Q + W - t
    unsigned carried_at[8];
    int prev = 0;
    for (int lam = 0; lam < p.lanes; ++lam) {
        const int ell = (p.W > 0) ? (int)(__brev((unsigned)lam) >> (32 - p.W)) : 0;
        const int t0 = (lam == 0) ? 0 : __ffs(ell ^ prev) - 1;
        if (lam > 0) {
            load_node(stack + (size_t)t0 * slot, M, C, lane, m - top - t0);
            carried = carried_at[t0];
        } else {
            carried = carried_top;
        }
        for (int t = t0; t < p.W; ++t) {
            const int rows = m - top - t;
            save_node(stack + (size_t)t * slot, M, C, lane, rows);
            carried_at[t] = carried;
            decide(M, C, carried, lane, top + t, rows, ((ell >> t) & 1) != 0);
        }
        write_leaf(M, C, p, lane, carried, ell, rec, chk);
        prev = ell;
    }
}

template <typename T>
__global__ void __launch_bounds__(32) roots_kernel(const Plan p, char* ws) {
    roots_body<T>(reinterpret_cast<const double*>(ws + p.off_r0), p,
                  reinterpret_cast<T*>(ws + p.off_leaves),
                  reinterpret_cast<unsigned long long*>(ws + p.off_status + kCheckOffset),
                  blockIdx.x);
}

template <typename T>
__global__ void __launch_bounds__(32) roots_kernel_b(const BatchView v) {
    int64_t local;
    const int d = batch_locate(v, v.cta_prefix, blockIdx.x, local);
    const Plan& p = v.plans[d];
    char* ws = v.ws[d];
    roots_body<T>(reinterpret_cast<const double*>(ws + p.off_r0), p,
                  reinterpret_cast<T*>(ws + p.off_leaves),
                  reinterpret_cast<unsigned long long*>(ws + p.off_status + kCheckOffset),
                  (uint64_t)local);
}

template <typename T>
size_t roots_smem(int Q, int W) {
    return sizeof(T) * (size_t)(Q + W + 1) * 32 * (size_t)(W > 0 ? W : 1);
}

template <typename T>
int set_roots_smem() {
    static bool attr_set = false;  // per process; every device gets the same attribute value
    if (!attr_set) {
        const int bytes = (int)roots_smem<T>(kMaxRows, kLaneBits);
        if (cudaFuncSetAttribute(roots_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 bytes) != cudaSuccess ||
            cudaFuncSetAttribute(roots_kernel_b<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 bytes) != cudaSuccess)
            return GBN_ERR_CUDA;
        attr_set = true;
    }
    return GBN_OK;
}

template <typename T>
int launch_roots_t(const Plan& p, char* ws, cudaStream_t stream) {
    if (set_roots_smem<T>()) return GBN_ERR_CUDA;
    roots_kernel<T><<<(unsigned)p.n_cta, 32, roots_smem<T>(p.Q, p.W), stream>>>(p, ws);
    return cudaGetLastError() == cudaSuccess ? GBN_OK : GBN_ERR_CUDA;
}

template <typename T>
int launch_roots_batched_t(const BatchView& v, int64_t total_cta, int Q, int max_w,
                           cudaStream_t stream) {
    if (set_roots_smem<T>()) return GBN_ERR_CUDA;
    roots_kernel_b<T><<<(unsigned)total_cta, 32, roots_smem<T>(Q, max_w), stream>>>(v);
    return cudaGetLastError() == cudaSuccess ? GBN_OK : GBN_ERR_CUDA;
}

}  // namespace

int launch_roots(const Plan& p, char* ws, cudaStream_t stream) {
    return p.precision ? launch_roots_t<double>(p, ws, stream)
                       : launch_roots_t<float>(p, ws, stream);
}

int launch_roots_batched(const BatchView& v, int64_t total_cta, int Q, int max_w, int precision,
                         cudaStream_t stream) {
    return precision ? launch_roots_batched_t<double>(v, total_cta, Q, max_w, stream)
                     : launch_roots_batched_t<float>(v, total_cta, Q, max_w, stream);
}

}  // namespace gbn

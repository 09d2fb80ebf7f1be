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
// remaining variable either joins F -- drop the first row and column, since
// the rest of R is already the factor of the remaining columns after
// projecting it out -- or joins B -- delete its column, re-triangularise the
// remaining upper-Hessenberg block with one Givens rotation per row pair, and
// carry the deleted column along as a vector rotated with the rest.
//
// One warp per CTA of the walk: it follows its CTA's path through the k - W
// top levels, then enumerates the 2^W leaves of the last W levels depth first
// and writes them, lane-interleaved, to the leaf record the walk reads.
#include <math.h>

#include "gbn_internal.cuh"

namespace gbn {
namespace {

constexpr int kNodeLd = 32;  // row stride of a node matrix

// Node matrices are flat arrays indexed [row * kNodeLd + column]: with this
// toolchain, runtime-indexed two-dimensional shared-memory arrays were
// mis-addressed in sm_103 code while flat ones were not.
template <typename T>
struct Node {
    T M[32 * kNodeLd];  // row-major; columns [0,p) = R, [p, p+nc) = carried vectors
    T C[32];      // residual of each carried column below row p
    int var[32];  // variable of each column
    int p, nc;
};

__device__ __forceinline__ float rsqrt_t(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsqrt_t(double x) { return rsqrt(x); }

template <typename T>
__device__ __forceinline__ void givens(T a, T b, T& c, T& s, T& rho) {
    const T rho2 = a * a + b * b;
    if (rho2 > T(0)) {
        const T inv = rsqrt_t(rho2);
        c = a * inv;
        s = b * inv;
        rho = rho2 * inv;
    } else {
        c = T(1);
        s = T(0);
        rho = T(0);
    }
}

// Child where the first variable joins the front set F.
template <typename T>
__device__ void node_include(const Node<T>& s, Node<T>& d, int lane, unsigned long long* chk) {
    const int p = s.p, nc = s.nc;
    const int ncol = p - 1 + nc;
    if (lane < ncol && GBN_IN(chk, 201, lane + 1, 32) && GBN_IN(chk, 202, p, 33)) {
        for (int r = 0; r < p - 1; ++r) d.M[(r) * kNodeLd + (lane)] = s.M[(r + 1) * kNodeLd + (lane + 1)];
        d.C[lane] = s.C[lane + 1];
        d.var[lane] = s.var[lane + 1];
    }
    if (lane == 0) {
        d.p = p - 1;
        d.nc = nc;
    }
    __syncwarp();
}

// Child where the first variable joins the back set B.
template <typename T>
__device__ void node_exclude(const Node<T>& s, Node<T>& d, int lane, unsigned long long* chk) {
    const int p = s.p, nc = s.nc;
    const int ncol = p + nc;
    if (!GBN_IN(chk, 211, ncol, 33) || !GBN_IN(chk, 212, p, 33) || !GBN_IN(chk, 213, p - 1, 32)) {
        __syncwarp();
        return;
    }
    if (lane < ncol) {
        const int src = (lane < ncol - 1) ? lane + 1 : 0;
        for (int r = 0; r < p; ++r) d.M[(r) * kNodeLd + (lane)] = s.M[(r) * kNodeLd + (src)];
        d.C[lane] = (lane < ncol - 1) ? s.C[src] : T(0);
        d.var[lane] = s.var[src];
    }
    __syncwarp();
    for (int j = 0; j + 1 < p; ++j) {
        const T a = d.M[(j) * kNodeLd + (j)], b = d.M[(j + 1) * kNodeLd + (j)];
        T c, sn, rho;
        givens(a, b, c, sn, rho);
        T x = T(0), y = T(0);
        if (lane < ncol) {
            x = d.M[(j) * kNodeLd + (lane)];
            y = d.M[(j + 1) * kNodeLd + (lane)];
        }
        __syncwarp();
        if (lane < ncol) {
            T nx = c * x + sn * y, ny = c * y - sn * x;
            if (lane == j) {
                nx = rho;
                ny = T(0);
            }
            d.M[(j) * kNodeLd + (lane)] = nx;
            d.M[(j + 1) * kNodeLd + (lane)] = ny;
        }
        __syncwarp();
    }
    if (lane < ncol) {
        if (lane >= p - 1) {
            const T y = d.M[(p - 1) * kNodeLd + (lane)];
            d.C[lane] += y * y;
        }
        d.M[(p - 1) * kNodeLd + (lane)] = T(0);
    }
    if (lane == 0) {
        d.p = p - 1;
        d.nc = nc + 1;
    }
    __syncwarp();
}

template <typename T>
__device__ void write_leaf(const Node<T>& nd, int ell, int Q, T* rec, int lane, size_t stride,
                           unsigned long long* chk) {
    const int LQ = Q * (Q + 1) / 2;
    for (int e = lane; e < LQ; e += 32) {
        int pc = 0;
        while ((pc + 1) * (pc + 2) / 2 <= e) ++pc;
        const int r = e - pc * (pc + 1) / 2;
        if (GBN_IN(chk, 221, (size_t)e * 32 + ell, stride) && GBN_IN(chk, 222, r * 32 + pc, 1024))
            rec[(size_t)e * 32 + ell] = nd.M[(r) * kNodeLd + (pc)];
    }
    const int nc = nd.nc;
    for (int e = lane; e < nc * (Q + 1); e += 32) {
        const int col = Q + e / (Q + 1), row = e % (Q + 1);
        if (!GBN_IN(chk, 223, col, 32)) continue;
        const int v = nd.var[col];
        const T val = (row < Q) ? nd.M[(row) * kNodeLd + (col)] : nd.C[col];
        if (GBN_IN(chk, 224, (size_t)(LQ + v * (Q + 1) + row) * 32 + ell, stride))
            rec[(size_t)(LQ + v * (Q + 1) + row) * 32 + ell] = val;
    }
    __syncwarp();
}

template <typename T>
__device__ __forceinline__ void roots_body(const double* __restrict__ R0, const Plan& p,
                                           T* __restrict__ leaves, unsigned long long* chk,
                                           uint64_t cta) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Node<T>* nodes = reinterpret_cast<Node<T>*>(smem_raw);
    const int lane = threadIdx.x;
    const int m = p.m;
    Node<T>& n0 = nodes[0];
    if (lane < m) {
        for (int r = 0; r < m; ++r)
            if (GBN_IN(chk, 231, r * 32 + lane, 1024)) n0.M[(r) * kNodeLd + (lane)] = (T)R0[r * m + lane];
        n0.C[lane] = T(0);
        n0.var[lane] = p.order[lane];
    }
    if (lane == 0) {
        n0.p = m;
        n0.nc = 0;
    }
    __syncwarp();
    int cur = 0;
    for (int j = 0; j < p.k - p.W; ++j) {
        if ((cta >> j) & 1ull)
            node_include(nodes[cur], nodes[cur ^ 1], lane, chk);
        else
            node_exclude(nodes[cur], nodes[cur ^ 1], lane, chk);
        cur ^= 1;
    }
    T* rec = leaves + (size_t)cta * p.leaf_stride;
    Node<T>* lvl[8];
    lvl[0] = &nodes[cur];
    for (int t = 1; t <= p.W; ++t) lvl[t] = &nodes[1 + t];
    int prev = 0;
    for (int lam = 0; lam < p.lanes; ++lam) {
        const int ell = (p.W > 0) ? (int)(__brev((unsigned)lam) >> (32 - p.W)) : 0;
        const int t0 = (lam == 0) ? 0 : __ffs(ell ^ prev) - 1;
        for (int t = t0; t < p.W; ++t) {
            if ((ell >> t) & 1)
                node_include(*lvl[t], *lvl[t + 1], lane, chk);
            else
                node_exclude(*lvl[t], *lvl[t + 1], lane, chk);
        }
        write_leaf(*lvl[p.W], ell, p.Q, rec, lane, p.leaf_stride, chk);
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
int set_roots_smem() {
    static bool attr_set = false;  // per process; every device gets the same attribute value
    if (!attr_set) {
        if (cudaFuncSetAttribute(roots_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(sizeof(Node<T>) * 7)) != cudaSuccess ||
            cudaFuncSetAttribute(roots_kernel_b<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(sizeof(Node<T>) * 7)) != cudaSuccess)
            return GBN_ERR_CUDA;
        attr_set = true;
    }
    return GBN_OK;
}

template <typename T>
int launch_roots_t(const Plan& p, char* ws, cudaStream_t stream) {
    if (set_roots_smem<T>()) return GBN_ERR_CUDA;
    const size_t smem = sizeof(Node<T>) * (size_t)(p.W + 2);
    roots_kernel<T><<<(unsigned)p.n_cta, 32, smem, stream>>>(p, ws);
    return cudaGetLastError() == cudaSuccess ? GBN_OK : GBN_ERR_CUDA;
}

template <typename T>
int launch_roots_batched_t(const BatchView& v, int64_t total_cta, int max_w, cudaStream_t stream) {
    if (set_roots_smem<T>()) return GBN_ERR_CUDA;
    const size_t smem = sizeof(Node<T>) * (size_t)(max_w + 2);
    roots_kernel_b<T><<<(unsigned)total_cta, 32, smem, stream>>>(v);
    return cudaGetLastError() == cudaSuccess ? GBN_OK : GBN_ERR_CUDA;
}

}  // namespace

int launch_roots(const Plan& p, char* ws, cudaStream_t stream) {
    return p.precision ? launch_roots_t<double>(p, ws, stream)
                       : launch_roots_t<float>(p, ws, stream);
}

int launch_roots_batched(const BatchView& v, int64_t total_cta, int max_w, int precision,
                         cudaStream_t stream) {
    return precision ? launch_roots_batched_t<double>(v, total_cta, max_w, stream)
                     : launch_roots_batched_t<float>(v, total_cta, max_w, stream);
}

}  // namespace gbn

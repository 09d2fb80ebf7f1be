// Adjoint of the all-family scores: grad_X of L = sum_f w_f * score_f.
//
// Every score depends on X only through the centred Gram G = Xc^T Xc: for a
// family f = (c, S) with least-squares coefficients beta_f, RSS_f = v_f^T G v_f
// with v_f = e_c - beta_f (beta_f placed on S), and at the optimum
// dRSS_f = v_f^T dG v_f.  So
//     dL = <Gbar, dG>,   Gbar = sum_f alpha_f v_f v_f^T,   alpha_f = w_f * n / RSS_f,
// and grad_X = Xc (Gbar + Gbar^T) (the centring adjoint vanishes because the
// columns of Xc sum to zero).
//
// Gbar is gathered along the same Givens walk as the forward pass (Sec. 1.3,
// Sec. 2, Algorithm 1), one sub-walk per warp (Algorithm 2, corrected reading;
// front set F over the fixed variables).  For a family read off the current
// factor R at prefix length a, v_f = R^{-1} u_f with u_f = (rows a.. of the
// child's column, zero above).  The warp keeps
//     A = sum_f alpha_f u_f u_f^T
// in the row basis of the current R: a GRC step R -> G R P conjugates A by the
// same rotation (A -> G A G^T), so at the end of the sub-walk
//     Gbar_sub = R_T^{-1} A R_T^{-T}      (columns in the final ordering).
// The sub-walk's starting factor is re-formed from the R0 checkpoint by GRC
// steps (adjacent swaps, one rotation each), which sort R0's column order into
// the sub-walk's ordering [F, L, H \ F].
//
// One warp per sub-walk, lane = column slot of R.  Warps loop over sub-walks
// in a fixed order and keep a private FP64 sum of their Gbar_sub; a second
// kernel adds the per-warp sums in a fixed order and forms grad_X, so the
// result is deterministic.
#include <math.h>

#include "gbn_internal.cuh"

namespace gbn {
namespace {

constexpr int kBwdWarps = 2;  // warps per block
constexpr int kLd = 32;       // row stride of R and A (one slot per lane)
constexpr int kLdY = 33;      // row stride of the FP64 transform scratch

template <typename T>
struct BwdWarpSmem {
    T R[32 * kLd];        // R[row * kLd + slot]
    T A[32 * kLd];        // A[row * kLd + col], rows and columns in the R row basis
    double Y[32 * kLdY];  // R_T^{-1} A, then Gbar_sub (positions)
    double Gp[32 * kLd];  // this warp's running sum of Gbar (variable order)
    int var_at_pos[32];
    int slot_at_pos[32];
};

struct BwdArgs {
    const double* R0;      // m x m, plan column order
    const void* w;         // weights, table layout (T)
    double* partials;      // [total_warps][m*m]
    int* status;
    unsigned long long* chk;
    int m, k, Q;
    int64_t n_sub;         // 2^k sub-walks
    int64_t total_warps;
    double n;              // samples
    int order[32];         // plan order: position -> variable of R0's columns
};

template <typename T>
__device__ __forceinline__ void givens_cs(T a, T b, T& c, T& s, T& rho) {
    const T r2 = a * a + b * b;
    if (r2 > T(0)) {
        const T r = sqrt(r2);
        c = a / r;
        s = b / r;
        rho = r;
    } else {
        c = T(1);
        s = T(0);
        rho = T(0);
    }
}

// GRC at position s: swap the columns at positions s and s+1, then restore
// triangularity with one rotation of rows s, s+1; with_A also conjugates A.
template <typename T>
__device__ __forceinline__ void grc(BwdWarpSmem<T>& S, int lane, int& mypos, int s, bool with_A) {
    if (mypos == s)
        mypos = s + 1;
    else if (mypos == s + 1)
        mypos = s;
    const unsigned at_s = __ballot_sync(0xffffffffu, mypos == s);
    const int ls = __ffs(at_s) - 1;
    const T a = S.R[s * kLd + ls], b = S.R[(s + 1) * kLd + ls];
    T c, sn, rho;
    givens_cs(a, b, c, sn, rho);
    const T x = S.R[s * kLd + lane], y = S.R[(s + 1) * kLd + lane];
    __syncwarp();
    S.R[s * kLd + lane] = (lane == ls) ? rho : c * x + sn * y;
    S.R[(s + 1) * kLd + lane] = (lane == ls) ? T(0) : c * y - sn * x;
    if (with_A) {
        const T ax = S.A[s * kLd + lane], ay = S.A[(s + 1) * kLd + lane];
        __syncwarp();
        S.A[s * kLd + lane] = c * ax + sn * ay;
        S.A[(s + 1) * kLd + lane] = c * ay - sn * ax;
        __syncwarp();
        const T bx = S.A[lane * kLd + s], by = S.A[lane * kLd + s + 1];
        __syncwarp();
        S.A[lane * kLd + s] = c * bx + sn * by;
        S.A[lane * kLd + s + 1] = c * by - sn * bx;
    }
    __syncwarp();
}

// Families of the current ordering with prefix length a0: every column at a
// position >= a0 is a child, the parents are the columns at positions < a0.
template <typename T>
__device__ __forceinline__ void emit(BwdWarpSmem<T>& S, const BwdArgs& g, const T* __restrict__ w,
                                     int lane, int mypos, int myvar, int a0) {
    const int m = g.m;
    const unsigned mask = __reduce_or_sync(0xffffffffu,
                                           (lane < m && mypos < a0) ? (1u << myvar) : 0u);
    const bool child = lane < m && mypos >= a0;
    T rss = T(0);
    for (int r = a0; r < m; ++r) {
        const T z = S.R[r * kLd + lane];
        rss += z * z;
    }
    T alpha = T(0);
    if (child) {
        const unsigned low = mask & ((1u << myvar) - 1u);
        const unsigned high = (mask >> (myvar + 1)) << myvar;
        const int64_t slot = ((int64_t)myvar << (m - 1)) + (int64_t)(low | high);
        if (GBN_IN(g.chk, 301, slot, (int64_t)m << (m - 1))) {
            const T wf = w[slot];
            if (rss > T(0)) alpha = wf * (T)g.n / rss;
        }
    }
    unsigned cm = __ballot_sync(0xffffffffu, child && alpha != T(0));
    while (cm) {
        const int c = __ffs(cm) - 1;
        cm &= cm - 1;
        const T al = __shfl_sync(0xffffffffu, alpha, c);
        const T tb = (lane >= a0 && lane < m) ? al * S.R[lane * kLd + c] : T(0);
        if (tb != T(0))
            for (int r = a0; r < m; ++r) S.A[r * kLd + lane] += tb * S.R[r * kLd + c];
    }
    __syncwarp();
}

template <typename T>
__global__ void __launch_bounds__(32 * kBwdWarps) bwd_walk_kernel(BwdArgs g) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    BwdWarpSmem<T>& S = reinterpret_cast<BwdWarpSmem<T>*>(smem_raw)[threadIdx.x >> 5];
    const int lane = threadIdx.x & 31;
    const int64_t wid = (int64_t)blockIdx.x * kBwdWarps + (threadIdx.x >> 5);
    const int m = g.m, k = g.k, Q = g.Q;
    const T* __restrict__ w = static_cast<const T*>(g.w);
    for (int e = lane; e < 32 * kLd; e += 32) S.Gp[e] = 0.0;
    const int64_t nsteps = ((int64_t)1 << Q) - Q - 1;
    const unsigned hmask = k > 0 ? (unsigned)((1ull << k) - 1ull) : 0u;

    for (int64_t sub = wid; sub < g.n_sub; sub += g.total_warps) {
        const unsigned F = (unsigned)sub;  // bit v set: fixed variable v is in the front set
        const int d = __popc(F);
        // checkpoint: R0 in plan order, slot = plan position
        for (int r = 0; r < 32; ++r) {
            T v = T(0);
            if (lane < m && r < m && GBN_IN(g.chk, 302, r * m + lane, m * m)) v = (T)g.R0[r * m + lane];
            S.R[r * kLd + lane] = v;
            S.A[r * kLd + lane] = T(0);
        }
        const int myvar = lane < m ? g.order[lane] : 0;
        int mypos = lane;
        // target position in [F ascending, L = k..m-1, (H \ F) ascending]
        int tpos = lane;
        if (lane < m) {
            const unsigned below = (1u << myvar) - 1u;
            if (myvar >= k)
                tpos = d + (myvar - k);
            else if ((F >> myvar) & 1u)
                tpos = __popc(F & below);
            else
                tpos = d + Q + __popc(~F & hmask & below);
        }
        __syncwarp();
        for (int p = 0; p < m; ++p) {  // sort by GRC steps; positions < p are final
            const int owner = __ffs(__ballot_sync(0xffffffffu, lane < m && tpos == p)) - 1;
            const int q = __shfl_sync(0xffffffffu, mypos, owner);
            for (int s = q - 1; s >= p; --s) grc(S, lane, mypos, s, false);
        }
        // the sub-walk: families at the root, then one new prefix per swap
        for (int a0 = d; a0 <= d + Q; ++a0) emit(S, g, w, lane, mypos, myvar, a0);
        for (int64_t t = 0; t < nsteps; ++t) {
            const int s = d + upsilon_at(Q, t) - 1;
            grc(S, lane, mypos, s, true);
            emit(S, g, w, lane, mypos, myvar, s + 1);
        }
        // Gbar_sub = R_T^{-1} A R_T^{-T} in FP64, columns by final position
        if (lane < m) {
            S.var_at_pos[mypos] = myvar;
            S.slot_at_pos[mypos] = lane;
        }
        __syncwarp();
        const double diag = lane < m ? (double)S.R[lane * kLd + S.slot_at_pos[lane]] : 1.0;
        if (__any_sync(0xffffffffu, diag == 0.0)) {  // singular factor: flag, skip
            if (lane == 0) atomicOr(g.status, GBN_STATUS_RANK_DEFICIENT);
            continue;
        }
        if (lane < m) {  // Y = R_T^{-1} A, lane = column of A
            for (int p = m - 1; p >= 0; --p) {
                double acc = (double)S.A[p * kLd + lane];
                for (int q = p + 1; q < m; ++q)
                    acc -= (double)S.R[p * kLd + S.slot_at_pos[q]] * S.Y[q * kLdY + lane];
                S.Y[p * kLdY + lane] = acc / (double)S.R[p * kLd + S.slot_at_pos[p]];
            }
        }
        __syncwarp();
        if (lane < m) {  // Gbar_sub = Y R_T^{-T}, lane = row, in place
            for (int p = m - 1; p >= 0; --p) {
                double acc = S.Y[lane * kLdY + p];
                for (int q = p + 1; q < m; ++q)
                    acc -= (double)S.R[p * kLd + S.slot_at_pos[q]] * S.Y[lane * kLdY + q];
                S.Y[lane * kLdY + p] = acc / (double)S.R[p * kLd + S.slot_at_pos[p]];
            }
            const int vr = S.var_at_pos[lane];
            for (int q = 0; q < m; ++q) S.Gp[vr * kLd + S.var_at_pos[q]] += S.Y[lane * kLdY + q];
        }
        __syncwarp();
    }
    if (wid < g.total_warps)
        for (int e = lane; e < m * m; e += 32)
            g.partials[wid * (int64_t)(m * m) + e] = S.Gp[(e / m) * kLd + e % m];
}

// Gsym = Gbar + Gbar^T from the per-warp sums (one warp per entry, lanes over
// the partial sums, fixed shuffle tree), and the column means by variable.
__global__ void bwd_reduce_kernel(const double* __restrict__ partials, int64_t total_warps, int m,
                                  const double* __restrict__ mu_plan, Plan plan,
                                  double* __restrict__ gsym, double* __restrict__ mu_var) {
    const int lane = threadIdx.x & 31;
    const int nw = blockDim.x >> 5;
    const int mm = m * m;
    for (int e = (threadIdx.x >> 5) + blockIdx.x * nw; e < mm; e += nw * gridDim.x) {
        const int i = e / m, j = e % m;
        double s = 0.0;
        for (int64_t wdx = lane; wdx < total_warps; wdx += 32)
            s += partials[wdx * mm + i * m + j] + partials[wdx * mm + j * m + i];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) gsym[e] = s;
    }
    if (blockIdx.x == 0 && threadIdx.x < m) mu_var[plan.order[threadIdx.x]] = mu_plan[threadIdx.x];
}

// grad_X[t][j] = sum_l (X[t][l] - mu[l]) * Gsym[l][j]
__global__ void bwd_grad_kernel(const double* __restrict__ X, int64_t n, int m,
                                const double* __restrict__ gsym, const double* __restrict__ mu_var,
                                double* __restrict__ grad) {
    __shared__ double gs[32 * 32];
    __shared__ double mu[32];
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) gs[e] = gsym[e];
    if (threadIdx.x < m) mu[threadIdx.x] = mu_var[threadIdx.x];
    __syncthreads();
    const int64_t total = n * m;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = e / m;
        const int j = (int)(e % m);
        double acc = 0.0;
        for (int l = 0; l < m; ++l) acc = fma(X[t * m + l] - mu[l], gs[l * m + j], acc);
        grad[e] = acc;
    }
}

struct BwdPlan {
    Plan p;         // R0 stage layout (plan order, means, Gram panels, R1, R0)
    int Qb = 0;     // sub-walk size of the backward walk
    int kb = 0;
    int64_t n_sub = 0, total_warps = 0;
    size_t off_partials = 0, off_gsym = 0, off_muv = 0, total = 0;
};

constexpr int64_t kBwdMaxWarps = 4096;

int make_bwd_plan(int64_t n, int32_t m, const givensbn_opts* opts, BwdPlan* b) {
    givensbn_opts o;
    givensbn_default_opts(&o);
    if (opts) o = *opts;
    if (o.shard_count > 1) return GBN_ERR_OPTS;  // the gradient sums over every family
    const int qreq = o.q;
    o.q = 0;
    o.consumer_warps = 0;
    o.tune_cache = nullptr;
    o.debug_coverage = 0;
    o.fixup_tau = 0.0;  // no fix-up stage: its workspace region is reused below
    int rc = make_plan(n, m, &o, &b->p);
    if (rc) return rc;
    int Qb = qreq > 0 ? qreq : m - 10;
    if (qreq <= 0) {
        if (Qb < 2) Qb = 2;
        if (Qb > m) Qb = m;
    }
    if (Qb < 1 || Qb > m || m - Qb > 30) return GBN_ERR_Q;
    b->Qb = Qb;
    b->kb = m - Qb;
    b->n_sub = (int64_t)1 << b->kb;
    b->total_warps = b->n_sub < kBwdMaxWarps ? b->n_sub : kBwdMaxWarps;
    size_t off = b->p.off_leaves;  // the forward leaf records are not needed here
    auto up = [](size_t x) { return (x + 255) / 256 * 256; };
    b->off_partials = off;
    off = up(off + sizeof(double) * (size_t)b->total_warps * m * m);
    b->off_gsym = off;
    off = up(off + sizeof(double) * (size_t)m * m);
    b->off_muv = off;
    off = up(off + sizeof(double) * 32);
    b->total = off;
    return GBN_OK;
}

template <typename T>
int launch_bwd(const BwdPlan& b, const double* X, const void* w, double* grad, char* ws,
               cudaStream_t stream) {
    const Plan& p = b.p;
    BwdArgs g;
    g.R0 = reinterpret_cast<const double*>(ws + p.off_r0);
    g.w = w;
    g.partials = reinterpret_cast<double*>(ws + b.off_partials);
    g.status = reinterpret_cast<int*>(ws + p.off_status);
    g.chk = reinterpret_cast<unsigned long long*>(ws + p.off_status + kCheckOffset);
    g.m = p.m;
    g.k = b.kb;
    g.Q = b.Qb;
    g.n_sub = b.n_sub;
    g.total_warps = b.total_warps;
    g.n = (double)p.n;
    for (int i = 0; i < 32; ++i) g.order[i] = p.order[i];
    const size_t smem = sizeof(BwdWarpSmem<T>) * kBwdWarps;
    if (cudaFuncSetAttribute(bwd_walk_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess)
        return GBN_ERR_CUDA;
    const unsigned blocks = (unsigned)((b.total_warps + kBwdWarps - 1) / kBwdWarps);
    double* gsym = reinterpret_cast<double*>(ws + b.off_gsym);
    double* muv = reinterpret_cast<double*>(ws + b.off_muv);
    const double* mu = reinterpret_cast<const double*>(ws + p.off_mu);
    const double* partials = g.partials;
    const cudaError_t e[] = {
        launch_plain(bwd_walk_kernel<T>, dim3(blocks), dim3(32 * kBwdWarps), smem, stream, g),
        launch_plain(bwd_reduce_kernel, dim3(8), dim3(256), 0, stream, partials, b.total_warps, p.m,
                     mu, p, gsym, muv),
        launch_plain(bwd_grad_kernel, dim3(304), dim3(256), 0, stream, X, p.n, p.m,
                     (const double*)gsym, (const double*)muv, grad)};
    for (cudaError_t x : e)
        if (x != cudaSuccess) return GBN_ERR_CUDA;
    return GBN_OK;
}

}  // namespace
}  // namespace gbn

using namespace gbn;

extern "C" int givensbn_backward_workspace_size(int64_t n, int32_t m, const givensbn_opts* opts,
                                                size_t* bytes) {
    if (!bytes) return GBN_ERR_NULL;
    BwdPlan b;
    const int rc = make_bwd_plan(n, m, opts, &b);
    if (rc) return rc;
    *bytes = b.total;
    return GBN_OK;
}

extern "C" int score_all_families_backward(const double* X, int64_t n, int32_t m, const void* w,
                                           double* grad_X, const givensbn_opts* opts) {
    if (!opts) return GBN_ERR_NULL;
    BwdPlan b;
    int rc = make_bwd_plan(n, m, opts, &b);
    if (rc) return rc;
    if (!X || !w || !grad_X) return GBN_ERR_NULL;
    if (((uintptr_t)X & 7u) || ((uintptr_t)w & 15u) || ((uintptr_t)grad_X & 7u)) return GBN_ERR_ALIGN;
    if (!opts->workspace || opts->workspace_bytes < b.total) return GBN_ERR_WORKSPACE;
    if ((uintptr_t)opts->workspace & 255u) return GBN_ERR_ALIGN;
    char* ws = static_cast<char*>(opts->workspace);
    cudaStream_t stream = static_cast<cudaStream_t>(opts->stream);
    if ((rc = launch_r0(b.p, X, ws, stream))) return rc;
    return b.p.precision ? launch_bwd<double>(b, X, w, grad_X, ws, stream)
                         : launch_bwd<float>(b, X, w, grad_X, ws, stream);
}

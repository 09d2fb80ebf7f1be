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
constexpr int64_t kBwdMaxWarps = 4096;  // warps given to one dataset
constexpr int kLd = 33;       // row stride of R and A (one slot per lane; odd: conflict-free)
constexpr int kLdW = 33;      // row stride of the tail sums
constexpr int kLdY = 33;      // row stride of the FP64 transform scratch

// Per warp.  The tail sums and the children's alphas are needed during the
// walk only, the FP64 transform scratch after it: they share storage.
template <typename T>
struct BwdWarpSmem {
    T R[32 * kLd];  // R[row * kLd + slot]
    T A[32 * kLd];  // A[row * kLd + col] (symmetric, both triangles), R's row basis
    union {
        struct {
            T Wt[33 * kLdW];  // Wt[r * kLdW + slot] = sum_{t >= r} R[t][slot]^2
            T P[32];          // alpha of each child slot of the current prefix
        };
        double Y[32 * kLdY];  // R_T^{-1} A, then Gbar_sub (positions)
    };
    double dinv[32];  // 1 / R_T[p][p] by position
    int var_at_pos[32];
    int slot_at_pos[32];
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
// triangularity with one rotation of rows s, s+1.  with_A also conjugates A
// (A -> G A G^T): lane j rotates its entries of rows s, s+1; by symmetry
// they are also column j's entries of columns s, s+1, except in the 2 x 2
// block, which lane s rotates on both sides; and the tail sums of row s+1.
template <typename T>
__device__ __forceinline__ void grc(BwdWarpSmem<T>& S, int m, int lane, int& mypos, int s,
                                    bool with_A) {
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
    T ax = T(0), ay = T(0);
    if (with_A) {
        ax = S.A[s * kLd + lane];
        ay = S.A[(s + 1) * kLd + lane];
    }
    __syncwarp();
    const T ry = (lane == ls) ? T(0) : c * y - sn * x;
    S.R[s * kLd + lane] = (lane == ls) ? rho : c * x + sn * y;
    S.R[(s + 1) * kLd + lane] = ry;
    if (with_A) {
        const T nx = c * ax + sn * ay, ny = c * ay - sn * ax;  // rows of G A
        const T nxs = __shfl_sync(0xffffffffu, nx, s), nxs1 = __shfl_sync(0xffffffffu, nx, s + 1);
        const T nys = __shfl_sync(0xffffffffu, ny, s), nys1 = __shfl_sync(0xffffffffu, ny, s + 1);
        if (lane < m && lane != s && lane != s + 1) {
            S.A[s * kLd + lane] = nx;
            S.A[(s + 1) * kLd + lane] = ny;
            S.A[lane * kLd + s] = nx;
            S.A[lane * kLd + s + 1] = ny;
        }
        if (lane == s) {
            S.A[s * kLd + s] = c * nxs + sn * nxs1;
            S.A[s * kLd + s + 1] = c * nxs1 - sn * nxs;
            S.A[(s + 1) * kLd + s] = c * nys + sn * nys1;
            S.A[(s + 1) * kLd + s + 1] = c * nys1 - sn * nys;
        }
        // the rotation keeps R[s][j]^2 + R[s+1][j]^2: only row s+1's tail sum changes
        S.Wt[(s + 1) * kLdW + lane] = fma(ry, ry, S.Wt[(s + 2) * kLdW + lane]);
    }
    __syncwarp();
}

// Families of the current ordering with prefix length a0: every column at a
// position >= a0 is a child (its RSS the tail sum of its slot from row a0),
// the parents are the columns at positions < a0.  Then
// A[r][j] += sum_c alpha_c R[r][c] R[j][c] for rows r, j >= a0 (lane = j).
template <typename T>
__device__ __forceinline__ void emit(BwdWarpSmem<T>& S, const BwdArgs& g, const T* __restrict__ w,
                                     int lane, int mypos, int myvar, int a0) {
    const int m = g.m;
    const unsigned mask = __reduce_or_sync(0xffffffffu,
                                           (lane < m && mypos < a0) ? (1u << myvar) : 0u);
    const bool child = lane < m && mypos >= a0;
    T alpha = T(0);
    if (child) {
        const unsigned low = mask & ((1u << myvar) - 1u);
        const unsigned high = (mask >> (myvar + 1)) << myvar;
        const int64_t slot = ((int64_t)myvar << (m - 1)) + (int64_t)(low | high);
        const T rss = S.Wt[a0 * kLdW + lane];
        if (GBN_IN(g.chk, 301, slot, (int64_t)m << (m - 1))) {
            const T wf = w[slot];
            if (rss > T(0)) alpha = wf * (T)g.n / rss;
        }
    }
    S.P[lane] = alpha;
    const unsigned cm = __ballot_sync(0xffffffffu, child && alpha != T(0));
    __syncwarp();
    if (!cm) return;
    // the children as a list (warp-uniform): slot c_i and t_i = alpha_i R[lane][c_i] in
    // registers, so each (row, child) term is one broadcast load and one FMA
    const int nc = __popc(cm);
    int cs[32];
    T t[32];
    unsigned rest = cm;
#pragma unroll
    for (int i = 0; i < 32; ++i) {
        if (i < nc) {
            const int c = __ffs(rest) - 1;
            rest &= rest - 1;
            cs[i] = c;
            t[i] = S.P[c] * S.R[lane * kLd + c];
        }
    }
    if (lane >= a0 && lane < m) {
        for (int r = a0; r < m; ++r) {
            const T* Rr = S.R + r * kLd;
            T acc0 = S.A[r * kLd + lane], acc1 = T(0);
#pragma unroll
            for (int i = 0; i < 32; i += 2) {
                if (i < nc) acc0 = fma(t[i], Rr[cs[i]], acc0);
                if (i + 1 < nc) acc1 = fma(t[i + 1], Rr[cs[i + 1]], acc1);
            }
            S.A[r * kLd + lane] = acc0 + acc1;
        }
    }
    __syncwarp();
}

// The sub-walks lw, lw + nw, ... of one dataset, by one warp; Gbar_sub of
// each is added to this warp's FP64 partial sum (partials slot lw).
template <typename T>
__device__ __forceinline__ void bwd_subwalks(const BwdArgs& g, int64_t lw, int64_t nw,
                                             BwdWarpSmem<T>& S) {
    const int lane = threadIdx.x & 31;
    const int m = g.m, k = g.k, Q = g.Q;
    const T* __restrict__ w = static_cast<const T*>(g.w);
    double* part = g.partials + lw * (int64_t)(m * m);
    for (int e = lane; e < m * m; e += 32) part[e] = 0.0;
    const int64_t nsteps = ((int64_t)1 << Q) - Q - 1;
    const unsigned hmask = k > 0 ? (unsigned)((1ull << k) - 1ull) : 0u;

    for (int64_t sub = lw; sub < g.n_sub; sub += nw) {
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
            for (int s = q - 1; s >= p; --s) grc(S, m, lane, mypos, s, false);
        }
        {  // tail sums of every slot from every row
            T acc = T(0);
            S.Wt[32 * kLdW + lane] = T(0);
            for (int r = 31; r >= 0; --r) {
                const T z = S.R[r * kLd + lane];
                acc = fma(z, z, acc);
                S.Wt[r * kLdW + lane] = acc;
            }
        }
        __syncwarp();
        // the sub-walk: families at the root, then one new prefix per swap
        for (int a0 = d; a0 <= d + Q; ++a0) emit(S, g, w, lane, mypos, myvar, a0);
        for (int64_t t = 0; t < nsteps; ++t) {
            const int s = d + upsilon_at(Q, t) - 1;
            grc(S, m, lane, mypos, s, true);
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
        S.dinv[lane] = 1.0 / diag;  // every pivot's reciprocal at once (FP64 division is slow)
        __syncwarp();
        if (lane < m) {  // Y = R_T^{-1} A, lane = column of A
            for (int p = m - 1; p >= 0; --p) {
                double acc = (double)S.A[p * kLd + lane];
                for (int q = p + 1; q < m; ++q)
                    acc -= (double)S.R[p * kLd + S.slot_at_pos[q]] * S.Y[q * kLdY + lane];
                S.Y[p * kLdY + lane] = acc * S.dinv[p];
            }
        }
        __syncwarp();
        if (lane < m) {  // Gbar_sub = Y R_T^{-T}, lane = row, in place
            for (int p = m - 1; p >= 0; --p) {
                double acc = S.Y[lane * kLdY + p];
                for (int q = p + 1; q < m; ++q)
                    acc -= (double)S.R[p * kLd + S.slot_at_pos[q]] * S.Y[lane * kLdY + q];
                S.Y[lane * kLdY + p] = acc * S.dinv[p];
            }
            const int vr = S.var_at_pos[lane];
            for (int q = 0; q < m; ++q) part[vr * m + S.var_at_pos[q]] += S.Y[lane * kLdY + q];
        }
        __syncwarp();
    }
}

// One dataset: warp wid takes sub-walks wid, wid + warps, ...
template <typename T>
__global__ void __launch_bounds__(32 * kBwdWarps) bwd_walk_kernel(BwdArgs g) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    BwdWarpSmem<T>& S = reinterpret_cast<BwdWarpSmem<T>*>(smem_raw)[threadIdx.x >> 5];
    grid_dep_wait();
    const int64_t wid = (int64_t)blockIdx.x * kBwdWarps + (threadIdx.x >> 5);
    if (wid < g.warps) bwd_subwalks<T>(g, wid, g.warps, S);
}

// A batch: warp gw belongs to dataset d with warp_prefix[d] <= gw < warp_prefix[d+1].
template <typename T>
__global__ void __launch_bounds__(32 * kBwdWarps)
    bwd_walk_kernel_b(const BwdArgs* __restrict__ args, const int64_t* __restrict__ warp_prefix,
                      int B) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    BwdWarpSmem<T>& S = reinterpret_cast<BwdWarpSmem<T>*>(smem_raw)[threadIdx.x >> 5];
    const int64_t gw = (int64_t)blockIdx.x * kBwdWarps + (threadIdx.x >> 5);
    if (gw >= warp_prefix[B]) return;
    int lo = 0, hi = B;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (warp_prefix[mid] <= gw)
            lo = mid;
        else
            hi = mid;
    }
    const BwdArgs& g = args[lo];  // read from global memory where used
    bwd_subwalks<T>(g, gw - warp_prefix[lo], g.warps, S);
}

// Gsym = Gbar + Gbar^T from the per-warp sums (one warp per entry, lanes over
// the partial sums, fixed shuffle tree), and the column means by variable.
__device__ __forceinline__ void bwd_reduce_body(const double* __restrict__ partials,
                                                int64_t warps, int m,
                                                const double* __restrict__ mu_plan,
                                                const int* order, double* __restrict__ gsym,
                                                double* __restrict__ mu_var, int blk, int nblk) {
    const int lane = threadIdx.x & 31;
    const int nw = blockDim.x >> 5;
    const int mm = m * m;
    for (int e = (threadIdx.x >> 5) + blk * nw; e < mm; e += nw * nblk) {
        const int i = e / m, j = e % m;
        double s = 0.0;
        for (int64_t wdx = lane; wdx < warps; wdx += 32)
            s += partials[wdx * mm + i * m + j] + partials[wdx * mm + j * m + i];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) gsym[e] = s;
    }
    if (blk == 0 && threadIdx.x < m) mu_var[order[threadIdx.x]] = mu_plan[threadIdx.x];
}

// grad_X[t][j] = sum_l (X[t][l] - mu[l]) * Gsym[l][j]
__device__ __forceinline__ void bwd_grad_body(const double* __restrict__ X, int64_t n, int m,
                                              const double* __restrict__ gsym,
                                              const double* __restrict__ mu_var,
                                              double* __restrict__ grad, int blk, int nblk) {
    __shared__ double gs[32 * 32];
    __shared__ double mu[32];
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) gs[e] = gsym[e];
    if (threadIdx.x < m) mu[threadIdx.x] = mu_var[threadIdx.x];
    __syncthreads();
    const int64_t total = n * m;
    for (int64_t e = (int64_t)blk * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)nblk * blockDim.x) {
        const int64_t t = e / m;
        const int j = (int)(e % m);
        double acc = 0.0;
        for (int l = 0; l < m; ++l) acc = fma(X[t * m + l] - mu[l], gs[l * m + j], acc);
        grad[e] = acc;
    }
}

__global__ void bwd_reduce_kernel(const double* __restrict__ partials, int64_t warps, int m,
                                  const double* __restrict__ mu_plan, Plan plan,
                                  double* __restrict__ gsym, double* __restrict__ mu_var) {
    grid_dep_wait();
    bwd_reduce_body(partials, warps, m, mu_plan, plan.order, gsym, mu_var, blockIdx.x, gridDim.x);
}

__global__ void bwd_grad_kernel(const double* __restrict__ X, int64_t n, int m,
                                const double* __restrict__ gsym, const double* __restrict__ mu_var,
                                double* __restrict__ grad) {
    grid_dep_wait();
    bwd_grad_body(X, n, m, gsym, mu_var, grad, blockIdx.x, gridDim.x);
}

// Batched reduction and gradient: grid.y = dataset.
__global__ void bwd_reduce_kernel_b(const BwdArgs* __restrict__ args) {
    const BwdArgs& g = args[blockIdx.y];
    bwd_reduce_body(g.partials, g.warps, g.m, g.mu_plan, g.order, g.gsym, g.mu_var, blockIdx.x,
                    gridDim.x);
}
__global__ void bwd_grad_kernel_b(const BwdArgs* __restrict__ args) {
    const BwdArgs& g = args[blockIdx.y];
    bwd_grad_body(g.X, g.rows, g.m, g.gsym, g.mu_var, g.grad, blockIdx.x, gridDim.x);
}

struct BwdPlan {
    Plan p;         // R0 stage layout (plan order, means, Gram panels, R1, R0)
    int Qb = 0;     // sub-walk size of the backward walk
    int kb = 0;
    int64_t n_sub = 0, warps = 0;
    size_t off_partials = 0, off_gsym = 0, off_muv = 0, total = 0;
};

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
    rc = bwd_subwalk_plan(m, qreq, &b->Qb, &b->n_sub, &b->warps);
    if (rc) return rc;
    b->kb = m - b->Qb;
    size_t off = b->p.off_leaves;  // the forward leaf records are not needed here
    auto up = [](size_t x) { return (x + 255) / 256 * 256; };
    b->off_partials = off;
    off = up(off + sizeof(double) * (size_t)b->warps * m * m);
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
    BwdArgs g = bwd_args(p, ws, X, w, grad, b.Qb, b.n_sub, b.warps,
                         reinterpret_cast<double*>(ws + b.off_partials),
                         reinterpret_cast<double*>(ws + b.off_gsym),
                         reinterpret_cast<double*>(ws + b.off_muv));
    const size_t smem = sizeof(BwdWarpSmem<T>) * kBwdWarps;
    if (cudaFuncSetAttribute(bwd_walk_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess)
        return GBN_ERR_CUDA;
    const unsigned blocks = (unsigned)((b.warps + kBwdWarps - 1) / kBwdWarps);
    const cudaError_t e[] = {
        launch_dep(bwd_walk_kernel<T>, dim3(blocks), dim3(32 * kBwdWarps), smem, stream, g),
        launch_dep(bwd_reduce_kernel, dim3(8), dim3(256), 0, stream, (const double*)g.partials,
                   g.warps, p.m, g.mu_plan, p, g.gsym, g.mu_var),
        launch_dep(bwd_grad_kernel, dim3(304), dim3(256), 0, stream, X, p.n, p.m,
                   (const double*)g.gsym, (const double*)g.mu_var, grad)};
    for (cudaError_t x : e)
        if (x != cudaSuccess) return GBN_ERR_CUDA;
    return GBN_OK;
}

template <typename T>
int launch_bwd_batched_t(const BwdArgs* args, const int64_t* warp_prefix, int B,
                         int64_t total_warps, cudaStream_t stream) {
    const size_t smem = sizeof(BwdWarpSmem<T>) * kBwdWarps;
    if (cudaFuncSetAttribute(bwd_walk_kernel_b<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess)
        return GBN_ERR_CUDA;
    const unsigned blocks = (unsigned)((total_warps + kBwdWarps - 1) / kBwdWarps);
    const cudaError_t e[] = {
        launch_plain(bwd_walk_kernel_b<T>, dim3(blocks), dim3(32 * kBwdWarps), smem, stream, args,
                     warp_prefix, B),
        launch_plain(bwd_reduce_kernel_b, dim3(4, (unsigned)B), dim3(256), 0, stream, args),
        launch_plain(bwd_grad_kernel_b, dim3(32, (unsigned)B), dim3(256), 0, stream, args)};
    for (cudaError_t x : e)
        if (x != cudaSuccess) return GBN_ERR_CUDA;
    return GBN_OK;
}

}  // namespace

int bwd_subwalk_plan(int m, int q_requested, int* Qb, int64_t* n_sub, int64_t* warps) {
    int q = q_requested > 0 ? q_requested : m - 10;
    if (q_requested <= 0) {
        if (q < 2) q = 2;
        if (q > m) q = m;
    }
    if (q < 1 || q > m || m - q > 30) return GBN_ERR_Q;
    *Qb = q;
    *n_sub = (int64_t)1 << (m - q);
    *warps = *n_sub < kBwdMaxWarps ? *n_sub : kBwdMaxWarps;
    return GBN_OK;
}

BwdArgs bwd_args(const Plan& p, char* ws, const double* X, const void* w, double* grad, int Qb,
                 int64_t n_sub, int64_t warps, double* partials, double* gsym, double* mu_var) {
    BwdArgs g;
    g.R0 = reinterpret_cast<const double*>(ws + p.off_r0);
    g.w = w;
    g.partials = partials;
    g.status = reinterpret_cast<int*>(ws + p.off_status);
    g.chk = reinterpret_cast<unsigned long long*>(ws + p.off_status + kCheckOffset);
    g.m = p.m;
    g.k = p.m - Qb;
    g.Q = Qb;
    g.n_sub = n_sub;
    g.warps = warps;
    g.n = (double)p.n;
    for (int i = 0; i < 32; ++i) g.order[i] = p.order[i];
    g.X = X;
    g.rows = p.n;
    g.mu_plan = reinterpret_cast<const double*>(ws + p.off_mu);
    g.gsym = gsym;
    g.mu_var = mu_var;
    g.grad = grad;
    return g;
}

int launch_bwd_batched(const BwdArgs* args, const int64_t* warp_prefix, int B, int64_t total_warps,
                       int precision, cudaStream_t stream) {
    return precision ? launch_bwd_batched_t<double>(args, warp_prefix, B, total_warps, stream)
                     : launch_bwd_batched_t<float>(args, warp_prefix, B, total_warps, stream);
}

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

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
constexpr int kStepTab = 1024;  // swap positions kept per warp (every Q <= 10)

// Per warp; MW (16 or 32) is the widest factor the warp holds.  For MW = 16
// the two half-warps hold the same columns and split the rows of the rank
// update between them.  The tail sums and the children's list are needed
// during the walk only, the FP64 transform scratch after it: they share
// storage.
template <typename T, int MW>
struct BwdWarpSmem {
    static constexpr int LD = MW + 1;  // odd row stride: conflict-free column reads
    T R[MW * LD];                      // R[row * LD + slot]
    T A[MW * LD];                      // A[row * LD + col] (symmetric), R's row basis
    union {
        struct {
            T Wt[(MW + 1) * LD];  // Wt[r * LD + slot] = sum_{t >= r} R[t][slot]^2
            T P[MW];              // alpha of the current prefix's children, by rank
            int cl[MW];           // their slots, by rank
        };
        double Y[MW * LD];  // R_T^{-1} A, then Gbar_sub (positions)
    };
    double dinv[MW];  // 1 / R_T[p][p] by position
    int var_at_pos[MW];
    int slot_at_pos[MW];
    unsigned char ups[kStepTab];  // Upsilon(Q): the swap position of every step
};

__device__ __forceinline__ float rsqrt_t(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsqrt_t(double x) { return rsqrt(x); }

template <typename T>
__device__ __forceinline__ void givens_cs(T a, T b, T& c, T& s, T& rho) {
    const T r2 = a * a + b * b;
    if (r2 > T(0)) {
        const T inv = rsqrt_t(r2);
        c = a * inv;
        s = b * inv;
        rho = r2 * inv;
    } else {
        c = T(1);
        s = T(0);
        rho = T(0);
    }
}

// alpha = w n / RSS: the fast reciprocal-multiply in FP32 (2 ulp), IEEE in FP64
__device__ __forceinline__ float fast_div(float x, float y) { return __fdividef(x, y); }
__device__ __forceinline__ double fast_div(double x, double y) { return x / y; }

__device__ __forceinline__ int swapped(int pos, int s) {
    return pos == s ? s + 1 : (pos == s + 1 ? s : pos);
}

// GRC at position s: swap the columns at positions s and s+1, then restore
// triangularity with one rotation of rows s, s+1.  with_A also conjugates A
// (A -> G A G^T): lane j rotates its entries of rows s, s+1; by symmetry
// they are also column j's entries of columns s, s+1, except in the 2 x 2
// block, which lane s rotates on both sides; and the tail sums of row s+1.
// col = the lane's column slot; only the lead half-warp stores.
template <typename T, int MW>
__device__ __forceinline__ void grc(BwdWarpSmem<T, MW>& S, int m, int col, bool lead, int& mypos,
                                    int s, bool with_A) {
    constexpr int LD = MW + 1;
    mypos = swapped(mypos, s);
    const unsigned at_s = __ballot_sync(0xffffffffu, mypos == s);
    const int ls = __ffs(at_s) - 1;  // a lead lane: the lowest set bit
    const T a = S.R[s * LD + ls], b = S.R[(s + 1) * LD + ls];
    T c, sn, rho;
    givens_cs(a, b, c, sn, rho);
    const T x = S.R[s * LD + col], y = S.R[(s + 1) * LD + col];
    T ax = T(0), ay = T(0);
    if (with_A) {
        ax = S.A[s * LD + col];
        ay = S.A[(s + 1) * LD + col];
    }
    __syncwarp();
    const T ry = (col == ls) ? T(0) : c * y - sn * x;
    if (lead) {
        S.R[s * LD + col] = (col == ls) ? rho : c * x + sn * y;
        S.R[(s + 1) * LD + col] = ry;
    }
    if (with_A) {
        const T nx = c * ax + sn * ay, ny = c * ay - sn * ax;  // rows of G A
        const T nxs = __shfl_sync(0xffffffffu, nx, s), nxs1 = __shfl_sync(0xffffffffu, nx, s + 1);
        const T nys = __shfl_sync(0xffffffffu, ny, s), nys1 = __shfl_sync(0xffffffffu, ny, s + 1);
        if (lead && col < m && col != s && col != s + 1) {
            S.A[s * LD + col] = nx;
            S.A[(s + 1) * LD + col] = ny;
            S.A[col * LD + s] = nx;
            S.A[col * LD + s + 1] = ny;
        }
        if (lead && col == s) {
            S.A[s * LD + s] = c * nxs + sn * nxs1;
            S.A[s * LD + s + 1] = c * nxs1 - sn * nxs;
            S.A[(s + 1) * LD + s] = c * nys + sn * nys1;
            S.A[(s + 1) * LD + s + 1] = c * nys1 - sn * nys;
        }
        // the rotation keeps R[s][j]^2 + R[s+1][j]^2: only row s+1's tail sum changes
        if (lead) S.Wt[(s + 1) * LD + col] = fma(ry, ry, S.Wt[(s + 2) * LD + col]);
    }
    __syncwarp();
}

// The weight w_f of this lane's family when the prefix has length a0 and the
// lane's column sits at position pos (0 unless that column is a child).  Its
// load is issued one step ahead of the family's rank update.
template <typename T>
__device__ __forceinline__ T family_weight(const BwdArgs& g, const T* __restrict__ w, int col,
                                           int pos, int var, int a0) {
    const int m = g.m;
    const unsigned mask = __reduce_or_sync(0xffffffffu,
                                           (col < m && pos < a0) ? (1u << var) : 0u);
    if (!(col < m && pos >= a0)) return T(0);
    const unsigned low = mask & ((1u << var) - 1u);
    const unsigned high = (mask >> (var + 1)) << var;
    const int64_t slot = ((int64_t)var << (m - 1)) + (int64_t)(low | high);
    return GBN_IN(g.chk, 301, slot, (int64_t)m << (m - 1)) ? w[slot] : T(0);
}

// Families of the current ordering with prefix length a0: every column at a
// position >= a0 is a child (its RSS the tail sum of its slot from row a0),
// the parents are the columns at positions < a0.  Then
// A[r][j] += sum_c alpha_c R[r][c] R[j][c] for rows r, j >= a0 (j = col).
template <typename T, int MW>
__device__ __forceinline__ void emit(BwdWarpSmem<T, MW>& S, const BwdArgs& g, int col, int ph,
                                     int mypos, int a0, T wf) {
    constexpr int LD = MW + 1;
    const int m = g.m;
    const bool child = col < m && mypos >= a0;
    T alpha = T(0);
    if (child) {
        const T rss = S.Wt[a0 * LD + col];
        if (rss > T(0)) alpha = fast_div(wf * (T)g.n, rss);
    }
    const unsigned cm = __ballot_sync(0xffffffffu, child && alpha != T(0)) &
                        (MW == 32 ? 0xffffffffu : ((1u << MW) - 1u));
    // the children as a list (warp-uniform): each child lane puts its slot and alpha at
    // its rank
    if (ph == 0 && ((cm >> col) & 1u)) {
        const int rank = __popc(cm & ((1u << col) - 1u));
        S.cl[rank] = col;
        S.P[rank] = alpha;
    }
    __syncwarp();
    if (!cm) return;
    const int nc = __popc(cm);
    if constexpr (MW == 16) {
        // children outer, this half's rows ph, ph + 2, ... in registers: per child one
        // t_i = alpha_i R[col][c_i], then one broadcast load and one FMA per row
        T acc[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[j] = T(0);
        for (int i = 0; i < nc; ++i) {
            const int c = S.cl[i];
            const T ti = S.P[i] * S.R[col * LD + c];
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[j] = fma(ti, S.R[(ph + 2 * j) * LD + c], acc[j]);
        }
        if (col >= a0 && col < m) {
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int r = ph + 2 * j;
                if (r >= a0 && r < m) S.A[r * LD + col] += acc[j];
            }
        }
    } else {  // MW = 32: rows outer, the children (slot c_i and t_i) in registers
        int cs[MW];
        T t[MW];
#pragma unroll
        for (int i = 0; i < MW; ++i) {
            if (i < nc) {
                const int c = S.cl[i];
                cs[i] = c;
                t[i] = S.P[i] * S.R[col * LD + c];
            }
        }
        if (col >= a0 && col < m) {
            for (int r = a0; r < m; ++r) {
                const T* Rr = S.R + r * LD;
                T acc0 = S.A[r * LD + col], acc1 = T(0);
#pragma unroll
                for (int i = 0; i < MW; i += 2) {
                    if (i < nc) acc0 = fma(t[i], Rr[cs[i]], acc0);
                    if (i + 1 < nc) acc1 = fma(t[i + 1], Rr[cs[i + 1]], acc1);
                }
                S.A[r * LD + col] = acc0 + acc1;
            }
        }
    }
    __syncwarp();
}

// The sub-walks lw, lw + nw, ... of one dataset, by one warp; Gbar_sub of
// each is added to this warp's FP64 partial sum (partials slot lw).
template <typename T, int MW>
__device__ __forceinline__ void bwd_subwalks(const BwdArgs& g, int64_t lw, int64_t nw,
                                             BwdWarpSmem<T, MW>& S) {
    constexpr int LD = MW + 1;
    constexpr int kPh = 32 / MW;
    const int lane = threadIdx.x & 31;
    const int col = lane & (MW - 1);
    const int ph = lane / MW;
    const bool lead = ph == 0;
    const int m = g.m, k = g.k, Q = g.Q;
    const T* __restrict__ w = static_cast<const T*>(g.w);
    double* part = g.partials + lw * (int64_t)(m * m);
    for (int e = lane; e < m * m; e += 32) part[e] = 0.0;
    const int64_t nsteps = ((int64_t)1 << Q) - Q - 1;
    const unsigned hmask = k > 0 ? (unsigned)((1ull << k) - 1ull) : 0u;
    const bool tab = nsteps <= kStepTab;  // the sequence once per warp, else step by step
    if (tab)
        for (int64_t t = lane; t < nsteps; t += 32) S.ups[t] = (unsigned char)upsilon_at(Q, t);
    __syncwarp();
    auto ups_at = [&](int64_t t) { return tab ? (int)S.ups[t] : upsilon_at(Q, t); };

    for (int64_t sub = lw; sub < g.n_sub; sub += nw) {
        const unsigned F = (unsigned)sub;  // bit v set: fixed variable v is in the front set
        const int d = __popc(F);
        // checkpoint: R0 in plan order, slot = plan position
        for (int r = ph; r < MW; r += kPh) {
            T v = T(0);
            if (col < m && r < m && GBN_IN(g.chk, 302, r * m + col, m * m)) v = (T)g.R0[r * m + col];
            S.R[r * LD + col] = v;
            S.A[r * LD + col] = T(0);
        }
        const int myvar = col < m ? g.order[col] : 0;
        int mypos = col;
        // target position in [F ascending, L = k..m-1, (H \ F) ascending]
        int tpos = col;
        if (col < m) {
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
            const int owner = __ffs(__ballot_sync(0xffffffffu, col < m && tpos == p)) - 1;
            const int q = __shfl_sync(0xffffffffu, mypos, owner);
            for (int s = q - 1; s >= p; --s) grc(S, m, col, lead, mypos, s, false);
        }
        if (lead) {  // tail sums of every slot from every row
            T acc = T(0);
            S.Wt[MW * LD + col] = T(0);
            for (int r = MW - 1; r >= 0; --r) {
                const T z = S.R[r * LD + col];
                acc = fma(z, z, acc);
                S.Wt[r * LD + col] = acc;
            }
        }
        __syncwarp();
        // the sub-walk: families at the root, then one new prefix per swap; each
        // step's weights are loaded while the previous step's update runs
        int s = nsteps > 0 ? d + ups_at(0) - 1 : 0;
        T wf = family_weight(g, w, col, mypos, myvar, d);
        for (int a0 = d; a0 <= d + Q; ++a0) {
            T wn = T(0);
            if (a0 < d + Q)
                wn = family_weight(g, w, col, mypos, myvar, a0 + 1);
            else if (nsteps > 0)
                wn = family_weight(g, w, col, swapped(mypos, s), myvar, s + 1);
            emit(S, g, col, ph, mypos, a0, wf);
            wf = wn;
        }
        for (int64_t t = 0; t < nsteps; ++t) {
            grc(S, m, col, lead, mypos, s, true);
            T wn = T(0);
            int s_next = 0;
            if (t + 1 < nsteps) {
                s_next = d + ups_at(t + 1) - 1;
                wn = family_weight(g, w, col, swapped(mypos, s_next), myvar, s_next + 1);
            }
            emit(S, g, col, ph, mypos, s + 1, wf);
            wf = wn;
            s = s_next;
        }
        // Gbar_sub = R_T^{-1} A R_T^{-T} in FP64, columns by final position
        if (lead && col < m) {
            S.var_at_pos[mypos] = myvar;
            S.slot_at_pos[mypos] = col;
        }
        __syncwarp();
        const double diag = col < m ? (double)S.R[col * LD + S.slot_at_pos[col]] : 1.0;
        if (__any_sync(0xffffffffu, diag == 0.0)) {  // singular factor: flag, skip
            if (lane == 0) atomicOr(g.status, GBN_STATUS_RANK_DEFICIENT);
            continue;
        }
        if (lead) S.dinv[col] = 1.0 / diag;  // every pivot's reciprocal at once
        __syncwarp();
        if (lead && col < m) {  // Y = R_T^{-1} A, lane = column of A
            for (int p = m - 1; p >= 0; --p) {
                double acc = (double)S.A[p * LD + col];
                for (int q = p + 1; q < m; ++q)
                    acc -= (double)S.R[p * LD + S.slot_at_pos[q]] * S.Y[q * LD + col];
                S.Y[p * LD + col] = acc * S.dinv[p];
            }
        }
        __syncwarp();
        if (lead && col < m) {  // Gbar_sub = Y R_T^{-T}, lane = row, in place
            for (int p = m - 1; p >= 0; --p) {
                double acc = S.Y[col * LD + p];
                for (int q = p + 1; q < m; ++q)
                    acc -= (double)S.R[p * LD + S.slot_at_pos[q]] * S.Y[col * LD + q];
                S.Y[col * LD + p] = acc * S.dinv[p];
            }
            const int vr = S.var_at_pos[col];
            for (int q = 0; q < m; ++q) part[vr * m + S.var_at_pos[q]] += S.Y[col * LD + q];
        }
        __syncwarp();
    }
}

// One dataset: warp wid takes sub-walks wid, wid + warps, ...
template <typename T, int MW>
__global__ void __launch_bounds__(32 * kBwdWarps) bwd_walk_kernel(BwdArgs g) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    BwdWarpSmem<T, MW>& S = reinterpret_cast<BwdWarpSmem<T, MW>*>(smem_raw)[threadIdx.x >> 5];
    grid_dep_wait();
    const int64_t wid = (int64_t)blockIdx.x * kBwdWarps + (threadIdx.x >> 5);
    if (wid < g.warps) bwd_subwalks<T, MW>(g, wid, g.warps, S);
}

// A batch: warp gw belongs to dataset d with warp_prefix[d] <= gw < warp_prefix[d+1].
template <typename T, int MW>
__global__ void __launch_bounds__(32 * kBwdWarps)
    bwd_walk_kernel_b(const BwdArgs* __restrict__ args, const int64_t* __restrict__ warp_prefix,
                      int B) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    BwdWarpSmem<T, MW>& S = reinterpret_cast<BwdWarpSmem<T, MW>*>(smem_raw)[threadIdx.x >> 5];
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
    bwd_subwalks<T, MW>(g, gw - warp_prefix[lo], g.warps, S);
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
    if (o.score == GBN_SCORE_BGE) return GBN_ERR_OPTS;  // the adjoint is that of n ln RSS
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

template <typename T, int MW>
int launch_bwd_w(const BwdPlan& b, const double* X, const void* w, double* grad, char* ws,
                 cudaStream_t stream) {
    const Plan& p = b.p;
    BwdArgs g = bwd_args(p, ws, X, w, grad, b.Qb, b.n_sub, b.warps,
                         reinterpret_cast<double*>(ws + b.off_partials),
                         reinterpret_cast<double*>(ws + b.off_gsym),
                         reinterpret_cast<double*>(ws + b.off_muv));
    const size_t smem = sizeof(BwdWarpSmem<T, MW>) * kBwdWarps;
    if (cudaFuncSetAttribute(bwd_walk_kernel<T, MW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess)
        return GBN_ERR_CUDA;
    const unsigned blocks = (unsigned)((b.warps + kBwdWarps - 1) / kBwdWarps);
    const cudaError_t e[] = {
        launch_dep(bwd_walk_kernel<T, MW>, dim3(blocks), dim3(32 * kBwdWarps), smem, stream, g),
        launch_dep(bwd_reduce_kernel, dim3(8), dim3(256), 0, stream, (const double*)g.partials,
                   g.warps, p.m, g.mu_plan, p, g.gsym, g.mu_var),
        launch_dep(bwd_grad_kernel, dim3(304), dim3(256), 0, stream, X, p.n, p.m,
                   (const double*)g.gsym, (const double*)g.mu_var, grad)};
    for (cudaError_t x : e)
        if (x != cudaSuccess) return GBN_ERR_CUDA;
    return GBN_OK;
}

template <typename T>
int launch_bwd(const BwdPlan& b, const double* X, const void* w, double* grad, char* ws,
               cudaStream_t stream) {
    return b.p.m <= 16 ? launch_bwd_w<T, 16>(b, X, w, grad, ws, stream)
                       : launch_bwd_w<T, 32>(b, X, w, grad, ws, stream);
}

// The walk over datasets [0, B) of args with one width.
template <typename T, int MW>
int launch_bwd_walk_group(const BwdArgs* args, const int64_t* warp_prefix, int B, int64_t warps,
                          cudaStream_t stream) {
    if (B == 0 || warps == 0) return GBN_OK;
    const size_t smem = sizeof(BwdWarpSmem<T, MW>) * kBwdWarps;
    if (cudaFuncSetAttribute(bwd_walk_kernel_b<T, MW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess)
        return GBN_ERR_CUDA;
    const unsigned blocks = (unsigned)((warps + kBwdWarps - 1) / kBwdWarps);
    return launch_rc(launch_plain(bwd_walk_kernel_b<T, MW>, dim3(blocks), dim3(32 * kBwdWarps),
                                  smem, stream, args, warp_prefix, B));
}

template <typename T>
int launch_bwd_batched_t(const BwdArgs* args, const int64_t* prefix, int B, int B_narrow,
                         int64_t warps_narrow, int64_t warps_wide, cudaStream_t stream) {
    int rc = launch_bwd_walk_group<T, 16>(args, prefix, B_narrow, warps_narrow, stream);
    if (rc == GBN_OK)
        rc = launch_bwd_walk_group<T, 32>(args + B_narrow, prefix + B_narrow + 1, B - B_narrow,
                                          warps_wide, stream);
    if (rc) return rc;
    const cudaError_t e[] = {
        launch_plain(bwd_reduce_kernel_b, dim3(4, (unsigned)B), dim3(256), 0, stream, args),
        launch_plain(bwd_grad_kernel_b, dim3(32, (unsigned)B), dim3(256), 0, stream, args)};
    for (cudaError_t x : e)
        if (x != cudaSuccess) return GBN_ERR_CUDA;
    return GBN_OK;
}

}  // namespace

int bwd_subwalk_plan(int m, int q_requested, int* Qb, int64_t* n_sub, int64_t* warps) {
    int q = q_requested > 0 ? q_requested : m - 9;
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

int launch_bwd_batched(const BwdArgs* args, const int64_t* prefix, int B, int B_narrow,
                       int64_t warps_narrow, int64_t warps_wide, int precision,
                       cudaStream_t stream) {
    return precision ? launch_bwd_batched_t<double>(args, prefix, B, B_narrow, warps_narrow,
                                                    warps_wide, stream)
                     : launch_bwd_batched_t<float>(args, prefix, B, B_narrow, warps_narrow,
                                                   warps_wide, stream);
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

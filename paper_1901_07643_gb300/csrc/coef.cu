// Least-squares coefficients of listed families (Sec. 1.1: the regression of
// a child on a parent set), from the same initial QR decomposition R0 that
// the walk starts from (Sec. 2).
//
// Xc = Q R0 with Q orthonormal, so for a family (c, S) the least-squares
// problem min |Xc_c - Xc_S b| is the m-row problem min |R0_c - R0_S b|.  One
// warp per family gathers R0's columns for S (ascending variable) and c into
// an m x (|S|+1) tile, triangularises it with |S| Householder reflections
// (FP64), takes the residual sum of squares from the trailing entries of the
// last column and solves the |S| x |S| triangle for b by back substitution.
// The intercept of the uncentred regression is mean_c - sum_v b_v mean_v.
// Numerically dependent parents -- a pivot |r_jj| at most 1e-12 times the
// norm of parent j's column -- give NaN coefficients (the RSS is kept).
#include <math.h>

#include "gbn_internal.cuh"

namespace gbn {
namespace {

constexpr int kCoefWarps = 4;
constexpr int kLdC = 33;

__device__ __forceinline__ double warp_sum(double x) {
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

__global__ void __launch_bounds__(32 * kCoefWarps)
    coef_kernel(const Plan p, char* ws, const int32_t* __restrict__ child,
                const uint64_t* __restrict__ parents, int64_t count, double* __restrict__ beta,
                double* __restrict__ rss_out) {
    __shared__ double M[kCoefWarps * 32 * kLdC];
    __shared__ int pos_of[32];
    __shared__ double mu_var[32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, m = p.m;
    grid_dep_wait();
    const double* mu = reinterpret_cast<const double*>(ws + p.off_mu);  // plan order
    if (threadIdx.x < m) {
        pos_of[p.order[threadIdx.x]] = threadIdx.x;
        mu_var[p.order[threadIdx.x]] = mu[threadIdx.x];
    }
    __syncthreads();
    const double* R0 = reinterpret_cast<const double*>(ws + p.off_r0);
    int* status = reinterpret_cast<int*>(ws + p.off_status);
    double* Mw = M + warp * 32 * kLdC;
    const double nan = __longlong_as_double(0x7ff8000000000000ll);
    for (int64_t f = (int64_t)blockIdx.x * kCoefWarps + warp; f < count;
         f += (int64_t)gridDim.x * kCoefWarps) {
        const int c = child[f];
        const uint64_t S = parents[f];
        double* bf = beta + f * (int64_t)(m + 1);
        const bool valid = c >= 0 && c < m && !((S >> c) & 1ull) && (m >= 64 || (S >> m) == 0ull);
        if (!valid) {  // an invalid family: NaN outputs, status bit
            if (lane <= m) bf[lane] = nan;
            if (lane == 0) {
                if (rss_out) rss_out[f] = nan;
                atomicOr(status, GBN_STATUS_BAD_FAMILY);
            }
            continue;
        }
        const int k = __popcll(S);
        int j = 0;
        int var_of_col[32];
        double norm[32];
        for (uint64_t rest = S; rest; rest &= rest - 1, ++j) {
            const int v = __ffsll((long long)rest) - 1;
            var_of_col[j] = v;
            const double x = lane < m ? R0[lane * m + pos_of[v]] : 0.0;
            Mw[lane * kLdC + j] = x;
            norm[j] = sqrt(warp_sum(x * x));
        }
        Mw[lane * kLdC + k] = lane < m ? R0[lane * m + pos_of[c]] : 0.0;
        __syncwarp();
        for (int jj = 0; jj < k; ++jj) {  // reflection zeroing column jj below row jj
            const double x = (lane >= jj && lane < m) ? Mw[lane * kLdC + jj] : 0.0;
            const double nrm2 = warp_sum(x * x);
            if (nrm2 == 0.0) continue;  // a zero column: its pivot stays 0 (flagged below)
            const double xj = __shfl_sync(0xffffffffu, x, jj);
            const double nrm = sqrt(nrm2);
            const double alpha = xj >= 0.0 ? -nrm : nrm;
            const double v = (lane == jj) ? xj - alpha : x;
            const double vtv = nrm2 - xj * xj + (xj - alpha) * (xj - alpha);
            for (int l = jj; l <= k; ++l) {
                const double y = (lane >= jj && lane < m) ? Mw[lane * kLdC + l] : 0.0;
                const double dot = warp_sum(v * y);
                if (lane >= jj && lane < m) Mw[lane * kLdC + l] = y - (2.0 * dot / vtv) * v;
            }
            __syncwarp();
        }
        const double t = (lane >= k && lane < m) ? Mw[lane * kLdC + k] : 0.0;
        const double rss = warp_sum(t * t);
        // back substitution on lane 0 (k <= 31 unknowns), then the scatter
        double b[32];
        bool singular = false;
        if (lane == 0) {
            for (int i = k - 1; i >= 0; --i) {
                double s = Mw[i * kLdC + k];
                for (int l = i + 1; l < k; ++l) s -= Mw[i * kLdC + l] * b[l];
                const double d = Mw[i * kLdC + i];
                if (!(fabs(d) > 1e-12 * norm[i])) singular = true;
                b[i] = s / d;
            }
        }
        singular = __shfl_sync(0xffffffffu, singular ? 1 : 0, 0) != 0;
        __syncwarp();
        if (lane == 0) {
            for (int v = 0; v <= m; ++v) bf[v] = 0.0;
            double icpt = mu_var[c];
            for (int i = 0; i < k; ++i) {
                const double bi = singular ? nan : b[i];
                bf[var_of_col[i]] = bi;
                icpt -= bi * mu_var[var_of_col[i]];
            }
            bf[m] = icpt;
            if (rss_out) rss_out[f] = rss;
            if (singular) atomicOr(status, GBN_STATUS_RANK_DEFICIENT);
        }
        __syncwarp();
    }
}

}  // namespace
}  // namespace gbn

using namespace gbn;

extern "C" int givensbn_coefficients_workspace_size(int64_t n, int32_t m, const givensbn_opts* opts,
                                                    size_t* bytes) {
    if (!bytes) return GBN_ERR_NULL;
    givensbn_opts o;
    givensbn_default_opts(&o);
    if (opts) o = *opts;
    o.precision = 0;
    o.q = 0;
    o.tune_cache = nullptr;
    o.score = GBN_SCORE_BIC;  // coefficients do not depend on the score
    Plan p;
    const int rc = make_plan(n, m, &o, &p);
    if (rc) return rc;
    *bytes = p.off_leaves;  // the R0 stage only
    return GBN_OK;
}

extern "C" int givensbn_family_coefficients(const double* X, int64_t n, int32_t m,
                                            const int32_t* child, const uint64_t* parents,
                                            int64_t count, double* beta, double* rss,
                                            const givensbn_opts* opts) {
    if (!opts) return GBN_ERR_NULL;
    givensbn_opts o = *opts;
    o.precision = 0;
    o.q = 0;
    o.tune_cache = nullptr;
    o.score = GBN_SCORE_BIC;  // coefficients do not depend on the score
    o.fixup_tau = 0.0;
    Plan p;
    int rc = make_plan(n, m, &o, &p);
    if (rc) return rc;
    if (count < 0) return GBN_ERR_BATCH;
    if (!X || (count > 0 && (!child || !parents || !beta))) return GBN_ERR_NULL;
    if (((uintptr_t)X & 7u) || ((uintptr_t)beta & 7u) || ((uintptr_t)rss & 7u) ||
        ((uintptr_t)parents & 7u) || ((uintptr_t)child & 3u))
        return GBN_ERR_ALIGN;
    if (!opts->workspace || opts->workspace_bytes < p.off_leaves) return GBN_ERR_WORKSPACE;
    if ((uintptr_t)opts->workspace & 255u) return GBN_ERR_ALIGN;
    char* ws = static_cast<char*>(opts->workspace);
    cudaStream_t stream = static_cast<cudaStream_t>(opts->stream);
    if ((rc = launch_r0(p, X, ws, stream))) return rc;
    if (count == 0) return GBN_OK;
    const int64_t want = (count + kCoefWarps - 1) / kCoefWarps;
    const unsigned blocks = (unsigned)(want < 4096 ? want : 4096);
    return launch_rc(launch_dep(coef_kernel, dim3(blocks), dim3(32 * kCoefWarps), 0, stream, p, ws,
                                child, parents, count, beta, rss));
}

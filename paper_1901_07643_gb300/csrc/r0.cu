// Initial QR decomposition R0 of the centred data (the "initial QRD" that the
// walk starts from, Sec. 2 and Sec. 1.3), computed as CholeskyQR2 in FP64:
//   means:  mu = column means (per-panel partial sums, then one reduction)
//   pass 1: G1 = Xc^T Xc (row panels, then summed over panels), R1 = chol(G1)
//   pass 2: Q1 = Xc R1^{-1} (explicit triangular inverse), G2 = Q1^T Q1,
//           R2 = chol(G2), R0 = R2 R1.
// Pass 2 exists for ill-conditioned data: an RSS read from R1 has relative
// error about eps ||x_c||^2 / RSS, the RSS of the explicitly orthogonalised Q1
// about eps ||x_c|| / sqrt(RSS).  When every column's smallest possible RSS
// (on all the other columns, 1 / (G1^{-1})_cc) is at least kOnePassRatio of its
// sum of squares, R1 is already that accurate (eps / 1e-3, about 1e-13): the
// pass-1 Cholesky kernel then writes R0 = R1 and raises a flag in the status
// block, and the pass-2 kernels return at once.
// Columns are taken in the plan's order (the order the sub-walk tree decides
// variables in), so R0 is the R factor of Xc[:, order].
#include <math.h>

#include <algorithm>

#include "gbn_internal.cuh"

namespace gbn {
namespace {

constexpr int kPanelChunk = 32;  // rows staged in shared memory at a time (even: see gram_body)
constexpr int kLd = 33;          // row stride of the m x m shared-memory tiles
constexpr int kRedThreads = 1024; // threads of the reduction kernels
constexpr int kColsumThreads = 128;  // threads of a column-sum block (16 blocks per SM)
constexpr int kCholThreads = 1024;  // threads of the Cholesky kernel (one barrier per column)
constexpr double kOnePassRatio = 1e-3;  // smallest RSS / sum of squares for one pass

// All shared-memory tiles here are flat 1-D arrays indexed as [row * kLd + col]:
// with this toolchain, runtime-indexed two-dimensional __shared__ arrays were
// mis-addressed in sm_103 code while the same accesses on flat arrays were not.

__device__ __forceinline__ void colsum_body(int b, const double* __restrict__ X, int64_t n, int m,
                                            int rows_per, double* __restrict__ colsum, int panels,
                                            unsigned long long* chk) {
    __shared__ double red[256];
    __shared__ int rede[256];
    const int64_t r0 = (int64_t)b * rows_per;
    const int64_t r1 = (r0 + rows_per < n) ? r0 + rows_per : n;
    const int per = blockDim.x / m;  // row lanes
    const int j = threadIdx.x % m;
    const int rl = threadIdx.x / m;
    double s = 0.0;
    int emax = 0;  // the largest biased binary exponent of |x| (integer operations only)
    if (rl < per)
        for (int64_t t = r0 + rl; t < r1; t += per)
            if (GBN_IN(chk, 101, t * m + j, n * m)) {
                const double x = X[t * m + j];
                s += x;
                emax = max(emax, (int)((__double_as_longlong(x) >> 52) & 0x7ff));
            }
    if (GBN_IN(chk, 102, threadIdx.x, 256)) {
        red[threadIdx.x] = (rl < per) ? s : 0.0;
        rede[threadIdx.x] = (rl < per) ? emax : 0;
    }
    __syncthreads();
    if (threadIdx.x < m) {
        double acc = 0.0;
        int em = 0;
        for (int l = 0; l < per; ++l)
            if (GBN_IN(chk, 103, l * m + threadIdx.x, 256)) {
                acc += red[l * m + threadIdx.x];
                em = max(em, rede[l * m + threadIdx.x]);
            }
        if (GBN_IN(chk, 104, (int64_t)b * m + threadIdx.x, (int64_t)panels * m)) {
            colsum[(int64_t)b * m + threadIdx.x] = acc;
            // the exponent maxima follow the sums, one integer per double slot
            reinterpret_cast<long long*>(colsum)[(int64_t)(panels + b) * m + threadIdx.x] = em;
        }
    }
}

// mu[j] = column mean of variable order[j] (zero when centring is off), and
// mu[32 + j] = that column's scale exponent: the unbiased binary exponent of its
// largest |x| (0 for a zero column).  The Gram passes hold each centred column
// times 2^-exponent (|y| < 4), so that their FP32-pair arithmetic stays inside
// FP32's range for data of any scale.  Threads split the panels of each column.
__device__ __forceinline__ void mean_body(const double* __restrict__ colsum, int panels, int m,
                                          int64_t n, int center, const Plan& plan,
                                          double* __restrict__ mu, unsigned long long* chk) {
    __shared__ double red[kRedThreads];
    __shared__ int rede[kRedThreads];
    const int per = kRedThreads / m;  // threads per column
    const int j = threadIdx.x % m;
    const int l = threadIdx.x / m;
    const long long* cexp = reinterpret_cast<const long long*>(colsum) + (int64_t)panels * m;
    double s = 0.0;
    int em = 0;
    if (l < per) {
        const int v = plan.order[j];
        for (int b = l; b < panels; b += per)
            if (GBN_IN(chk, 131, (int64_t)b * m + v, (int64_t)panels * m)) {
                if (center) s += colsum[(int64_t)b * m + v];
                em = max(em, (int)cexp[(int64_t)b * m + v]);
            }
    }
    red[threadIdx.x] = (l < per) ? s : 0.0;
    rede[threadIdx.x] = (l < per) ? em : 0;
    __syncthreads();
    if (threadIdx.x < m) {
        double acc = 0.0;
        int e = 0;
        for (int t = 0; t < per; ++t) {
            acc += red[t * m + threadIdx.x];
            e = max(e, rede[t * m + threadIdx.x]);
        }
        mu[threadIdx.x] = center ? acc / (double)n : 0.0;
        mu[32 + threadIdx.x] = e > 0 ? (double)(e - 1023) : 0.0;
    }
}

// FP32-pair ("double-float") arithmetic for the panel Grams: a value is the
// unevaluated sum hi + lo of two floats (47 significant bits here), products by
// Dekker's method with FMA and sums by Knuth's TwoSum (Dekker, "A floating-point
// technique for extending the available precision", Numer. Math. 18, 1971;
// Knuth, TAOCP vol. 2, 4.2.2).  GB300 runs FP32 at 74 times its FP64 rate and
// the Gram passes were bound by the FP64 pipe; here the centring subtraction
// and the panel's final sums are the only FP64 operations.  The _rn intrinsics
// keep the compiler from fusing the steps of the error-free transformations.
//
// y * 2^-s split into floats by integer operations (FP64 <-> FP32 conversions
// also run on the slow FP64 pipe): hi = the sign, exponent and top 23 mantissa
// bits; lo = the remaining 29 bits, normalised and truncated to 24.  Parts below
// FP32's normal range (2^-126, relative to a column whose largest |x| is scaled
// to [1, 2)) are dropped.
__device__ __forceinline__ float2 df_split_int(double y, int s) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(y);
    const int eb = (int)((b >> 52) & 0x7ff);
    if (eb == 0) return make_float2(0.f, 0.f);  // zero (or subnormal)
    const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
    const int E = eb - 1023 - s;  // unbiased exponent of y * 2^-s
    const int ehi = E + 127;
    if (ehi <= 0) return make_float2(0.f, 0.f);
    const unsigned long long mant = b & 0x000FFFFFFFFFFFFFull;
    const float hi = __uint_as_float(sign | ((unsigned)ehi << 23) | (unsigned)(mant >> 29));
    const unsigned r = (unsigned)(mant & 0x1FFFFFFFull);  // value r * 2^(E - 52)
    float lo = 0.f;
    if (r) {
        const int lz = __clz(r);  // >= 3
        const int elo = E - 52 + (31 - lz) + 127;
        if (elo > 0) lo = __uint_as_float(sign | ((unsigned)elo << 23) | ((r << (lz + 1)) >> 9));
    }
    return make_float2(hi, lo);
}

__device__ __forceinline__ float2 df_split(double x) {  // via conversions (a few per block)
    const float h = __double2float_rn(x);
    return make_float2(h, __double2float_rn(x - (double)h));
}

// (sh, sl) += a * b
__device__ __forceinline__ void df_fma(float2 a, float2 b, float& sh, float& sl) {
    const float p = __fmul_rn(a.x, b.x);
    float e = __fmaf_rn(a.x, b.x, -p);  // the product's rounding error, exactly
    e = __fmaf_rn(a.x, b.y, e);
    e = __fmaf_rn(a.y, b.x, e);
    const float t = __fadd_rn(sh, p);  // TwoSum(sh, p) = t + w exactly
    const float v = __fsub_rn(t, sh);
    const float w = __fadd_rn(__fsub_rn(sh, __fsub_rn(t, v)), __fsub_rn(p, v));
    const float lo = __fadd_rn(sl, __fadd_rn(e, w));
    sh = __fadd_rn(t, lo);  // renormalise
    sl = __fsub_rn(lo, __fsub_rn(sh, t));
}

// Partial Gram of one row panel: sum over its rows of y y^T (upper triangle,
// packed by pairs i <= j), where y is the centred row in plan order (centred in
// FP64, scaled by the column's power of two and split into an FP32 pair), or for
// pass 2 the row of Q1 = y R1^{-1} (Rinv = R1^{-1}, upper triangular; Q1's
// entries are at most about 1), both accumulated in FP32 pairs.  Each pair's
// thread adds the panel's even rows into one sum and the odd rows into another
// (rows staged kPanelChunk at a time; the chunk size is even, so the split,
// and the result, do not depend on it).  The panel's sums leave as FP64,
// pass 1's scaled back exactly.
__device__ __forceinline__ void gram_body(int blk, const double* __restrict__ X, int64_t n, int m,
                                          int rows_per, const double* __restrict__ mu_g, int panels,
                                          const double* __restrict__ Rinv, const Plan& plan,
                                          double* __restrict__ gram, unsigned long long* chk) {
    __shared__ double mu[32];
    __shared__ int sx[32];  // column scale exponents: y' = y 2^-sx
    __shared__ float2 rows[kPanelChunk * kLd];
    __shared__ float2 qrows[kPanelChunk * kLd];
    __shared__ float2 ri[32 * kLd];
    __shared__ int ord[32];  // the plan's column order (the plan may live in global memory)
    const int tid = threadIdx.x;
    if (tid < m) {
        mu[tid] = mu_g[tid];
        sx[tid] = (int)mu_g[32 + tid];
        ord[tid] = plan.order[tid];
    }
    __syncthreads();
    if (Rinv)  // row i of R1^{-1} times 2^sx[i], so that y' Rinv' = y R1^{-1}
        for (int e = tid; e < m * m; e += blockDim.x)
            if (GBN_IN(chk, 112, (e / m) * kLd + e % m, 32 * kLd))
                ri[(e / m) * kLd + e % m] = df_split(ldexp(Rinv[e], sx[e / m]));
    const int npair = m * (m + 1) / 2;
    int pi = 0, pj = 0;
    if (tid < npair) {  // unpack pair index -> (i, j), i <= j
        int e = tid, i = 0;
        while (e >= m - i) {
            e -= m - i;
            ++i;
        }
        pi = i;
        pj = i + e;
    }
    float h0 = 0.f, l0 = 0.f, h1 = 0.f, l1 = 0.f;
    const int64_t r0 = (int64_t)blk * rows_per;
    const int64_t rend = (r0 + rows_per < n) ? r0 + rows_per : n;
    const float2* src = Rinv ? qrows : rows;
    __syncthreads();
    for (int64_t c0 = r0; c0 < rend; c0 += kPanelChunk) {
        const int cnt = (rend - c0 < kPanelChunk) ? (int)(rend - c0) : kPanelChunk;
        for (int e = tid; e < cnt * m; e += blockDim.x) {
            const int t = e / m, j = e % m;
            const int64_t xi = (c0 + t) * m + ord[j];
            if (GBN_IN(chk, 113, xi, n * m) && GBN_IN(chk, 114, t * kLd + j, kPanelChunk * kLd))
                rows[t * kLd + j] = df_split_int(X[xi] - mu[j], sx[j]);
        }
        __syncthreads();
        if (Rinv) {  // Q1 rows: q[t][j] = sum_{i <= j} y[t][i] Rinv[i][j], one entry per thread
            for (int e = tid; e < cnt * m; e += blockDim.x) {
                const int t = e / m, j = e % m;
                float sh = 0.f, sl = 0.f;
                for (int i = 0; i <= j; ++i) df_fma(rows[t * kLd + i], ri[i * kLd + j], sh, sl);
                qrows[t * kLd + j] = make_float2(sh, sl);
            }
            __syncthreads();
        }
        if (tid < npair) {
            int t = 0;
            for (; t + 1 < cnt; t += 2) {
                df_fma(src[t * kLd + pi], src[t * kLd + pj], h0, l0);
                df_fma(src[(t + 1) * kLd + pi], src[(t + 1) * kLd + pj], h1, l1);
            }
            if (t < cnt) df_fma(src[t * kLd + pi], src[t * kLd + pj], h0, l0);
        }
        __syncthreads();
    }
    if (tid < npair && GBN_IN(chk, 115, (int64_t)blk * npair + tid, (int64_t)panels * npair)) {
        const double g = ((double)h0 + (double)l0) + ((double)h1 + (double)l1);
        gram[(int64_t)blk * npair + tid] = Rinv ? g : ldexp(g, sx[pi] + sx[pj]);
    }
}

// Sum of the panel Grams for pairs [32 g, 32 g + 32): lane l of warp w adds
// pair 32 g + l over panels w, w + 32, ... (the loads of a warp contiguous),
// then warp 0 adds the 32 slice sums in a fixed order.  GB300's FP64 rate is
// low (two FMAs per clock per SM), so the sum is spread over blocks.
__device__ __forceinline__ void gram_sum_body(int g, const double* __restrict__ gram, int panels,
                                              int m, double* __restrict__ gsum,
                                              unsigned long long* chk) {
    __shared__ double part[32 * 33];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int npair = m * (m + 1) / 2;
    const int e = g * 32 + lane;
    double a0 = 0.0, a1 = 0.0;
    if (e < npair) {
        int b = w;
        for (; b + 32 < panels; b += 64) {
            if (GBN_IN(chk, 121, (int64_t)(b + 32) * npair + e, (int64_t)panels * npair)) {
                a0 += gram[(int64_t)b * npair + e];
                a1 += gram[(int64_t)(b + 32) * npair + e];
            }
        }
        if (b < panels && GBN_IN(chk, 122, (int64_t)b * npair + e, (int64_t)panels * npair))
            a0 += gram[(int64_t)b * npair + e];
    }
    part[w * 33 + lane] = a0 + a1;
    __syncthreads();
    if (w == 0 && e < npair) {
        double acc = 0.0;
        for (int k = 0; k < 32; ++k) acc += part[k * 33 + lane];
        gsum[e] = acc;
    }
}

// Cholesky-factor the summed Gram (upper R with R^T R = G, pairs packed by
// rows).  Pass 1 (R1 == nullptr): writes R1 to Rout and its inverse to
// Rinv_out.  Pass 2: the factor is R2 and R0 = R2 * R1 is written to Rout.
// Both the factorisation and the inverse are right-looking with one barrier
// per column: the threads of the row that a step completes scale it at once
// (each forms the pivot's 1/sqrt itself from values nobody writes in that
// step), so the next step reads it final.  The operations and their order
// per element are those of the textbook right-looking forms.
__device__ __forceinline__ void chol_body(const double* __restrict__ gsum, int m,
                                          const double* __restrict__ R1, double* __restrict__ Rout,
                                          double* __restrict__ Rinv_out, int* __restrict__ status,
                                          unsigned long long* chk,
                                          double* __restrict__ R0_one = nullptr,
                                          int* __restrict__ onepass = nullptr) {
    __shared__ double G[32 * kLd];
    __shared__ double R1s[32 * kLd];
    // pair table: pairs (a, b), a <= b, ordered by a, so that the pairs with
    // a > j are a suffix starting at pair_start[j + 1]
    __shared__ short2 pairs[32 * 33 / 2 + 1];
    __shared__ int pair_start[33];
    __shared__ double dinv[32], diag[32];
    const int tid = threadIdx.x;
    const int npair = m * (m + 1) / 2;
    for (int e = tid; e < 32 * kLd; e += blockDim.x) G[e] = 0.0;
    if (R1)
        for (int e = tid; e < m * m; e += blockDim.x) R1s[(e / m) * kLd + e % m] = R1[e];
    if (tid <= m) {
        int st = 0;
        for (int a = 0; a < tid; ++a) st += m - a;
        pair_start[tid] = st;
    }
    for (int e = tid; e < npair; e += blockDim.x) {
        int q = e, a = 0;
        while (q >= m - a) {
            q -= m - a;
            ++a;
        }
        pairs[e] = make_short2((short)a, (short)(a + q));
    }
    __syncthreads();
    for (int e = tid; e < npair; e += blockDim.x) {
        const short2 ab = pairs[e];
        if (GBN_IN(chk, 123, ab.x * kLd + ab.y, 32 * kLd)) G[ab.x * kLd + ab.y] = gsum[e];
    }
    __syncthreads();
    // Cholesky.  Step j (-1 .. m-2) completes row j+1: its owners take the
    // pivot d = G_{j+1,j+1} - r_{j,j+1}^2 (the diagonal is never written
    // during a step: the scaled diagonal goes to diag[]) and scale by 1/sqrt(d).
    for (int j = -1; j < m - 1; ++j) {
        const int r = j + 1;  // the row this step completes
        for (int e = pair_start[r] + tid; e < npair; e += blockDim.x) {
            const short2 ab = pairs[e];
            double v = G[ab.x * kLd + ab.y];
            if (j >= 0) v -= G[j * kLd + ab.x] * G[j * kLd + ab.y];
            if (ab.x == r) {
                double d = G[r * kLd + r];
                if (j >= 0) d -= G[j * kLd + r] * G[j * kLd + r];
                const double inv = d > 0.0 ? rsqrt(d) : 0.0;
                if (ab.y == r) {
                    if (!(d > 0.0)) atomicOr(status, GBN_STATUS_RANK_DEFICIENT);
                    dinv[r] = inv;
                    diag[r] = d * inv;
                } else {
                    G[ab.x * kLd + ab.y] = v * inv;
                }
            } else {
                G[ab.x * kLd + ab.y] = v;
            }
        }
        __syncthreads();
    }
    for (int r = tid; r < m; r += blockDim.x) G[r * kLd + r] = diag[r];
    __syncthreads();
    if (!R1 && Rinv_out) {
        // R^{-1} = B right-looking from the last row: row j of B is B_j / R_jj,
        // then rows i < j lose R_ij * (row j).  Step j updates columns c >= j
        // of rows i < j and completes row j - 1 (scaled by 1/R_{j-1,j-1}).
        double* B = R1s;  // unused in this pass
        for (int e = tid; e < 32 * kLd; e += blockDim.x) B[e] = 0.0;
        __syncthreads();
        for (int e = tid; e < m; e += blockDim.x) B[e * kLd + e] = (e == m - 1) ? dinv[e] : 1.0;
        __syncthreads();
        for (int j = m - 1; j >= 1; --j) {
            const int w = m - j;  // columns j .. m-1
            for (int e = tid; e <= j * w; e += blockDim.x) {
                if (e == j * w) {  // the diagonal of the completed row
                    B[(j - 1) * kLd + (j - 1)] = dinv[j - 1];
                    continue;
                }
                const int i = e / w, c = j + e % w;
                double v = B[i * kLd + c] - G[i * kLd + j] * B[j * kLd + c];
                if (i == j - 1) v *= dinv[j - 1];
                B[i * kLd + c] = v;
            }
            __syncthreads();
        }
        for (int e = tid; e < m * m; e += blockDim.x) {
            const int i = e / m, c = e % m;
            if (GBN_IN(chk, 126, e, m * m)) Rinv_out[e] = (i <= c) ? B[i * kLd + c] : 0.0;
        }
    }
    bool one = false;
    if (!R1 && onepass) {  // is R1 accurate enough to be R0?  (see the top of this file)
        bool ok = true;
        if (tid < m) {
            double cn2 = 0.0, ginv = 0.0;
            for (int i = 0; i <= tid; ++i) cn2 = fma(G[i * kLd + tid], G[i * kLd + tid], cn2);
            for (int j = tid; j < m; ++j) ginv = fma(R1s[tid * kLd + j], R1s[tid * kLd + j], ginv);
            ok = cn2 > 0.0 && ginv > 0.0 && ginv * cn2 <= 1.0 / kOnePassRatio;
        }
        one = __syncthreads_and(ok) != 0;
        if (one && tid == 0) *onepass = 1;
    }
    __syncthreads();
    for (int e = tid; e < m * m; e += blockDim.x) {
        const int i = e / m, j = e % m;
        double v = 0.0;
        if (i <= j) {
            if (R1) {
                for (int l = i; l <= j; ++l) v = fma(G[i * kLd + l], R1s[l * kLd + j], v);
            } else {
                v = G[i * kLd + j];
            }
        }
        if (GBN_IN(chk, 125, e, m * m)) {
            Rout[e] = v;
            if (one) R0_one[e] = v;
        }
    }
}

// Stage pointers of one dataset inside its workspace region.
struct R0Ptrs {
    double *colsum, *mu, *gram, *gsum, *r1, *r1inv, *r0;
    int* status;
    int* onepass;  // set by pass 1 when pass 2 is not needed
    unsigned long long* chk;
};

__device__ __host__ __forceinline__ R0Ptrs r0_ptrs(const Plan& p, char* ws) {
    R0Ptrs q;
    q.colsum = reinterpret_cast<double*>(ws + p.off_colsum);
    q.mu = reinterpret_cast<double*>(ws + p.off_mu);
    q.gram = reinterpret_cast<double*>(ws + p.off_gram);
    q.gsum = reinterpret_cast<double*>(ws + p.off_gsum);
    q.r1 = reinterpret_cast<double*>(ws + p.off_r1);
    q.r1inv = reinterpret_cast<double*>(ws + p.off_r1inv);
    q.r0 = reinterpret_cast<double*>(ws + p.off_r0);
    q.status = reinterpret_cast<int*>(ws + p.off_status);
    q.onepass = reinterpret_cast<int*>(ws + p.off_status + kR0OnePassOffset);
    q.chk = reinterpret_cast<unsigned long long*>(ws + p.off_status + kCheckOffset);
    return q;
}

// Threads of a Gram block: one per column pair (i <= j), in whole warps of 256
// or 512.  The smaller block leaves fewer idle warps at the panel's barriers and
// fits twice as many blocks on an SM; a pair's sum does not depend on it.
inline unsigned gram_threads(int m) { return m * (m + 1) / 2 <= 256 ? 256u : 512u; }

// One dataset: the plan travels as a kernel parameter.
__global__ void colsum_kernel(const Plan p, const double* __restrict__ X, char* ws) {
    const R0Ptrs q = r0_ptrs(p, ws);
    colsum_body(blockIdx.x, X, p.n, p.m, p.rows_per_panel, q.colsum, p.panels, q.chk);
}
__global__ void __launch_bounds__(kRedThreads) mean_kernel(const Plan p, char* ws) {
    grid_dep_wait();
    grid_dep_launch();
    const R0Ptrs q = r0_ptrs(p, ws);
    mean_body(q.colsum, p.panels, p.m, p.n, p.center, p, q.mu, q.chk);
}
__global__ void gram_kernel(const Plan p, const double* __restrict__ X, char* ws, int pass) {
    grid_dep_wait();
    const R0Ptrs q = r0_ptrs(p, ws);
    if (pass && *q.onepass) return;
    gram_body(blockIdx.x, X, p.n, p.m, p.rows_per_panel, q.mu, p.panels, pass ? q.r1inv : nullptr,
              p, q.gram, q.chk);
}
__global__ void __launch_bounds__(kRedThreads) gram_sum_kernel(const Plan p, char* ws, int pass) {
    grid_dep_wait();
    grid_dep_launch();
    const R0Ptrs q = r0_ptrs(p, ws);
    if (pass && *q.onepass) return;
    gram_sum_body(blockIdx.x, q.gram, p.panels, p.m, q.gsum, q.chk);
}
__global__ void __launch_bounds__(kCholThreads) chol_kernel(const Plan p, char* ws, int pass) {
    grid_dep_wait();
    grid_dep_launch();
    const R0Ptrs q = r0_ptrs(p, ws);
    if (pass) {
        if (!*q.onepass) chol_body(q.gsum, p.m, q.r1, q.r0, nullptr, q.status, q.chk);
    } else {
        chol_body(q.gsum, p.m, nullptr, q.r1, q.r1inv, q.status, q.chk, q.r0, q.onepass);
    }
}

// A batch: the position maps (block -> launch position) of panels (y = 0) and of
// sub-walk CTAs (y = 1), one block per launch position.
__global__ void batch_pos_kernel(const BatchView v) {
    const int l = blockIdx.x;
    const int64_t* prefix = blockIdx.y ? v.cta_prefix : v.panel_prefix;
    int32_t* pos = blockIdx.y ? v.cta_pos : v.panel_pos;
    for (int64_t i = prefix[l] + threadIdx.x; i < prefix[l + 1]; i += blockDim.x) pos[i] = l;
}

// A batch: blocks are mapped to (dataset, panel) through the prefix of panels.
__global__ void status_clear_kernel_b(const BatchView v) {
    const int d = blockIdx.x;
    int* st = reinterpret_cast<int*>(v.ws[d] + v.plans[d].off_status);
    for (int i = threadIdx.x; i < 64; i += blockDim.x) st[i] = 0;
}
// The batched column sums loop over the batch's row panels on a few blocks per
// SM (grid-stride): one small block per panel, about 20,000 for the bootstrap
// batch, cost more to launch than the panels' work (51 -> 43 us).
__global__ void colsum_kernel_b(const BatchView v, int64_t P) {
    for (int64_t g = blockIdx.x; g < P; g += gridDim.x) {
        int64_t local;
        const int d = batch_locate(v, v.panel_prefix, v.panel_pos, g, local);
        const Plan& p = v.plans[d];
        const R0Ptrs q = r0_ptrs(p, v.ws[d]);
        colsum_body((int)local, v.X[d], p.n, p.m, p.rows_per_panel, q.colsum, p.panels, q.chk);
        __syncthreads();  // the shared reduction buffers are reused by the next panel
    }
}
__global__ void __launch_bounds__(kRedThreads) mean_kernel_b(const BatchView v) {
    const int d = blockIdx.x;
    const Plan& p = v.plans[d];
    const R0Ptrs q = r0_ptrs(p, v.ws[d]);
    mean_body(q.colsum, p.panels, p.m, p.n, p.center, p, q.mu, q.chk);
}
// The row panels of the datasets that need the second CholeskyQR pass, as a
// prefix over launch positions (datasets that took one pass count none): one
// block scans the one-pass flags after the first pass, so that the second
// pass's Gram blocks map onto that work alone, and the rest return after one
// load instead of each looking its dataset and flag up (the bootstrap batch's
// datasets are mostly well conditioned).
__global__ void __launch_bounds__(1024) pass2_prefix_kernel_b(const BatchView v) {
    __shared__ int64_t part[1024];
    __shared__ int64_t carry;
    if (threadIdx.x == 0) {
        carry = 0;
        v.pass2_prefix[0] = 0;
    }
    __syncthreads();
    for (int b0 = 0; b0 < v.B; b0 += blockDim.x) {
        const int l = b0 + (int)threadIdx.x;
        int64_t c = 0;
        if (l < v.B) {
            const int d = v.dataset_of[l];
            const Plan& p = v.plans[d];
            const R0Ptrs q = r0_ptrs(p, v.ws[d]);
            c = *q.onepass ? 0 : p.panels;
        }
        part[threadIdx.x] = c;
        __syncthreads();
        for (unsigned o = 1; o < blockDim.x; o <<= 1) {  // inclusive scan
            const int64_t t = threadIdx.x >= o ? part[threadIdx.x - o] : 0;
            __syncthreads();
            part[threadIdx.x] += t;
            __syncthreads();
        }
        if (l < v.B) v.pass2_prefix[l + 1] = carry + part[threadIdx.x];
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry += part[threadIdx.x];
        __syncthreads();
    }
}
// Pass 1: one block per row panel of the batch.  Pass 2: block bx is panel bx of
// the pass-2 prefix (a binary search for its launch position), if there is one.
// (A grid-stride form of either pass, a few blocks per SM looping over the
// panels, measured slower: the Gram is bound by its work, not by its launch.)
__global__ void gram_kernel_b(const BatchView v, int pass) {
    int64_t local;
    int d;
    if (pass) {
        const int64_t bx = blockIdx.x;
        if (bx >= v.pass2_prefix[v.B]) return;
        int lo = 0, hi = v.B;  // pass2_prefix[lo] <= bx < pass2_prefix[hi]
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (v.pass2_prefix[mid] <= bx)
                lo = mid;
            else
                hi = mid;
        }
        local = bx - v.pass2_prefix[lo];
        d = v.dataset_of[lo];
    } else {
        d = batch_locate(v, v.panel_prefix, v.panel_pos, blockIdx.x, local);
    }
    const Plan& p = v.plans[d];
    const R0Ptrs q = r0_ptrs(p, v.ws[d]);
    gram_body((int)local, v.X[d], p.n, p.m, p.rows_per_panel, q.mu, p.panels,
              pass ? q.r1inv : nullptr, p, q.gram, q.chk);
}
// grid (pair groups of the largest m, datasets)
__global__ void __launch_bounds__(kRedThreads) gram_sum_kernel_b(const BatchView v, int pass) {
    const int d = blockIdx.y;
    const Plan& p = v.plans[d];
    if ((int)blockIdx.x * 32 >= p.m * (p.m + 1) / 2) return;
    const R0Ptrs q = r0_ptrs(p, v.ws[d]);
    if (pass && *q.onepass) return;
    gram_sum_body(blockIdx.x, q.gram, p.panels, p.m, q.gsum, q.chk);
}
__global__ void __launch_bounds__(kCholThreads) chol_kernel_b(const BatchView v, int pass) {
    const int d = blockIdx.x;
    const Plan& p = v.plans[d];
    const R0Ptrs q = r0_ptrs(p, v.ws[d]);
    if (pass) {
        if (!*q.onepass) chol_body(q.gsum, p.m, q.r1, q.r0, nullptr, q.status, q.chk);
    } else {
        chol_body(q.gsum, p.m, nullptr, q.r1, q.r1inv, q.status, q.chk, q.r0, q.onepass);
    }
}

}  // namespace

int launch_r0(const Plan& p, const double* X, char* ws, cudaStream_t stream) {
    if (cudaMemsetAsync(ws + p.off_status, 0, 256, stream) != cudaSuccess) return GBN_ERR_CUDA;
    if (launch_plain(colsum_kernel, dim3(p.panels), dim3(kColsumThreads), 0, stream, p, X, ws) !=
        cudaSuccess)
        return GBN_ERR_CUDA;
    const unsigned groups = (unsigned)((p.m * (p.m + 1) / 2 + 31) / 32);
    const cudaError_t e[] = {
        launch_dep(mean_kernel, dim3(1), dim3(kRedThreads), 0, stream, p, ws),
        launch_dep(gram_kernel, dim3(p.panels), dim3(gram_threads(p.m)), 0, stream, p, X, ws, 0),
        launch_dep(gram_sum_kernel, dim3(groups), dim3(kRedThreads), 0, stream, p, ws, 0),
        launch_dep(chol_kernel, dim3(1), dim3(kCholThreads), 0, stream, p, ws, 0),
        launch_dep(gram_kernel, dim3(p.panels), dim3(gram_threads(p.m)), 0, stream, p, X, ws, 1),
        launch_dep(gram_sum_kernel, dim3(groups), dim3(kRedThreads), 0, stream, p, ws, 1),
        launch_dep(chol_kernel, dim3(1), dim3(kCholThreads), 0, stream, p, ws, 1)};
    for (cudaError_t x : e)
        if (x != cudaSuccess) return GBN_ERR_CUDA;
    return GBN_OK;
}

constexpr int kColsumBlocksPerSm = 16;

int launch_r0_batched(const BatchView& v, int64_t total_panels, int max_m, cudaStream_t stream) {
    const unsigned B = (unsigned)v.B;
    const int64_t P = total_panels;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return GBN_ERR_CUDA;
    const unsigned g_colsum = (unsigned)std::min<int64_t>(P, (int64_t)sms * kColsumBlocksPerSm);
    const dim3 sum_grid((unsigned)((max_m * (max_m + 1) / 2 + 31) / 32), B);
    const cudaError_t e[] = {
        launch_plain(batch_pos_kernel, dim3(B, 2), dim3(256), 0, stream, v),
        launch_plain(status_clear_kernel_b, dim3(B), dim3(64), 0, stream, v),
        launch_plain(colsum_kernel_b, dim3(g_colsum), dim3(kColsumThreads), 0, stream, v, P),
        launch_plain(mean_kernel_b, dim3(B), dim3(kRedThreads), 0, stream, v),
        launch_plain(gram_kernel_b, dim3((unsigned)P), dim3(gram_threads(max_m)), 0, stream, v, 0),
        launch_plain(gram_sum_kernel_b, sum_grid, dim3(kRedThreads), 0, stream, v, 0),
        launch_plain(chol_kernel_b, dim3(B), dim3(kCholThreads), 0, stream, v, 0),
        launch_plain(pass2_prefix_kernel_b, dim3(1), dim3(1024), 0, stream, v),
        launch_plain(gram_kernel_b, dim3((unsigned)P), dim3(gram_threads(max_m)), 0, stream, v, 1),
        launch_plain(gram_sum_kernel_b, sum_grid, dim3(kRedThreads), 0, stream, v, 1),
        launch_plain(chol_kernel_b, dim3(B), dim3(kCholThreads), 0, stream, v, 1)};
    for (cudaError_t x : e)
        if (x != cudaSuccess) return GBN_ERR_CUDA;
    return GBN_OK;
}

}  // namespace gbn

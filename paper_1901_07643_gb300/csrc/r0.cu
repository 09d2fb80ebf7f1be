// Initial QR decomposition R0 of the centred data (the "initial QRD" that the
// walk starts from, Sec. 2 and Sec. 1.3), computed as CholeskyQR2 in FP64:
//   pass 1: G1 = Xc^T Xc (row panels, reduced), R1 = chol(G1)
//   pass 2: Q1 = Xc R1^{-1} (per row), G2 = Q1^T Q1, R2 = chol(G2), R0 = R2 R1.
// Columns are taken in the plan's order (the order the sub-walk tree decides
// variables in), so R0 is the R factor of Xc[:, order].
#include <math.h>

#include "gbn_internal.cuh"

namespace gbn {
namespace {

constexpr int kPanelChunk = 32;  // rows staged in shared memory at a time
constexpr int kLd = 33;          // row stride of the m x m shared-memory tiles

// All shared-memory tiles here are flat 1-D arrays indexed as [row * kLd + col]:
// with this toolchain, runtime-indexed two-dimensional __shared__ arrays were
// mis-addressed in sm_103 code while the same accesses on flat arrays were not.

__global__ void colsum_kernel(const double* __restrict__ X, int64_t n, int m, int rows_per,
                              double* __restrict__ colsum, int panels,
                              unsigned long long* chk) {
    __shared__ double red[256];
    const int b = blockIdx.x;
    const int64_t r0 = (int64_t)b * rows_per;
    const int64_t r1 = (r0 + rows_per < n) ? r0 + rows_per : n;
    const int per = blockDim.x / m;  // row lanes
    const int j = threadIdx.x % m;
    const int rl = threadIdx.x / m;
    double s = 0.0;
    if (rl < per)
        for (int64_t t = r0 + rl; t < r1; t += per)
            if (GBN_IN(chk, 101, t * m + j, n * m)) s += X[t * m + j];
    if (GBN_IN(chk, 102, threadIdx.x, 256)) red[threadIdx.x] = (rl < per) ? s : 0.0;
    __syncthreads();
    if (threadIdx.x < m) {
        double acc = 0.0;
        for (int l = 0; l < per; ++l)
            if (GBN_IN(chk, 103, l * m + threadIdx.x, 256)) acc += red[l * m + threadIdx.x];
        if (GBN_IN(chk, 104, (int64_t)b * m + threadIdx.x, (int64_t)panels * m))
            colsum[(int64_t)b * m + threadIdx.x] = acc;
    }
}

// Partial Gram of one row panel: sum over its rows of y y^T (upper triangle,
// packed by pairs i <= j), where y is the centred row in plan order, or for
// pass 2 the row of Q1 solving y R1 = xc.
__global__ void gram_kernel(const double* __restrict__ X, int64_t n, int m, int rows_per,
                            const double* __restrict__ colsum, int panels, int center,
                            const double* __restrict__ R1, Plan plan, double* __restrict__ gram,
                            unsigned long long* chk) {
    __shared__ double mu[32];
    __shared__ double rows[kPanelChunk * kLd];
    __shared__ double r1[32 * kLd];
    const int tid = threadIdx.x;
    if (tid < m) {
        double s = 0.0;
        if (center)
            for (int b = 0; b < panels; ++b)
                if (GBN_IN(chk, 111, (int64_t)b * m + plan.order[tid], (int64_t)panels * m))
                    s += colsum[(int64_t)b * m + plan.order[tid]];
        mu[tid] = center ? s / (double)n : 0.0;
    }
    if (R1)
        for (int e = tid; e < m * m; e += blockDim.x)
            if (GBN_IN(chk, 112, (e / m) * kLd + e % m, 32 * kLd)) r1[(e / m) * kLd + e % m] = R1[e];
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
    double acc = 0.0;
    const int64_t r0 = (int64_t)blockIdx.x * rows_per;
    const int64_t rend = (r0 + rows_per < n) ? r0 + rows_per : n;
    __syncthreads();
    for (int64_t c0 = r0; c0 < rend; c0 += kPanelChunk) {
        const int cnt = (rend - c0 < kPanelChunk) ? (int)(rend - c0) : kPanelChunk;
        for (int e = tid; e < cnt * m; e += blockDim.x) {
            const int t = e / m, j = e % m;
            const int64_t xi = (c0 + t) * m + plan.order[j];
            if (GBN_IN(chk, 113, xi, n * m) && GBN_IN(chk, 114, t * kLd + j, kPanelChunk * kLd))
                rows[t * kLd + j] = X[xi] - mu[j];
        }
        __syncthreads();
        if (R1 && tid < cnt) {  // forward substitution y R1 = xc, one row per thread
            double* y = rows + tid * kLd;
            for (int j = 0; j < m; ++j) {
                double s = y[j];
                for (int i = 0; i < j; ++i) s -= y[i] * r1[i * kLd + j];
                const double d = r1[j * kLd + j];
                y[j] = (d != 0.0) ? s / d : 0.0;
            }
        }
        __syncthreads();
        if (tid < npair)
            for (int t = 0; t < cnt; ++t) acc = fma(rows[t * kLd + pi], rows[t * kLd + pj], acc);
        __syncthreads();
    }
    if (tid < npair && GBN_IN(chk, 115, (int64_t)blockIdx.x * npair + tid, (int64_t)panels * npair))
        gram[(int64_t)blockIdx.x * npair + tid] = acc;
}

// Sum the panel Grams, Cholesky-factor (upper R with R^T R = G).  If R1 is
// given, the result is R2 and R0 = R2 * R1 is written to Rout; otherwise the
// factor itself is written to Rout.
__global__ void chol_kernel(const double* __restrict__ gram, int panels, int m,
                            const double* __restrict__ R1, double* __restrict__ Rout,
                            int* __restrict__ status, unsigned long long* chk) {
    __shared__ double G[32 * kLd];
    __shared__ double R[32 * kLd];
    const int tid = threadIdx.x;
    const int npair = m * (m + 1) / 2;
    for (int e = tid; e < npair; e += blockDim.x) {
        int q = e, i = 0;
        while (q >= m - i) {
            q -= m - i;
            ++i;
        }
        const int j = i + q;
        double s = 0.0;
        for (int b = 0; b < panels; ++b)
            if (GBN_IN(chk, 121, (int64_t)b * npair + e, (int64_t)panels * npair))
                s += gram[(int64_t)b * npair + e];
        if (GBN_IN(chk, 122, i * kLd + j, 32 * kLd)) G[i * kLd + j] = s;
    }
    for (int e = tid; e < 32 * kLd; e += blockDim.x) R[e] = 0.0;
    __syncthreads();
    for (int j = 0; j < m; ++j) {
        if (tid == 0) {
            double d = G[j * kLd + j];
            for (int i = 0; i < j; ++i) d -= R[i * kLd + j] * R[i * kLd + j];
            if (d > 0.0) {
                R[j * kLd + j] = sqrt(d);
            } else {
                R[j * kLd + j] = 0.0;  // column j lies in the span of the earlier ones
                atomicOr(status, GBN_STATUS_RANK_DEFICIENT);
            }
        }
        __syncthreads();
        const double rjj = R[j * kLd + j];
        for (int l = j + 1 + tid; l < m; l += blockDim.x) {
            double s = G[j * kLd + l];
            for (int i = 0; i < j; ++i) s -= R[i * kLd + j] * R[i * kLd + l];
            R[j * kLd + l] = (rjj != 0.0) ? s / rjj : 0.0;
        }
        __syncthreads();
    }
    for (int e = tid; e < m * m; e += blockDim.x) {
        const int i = e / m, j = e % m;
        double v = 0.0;
        if (i <= j) {
            if (R1) {
                for (int l = i; l <= j; ++l)
                    if (GBN_IN(chk, 123, l * m + j, m * m)) v += R[i * kLd + l] * R1[l * m + j];
            } else {
                v = R[i * kLd + j];
            }
        }
        if (GBN_IN(chk, 124, e, m * m)) Rout[e] = v;
    }
}

}  // namespace

int launch_r0(const Plan& p, const double* X, char* ws, cudaStream_t stream) {
    double* colsum = reinterpret_cast<double*>(ws + p.off_colsum);
    double* gram = reinterpret_cast<double*>(ws + p.off_gram);
    double* r1 = reinterpret_cast<double*>(ws + p.off_r1);
    double* r0 = reinterpret_cast<double*>(ws + p.off_r0);
    int* status = reinterpret_cast<int*>(ws + p.off_status);
    unsigned long long* chk = reinterpret_cast<unsigned long long*>(ws + p.off_status + kCheckOffset);
    if (cudaMemsetAsync(ws + p.off_status, 0, 256, stream) != cudaSuccess) return GBN_ERR_CUDA;
    if (p.center)
        colsum_kernel<<<p.panels, 256, 0, stream>>>(X, p.n, p.m, p.rows_per_panel, colsum, p.panels,
                                                    chk);
    gram_kernel<<<p.panels, 512, 0, stream>>>(X, p.n, p.m, p.rows_per_panel, colsum, p.panels,
                                              p.center, nullptr, p, gram, chk);
    chol_kernel<<<1, 256, 0, stream>>>(gram, p.panels, p.m, nullptr, r1, status, chk);
    gram_kernel<<<p.panels, 512, 0, stream>>>(X, p.n, p.m, p.rows_per_panel, colsum, p.panels,
                                              p.center, r1, p, gram, chk);
    chol_kernel<<<1, 256, 0, stream>>>(gram, p.panels, p.m, r1, r0, status, chk);
    return cudaGetLastError() == cudaSuccess ? GBN_OK : GBN_ERR_CUDA;
}

}  // namespace gbn

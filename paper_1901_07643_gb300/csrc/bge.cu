// BGe scores of every family from the Givens walk.
//
// The BGe score (Geiger and Heckerman 2002, corrected by Kuipers, Moffa and
// Heckerman 2014) of child c with parents S, l = |S|, is
//     ln p(d_{S u c}) - ln p(d_S)
//       = K(l) - a(l) ln rho(c | S) - L[S] / 2,
//     K(l) = ln(alpha_mu / (n + alpha_mu)) / 2 - (n / 2) ln pi
//            + ln Gamma((n + alpha_w - m + l + 1) / 2) - ln Gamma((alpha_w - m + l + 1) / 2)
//            + ((alpha_w - m + 2 l + 1) / 2) ln t,
//     a(l) = (n + alpha_w - m + l + 1) / 2,
// with R = t I + S_n the posterior matrix (prior mean = sample mean, T0 = t I),
// rho(c | S) = det R_{S u c} / det R_S its Schur complement and L[S] = ln det R_SS
// (the multivariate gamma ratio of consecutive sizes leaves one gamma each).
//
// The Schur complements are exactly what the walk reads off as RSS when it runs
// over an upper factor of R instead of the data's: the prior stage replaces R0
// (R0^T R0 = S_n) by the Cholesky factor of R0^T R0 + t I, and the walk runs in
// penalty mode with no penalty, storing n ln(rho / n).  After it:
//   * L over every variable set by the recursion L[S] = L[S - h] + ln rho(h | S - h),
//     h the highest variable of S: the family (h, S - h) sits at slot
//     h 2^(m-1) + (S - h) because S - h has no variable above h, so level h reads
//     one contiguous block of the table (levels below kLowLevels in one block);
//   * every slot rewritten in place as the BGe score.
// Families with more than the in-degree bound's parents are not touched, and L is
// formed only for the sets they need.
#include <math.h>

#include "gbn_internal.cuh"

namespace gbn {
namespace {

constexpr int kPriorThreads = 256;
constexpr int kLowLevels = 12;  // levels h < 12 (4096 sets) in one block
constexpr int kLd = 33;

// R0 <- U with U^T U = R0^T R0 + t I (FP64, one block; R0 upper triangular, m x m
// row-major in plan order: t I is invariant under the column order).
__global__ void __launch_bounds__(kPriorThreads) bge_prior_kernel(const Plan p, char* ws) {
    __shared__ double A[32 * kLd];
    __shared__ double M[32 * kLd];
    __shared__ double piv;
    grid_dep_wait();
    double* R0 = reinterpret_cast<double*>(ws + p.off_r0);
    const int m = p.m;
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) A[(e / m) * kLd + e % m] = R0[e];
    __syncthreads();
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {  // M = A^T A + t I, upper part
        const int i = e / m, j = e % m;
        if (i > j) continue;
        double s = (i == j) ? p.bge_t : 0.0;
        for (int k = 0; k <= i; ++k) s = fma(A[k * kLd + i], A[k * kLd + j], s);
        M[i * kLd + j] = s;
    }
    __syncthreads();
    for (int i = 0; i < m; ++i) {  // right-looking Cholesky: row i of U per step
        if (threadIdx.x == 0) {
            const double inv = rsqrt(M[i * kLd + i]);
            M[i * kLd + i] *= inv;  // sqrt(M_ii)
            piv = inv;
        }
        __syncthreads();
        for (int j = i + 1 + threadIdx.x; j < m; j += blockDim.x) M[i * kLd + j] *= piv;
        __syncthreads();
        for (int e = threadIdx.x; e < m * m; e += blockDim.x) {  // trailing block, i < r <= j
            const int r = e / m, j = e % m;
            if (r > i && r <= j) M[r * kLd + j] = fma(-M[i * kLd + r], M[i * kLd + j], M[r * kLd + j]);
        }
        __syncthreads();
    }
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
        const int i = e / m, j = e % m;
        R0[e] = (i <= j) ? M[i * kLd + j] : 0.0;
    }
}

struct BgeCoef {
    double K[32];  // K(l) by parent count
    double a[32];  // a(l)
    double inv_n, ln_n;
};

// ln rho from the walk's n ln(rho / n)
template <typename T>
__device__ __forceinline__ T ln_rho(T v, T inv_n, T ln_n) { return fma(v, inv_n, ln_n); }

// L of the sets S' + 2^h for S' < 2^h (sets with more than kmax variables need none).
template <typename T>
__device__ __forceinline__ void logdet_level(const Plan& p, const T* __restrict__ table,
                                             T* __restrict__ L, int h, int64_t i, int64_t stride,
                                             T inv_n, T ln_n) {
    const int64_t half = (int64_t)1 << (p.m - 1);
    const int64_t cnt = (int64_t)1 << h;
    for (; i < cnt; i += stride) {
        T v = T(0);
        if (__popcll((unsigned long long)i) < p.kmax)  // the set has <= kmax variables
            v = L[i] + ln_rho(table[(int64_t)h * half + i], inv_n, ln_n);
        L[cnt + i] = v;
    }
}

template <typename T>
__global__ void __launch_bounds__(1024) bge_logdet_low_kernel(const Plan p, const T* table, T* L,
                                                              int levels, const BgeCoef co) {
    grid_dep_wait();
    if (threadIdx.x == 0) L[0] = T(0);
    __syncthreads();
    for (int h = 0; h < levels; ++h) {
        logdet_level(p, table, L, h, threadIdx.x, blockDim.x, (T)co.inv_n, (T)co.ln_n);
        __syncthreads();
    }
}

template <typename T>
__global__ void __launch_bounds__(256) bge_logdet_kernel(const Plan p, const T* table, T* L, int h,
                                                         const BgeCoef co) {
    grid_dep_wait();
    logdet_level(p, table, L, h, (int64_t)blockIdx.x * blockDim.x + threadIdx.x,
                 (int64_t)gridDim.x * blockDim.x, (T)co.inv_n, (T)co.ln_n);
}

__device__ __forceinline__ uint64_t parent_set(int c, uint64_t cm) {
    return (cm & ((1ull << c) - 1ull)) | ((cm >> c) << (c + 1));
}
// The compressed mask of set S for child c (S without c): bit c removed.
__device__ __forceinline__ uint64_t parent_set_inv(int c, uint64_t S) {
    return (S & ((1ull << c) - 1ull)) | ((S >> (c + 1)) << c);
}

template <typename T>
__device__ __forceinline__ T bge_value(T v, T Ls, int l, const T* K, const T* a, T inv_n, T ln_n) {
    return fma(-a[l], ln_rho(v, inv_n, ln_n), fma(T(-0.5), Ls, K[l]));
}

// Every written slot rewritten in place.  FP32 with m >= 3: four consecutive slots per
// thread (one child, parent masks 4i .. 4i + 3), one 16-byte load and store of the table,
// and for children c >= 2 one 16-byte load of L (the two low mask bits are below c, so the
// four parent sets are consecutive and start at a multiple of 4).  A slot above the
// in-degree bound is stored back unchanged.
template <typename T>
__global__ void __launch_bounds__(256) bge_finalize_kernel(const Plan p, T* __restrict__ table,
                                                           const T* __restrict__ L,
                                                           const BgeCoef co) {
    __shared__ T K[32], a[32];
    if (threadIdx.x < 32) {
        K[threadIdx.x] = (T)co.K[threadIdx.x];
        a[threadIdx.x] = (T)co.a[threadIdx.x];
    }
    grid_dep_wait();
    __syncthreads();
    const int m = p.m;
    const int64_t half = (int64_t)1 << (m - 1);
    const int64_t total = (int64_t)m * half;
    const T inv_n = (T)co.inv_n, ln_n = (T)co.ln_n;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    if constexpr (sizeof(T) == 4) {
        if (m >= 3) {
            float4* t4 = reinterpret_cast<float4*>(table);
            for (int64_t qd = tid; qd < total / 4; qd += stride) {
                const int64_t slot = qd * 4;
                const int c = (int)(slot >> (m - 1));
                const uint64_t cm = (uint64_t)(slot & (half - 1));
                const uint64_t S = parent_set(c, cm);
                float4 v = t4[qd];
                float Ls[4];
                if (c >= 2) {
                    const float4 l4 = reinterpret_cast<const float4*>(L)[S >> 2];
                    Ls[0] = l4.x; Ls[1] = l4.y; Ls[2] = l4.z; Ls[3] = l4.w;
                } else {
#pragma unroll
                    for (int i = 0; i < 4; ++i) Ls[i] = L[parent_set(c, cm + i)];
                }
                float* vv = reinterpret_cast<float*>(&v);
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int l = __popcll(cm + i);
                    if (l <= p.kmax) vv[i] = bge_value(vv[i], Ls[i], l, K, a, inv_n, ln_n);
                }
                t4[qd] = v;
            }
            return;
        }
    }
    for (int64_t slot = tid; slot < total; slot += stride) {
        const int c = (int)(slot >> (m - 1));
        const uint64_t cm = (uint64_t)(slot & (half - 1));
        const int l = __popcll(cm);
        if (l > p.kmax) continue;
        table[slot] = bge_value(table[slot], L[parent_set(c, cm)], l, K, a, inv_n, ln_n);
    }
}

// FP32 with m >= 13: one block per block of 4096 variable sets S = H | low (H the
// sets' bits from 12 up, low < 4096): their L values are read once into shared
// memory, then every child's slots for these sets are rewritten.  For a child
// c >= 12 outside H the 4096 slots are contiguous (compress keeps the low 12
// bits); for c < 12 the 2048 sets without c are, at c 2^(m-1) + H/2 + j with
// low the 12-bit value j spread around bit c.  So L is read once (2^m elements)
// instead of once per child.
__global__ void __launch_bounds__(256) bge_finalize_sets_kernel(const Plan p,
                                                                float* __restrict__ table,
                                                                const float* __restrict__ L,
                                                                const BgeCoef co) {
    __shared__ float Ls[4096];
    __shared__ float K[32], a[32];
    if (threadIdx.x < 32) {
        K[threadIdx.x] = (float)co.K[threadIdx.x];
        a[threadIdx.x] = (float)co.a[threadIdx.x];
    }
    grid_dep_wait();
    const uint64_t H = (uint64_t)blockIdx.x << 12;
    for (int i = threadIdx.x; i < 1024; i += blockDim.x)
        reinterpret_cast<float4*>(Ls)[i] = reinterpret_cast<const float4*>(L + H)[i];
    __syncthreads();
    const int m = p.m;
    const int64_t half = (int64_t)1 << (m - 1);
    const float inv_n = (float)co.inv_n, ln_n = (float)co.ln_n;
    const int hp = __popcll(H);
    for (int c = 0; c < m; ++c) {
        if (c >= 12) {
            if ((H >> c) & 1ull) continue;  // every set of the block holds c
            float4* t4 = reinterpret_cast<float4*>(table + (int64_t)c * half +
                                                   (int64_t)parent_set_inv(c, H));
            for (int q = threadIdx.x; q < 1024; q += blockDim.x) {
                float4 v = t4[q];
                float* vv = reinterpret_cast<float*>(&v);
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int low = 4 * q + i;
                    const int l = hp + __popc(low);
                    if (l <= p.kmax) vv[i] = bge_value(vv[i], Ls[low], l, K, a, inv_n, ln_n);
                }
                t4[q] = v;
            }
        } else {
            float4* t4 = reinterpret_cast<float4*>(table + (int64_t)c * half + (int64_t)(H >> 1));
            const unsigned below = (1u << c) - 1u;
            for (int q = threadIdx.x; q < 512; q += blockDim.x) {
                float4 v = t4[q];
                float* vv = reinterpret_cast<float*>(&v);
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const unsigned j = 4u * q + i;
                    const unsigned low = (j & below) | ((j & ~below) << 1);
                    const int l = hp + __popc(low);
                    if (l <= p.kmax) vv[i] = bge_value(vv[i], Ls[low], l, K, a, inv_n, ln_n);
                }
                t4[q] = v;
            }
        }
    }
}

template <typename T>
int launch_finalize_t(const Plan& p, char* ws, T* out, cudaStream_t stream) {
    T* L = reinterpret_cast<T*>(ws + p.off_bge);
    const int m = p.m;
    const double n = (double)p.n, am = p.bge_alpha_mu, aw = p.bge_alpha_w, t = p.bge_t;
    const double kPi = 3.14159265358979323846;
    BgeCoef co;
    co.inv_n = 1.0 / n;
    co.ln_n = log(n);
    for (int l = 0; l < 32; ++l) {
        co.a[l] = (n + aw - m + l + 1) / 2.0;
        co.K[l] = 0.5 * log(am / (n + am)) - 0.5 * n * log(kPi) +
                  lgamma((n + aw - m + l + 1) / 2.0) - lgamma((aw - m + l + 1) / 2.0) +
                  (aw - m + 2.0 * l + 1) / 2.0 * log(t);
    }
    const int low = m < kLowLevels ? m : kLowLevels;
    if (launch_dep(bge_logdet_low_kernel<T>, dim3(1), dim3(1024), 0, stream, p, (const T*)out, L,
                   low, co) != cudaSuccess)
        return GBN_ERR_CUDA;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return GBN_ERR_CUDA;
    for (int h = low; h < m; ++h) {
        const int64_t cnt = (int64_t)1 << h;
        const int64_t want = (cnt + 255) / 256;
        const unsigned nb = (unsigned)(want < (int64_t)sms * 8 ? want : (int64_t)sms * 8);
        if (launch_dep(bge_logdet_kernel<T>, dim3(nb), dim3(256), 0, stream, p, (const T*)out, L,
                       h, co) != cudaSuccess)
            return GBN_ERR_CUDA;
    }
    if constexpr (sizeof(T) == 4) {
        if (m >= 13)
            return launch_rc(launch_dep(bge_finalize_sets_kernel, dim3((unsigned)(1u << (m - 12))),
                                        dim3(256), 0, stream, p, (float*)out, (const float*)L, co));
    }
    const int64_t total = (int64_t)m << (m - 1);
    const int64_t want = (total / 4 + 255) / 256 + 1;
    const unsigned nb = (unsigned)(want < (int64_t)sms * 16 ? want : (int64_t)sms * 16);
    if (launch_dep(bge_finalize_kernel<T>, dim3(nb), dim3(256), 0, stream, p, out, (const T*)L,
                   co) != cudaSuccess)
        return GBN_ERR_CUDA;
    return GBN_OK;
}

}  // namespace

int launch_bge_prior(const Plan& p, char* ws, cudaStream_t stream) {
    return launch_rc(launch_dep(bge_prior_kernel, dim3(1), dim3(kPriorThreads), 0, stream, p, ws));
}

int launch_bge_finalize(const Plan& p, char* ws, void* out, cudaStream_t stream) {
    return p.precision ? launch_finalize_t<double>(p, ws, static_cast<double*>(out), stream)
                       : launch_finalize_t<float>(p, ws, static_cast<float*>(out), stream);
}

}  // namespace gbn

// FP64 fix-up of ill-conditioned families in the FP32 walk.
//
// Before the walk, one warp flags the variables whose smallest possible RSS
// (the residual on all other variables, 1 / (G^{-1})_vv from R0) is below ten
// times fixup_tau times their centred sum of squares, and stores per variable
// the listing threshold fixup_tau * ||x_v||^2.  After the walk, the table
// blocks of flagged children only are scanned: a family whose FP32 score
// says RSS < threshold, i.e. score < n ln(thr / n) + |S| ln n, is listed.
// Each listed family is then solved again in FP64 from R0 -- Householder QR
// of the m x (|S|+1) matrix of R0's columns for S and the child, the
// least-squares problem of Sec. 1 on the initial QRD of Sec. 2 -- and its
// score is recomputed in FP64 and stored over the FP32 one.  Unflagged
// variables cost one early-exit block each; the walk itself is untouched.
#include <math.h>

#include "gbn_internal.cuh"

namespace gbn {
namespace {

constexpr int kFixWarps = 4;
constexpr int kLdF = 33;

// 32 warps load R0 (one element per thread, one round of loads); warp 0 does
// the rest.
__global__ void __launch_bounds__(1024) fix_flags_kernel(const Plan p, char* ws) {
    __shared__ float R[32 * kLdF];
    __shared__ float Ri[32 * kLdF];
    grid_dep_wait();
    grid_dep_launch();
    const int lane = threadIdx.x & 31, m = p.m;
    const double* R0 = reinterpret_cast<const double*>(ws + p.off_r0);
    {
        const int r = threadIdx.x >> 5;
        R[r * kLdF + lane] = (r < m && lane < m) ? (float)R0[r * m + lane] : 0.f;
        Ri[r * kLdF + lane] = 0.f;
    }
    __syncthreads();
    if (threadIdx.x >= 32) return;
    if (lane < m) {  // column `lane` of R0^{-1}
        for (int i = lane; i >= 0; --i) {
            float s = (i == lane) ? 1.f : 0.f;
            for (int l = i + 1; l <= lane; ++l) s -= R[i * kLdF + l] * Ri[l * kLdF + lane];
            Ri[i * kLdF + lane] = s / R[i * kLdF + i];  // a zero pivot gives inf: flagged below
        }
    }
    __syncwarp();
    float ginv = 0.f, cn2 = 0.f;
    if (lane < m) {
        for (int j = 0; j < m; ++j) ginv += Ri[lane * kLdF + j] * Ri[lane * kLdF + j];
        for (int i = 0; i <= lane; ++i) cn2 += R[i * kLdF + lane] * R[i * kLdF + lane];
    }
    const float tau = (float)p.fix_tau;
    const float rssmin = 1.f / ginv;
    const bool flag = lane < m && !(rssmin >= 10.f * tau * cn2);
    const int var = lane < m ? p.order[lane] : 0;
    const unsigned mask = __reduce_or_sync(0xffffffffu, flag ? (1u << var) : 0u);
    float* thr = reinterpret_cast<float*>(ws + p.off_fix + 16);
    if (lane < m) thr[var] = (float)((double)p.n * log((double)tau * (double)cn2 / (double)p.n));
    if (lane == 0) *reinterpret_cast<unsigned*>(ws + p.off_fix) = mask;
}

constexpr int kScanBlocksPerChild = 64;

// List the families of flagged children whose score is below the threshold.
__global__ void fix_scan_kernel(const Plan p, char* ws, const float* __restrict__ out) {
    grid_dep_wait();
    grid_dep_launch();
    const int c = blockIdx.y;
    const unsigned mask = *reinterpret_cast<const unsigned*>(ws + p.off_fix);
    if (!((mask >> c) & 1u)) return;
    const float base = reinterpret_cast<const float*>(ws + p.off_fix + 16)[c];  // n ln(thr/n)
    const float lam = (float)p.lam;
    unsigned* count = reinterpret_cast<unsigned*>(ws + p.off_status + kFixCountOffset);
    long long* list = reinterpret_cast<long long*>(ws + p.off_fix + 256);
    int* status = reinterpret_cast<int*>(ws + p.off_status);
    const int m = p.m;
    const int64_t block = (int64_t)1 << (m - 1);
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    // every lane of a warp runs the same number of iterations (block is a multiple of 32,
    // or smaller than one warp and then the extra lanes only vote false)
    for (int64_t s0 = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); s0 < block;
         s0 += stride) {
        const int64_t s = s0 + lane;
        bool f = false;
        if (s < block && slot_written(p, c, s)) {
            const float sc = out[((int64_t)c << (m - 1)) + s];
            f = sc < base + (float)__popcll((unsigned long long)s) * lam;
        }
        const unsigned bal = __ballot_sync(0xffffffffu, f);
        if (bal) {
            const int leader = __ffs(bal) - 1;
            unsigned first = 0;
            if (lane == leader) first = atomicAdd(count, (unsigned)__popc(bal));
            first = __shfl_sync(0xffffffffu, first, leader);
            if (f) {
                const unsigned idx = first + __popc(bal & ((1u << lane) - 1u));
                if (idx < (unsigned)p.fix_cap)
                    list[idx] = ((long long)c << (m - 1)) + s;
                else
                    atomicOr(status, GBN_STATUS_FIXUP_OVERFLOW);
            }
        }
    }
}

__device__ __forceinline__ double warp_sum(double x) {
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

__global__ void __launch_bounds__(32 * kFixWarps) fixup_kernel(const Plan p, char* ws, float* out) {
    __shared__ double M[kFixWarps * 32 * kLdF];
    __shared__ int pos_of[32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, m = p.m;
    grid_dep_wait();
    if (threadIdx.x < m) pos_of[p.order[threadIdx.x]] = threadIdx.x;
    __syncthreads();
    const unsigned listed = *reinterpret_cast<const unsigned*>(ws + p.off_status + kFixCountOffset);
    const unsigned count = listed < (unsigned)p.fix_cap ? listed : (unsigned)p.fix_cap;
    const long long* list = reinterpret_cast<const long long*>(ws + p.off_fix + 256);
    const double* R0 = reinterpret_cast<const double*>(ws + p.off_r0);
    double* Mw = M + warp * 32 * kLdF;
    const double n = (double)p.n, lam = p.lam;
    const long long table = (long long)m << (m - 1);
    for (unsigned i = blockIdx.x * kFixWarps + warp; i < count; i += gridDim.x * kFixWarps) {
        const long long slot = list[i];
        if (slot < 0 || slot >= table) continue;  // cannot happen: slots come from the walk
        const int c = (int)(slot >> (m - 1));
        const unsigned cm = (unsigned)(slot & ((1ll << (m - 1)) - 1));
        const unsigned S = (cm & ((1u << c) - 1u)) | ((cm >> c) << (c + 1));
        const int k = __popc(S);
        int j = 0;
        for (unsigned rest = S; rest; rest &= rest - 1, ++j) {
            const int v = __ffs(rest) - 1;
            Mw[lane * kLdF + j] = lane < m ? R0[lane * m + pos_of[v]] : 0.0;
        }
        Mw[lane * kLdF + k] = lane < m ? R0[lane * m + pos_of[c]] : 0.0;
        __syncwarp();
        for (int jj = 0; jj < k; ++jj) {  // Householder reflection zeroing column jj below row jj
            const double x = (lane >= jj && lane < m) ? Mw[lane * kLdF + jj] : 0.0;
            const double nrm2 = warp_sum(x * x);
            if (nrm2 == 0.0) continue;
            const double xj = __shfl_sync(0xffffffffu, x, jj);
            const double nrm = sqrt(nrm2);
            const double alpha = xj >= 0.0 ? -nrm : nrm;
            const double v = (lane == jj) ? xj - alpha : x;
            const double vtv = nrm2 - xj * xj + (xj - alpha) * (xj - alpha);
            for (int l = jj + 1; l <= k; ++l) {
                const double y = lane < m ? Mw[lane * kLdF + l] : 0.0;
                const double dot = warp_sum(v * y);
                if (lane < m) Mw[lane * kLdF + l] = y - (2.0 * dot / vtv) * v;
            }
            __syncwarp();
        }
        const double t = (lane >= k && lane < m) ? Mw[lane * kLdF + k] : 0.0;
        const double rss = warp_sum(t * t);
        if (lane == 0) out[slot] = rss > 0.0 ? (float)(n * log(rss / n) + k * lam) : -INFINITY;
        __syncwarp();
    }
}

}  // namespace

int launch_fix_flags(const Plan& p, char* ws, cudaStream_t stream) {
    return launch_rc(launch_dep(fix_flags_kernel, dim3(1), dim3(1024), 0, stream, p, ws));
}

int launch_fixup(const Plan& p, char* ws, void* out, cudaStream_t stream) {
    if (launch_dep(fix_scan_kernel, dim3(kScanBlocksPerChild, p.m), dim3(256), 0, stream, p, ws,
                   static_cast<const float*>(out)) != cudaSuccess ||
        launch_dep(fixup_kernel, dim3(304), dim3(32 * kFixWarps), 0, stream, p, ws,
                   static_cast<float*>(out)) != cudaSuccess)
        return GBN_ERR_CUDA;
    return GBN_OK;
}

}  // namespace gbn

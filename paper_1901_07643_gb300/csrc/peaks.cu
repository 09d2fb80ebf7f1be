// Arithmetic-pipe peaks of the device, measured: the denominators of the
// compute rooflines of the FP32 walk, the FP64 walk and the FP64 Gram passes.
// Each thread runs kChains independent chains of fused multiply-adds
// (x = x * a + b) for `iters` rounds; enough blocks fill every SM several
// times over, so the pipe, not latency, bounds the rate.  FLOPs are counted
// as 2 per FMA.  The FP64 tensor-core rate (mma.sync m8n8k4 f64, the only
// FP64 matrix instruction of the architecture) is measured the same way:
// independent accumulator chains per warp, 2 * 8 * 8 * 4 flops per
// instruction.  Not part of the scoring method.
#include "gbn_internal.cuh"

namespace gbn {
namespace {

constexpr int kChains = 8;
constexpr int kPeakThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kPeakThreads) fma_chains_kernel(T* out, T a, T b, int iters) {
    T x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (T)(threadIdx.x + c);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == (T)12345.6789) out[0] = s;  // keeps the chains live; never true for these inputs
}

template <typename T>
int time_fma(T* scratch, cudaStream_t stream, double* tflops) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return GBN_ERR_CUDA;
    const int blocks = sms * 8;
    const int iters = sizeof(T) == 8 ? 2048 : 65536;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return GBN_ERR_CUDA;
    int rc = launch_rc(launch_plain(fma_chains_kernel<T>, dim3(blocks), dim3(kPeakThreads), 0,
                                    stream, scratch, (T)0.999999, (T)1e-7, iters));  // warm-up
    float best = 1e30f;
    for (int r = 0; r < 3 && rc == GBN_OK; ++r) {
        if (cudaEventRecord(e0, stream) != cudaSuccess) rc = GBN_ERR_CUDA;
        if (rc == GBN_OK)
            rc = launch_rc(launch_plain(fma_chains_kernel<T>, dim3(blocks), dim3(kPeakThreads), 0,
                                        stream, scratch, (T)0.999999, (T)1e-7, iters));
        float ms = 0.f;
        if (rc == GBN_OK && (cudaEventRecord(e1, stream) != cudaSuccess ||
                             cudaEventSynchronize(e1) != cudaSuccess ||
                             cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
            rc = GBN_ERR_CUDA;
        if (rc == GBN_OK && ms < best) best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    const double flops = 2.0 * kChains * (double)iters * blocks * kPeakThreads;
    *tflops = flops / (best * 1e-3) / 1e12;
    return GBN_OK;
}

// One m8n8k4 FP64 MMA per chain and round: D (8 x 8, two doubles per lane)
// += A (8 x 4, one per lane) * B (4 x 8, one per lane).
__global__ void __launch_bounds__(kPeakThreads) dmma_chains_kernel(double* out, double a,
                                                                    int iters) {
    double d0[kChains], d1[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) d0[c] = d1[c] = (double)(threadIdx.x + c);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < kChains; ++c)
            asm("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
                : "+d"(d0[c]), "+d"(d1[c])
                : "d"(a), "d"(a));
    }
    double s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += d0[c] + d1[c];
    if (s == 12345.6789) out[0] = s;  // keeps the chains live; never true for these inputs
}

int time_dmma(double* scratch, cudaStream_t stream, double* tflops) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return GBN_ERR_CUDA;
    const int blocks = sms * 8;
    const int iters = 1024;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return GBN_ERR_CUDA;
    int rc = launch_rc(launch_plain(dmma_chains_kernel, dim3(blocks), dim3(kPeakThreads), 0,
                                    stream, scratch, 1e-4, iters));  // warm-up
    float best = 1e30f;
    for (int r = 0; r < 3 && rc == GBN_OK; ++r) {
        if (cudaEventRecord(e0, stream) != cudaSuccess) rc = GBN_ERR_CUDA;
        if (rc == GBN_OK)
            rc = launch_rc(launch_plain(dmma_chains_kernel, dim3(blocks), dim3(kPeakThreads), 0,
                                        stream, scratch, 1e-4, iters));
        float ms = 0.f;
        if (rc == GBN_OK && (cudaEventRecord(e1, stream) != cudaSuccess ||
                             cudaEventSynchronize(e1) != cudaSuccess ||
                             cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
            rc = GBN_ERR_CUDA;
        if (rc == GBN_OK && ms < best) best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    const double warps = (double)blocks * (kPeakThreads / 32);
    const double flops = 2.0 * 8 * 8 * 4 * kChains * (double)iters * warps;
    *tflops = flops / (best * 1e-3) / 1e12;
    return GBN_OK;
}

}  // namespace
}  // namespace gbn

using namespace gbn;

extern "C" int givensbn_dmma_peak(void* scratch, void* stream, double* tflops) {
    if (!scratch || !tflops) return GBN_ERR_NULL;
    if ((uintptr_t)scratch & 7u) return GBN_ERR_ALIGN;
    return time_dmma(static_cast<double*>(scratch), static_cast<cudaStream_t>(stream), tflops);
}

extern "C" int givensbn_pipe_peaks(void* scratch, void* stream, double* fp32_tflops,
                                   double* fp64_tflops) {
    if (!scratch || !fp32_tflops || !fp64_tflops) return GBN_ERR_NULL;
    if ((uintptr_t)scratch & 7u) return GBN_ERR_ALIGN;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int rc = time_fma<float>(static_cast<float*>(scratch), s, fp32_tflops);
    if (rc) return rc;
    return time_fma<double>(static_cast<double*>(scratch), s, fp64_tflops);
}

// score_all_families_noalloc: the scoring pipeline with its scratch in a
// file-scope device array instead of a caller-supplied workspace.
//
// Who needs it: callers that cannot allocate device memory at the point of
// the call — a host runtime whose own pool already owns all free HBM (so a
// cudaMalloc would fail or evict), or a latency-critical loop where
// cudaMalloc/cudaFree would implicitly synchronise the device and stall the
// other streams.  Such callers also cannot size and hand over a workspace of
// their own.  This entry point calls no allocating routine: the scratch below
// is part of the library's device image, and its address is looked up once
// per device.
//
// Limits and rules:
//  * kStaticScratchBytes = 16 MiB, enough for every n at m <= 20 with the
//    automatic q (FP32).  Larger inputs are rejected with
//    GBN_ERR_STATIC_SCRATCH before any device work.
//  * What must start at zero: only the 256-byte status block at the start of
//    the scratch; every call clears it on its own stream (cudaMemsetAsync)
//    before its first kernel.  Everything else is written before it is read.
//  * Overlapping calls race: all calls on one device share the one scratch,
//    so a call must not start (on any stream or host thread) until the
//    previous call's kernels have finished.
//  * The first call on a device does the symbol lookup; make that first call
//    before any stream capture begins.  The address is kept for the life of
//    the process: after cudaDeviceReset (or anything else that destroys the
//    device's primary context) it names memory of the old context, so a
//    process that resets a device must not call this entry point again.
#include <mutex>

#include "gbn_internal.cuh"

namespace gbn {
namespace {

constexpr size_t kStaticScratchBytes = size_t(16) << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_setup_mutex;
void* g_scratch_ptr[kMaxDevices] = {};

// Address of this device's copy of g_static_scratch (the current device),
// looked up once per device.
int scratch_for_current_device(char** ptr) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return GBN_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) return GBN_ERR_CUDA;
        g_scratch_ptr[dev] = p;
    }
    *ptr = static_cast<char*>(g_scratch_ptr[dev]);
    return GBN_OK;
}

}  // namespace
}  // namespace gbn

using namespace gbn;

extern "C" int score_all_families_noalloc(const double* X, int64_t n, int32_t m,
                                          float* out_scores, void* stream) {
    givensbn_opts opts;
    givensbn_default_opts(&opts);  // FP32, centring, automatic q
    Plan p;
    int rc = make_plan(n, m, &opts, &p);
    if (rc) return rc;
    if (p.total_bytes > kStaticScratchBytes) return GBN_ERR_STATIC_SCRATCH;
    if (!X || !out_scores) return GBN_ERR_NULL;
    if (((uintptr_t)X & 7u) || ((uintptr_t)out_scores & 15u)) return GBN_ERR_ALIGN;
    char* ws = nullptr;
    if ((rc = scratch_for_current_device(&ws))) return rc;
    return run_pipeline(p, X, ws, out_scores, static_cast<cudaStream_t>(stream), nullptr);
}

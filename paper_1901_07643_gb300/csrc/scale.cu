// Power-of-two column equilibration of R0 for the FP32 stages.
//
// The FP32 roots and walk form squares of R entries (a rotation's r^2 = x^2 + y^2,
// the tail sums): a column whose entries exceed about 2^64 overflows them and one
// below about 2^-63 underflows them.  Data of any scale reach the walk safely if
// each column j of R0 whose squared norm lies outside [2^-60, 2^60] is scaled by
// a power of two 2^e_j that brings it near 1 -- exact in FP64 and FP32, since only
// the exponent changes.  Scaling a parent column leaves every residual unchanged
// (it only rescales that parent's coefficient); scaling the child column c scales
// the family's RSS by exactly 2^(2 e_c).  So after the walk and the FP64 fix-up,
// which both see the scaled R0, each written score of child c is corrected by
// -2 e_c n ln 2 (the score is n ln(RSS / n) + penalty).  Columns already in range
// are untouched, so ordinary data give the same bits as without this stage; the
// correction kernel then finds nothing to do and returns at once.
//
// FP32 single-dataset path only: the FP64 walk's range holds any finite data whose
// squares are finite, and the batched path does not equilibrate.
#include <math.h>

#include "gbn_internal.cuh"

namespace gbn {
namespace {

constexpr double kLoNorm2 = 0x1p-60;
constexpr double kHiNorm2 = 0x1p60;

// One warp: lane j scales R0's column j (plan order) and records its exponent by
// variable; word 32 is set when any column was scaled.
__global__ void __launch_bounds__(32) scale_r0_kernel(const Plan p, char* ws) {
    grid_dep_wait();
    const int j = threadIdx.x;
    const int m = p.m;
    double* R0 = reinterpret_cast<double*>(ws + p.off_r0);
    int* ex = reinterpret_cast<int*>(ws + p.off_scale);
    int e = 0;
    if (j < m) {
        double s = 0.0;
        for (int r = 0; r <= j; ++r) s = fma(R0[r * m + j], R0[r * m + j], s);
        if (s > 0.0 && (s < kLoNorm2 || s > kHiNorm2)) e = -(ilogb(s) / 2);
        if (e != 0)
            for (int r = 0; r <= j; ++r) R0[r * m + j] = ldexp(R0[r * m + j], e);
        ex[p.order[j]] = e;
    }
    const unsigned any = __ballot_sync(0xffffffffu, e != 0);
    if (j == 0) ex[32] = any != 0u;
}

// Written scores of child c (grid.y) less 2 e_c n ln 2.
__global__ void __launch_bounds__(256) unscale_kernel(const Plan p, const char* ws,
                                                      float* __restrict__ out) {
    grid_dep_wait();
    const int* ex = reinterpret_cast<const int*>(ws + p.off_scale);
    if (ex[32] == 0) return;
    const int c = blockIdx.y;
    const int e = ex[c];
    if (e == 0) return;
    const float shift = (float)(2.0 * (double)e * (double)p.n * 0.69314718055994530942);
    const int64_t half = (int64_t)1 << (p.m - 1);
    float* blk = out + (int64_t)c * half;
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < half;
         s += (int64_t)gridDim.x * blockDim.x)
        if (slot_written(p, c, s)) blk[s] -= shift;
}

}  // namespace

int launch_scale_r0(const Plan& p, char* ws, cudaStream_t stream) {
    return launch_rc(launch_dep(scale_r0_kernel, dim3(1), dim3(32), 0, stream, p, ws));
}

int launch_unscale(const Plan& p, char* ws, void* out, cudaStream_t stream) {
    const int64_t half = (int64_t)1 << (p.m - 1);
    const int64_t want = (half + 255) / 256;
    const unsigned bx = (unsigned)(want < 64 ? want : 64);
    return launch_rc(launch_dep(unscale_kernel, dim3(bx, (unsigned)p.m), dim3(256), 0, stream, p,
                                (const char*)ws, static_cast<float*>(out)));
}

}  // namespace gbn

// Dispatch from a plan to the compiled walk instantiation.
#include <math.h>

#include "walk3.cuh"

#define GBN_DECL_ALL(T, COV)     \
    GBN_WALK_DECL(T, 2, COV);    \
    GBN_WALK_DECL(T, 3, COV);    \
    GBN_WALK_DECL(T, 4, COV);    \
    GBN_WALK_DECL(T, 5, COV);    \
    GBN_WALK_DECL(T, 6, COV);    \
    GBN_WALK_DECL(T, 7, COV);    \
    GBN_WALK_DECL(T, 8, COV);    \
    GBN_WALK_DECL(T, 9, COV);
#define GBN_DECL_FP64(COV)       \
    GBN_WALK_DECL(double, 2, COV); \
    GBN_WALK_DECL(double, 3, COV); \
    GBN_WALK_DECL(double, 4, COV); \
    GBN_WALK_DECL(double, 5, COV); \
    GBN_WALK_DECL(double, 6, COV); \
    GBN_WALK_DECL(double, 7, COV); \
    GBN_WALK_DECL(double, 8, COV);
GBN_DECL_ALL(float, 0)
GBN_DECL_ALL(float, 1)
GBN_DECL_FP64(0)
GBN_DECL_FP64(1)

namespace gbn {

// A wait inside the walk that lasts this long means the schedule is broken.
constexpr long long kWatchdogNs = 2000000000ll;

template <typename T>
static WalkArgs<T> walk_args(const Plan& p, char* ws, void* out) {
    WalkArgs<T> a;
    a.out = out;
    a.leaves = reinterpret_cast<const T*>(ws + p.off_leaves);
    a.leaf_stride = p.leaf_stride;
    a.m = p.m;
    a.k = p.k;
    a.W = p.W;
    a.lanes = p.lanes;
    const double n = (double)p.n;
    a.alpha = (T)(n * 0.69314718055994530942);
    a.lnn = (T)log(n);
    a.nlnn = (T)(n * log(n));
    a.chk = reinterpret_cast<unsigned long long*>(ws + p.off_status + kCheckOffset);
    a.timing = reinterpret_cast<unsigned long long*>(ws + p.off_status + kTimingOffset);
    a.status = reinterpret_cast<int*>(ws + p.off_status);
    a.out_size = (size_t)p.m << (p.m - 1);
    a.n_cwarps = p.n_bwarps;
    a.watchdog_ns = kWatchdogNs;
    return a;
}

#define GBN_CASE(T, Q)                                                       \
    case Q:                                                                  \
        return p.coverage ? GBN_WALK_INST_NAME(T, Q, 1)(a, p.n_cta, stream) \
                          : GBN_WALK_INST_NAME(T, Q, 0)(a, p.n_cta, stream);
int launch_walk(const Plan& p, char* ws, void* out, cudaStream_t stream) {
    if (p.precision) {
        const WalkArgs<double> a = walk_args<double>(p, ws, out);
        switch (p.Q) {
            GBN_CASE(double, 2)
            GBN_CASE(double, 3)
            GBN_CASE(double, 4)
            GBN_CASE(double, 5)
            GBN_CASE(double, 6)
            GBN_CASE(double, 7)
            GBN_CASE(double, 8)
            default:
                return GBN_ERR_Q;
        }
    }
    const WalkArgs<float> a = walk_args<float>(p, ws, out);
    switch (p.Q) {
        GBN_CASE(float, 2)
        GBN_CASE(float, 3)
        GBN_CASE(float, 4)
        GBN_CASE(float, 5)
        GBN_CASE(float, 6)
        GBN_CASE(float, 7)
        GBN_CASE(float, 8)
        GBN_CASE(float, 9)
        default:
            return GBN_ERR_Q;
    }
}

}  // namespace gbn

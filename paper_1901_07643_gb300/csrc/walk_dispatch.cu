// Dispatch from a plan to the compiled walk instantiation.
#include <math.h>

#include "walk3.cuh"

#define GBN_DECL_BOTH(T, Q, COV) \
    GBN_WALK_DECL(T, Q, COV);       \
    GBN_WALK_B_DECL(T, Q, COV);
#define GBN_DECL_ALL(T, COV)       \
    GBN_DECL_BOTH(T, 2, COV)       \
    GBN_DECL_BOTH(T, 3, COV)       \
    GBN_DECL_BOTH(T, 4, COV)       \
    GBN_DECL_BOTH(T, 5, COV)       \
    GBN_DECL_BOTH(T, 6, COV)       \
    GBN_DECL_BOTH(T, 7, COV)       \
    GBN_DECL_BOTH(T, 8, COV)       \
    GBN_DECL_BOTH(T, 9, COV)
#define GBN_DECL_FP64(COV)          \
    GBN_DECL_BOTH(double, 2, COV)   \
    GBN_DECL_BOTH(double, 3, COV)   \
    GBN_DECL_BOTH(double, 4, COV)   \
    GBN_DECL_BOTH(double, 5, COV)   \
    GBN_DECL_BOTH(double, 6, COV)   \
    GBN_DECL_BOTH(double, 7, COV)   \
    GBN_DECL_BOTH(double, 8, COV)
GBN_DECL_ALL(float, 0)
GBN_DECL_ALL(float, 1)
GBN_DECL_FP64(0)
GBN_DECL_FP64(1)

namespace gbn {

#define GBN_CASE(T, Q)                                                       \
    case Q:                                                                  \
        return p.coverage ? GBN_WALK_INST_NAME(T, Q, 1)(a, p.n_cta, stream) \
                          : GBN_WALK_INST_NAME(T, Q, 0)(a, p.n_cta, stream);
int launch_walk(const Plan& p, char* ws, void* out, cudaStream_t stream) {
    if (p.precision) {
        const WalkArgs<double> a = make_walk_args<double>(p, ws, out);
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
    const WalkArgs<float> a = make_walk_args<float>(p, ws, out);
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

namespace gbn {

#define GBN_BCASE(T, Q)                                                               \
    case Q:                                                                           \
        return coverage ? GBN_WALK_B_INST_NAME(T, Q, 1)(v, total_cta, n_cwarps, stream) \
                        : GBN_WALK_B_INST_NAME(T, Q, 0)(v, total_cta, n_cwarps, stream);
int launch_walk_batched(const BatchView& v, int64_t total_cta, int Q, int precision, bool coverage,
                        int n_cwarps, cudaStream_t stream) {
    if (precision) {
        switch (Q) {
            GBN_BCASE(double, 2)
            GBN_BCASE(double, 3)
            GBN_BCASE(double, 4)
            GBN_BCASE(double, 5)
            GBN_BCASE(double, 6)
            GBN_BCASE(double, 7)
            GBN_BCASE(double, 8)
            default:
                return GBN_ERR_Q;
        }
    }
    switch (Q) {
        GBN_BCASE(float, 2)
        GBN_BCASE(float, 3)
        GBN_BCASE(float, 4)
        GBN_BCASE(float, 5)
        GBN_BCASE(float, 6)
        GBN_BCASE(float, 7)
        GBN_BCASE(float, 8)
        GBN_BCASE(float, 9)
        default:
            return GBN_ERR_Q;
    }
}

}  // namespace gbn

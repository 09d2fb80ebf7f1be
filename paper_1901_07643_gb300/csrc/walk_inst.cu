// One instantiation of the Givens walk, selected at compile time by
// GBN_T (float or double), GBN_Q (free variables per sub-walk) and GBN_COV
// (1: coverage counters instead of scores).
#if !defined(GBN_T) || !defined(GBN_Q) || !defined(GBN_COV)
#error "walk_inst.cu needs -DGBN_T=... -DGBN_Q=... -DGBN_COV=..."
#endif

#include "walk3.cuh"

#define GBN_XNAME(T, Q, C) GBN_WALK_INST_NAME(T, Q, C)
int GBN_XNAME(GBN_T, GBN_Q, GBN_COV)(const gbn::WalkArgs<GBN_T>& a, int64_t n_cta,
                                      cudaStream_t s) {
    return gbn::launch_walk_q<GBN_T, GBN_Q, (GBN_COV != 0)>(a, n_cta, s);
}

#define GBN_XBNAME(T, Q, C) GBN_WALK_B_INST_NAME(T, Q, C)
int GBN_XBNAME(GBN_T, GBN_Q, GBN_COV)(const gbn::BatchView& v, int64_t total_cta, int nw,
                                       cudaStream_t s) {
    return gbn::launch_walk_batched_q<GBN_T, GBN_Q, (GBN_COV != 0)>(v, total_cta, nw, s);
}

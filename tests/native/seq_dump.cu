// Prints the compile-time swap tables the CUDA walk is built from, so that a
// CPU test can compare them with the oracle's GreedySwaps.  Host code only.
#include <cstdio>

#include "../../paper_1901_07643_gb300/csrc/gbn_internal.cuh"

template <int Q>
void dump() {
    constexpr auto& s = gbn::kWalkSeq<Q>;
    for (int t = 0; t < gbn::WalkSeq<Q>::N; ++t) {
        std::printf("%d %d %u", Q, s.idx[t], s.prefix[t]);
        for (int p = 0; p < Q; ++p) std::printf(" %d", s.var_at[t][p]);
        std::printf("\n");
    }
}

int main() {
    dump<2>(); dump<3>(); dump<4>(); dump<5>(); dump<6>(); dump<7>(); dump<8>();
    return 0;
}

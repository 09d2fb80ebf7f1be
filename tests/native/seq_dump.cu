// Prints the compile-time swap table the CUDA walk is built from, so that a
// CPU test can compare it with the oracle's GreedySwaps.  Host code only.
#include <cstdio>

#include "../../paper_1901_07643_gb300/csrc/walk3.cuh"

template <int Q>
void dump() {
    constexpr auto tab = gbn::make_step_tab<Q>();
    for (int t = 0; t < gbn::StepTab<Q>::N; ++t)
        std::printf("%d %u %u\n", Q, (unsigned)tab.row[t] + 1u, (unsigned)tab.pre[t]);
}

int main() {
    dump<2>(); dump<3>(); dump<4>(); dump<5>(); dump<6>(); dump<7>(); dump<8>();
    dump<9>(); dump<10>(); dump<11>(); dump<12>();
    return 0;
}

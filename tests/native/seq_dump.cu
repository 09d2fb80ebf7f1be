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

// upsilon_at (the run-time generator used by the adjoint walk): "U Q index"
void dump_runtime(int Q) {
    const long long n = (1ll << Q) - Q - 1;
    for (long long t = 0; t < n; ++t) std::printf("U %d %d\n", Q, gbn::upsilon_at(Q, t));
    std::printf("U %d %d\n", Q, gbn::upsilon_at(Q, n));  // past the end: 0
}

// The consumers' compressed slot table: "S Q t jj value"
template <int Q>
void dump_slots() {
    constexpr auto tab = gbn::make_slot_tab<Q>();
    for (int t = 0; t < gbn::StepTab<Q>::N; ++t)
        for (int jj = 0; jj <= Q; ++jj) std::printf("S %d %d %d %u\n", Q, t, jj, (unsigned)tab.v[t * (Q + 1) + jj]);
}

int main() {
    dump_slots<3>(); dump_slots<5>(); dump_slots<7>(); dump_slots<8>();
    for (int Q = 2; Q <= 14; ++Q) dump_runtime(Q);
    dump<2>(); dump<3>(); dump<4>(); dump<5>(); dump<6>(); dump<7>(); dump<8>();
    dump<9>(); dump<10>(); dump<11>(); dump<12>();
    return 0;
}

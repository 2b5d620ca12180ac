// Test driver for the warp-blocked table's slot schedule (pd_wb_sched.h), built
// by tests/test_wb_sched.py with the host C++ compiler.
//
// stdin:  NL G count, then per instance: slots, followed by 32 * slots targets
//         (lane-major: lane l, slot s at l * slots + s; -1 = empty slot)
// stdout: the scheduled instances in the same layout, one per line.
#include <cstdio>
#include <vector>

#include "pd_wb_sched.h"

int main() {
    int NL = 0, G = 0, count = 0;
    if (std::scanf("%d %d %d", &NL, &G, &count) != 3) return 1;
    const pd_wb::BankLayout bl{NL, G};
    for (int n = 0; n < count; ++n) {
        int slots = 0;
        if (std::scanf("%d", &slots) != 1 || slots < 0) return 1;
        std::vector<int32_t> grid((size_t)32 * slots);
        for (auto &v : grid)
            if (std::scanf("%d", &v) != 1) return 1;
        pd_wb::balance_banks(grid, slots, bl);
        std::printf("%d", slots);
        for (int32_t v : grid) std::printf(" %d", v);
        std::printf("\n");
    }
    return 0;
}

// Test driver for the invariant-divisor quotient (pd_divmagic.h), built by
// tests/test_divmagic.py with the host C++ compiler.
// stdin: count, then count lines "n d"; stdout: floor(n / d) per line.
#include <cstdio>

#include "pd_divmagic.h"

int main() {
    unsigned long long count = 0;
    if (std::scanf("%llu", &count) != 1) return 1;
    for (unsigned long long i = 0; i < count; ++i) {
        unsigned long long n = 0, d = 0;
        if (std::scanf("%llu %llu", &n, &d) != 2 || d == 0) return 1;
        std::printf("%llu\n", (unsigned long long)divmagic_q(n, make_divmagic(d)));
    }
    return 0;
}

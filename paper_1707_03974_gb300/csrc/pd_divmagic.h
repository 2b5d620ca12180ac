// Division of 64-bit integers by a divisor fixed for many quotients (host and
// device; plain C++ otherwise, compiled on its own by the CPU tests).
//
// Method: Granlund & Montgomery, "Division by invariant integers using
// multiplication" (PLDI 1994), the unsigned N-bit algorithm of their Fig. 4.1
// with N = 64.  For a divisor d >= 1 let l = ceil(log2 d) and
//     m = floor(2^64 (2^l - d) / d) + 1   (< 2^64),
// then for every 0 <= n < 2^64, with t = floor(m n / 2^64),
//     floor(n / d) = (t + ((n - t) >> min(l, 1))) >> max(l - 1, 0).
// The basis maps split a combined index I into (I / D_dn, I mod D_dn) once
// per element; this replaces the 64-bit division routine by one high
// multiply, a subtraction and two shifts.
#pragma once

#include <stdint.h>

#ifdef __CUDACC__
#define PD_DM_HD __host__ __device__
#else
#define PD_DM_HD
#endif

struct DivMagic {
    uint64_t m = 1;
    int sh1 = 0, sh2 = 0;
};

// host only: the constants for divisor d (d >= 1)
inline DivMagic make_divmagic(uint64_t d) {
    DivMagic r;
    int l = 0;
    while (l < 64 && ((uint64_t)1 << l) < d) ++l;  // l = ceil(log2 d)
    const unsigned __int128 two_l = (unsigned __int128)1 << l;
    r.m = (uint64_t)(((two_l - d) << 64) / d) + 1;
    r.sh1 = l < 1 ? l : 1;
    r.sh2 = l > 1 ? l - 1 : 0;
    return r;
}

PD_DM_HD inline uint64_t divmagic_hi(uint64_t a, uint64_t b) {
#ifdef __CUDA_ARCH__
    return __umul64hi(a, b);
#else
    return (uint64_t)(((unsigned __int128)a * b) >> 64);
#endif
}

// floor(n / d) for the d the constants were made for
PD_DM_HD inline uint64_t divmagic_q(uint64_t n, const DivMagic &dm) {
    const uint64_t t = divmagic_hi(dm.m, n);
    return (t + ((n - t) >> dm.sh1)) >> dm.sh2;
}

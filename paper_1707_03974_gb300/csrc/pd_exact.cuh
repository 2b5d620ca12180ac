// Exact reductions shared by the Lanczos kernels (internal header).
//
// Dot products of fixed-point (HB_FX64) vectors are exact: every 64 x 64-bit
// product is kept as a 128-bit integer and summed in 128 bits (per thread, per
// block, across blocks), then converted to float64 once.  The Lanczos
// coefficients follow from the exact sums in double-double arithmetic (the
// error-free transformations of Knuth and Dekker), so
//   alpha = <w, v>,  beta^2 = <w,w> - 2 alpha <w,v> + alpha^2 <v,v>
// lose nothing to cancellation.
#pragma once

#include <stdint.h>

namespace pdx {

struct I128 {
    uint64_t lo = 0;
    int64_t hi = 0;
};

__device__ __forceinline__ void i128_add(I128 &s, const I128 &t) {
    const uint64_t lo = s.lo + t.lo;
    s.hi += t.hi + (lo < t.lo ? 1 : 0);
    s.lo = lo;
}

// s += a * b exactly
__device__ __forceinline__ void i128_add_prod(I128 &s, int64_t a, int64_t b) {
    const int64_t ph = __mul64hi(a, b);
    const uint64_t pl = (uint64_t)a * (uint64_t)b;
    const uint64_t lo = s.lo + pl;
    s.hi += ph + (lo < pl ? 1 : 0);
    s.lo = lo;
}

// Sum over the block (warp shuffles, then one warp); the result is valid in thread 0.
__device__ __forceinline__ I128 block_sum128(I128 v) {
    __shared__ uint64_t s_lo[32];
    __shared__ int64_t s_hi[32];
    for (int o = 16; o > 0; o >>= 1) {
        I128 t;
        t.lo = __shfl_down_sync(0xffffffffu, v.lo, o);
        t.hi = __shfl_down_sync(0xffffffffu, v.hi, o);
        i128_add(v, t);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) {
        s_lo[wid] = v.lo;
        s_hi[wid] = v.hi;
    }
    __syncthreads();
    I128 r;
    if (wid == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        if (lane < nw) {
            r.lo = s_lo[lane];
            r.hi = s_hi[lane];
        }
        for (int o = 16; o > 0; o >>= 1) {
            I128 t;
            t.lo = __shfl_down_sync(0xffffffffu, r.lo, o);
            t.hi = __shfl_down_sync(0xffffffffu, r.hi, o);
            i128_add(r, t);
        }
    }
    return r;
}

// float64 sum over the block in a fixed tree order; valid in thread 0.
__device__ __forceinline__ double block_sum_d(double v) {
    __shared__ double s_w[32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) s_w[wid] = v;
    __syncthreads();
    double r = 0.0;
    if (wid == 0) {
        r = lane < (int)((blockDim.x + 31) >> 5) ? s_w[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) r += __shfl_down_sync(0xffffffffu, r, o);
    }
    return r;
}

// ---- double-double (Dekker / Knuth error-free transformations) ----
struct DD {
    double h, l;
};
__device__ __forceinline__ DD dd_two_sum(double a, double b) {
    const double s = a + b, bb = s - a;
    return {s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ DD dd_norm(double s, double e) {
    const double t = s + e;
    return {t, e - (t - s)};
}
__device__ __forceinline__ DD dd_add(DD x, DD y) {
    DD s = dd_two_sum(x.h, y.h);
    return dd_norm(s.h, s.l + x.l + y.l);
}
__device__ __forceinline__ DD dd_mul_d(DD x, double y) {
    const double p = x.h * y;
    return dd_norm(p, fma(x.h, y, -p) + x.l * y);
}
// a 128-bit integer times 2^sh as a double-double: the four 32-bit pieces are exact doubles
__device__ __forceinline__ DD dd_of_i128(I128 s, int sh) {
    const double h1 = ldexp((double)(int32_t)(uint32_t)((uint64_t)s.hi >> 32), 96 + sh);
    const double h0 = ldexp((double)(uint32_t)((uint64_t)s.hi & 0xFFFFFFFFu), 64 + sh);
    const double l1 = ldexp((double)(uint32_t)(s.lo >> 32), 32 + sh);
    const double l0 = ldexp((double)(uint32_t)(s.lo & 0xFFFFFFFFu), sh);
    DD r = {h1, 0.0};
    r = dd_add(r, {h0, 0.0});
    r = dd_add(r, {l1, 0.0});
    return dd_add(r, {l0, 0.0});
}

__device__ __forceinline__ double dd_value(DD x) { return x.h + x.l; }

// alpha and beta of a fixed-point Lanczos step from the exact sums
// t[0] = <w, v>, t[1] = <w, w>, t[2] = <v, v> of integer vectors with F fractional bits
__device__ __forceinline__ void fx_alpha_beta(const I128 (&t)[3], int F, double *alpha, double *beta) {
    const DD swv = dd_of_i128(t[0], -2 * F), sww = dd_of_i128(t[1], -2 * F), svv = dd_of_i128(t[2], -2 * F);
    const double al = swv.h + swv.l;
    DD b2 = dd_add(sww, dd_mul_d(swv, -2.0 * al));
    b2 = dd_add(b2, dd_mul_d(dd_mul_d(svv, al), al));
    const double v = b2.h + b2.l;
    *alpha = al;
    *beta = v > 0.0 ? sqrt(v) : 0.0;
}

}  // namespace pdx

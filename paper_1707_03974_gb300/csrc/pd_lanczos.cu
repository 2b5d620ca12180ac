// Lanczos ground state on top of the matrix-free H·v.
//
// The paper names Lanczos as the eigensolver (Sec. I) without specifying it;
// this is the textbook three-term recurrence (Golub & Van Loan, Sec. 10.1):
//   w = H v_j - beta_{j-1} v_{j-1};  alpha_j = <w, v_j>;  w -= alpha_j v_j;
//   [full reorthogonalisation: w -= V (V^T w), twice];
//   beta_j = ||w||;  v_{j+1} = w / beta_j,
// and the lowest eigenpair of the tridiagonal T_j solved on the host.
//
// Precision: alpha, beta, every dot product and norm are float64 values.  For
// float64 vectors the reductions accumulate in float64; for float32 vectors
// each thread accumulates exact products (TwoProd by fused multiply-add) in a
// float32 pair with TwoSum (Knuth / Dekker error-free transformations), so the
// reduction keeps ~48 significant bits at float32 throughput, and the float64
// per-thread values are then combined in a fixed tree order (deterministic).
#include <algorithm>
#include <chrono>
#include <complex>
#include <cfloat>
#include <cmath>
#include <type_traits>
#include <vector>

#include "pd_common.cuh"
#include "pd_exact.cuh"

namespace {

constexpr int kRedThreads = 256;
constexpr int kFinalThreads = 1024;
constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;

// ---------------- per-thread accumulators ----------------
struct AccF64 {
    double s = 0.0;
    __device__ void add_prod(double a, double b) { s = fma(a, b, s); }
    __device__ double value() const { return s; }
};

struct AccF32x2 {
    float hi = 0.f, lo = 0.f;
    __device__ void add_prod(float a, float b) {
        const float p = a * b;
        const float e = fmaf(a, b, -p);  // a*b = p + e exactly
        const float t = hi + p;
        const float bp = t - hi;
        const float err = (hi - (t - bp)) + (p - bp);  // hi + p = t + err exactly
        hi = t;
        lo += err + e;
    }
    __device__ double value() const { return (double)hi + (double)lo; }
};

template <typename T>
struct AccFor;
template <>
struct AccFor<double> {
    using type = AccF64;
};
template <>
struct AccFor<float> {
    using type = AccF32x2;
};

__device__ __forceinline__ double block_sum(double v) {
    __shared__ double s_warp[32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) s_warp[wid] = v;
    __syncthreads();
    double r = 0.0;
    if (wid == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        r = lane < nw ? s_warp[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) r += __shfl_down_sync(0xffffffffu, r, o);
    }
    return r;  // valid in thread 0
}

// Grid-stride loop over [0, n) that hands f four independent indices at a
// time (i, i + stride, i + 2 stride, i + 3 stride), so each thread keeps
// several loads in flight; the remainder one by one.  f(i) must not depend on
// another index's result.
template <typename Fn>
__device__ __forceinline__ void for_each_x4(uint64_t n, Fn f) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    for (; i + 3 * stride < n; i += 4 * stride) f(i, i + stride, i + 2 * stride, i + 3 * stride);
    for (; i < n; i += stride) f(i);
}

// ---------------- vector kernels ----------------
template <typename T>
__global__ void k_fill_random(T *__restrict__ v, uint64_t n, uint64_t seed) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t z = seed + (i + 1) * kGamma;  // state of the (i+1)-th SplitMix64 output
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z = z ^ (z >> 31);
        const double u = (double)(z >> 11) * 0x1.0p-52 - 1.0;
        v[i] = (T)u;
    }
}

// partial <a, b> per block
template <typename T>
__global__ void k_dot(const T *__restrict__ a, const T *__restrict__ b, uint64_t n, double *__restrict__ partials) {
    typename AccFor<T>::type acc;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        acc.add_prod(a[i], b[i]);
    const double s = block_sum(acc.value());
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// w -= beta_prev * vprev (if beta_prev); partial <w, v>
template <typename T>
__global__ void k_axpy_dot(T *__restrict__ w, const T *__restrict__ vprev, const double *__restrict__ beta_prev,
                           const T *__restrict__ v, uint64_t n, double *__restrict__ partials) {
    typename AccFor<T>::type acc;
    const T b = beta_prev ? (T)(*beta_prev) : T(0);
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        T wi = w[i];
        if (beta_prev) {
            wi = wi - b * vprev[i];
            w[i] = wi;
        }
        acc.add_prod(wi, v[i]);
    }
    const double s = block_sum(acc.value());
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// w -= alpha * v; partial ||w||^2 (when partials != nullptr)
template <typename T>
__global__ void k_axpy_norm(T *__restrict__ w, const T *__restrict__ v, const double *__restrict__ alpha, uint64_t n,
                            double *__restrict__ partials) {
    typename AccFor<T>::type acc;
    const T al = (T)(*alpha);
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const T wi = w[i] - al * v[i];
        w[i] = wi;
        acc.add_prod(wi, wi);
    }
    const double s = block_sum(acc.value());
    if (partials && threadIdx.x == 0) partials[blockIdx.x] = s;
}

// v *= 1 / *den  (den = beta or a norm)
template <typename T>
__global__ void k_scale(T *__restrict__ v, const double *__restrict__ den, uint64_t n) {
    const double d = *den;
    const T f = d != 0.0 ? (T)(1.0 / d) : T(0);
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        v[i] = v[i] * f;
}

// ---- float32 step in two passes (as the fixed-point one): pass 1 forms
// w = H v - beta_prev vprev and the sums <w,v>, <w,w>, <v,v> (float32 pairs,
// exact products); beta^2 = <w,w> - 2 alpha <w,v> + alpha^2 <v,v> in float64;
// pass 2 writes (w - alpha v) * (1 / beta), the same float32 operations the
// recurrence replay (k_regen_f32) performs.
__global__ void k_axpy_dot3_f32(float *__restrict__ w, const float *__restrict__ vprev,
                                const double *__restrict__ beta_prev, const float *__restrict__ v, uint64_t n,
                                double *__restrict__ partials) {
    AccF32x2 swv, sww, svv;
    const float b = beta_prev ? (float)(*beta_prev) : 0.f;
    auto one = [&](uint64_t i, float wi, float vi) {
        swv.add_prod(wi, vi);
        sww.add_prod(wi, wi);
        svv.add_prod(vi, vi);
    };
    for_each_x4(n, [&](uint64_t i0, auto... rest) {
        constexpr int U = 1 + sizeof...(rest);
        const uint64_t idx[U] = {i0, rest...};
        float wv[U], vv[U], pv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            wv[u] = w[idx[u]];
            vv[u] = v[idx[u]];
            pv[u] = beta_prev ? vprev[idx[u]] : 0.f;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (beta_prev) {
                wv[u] = wv[u] - b * pv[u];
                w[idx[u]] = wv[u];
            }
            one(idx[u], wv[u], vv[u]);
        }
    });
    const double a = block_sum(swv.value());
    const double c = block_sum(sww.value());
    const double d = block_sum(svv.value());
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = a;
        partials[gridDim.x + blockIdx.x] = c;
        partials[2 * gridDim.x + blockIdx.x] = d;
    }
}

__global__ void k_alpha_beta_f32(const double *__restrict__ partials, int nb, double *__restrict__ alpha,
                                 double *__restrict__ beta) {
    double t[3];
    for (int k = 0; k < 3; ++k) {
        double s = 0.0;
        for (int i = threadIdx.x; i < nb; i += blockDim.x) s += partials[k * nb + i];
        t[k] = block_sum(s);
    }
    if (threadIdx.x == 0) {
        const double al = t[0];
        // the float32 value of alpha is what pass 2 applies
        const double af = (double)(float)al;
        const double b2 = t[1] - 2.0 * af * t[0] + af * af * t[2];
        alpha[0] = al;
        beta[0] = b2 > 0.0 ? sqrt(b2) : 0.0;
    }
}

__global__ void k_update_f32(float *__restrict__ w, const float *__restrict__ v, const double *__restrict__ alpha,
                             const double *__restrict__ beta, int scale, uint64_t n) {
    const float al = (float)(*alpha);
    const double bb = *beta;
    const float f = scale ? (bb != 0.0 ? (float)(1.0 / bb) : 0.f) : 1.f;
    for_each_x4(n, [&](uint64_t i0, auto... rest) {
        constexpr int U = 1 + sizeof...(rest);
        const uint64_t idx[U] = {i0, rest...};
        float wv[U], vv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) wv[u] = w[idx[u]], vv[u] = v[idx[u]];
#pragma unroll
        for (int u = 0; u < U; ++u) w[idx[u]] = scale ? (wv[u] - al * vv[u]) * f : wv[u] - al * vv[u];
    });
}

// Full reorthogonalisation: partial dots of w with the stored vectors V[0..m),
// block (blockIdx.x, blockIdx.y) covers a slice of vector blockIdx.y.
template <typename T>
__global__ void k_multi_dot(const T *__restrict__ V, uint64_t stride, int m, const T *__restrict__ w, uint64_t n,
                            double *__restrict__ partials) {
    const int k = blockIdx.y;
    const T *vk = V + (uint64_t)k * stride;
    typename AccFor<T>::type acc;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        acc.add_prod(vk[i], w[i]);
    const double s = block_sum(acc.value());
    if (threadIdx.x == 0) partials[(uint64_t)k * gridDim.x + blockIdx.x] = s;
}

// w -= sum_k c_k V_k
template <typename T>
__global__ void k_multi_axpy(const T *__restrict__ V, uint64_t stride, int m, const double *__restrict__ c,
                             T *__restrict__ w, uint64_t n) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        T acc = w[i];
        for (int k = 0; k < m; ++k) acc -= (T)c[k] * V[(uint64_t)k * stride + i];
        w[i] = acc;
    }
}

// out[k] = sum of partials[k*nb .. k*nb+nb) (mode 0) or its square root (mode 1).
// One block per k, fixed summation order: deterministic.
__global__ void k_reduce(const double *__restrict__ partials, int nb, double *__restrict__ out, int mode) {
    double s = 0.0;
    const double *p = partials + (uint64_t)blockIdx.x * nb;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) s += p[i];
    s = block_sum(s);
    if (threadIdx.x == 0) out[blockIdx.x] = mode == 1 ? sqrt(s) : s;
}

// y = sum_k c_k V_k over m stored float32 vectors, accumulated in float64 (the
// Ritz vector of a float32 phase whose Krylov vectors were kept)
__global__ void k_combine_f32(const float *__restrict__ V, uint64_t stride, int m, const double *__restrict__ c,
                              float *__restrict__ y, uint64_t n) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int k = 0; k < m; ++k) acc = fma(c[k], (double)V[(uint64_t)k * stride + i], acc);
        y[i] = (float)acc;
    }
}

// y += c * v, float32 storage (Ritz vector assembly)
__global__ void k_axpy_scalar_f32(float *__restrict__ y, const float *__restrict__ v, float c, uint64_t n) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        y[i] += c * v[i];
}

// w = (w - alpha v - beta_prev vprev) / beta  with host scalars (regeneration of
// the float32 Krylov vectors with the recorded recurrence coefficients)
__global__ void k_regen_f32(float *__restrict__ w, const float *__restrict__ v, const float *__restrict__ vprev,
                            float al, float bp, float inv_b, uint64_t n) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        float wi = w[i];
        if (vprev) wi = wi - bp * vprev[i];
        wi = wi - al * v[i];
        w[i] = wi * inv_b;
    }
}

__global__ void k_f32_to_f64(const float *__restrict__ a, double *__restrict__ b, uint64_t n) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        b[i] = (double)a[i];
}

__global__ void k_copy_f32(const float *__restrict__ a, float *__restrict__ b, uint64_t n) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        b[i] = a[i];
}

template <typename T>
__global__ void k_copy(const T *__restrict__ a, T *__restrict__ b, uint64_t n) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        b[i] = a[i];
}

// ---------------- fixed-point (HB_FX64) vector kernels ----------------
// Dot products of fixed-point vectors are exact (pd_exact.cuh): 128-bit sums of
// the 64 x 64-bit products, per thread, per block and across blocks in a fixed
// order, converted to float64 once.
using pdx::I128;
using pdx::block_sum128;
using pdx::i128_add;
using pdx::i128_add_prod;

__global__ void k_fx_scale(int64_t *__restrict__ v, const double *__restrict__ den, uint64_t n) {
    const double d = *den;
    const FxCoef f = fx_coef_dev(d != 0.0 ? 1.0 / d : 0.0);
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        v[i] = fx_mul(v[i], f.K, f.G);
}

// Exact 128-bit sum of block partials, converted once: value * 2^(sh - 2F); mode 1 takes the square root.
__global__ void k_reduce128(const I128 *__restrict__ partials, int nb, double *__restrict__ out, int mode, int F,
                            int sh = 0) {
    I128 s;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) i128_add(s, partials[i]);
    s = block_sum128(s);
    if (threadIdx.x == 0) {
        const double v = ldexp((double)s.hi * 18446744073709551616.0 + (double)s.lo, sh - 2 * F);
        out[0] = mode == 1 ? sqrt(v) : v;
    }
}

// ---- fused fixed-point step: two passes instead of three ----
// Pass 1 forms w = H v - beta_prev vprev and the exact sums <w, v>, <w, w>,
// <v, v>; alpha = <w, v> and beta^2 = ||w - alpha v||^2 = <w,w> - 2 alpha <w,v>
// + alpha^2 <v,v> follow in double-double arithmetic from the exact 128-bit
// sums (no cancellation loss); pass 2 writes (w - alpha v) / beta.
__global__ void k_fx_axpy_dot3(int64_t *__restrict__ w, const int64_t *__restrict__ vprev,
                               const double *__restrict__ beta_prev, const int64_t *__restrict__ v, uint64_t n,
                               I128 *__restrict__ partials) {
    I128 swv, sww, svv;
    const FxCoef b = beta_prev ? fx_coef_dev(*beta_prev) : FxCoef();
    for_each_x4(n, [&](uint64_t i0, auto... rest) {
        constexpr int U = 1 + sizeof...(rest);
        const uint64_t idx[U] = {i0, rest...};
        int64_t wv[U], vv[U], pv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            wv[u] = w[idx[u]];
            vv[u] = v[idx[u]];
            pv[u] = beta_prev ? vprev[idx[u]] : 0;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (beta_prev) {
                wv[u] -= fx_mul(pv[u], b.K, b.G);
                w[idx[u]] = wv[u];
            }
            i128_add_prod(swv, wv[u], vv[u]);
            i128_add_prod(sww, wv[u], wv[u]);
            i128_add_prod(svv, vv[u], vv[u]);
        }
    });
    const I128 a = block_sum128(swv);
    const I128 c = block_sum128(sww);
    const I128 d = block_sum128(svv);
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = a;
        partials[gridDim.x + blockIdx.x] = c;
        partials[2 * gridDim.x + blockIdx.x] = d;
    }
}

// alpha = <w, v>; beta = sqrt(<w,w> - 2 alpha <w,v> + alpha^2 <v,v>) with the
// alpha that pass 2 applies (the float64 value written to *alpha)
__global__ void k_fx_alpha_beta(const I128 *__restrict__ partials, int nb, double *__restrict__ alpha,
                                double *__restrict__ beta, int F) {
    I128 t[3];
    for (int k = 0; k < 3; ++k) {
        I128 s;
        for (int i = threadIdx.x; i < nb; i += blockDim.x) i128_add(s, partials[k * nb + i]);
        t[k] = block_sum128(s);
    }
    if (threadIdx.x == 0) pdx::fx_alpha_beta(t, F, alpha, beta);
}

// w = (w - alpha v) / beta  (without the division when !scale)
__global__ void k_fx_update(int64_t *__restrict__ w, const int64_t *__restrict__ v, const double *__restrict__ alpha,
                            const double *__restrict__ beta, int scale, uint64_t n) {
    const FxCoef al = fx_coef_dev(*alpha);
    const double b = *beta;
    const FxCoef f = fx_coef_dev(b != 0.0 ? 1.0 / b : 0.0);
    for_each_x4(n, [&](uint64_t i0, auto... rest) {
        constexpr int U = 1 + sizeof...(rest);
        const uint64_t idx[U] = {i0, rest...};
        int64_t wv[U], vv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) wv[u] = w[idx[u]], vv[u] = v[idx[u]];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t wi = wv[u] - fx_mul(vv[u], al.K, al.G);
            w[idx[u]] = scale ? fx_mul(wi, f.K, f.G) : wi;
        }
    });
}

// Uniform [-1, 1) start vector in fixed point: SplitMix64 output k = z >> 11
// stands for k * 2^-52 - 1 (exact when F >= 52).
__global__ void k_fill_random_fx(int64_t *__restrict__ v, uint64_t n, uint64_t seed, int F) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t z = seed + (i + 1) * kGamma;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z = z ^ (z >> 31);
        const int64_t k = (int64_t)(z >> 11);
        const int64_t q = F >= 52 ? (k << (F - 52)) : ((k + (1ll << (51 - F))) >> (52 - F));
        v[i] = q - (1ll << F);
    }
}

// partial sums of (q 2^-F)^2 in float64: the norm of a fixed-point vector of any
// scale (a start vector need not be near unit norm), once per solve
__global__ void k_fx_norm2_f64(const int64_t *__restrict__ v, uint64_t n, int F, double *__restrict__ partials) {
    double acc = 0.0;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const double t = ldexp((double)v[i], -F);
        acc = fma(t, t, acc);
    }
    const double s = block_sum(acc);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

__global__ void k_f32_to_fx(const float *__restrict__ a, int64_t *__restrict__ b, uint64_t n, int F) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        b[i] = __double2ll_rn(ldexp((double)a[i], F));
}

// ---------------- host: tridiagonal lowest eigenpair ----------------
int sturm_below(const double *a, const double *b, int n, double x) {
    int c = 0;
    double q = 1.0;
    for (int i = 0; i < n; ++i) {
        const double bb = i > 0 ? b[i - 1] * b[i - 1] : 0.0;
        q = (a[i] - x) - (i > 0 ? bb / q : 0.0);
        if (q == 0.0) q = -DBL_EPSILON * (std::fabs(a[i]) + std::fabs(x) + DBL_MIN);
        if (q < 0.0) ++c;
    }
    return c;
}

// Solve (T - theta I) z = rhs in place by Gaussian elimination with partial
// pivoting on the tridiagonal (the row-interchange scheme of LAPACK's gttrf).
void shifted_tridiag_solve(const double *a, const double *b, int n, double theta, double *z) {
    std::vector<double> dl(n > 1 ? n - 1 : 1), d(n), du(n > 1 ? n - 1 : 1), du2(n > 2 ? n - 2 : 1);
    std::vector<int> piv(n);
    double scale = 0.0;
    for (int i = 0; i < n; ++i) {
        d[i] = a[i] - theta;
        scale = std::max(scale, std::fabs(a[i]) + (i > 0 ? std::fabs(b[i - 1]) : 0.0) + (i + 1 < n ? std::fabs(b[i]) : 0.0));
    }
    for (int i = 0; i + 1 < n; ++i) dl[i] = du[i] = b[i];
    const double tiny = DBL_EPSILON * (scale > 0 ? scale : 1.0);
    for (int i = 0; i + 1 < n; ++i) {
        if (std::fabs(d[i]) >= std::fabs(dl[i])) {
            if (d[i] == 0.0) d[i] = tiny;
            const double f = dl[i] / d[i];
            dl[i] = f;
            d[i + 1] -= f * du[i];
            if (i + 2 < n) du2[i] = 0.0;
            piv[i] = i;
        } else {
            const double f = d[i] / dl[i];
            d[i] = dl[i];
            dl[i] = f;
            const double tmp = du[i];
            du[i] = d[i + 1];
            d[i + 1] = tmp - f * d[i + 1];
            if (i + 2 < n) {
                du2[i] = du[i + 1];
                du[i + 1] = -f * du[i + 1];
            }
            piv[i] = i + 1;
        }
    }
    if (d[n - 1] == 0.0) d[n - 1] = tiny;
    for (int i = 0; i + 1 < n; ++i) {
        if (piv[i] == i) {
            z[i + 1] -= dl[i] * z[i];
        } else {
            const double tmp = z[i];
            z[i] = z[i + 1];
            z[i + 1] = tmp - dl[i] * z[i];
        }
    }
    z[n - 1] /= d[n - 1];
    if (n > 1) z[n - 2] = (z[n - 2] - du[n - 2] * z[n - 1]) / d[n - 2];
    for (int i = n - 3; i >= 0; --i) z[i] = (z[i] - du[i] * z[i + 1] - du2[i] * z[i + 2]) / d[i];
}

// Lowest eigenvalue by Sturm bisection to full precision, eigenvector by two
// steps of inverse iteration; returns the eigenvector's last component and,
// optionally, the whole normalised eigenvector.
void tridiag_lowest_host(const double *a, const double *b, int n, double *theta, double *s_last,
                         std::vector<double> *vec) {
    if (n == 1) {
        *theta = a[0];
        *s_last = 1.0;
        if (vec) vec->assign(1, 1.0);
        return;
    }
    double lo = a[0], hi = a[0];
    for (int i = 0; i < n; ++i) {
        const double r = (i > 0 ? std::fabs(b[i - 1]) : 0.0) + (i + 1 < n ? std::fabs(b[i]) : 0.0);
        lo = std::min(lo, a[i] - r);
        hi = std::max(hi, a[i] + r);
    }
    for (int it = 0; it < 200; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if (sturm_below(a, b, n, mid) >= 1)
            hi = mid;
        else
            lo = mid;
    }
    *theta = 0.5 * (lo + hi);
    std::vector<double> z(n, 1.0);
    for (int it = 0; it < 3; ++it) {
        shifted_tridiag_solve(a, b, n, *theta, z.data());
        double nrm = 0.0;
        for (double v : z) nrm += v * v;
        nrm = std::sqrt(nrm);
        if (!(nrm > 0.0) || !std::isfinite(nrm)) break;
        for (double &v : z) v /= nrm;
    }
    *s_last = z[n - 1];
    if (vec) *vec = z;
}

// ---------------- driver ----------------
struct Layout {
    uint64_t partials = 0, scal = 0, vec = 0, vec2 = 0, total = 0;
    int nblk = 0, nvec = 0, nvec2 = 0, maxit = 0;
};

uint64_t align256(uint64_t x) { return (x + 255) & ~255ull; }

Layout make_layout(hb_handle h, const hb_lanczos_opts &o) {
    Layout L;
    L.maxit = o.maxit;
    const uint64_t D = h->D;
    L.nblk = (int)std::max<uint64_t>(1, std::min<uint64_t>((uint64_t)h->sm_count * 4, (D + kRedThreads - 1) / kRedThreads));
    // partial sums per reduction block: three 128-bit integers (the fixed-point
    // step), or one float64 per block and stored vector (full reorthogonalisation)
    const uint64_t npart = std::max<uint64_t>(6ull * L.nblk, o.reorth ? (uint64_t)L.nblk * (o.maxit + 1) : 0ull);
    const uint64_t es = o.vec_dtype == HB_F32 ? 4 : 8;
    L.partials = 0;
    L.scal = align256(npart * 8);
    // scalars: alpha[maxit+1], beta[maxit+1], coef[maxit+1], misc[8]
    L.vec = L.scal + align256((uint64_t)(3 * (o.maxit + 1) + 8) * 8);
    L.nvec = o.reorth ? o.maxit + 1 : 3;
    if (o.vec_dtype == HB_F32 && o.fp64_finish && !o.reorth && o.store_basis > 0)
        L.nvec = std::min(o.maxit, o.store_basis) + 1;  // the float32 phase keeps v_0 .. v_K
    const uint64_t vbytes = align256(D * es);
    L.vec2 = L.vec + vbytes * L.nvec;
    L.nvec2 = 0;
    L.total = L.vec2;
    if (o.vec_dtype == HB_F32 && o.fp64_finish && !o.reorth) {
        L.nvec2 = 4;  // one float32 accumulator + three float64 vectors (in float32-size units: 1 + 6)
        L.total = L.vec2 + align256(D * 4) + 3 * align256(D * 8);
    }
    return L;
}

struct Solve {
    hb_handle h;
    cudaStream_t st;
    uint64_t D;
    int nblk;
    double *partials;
    double *d_alpha, *d_beta, *d_coef, *d_misc;
    int grid_vec;
};

template <typename T>
hb_status normalise(Solve &s, T *v) {
    if constexpr (std::is_same<T, int64_t>::value) {
        // a fresh start vector can be of any scale: its norm is taken in float64 (once per solve)
        k_fx_norm2_f64<<<s.nblk, kRedThreads, 0, s.st>>>(v, s.D, s.h->fx_frac, s.partials);
        k_reduce<<<1, kFinalThreads, 0, s.st>>>(s.partials, s.nblk, s.d_misc, 1);
        k_fx_scale<<<s.grid_vec, kRedThreads, 0, s.st>>>(v, s.d_misc, s.D);
    } else {
        k_dot<T><<<s.nblk, kRedThreads, 0, s.st>>>(v, v, s.D, s.partials);
        k_reduce<<<1, kFinalThreads, 0, s.st>>>(s.partials, s.nblk, s.d_misc, 1);
        k_scale<T><<<s.grid_vec, kRedThreads, 0, s.st>>>(v, s.d_misc, s.D);
    }
    PD_CUDA(cudaGetLastError());
    return HB_OK;
}

// One three-term step on the stream: w = H v - beta_prev vprev; alpha = <w, v>;
// w -= alpha v; beta = ||w||; and, when `scale`, w /= beta.  6 kernel launches.
template <typename T>
hb_status three_term_step(Solve &s, hb_dtype dt, const T *v, const T *vp, T *w, const double *beta_prev,
                          double *alpha, double *beta, bool scale, cudaEvent_t ev0, cudaEvent_t ev1) {
    if (ev0) PD_CUDA(cudaEventRecord(ev0, s.st));
    hb_status st = pd_apply(s.h, dt, v, w, s.st);
    if (st != HB_OK) return st;
    if (ev1) PD_CUDA(cudaEventRecord(ev1, s.st));
    if constexpr (std::is_same<T, float>::value) {  // two passes, see k_axpy_dot3_f32
        k_axpy_dot3_f32<<<s.nblk, kRedThreads, 0, s.st>>>(w, vp, vp ? beta_prev : nullptr, v, s.D, s.partials);
        k_alpha_beta_f32<<<1, kFinalThreads, 0, s.st>>>(s.partials, s.nblk, alpha, beta);
        k_update_f32<<<s.grid_vec, kRedThreads, 0, s.st>>>(w, v, alpha, beta, scale ? 1 : 0, s.D);
    } else {  // float64: the textbook three passes (the plain method)
        k_axpy_dot<T><<<s.nblk, kRedThreads, 0, s.st>>>(w, vp, vp ? beta_prev : nullptr, v, s.D, s.partials);
        k_reduce<<<1, kFinalThreads, 0, s.st>>>(s.partials, s.nblk, alpha, 0);
        k_axpy_norm<T><<<s.nblk, kRedThreads, 0, s.st>>>(w, v, alpha, s.D, s.partials);
        k_reduce<<<1, kFinalThreads, 0, s.st>>>(s.partials, s.nblk, beta, 1);
        if (scale) k_scale<T><<<s.grid_vec, kRedThreads, 0, s.st>>>(w, beta, s.D);
    }
    PD_CUDA(cudaGetLastError());
    return HB_OK;
}

// The fixed-point step in two passes (see k_fx_axpy_dot3): 4 kernel launches
// after the H·v.
hb_status three_term_step_fx(Solve &s, const int64_t *v, const int64_t *vp, int64_t *w, const double *beta_prev,
                             double *alpha, double *beta, bool scale, cudaEvent_t ev0, cudaEvent_t ev1) {
    const int nb = s.nblk;
    I128 *part = reinterpret_cast<I128 *>(s.partials);
    const int F = s.h->fx_frac;
    if (ev0) PD_CUDA(cudaEventRecord(ev0, s.st));
    hb_status st = pd_apply(s.h, HB_FX64, v, w, s.st);
    if (st != HB_OK) return st;
    if (ev1) PD_CUDA(cudaEventRecord(ev1, s.st));
    k_fx_axpy_dot3<<<nb, kRedThreads, 0, s.st>>>(w, vp, vp ? beta_prev : nullptr, v, s.D, part);
    k_fx_alpha_beta<<<1, kFinalThreads, 0, s.st>>>(part, nb, alpha, beta, F);
    k_fx_update<<<s.grid_vec, kRedThreads, 0, s.st>>>(w, v, alpha, beta, scale ? 1 : 0, s.D);
    PD_CUDA(cudaGetLastError());
    return HB_OK;
}

// the fixed-point and float32 steps divide by beta in their last pass
template <typename T>
constexpr bool kScalesInStep = !std::is_same<T, double>::value;

template <typename T>
hb_status step_any(Solve &s, hb_dtype dt, const T *v, const T *vp, T *w, const double *beta_prev, double *alpha,
                   double *beta, bool scale, cudaEvent_t ev0, cudaEvent_t ev1) {
    if constexpr (std::is_same<T, int64_t>::value)
        return three_term_step_fx(s, v, vp, w, beta_prev, alpha, beta, scale, ev0, ev1);
    else
        return three_term_step<T>(s, dt, v, vp, w, beta_prev, alpha, beta, scale, ev0, ev1);
}

template <typename T>
void scale_any(Solve &s, T *w, const double *den) {
    if constexpr (std::is_same<T, int64_t>::value)
        k_fx_scale<<<s.grid_vec, kRedThreads, 0, s.st>>>(w, den, s.D);
    else
        k_scale<T><<<s.grid_vec, kRedThreads, 0, s.st>>>(w, den, s.D);
}

struct PhaseResult {
    double theta = NAN, res = INFINITY;
    int iters = 0;
    bool converged = false;
    std::vector<double> alpha, beta;
};

// One Lanczos run.  V: base of the vector slots (slot stride `stride` elements);
// slot 0 must hold the normalised start vector.  reorth or keep: slot j holds
// v_j (keep: the three-term recurrence, the vectors only stored).  Otherwise
// three rotating slots.  Stops on tol (if tol > 0) or maxit.
template <typename T>
hb_status lanczos_run(Solve &s, hb_dtype dt, T *V, uint64_t stride, int maxit, bool reorth, double tol, int check,
                      PhaseResult &out, bool keep = false) {
    out = PhaseResult();
    std::vector<double> ha(maxit + 1), hb(maxit + 1);
    int iv = 0, ip = -1, iw = 1;  // slots of v_j, v_{j-1}, w
    for (int j = 0; j < maxit; ++j) {
        T *v = V + (uint64_t)iv * stride;
        T *w = V + (uint64_t)iw * stride;
        T *vp = ip >= 0 ? V + (uint64_t)ip * stride : nullptr;
        if (!reorth) {
            // the fixed-point and float32 steps divide by beta in their last pass, float64 below
            hb_status st = step_any<T>(s, dt, v, vp, w, vp ? s.d_beta + (j - 1) : nullptr, s.d_alpha + j,
                                       s.d_beta + j, kScalesInStep<T>, nullptr, nullptr);
            if (st != HB_OK) return st;
        } else if constexpr (std::is_same<T, int64_t>::value) {
            return HB_ERR_INVALID_ARG;  // full reorthogonalisation is float only
        } else {
            hb_status st = pd_apply(s.h, dt, v, w, s.st);
            if (st != HB_OK) return st;
            k_axpy_dot<T><<<s.nblk, kRedThreads, 0, s.st>>>(w, vp, vp ? s.d_beta + (j - 1) : nullptr, v, s.D,
                                                            s.partials);
            k_reduce<<<1, kFinalThreads, 0, s.st>>>(s.partials, s.nblk, s.d_alpha + j, 0);
            k_axpy_norm<T><<<s.nblk, kRedThreads, 0, s.st>>>(w, v, s.d_alpha + j, s.D, nullptr);
            const int m = j + 1;
            for (int pass = 0; pass < 2; ++pass) {
                dim3 g(s.nblk, m);
                k_multi_dot<T><<<g, kRedThreads, 0, s.st>>>(V, stride, m, w, s.D, s.partials);
                k_reduce<<<m, kFinalThreads, 0, s.st>>>(s.partials, s.nblk, s.d_coef, 0);
                k_multi_axpy<T><<<s.grid_vec, kRedThreads, 0, s.st>>>(V, stride, m, s.d_coef, w, s.D);
            }
            k_dot<T><<<s.nblk, kRedThreads, 0, s.st>>>(w, w, s.D, s.partials);
            k_reduce<<<1, kFinalThreads, 0, s.st>>>(s.partials, s.nblk, s.d_beta + j, 1);
            PD_CUDA(cudaGetLastError());
        }
        const bool last = (j + 1 == maxit) || (uint64_t)(j + 1) >= s.D;
        if ((j + 1) % check == 0 || last) {
            PD_CUDA(cudaMemcpyAsync(ha.data(), s.d_alpha, sizeof(double) * (j + 1), cudaMemcpyDeviceToHost, s.st));
            PD_CUDA(cudaMemcpyAsync(hb.data(), s.d_beta, sizeof(double) * (j + 1), cudaMemcpyDeviceToHost, s.st));
            PD_CUDA(cudaStreamSynchronize(s.st));
            double th, sl;
            tridiag_lowest_host(ha.data(), hb.data(), j + 1, &th, &sl, nullptr);
            out.theta = th;
            out.res = hb[j] * std::fabs(sl);
            out.iters = j + 1;
            if (!std::isfinite(th) || !std::isfinite(hb[j])) return HB_ERR_INVALID_STATE;
            const bool exhausted = hb[j] == 0.0 || (uint64_t)(j + 1) >= s.D;
            if ((tol > 0 && out.res <= tol * std::max(1.0, std::fabs(th))) || exhausted) {
                out.converged = true;
                out.alpha.assign(ha.begin(), ha.begin() + j + 1);
                out.beta.assign(hb.begin(), hb.begin() + j + 1);
                return HB_OK;
            }
            if (last) {
                out.alpha.assign(ha.begin(), ha.begin() + j + 1);
                out.beta.assign(hb.begin(), hb.begin() + j + 1);
                return HB_OK;
            }
        }
        if (reorth || !kScalesInStep<T>) scale_any<T>(s, w, s.d_beta + j);
        if (reorth || keep) {  // slot j holds v_j
            ip = iv;
            iv = j + 1;
            iw = j + 2;
        } else {
            const int old_p = ip < 0 ? 2 : ip;
            ip = iv;
            iv = iw;
            iw = old_p;
        }
    }
    out.iters = maxit;
    return HB_OK;
}


// Ritz vector y = sum_k s_k v_k of a float32 run: replay the recurrence from
// the stored start vector with the recorded alpha, beta (three slots: V slots
// 1, 2 and the start copy), accumulating y in V slot 0.  The replayed vectors
// are bit-identical to the first pass (same kernels, same scalars).
hb_status replay_ritz_f32(Solve &s, const PhaseResult &r, float *start_copy, float *V, uint64_t stride) {
    const uint64_t D = s.D;
    const int m = r.iters;
    std::vector<double> svec;
    double th, sl;
    tridiag_lowest_host(r.alpha.data(), r.beta.data(), m, &th, &sl, &svec);
    float *y = V;
    float *a = V + 1 * stride, *b = V + 2 * stride;
    float *vj = start_copy, *vp = nullptr, *wbuf = a, *spare = b;
    PD_CUDA(cudaMemsetAsync(y, 0, D * 4, s.st));
    for (int k = 0; k < m; ++k) {
        k_axpy_scalar_f32<<<s.grid_vec, kRedThreads, 0, s.st>>>(y, vj, (float)svec[k], D);
        if (k + 1 == m) break;
        hb_status st = pd_apply(s.h, HB_F32, vj, wbuf, s.st);
        if (st != HB_OK) return st;
        const double bk = r.beta[k];
        k_regen_f32<<<s.grid_vec, kRedThreads, 0, s.st>>>(wbuf, vj, vp, (float)r.alpha[k],
                                                          k > 0 ? (float)r.beta[k - 1] : 0.f,
                                                          bk != 0 ? (float)(1.0 / bk) : 0.f, D);
        float *old_vp = vp ? vp : spare;  // rotate: vp <- vj, vj <- wbuf, wbuf <- old vp
        vp = vj;
        vj = wbuf;
        wbuf = old_vp;
    }
    PD_CUDA(cudaGetLastError());
    return HB_OK;
}

// Ritz vector of float64 Lanczos: the same replay in float64 (the regeneration
// repeats the float64 step's operations: w - beta_prev vprev, - alpha v, * (1/beta))
__global__ void k_axpy_scalar_f64(double *__restrict__ y, const double *__restrict__ v, double c, uint64_t n) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        y[i] += c * v[i];
}

__global__ void k_regen_f64(double *__restrict__ w, const double *__restrict__ v, const double *__restrict__ vprev,
                            double al, double bp, double inv_b, uint64_t n) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        double wi = w[i];
        if (vprev) wi = wi - bp * vprev[i];
        wi = wi - al * v[i];
        w[i] = wi * inv_b;
    }
}

hb_status replay_ritz_f64(Solve &s, const PhaseResult &r, double *start_copy, double *V, uint64_t stride) {
    const uint64_t D = s.D;
    const int m = r.iters;
    std::vector<double> svec;
    double th, sl;
    tridiag_lowest_host(r.alpha.data(), r.beta.data(), m, &th, &sl, &svec);
    double *y = V;
    double *a = V + 1 * stride, *b = V + 2 * stride;
    double *vj = start_copy, *vp = nullptr, *wbuf = a, *spare = b;
    PD_CUDA(cudaMemsetAsync(y, 0, D * 8, s.st));
    for (int k = 0; k < m; ++k) {
        k_axpy_scalar_f64<<<s.grid_vec, kRedThreads, 0, s.st>>>(y, vj, svec[k], D);
        if (k + 1 == m) break;
        hb_status st = pd_apply(s.h, HB_F64, vj, wbuf, s.st);
        if (st != HB_OK) return st;
        const double bk = r.beta[k];
        k_regen_f64<<<s.grid_vec, kRedThreads, 0, s.st>>>(wbuf, vj, vp, r.alpha[k], k > 0 ? r.beta[k - 1] : 0.0,
                                                          bk != 0 ? 1.0 / bk : 0.0, D);
        double *old_vp = vp ? vp : spare;
        vp = vj;
        vj = wbuf;
        wbuf = old_vp;
    }
    PD_CUDA(cudaGetLastError());
    return HB_OK;
}

}  // namespace

extern "C" {

hb_status hb_continued_fraction(const double *alpha, const double *beta, int n, double norm2, double E0,
                                const double *z_re, const double *z_im, int nz, double *g_re, double *g_im) {
    if (!alpha || n < 1 || (n > 1 && !beta) || nz < 0 || (nz > 0 && (!z_re || !z_im || !g_re || !g_im)))
        return HB_ERR_INVALID_ARG;
    for (int q = 0; q < nz; ++q) {
        const std::complex<double> z(z_re[q] + E0, z_im[q]);
        std::complex<double> g = z - alpha[n - 1];
        for (int j = n - 2; j >= 0; --j) g = z - alpha[j] - beta[j] * beta[j] / g;
        const std::complex<double> G = norm2 / g;
        g_re[q] = G.real();
        g_im[q] = G.imag();
    }
    return HB_OK;
}

hb_status hb_tridiag_lowest(const double *alpha, const double *beta, int n, double *theta, double *s_last) {
    if (!alpha || n < 1 || (n > 1 && !beta) || !theta || !s_last) return HB_ERR_INVALID_ARG;
    tridiag_lowest_host(alpha, beta, n, theta, s_last, nullptr);
    return HB_OK;
}

hb_status lanczos_step_scratch_bytes(hb_handle h, uint64_t *bytes) {
    if (!h || !bytes) return HB_ERR_INVALID_ARG;
    hb_lanczos_opts o{};
    o.maxit = 1;
    o.vec_dtype = HB_F64;
    *bytes = (uint64_t)make_layout(h, o).nblk * 48;  // three 16-byte partials per reduction block
    return HB_OK;
}

// reduction blocks of one step (the partial sums above are per block)
int step_blocks(hb_handle h) {
    hb_lanczos_opts o{};
    o.maxit = 1;
    o.vec_dtype = HB_F64;
    return make_layout(h, o).nblk;
}

hb_status lanczos_step(hb_handle h, hb_dtype dt, const void *v, const void *vprev, void *w, const double *beta_prev,
                       double *alpha, double *beta, void *scratch, uint64_t scratch_bytes, void *ev_hv_begin,
                       void *ev_hv_end, uint32_t *launches, void *stream) {
    if (!h || !v || !w || !alpha || !beta || !scratch || (dt != HB_F64 && dt != HB_F32 && dt != HB_FX64))
        return HB_ERR_INVALID_ARG;
    if ((vprev == nullptr) != (beta_prev == nullptr)) return HB_ERR_INVALID_ARG;
    if (dt == HB_FX64 && !h->fx_ok) return HB_ERR_INVALID_ARG;
    if ((uintptr_t)scratch % 16 != 0) return HB_ERR_INVALID_ARG;
    uint64_t need = 0;
    lanczos_step_scratch_bytes(h, &need);
    if (scratch_bytes < need) return HB_ERR_NO_MEMORY;
    const size_t es = dt == HB_F32 ? 4 : 8;
    const uintptr_t n = (uintptr_t)(h->D * es), wb = (uintptr_t)w;
    for (const void *p : {v, vprev}) {
        const uintptr_t pb = (uintptr_t)p;
        if (p && pb < wb + n && wb < pb + n) return HB_ERR_INVALID_ARG;  // w overlaps an input
    }
    hb_status st = pd_build_tables(h);
    if (st != HB_OK) return st;
    Solve s;
    s.h = h;
    s.st = reinterpret_cast<cudaStream_t>(stream);
    s.D = h->D;
    s.nblk = step_blocks(h);
    s.partials = static_cast<double *>(scratch);
    s.grid_vec = h->sm_count * 8;
    cudaEvent_t e0 = reinterpret_cast<cudaEvent_t>(ev_hv_begin), e1 = reinterpret_cast<cudaEvent_t>(ev_hv_end);
    if (dt == HB_F64)
        st = three_term_step<double>(s, dt, static_cast<const double *>(v), static_cast<const double *>(vprev),
                                     static_cast<double *>(w), beta_prev, alpha, beta, true, e0, e1);
    else if (dt == HB_FX64)
        st = three_term_step_fx(s, static_cast<const int64_t *>(v), static_cast<const int64_t *>(vprev),
                                static_cast<int64_t *>(w), beta_prev, alpha, beta, true, e0, e1);
    else
        st = three_term_step<float>(s, dt, static_cast<const float *>(v), static_cast<const float *>(vprev),
                                    static_cast<float *>(w), beta_prev, alpha, beta, true, e0, e1);
    if (st == HB_OK && launches) *launches += (uint32_t)(pd_hv_launches(h, dt) + (dt == HB_F64 ? 5 : 3));
    return st;
}

hb_status lanczos_workspace_bytes(hb_handle h, const hb_lanczos_opts *o, uint64_t *bytes) {
    if (!h || !o || !bytes || o->maxit < 1) return HB_ERR_INVALID_ARG;
    if (o->vec_dtype != HB_F64 && o->vec_dtype != HB_F32 && o->vec_dtype != HB_FX64) return HB_ERR_INVALID_ARG;
    *bytes = make_layout(h, *o).total;
    return HB_OK;
}

hb_status lanczos_ground_state(hb_handle h, const hb_lanczos_opts *o, const void *v0, void *workspace,
                               uint64_t workspace_bytes, double *alphas, double *betas, double *E0,
                               hb_lanczos_info *info, void *stream) {
    const auto t0 = std::chrono::steady_clock::now();
    if (!h || !o || !E0 || !workspace || o->maxit < 1 || o->check_every < 1) return HB_ERR_INVALID_ARG;
    if (o->vec_dtype != HB_F64 && o->vec_dtype != HB_F32 && o->vec_dtype != HB_FX64) return HB_ERR_INVALID_ARG;
    if ((o->vec_dtype == HB_FX64 || o->fp64_finish == 2) && (!h->fx_ok || o->reorth)) return HB_ERR_INVALID_ARG;
    if (o->fp64_finish < 0 || o->fp64_finish > 2) return HB_ERR_INVALID_ARG;
    const Layout L = make_layout(h, *o);
    if (workspace_bytes < L.total) return HB_ERR_NO_MEMORY;
    if ((uintptr_t)workspace % 256 != 0) return HB_ERR_INVALID_ARG;
    hb_status st = pd_build_tables(h);
    if (st != HB_OK) return st;

    char *ws = static_cast<char *>(workspace);
    Solve s;
    s.h = h;
    s.st = reinterpret_cast<cudaStream_t>(stream);
    s.D = h->D;
    s.nblk = L.nblk;
    s.partials = reinterpret_cast<double *>(ws + L.partials);
    s.d_alpha = reinterpret_cast<double *>(ws + L.scal);
    s.d_beta = s.d_alpha + (o->maxit + 1);
    s.d_coef = s.d_beta + (o->maxit + 1);
    s.d_misc = s.d_coef + (o->maxit + 1);
    s.grid_vec = h->sm_count * 8;
    const uint64_t D = h->D;
    const hb_dtype dt = (hb_dtype)o->vec_dtype;
    const uint64_t es = dt == HB_F32 ? 4 : 8;
    const uint64_t stride = align256(D * es) / es;
    const bool reorth = o->reorth != 0;
    const double tol = o->tol;

    PhaseResult r;
    int iters_f32 = 0;
    bool ran_finish = false;
    if (dt == HB_F64) {
        double *V = reinterpret_cast<double *>(ws + L.vec);
        if (v0)
            k_copy<double><<<s.grid_vec, kRedThreads, 0, s.st>>>(static_cast<const double *>(v0), V, D);
        else
            k_fill_random<double><<<s.grid_vec, kRedThreads, 0, s.st>>>(V, D, o->seed);
        if ((st = normalise(s, V)) != HB_OK) return st;
        st = lanczos_run<double>(s, HB_F64, V, stride, o->maxit, reorth, tol, o->check_every, r);
    } else if (dt == HB_FX64) {
        int64_t *V = reinterpret_cast<int64_t *>(ws + L.vec);
        if (v0)
            k_copy<int64_t><<<s.grid_vec, kRedThreads, 0, s.st>>>(static_cast<const int64_t *>(v0), V, D);
        else
            k_fill_random_fx<<<s.grid_vec, kRedThreads, 0, s.st>>>(V, D, o->seed, h->fx_frac);
        if ((st = normalise(s, V)) != HB_OK) return st;
        st = lanczos_run<int64_t>(s, HB_FX64, V, stride, o->maxit, false, tol, o->check_every, r);
    } else {
        float *V = reinterpret_cast<float *>(ws + L.vec);
        if (v0)
            k_copy_f32<<<s.grid_vec, kRedThreads, 0, s.st>>>(static_cast<const float *>(v0), V, D);
        else
            k_fill_random<float><<<s.grid_vec, kRedThreads, 0, s.st>>>(V, D, o->seed);
        if ((st = normalise(s, V)) != HB_OK) return st;
        const bool finish = o->fp64_finish && !reorth;
        const double tol32 = finish ? std::pow(10.0, o->f32_tol_exp != 0 ? o->f32_tol_exp : -5) : tol;
        // keep a copy of the normalised start: the Ritz vector is regenerated from it
        float *start_copy = finish ? reinterpret_cast<float *>(ws + L.vec2) : nullptr;
        if (finish) k_copy_f32<<<s.grid_vec, kRedThreads, 0, s.st>>>(V, start_copy, D);
        const bool keep = finish && o->store_basis > 0;
        const int maxit32 = keep ? std::min(o->maxit, o->store_basis) : o->maxit;
        st = lanczos_run<float>(s, HB_F32, V, stride, maxit32, reorth, tol32, o->check_every, r, keep);
        iters_f32 = r.iters;
        if (st == HB_OK && finish && !(r.converged && tol32 <= tol)) {
            // Ritz vector of the float32 phase, then continue in float64 / fixed point: one
            // combination pass over the kept vectors, or a replay of the recurrence from the start
            const int m = r.iters;
            float *y = V;
            if (keep) {
                std::vector<double> svec;
                double th, sl;
                tridiag_lowest_host(r.alpha.data(), r.beta.data(), m, &th, &sl, &svec);
                PD_CUDA(cudaMemcpyAsync(s.d_coef, svec.data(), sizeof(double) * m, cudaMemcpyHostToDevice, s.st));
                y = start_copy;  // the start copy is not needed: the vectors are kept
                k_combine_f32<<<s.grid_vec, kRedThreads, 0, s.st>>>(V, stride, m, s.d_coef, y, D);
            } else if ((st = replay_ritz_f32(s, r, start_copy, V, stride)) != HB_OK) {
                return st;
            }
            PD_CUDA(cudaGetLastError());
            const uint64_t stride64 = align256(D * 8) / 8;
            const int rest = std::max(1, o->maxit - m);
            ran_finish = true;
            if (o->fp64_finish == 2) {
                int64_t *Vfx = reinterpret_cast<int64_t *>(ws + L.vec2 + align256(D * 4));
                k_f32_to_fx<<<s.grid_vec, kRedThreads, 0, s.st>>>(y, Vfx, D, h->fx_frac);
                if ((st = normalise(s, Vfx)) != HB_OK) return st;
                st = lanczos_run<int64_t>(s, HB_FX64, Vfx, stride64, rest, false, tol, o->check_every, r);
            } else {
                double *V64 = reinterpret_cast<double *>(ws + L.vec2 + align256(D * 4));
                k_f32_to_f64<<<s.grid_vec, kRedThreads, 0, s.st>>>(y, V64, D);
                if ((st = normalise(s, V64)) != HB_OK) return st;
                st = lanczos_run<double>(s, HB_F64, V64, stride64, rest, false, tol, o->check_every, r);
            }
        }
    }
    PD_CUDA(cudaStreamSynchronize(s.st));
    if (st != HB_OK) return st;
    *E0 = r.theta;
    if (alphas) std::copy(r.alpha.begin(), r.alpha.end(), alphas);
    if (betas) std::copy(r.beta.begin(), r.beta.end(), betas);
    const hb_status outcome = r.converged || tol <= 0 ? HB_OK : HB_ERR_NOT_CONVERGED;
    if (info) {
        info->E0 = r.theta;
        info->residual = r.res;
        info->iterations = ran_finish ? iters_f32 + r.iters : r.iters;
        info->iterations_f32 = dt == HB_F32 ? iters_f32 : 0;
        info->status = outcome;
        info->converged = r.converged ? 1 : 0;
        info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    return outcome;
}

hb_status lanczos_ritz_vector_f32(hb_handle h, const hb_lanczos_opts *o, const void *v0, void *workspace,
                                  uint64_t workspace_bytes, float *ritz, double *E0, hb_lanczos_info *info,
                                  void *stream) {
    if (!h || !o || !workspace || !ritz || !E0 || o->maxit < 1 || o->check_every < 1 || o->reorth)
        return HB_ERR_INVALID_ARG;
    hb_lanczos_opts oo = *o;
    oo.vec_dtype = HB_F32;
    oo.fp64_finish = 1;  // same workspace layout (keeps the start copy)
    const Layout L = make_layout(h, oo);
    if (workspace_bytes < L.total) return HB_ERR_NO_MEMORY;
    if ((uintptr_t)workspace % 256 != 0) return HB_ERR_INVALID_ARG;
    hb_status st = pd_build_tables(h);
    if (st != HB_OK) return st;
    const auto t0 = std::chrono::steady_clock::now();
    char *ws = static_cast<char *>(workspace);
    Solve s;
    s.h = h;
    s.st = reinterpret_cast<cudaStream_t>(stream);
    s.D = h->D;
    s.nblk = L.nblk;
    s.partials = reinterpret_cast<double *>(ws + L.partials);
    s.d_alpha = reinterpret_cast<double *>(ws + L.scal);
    s.d_beta = s.d_alpha + (oo.maxit + 1);
    s.d_coef = s.d_beta + (oo.maxit + 1);
    s.d_misc = s.d_coef + (oo.maxit + 1);
    s.grid_vec = h->sm_count * 8;
    const uint64_t D = h->D, stride = align256(D * 4) / 4;
    float *V = reinterpret_cast<float *>(ws + L.vec);
    float *start_copy = reinterpret_cast<float *>(ws + L.vec2);
    if (v0)
        k_copy_f32<<<s.grid_vec, kRedThreads, 0, s.st>>>(static_cast<const float *>(v0), V, D);
    else
        k_fill_random<float><<<s.grid_vec, kRedThreads, 0, s.st>>>(V, D, oo.seed);
    if ((st = normalise(s, V)) != HB_OK) return st;
    k_copy_f32<<<s.grid_vec, kRedThreads, 0, s.st>>>(V, start_copy, D);
    PhaseResult r;
    st = lanczos_run<float>(s, HB_F32, V, stride, oo.maxit, false, oo.tol, oo.check_every, r);
    if (st != HB_OK) return st;
    if ((st = replay_ritz_f32(s, r, start_copy, V, stride)) != HB_OK) return st;
    if ((st = normalise(s, V)) != HB_OK) return st;
    k_copy_f32<<<s.grid_vec, kRedThreads, 0, s.st>>>(V, ritz, D);
    PD_CUDA(cudaStreamSynchronize(s.st));
    *E0 = r.theta;
    if (info) {
        info->E0 = r.theta;
        info->residual = r.res;
        info->iterations = r.iters;
        info->iterations_f32 = r.iters;
        info->status = r.converged ? HB_OK : HB_ERR_NOT_CONVERGED;
        info->converged = r.converged;
        info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    return r.converged ? HB_OK : HB_ERR_NOT_CONVERGED;
}

hb_status lanczos_ritz_vector_f64(hb_handle h, const hb_lanczos_opts *o, const void *v0, void *workspace,
                                  uint64_t workspace_bytes, double *ritz, double *E0, hb_lanczos_info *info,
                                  void *stream) {
    if (!h || !o || !workspace || !ritz || !E0 || o->maxit < 1 || o->check_every < 1 || o->reorth)
        return HB_ERR_INVALID_ARG;
    hb_lanczos_opts oo = *o;
    oo.vec_dtype = HB_F64;
    oo.fp64_finish = 0;
    const Layout L = make_layout(h, oo);
    const uint64_t D = h->D, stride = align256(D * 8) / 8;
    if (workspace_bytes < L.total + align256(D * 8)) return HB_ERR_NO_MEMORY;
    if ((uintptr_t)workspace % 256 != 0) return HB_ERR_INVALID_ARG;
    hb_status st = pd_build_tables(h);
    if (st != HB_OK) return st;
    const auto t0 = std::chrono::steady_clock::now();
    char *ws = static_cast<char *>(workspace);
    Solve s;
    s.h = h;
    s.st = reinterpret_cast<cudaStream_t>(stream);
    s.D = D;
    s.nblk = L.nblk;
    s.partials = reinterpret_cast<double *>(ws + L.partials);
    s.d_alpha = reinterpret_cast<double *>(ws + L.scal);
    s.d_beta = s.d_alpha + (oo.maxit + 1);
    s.d_coef = s.d_beta + (oo.maxit + 1);
    s.d_misc = s.d_coef + (oo.maxit + 1);
    s.grid_vec = h->sm_count * 8;
    double *V = reinterpret_cast<double *>(ws + L.vec);
    double *start_copy = reinterpret_cast<double *>(ws + L.total);
    if (v0)
        k_copy<double><<<s.grid_vec, kRedThreads, 0, s.st>>>(static_cast<const double *>(v0), V, D);
    else
        k_fill_random<double><<<s.grid_vec, kRedThreads, 0, s.st>>>(V, D, oo.seed);
    if ((st = normalise(s, V)) != HB_OK) return st;
    k_copy<double><<<s.grid_vec, kRedThreads, 0, s.st>>>(V, start_copy, D);
    PhaseResult r;
    st = lanczos_run<double>(s, HB_F64, V, stride, oo.maxit, false, oo.tol, oo.check_every, r);
    if (st != HB_OK) return st;
    if ((st = replay_ritz_f64(s, r, start_copy, V, stride)) != HB_OK) return st;
    if ((st = normalise(s, V)) != HB_OK) return st;
    k_copy<double><<<s.grid_vec, kRedThreads, 0, s.st>>>(V, ritz, D);
    PD_CUDA(cudaStreamSynchronize(s.st));
    *E0 = r.theta;
    if (info) {
        info->E0 = r.theta;
        info->residual = r.res;
        info->iterations = r.iters;
        info->iterations_f32 = 0;
        info->status = r.converged ? HB_OK : HB_ERR_NOT_CONVERGED;
        info->converged = r.converged;
        info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    return r.converged ? HB_OK : HB_ERR_NOT_CONVERGED;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free variant of lanczos_step.
//
// The only scratch lanczos_step needs is one float64 partial sum per reduction
// block (three for the float32 step's fused sums).  This variant keeps that scratch in a fixed file-scope device array,
// so neither the library nor the caller allocates anything per call.  In host
// code `g_noalloc_partials` names a host-side shadow, not device memory: its
// device address is looked up with cudaGetSymbolAddress on every call, with the
// handle's device current, so a device or context reset between two calls can
// never leave a stale address behind (the lookup costs about a microsecond once
// the module is loaded).  Every block of the two reductions overwrites its own slot
// before the final reduction reads it, so no slot has to start at zero; the
// array simply keeps whatever the previous call left.  All calls on a device
// share the array: two calls whose kernels overlap on the GPU race on it.
// The fixed-point step needs three 128-bit partials per block (six doubles),
// more than the array holds on a GB300, so HB_FX64 is refused.

#define PD_NOALLOC_PARTIALS 2048  // capacity: 2048 doubles = 16 KiB per device

static __device__ __align__(256) double g_noalloc_partials[PD_NOALLOC_PARTIALS];

extern "C" hb_status lanczos_step_noalloc(hb_handle h, hb_dtype dt, const void *v, const void *vprev, void *w,
                                          const double *beta_prev, double *alpha, double *beta, void *ev_hv_begin,
                                          void *ev_hv_end, uint32_t *launches, void *stream) {
    if (!h || !v || !w || !alpha || !beta || (dt != HB_F64 && dt != HB_F32)) return HB_ERR_INVALID_ARG;
    if ((vprev == nullptr) != (beta_prev == nullptr)) return HB_ERR_INVALID_ARG;
    int dev = -1;
    PD_CUDA(cudaGetDevice(&dev));
    if (dev != h->device) return HB_ERR_INVALID_ARG;  // checked before anything is enqueued
    if (!h->tables_built) return HB_ERR_INVALID_STATE;  // building them would allocate
    const size_t es = dt == HB_F64 ? 8 : 4;
    const uintptr_t n = (uintptr_t)(h->D * es), wb = (uintptr_t)w;
    for (const void *p : {v, vprev}) {
        const uintptr_t pb = (uintptr_t)p;
        if (p && pb < wb + n && wb < pb + n) return HB_ERR_INVALID_ARG;
    }
    const uint64_t nblk = (uint64_t)step_blocks(h);  // up to three float64 partials per block are used here
    if (3 * nblk > PD_NOALLOC_PARTIALS) return HB_ERR_NO_MEMORY;  // device wider than the fixed scratch
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_partials) != cudaSuccess || !p) return HB_ERR_CUDA;
    Solve s;
    s.h = h;
    s.st = reinterpret_cast<cudaStream_t>(stream);
    s.D = h->D;
    s.nblk = (int)nblk;
    s.partials = static_cast<double *>(p);
    s.grid_vec = h->sm_count * 8;
    cudaEvent_t e0 = reinterpret_cast<cudaEvent_t>(ev_hv_begin), e1 = reinterpret_cast<cudaEvent_t>(ev_hv_end);
    hb_status st;
    if (dt == HB_F64)
        st = three_term_step<double>(s, dt, static_cast<const double *>(v), static_cast<const double *>(vprev),
                                     static_cast<double *>(w), beta_prev, alpha, beta, true, e0, e1);
    else
        st = three_term_step<float>(s, dt, static_cast<const float *>(v), static_cast<const float *>(vprev),
                                    static_cast<float *>(w), beta_prev, alpha, beta, true, e0, e1);
    if (st == HB_OK && launches) *launches += (uint32_t)(pd_hv_launches(h, dt) + (dt == HB_F64 ? 5 : 3));
    return st;
}

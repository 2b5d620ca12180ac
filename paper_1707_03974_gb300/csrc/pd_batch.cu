// Batched Hubbard problems: many clusters / sectors / U values of uneven
// dimension in single launches, and a batched Lanczos run by one persistent
// cooperative kernel (grid barriers whose waits give up after a limit), whose
// chunks of steps are replayed from a captured CUDA graph.
//
// The paper's method per instance is unchanged (Eq. 1 with Paradeisos-ranked
// hop tables, Eq. 3); the batch only concatenates the instances' vectors and
// flattens their row groups into one work list.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <new>
#include <vector>

#include <cfloat>
#include <type_traits>

#include "pd_exact.cuh"
#include "pd_hv_body.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kFinal = 512;
constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;

struct Inst {
    HvArgs<double> f64;
    HvArgs<float> f32;
    FxArgs fx;
    uint64_t off;  // element offset of the instance's vector in the batch vector
    uint64_t D;
    int F;         // fixed-point fractional bits of this instance
};

// Copies one instance descriptor into shared memory (all threads cooperate).
__device__ __forceinline__ void copy_inst(Inst *dst, const Inst *src) {
    const uint64_t *s = reinterpret_cast<const uint64_t *>(src);
    uint64_t *d = reinterpret_cast<uint64_t *>(dst);
    for (int i = threadIdx.x; i < (int)(sizeof(Inst) / 8); i += blockDim.x) d[i] = s[i];
}

__device__ __forceinline__ int find_inst(const uint64_t *prefix, int n, uint64_t item) {
    int lo = 0, hi = n - 1;  // largest k with prefix[k] <= item
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (prefix[mid] <= item) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// mode 0: float64, 1: float32, 2: fixed point
template <int R, int MODE, int NC>
__global__ void __launch_bounds__(512) k_batch_hv(const Inst *__restrict__ inst, const uint64_t *__restrict__ prefix,
                                                  int n, const int *__restrict__ active, const void *x, void *y) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ __align__(16) unsigned char s_inst_raw[sizeof(Inst)];  // filled by copy_inst, no constructor
    Inst &s_inst = *reinterpret_cast<Inst *>(s_inst_raw);
    __shared__ int s_k;
    const uint64_t total = prefix[n];
    int cur = -1;
    for (uint64_t it = blockIdx.x; it < total; it += gridDim.x) {
        __syncthreads();  // every thread is done with the previous item
        if (threadIdx.x == 0) s_k = find_inst(prefix, n, it);
        __syncthreads();
        const int k = s_k;
        if (active && !active[k]) continue;  // uniform across the CTA
        if (k != cur) {
            copy_inst(&s_inst, inst + k);
            __syncthreads();
            if (MODE == 2) hv_fx_load_diag(s_inst.fx, smem);
            cur = k;
        }
        const uint64_t g = it - prefix[k];
        const uint64_t off = s_inst.off;
        if (MODE == 0)
            hv_group<R, double, true>(s_inst.f64, static_cast<const double *>(x) + off, static_cast<double *>(y) + off,
                                      g, smem);
        else if (MODE == 1)
            hv_group<R, float, true>(s_inst.f32, static_cast<const float *>(x) + off, static_cast<float *>(y) + off, g,
                                     smem);
        else
            hv_fx_group<R, NC, true>(s_inst.fx, static_cast<const int64_t *>(x) + off,
                                     static_cast<int64_t *>(y) + off, g, smem);
    }
}

// ---- split form of the batched fixed-point H·v ----
// Row pass: items (instance k, row group g of R rows), y = diag + spin-down hops
// on the instance's warp-blocked table.  Spin-up pass: items (instance k,
// column block j, row group g), column-block-major within an instance, y +=
// spin-up hops; pairs of columns per thread where D_dn is even.
template <int R, int NC>
__global__ void __launch_bounds__(512) k_batch_row(const Inst *__restrict__ inst, const uint64_t *__restrict__ prefix,
                                                   int n, const int *__restrict__ active, const int64_t *x,
                                                   int64_t *y) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ __align__(16) unsigned char s_inst_raw[sizeof(Inst)];
    Inst &s_inst = *reinterpret_cast<Inst *>(s_inst_raw);
    __shared__ int s_k;
    const uint64_t total = prefix[n];
    int cur = -1;
    for (uint64_t it = blockIdx.x; it < total; it += gridDim.x) {
        __syncthreads();
        if (threadIdx.x == 0) s_k = find_inst(prefix, n, it);
        __syncthreads();
        const int k = s_k;
        if (active && !active[k]) continue;  // uniform across the CTA
        if (k != cur) {
            copy_inst(&s_inst, inst + k);
            __syncthreads();
            hv_fx_load_diag(s_inst.fx, smem);
            cur = k;
        }
        hv_fx_wb_group<R, NC>(s_inst.fx, x + s_inst.off, y + s_inst.off, it - prefix[k], smem);
    }
}

// column block j and row group g of spin-up item `local` of an instance
__device__ __forceinline__ void up_item_of(const FxArgs &a, uint64_t local, int RA, uint64_t *j, uint64_t *g) {
    const uint64_t ng = (a.Du + RA - 1) / RA;
    *j = local / ng;
    *g = local - *j * ng;
}

template <int RR, int NC>
__global__ void __launch_bounds__(512) k_batch_up(const Inst *__restrict__ inst, const uint64_t *__restrict__ up_prefix,
                                                  int n, const int *__restrict__ active, const int64_t *x,
                                                  int64_t *y, int W, int S) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ __align__(16) unsigned char s_inst_raw[sizeof(Inst)];
    Inst &s_inst = *reinterpret_cast<Inst *>(s_inst_raw);
    __shared__ int s_k;
    const uint64_t total = up_prefix[n];
    int cur = -1;
    for (uint64_t it = blockIdx.x; it < total; it += gridDim.x) {
        __syncthreads();
        if (threadIdx.x == 0) s_k = find_inst(up_prefix, n, it);
        __syncthreads();
        const int k = s_k;
        if (active && !active[k]) continue;
        if (k != cur) {
            copy_inst(&s_inst, inst + k);
            __syncthreads();
            cur = k;
        }
        uint64_t j, g;
        up_item_of(s_inst.fx, it - up_prefix[k], S * RR, &j, &g);
        const int64_t *xk = x + s_inst.off;
        int64_t *yk = y + s_inst.off;
        if (s_inst.fx.Dd % 2 == 0)
            hv_fx_up_item<RR, NC, true, 2>(s_inst.fx, xk, yk, j, g, W, S, smem);
        else
            hv_fx_up_item<RR, NC, true, 1>(s_inst.fx, xk, yk, j, g, W, S, smem);
    }
}

// ---------------- batched Lanczos: one persistent kernel for all instances ----------------
using pdx::block_sum128;
using pdx::block_sum_d;
using pdx::I128;
using pdx::i128_add;
using pdx::i128_add_prod;

// Start vectors (instance k: SplitMix64 seeded with seed + k, normalised).
// Grid: x = blocks per instance, y = instance.
struct StartState {
    const Inst *inst;
    void *V;    // slot 0 of the batch vector
    I128 *part; // [n][nb]
    int nb;
};

template <bool FX>
__global__ void k_b_fill(StartState s, uint64_t seed) {
    const int k = blockIdx.y;
    const Inst &in = s.inst[k];
    const uint64_t sk = seed + (uint64_t)k;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < in.D; i += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t z = sk + (i + 1) * kGamma;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z = z ^ (z >> 31);
        if (FX) {
            // scaled by 2^-16 so that the un-normalised norm stays far inside 128 bits
            const int64_t kq = (int64_t)(z >> 11);
            const int sh = 52 - (in.F - 16);
            const int64_t q = sh >= 0 ? ((kq + (sh > 0 ? (1ll << (sh - 1)) : 0)) >> sh) : (kq << -sh);
            static_cast<int64_t *>(s.V)[in.off + i] = q - (1ll << (in.F - 16));
        } else {
            static_cast<double *>(s.V)[in.off + i] = (double)(z >> 11) * 0x1.0p-52 - 1.0;
        }
    }
}

template <bool FX>
__global__ void k_b_norm_partials(StartState s) {
    const int k = blockIdx.y;
    const Inst &in = s.inst[k];
    if (FX) {
        const int64_t *v = static_cast<const int64_t *>(s.V) + in.off;
        I128 acc;
        for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < in.D; i += (uint64_t)gridDim.x * blockDim.x)
            i128_add_prod(acc, v[i], v[i]);
        const I128 t = block_sum128(acc);
        if (threadIdx.x == 0) s.part[k * s.nb + blockIdx.x] = t;
    } else {
        const double *v = static_cast<const double *>(s.V) + in.off;
        double acc = 0.0;
        for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < in.D; i += (uint64_t)gridDim.x * blockDim.x)
            acc = fma(v[i], v[i], acc);
        const double t = block_sum_d(acc);
        if (threadIdx.x == 0) reinterpret_cast<double *>(s.part)[2 * (k * s.nb + blockIdx.x)] = t;
    }
}

// slot 0 of instance k *= 1 / sqrt(sum of its partials)
template <bool FX>
__global__ void k_b_normalise(StartState s) {
    const int k = blockIdx.x;
    const Inst &in = s.inst[k];
    __shared__ double s_f;
    double nrm2;
    if (FX) {
        I128 acc;
        for (int i = threadIdx.x; i < s.nb; i += blockDim.x) i128_add(acc, s.part[k * s.nb + i]);
        acc = block_sum128(acc);
        nrm2 = ldexp((double)acc.hi * 18446744073709551616.0 + (double)acc.lo, -2 * in.F);
    } else {
        double acc = 0.0;
        for (int i = threadIdx.x; i < s.nb; i += blockDim.x) acc += reinterpret_cast<const double *>(s.part)[2 * (k * s.nb + i)];
        nrm2 = block_sum_d(acc);
    }
    if (threadIdx.x == 0) s_f = nrm2 > 0 ? 1.0 / sqrt(nrm2) : 0.0;
    __syncthreads();
    const double f = s_f;
    if (FX) {
        int64_t *v = static_cast<int64_t *>(s.V) + in.off;
        const FxCoef c = fx_coef_dev(f);
        for (uint64_t i = threadIdx.x; i < in.D; i += blockDim.x) v[i] = fx_mul(v[i], c.K, c.G);
    } else {
        double *v = static_cast<double *>(s.V) + in.off;
        for (uint64_t i = threadIdx.x; i < in.D; i += blockDim.x) v[i] *= f;
    }
}

// ---- bounded grid barrier ----
// All CTAs of a cooperative launch meet here.  A CTA whose wait exceeds
// limit_ns (measured on the global nanosecond timer; a poll count caps it as
// well) raises `abort` and records where; every CTA then leaves the kernel at
// its next barrier, so nothing waits forever and the host reads HB_ERR_TIMEOUT.
struct GridSync {
    unsigned count;  // arrivals in the current generation
    unsigned gen;    // generation, bumped by the last arrival
    unsigned abort;  // 1 once a wait gave up
    unsigned where;  // 1 + index of the barrier that gave up
};

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(unsigned *p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ bool grid_barrier(GridSync *gs, unsigned long long limit_ns, unsigned tag) {
    __shared__ int s_ok;
    __syncthreads();  // the CTA's work of this phase is done
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned g = ld_acquire(&gs->gen);
        __threadfence();  // this CTA's writes are visible before its arrival counts
        if (atomicAdd(&gs->count, 1u) == gridDim.x - 1) {
            atomicExch(&gs->count, 0u);
            __threadfence();
            st_release(&gs->gen, g + 1);
        } else {
            const unsigned long long t0 = global_ns();
            const unsigned long long max_polls = (limit_ns >> 5) + 1024;
            for (unsigned long long polls = 0; ld_acquire(&gs->gen) == g; ++polls) {
                if (ld_acquire(&gs->abort)) {
                    ok = 0;
                    break;
                }
                if (polls >= max_polls || global_ns() - t0 > limit_ns) {
                    atomicExch(&gs->where, tag + 1);
                    atomicExch(&gs->abort, 1u);
                    ok = 0;
                    break;
                }
                __nanosleep(32);
            }
        }
        if (ok && ld_acquire(&gs->abort)) ok = 0;
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// ---- lowest eigenpair of the Lanczos tridiagonal, on the device (one warp) ----
// FP64 runs at a small fraction of the FP32 rate on this GPU, so the check is
// written to need few FP64 instructions per row: the Sturm counts and Newton
// corrections come from the three-term recurrence of the leading principal
// minors (no division per row), and the eigenvector's last component from one
// twisted factorisation instead of inverse iteration.

// p_i = det(T_i - x I) (T_i the leading i x i block; p_0 = 1) and its derivative
// in x, by p_i = (a_i - x) p_{i-1} - b_{i-1}^2 p_{i-2}; both are rescaled by a
// power of two whenever they leave [2^-256, 2^256].  count = sign changes of
// p_0 .. p_n = eigenvalues of T_n below x (a zero p_i takes the sign opposite
// to p_{i-1}).  b2: squared off-diagonals.
struct TriEval {
    int count;
    double p, dp;
};
__device__ __forceinline__ int exp_of(double v) { return ((__double2hiint(v) >> 20) & 0x7ff) - 1023; }
__device__ TriEval tri_eval(const double *a, const double *b2, int n, double x) {
    double p2 = 0.0, p1 = 1.0, d2 = 0.0, d1 = 0.0;
    int s1 = 0, c = 0;
    for (int i = 0; i < n; ++i) {
        const double bb = i > 0 ? b2[i - 1] : 0.0;
        const double d = a[i] - x;
        const double p = fma(d, p1, -bb * p2);
        const double dp = fma(d, d1, -fma(bb, d2, p1));
        const int s = p != 0.0 ? (p < 0.0 ? 1 : 0) : 1 - s1;
        c += s != s1;
        p2 = p1;
        p1 = p;
        d2 = d1;
        d1 = dp;
        s1 = s;
        const int e = min(max(exp_of(p1), exp_of(d1)), 1022);
        if (e > 256 || e < -256) {
            const double f = __hiloint2double((1023 - e) << 20, 0);  // 2^-e, exact
            p2 *= f;
            p1 *= f;
            d2 *= f;
            d1 *= f;
        }
    }
    return {c, p1, d1};
}

__device__ __forceinline__ double warp_min_d(double v) {
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ double warp_max_d(double v) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// theta = lowest eigenvalue of T_n (diagonal a[0..n), squared off-diagonal
// b2[0..n-1), off-diagonal b[0..n-1)) and s_last = |last component| of its
// normalised eigenvector.  Called by all 32 lanes of one warp; dp, dm: n
// doubles each (work).
//
// theta: each pass evaluates the recurrence at 32 points of the bracket
// [lo, hi] (lane 0 at lo).  A point with no eigenvalue below it is a lower
// bound, and so is its Newton iterate on det(T_n - x I): left of the smallest
// root of a polynomial with real roots, Newton steps rise monotonically
// towards that root.  A point with an eigenvalue below it is an upper bound.
// Passes stop when lo's Newton correction is at rounding level, or the bracket
// stops shrinking.
//
// s_last: the twisted factorisation of T_n - theta I (Dhillon and Parlett):
// forward pivots dp (lane 0) and backward pivots dm (lane 1) in one pass,
// gamma_k = dp_k + dm_k - (a_k - theta), and the eigenvector solved from the
// row k of smallest |gamma_k| outwards with z_k = 1.
__device__ void tri_lowest_warp(const double *a, const double *b2, const double *b, int n, double *dp,
                                double *dm, double *theta, double *s_last) {
    const int lane = threadIdx.x & 31;
    if (n == 1) {
        *theta = a[0];
        *s_last = 1.0;
        return;
    }
    double lo = INFINITY, hi = -INFINITY, amax = 0.0;
    for (int i = lane; i < n; i += 32) {
        const double r = (i > 0 ? fabs(b[i - 1]) : 0.0) + (i + 1 < n ? fabs(b[i]) : 0.0);
        lo = fmin(lo, a[i] - r);
        hi = fmax(hi, a[i] + r);
        amax = fmax(amax, fabs(a[i]) + r);
    }
    lo = warp_min_d(lo);
    hi = warp_max_d(hi);
    amax = warp_max_d(amax);
    for (int pass = 0; pass < 64; ++pass) {
        const double x = lane == 0 ? lo : lo + (hi - lo) * ((double)lane / 32.0);
        const TriEval ev = tri_eval(a, b2, n, x);
        double up = INFINITY, down = -INFINITY;
        bool small = false;
        if (ev.count >= 1) {
            up = x;
        } else {
            down = x;
            if (ev.dp != 0.0) {
                const double step = -ev.p / ev.dp;  // >= 0 below the smallest root
                if (step > 0.0 && isfinite(step)) down = x + step;
                small = !(fabs(step) > 4.0 * DBL_EPSILON * fmax(fabs(x), DBL_EPSILON * amax));
            }
        }
        const bool stop = __shfl_sync(0xffffffffu, small ? 1 : 0, 0) != 0;  // lo's correction is negligible
        const double nhi = fmin(hi, warp_min_d(up));
        double nlo = fmax(lo, warp_max_d(down));
        if (nlo > nhi) nlo = nhi;  // a Newton iterate past an upper bound is rounding
        const bool progress = nhi - nlo < hi - lo;
        if (progress) {
            lo = nlo;
            hi = nhi;
        }
        if (stop || !progress || !(hi - lo > 4.0 * DBL_EPSILON * fmax(fabs(lo), fabs(hi)))) break;
    }
    const double th = lo;
    // forward (lane 0) and backward (lane 1) pivots of T_n - th I
    const double tiny = DBL_EPSILON * (amax > 0.0 ? amax : 1.0);
    if (lane < 2) {
        double prev = 1.0;
        double *out = lane == 0 ? dp : dm;
        for (int t = 0; t < n; ++t) {
            const int i = lane == 0 ? t : n - 1 - t;
            double d = a[i] - th;
            if (t > 0) d -= b2[lane == 0 ? i - 1 : i] / prev;
            if (d == 0.0) d = tiny;
            out[i] = d;
            prev = d;
        }
    }
    __syncwarp();
    double g = INFINITY;
    int k = n;
    for (int i = lane; i < n; i += 32) {
        const double gi = fabs(dp[i] + dm[i] - (a[i] - th));
        if (gi < g) {
            g = gi;
            k = i;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        const double go = __shfl_xor_sync(0xffffffffu, g, o);
        const int ko = __shfl_xor_sync(0xffffffffu, k, o);
        if (go < g || (go == g && ko < k)) {
            g = go;
            k = ko;
        }
    }
    if (k >= n) k = 0;  // every gamma was NaN: fall back to the first row
    // z: lane 0 from row k towards row 0, lane 1 from row k towards row n - 1
    double z = 1.0, ss = 0.0;
    if (lane < 2) {
        const int len = lane == 0 ? k : n - 1 - k;
        for (int t = 0; t < len; ++t) {
            const int i = lane == 0 ? k - 1 - t : k + t;
            const double piv = lane == 0 ? dp[i] : dm[i + 1];
            z = -(b[i] / piv) * z;
            ss = fma(z, z, ss);
        }
    }
    const double ss0 = __shfl_sync(0xffffffffu, ss, 0), ss1 = __shfl_sync(0xffffffffu, ss, 1);
    const double zl = __shfl_sync(0xffffffffu, z, 1);
    *theta = th;
    *s_last = fabs(zl) / sqrt(1.0 + ss0 + ss1);
}

// ---- the persistent kernel ----
struct PState {
    const Inst *inst;
    const uint64_t *prefix;  // [n+1] prefix sums of row groups (items)
    int n;
    int *active;             // [n]
    int *jdev;               // step index, carried across launches
    int *n_active;           // active instances after the launch
    int chunk, maxit, maxit1, check_every;
    double tol;
    uint64_t stride;         // elements per vector slot
    uint64_t total;          // elements of one batch vector (instance k at [off_k, off_k + D_k))
    void *V;                 // three slots
    I128 *part;              // [n][grid][3] per-CTA partial sums
    double *alpha, *beta;    // [n][maxit1]
    double *theta, *res;     // [n]
    int *iters, *conv;       // [n]
    double *tri_ws;          // [n][3 maxit1]: beta^2 and the pivots of checks longer than kTriSmem
    GridSync *gs;
    unsigned long long limit_ns;
    int withhold;            // CTA that leaves before its first arrival (the wait self-test), -1: none
    const uint64_t *up_prefix;  // split form: prefix sums of the spin-up items
    int up_W, up_S;             // split form: spin-up columns per block and row slots (up_W * up_S threads)
    I128 *item_part;            // [items of the fused pass][8 warps]: per-warp partials of <w, v>
};

// Store hook of the H·v (fixed point): w = H v - beta_prev vprev and the exact
// sum <w, v> of the elements this thread wrote.
struct FxStepEpi {
    int64_t *w;
    const int64_t *vprev;
    int64_t Kb;
    int Gb, has_prev;
    I128 swv;
    __device__ __forceinline__ void store(uint64_t i, int64_t hv, int64_t v) {
        int64_t wi = hv;
        if (has_prev) wi -= fx_mul(vprev[i], Kb, Gb);
        w[i] = wi;
        i128_add_prod(swv, wi, v);
    }
};

// float64: w = H v - beta_prev vprev and <w, v> (the textbook first reduction)
struct F64StepEpi {
    double *w;
    const double *vprev;
    double bprev;
    int has_prev;
    double swv;
    __device__ __forceinline__ void store(uint64_t i, double hv, double v) {
        double wi = hv;
        if (has_prev) wi = wi - bprev * vprev[i];
        w[i] = wi;
        swv = fma(wi, v, swv);
    }
};

constexpr int kPThreads = 256;
constexpr int kPUpRR = 4;        // spin-up rows per thread in the persistent kernel
constexpr int kPMinBlocks = 4;    // CTAs per SM the persistent kernel's light variants are compiled for
constexpr int kSmemPrefix = 512;  // batches of up to this many instances keep their item prefix sums in shared memory
constexpr int kTriSmem = 768;     // Lanczos lengths up to this are checked with the tridiagonal in shared memory
constexpr size_t kTriSmemBytes = (size_t)5 * kTriSmem * 8;  // alpha, beta, beta^2 and two pivot arrays

// w[e] = f(w[e], v[e]) for every element e of [e0, e1) handled by this thread
// (v may be null: f then gets 0): the loads of four elements (e, e + T, e + 2T,
// e + 3T) are issued before any of their stores, so each thread keeps eight
// loads in flight (the pointers are restrict: w and v never overlap).  f may
// accumulate on the side; it must not depend on another element's result.
template <typename T, typename Fn>
__device__ __forceinline__ void slice_update(uint64_t e0, uint64_t e1, T *__restrict__ w, const T *__restrict__ v,
                                             Fn f) {
    const uint64_t Tn = blockDim.x;
    uint64_t e = e0 + threadIdx.x;
    for (; e + 3 * Tn < e1; e += 4 * Tn) {
        T wv[4], vv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            wv[u] = w[e + u * Tn];
            vv[u] = v ? v[e + u * Tn] : T(0);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) w[e + u * Tn] = f(wv[u], vv[u]);
    }
    for (; e < e1; e += Tn) w[e] = f(w[e], v ? v[e] : T(0));
}

// The next item at or after `it` (items of this CTA are it, it + G, ...) whose
// instance is active: items of an inactive instance are skipped in one jump.
// Every thread of the CTA computes the same answer from the same data, so the
// loop needs no barrier.  Returns false when no such item is left.
__device__ __forceinline__ bool next_active_item(const uint64_t *pre, int n, const int *active, uint64_t total,
                                                 unsigned G, uint64_t &it, int &k) {
    while (it < total) {
        k = find_inst(pre, n, it);
        if (active[k]) return true;
        const uint64_t end = pre[k + 1];  // first item of the next instance
        it += (end - it + G - 1) / G * G;
    }
    return false;
}

// first instance whose vector ends after element e (instances ordered by offset)
__device__ __forceinline__ int inst_at(const Inst *inst, int n, uint64_t e) {
    int lo = 0, hi = n - 1;  // largest k with off_k <= e
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (inst[mid].off <= e) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Lanczos steps j = *jdev .. for every active instance, until chunk steps, maxit
// or convergence of all.  Per step: phase A, the H·v of all row groups of all
// active instances fused with w = H v - beta vprev and the first reduction
// <w, v> (per-CTA partials per instance); barrier; phase B, alpha = <w, v>,
// w -= alpha v and the partials of ||w||^2 over a contiguous slice of the batch
// vector per CTA; barrier; phase C, beta = ||w||, w /= beta, and, every
// check_every steps, the tridiagonal solve of each instance by the CTA that
// holds its first element; barrier.  With fixed-point vectors both reductions
// are exact 128-bit sums (converted to float64 once, through double-double).
template <int R, int NC, bool FX, bool SPLIT>
__global__ void __launch_bounds__(kPThreads, (FX && NC <= 2 && R <= 2) ? kPMinBlocks : 3) k_batch_lanczos(PState p) {
    static_assert(FX || !SPLIT, "the split form is fixed point only");
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ __align__(16) unsigned char s_inst_raw[sizeof(Inst)];  // filled by copy_inst, no constructor
    Inst &s_inst = *reinterpret_cast<Inst *>(s_inst_raw);
    __shared__ double s_ab[2];
    __shared__ uint64_t s_prefix[kSmemPrefix + 1];  // item prefix sums, when the batch is small enough
    __shared__ uint64_t s_up_prefix[SPLIT ? kSmemPrefix + 1 : 1];
    __shared__ uint64_t s_apre[2 * kPThreads];  // active elements' prefix sums (phases B and C)
    __shared__ uint64_t s_wsum[kPThreads / 32];
    const bool compact = p.n < 2 * kPThreads;
    const bool pre_smem = p.n <= kSmemPrefix;
    if (pre_smem)
        for (int k = threadIdx.x; k <= p.n; k += blockDim.x) {
            s_prefix[k] = p.prefix[k];
            if (SPLIT) s_up_prefix[k] = p.up_prefix[k];
        }
    __syncthreads();
    const uint64_t *prefix = pre_smem ? s_prefix : p.prefix;
    const uint64_t *up_prefix = SPLIT ? (pre_smem ? s_up_prefix : p.up_prefix) : nullptr;
    using T = typename std::conditional<FX, int64_t, double>::type;
    const unsigned G = gridDim.x;
    const uint64_t n_items = p.prefix[p.n];
    T *V = static_cast<T *>(p.V);
    // this CTA's slice of the batch vector (phases B and C)
    const uint64_t per = ((p.total + G - 1) / G + 3) & ~3ull;
    const uint64_t c0 = min(p.total, (uint64_t)blockIdx.x * per), c1 = min(p.total, c0 + per);
    int j = *p.jdev;
    const int j_end = min(j + p.chunk, p.maxit);
    unsigned tag = 0;
    if ((int)blockIdx.x == p.withhold) return;  // self-test: this CTA never arrives
    for (; j < j_end; ++j) {
        int na = 0;
        for (int k = 0; k < p.n; ++k) na += p.active[k];
        if (na == 0) break;  // every CTA reads the same flags (set before the last barrier)
        const int iv = j % 3, ip = (j + 2) % 3, iw = (j + 1) % 3;
        // ---------------- phase A: H·v + first vector pass ----------------
        typename std::conditional<FX, FxStepEpi, F64StepEpi>::type epi{};
        int cur = -1;
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        // the warp's partial <w, v> of item `it`, then a fresh accumulator (no CTA barrier)
        auto item_done = [&](uint64_t it) {
            if constexpr (FX) {
                I128 v = epi.swv;
                for (int o = 16; o > 0; o >>= 1) {
                    I128 t;
                    t.lo = __shfl_down_sync(0xffffffffu, v.lo, o);
                    t.hi = __shfl_down_sync(0xffffffffu, v.hi, o);
                    i128_add(v, t);
                }
                if (lane == 0) p.item_part[it * (kPThreads / 32) + warp] = v;
                epi.swv = I128();
            } else {
                double v = epi.swv;
                for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
                if (lane == 0) reinterpret_cast<double *>(p.item_part + it * (kPThreads / 32) + warp)[0] = v;
                epi.swv = 0.0;
            }
        };
        // instance k becomes the CTA's current one: descriptor, diagonal table, hook pointers
        auto enter = [&](int k, bool diag) {
            __syncthreads();
            copy_inst(&s_inst, p.inst + k);
            __syncthreads();
            if (diag) hv_fx_load_diag(s_inst.fx, smem);
            cur = k;
            const uint64_t off = s_inst.off;
            epi.w = V + iw * p.stride + off;
            epi.vprev = V + ip * p.stride + off;
            epi.has_prev = j > 0;
            const double bp = j > 0 ? p.beta[(uint64_t)k * p.maxit1 + j - 1] : 0.0;
            if constexpr (FX) {
                const FxCoef c = fx_coef_dev(bp);
                epi.Kb = c.K;
                epi.Gb = c.G;
            } else {
                epi.bprev = bp;
            }
        };
        int k = 0;
        if constexpr (SPLIT) {
            // row pass of every active instance: w = diag + spin-down hops
            for (uint64_t it = blockIdx.x; next_active_item(prefix, p.n, p.active, n_items, G, it, k); it += G) {
                if (k != cur) enter(k, true);
                hv_fx_wb_group<R, NC>(s_inst.fx, V + iv * p.stride + s_inst.off, V + iw * p.stride + s_inst.off,
                                      it - prefix[k], smem);
            }
            if (!grid_barrier(p.gs, p.limit_ns, tag++)) return;
            // spin-up pass; its hook adds - beta vprev and accumulates <w, v>
            cur = -1;
            const uint64_t n_up = up_prefix[p.n];
            for (uint64_t it = blockIdx.x; next_active_item(up_prefix, p.n, p.active, n_up, G, it, k); it += G) {
                if (k != cur) enter(k, false);
                uint64_t jb, g;
                up_item_of(s_inst.fx, it - up_prefix[k], p.up_S * kPUpRR, &jb, &g);
                const int64_t *v = V + iv * p.stride + s_inst.off;
                if (s_inst.fx.Dd % 2 == 0)
                    hv_fx_up_item<kPUpRR, NC, true, 2, FxStepEpi>(s_inst.fx, v, epi.w, jb, g, p.up_W, p.up_S, smem, &epi);
                else
                    hv_fx_up_item<kPUpRR, NC, true, 1, FxStepEpi>(s_inst.fx, v, epi.w, jb, g, p.up_W, p.up_S, smem, &epi);
                item_done(it);
            }
        } else {
            for (uint64_t it = blockIdx.x; next_active_item(prefix, p.n, p.active, n_items, G, it, k); it += G) {
                if (k != cur) enter(k, FX);
                const uint64_t g = it - prefix[k];
                const T *v = V + iv * p.stride + s_inst.off;
                if constexpr (FX)
                    hv_fx_group<R, NC, true, true, FxStepEpi>(s_inst.fx, v, nullptr, g, smem, &epi);
                else
                    hv_group<R, double, true, true, F64StepEpi>(s_inst.f64, v, nullptr, g, smem, &epi);
                item_done(it);
            }
        }
        if (!grid_barrier(p.gs, p.limit_ns, tag++)) return;
        // items whose warp partials hold <w, v>: the fused pass's, or the spin-up pass's in the split form
        const uint64_t *epre = SPLIT ? up_prefix : prefix;
        // ---------------- slices of phases B and C ----------------
        // Batches of fewer than 2 kPThreads instances split the elements of the instances active
        // at this step evenly over the CTAs (s_apre: their exclusive prefix sums, taken from the
        // flags as they stand after the last step's checks and kept for phase C, whose owners
        // change the flags); larger batches split the whole batch vector.
        if (compact) {
            const int t = threadIdx.x, k0 = 2 * t, k1 = 2 * t + 1;
            const uint64_t v0 = (k0 < p.n && p.active[k0]) ? p.inst[k0].D : 0;
            const uint64_t v1 = (k1 < p.n && p.active[k1]) ? p.inst[k1].D : 0;
            const uint64_t s = v0 + v1;
            uint64_t incl = s;
            for (int o = 1; o < 32; o <<= 1) {
                const uint64_t y = __shfl_up_sync(0xffffffffu, incl, o);
                if ((t & 31) >= o) incl += y;
            }
            if ((t & 31) == 31) s_wsum[t >> 5] = incl;
            __syncthreads();
            uint64_t base = 0;
            for (int w = 0; w < (t >> 5); ++w) base += s_wsum[w];
            const uint64_t excl = base + incl - s;
            if (k0 <= p.n) s_apre[k0] = excl;
            if (k1 <= p.n) s_apre[k1] = excl + v0;
            __syncthreads();
        }
        // fn(k, e0, e1, owner) for each instance k this CTA updates: elements [e0, e1) of the
        // batch vector; owner: the CTA holds the instance's first element of the split
        auto for_slices = [&](auto &&fn) {
            if (compact) {
                const uint64_t A = s_apre[p.n];
                const uint64_t pa = ((A + G - 1) / G + 3) & ~3ull;
                const uint64_t a0 = min(A, (uint64_t)blockIdx.x * pa), a1 = min(A, a0 + pa);
                if (a0 >= a1) return;
                int lo = 0, hi = p.n - 1;  // first k with s_apre[k + 1] > a0
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (s_apre[mid + 1] > a0) hi = mid; else lo = mid + 1;
                }
                for (int k = lo; k < p.n && s_apre[k] < a1; ++k) {
                    if (s_apre[k + 1] == s_apre[k]) continue;  // inactive at this step
                    const uint64_t off = p.inst[k].off;
                    fn(k, off + (max(a0, s_apre[k]) - s_apre[k]), off + (min(a1, s_apre[k + 1]) - s_apre[k]),
                       s_apre[k] >= a0);
                }
            } else if (c0 < c1) {
                for (int k = inst_at(p.inst, p.n, c0); k < p.n && p.inst[k].off < c1; ++k) {
                    if (!p.active[k]) continue;
                    const Inst &in = p.inst[k];
                    fn(k, max(c0, in.off), min(c1, in.off + in.D), in.off >= c0);
                }
            }
        };
        // ---------------- phase B: alpha = <w, v>; w -= alpha v; partial ||w||^2 ----------------
        for (int k = threadIdx.x; k < p.n; k += blockDim.x) p.part[((uint64_t)k * G + blockIdx.x) * 3 + 1] = I128();
        for_slices([&](int k, uint64_t e0, uint64_t e1, bool owner) {
            const int F = p.inst[k].F;
            const uint64_t q0 = epre[k] * (kPThreads / 32), q1 = epre[k + 1] * (kPThreads / 32);
            if constexpr (FX) {
                I128 sa;
                for (uint64_t q = q0 + threadIdx.x; q < q1; q += blockDim.x) i128_add(sa, p.item_part[q]);
                sa = block_sum128(sa);
                if (threadIdx.x == 0) s_ab[0] = pdx::dd_value(pdx::dd_of_i128(sa, -2 * F));
            } else {
                double sa = 0.0;
                for (uint64_t q = q0 + threadIdx.x; q < q1; q += blockDim.x)
                    sa += reinterpret_cast<const double *>(p.item_part + q)[0];
                sa = block_sum_d(sa);
                if (threadIdx.x == 0) s_ab[0] = sa;
            }
            __syncthreads();
            const double al = s_ab[0];
            if (owner && threadIdx.x == 0) p.alpha[(uint64_t)k * p.maxit1 + j] = al;
            T *w = V + iw * p.stride;
            const T *v = V + iv * p.stride;
            if constexpr (FX) {
                const FxCoef ca = fx_coef_dev(al);
                I128 acc;
                slice_update<int64_t>(e0, e1, w, v, [&](int64_t wv, int64_t vv) {
                    const int64_t wi = wv - fx_mul(vv, ca.K, ca.G);
                    i128_add_prod(acc, wi, wi);
                    return wi;
                });
                acc = block_sum128(acc);
                if (threadIdx.x == 0) p.part[((uint64_t)k * G + blockIdx.x) * 3 + 1] = acc;
            } else {
                double acc = 0.0;
                slice_update<double>(e0, e1, w, v, [&](double wv, double vv) {
                    const double wi = wv - al * vv;
                    acc = fma(wi, wi, acc);
                    return wi;
                });
                acc = block_sum_d(acc);
                if (threadIdx.x == 0) reinterpret_cast<double *>(p.part + ((uint64_t)k * G + blockIdx.x) * 3 + 1)[0] = acc;
            }
            __syncthreads();
        });
        if (!grid_barrier(p.gs, p.limit_ns, tag++)) return;
        // ---------------- phase C: alpha, beta; w = (w - alpha v) / beta; checks ----------------
        const bool check = (j + 1) % p.check_every == 0;
        for_slices([&](int k, uint64_t e0, uint64_t e1, bool owner) {
            const Inst &in = p.inst[k];
            if constexpr (FX) {
                I128 sb;
                for (unsigned b = threadIdx.x; b < G; b += blockDim.x) i128_add(sb, p.part[((uint64_t)k * G + b) * 3 + 1]);
                sb = block_sum128(sb);
                if (threadIdx.x == 0) {
                    const double b2 = pdx::dd_value(pdx::dd_of_i128(sb, -2 * in.F));
                    s_ab[1] = b2 > 0.0 ? sqrt(b2) : 0.0;
                }
            } else {
                double sb = 0.0;
                for (unsigned b = threadIdx.x; b < G; b += blockDim.x)
                    sb += reinterpret_cast<const double *>(p.part + ((uint64_t)k * G + b) * 3)[2];
                sb = block_sum_d(sb);
                if (threadIdx.x == 0) {
                    s_ab[1] = sqrt(sb);
                }
            }
            __syncthreads();
            const double be = s_ab[1];
            if (owner && threadIdx.x == 0) p.beta[(uint64_t)k * p.maxit1 + j] = be;  // alpha: phase B
            T *w = V + iw * p.stride;
            if constexpr (FX) {
                const FxCoef cf = fx_coef_dev(be != 0.0 ? 1.0 / be : 0.0);
                slice_update<int64_t>(e0, e1, w, nullptr, [&](int64_t wv, int64_t) { return fx_mul(wv, cf.K, cf.G); });
            } else {
                const double f = be != 0.0 ? 1.0 / be : 0.0;
                slice_update<double>(e0, e1, w, nullptr, [&](double wv, double) { return wv * f; });
            }
            const bool last = j + 1 >= p.maxit;
            if (owner && (check || be == 0.0 || (uint64_t)(j + 1) >= in.D || last)) {
                __threadfence_block();
                __syncthreads();
                if (threadIdx.x < 32) {
                    double th = 0.0, sl = 0.0;
                    const int nn = j + 1;
                    const double *ga = p.alpha + (uint64_t)k * p.maxit1, *gb = p.beta + (uint64_t)k * p.maxit1;
                    // the coefficients and the work arrays: shared memory (free during this phase) up to
                    // kTriSmem steps, so every dependent access of the passes stays on chip; else global
                    const bool on_chip = nn <= kTriSmem;
                    double *sa = reinterpret_cast<double *>(smem);
                    double *sb = on_chip ? sa + kTriSmem : nullptr;
                    double *w0 = on_chip ? sa + 2 * kTriSmem : p.tri_ws + (uint64_t)k * 3 * p.maxit1;
                    double *sb2 = w0, *sdp = w0 + (on_chip ? kTriSmem : p.maxit1), *sdm = sdp + (on_chip ? kTriSmem : p.maxit1);
                    for (int i = threadIdx.x; i < nn; i += 32) {
                        if (on_chip) {
                            sa[i] = ga[i];
                            sb[i] = gb[i];
                        }
                        sb2[i] = gb[i] * gb[i];
                    }
                    __syncwarp();
                    if (on_chip)
                        tri_lowest_warp(sa, sb2, sb, nn, sdp, sdm, &th, &sl);
                    else
                        tri_lowest_warp(ga, sb2, gb, nn, sdp, sdm, &th, &sl);
                    if (threadIdx.x == 0) {
                        const double r = be * fabs(sl);
                        p.theta[k] = th;
                        p.res[k] = r;
                        p.iters[k] = nn;
                        const bool done = (p.tol > 0 && r <= p.tol * fmax(1.0, fabs(th))) || be == 0.0 ||
                                          (uint64_t)nn >= in.D;
                        if (done) {
                            p.conv[k] = 1;
                            p.active[k] = 0;
                        }
                    }
                }
            }
            __syncthreads();
        });
        if (!grid_barrier(p.gs, p.limit_ns, tag++)) return;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        int na = 0;
        for (int k = 0; k < p.n; ++k) na += p.active[k];
        *p.jdev = j;
        *p.n_active = na;
    }
}

uint64_t align256(uint64_t x) { return (x + 255) & ~255ull; }

}  // namespace

struct hb_batch {
    int n = 0;
    int device = 0, sm_count = 0;
    std::vector<hb_handle> h;
    std::vector<uint64_t> off, items;  // items: prefix sums of row groups (for the configured R)
    uint64_t total = 0;
    Inst *d_inst = nullptr;
    uint64_t *d_prefix = nullptr;
    int *d_all_active = nullptr;
    int max_classes = 1;
    int rows = 2, threads = 256;  // batched H·v launch configuration
    hb_dtype desc_dtype = HB_F64;
    // split form (fixed point): row pass on each instance's warp-blocked table, then the
    // column-blocked spin-up pass; items of the spin-up pass: prefix over instances
    int split = 0;
    bool split_ok = false;  // every instance has a warp-blocked table and D < 2^32
    int up_W = 128, up_S = 2, up_RR = 2, up_threads = 256;
    uint64_t *d_up_prefix = nullptr;
    std::vector<uint64_t> up_items;
};

namespace {

hb_status build_desc(hb_batch *b, int R) {
    std::vector<Inst> host(b->n);
    std::vector<uint64_t> prefix(b->n + 1, 0);
    for (int k = 0; k < b->n; ++k) {
        hb_handle h = b->h[k];
        Inst &I = host[k];
        I.off = b->off[k];
        I.D = h->D;
        I.F = h->fx_frac;
        HvArgs<double> &a = I.f64;
        a.Du = h->D_up;
        a.Dd = h->D_dn;
        a.U = h->U;
        a.str_up = h->up.str;
        a.str_dn = h->dn.str;
        a.cnt_up = h->up.count;
        a.cnt_dn = h->dn.count;
        a.tgt_up = h->up.target;
        a.tgt_dn = h->dn.target;
        a.val_up = h->up.val;
        a.val_dn = h->dn.val;
        a.order = h->d_row_order;
        a.zmax_up = h->up.zmax;
        HvArgs<float> &f = I.f32;
        f.Du = a.Du;
        f.Dd = a.Dd;
        f.U = (float)h->U;
        f.str_up = a.str_up;
        f.str_dn = a.str_dn;
        f.cnt_up = a.cnt_up;
        f.cnt_dn = a.cnt_dn;
        f.tgt_up = a.tgt_up;
        f.tgt_dn = a.tgt_dn;
        f.val_up = h->up.valf;
        f.val_dn = h->dn.valf;
        f.order = a.order;
        f.zmax_up = a.zmax_up;
        FxArgs &x = I.fx;
        x.Du = a.Du;
        x.Dd = a.Dd;
        x.str_up = a.str_up;
        x.str_dn = a.str_dn;
        x.seg_up = h->up.seg;
        x.seg_dn = h->dn.seg;
        x.ft_up = h->up.ftarget;
        x.ft_dn = h->dn.ftarget;
        x.order = a.order;
        x.zmax_up = a.zmax_up;
        if (h->fx_ok) {
            FxCoef diag[PD_MAXL + 1], cls[PD_FX_MAXC];
            pd_fx_coefs(h, diag, cls);
            for (int q = 0; q <= PD_MAXL; ++q) {
                x.Kd[q] = diag[q].K;
                x.Gd[q] = diag[q].G;
            }
            for (int c = 0; c < PD_FX_MAXC; ++c) {
                x.Kc[c] = cls[c].K;
                x.Gc[c] = cls[c].G;
            }
        }
        if (h->dn.wb_ok) {
            x.wb_perm = h->dn.wb_perm;
            x.wb_str = h->dn.wb_str;
            x.wb_base = h->dn.wb_base;
            x.wb_ent = h->dn.wb_ent;
            x.wb_caps = h->dn.wb_caps;
            x.wb_nblk = h->dn.wb_nblk;
        }
        prefix[k + 1] = prefix[k] + (h->D_up + R - 1) / R;
    }
    // spin-up pass items: (column block, row group) of every instance, column-block-major
    b->split_ok = true;
    std::vector<uint64_t> up(b->n + 1, 0);
    const uint64_t RA = (uint64_t)b->up_S * b->up_RR;
    for (int k = 0; k < b->n; ++k) {
        hb_handle h = b->h[k];
        b->split_ok = b->split_ok && h->fx_ok && h->dn.wb_ok && h->D < (1ull << 32);
        const uint64_t V = h->D_dn % 2 == 0 ? 2 : 1;
        const uint64_t cols = (uint64_t)b->up_W * V;
        up[k + 1] = up[k] + (h->D_dn + cols - 1) / cols * ((h->D_up + RA - 1) / RA);
    }
    PD_CUDA(cudaMemcpy(b->d_inst, host.data(), sizeof(Inst) * b->n, cudaMemcpyHostToDevice));
    PD_CUDA(cudaMemcpy(b->d_prefix, prefix.data(), sizeof(uint64_t) * (b->n + 1), cudaMemcpyHostToDevice));
    PD_CUDA(cudaMemcpy(b->d_up_prefix, up.data(), sizeof(uint64_t) * (b->n + 1), cudaMemcpyHostToDevice));
    b->items = prefix;
    b->up_items = up;
    return HB_OK;
}

size_t batch_smem(const hb_batch *b, int R, hb_dtype dt) {
    size_t m = 0;
    for (hb_handle h : b->h) {
        const size_t s = dt == HB_FX64 ? hv_fx_smem_bytes(R, h->up.zmax, h->D_dn)
                                       : hv_smem_bytes(R, h->up.zmax, dt == HB_F32 ? 4 : 8, h->D_dn, true);
        m = std::max(m, s);
    }
    return m;
}

template <int R, int MODE, int NC>
hb_status launch_batch_hv(hb_batch *b, const void *x, void *y, const int *active, cudaStream_t st, size_t smem) {
    auto kern = k_batch_hv<R, MODE, NC>;
    PD_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    PD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, b->threads, smem));
    if (per_sm < 1) return HB_ERR_NO_MEMORY;
    const uint64_t grid = std::min<uint64_t>(b->items[b->n], (uint64_t)per_sm * b->sm_count);
    kern<<<(unsigned)std::max<uint64_t>(grid, 1), b->threads, smem, st>>>(b->d_inst, b->d_prefix, b->n, active, x, y);
    PD_CUDA(cudaGetLastError());
    return HB_OK;
}

template <int R>
hb_status batch_hv_r(hb_batch *b, hb_dtype dt, const void *x, void *y, const int *active, cudaStream_t st) {
    const size_t smem = batch_smem(b, R, dt);
    if (dt == HB_F64) return launch_batch_hv<R, 0, 1>(b, x, y, active, st, smem);
    if (dt == HB_F32) return launch_batch_hv<R, 1, 1>(b, x, y, active, st, smem);
    switch (b->max_classes) {
        case 1: return launch_batch_hv<R, 2, 1>(b, x, y, active, st, smem);
        case 2: return launch_batch_hv<R, 2, 2>(b, x, y, active, st, smem);
        case 3: return launch_batch_hv<R, 2, 3>(b, x, y, active, st, smem);
        default: return launch_batch_hv<R, 2, 4>(b, x, y, active, st, smem);
    }
}

size_t batch_row_smem(const hb_batch *b, int R) {
    size_t m = 0;
    for (hb_handle h : b->h) m = std::max(m, hv_fx_wb_smem_bytes(R, h->D_dn));
    return m;
}
size_t batch_up_smem(const hb_batch *b) {
    size_t m = 0;
    for (hb_handle h : b->h) m = std::max(m, hv_fx_up_smem_bytes<true>(b->up_S * b->up_RR, h->up.zmax));
    return m;
}

template <int R, int NC>
hb_status launch_batch_row(hb_batch *b, const int64_t *x, int64_t *y, const int *active, cudaStream_t st) {
    auto kern = k_batch_row<R, NC>;
    const size_t smem = batch_row_smem(b, R);
    PD_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    PD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, b->threads, smem));
    if (per_sm < 1) return HB_ERR_NO_MEMORY;
    const uint64_t grid = std::min<uint64_t>(b->items[b->n], (uint64_t)per_sm * b->sm_count);
    kern<<<(unsigned)std::max<uint64_t>(grid, 1), b->threads, smem, st>>>(b->d_inst, b->d_prefix, b->n, active, x, y);
    PD_CUDA(cudaGetLastError());
    return HB_OK;
}

template <int RR, int NC>
hb_status launch_batch_up(hb_batch *b, const int64_t *x, int64_t *y, const int *active, cudaStream_t st) {
    auto kern = k_batch_up<RR, NC>;
    const size_t smem = batch_up_smem(b);
    const int threads = b->up_W * b->up_S;
    PD_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    PD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem));
    if (per_sm < 1) return HB_ERR_NO_MEMORY;
    const uint64_t grid = std::min<uint64_t>(b->up_items[b->n], (uint64_t)per_sm * b->sm_count);
    kern<<<(unsigned)std::max<uint64_t>(grid, 1), threads, smem, st>>>(b->d_inst, b->d_up_prefix, b->n, active, x, y,
                                                                       b->up_W, b->up_S);
    PD_CUDA(cudaGetLastError());
    return HB_OK;
}

template <int NC>
hb_status batch_hv_split_nc(hb_batch *b, const int64_t *x, int64_t *y, const int *active, cudaStream_t st) {
    hb_status s = b->rows == 1 ? launch_batch_row<1, NC>(b, x, y, active, st) : launch_batch_row<2, NC>(b, x, y, active, st);
    if (s != HB_OK) return s;
    if (b->up_RR == 4) return launch_batch_up<4, NC>(b, x, y, active, st);
    if (b->up_RR == 2) return launch_batch_up<2, NC>(b, x, y, active, st);
    return launch_batch_up<1, NC>(b, x, y, active, st);
}

hb_status batch_hv_split(hb_batch *b, const void *x, void *y, const int *active, cudaStream_t st) {
    const int64_t *xi = static_cast<const int64_t *>(x);
    int64_t *yi = static_cast<int64_t *>(y);
    switch (b->max_classes) {
        case 1: return batch_hv_split_nc<1>(b, xi, yi, active, st);
        case 2: return batch_hv_split_nc<2>(b, xi, yi, active, st);
        case 3: return batch_hv_split_nc<3>(b, xi, yi, active, st);
        default: return batch_hv_split_nc<4>(b, xi, yi, active, st);
    }
}

hb_status batch_hv(hb_batch *b, hb_dtype dt, const void *x, void *y, const int *active, cudaStream_t st) {
    if (dt == HB_FX64 && b->split && b->split_ok) return batch_hv_split(b, x, y, active, st);
    if (b->rows == 4) return batch_hv_r<4>(b, dt, x, y, active, st);
    if (b->rows == 1) return batch_hv_r<1>(b, dt, x, y, active, st);
    return batch_hv_r<2>(b, dt, x, y, active, st);
}

hb_status batch_prepare(hb_batch *b) {
    for (hb_handle h : b->h) {
        hb_status s = pd_build_tables(h);
        if (s != HB_OK) return s;
    }
    return build_desc(b, b->rows);
}

}  // namespace

extern "C" {

hb_status hubbard_batch_create(int n, const hb_handle *handles, hb_batch_handle *out) {
    if (!out || n < 1 || !handles) return HB_ERR_INVALID_ARG;
    *out = nullptr;
    hb_batch *b = new (std::nothrow) hb_batch();
    if (!b) return HB_ERR_NO_MEMORY;
    b->n = n;
    b->h.assign(handles, handles + n);
    b->off.assign(n + 1, 0);
    for (int k = 0; k < n; ++k) {
        if (!handles[k] || handles[k]->device != handles[0]->device) {
            delete b;
            return HB_ERR_INVALID_ARG;
        }
        b->off[k + 1] = b->off[k] + ((handles[k]->D + 63) / 64) * 64;  // 512-byte aligned instance vectors
        b->max_classes = std::max(b->max_classes, handles[k]->n_classes);
    }
    b->total = b->off[n];
    b->device = handles[0]->device;
    b->sm_count = handles[0]->sm_count;
    if (cudaMalloc(&b->d_inst, sizeof(Inst) * n) != cudaSuccess ||
        cudaMalloc(&b->d_prefix, sizeof(uint64_t) * (n + 1)) != cudaSuccess ||
        cudaMalloc(&b->d_all_active, sizeof(int) * n) != cudaSuccess ||
        cudaMalloc(&b->d_up_prefix, sizeof(uint64_t) * (n + 1)) != cudaSuccess) {
        hubbard_batch_destroy(b);
        return HB_ERR_NO_MEMORY;
    }
    std::vector<int> ones(n, 1);
    cudaMemcpy(b->d_all_active, ones.data(), sizeof(int) * n, cudaMemcpyHostToDevice);
    *out = b;
    return HB_OK;
}

hb_status hubbard_batch_destroy(hb_batch_handle b) {
    if (!b) return HB_ERR_INVALID_ARG;
    cudaFree(b->d_inst);
    cudaFree(b->d_prefix);
    cudaFree(b->d_all_active);
    cudaFree(b->d_up_prefix);
    delete b;
    return HB_OK;
}

hb_status hubbard_batch_layout(hb_batch_handle b, uint64_t *offsets) {
    if (!b || !offsets) return HB_ERR_INVALID_ARG;
    std::copy(b->off.begin(), b->off.end(), offsets);
    return HB_OK;
}

hb_status hubbard_batch_apply(hb_batch_handle b, hb_dtype dt, const void *x, void *y, void *stream) {
    if (!b || !x || !y || (dt != HB_F64 && dt != HB_F32 && dt != HB_FX64)) return HB_ERR_INVALID_ARG;
    if (dt == HB_FX64)
        for (hb_handle h : b->h)
            if (!h->fx_ok) return HB_ERR_INVALID_ARG;
    hb_status s = batch_prepare(b);
    if (s != HB_OK) return s;
    return batch_hv(b, dt, x, y, nullptr, reinterpret_cast<cudaStream_t>(stream));
}

hb_status hubbard_batch_get_config(hb_batch_handle b, hb_hv_config *cfg) {
    if (!b || !cfg) return HB_ERR_INVALID_ARG;
    cfg->rows_per_cta = b->rows;
    cfg->threads_per_cta = b->threads;
    cfg->visit_order = 1;
    cfg->ms = 0.f;
    cfg->split = b->split;
    cfg->up_block = b->split ? b->up_W : 0;
    cfg->up_threads = b->split ? b->up_W * b->up_S : 0;
    cfg->up_rows = b->split ? b->up_RR : 0;
    return HB_OK;
}

hb_status hubbard_batch_set_config(hb_batch_handle b, const hb_hv_config *c) {
    if (!b || !c) return HB_ERR_INVALID_ARG;
    const int R = c->rows_per_cta ? c->rows_per_cta : 2, T = c->threads_per_cta ? c->threads_per_cta : 256;
    if ((R != 1 && R != 2 && R != 4) || T < 32 || T > 512 || T % 32 || (c->split != 0 && c->split != 1))
        return HB_ERR_INVALID_ARG;
    int W = b->up_W, S = b->up_S, RR = b->up_RR;
    if (c->split) {
        W = c->up_block ? c->up_block : 128;
        const int UT = c->up_threads ? c->up_threads : 256;
        RR = c->up_rows ? c->up_rows : 2;
        if (W < 32 || W % 32 || UT % W || UT > 512 || (RR != 1 && RR != 2 && RR != 4) || R == 4)
            return HB_ERR_INVALID_ARG;
        S = UT / W;
    }
    hb_status s = batch_prepare(b);  // builds the tables, so that split_ok is known
    if (s != HB_OK) return s;
    if (c->split && !b->split_ok) return HB_ERR_INVALID_ARG;
    b->rows = R, b->threads = T, b->split = c->split, b->up_W = W, b->up_S = S, b->up_RR = RR;
    return batch_prepare(b);
}

hb_status hubbard_batch_autotune(hb_batch_handle b, hb_dtype dt, const void *x, void *y, int32_t reps,
                                 hb_hv_config *best, void *stream) {
    if (!b || !x || !y || reps < 1) return HB_ERR_INVALID_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    cudaEvent_t e0, e1;
    PD_CUDA(cudaEventCreate(&e0));
    PD_CUDA(cudaEventCreate(&e1));
    // average time of reps batched applications under the batch's current configuration
    auto time_cfg = [&](float *ms) -> hb_status {
        hb_status s = batch_prepare(b);
        if (s != HB_OK || (s = batch_hv(b, dt, x, y, nullptr, st)) != HB_OK) return s;
        cudaEventRecord(e0, st);
        for (int k = 0; k < reps && s == HB_OK; ++k) s = batch_hv(b, dt, x, y, nullptr, st);
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        float t = 0.f;
        cudaEventElapsedTime(&t, e0, e1);
        *ms = t / reps;
        return s;
    };
    struct Cfg {
        int split, R, T, W, S, RR;
    };
    Cfg bestc = {0, b->rows, b->threads, b->up_W, b->up_S, b->up_RR};
    float best_ms = 3.4e38f;
    hb_status s = HB_OK;
    auto apply = [&](const Cfg &c) {
        b->split = c.split, b->rows = c.R, b->threads = c.T, b->up_W = c.W, b->up_S = c.S, b->up_RR = c.RR;
    };
    auto consider = [&](const Cfg &c) {
        if (s != HB_OK) return;
        apply(c);
        float ms = 0.f;
        s = time_cfg(&ms);
        if (s == HB_OK && ms < best_ms) best_ms = ms, bestc = c;
    };
    // one kernel over all terms
    for (int R : {1, 2, 4})
        for (int T : {128, 256, 512}) consider({0, R, T, b->up_W, b->up_S, b->up_RR});
    // split form (fixed point, every instance with a warp-blocked table): the row pass first, under
    // a default spin-up shape, then the spin-up shape under the best row pass
    apply(bestc);
    if (s == HB_OK && dt == HB_FX64 && batch_prepare(b) == HB_OK && b->split_ok) {
        Cfg row_best = {1, 2, 256, 128, 2, 2};
        float row_ms = 3.4e38f;
        for (int R : {1, 2})
            for (int T : {256, 512}) {
                if (s != HB_OK) break;
                const Cfg c = {1, R, T, 128, 2, 2};
                apply(c);
                float ms = 0.f;
                s = time_cfg(&ms);
                if (s == HB_OK && ms < row_ms) row_ms = ms, row_best = c;
                if (s == HB_OK && ms < best_ms) best_ms = ms, bestc = c;
            }
        const int shapes[][3] = {{32, 8, 2}, {64, 4, 2}, {64, 8, 1}, {128, 4, 1}, {128, 2, 4}, {256, 2, 2}, {512, 1, 2}};
        for (const auto &sh : shapes) consider({1, row_best.R, row_best.T, sh[0], sh[1], sh[2]});
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    apply(bestc);
    hb_status s2 = batch_prepare(b);
    if (s != HB_OK) return s;
    if (s2 != HB_OK) return s2;
    if (best) {
        best->rows_per_cta = bestc.R;
        best->threads_per_cta = bestc.T;
        best->visit_order = 1;
        best->ms = best_ms;
        best->split = bestc.split;
        best->up_block = bestc.split ? bestc.W : 0;
        best->up_threads = bestc.split ? bestc.W * bestc.S : 0;
        best->up_rows = bestc.split ? bestc.RR : 0;
    }
    return HB_OK;
}

}  // extern "C"

namespace {

// ---------------- batched Lanczos (host) ----------------
struct BatchWs {
    uint64_t vec, part_start, part, item, ab, tri, dbl, ints, sync, total;
    int nb, gmax;
};

// items of the pass that carries the first reduction, at most: rows of every instance (one-kernel
// form, one row per item) or the spin-up items of the persistent split shape (128 columns per block
// at one column per thread, kPThreads / 128 row slots of kPUpRR rows per item)
uint64_t max_epi_items(const hb_batch *b) {
    constexpr uint64_t rows_per_item = (kPThreads / 128) * kPUpRR;
    uint64_t rows = 0, up = 0;
    for (hb_handle h : b->h) {
        rows += h->D_up;
        up += (h->D_dn + 127) / 128 * ((h->D_up + rows_per_item - 1) / rows_per_item);
    }
    return std::max(rows, up);
}

static BatchWs batch_layout_ws(hb_batch_handle b, const hb_lanczos_opts *o) {
    BatchWs L;
    L.nb = std::max(1, std::min(b->sm_count * 2, (int)((b->off[1] + 1023) / 1024)));
    for (int k = 0; k < b->n; ++k) L.nb = std::max(L.nb, std::min(b->sm_count * 2, (int)((b->h[k]->D + 4095) / 4096)));
    L.gmax = b->sm_count * (2048 / kPThreads);  // co-resident CTAs of the persistent kernel, at most
    const uint64_t n = (uint64_t)b->n, m1 = (uint64_t)o->maxit + 1;
    L.vec = 0;
    L.part_start = L.vec + 3 * align256(b->total * 8);
    L.part = L.part_start + align256(n * L.nb * 16);
    L.item = L.part + align256(n * L.gmax * 3 * 16);
    L.ab = L.item + align256(max_epi_items(b) * (kPThreads / 32) * 16);
    L.tri = L.ab + align256(n * m1 * 8 * 2);
    L.dbl = L.tri + align256(n * 3 * m1 * 8);
    L.ints = L.dbl + align256(n * 2 * 8);
    L.sync = L.ints + align256((3 * n + 2) * 4);
    L.total = L.sync + 256;
    return L;
}

template <int R, int NC, bool FX, bool SPLIT>
hb_status pick_persistent(hb_batch *b, size_t smem, void **kern, int *per_sm) {
    auto k = k_batch_lanczos<R, NC, FX, SPLIT>;
    PD_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    PD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k, kPThreads, smem));
    *kern = reinterpret_cast<void *>(k);
    return HB_OK;
}

template <int R, bool SPLIT>
hb_status pick_persistent_r(hb_batch *b, bool fx, size_t smem, void **kern, int *per_sm) {
    if (!fx) return pick_persistent<R, 1, false, false>(b, smem, kern, per_sm);
    switch (b->max_classes) {
        case 1: return pick_persistent<R, 1, true, SPLIT>(b, smem, kern, per_sm);
        case 2: return pick_persistent<R, 2, true, SPLIT>(b, smem, kern, per_sm);
        case 3: return pick_persistent<R, 3, true, SPLIT>(b, smem, kern, per_sm);
        default: return pick_persistent<R, 4, true, SPLIT>(b, smem, kern, per_sm);
    }
}

// One cooperative launch of the persistent kernel (all CTAs co-resident, as its grid barriers need).
hb_status launch_persistent(void *kern, unsigned grid, size_t smem, const PState &p, cudaStream_t st) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kPThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    void *args[] = {const_cast<PState *>(&p)};
    PD_CUDA(cudaLaunchKernelExC(&cfg, kern, args));
    return HB_OK;
}

// The batched solve.  withhold >= 0 runs one step with that CTA leaving before
// its first arrival and the given wait limit (the bounded-wait self-test).
hb_status batch_lanczos(hb_batch *b, const hb_lanczos_opts *o, void *workspace, uint64_t workspace_bytes,
                        double *E0, hb_lanczos_info *info, cudaStream_t user, int withhold,
                        unsigned long long limit_ns) {
    const auto t0 = std::chrono::steady_clock::now();
    if (!b || !o || !workspace || o->maxit < 1 || o->check_every < 1 || o->reorth) return HB_ERR_INVALID_ARG;
    if (o->vec_dtype != HB_F64 && o->vec_dtype != HB_FX64) return HB_ERR_INVALID_ARG;
    const bool FX = o->vec_dtype == HB_FX64;
    if (FX)
        for (hb_handle h : b->h)
            if (!h->fx_ok) return HB_ERR_INVALID_ARG;
    const BatchWs L = batch_layout_ws(b, o);
    if (workspace_bytes < L.total) return HB_ERR_NO_MEMORY;
    int coop = 0;
    PD_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, b->device));
    if (!coop) return HB_ERR_CUDA;
    hb_status st = batch_prepare(b);
    if (st != HB_OK) return st;
    // the batched H·v's tuned form: the split form (fixed point, warp-blocked tables) or one kernel
    const bool split = FX && b->split && b->split_ok;
    const int R = split ? (b->rows == 1 ? 1 : 2) : (b->rows == 1 ? 1 : b->rows == 4 ? 4 : 2);
    // the spin-up shape of the persistent kernel: kPThreads threads, two rows per thread
    const int saved_W = b->up_W, saved_S = b->up_S, saved_RR = b->up_RR;
    if (split) {  // the shape max_epi_items counts with
        b->up_W = 128;
        b->up_S = kPThreads / 128;
        b->up_RR = kPUpRR;
    }
    st = build_desc(b, R);  // items of R rows and the spin-up items of that shape (batch_prepare rebuilds for apply)
    const int up_W = b->up_W, up_S = b->up_S;
    // dynamic shared memory: the H·v phases' needs, or the tridiagonal check's, whichever is larger
    const size_t smem = std::max(kTriSmemBytes, split ? std::max(batch_row_smem(b, R), batch_up_smem(b))
                                                      : batch_smem(b, R, FX ? HB_FX64 : HB_F64));
    b->up_W = saved_W, b->up_S = saved_S, b->up_RR = saved_RR;
    if (st != HB_OK) return st;
    void *kern = nullptr;
    int per_sm = 0;
    if (split)
        st = R == 1 ? pick_persistent_r<1, true>(b, FX, smem, &kern, &per_sm)
                    : pick_persistent_r<2, true>(b, FX, smem, &kern, &per_sm);
    else
        st = R == 1   ? pick_persistent_r<1, false>(b, FX, smem, &kern, &per_sm)
             : R == 4 ? pick_persistent_r<4, false>(b, FX, smem, &kern, &per_sm)
                      : pick_persistent_r<2, false>(b, FX, smem, &kern, &per_sm);
    if (st != HB_OK) return st;
    if (per_sm < 1) return HB_ERR_NO_MEMORY;
    const unsigned grid = (unsigned)std::min(per_sm * b->sm_count, L.gmax);

    char *ws = static_cast<char *>(workspace);
    const int n = b->n, maxit1 = o->maxit + 1;
    PState p;
    p.inst = b->d_inst;
    p.prefix = b->d_prefix;
    p.n = n;
    p.maxit = withhold >= 0 ? 1 : o->maxit;
    p.maxit1 = maxit1;
    p.check_every = o->check_every;
    p.tol = o->tol;
    p.chunk = withhold >= 0 ? 1 : std::min(o->maxit, 64);
    p.stride = align256(b->total * 8) / 8;
    p.total = b->total;
    p.V = ws + L.vec;
    p.part = reinterpret_cast<I128 *>(ws + L.part);
    p.alpha = reinterpret_cast<double *>(ws + L.ab);
    p.beta = p.alpha + (uint64_t)n * maxit1;
    p.tri_ws = reinterpret_cast<double *>(ws + L.tri);
    p.theta = reinterpret_cast<double *>(ws + L.dbl);
    p.res = p.theta + n;
    p.active = reinterpret_cast<int *>(ws + L.ints);
    p.iters = p.active + n;
    p.conv = p.iters + n;
    p.jdev = p.conv + n;
    p.n_active = p.jdev + 1;
    p.gs = reinterpret_cast<GridSync *>(ws + L.sync);
    p.limit_ns = limit_ns;
    p.withhold = withhold;
    p.up_prefix = b->d_up_prefix;
    p.up_W = up_W;
    p.up_S = up_S;
    p.item_part = reinterpret_cast<I128 *>(ws + L.item);

    cudaStream_t cs;
    PD_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaEvent_t ev;
    if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
        cudaStreamDestroy(cs);
        return HB_ERR_CUDA;
    }
    cudaEventRecord(ev, user);
    cudaStreamWaitEvent(cs, ev, 0);  // ordered after the caller's earlier work
    std::vector<int> ones(n, 1);
    cudaMemcpyAsync(p.active, ones.data(), sizeof(int) * n, cudaMemcpyHostToDevice, cs);
    cudaMemsetAsync(p.iters, 0, sizeof(int) * (2 * n + 2), cs);  // iters, conv, jdev, n_active
    cudaMemsetAsync(p.gs, 0, sizeof(GridSync), cs);
    cudaMemsetAsync(p.alpha, 0, sizeof(double) * 2 * (uint64_t)n * maxit1, cs);
    StartState ss{b->d_inst, p.V, reinterpret_cast<I128 *>(ws + L.part_start), L.nb};
    const dim3 gv(L.nb, n);
    if (FX) {
        k_b_fill<true><<<gv, kThreads, 0, cs>>>(ss, o->seed);
        k_b_norm_partials<true><<<gv, kThreads, 0, cs>>>(ss);
        k_b_normalise<true><<<n, kFinal, 0, cs>>>(ss);
    } else {
        k_b_fill<false><<<gv, kThreads, 0, cs>>>(ss, o->seed);
        k_b_norm_partials<false><<<gv, kThreads, 0, cs>>>(ss);
        k_b_normalise<false><<<n, kFinal, 0, cs>>>(ss);
    }
    hb_status run = cudaGetLastError() == cudaSuccess ? HB_OK : HB_ERR_CUDA;

    // one chunk of steps = one cooperative launch, captured once into a graph and replayed
    cudaGraphExec_t exec = nullptr;
    if (run == HB_OK && withhold < 0) {
        cudaGraph_t g = nullptr;
        if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) run = HB_ERR_CUDA;
        if (run == HB_OK) {
            const hb_status ls = launch_persistent(kern, grid, smem, p, cs);
            const cudaError_t ce = cudaStreamEndCapture(cs, &g);
            if (ls != HB_OK || ce != cudaSuccess) run = HB_ERR_CUDA;
        }
        if (run == HB_OK && cudaGraphInstantiate(&exec, g, 0) != cudaSuccess) run = HB_ERR_CUDA;
        if (g) cudaGraphDestroy(g);
    }
    struct {
        int j, n_active;
        GridSync gs;
    } hs = {};
    while (run == HB_OK) {
        if (withhold >= 0)
            run = launch_persistent(kern, grid, smem, p, cs);
        else if (cudaGraphLaunch(exec, cs) != cudaSuccess)
            run = HB_ERR_CUDA;
        if (run != HB_OK) break;
        cudaMemcpyAsync(&hs.j, p.jdev, sizeof(int) * 2, cudaMemcpyDeviceToHost, cs);
        cudaMemcpyAsync(&hs.gs, p.gs, sizeof(GridSync), cudaMemcpyDeviceToHost, cs);
        if (cudaStreamSynchronize(cs) != cudaSuccess) {
            run = HB_ERR_CUDA;
            break;
        }
        if (hs.gs.abort) {
            run = HB_ERR_TIMEOUT;
            break;
        }
        if (hs.n_active == 0 || hs.j >= p.maxit) break;
    }
    cudaStreamSynchronize(cs);
    if (exec) cudaGraphExecDestroy(exec);
    std::vector<double> ha((size_t)n * maxit1), hbv((size_t)n * maxit1);
    std::vector<int> iters(n), conv(n);
    if (run == HB_OK) {
        cudaMemcpyAsync(ha.data(), p.alpha, sizeof(double) * n * maxit1, cudaMemcpyDeviceToHost, cs);
        cudaMemcpyAsync(hbv.data(), p.beta, sizeof(double) * n * maxit1, cudaMemcpyDeviceToHost, cs);
        cudaMemcpyAsync(iters.data(), p.iters, sizeof(int) * n, cudaMemcpyDeviceToHost, cs);
        cudaMemcpyAsync(conv.data(), p.conv, sizeof(int) * n, cudaMemcpyDeviceToHost, cs);
        if (cudaStreamSynchronize(cs) != cudaSuccess) run = HB_ERR_CUDA;
    }
    cudaEventRecord(ev, cs);
    cudaStreamWaitEvent(user, ev, 0);
    cudaEventDestroy(ev);
    cudaStreamDestroy(cs);
    if (run != HB_OK) return run;
    // final values on the host from the recorded coefficients (the same solver as every other Lanczos call)
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    bool all = true;
    for (int k = 0; k < n; ++k) {
        const int nn = std::max(1, iters[k]);
        const double *a = ha.data() + (size_t)k * maxit1;
        const double *bb = hbv.data() + (size_t)k * maxit1;
        double th = NAN, sl = 0.0;
        hb_tridiag_lowest(a, bb, nn, &th, &sl);
        if (E0) E0[k] = th;
        all = all && conv[k];
        if (info) {
            info[k].E0 = th;
            info[k].residual = bb[nn - 1] * std::fabs(sl);
            info[k].iterations = nn;
            info[k].iterations_f32 = 0;
            info[k].status = conv[k] || o->tol <= 0 ? HB_OK : HB_ERR_NOT_CONVERGED;
            info[k].converged = conv[k];
            info[k].seconds = secs;
        }
    }
    return all || o->tol <= 0 ? HB_OK : HB_ERR_NOT_CONVERGED;
}

}  // namespace

extern "C" {

hb_status lanczos_batch_workspace_bytes(hb_batch_handle b, const hb_lanczos_opts *o, uint64_t *bytes) {
    if (!b || !o || !bytes || o->maxit < 1) return HB_ERR_INVALID_ARG;
    *bytes = batch_layout_ws(b, o).total;
    return HB_OK;
}

hb_status lanczos_batch_ground_state(hb_batch_handle b, const hb_lanczos_opts *o, void *workspace,
                                     uint64_t workspace_bytes, double *E0, hb_lanczos_info *info, void *stream) {
    if (!E0) return HB_ERR_INVALID_ARG;
    return batch_lanczos(b, o, workspace, workspace_bytes, E0, info, reinterpret_cast<cudaStream_t>(stream), -1,
                         5000000000ull);
}

hb_status lanczos_batch_wait_selftest(hb_batch_handle b, const hb_lanczos_opts *o, void *workspace,
                                      uint64_t workspace_bytes, int32_t withhold_cta, uint32_t limit_ms,
                                      void *stream) {
    if (withhold_cta < 0 || limit_ms < 1 || limit_ms > 10000) return HB_ERR_INVALID_ARG;
    return batch_lanczos(b, o, workspace, workspace_bytes, nullptr, nullptr, reinterpret_cast<cudaStream_t>(stream),
                         withhold_cta, (unsigned long long)limit_ms * 1000000ull);
}

}  // extern "C"

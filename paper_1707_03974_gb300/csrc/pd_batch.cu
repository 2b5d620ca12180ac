// Batched Hubbard problems: many clusters / sectors / U values of uneven
// dimension in single launches, and a batched Lanczos whose steps are replayed
// from a captured CUDA graph.
//
// The paper's method per instance is unchanged (Eq. 1 with Paradeisos-ranked
// hop tables, Eq. 3); the batch only concatenates the instances' vectors and
// flattens their row groups into one work list.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <new>
#include <vector>

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
    __shared__ Inst s_inst;
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

// ---------------- batched vector kernels (grid: x = blocks per instance, y = instance) ----------------
struct I128 {
    uint64_t lo = 0;
    int64_t hi = 0;
};
__device__ __forceinline__ void i128_add(I128 &s, const I128 &t) {
    const uint64_t lo = s.lo + t.lo;
    s.hi += t.hi + (lo < t.lo ? 1 : 0);
    s.lo = lo;
}
__device__ __forceinline__ void i128_add_prod(I128 &s, int64_t a, int64_t b, int sh) {
    const int64_t ph = __mul64hi(a, b);
    const uint64_t pl = (uint64_t)a * (uint64_t)b;
    I128 p;
    p.lo = sh == 0 ? pl : ((pl >> sh) | ((uint64_t)ph << (64 - sh)));
    p.hi = sh == 0 ? ph : (ph >> sh);
    i128_add(s, p);
}
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
        if (lane < (int)((blockDim.x + 31) >> 5)) {
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

// Per-step state on the device: the step counter j (slots and alpha/beta
// entries are derived from it), so the same captured graph replays every step.
struct BState {
    const Inst *inst;
    const int *active;
    const int *j;         // current step
    uint64_t stride;      // elements per slot (whole batch vector)
    int n, maxit1, nb;
    void *V;              // 3 slots
    I128 *part;           // [n][nb] (float64 runs use the lo word as a double)
    double *alpha, *beta; // [n][maxit1]
};

template <bool FX>
__global__ void k_b_axpy_dot(BState s) {
    const int k = blockIdx.y;
    if (!s.active[k]) return;
    const int j = *s.j;
    const Inst &in = s.inst[k];
    const uint64_t D = in.D;
    const int iv = j % 3, ip = (j + 2) % 3, iw = (j + 1) % 3;
    const double bprev = j > 0 ? s.beta[k * s.maxit1 + j - 1] : 0.0;
    if (FX) {
        int64_t *V = static_cast<int64_t *>(s.V);
        int64_t *w = V + iw * s.stride + in.off;
        const int64_t *v = V + iv * s.stride + in.off, *vp = V + ip * s.stride + in.off;
        const FxCoef b = fx_coef_dev(bprev);
        I128 acc;
        for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < D; i += (uint64_t)gridDim.x * blockDim.x) {
            int64_t wi = w[i];
            if (j > 0) {
                wi -= fx_mul(vp[i], b.K, b.G);
                w[i] = wi;
            }
            i128_add_prod(acc, wi, v[i], 0);
        }
        const I128 t = block_sum128(acc);
        if (threadIdx.x == 0) s.part[k * s.nb + blockIdx.x] = t;
    } else {
        double *V = static_cast<double *>(s.V);
        double *w = V + iw * s.stride + in.off;
        const double *v = V + iv * s.stride + in.off, *vp = V + ip * s.stride + in.off;
        double acc = 0.0;
        for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < D; i += (uint64_t)gridDim.x * blockDim.x) {
            double wi = w[i];
            if (j > 0) {
                wi = wi - bprev * vp[i];
                w[i] = wi;
            }
            acc = fma(wi, v[i], acc);
        }
        const double t = block_sum_d(acc);
        if (threadIdx.x == 0) reinterpret_cast<double *>(s.part)[2 * (k * s.nb + blockIdx.x)] = t;
    }
}

template <bool FX>
__global__ void k_b_axpy_norm(BState s) {
    const int k = blockIdx.y;
    if (!s.active[k]) return;
    const int j = *s.j;
    const Inst &in = s.inst[k];
    const uint64_t D = in.D;
    const int iv = j % 3, iw = (j + 1) % 3;
    const double al = s.alpha[k * s.maxit1 + j];
    if (FX) {
        int64_t *V = static_cast<int64_t *>(s.V);
        int64_t *w = V + iw * s.stride + in.off;
        const int64_t *v = V + iv * s.stride + in.off;
        const FxCoef a = fx_coef_dev(al);
        I128 acc;
        for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < D; i += (uint64_t)gridDim.x * blockDim.x) {
            const int64_t wi = w[i] - fx_mul(v[i], a.K, a.G);
            w[i] = wi;
            i128_add_prod(acc, wi, wi, 0);
        }
        const I128 t = block_sum128(acc);
        if (threadIdx.x == 0) s.part[k * s.nb + blockIdx.x] = t;
    } else {
        double *V = static_cast<double *>(s.V);
        double *w = V + iw * s.stride + in.off;
        const double *v = V + iv * s.stride + in.off;
        double acc = 0.0;
        for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < D; i += (uint64_t)gridDim.x * blockDim.x) {
            const double wi = w[i] - al * v[i];
            w[i] = wi;
            acc = fma(wi, wi, acc);
        }
        const double t = block_sum_d(acc);
        if (threadIdx.x == 0) reinterpret_cast<double *>(s.part)[2 * (k * s.nb + blockIdx.x)] = t;
    }
}

// which: 0 -> alpha[k][j] = sum, 1 -> beta[k][j] = sqrt(sum)
template <bool FX>
__global__ void k_b_reduce(BState s, int which) {
    const int k = blockIdx.x;
    if (!s.active[k]) return;
    const int j = *s.j;
    double v;
    if (FX) {
        I128 acc;
        for (int i = threadIdx.x; i < s.nb; i += blockDim.x) i128_add(acc, s.part[k * s.nb + i]);
        acc = block_sum128(acc);
        v = ldexp((double)acc.hi * 18446744073709551616.0 + (double)acc.lo, -2 * s.inst[k].F);
    } else {
        double acc = 0.0;
        for (int i = threadIdx.x; i < s.nb; i += blockDim.x) acc += reinterpret_cast<const double *>(s.part)[2 * (k * s.nb + i)];
        v = block_sum_d(acc);
    }
    if (threadIdx.x == 0) {
        if (which == 0) s.alpha[k * s.maxit1 + j] = v;
        else s.beta[k * s.maxit1 + j] = sqrt(v);
    }
}

template <bool FX>
__global__ void k_b_scale(BState s) {
    const int k = blockIdx.y;
    if (!s.active[k]) return;
    const int j = *s.j;
    const Inst &in = s.inst[k];
    const double b = s.beta[k * s.maxit1 + j];
    const double f = b != 0.0 ? 1.0 / b : 0.0;
    const int iw = (j + 1) % 3;
    if (FX) {
        int64_t *w = static_cast<int64_t *>(s.V) + iw * s.stride + in.off;
        const FxCoef c = fx_coef_dev(f);
        for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < in.D; i += (uint64_t)gridDim.x * blockDim.x)
            w[i] = fx_mul(w[i], c.K, c.G);
    } else {
        double *w = static_cast<double *>(s.V) + iw * s.stride + in.off;
        for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < in.D; i += (uint64_t)gridDim.x * blockDim.x)
            w[i] *= f;
    }
}

__global__ void k_b_advance(int *j) { *j += 1; }

// start vectors: instance k uses SplitMix64 seeded with seed + k; then normalised
template <bool FX>
__global__ void k_b_fill(BState s, uint64_t seed) {
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
__global__ void k_b_norm_partials(BState s) {
    const int k = blockIdx.y;
    const Inst &in = s.inst[k];
    if (FX) {
        const int64_t *v = static_cast<const int64_t *>(s.V) + in.off;
        I128 acc;
        for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < in.D; i += (uint64_t)gridDim.x * blockDim.x)
            i128_add_prod(acc, v[i], v[i], 0);
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
__global__ void k_b_normalise(BState s) {
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

uint64_t align256(uint64_t x) { return (x + 255) & ~255ull; }
void tridiag_lowest(const double *a, const double *b, int n, double *theta, double *s_last) {
    hb_tridiag_lowest(a, b, n, theta, s_last);
}

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
        prefix[k + 1] = prefix[k] + (h->D_up + R - 1) / R;
    }
    PD_CUDA(cudaMemcpy(b->d_inst, host.data(), sizeof(Inst) * b->n, cudaMemcpyHostToDevice));
    PD_CUDA(cudaMemcpy(b->d_prefix, prefix.data(), sizeof(uint64_t) * (b->n + 1), cudaMemcpyHostToDevice));
    b->items = prefix;
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

hb_status batch_hv(hb_batch *b, hb_dtype dt, const void *x, void *y, const int *active, cudaStream_t st) {
    if (b->rows == 4 && dt != HB_FX64) return batch_hv_r<4>(b, dt, x, y, active, st);
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
        cudaMalloc(&b->d_all_active, sizeof(int) * n) != cudaSuccess) {
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

hb_status hubbard_batch_autotune(hb_batch_handle b, hb_dtype dt, const void *x, void *y, int32_t reps,
                                 hb_hv_config *best, void *stream) {
    if (!b || !x || !y || reps < 1) return HB_ERR_INVALID_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    cudaEvent_t e0, e1;
    PD_CUDA(cudaEventCreate(&e0));
    PD_CUDA(cudaEventCreate(&e1));
    int bestR = b->rows, bestT = b->threads;
    float best_ms = 3.4e38f;
    hb_status s = HB_OK;
    for (int R : {1, 2, 4}) {
        if (R == 4 && dt == HB_FX64) continue;
        for (int T : {128, 256, 512}) {
            b->rows = R;
            b->threads = T;
            if ((s = batch_prepare(b)) != HB_OK) break;
            if ((s = batch_hv(b, dt, x, y, nullptr, st)) != HB_OK) break;
            cudaEventRecord(e0, st);
            for (int k = 0; k < reps && s == HB_OK; ++k) s = batch_hv(b, dt, x, y, nullptr, st);
            cudaEventRecord(e1, st);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            ms /= reps;
            if (s == HB_OK && ms < best_ms) {
                best_ms = ms;
                bestR = R;
                bestT = T;
            }
        }
        if (s != HB_OK) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->rows = bestR;
    b->threads = bestT;
    hb_status s2 = batch_prepare(b);
    if (s != HB_OK) return s;
    if (s2 != HB_OK) return s2;
    if (best) {
        best->rows_per_cta = bestR;
        best->threads_per_cta = bestT;
        best->visit_order = 1;
        best->ms = best_ms;
        best->split = 0;  // the batched H·v is always one kernel
        best->up_block = best->up_threads = best->up_rows = 0;
    }
    return HB_OK;
}

static void batch_layout_ws(hb_batch_handle b, const hb_lanczos_opts *o, uint64_t *vec, uint64_t *part,
                            uint64_t *ab, uint64_t *misc, uint64_t *total, int *nb) {
    *nb = std::max(1, std::min(b->sm_count * 2, (int)((b->off[1] + 1023) / 1024)));
    for (int k = 0; k < b->n; ++k) *nb = std::max(*nb, std::min(b->sm_count * 2, (int)((b->h[k]->D + 4095) / 4096)));
    *vec = 0;
    const uint64_t vbytes = align256(b->total * 8);
    *part = *vec + 3 * vbytes;
    *ab = *part + align256((uint64_t)b->n * (*nb) * 16);
    *misc = *ab + align256((uint64_t)b->n * (o->maxit + 1) * 8 * 2);
    *total = *misc + align256(sizeof(int) * (b->n + 1));
}

hb_status lanczos_batch_workspace_bytes(hb_batch_handle b, const hb_lanczos_opts *o, uint64_t *bytes) {
    if (!b || !o || !bytes || o->maxit < 1) return HB_ERR_INVALID_ARG;
    uint64_t v, p, a, m;
    int nb;
    batch_layout_ws(b, o, &v, &p, &a, &m, bytes, &nb);
    return HB_OK;
}

// Batched three-term Lanczos (float64 or fixed-point vectors).  One step of
// all active instances is 8 launches that take the step index from device
// memory; `check_every` steps are captured once into a CUDA graph and the
// graph is replayed between host-side convergence checks (per-instance
// tridiagonal solves).  Converged instances are masked out of later steps.
hb_status lanczos_batch_ground_state(hb_batch_handle b, const hb_lanczos_opts *o, void *workspace,
                                     uint64_t workspace_bytes, double *E0, hb_lanczos_info *info, void *stream) {
    const auto t0 = std::chrono::steady_clock::now();
    if (!b || !o || !workspace || !E0 || o->maxit < 1 || o->check_every < 1 || o->reorth) return HB_ERR_INVALID_ARG;
    if (o->vec_dtype != HB_F64 && o->vec_dtype != HB_FX64) return HB_ERR_INVALID_ARG;
    const bool FX = o->vec_dtype == HB_FX64;
    if (FX)
        for (hb_handle h : b->h)
            if (!h->fx_ok) return HB_ERR_INVALID_ARG;
    uint64_t ov, op, oab, om, total;
    int nb;
    batch_layout_ws(b, o, &ov, &op, &oab, &om, &total, &nb);
    if (workspace_bytes < total) return HB_ERR_NO_MEMORY;
    hb_status st = batch_prepare(b);
    if (st != HB_OK) return st;
    char *ws = static_cast<char *>(workspace);
    const int n = b->n, maxit1 = o->maxit + 1;
    BState S;
    S.inst = b->d_inst;
    S.stride = align256(b->total * 8) / 8;
    S.n = n;
    S.maxit1 = maxit1;
    S.nb = nb;
    S.V = ws + ov;
    S.part = reinterpret_cast<I128 *>(ws + op);
    S.alpha = reinterpret_cast<double *>(ws + oab);
    S.beta = S.alpha + (uint64_t)n * maxit1;
    int *d_active = reinterpret_cast<int *>(ws + om);
    int *d_j = d_active + n;
    S.active = d_active;
    S.j = d_j;

    cudaStream_t user = reinterpret_cast<cudaStream_t>(stream);
    cudaStream_t cs;
    PD_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaEvent_t ev;
    PD_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    cudaEventRecord(ev, user);
    cudaStreamWaitEvent(cs, ev, 0);  // ordered after the caller's earlier work
    std::vector<int> act(n, 1);
    cudaMemcpyAsync(d_active, act.data(), sizeof(int) * n, cudaMemcpyHostToDevice, cs);
    cudaMemsetAsync(d_j, 0, sizeof(int), cs);
    const dim3 gv(nb, n);
    // start vectors in slot 0, normalised
    if (FX) {
        k_b_fill<true><<<gv, kThreads, 0, cs>>>(S, o->seed);
        // norms of un-normalised vectors: products shifted as in the single-instance path
        k_b_norm_partials<true><<<gv, kThreads, 0, cs>>>(S);
        k_b_normalise<true><<<n, kFinal, 0, cs>>>(S);
    } else {
        k_b_fill<false><<<gv, kThreads, 0, cs>>>(S, o->seed);
        k_b_norm_partials<false><<<gv, kThreads, 0, cs>>>(S);
        k_b_normalise<false><<<n, kFinal, 0, cs>>>(S);
    }
    PD_CUDA(cudaGetLastError());
    const hb_dtype dt = FX ? HB_FX64 : HB_F64;
    // One graph per slot phase p = j mod 3 (the batched H·v takes its vector pointers as
    // launch arguments, the vector kernels read j from device memory); each graph holds one
    // step, and steps are replayed phase after phase.
    if ((st = batch_hv(b, dt, S.V, static_cast<char *>(S.V) + S.stride * 8, d_active, cs)) != HB_OK) return st;
    cudaGraphExec_t exec[3] = {nullptr, nullptr, nullptr};
    hb_status cap = HB_OK;
    for (int p = 0; p < 3 && cap == HB_OK; ++p) {
        const uint64_t es = 8;
        char *Vb = static_cast<char *>(S.V);
        const void *v = Vb + (uint64_t)(p % 3) * S.stride * es;
        void *w = Vb + (uint64_t)((p + 1) % 3) * S.stride * es;
        cudaGraph_t g;
        if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
            cap = HB_ERR_CUDA;
            break;
        }
        hb_status s1 = batch_hv(b, dt, v, w, d_active, cs);
        if (FX) {
            k_b_axpy_dot<true><<<gv, kThreads, 0, cs>>>(S);
            k_b_reduce<true><<<n, kFinal, 0, cs>>>(S, 0);
            k_b_axpy_norm<true><<<gv, kThreads, 0, cs>>>(S);
            k_b_reduce<true><<<n, kFinal, 0, cs>>>(S, 1);
            k_b_scale<true><<<gv, kThreads, 0, cs>>>(S);
        } else {
            k_b_axpy_dot<false><<<gv, kThreads, 0, cs>>>(S);
            k_b_reduce<false><<<n, kFinal, 0, cs>>>(S, 0);
            k_b_axpy_norm<false><<<gv, kThreads, 0, cs>>>(S);
            k_b_reduce<false><<<n, kFinal, 0, cs>>>(S, 1);
            k_b_scale<false><<<gv, kThreads, 0, cs>>>(S);
        }
        k_b_advance<<<1, 1, 0, cs>>>(d_j);
        cudaError_t ce = cudaStreamEndCapture(cs, &g);
        if (s1 != HB_OK || ce != cudaSuccess) {
            cap = s1 != HB_OK ? s1 : HB_ERR_CUDA;
            break;
        }
        if (cudaGraphInstantiate(&exec[p], g, 0) != cudaSuccess) cap = HB_ERR_CUDA;
        cudaGraphDestroy(g);
    }
    std::vector<double> ha((size_t)n * maxit1), hbv((size_t)n * maxit1);
    std::vector<int> iters(n, 0), conv(n, 0);
    std::vector<double> theta(n, NAN), res(n, INFINITY);
    int j = 0, n_active = n;
    while (cap == HB_OK && j < o->maxit && n_active > 0) {
        const int chunk = std::min(o->check_every, o->maxit - j);
        for (int c = 0; c < chunk; ++c, ++j)
            if (cudaGraphLaunch(exec[j % 3], cs) != cudaSuccess) {
                cap = HB_ERR_CUDA;
                break;
            }
        if (cap != HB_OK) break;
        cudaMemcpyAsync(ha.data(), S.alpha, sizeof(double) * n * maxit1, cudaMemcpyDeviceToHost, cs);
        cudaMemcpyAsync(hbv.data(), S.beta, sizeof(double) * n * maxit1, cudaMemcpyDeviceToHost, cs);
        if (cudaStreamSynchronize(cs) != cudaSuccess) {
            cap = HB_ERR_CUDA;
            break;
        }
        bool changed = false;
        for (int k = 0; k < n; ++k) {
            if (!act[k]) continue;
            const double *a = ha.data() + (size_t)k * maxit1;
            const double *bb = hbv.data() + (size_t)k * maxit1;
            double th, sl;
            tridiag_lowest(a, bb, j, &th, &sl);
            theta[k] = th;
            res[k] = bb[j - 1] * std::fabs(sl);
            iters[k] = j;
            const bool exhausted = bb[j - 1] == 0.0 || (uint64_t)j >= b->h[k]->D;
            if ((o->tol > 0 && res[k] <= o->tol * std::max(1.0, std::fabs(th))) || exhausted) {
                conv[k] = 1;
                act[k] = 0;
                --n_active;
                changed = true;
            }
        }
        if (changed) cudaMemcpyAsync(d_active, act.data(), sizeof(int) * n, cudaMemcpyHostToDevice, cs);
    }
    cudaStreamSynchronize(cs);
    for (auto &e : exec)
        if (e) cudaGraphExecDestroy(e);
    cudaEventRecord(ev, cs);
    cudaStreamWaitEvent(user, ev, 0);
    cudaEventDestroy(ev);
    cudaStreamDestroy(cs);
    if (cap != HB_OK) return cap;
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    bool all = true;
    for (int k = 0; k < n; ++k) {
        E0[k] = theta[k];
        all = all && conv[k];
        if (info) {
            info[k].E0 = theta[k];
            info[k].residual = res[k];
            info[k].iterations = iters[k];
            info[k].iterations_f32 = 0;
            info[k].status = conv[k] || o->tol <= 0 ? HB_OK : HB_ERR_NOT_CONVERGED;
            info[k].converged = conv[k];
            info[k].seconds = secs;
        }
    }
    return all || o->tol <= 0 ? HB_OK : HB_ERR_NOT_CONVERGED;
}

}  // extern "C"

// Matrix-free Hubbard H·v (Eq. 1) on the tensor-product basis.
//
// With x viewed as the row-major D_up x D_dn matrix X of the combined index
// (Sec. III), every spin-up hop changes only the row and every spin-down hop
// only the column (the other species adds no fermion sign), so
//     y[u, d] = U popcount(s_u & s_d) x[u, d]                     (Sec. II B)
//             + sum_{u' in hops(u)} h_up(u, u') x[u', d]
//             + sum_{d' in hops(d)} h_dn(d, d') x[u, d'].
// Hop targets are per-spin indices from the forward map (Eq. 3), computed once
// per spin string when the handle's tables are built.
//
// Kernel shape: a persistent grid walks groups of R rows (in the handle's visiting
// order, reverse Cuthill-McKee over the spin-up hop graph by default).  A CTA
// stages its R rows of x in shared memory (interleaved x_s[d * R + r]) so the
// spin-down gathers hit shared memory; the spin-up terms read whole rows
// x[u', :] from global memory, coalesced across the threads of the CTA.  When
// R rows do not fit in shared memory the down gathers read global memory.
#include <algorithm>

#include "pd_hv_body.cuh"
#include "pd_hv_f32wb.cuh"

namespace {

// part: 0 = the whole H·v as configured, 1 = row pass only (diagonal + spin-down),
// 2 = spin-up pass only (adds into y).  Parts 1 and 2 exist for the autotuner.
enum { kAll = 0, kRowPass = 1, kUpPass = 2 };

template <int R, typename T, bool SMEM, int LB, bool DO_A>
__global__ void __launch_bounds__(LB) k_hv(const HvArgs<T> a, const T *__restrict__ x, T *__restrict__ y) {
    extern __shared__ __align__(16) unsigned char smem[];
    const uint64_t ngroups = (a.Du + R - 1) / R;
    for (uint64_t g = blockIdx.x; g < ngroups; g += gridDim.x) hv_group<R, T, SMEM, DO_A>(a, x, y, g, smem);
}

template <int RR, typename T, bool IDX32, int LB, int V>
__global__ void __launch_bounds__(LB) k_hv_up(const HvArgs<T> a, const T *__restrict__ x, T *__restrict__ y, int W,
                                                uint64_t n_groups, uint64_t n_items) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int S = blockDim.x / W;
    ItemWalk w(n_groups);
    for (uint64_t it = blockIdx.x; it < n_items; it += gridDim.x, w.next())
        hv_up_item<RR, T, IDX32, V>(a, x, y, w.j, w.g, W, S, smem);
}

bool a_small(uint64_t Dd, int threads) { return Dd < (uint64_t)threads; }

template <typename K>
hb_status persistent_launch_dims(hb_handle h, K kern, int threads, size_t smem, uint64_t work, unsigned *grid) {
    PD_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    PD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem));
    if (per_sm < 1) return HB_ERR_NO_MEMORY;
    *grid = (unsigned)std::min<uint64_t>(work, (uint64_t)per_sm * h->sm_count);
    return HB_OK;
}

template <int R, typename T, bool SMEM, int LB, bool DO_A>
hb_status launch_hv_lb(hb_handle h, const HvArgs<T> &a, const T *x, T *y, cudaStream_t st, size_t smem,
                       int threads) {
    auto kern = k_hv<R, T, SMEM, LB, DO_A>;
    unsigned grid = 0;
    hb_status s = persistent_launch_dims(h, kern, threads, smem, (a.Du + R - 1) / R, &grid);
    if (s != HB_OK) return s;
    kern<<<grid, threads, smem, st>>>(a, x, y);
    PD_CUDA(cudaGetLastError());
    return HB_OK;
}

int pick_threads(const HvConfig &c, uint64_t Dd) {
    int threads = c.threads > 0 ? c.threads : 1024;
    if (a_small(Dd, threads)) threads = (int)std::max<uint64_t>(64, (Dd + 31) / 32 * 32);
    return threads;
}

// Spin-up pass shape: block width W (multiple of 32, no wider than the rows need),
// S = threads / W row slots, RR rows per thread.
struct UpShape {
    int W, S, RR;
};
UpShape up_shape(const HvConfig &c, uint64_t Dd) {
    UpShape u;
    int threads = c.up_threads > 0 ? c.up_threads : 1024;
    u.W = c.up_block > 0 ? c.up_block : 256;
    const int need = (int)std::min<uint64_t>(1024, (Dd + 31) / 32 * 32);
    if (u.W > need) u.W = need;
    if (u.W > threads) u.W = threads;
    u.S = std::max(1, threads / u.W);
    u.RR = c.up_rows == 4 ? 4 : c.up_rows == 2 ? 2 : 1;
    return u;
}

template <int R, typename T, bool SMEM, bool DO_A>
hb_status launch_hv(hb_handle h, const HvArgs<T> &a, const T *x, T *y, cudaStream_t st, size_t smem, int threads) {
    if (threads <= 512) return launch_hv_lb<R, T, SMEM, 512, DO_A>(h, a, x, y, st, smem, threads);
    return launch_hv_lb<R, T, SMEM, 1024, DO_A>(h, a, x, y, st, smem, threads);
}

// Two adjacent columns per thread (one vector load per operand) when every row
// of x and y starts on a 2-element boundary.
template <typename T>
bool up_pairs(uint64_t Dd, const void *x, const void *y) {
    return Dd % 2 == 0 && ((uintptr_t)x | (uintptr_t)y) % (2 * sizeof(T)) == 0;
}

template <int RR, typename T, bool IDX32, int V>
hb_status launch_up_v(hb_handle h, const HvArgs<T> &a, const T *x, T *y, cudaStream_t st, const UpShape &u) {
    const int RA = u.S * RR, threads = u.W * u.S;
    const size_t smem = hv_up_smem_bytes<IDX32>(RA, a.zmax_up, sizeof(T));
    const uint64_t n_groups = (a.Du + RA - 1) / RA, n_items = (a.Dd + (uint64_t)u.W * V - 1) / ((uint64_t)u.W * V) * n_groups;
    auto kern = threads <= 512 ? k_hv_up<RR, T, IDX32, 512, V> : k_hv_up<RR, T, IDX32, 1024, V>;
    unsigned grid = 0;
    hb_status s = persistent_launch_dims(h, kern, threads, smem, n_items, &grid);
    if (s != HB_OK) return s;
    kern<<<grid, threads, smem, st>>>(a, x, y, u.W, n_groups, n_items);
    PD_CUDA(cudaGetLastError());
    return HB_OK;
}

template <int RR, typename T, bool IDX32>
hb_status launch_up(hb_handle h, const HvArgs<T> &a, const T *x, T *y, cudaStream_t st, const UpShape &u) {
    return up_pairs<T>(a.Dd, x, y) ? launch_up_v<RR, T, IDX32, 2>(h, a, x, y, st, u)
                                   : launch_up_v<RR, T, IDX32, 1>(h, a, x, y, st, u);
}

template <int R, int NC, int LB>
__global__ void __launch_bounds__(LB) k_hv_f_wb(const FWbArgs a, const float *__restrict__ x, float *__restrict__ y) {
    extern __shared__ __align__(16) unsigned char smem[];
    const uint64_t ngroups = (a.Du + R - 1) / R;
    for (uint64_t g = blockIdx.x; g < ngroups; g += gridDim.x) hv_f_wb_group<R, NC>(a, x, y, g, smem);
}

template <int R, int NC>
hb_status launch_f_wb(hb_handle h, const FWbArgs &a, const float *x, float *y, cudaStream_t st, int threads) {
    auto kern = threads <= 512 ? k_hv_f_wb<R, NC, 512> : k_hv_f_wb<R, NC, 1024>;
    const size_t smem = hv_f_wb_smem_bytes(R, a.Dd);
    unsigned grid = 0;
    hb_status s = persistent_launch_dims(h, kern, threads, smem, (a.Du + R - 1) / R, &grid);
    if (s != HB_OK) return s;
    kern<<<grid, threads, smem, st>>>(a, x, y);
    PD_CUDA(cudaGetLastError());
    return HB_OK;
}

template <int R>
hb_status launch_f_wb_r(hb_handle h, const FWbArgs &a, const float *x, float *y, cudaStream_t st, int threads) {
    switch (std::max(1, h->n_classes)) {
        case 1: return launch_f_wb<R, 1>(h, a, x, y, st, threads);
        case 2: return launch_f_wb<R, 2>(h, a, x, y, st, threads);
        case 3: return launch_f_wb<R, 3>(h, a, x, y, st, threads);
        default: return launch_f_wb<R, 4>(h, a, x, y, st, threads);
    }
}

// Float32 row pass of the split form on the warp-blocked spin-down table, when
// the handle has one and R rows (requested, else the widest) fit in shared memory.
hb_status f32_wb_row_pass(hb_handle h, const HvArgs<float> &a, const float *x, float *y, cudaStream_t st,
                          const HvConfig &cfg, size_t budget, bool *done) {
    *done = false;
    if (!h->dn.wb_ok || h->dn.wb_nblk == 0) return HB_OK;
    auto fits = [&](int R) { return hv_f_wb_smem_bytes(R, a.Dd) <= budget; };
    int R = cfg.rows;
    if (R != 1 && R != 2 && R != 4) R = 0;
    if (R == 0 || !fits(R)) R = fits(4) ? 4 : fits(2) ? 2 : fits(1) ? 1 : 0;
    if (R == 0) return HB_OK;
    FWbArgs f;
    f.Du = a.Du;
    f.Dd = a.Dd;
    f.U = a.U;
    f.str_up = a.str_up;
    f.order = a.order;
    for (int c = 0; c < PD_FX_MAXC; ++c) f.tc[c] = c < h->n_classes ? (float)(-h->class_t[c]) : 0.0f;
    f.wb_perm = h->dn.wb_perm;
    f.wb_str = h->dn.wb_str;
    f.wb_base = h->dn.wb_base;
    f.wb_ent = h->dn.wb_ent;
    f.wb_caps = h->dn.wb_caps;
    f.wb_nblk = h->dn.wb_nblk;
    const int threads = pick_threads(cfg, a.Dd);
    *done = true;
    if (R == 4) return launch_f_wb_r<4>(h, f, x, y, st, threads);
    if (R == 2) return launch_f_wb_r<2>(h, f, x, y, st, threads);
    return launch_f_wb_r<1>(h, f, x, y, st, threads);
}

template <typename T, bool DO_A>
hb_status row_pass(hb_handle h, const HvArgs<T> &a, const T *x, T *y, cudaStream_t st, const HvConfig &cfg) {
    const int threads = pick_threads(cfg, a.Dd);
    int max_smem = 0;
    PD_CUDA(cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device));
    const size_t budget = (size_t)max_smem;
    if constexpr (std::is_same<T, float>::value && !DO_A) {
        bool done = false;
        hb_status s = f32_wb_row_pass(h, a, x, y, st, cfg, budget, &done);
        if (s != HB_OK || done) return s;
    }
    auto fits = [&](int R) { return hv_smem_bytes(R, a.zmax_up, sizeof(T), a.Dd, true) <= budget; };
    // requested row-group size if it fits, else the widest that fits
    int R = cfg.rows;
    if (R != 1 && R != 2 && R != 4) R = 0;
    if (R == 0 || !fits(R)) R = fits(4) ? 4 : fits(2) ? 2 : fits(1) ? 1 : 0;
    switch (R) {
        case 4:
            return launch_hv<4, T, true, DO_A>(h, a, x, y, st, hv_smem_bytes(4, a.zmax_up, sizeof(T), a.Dd, true),
                                               threads);
        case 2:
            return launch_hv<2, T, true, DO_A>(h, a, x, y, st, hv_smem_bytes(2, a.zmax_up, sizeof(T), a.Dd, true),
                                               threads);
        case 1:
            return launch_hv<1, T, true, DO_A>(h, a, x, y, st, hv_smem_bytes(1, a.zmax_up, sizeof(T), a.Dd, true),
                                               threads);
        default:  // rows too long for shared memory: gather from L2
            return launch_hv<1, T, false, DO_A>(h, a, x, y, st,
                                                hv_smem_bytes(1, a.zmax_up, sizeof(T), a.Dd, false), threads);
    }
}

template <typename T>
hb_status apply_t(hb_handle h, const T *x, T *y, cudaStream_t st, int part) {
    HvArgs<T> a;
    a.Du = h->D_up;
    a.Dd = h->D_dn;
    a.U = (T)h->U;
    a.str_up = h->up.str;
    a.str_dn = h->dn.str;
    a.cnt_up = h->up.count;
    a.cnt_dn = h->dn.count;
    a.tgt_up = h->up.target;
    a.tgt_dn = h->dn.target;
    if constexpr (sizeof(T) == 8) {
        a.val_up = reinterpret_cast<const T *>(h->up.val);
        a.val_dn = reinterpret_cast<const T *>(h->dn.val);
    } else {
        a.val_up = reinterpret_cast<const T *>(h->up.valf);
        a.val_dn = reinterpret_cast<const T *>(h->dn.valf);
    }
    a.zmax_up = h->up.zmax;
    const HvConfig &cfg = h->hv_cfg[sizeof(T) == 8 ? HB_F64 : HB_F32];
    a.order = cfg.order ? h->d_row_order : nullptr;
    const bool split = part != kAll || cfg.split;
    if (!split) return row_pass<T, true>(h, a, x, y, st, cfg);
    hb_status s = HB_OK;
    if (part != kUpPass && (s = row_pass<T, false>(h, a, x, y, st, cfg)) != HB_OK) return s;
    if (part == kRowPass) return HB_OK;
    const UpShape u = up_shape(cfg, a.Dd);
    if (h->D < (1ull << 32)) {
        if (u.RR == 4) return launch_up<4, T, true>(h, a, x, y, st, u);
        return u.RR == 2 ? launch_up<2, T, true>(h, a, x, y, st, u) : launch_up<1, T, true>(h, a, x, y, st, u);
    }
    if (u.RR == 4) return launch_up<4, T, false>(h, a, x, y, st, u);
    return u.RR == 2 ? launch_up<2, T, false>(h, a, x, y, st, u) : launch_up<1, T, false>(h, a, x, y, st, u);
}

template <int R, int NC, bool SMEM, int LB, bool DO_A>
__global__ void __launch_bounds__(LB) k_hv_fx(const FxArgs a, const int64_t *__restrict__ x,
                                              int64_t *__restrict__ y) {
    extern __shared__ __align__(16) unsigned char smem[];
    hv_fx_load_diag(a, smem);
    const uint64_t ngroups = (a.Du + R - 1) / R;
    for (uint64_t g = blockIdx.x; g < ngroups; g += gridDim.x) hv_fx_group<R, NC, SMEM, DO_A>(a, x, y, g, smem);
}

template <int R, int NC, int LB>
__global__ void __launch_bounds__(LB) k_hv_fx_wb(const FxArgs a, const int64_t *__restrict__ x,
                                                 int64_t *__restrict__ y) {
    extern __shared__ __align__(16) unsigned char smem[];
    hv_fx_load_diag(a, smem);
    const uint64_t ngroups = (a.Du + R - 1) / R;
    for (uint64_t g = blockIdx.x; g < ngroups; g += gridDim.x) hv_fx_wb_group<R, NC>(a, x, y, g, smem);
}

template <int R, int NC, int LB>
hb_status launch_hv_fx_wb_lb(hb_handle h, const FxArgs &a, const int64_t *x, int64_t *y, cudaStream_t st,
                             int threads) {
    auto kern = k_hv_fx_wb<R, NC, LB>;
    const size_t smem = hv_fx_wb_smem_bytes(R, a.Dd);
    unsigned grid = 0;
    hb_status s = persistent_launch_dims(h, kern, threads, smem, (a.Du + R - 1) / R, &grid);
    if (s != HB_OK) return s;
    kern<<<grid, threads, smem, st>>>(a, x, y);
    PD_CUDA(cudaGetLastError());
    return HB_OK;
}

template <int R, int NC>
hb_status launch_hv_fx_wb(hb_handle h, const FxArgs &a, const int64_t *x, int64_t *y, cudaStream_t st, int threads) {
    if (threads <= 512) return launch_hv_fx_wb_lb<R, NC, 512>(h, a, x, y, st, threads);
    return launch_hv_fx_wb_lb<R, NC, 1024>(h, a, x, y, st, threads);
}

template <int RR, int NC, bool IDX32, int LB, int V>
__global__ void __launch_bounds__(LB) k_hv_fx_up(const FxArgs a, const int64_t *__restrict__ x,
                                                   int64_t *__restrict__ y, int W, uint64_t n_groups,
                                                   uint64_t n_items) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int S = blockDim.x / W;
    ItemWalk w(n_groups);
    for (uint64_t it = blockIdx.x; it < n_items; it += gridDim.x, w.next())
        hv_fx_up_item<RR, NC, IDX32, V>(a, x, y, w.j, w.g, W, S, smem);
}

template <int R, int NC, bool SMEM, int LB, bool DO_A>
hb_status launch_hv_fx_lb(hb_handle h, const FxArgs &a, const int64_t *x, int64_t *y, cudaStream_t st, int threads) {
    auto kern = k_hv_fx<R, NC, SMEM, LB, DO_A>;
    const size_t smem = hv_fx_smem_bytes(R, a.zmax_up, a.Dd, SMEM);
    unsigned grid = 0;
    hb_status s = persistent_launch_dims(h, kern, threads, smem, (a.Du + R - 1) / R, &grid);
    if (s != HB_OK) return s;
    kern<<<grid, threads, smem, st>>>(a, x, y);
    PD_CUDA(cudaGetLastError());
    return HB_OK;
}

template <int R, int NC, bool SMEM, bool DO_A>
hb_status launch_hv_fx(hb_handle h, const FxArgs &a, const int64_t *x, int64_t *y, cudaStream_t st, int threads) {
    if (threads <= 512) return launch_hv_fx_lb<R, NC, SMEM, 512, DO_A>(h, a, x, y, st, threads);
    return launch_hv_fx_lb<R, NC, SMEM, 1024, DO_A>(h, a, x, y, st, threads);
}

template <int RR, int NC, bool IDX32, int V>
hb_status launch_fx_up_v(hb_handle h, const FxArgs &a, const int64_t *x, int64_t *y, cudaStream_t st,
                         const UpShape &u) {
    const int RA = u.S * RR, threads = u.W * u.S;
    const size_t smem = hv_fx_up_smem_bytes<IDX32>(RA, a.zmax_up);
    const uint64_t n_groups = (a.Du + RA - 1) / RA, n_items = (a.Dd + (uint64_t)u.W * V - 1) / ((uint64_t)u.W * V) * n_groups;
    auto kern = threads <= 512 ? k_hv_fx_up<RR, NC, IDX32, 512, V> : k_hv_fx_up<RR, NC, IDX32, 1024, V>;
    unsigned grid = 0;
    hb_status s = persistent_launch_dims(h, kern, threads, smem, n_items, &grid);
    if (s != HB_OK) return s;
    kern<<<grid, threads, smem, st>>>(a, x, y, u.W, n_groups, n_items);
    PD_CUDA(cudaGetLastError());
    return HB_OK;
}

template <int RR, int NC, bool IDX32>
hb_status launch_fx_up(hb_handle h, const FxArgs &a, const int64_t *x, int64_t *y, cudaStream_t st,
                       const UpShape &u) {
    return up_pairs<int64_t>(a.Dd, x, y) ? launch_fx_up_v<RR, NC, IDX32, 2>(h, a, x, y, st, u)
                                         : launch_fx_up_v<RR, NC, IDX32, 1>(h, a, x, y, st, u);
}

template <int NC, bool DO_A>
hb_status fx_row_pass(hb_handle h, const FxArgs &a, const int64_t *x, int64_t *y, cudaStream_t st, size_t budget,
                      const HvConfig &cfg) {
    const int threads = pick_threads(cfg, a.Dd);
    if (!DO_A && a.wb_nblk > 0) {  // split form: warp-blocked spin-down table
        auto fits_wb = [&](int R) { return hv_fx_wb_smem_bytes(R, a.Dd) <= budget; };
        int R = cfg.rows == 1 ? 1 : 2;
        if (!fits_wb(R)) R = 1;
        if (fits_wb(R))
            return R == 2 ? launch_hv_fx_wb<2, NC>(h, a, x, y, st, threads)
                          : launch_hv_fx_wb<1, NC>(h, a, x, y, st, threads);
    }
    auto fits = [&](int R) { return hv_fx_smem_bytes(R, a.zmax_up, a.Dd) <= budget; };
    int R = cfg.rows;
    if (R != 1 && R != 2) R = 0;
    if (R == 0 || !fits(R)) R = fits(2) ? 2 : fits(1) ? 1 : 0;
    if (R == 2) return launch_hv_fx<2, NC, true, DO_A>(h, a, x, y, st, threads);
    if (R == 1) return launch_hv_fx<1, NC, true, DO_A>(h, a, x, y, st, threads);
    return launch_hv_fx<1, NC, false, DO_A>(h, a, x, y, st, threads);  // rows too long for shared memory
}

template <int NC>
hb_status apply_fx_nc(hb_handle h, const FxArgs &a, const int64_t *x, int64_t *y, cudaStream_t st, size_t budget,
                      const HvConfig &cfg, int part) {
    const bool split = part != kAll || cfg.split;
    if (!split) return fx_row_pass<NC, true>(h, a, x, y, st, budget, cfg);
    hb_status s = HB_OK;
    if (part != kUpPass && (s = fx_row_pass<NC, false>(h, a, x, y, st, budget, cfg)) != HB_OK) return s;
    if (part == kRowPass) return HB_OK;
    const UpShape u = up_shape(cfg, a.Dd);
    if (h->D < (1ull << 32)) {
        if (u.RR == 4) return launch_fx_up<4, NC, true>(h, a, x, y, st, u);
        return u.RR == 2 ? launch_fx_up<2, NC, true>(h, a, x, y, st, u) : launch_fx_up<1, NC, true>(h, a, x, y, st, u);
    }
    if (u.RR == 4) return launch_fx_up<4, NC, false>(h, a, x, y, st, u);
    return u.RR == 2 ? launch_fx_up<2, NC, false>(h, a, x, y, st, u) : launch_fx_up<1, NC, false>(h, a, x, y, st, u);
}

hb_status apply_fx(hb_handle h, const int64_t *x, int64_t *y, cudaStream_t st, int part) {
    if (!h->fx_ok) return HB_ERR_INVALID_ARG;
    FxArgs a;
    a.Du = h->D_up;
    a.Dd = h->D_dn;
    a.str_up = h->up.str;
    a.str_dn = h->dn.str;
    a.seg_up = h->up.seg;
    a.seg_dn = h->dn.seg;
    a.ft_up = h->up.ftarget;
    a.ft_dn = h->dn.ftarget;
    a.zmax_up = h->up.zmax;
    if (h->dn.wb_ok) {
        a.wb_perm = h->dn.wb_perm;
        a.wb_str = h->dn.wb_str;
        a.wb_base = h->dn.wb_base;
        a.wb_ent = h->dn.wb_ent;
        a.wb_caps = h->dn.wb_caps;
        a.wb_nblk = h->dn.wb_nblk;
    }
    const HvConfig &cfg = h->hv_cfg[HB_FX64];
    a.order = cfg.order ? h->d_row_order : nullptr;
    FxCoef diag[PD_MAXL + 1], cls[PD_FX_MAXC];
    hb_status s = pd_fx_coefs(h, diag, cls);
    if (s != HB_OK) return s;
    for (int k = 0; k <= PD_MAXL; ++k) {
        a.Kd[k] = diag[k].K;
        a.Gd[k] = diag[k].G;
    }
    for (int c = 0; c < PD_FX_MAXC; ++c) {
        a.Kc[c] = cls[c].K;
        a.Gc[c] = cls[c].G;
    }
    int max_smem = 0;
    PD_CUDA(cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device));
    const size_t budget = (size_t)max_smem;
    switch (std::max(1, h->n_classes)) {
        case 1: return apply_fx_nc<1>(h, a, x, y, st, budget, cfg, part);
        case 2: return apply_fx_nc<2>(h, a, x, y, st, budget, cfg, part);
        case 3: return apply_fx_nc<3>(h, a, x, y, st, budget, cfg, part);
        default: return apply_fx_nc<4>(h, a, x, y, st, budget, cfg, part);
    }
}

hb_status apply_part(hb_handle h, hb_dtype dt, const void *x, void *y, cudaStream_t st, int part) {
    if (h->ks) return pd_k_apply(h, dt, x, y, st);  // momentum sector: one kernel, no parts
    if (dt == HB_F64) return apply_t<double>(h, static_cast<const double *>(x), static_cast<double *>(y), st, part);
    if (dt == HB_FX64) return apply_fx(h, static_cast<const int64_t *>(x), static_cast<int64_t *>(y), st, part);
    return apply_t<float>(h, static_cast<const float *>(x), static_cast<float *>(y), st, part);
}

}  // namespace

hb_status pd_apply(hb_handle h, hb_dtype dt, const void *x, void *y, cudaStream_t st) {
    if (h->ks) return pd_k_apply(h, dt, x, y, st);
    return apply_part(h, dt, x, y, st, kAll);
}

int pd_hv_launches(hb_handle h, hb_dtype dt) { return !h->ks && h->hv_cfg[dt].split ? 2 : 1; }

namespace {

void to_public(const HvConfig &c, float ms, hb_hv_config *out) {
    out->rows_per_cta = c.rows;
    out->threads_per_cta = c.threads;
    out->visit_order = c.order;
    out->ms = ms;
    out->split = c.split;
    out->up_block = c.up_block;
    out->up_threads = c.up_threads;
    out->up_rows = c.up_rows;
}

// Average time of reps launches of one part of H·v under configuration c.
hb_status time_part(hb_handle h, hb_dtype dt, const void *x, void *y, cudaStream_t st, int part, int reps,
                    cudaEvent_t e0, cudaEvent_t e1, float *ms) {
    hb_status s = apply_part(h, dt, x, y, st, part);  // warm-up
    if (s != HB_OK) return s;
    cudaEventRecord(e0, st);
    for (int k = 0; k < reps && s == HB_OK; ++k) s = apply_part(h, dt, x, y, st, part);
    cudaEventRecord(e1, st);
    if (cudaEventSynchronize(e1) != cudaSuccess) return HB_ERR_CUDA;
    if (s != HB_OK) return s;
    float t = 0.f;
    cudaEventElapsedTime(&t, e0, e1);
    *ms = t / (float)reps;
    return HB_OK;
}

}  // namespace

extern "C" hb_status hubbard_get_hv_config(hb_handle h, hb_dtype dt, hb_hv_config *cfg) {
    if (!h || !cfg || (dt != HB_F64 && dt != HB_F32 && dt != HB_FX64)) return HB_ERR_INVALID_ARG;
    to_public(h->hv_cfg[dt], 0.f, cfg);
    return HB_OK;
}

extern "C" hb_status hubbard_set_hv_config(hb_handle h, hb_dtype dt, const hb_hv_config *cfg) {
    if (!h || !cfg || (dt != HB_F64 && dt != HB_F32 && dt != HB_FX64)) return HB_ERR_INVALID_ARG;
    if (cfg->rows_per_cta < 0 || cfg->rows_per_cta > 4 || cfg->threads_per_cta < 0 || cfg->threads_per_cta > 1024 ||
        cfg->threads_per_cta % 32 != 0 || (cfg->visit_order != 0 && cfg->visit_order != 1))
        return HB_ERR_INVALID_ARG;
    if ((cfg->split != 0 && cfg->split != 1) || cfg->up_block < 0 || cfg->up_block % 32 != 0 ||
        cfg->up_threads < 0 || cfg->up_threads > 1024 || cfg->up_rows < 0 || cfg->up_rows > 4 || cfg->up_rows == 3)
        return HB_ERR_INVALID_ARG;
    const int ub = cfg->up_block > 0 ? cfg->up_block : 256, ut = cfg->up_threads > 0 ? cfg->up_threads : 1024;
    if (ub > ut || ut % ub != 0) return HB_ERR_INVALID_ARG;
    HvConfig &c = h->hv_cfg[dt];
    c.rows = cfg->rows_per_cta;
    c.threads = cfg->threads_per_cta;
    c.order = cfg->visit_order;
    c.split = cfg->split;
    c.up_block = cfg->up_block;
    c.up_threads = cfg->up_threads;
    c.up_rows = cfg->up_rows;
    return HB_OK;
}

// Times every (rows per group, threads, visiting order) candidate of the
// one-kernel form and of the split form's row pass, then every spin-up pass
// shape, on the caller's vectors with CUDA events; keeps the fastest whole.
extern "C" hb_status hubbard_autotune(hb_handle h, hb_dtype dt, const void *x, void *y, int32_t reps,
                                      hb_hv_config *best, void *stream) {
    if (!h || !x || !y || reps < 1 || (dt != HB_F64 && dt != HB_F32 && dt != HB_FX64)) return HB_ERR_INVALID_ARG;
    if (dt == HB_FX64 && !h->fx_ok) return HB_ERR_INVALID_ARG;
    hb_status s = pd_build_tables(h);
    if (s != HB_OK) return s;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    cudaEvent_t e0, e1;
    PD_CUDA(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return HB_ERR_CUDA;
    }
    if (h->ks) {  // momentum sectors have one launch shape: report its time
        float ms = 0.f;
        s = time_part(h, dt, x, y, st, kAll, reps, e0, e1, &ms);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (s == HB_OK && best) to_public(h->hv_cfg[dt], ms, best);
        return s;
    }
    const HvConfig saved = h->hv_cfg[dt];
    HvConfig fused_win = saved, row_win = saved;
    float fused_ms = 3.4e38f, row_ms = 3.4e38f;
    const int rows_c[3] = {1, 2, 4};
    const int thr_c[3] = {256, 512, 1024};
    for (int order = 0; order <= 1 && s == HB_OK; ++order)
        for (int ri = 0; ri < (dt == HB_FX64 ? 2 : 3) && s == HB_OK; ++ri)
            for (int ti = 0; ti < 3 && s == HB_OK; ++ti)
                for (int part = kAll; part <= kRowPass && s == HB_OK; ++part) {
                    HvConfig c;
                    c.rows = rows_c[ri];
                    c.threads = thr_c[ti];
                    c.order = order;
                    h->hv_cfg[dt] = c;
                    float ms = 0.f;
                    s = time_part(h, dt, x, y, st, part, reps, e0, e1, &ms);
                    if (s != HB_OK) break;
                    if (part == kAll && ms < fused_ms) fused_ms = ms, fused_win = c;
                    if (part == kRowPass && ms < row_ms) row_ms = ms, row_win = c;
                }
    HvConfig split_win = row_win;
    float up_ms = 3.4e38f;
    const int blk_c[3] = {128, 256, 512};
    const int uthr_c[2] = {512, 1024};
    for (int bi = 0; bi < 3 && s == HB_OK; ++bi)
        for (int ti = 0; ti < 2 && s == HB_OK; ++ti)
            for (int rr = 1; rr <= 4 && s == HB_OK; rr *= 2) {
                HvConfig c = row_win;
                c.split = 1;
                c.up_block = blk_c[bi];
                c.up_threads = uthr_c[ti];
                c.up_rows = rr;
                h->hv_cfg[dt] = c;
                float ms = 0.f;
                s = time_part(h, dt, x, y, st, kUpPass, reps, e0, e1, &ms);
                if (s == HB_OK && ms < up_ms) up_ms = ms, split_win = c;
            }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s != HB_OK) {
        h->hv_cfg[dt] = saved;
        return s;
    }
    const bool use_split = row_ms + up_ms < fused_ms;
    h->hv_cfg[dt] = use_split ? split_win : fused_win;
    if (best) to_public(h->hv_cfg[dt], use_split ? row_ms + up_ms : fused_ms, best);
    return HB_OK;
}

extern "C" hb_status hubbard_apply(hb_handle h, hb_dtype dt, const void *x, void *y, void *stream) {
    if (!h || !x || !y || (dt != HB_F64 && dt != HB_F32 && dt != HB_FX64)) return HB_ERR_INVALID_ARG;
    if (dt == HB_FX64 && !h->fx_ok) return HB_ERR_INVALID_ARG;
    const size_t es = dt == HB_F32 ? 4 : 8;
    const uintptr_t xb = (uintptr_t)x, yb = (uintptr_t)y, n = (uintptr_t)(h->D * es);
    if (xb < yb + n && yb < xb + n) return HB_ERR_INVALID_ARG;  // overlapping vectors
    hb_status s = pd_build_tables(h);
    if (s != HB_OK) return s;
    return pd_apply(h, dt, x, y, reinterpret_cast<cudaStream_t>(stream));
}

extern "C" hb_status hubbard_apply_timed(hb_handle h, hb_dtype dt, const void *x, void *y, void *ev_begin,
                                         void *ev_mid, void *ev_end, void *stream) {
    if (!h || !x || !y || !ev_begin || !ev_mid || !ev_end || (dt != HB_F64 && dt != HB_F32 && dt != HB_FX64))
        return HB_ERR_INVALID_ARG;
    if (dt == HB_FX64 && !h->fx_ok) return HB_ERR_INVALID_ARG;
    const size_t es = dt == HB_F32 ? 4 : 8;
    const uintptr_t xb = (uintptr_t)x, yb = (uintptr_t)y, n = (uintptr_t)(h->D * es);
    if (xb < yb + n && yb < xb + n) return HB_ERR_INVALID_ARG;
    hb_status s = pd_build_tables(h);
    if (s != HB_OK) return s;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    cudaEvent_t e0 = reinterpret_cast<cudaEvent_t>(ev_begin), e1 = reinterpret_cast<cudaEvent_t>(ev_mid),
                e2 = reinterpret_cast<cudaEvent_t>(ev_end);
    PD_CUDA(cudaEventRecord(e0, st));
    if (h->ks || !h->hv_cfg[dt].split) {
        if ((s = pd_apply(h, dt, x, y, st)) != HB_OK) return s;
        PD_CUDA(cudaEventRecord(e1, st));
    } else {
        if ((s = apply_part(h, dt, x, y, st, kRowPass)) != HB_OK) return s;
        PD_CUDA(cudaEventRecord(e1, st));
        if ((s = apply_part(h, dt, x, y, st, kUpPass)) != HB_OK) return s;
    }
    PD_CUDA(cudaEventRecord(e2, st));
    return HB_OK;
}

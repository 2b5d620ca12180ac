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

namespace {

template <int R, typename T, bool SMEM, int LB>
__global__ void __launch_bounds__(LB) k_hv(const HvArgs<T> a, const T *__restrict__ x, T *__restrict__ y) {
    extern __shared__ __align__(16) unsigned char smem[];
    const uint64_t ngroups = (a.Du + R - 1) / R;
    for (uint64_t g = blockIdx.x; g < ngroups; g += gridDim.x) hv_group<R, T, SMEM>(a, x, y, g, smem);
}


bool a_small(uint64_t Dd, int threads) { return Dd < (uint64_t)threads; }

template <int R, typename T, bool SMEM, int LB>
hb_status launch_hv_lb(hb_handle h, const HvArgs<T> &a, const T *x, T *y, cudaStream_t st, size_t smem,
                       int threads) {
    auto kern = k_hv<R, T, SMEM, LB>;
    PD_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    PD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem));
    if (per_sm < 1) return HB_ERR_NO_MEMORY;
    const uint64_t ngroups = (a.Du + R - 1) / R;
    const uint64_t grid = std::min<uint64_t>(ngroups, (uint64_t)per_sm * h->sm_count);
    kern<<<(unsigned)grid, threads, smem, st>>>(a, x, y);
    PD_CUDA(cudaGetLastError());
    return HB_OK;
}

int pick_threads(const HvConfig &c, uint64_t Dd) {
    int threads = c.threads > 0 ? c.threads : 1024;
    if (a_small(Dd, threads)) threads = (int)std::max<uint64_t>(64, (Dd + 31) / 32 * 32);
    return threads;
}

template <int R, typename T, bool SMEM>
hb_status launch_hv(hb_handle h, const HvArgs<T> &a, const T *x, T *y, cudaStream_t st, size_t smem, int threads) {
    if (threads <= 512) return launch_hv_lb<R, T, SMEM, 512>(h, a, x, y, st, smem, threads);
    return launch_hv_lb<R, T, SMEM, 1024>(h, a, x, y, st, smem, threads);
}

template <typename T>
hb_status apply_t(hb_handle h, const T *x, T *y, cudaStream_t st) {
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
    const int threads = pick_threads(cfg, a.Dd);
    int max_smem = 0;
    PD_CUDA(cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device));
    const size_t budget = (size_t)max_smem;
    auto fits = [&](int R) { return hv_smem_bytes(R, a.zmax_up, sizeof(T), a.Dd, true) <= budget; };
    // requested row-group size if it fits, else the widest that fits
    int R = cfg.rows;
    if (R != 1 && R != 2 && R != 4) R = 0;
    if (R == 0 || !fits(R)) R = fits(4) ? 4 : fits(2) ? 2 : fits(1) ? 1 : 0;
    switch (R) {
        case 4: return launch_hv<4, T, true>(h, a, x, y, st, hv_smem_bytes(4, a.zmax_up, sizeof(T), a.Dd, true), threads);
        case 2: return launch_hv<2, T, true>(h, a, x, y, st, hv_smem_bytes(2, a.zmax_up, sizeof(T), a.Dd, true), threads);
        case 1: return launch_hv<1, T, true>(h, a, x, y, st, hv_smem_bytes(1, a.zmax_up, sizeof(T), a.Dd, true), threads);
        default:  // rows too long for shared memory: gather from L2
            return launch_hv<1, T, false>(h, a, x, y, st, hv_smem_bytes(1, a.zmax_up, sizeof(T), a.Dd, false), threads);
    }
}

template <int R, int NC, bool SMEM, int LB>
__global__ void __launch_bounds__(LB) k_hv_fx(const FxArgs a, const int64_t *__restrict__ x,
                                              int64_t *__restrict__ y) {
    extern __shared__ __align__(16) unsigned char smem[];
    hv_fx_load_diag(a, smem);
    const uint64_t ngroups = (a.Du + R - 1) / R;
    for (uint64_t g = blockIdx.x; g < ngroups; g += gridDim.x) hv_fx_group<R, NC, SMEM>(a, x, y, g, smem);
}



template <int R, int NC, bool SMEM, int LB>
hb_status launch_hv_fx_lb(hb_handle h, const FxArgs &a, const int64_t *x, int64_t *y, cudaStream_t st, int threads) {
    auto kern = k_hv_fx<R, NC, SMEM, LB>;
    const size_t smem = hv_fx_smem_bytes(R, a.zmax_up, a.Dd, SMEM);
    PD_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    PD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem));
    if (per_sm < 1) return HB_ERR_NO_MEMORY;
    const uint64_t ngroups = (a.Du + R - 1) / R;
    const uint64_t grid = std::min<uint64_t>(ngroups, (uint64_t)per_sm * h->sm_count);
    kern<<<(unsigned)grid, threads, smem, st>>>(a, x, y);
    PD_CUDA(cudaGetLastError());
    return HB_OK;
}

template <int R, int NC, bool SMEM>
hb_status launch_hv_fx(hb_handle h, const FxArgs &a, const int64_t *x, int64_t *y, cudaStream_t st, int threads) {
    if (threads <= 512) return launch_hv_fx_lb<R, NC, SMEM, 512>(h, a, x, y, st, threads);
    return launch_hv_fx_lb<R, NC, SMEM, 1024>(h, a, x, y, st, threads);
}

template <int NC>
hb_status apply_fx_nc(hb_handle h, const FxArgs &a, const int64_t *x, int64_t *y, cudaStream_t st, size_t budget,
                      const HvConfig &cfg) {
    const int threads = pick_threads(cfg, a.Dd);
    auto fits = [&](int R) { return hv_fx_smem_bytes(R, a.zmax_up, a.Dd) <= budget; };
    int R = cfg.rows;
    if (R != 1 && R != 2) R = 0;
    if (R == 0 || !fits(R)) R = fits(2) ? 2 : fits(1) ? 1 : 0;
    if (R == 2) return launch_hv_fx<2, NC, true>(h, a, x, y, st, threads);
    if (R == 1) return launch_hv_fx<1, NC, true>(h, a, x, y, st, threads);
    return launch_hv_fx<1, NC, false>(h, a, x, y, st, threads);  // rows too long for shared memory
}

hb_status apply_fx(hb_handle h, const int64_t *x, int64_t *y, cudaStream_t st) {
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
        case 1: return apply_fx_nc<1>(h, a, x, y, st, budget, cfg);
        case 2: return apply_fx_nc<2>(h, a, x, y, st, budget, cfg);
        case 3: return apply_fx_nc<3>(h, a, x, y, st, budget, cfg);
        default: return apply_fx_nc<4>(h, a, x, y, st, budget, cfg);
    }
}

}  // namespace

hb_status pd_apply(hb_handle h, hb_dtype dt, const void *x, void *y, cudaStream_t st) {
    if (dt == HB_F64) return apply_t<double>(h, static_cast<const double *>(x), static_cast<double *>(y), st);
    if (dt == HB_FX64) return apply_fx(h, static_cast<const int64_t *>(x), static_cast<int64_t *>(y), st);
    return apply_t<float>(h, static_cast<const float *>(x), static_cast<float *>(y), st);
}

extern "C" hb_status hubbard_get_hv_config(hb_handle h, hb_dtype dt, hb_hv_config *cfg) {
    if (!h || !cfg || (dt != HB_F64 && dt != HB_F32 && dt != HB_FX64)) return HB_ERR_INVALID_ARG;
    const HvConfig &c = h->hv_cfg[dt];
    cfg->rows_per_cta = c.rows;
    cfg->threads_per_cta = c.threads;
    cfg->visit_order = c.order;
    cfg->ms = 0.f;
    return HB_OK;
}

extern "C" hb_status hubbard_set_hv_config(hb_handle h, hb_dtype dt, const hb_hv_config *cfg) {
    if (!h || !cfg || (dt != HB_F64 && dt != HB_F32 && dt != HB_FX64)) return HB_ERR_INVALID_ARG;
    if (cfg->rows_per_cta < 0 || cfg->rows_per_cta > 4 || cfg->threads_per_cta < 0 || cfg->threads_per_cta > 1024 ||
        cfg->threads_per_cta % 32 != 0 || (cfg->visit_order != 0 && cfg->visit_order != 1))
        return HB_ERR_INVALID_ARG;
    HvConfig &c = h->hv_cfg[dt];
    c.rows = cfg->rows_per_cta;
    c.threads = cfg->threads_per_cta;
    c.order = cfg->visit_order;
    return HB_OK;
}

// Times every (rows per group, threads, visiting order) candidate on the
// caller's vectors with CUDA events and keeps the fastest in the handle.
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
    const HvConfig saved = h->hv_cfg[dt];
    HvConfig win = saved;
    float win_ms = 3.4e38f;
    const int rows_c[3] = {1, 2, 4};
    const int thr_c[3] = {256, 512, 1024};
    for (int order = 0; order <= 1 && s == HB_OK; ++order)
        for (int ri = 0; ri < (dt == HB_FX64 ? 2 : 3) && s == HB_OK; ++ri)
            for (int ti = 0; ti < 3 && s == HB_OK; ++ti) {
                HvConfig c;
                c.rows = rows_c[ri];
                c.threads = thr_c[ti];
                c.order = order;
                h->hv_cfg[dt] = c;
                s = pd_apply(h, dt, x, y, st);  // warm-up
                if (s != HB_OK) break;
                cudaEventRecord(e0, st);
                for (int k = 0; k < reps && s == HB_OK; ++k) s = pd_apply(h, dt, x, y, st);
                cudaEventRecord(e1, st);
                if (cudaEventSynchronize(e1) != cudaSuccess) s = HB_ERR_CUDA;
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                ms /= (float)reps;
                if (s == HB_OK && ms < win_ms) {
                    win_ms = ms;
                    win = c;
                }
            }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    h->hv_cfg[dt] = s == HB_OK ? win : saved;
    if (s != HB_OK) return s;
    if (best) {
        best->rows_per_cta = win.rows;
        best->threads_per_cta = win.threads;
        best->visit_order = win.order;
        best->ms = win_ms;
    }
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

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
// Kernel shape: a persistent grid walks groups of R consecutive rows.  A CTA
// stages its R rows of x in shared memory (interleaved x_s[d * R + r]) so the
// spin-down gathers hit shared memory; the spin-up terms read whole rows
// x[u', :] from global memory, coalesced across the threads of the CTA.  When
// R rows do not fit in shared memory the down gathers read global memory.
#include <algorithm>

#include "pd_common.cuh"

namespace {

template <typename T>
struct HvArgs {
    uint64_t Du, Dd;
    T U;
    const uint32_t *str_up, *str_dn;
    const uint16_t *cnt_up, *cnt_dn;
    const uint32_t *tgt_up, *tgt_dn;
    const T *val_up, *val_dn;
    const uint32_t *order;  // row visiting order (nullptr: storage order)
    int zmax_up;
};

template <int R, typename T, bool SMEM>
__global__ void __launch_bounds__(1024) k_hv(const HvArgs<T> a, const T *__restrict__ x, T *__restrict__ y) {
    extern __shared__ __align__(16) unsigned char smem[];
    const uint64_t Dd = a.Dd;
    // shared layout: [up cols R*zmax u32][up vals R*zmax T][up counts R int][x rows R*Dd T (SMEM only)]
    uint32_t *s_ucol = reinterpret_cast<uint32_t *>(smem);
    const int zr = a.zmax_up > 0 ? a.zmax_up : 1;
    size_t off = ((size_t)R * zr * sizeof(uint32_t) + 15) & ~(size_t)15;
    T *s_uval = reinterpret_cast<T *>(smem + off);
    off = (off + (size_t)R * zr * sizeof(T) + 15) & ~(size_t)15;
    int *s_nup = reinterpret_cast<int *>(smem + off);
    off = (off + R * sizeof(int) + 15) & ~(size_t)15;
    T *s_x = reinterpret_cast<T *>(smem + off);

    const uint64_t ngroups = (a.Du + R - 1) / R;
    for (uint64_t g = blockIdx.x; g < ngroups; g += gridDim.x) {
        const uint64_t p0 = g * R;
        const uint64_t left = a.Du - p0;
        const int nr = left < (uint64_t)R ? (int)left : R;
        uint64_t ur[R];  // the rows of this group
#pragma unroll
        for (int r = 0; r < R; ++r) ur[r] = r < nr ? (a.order ? (uint64_t)a.order[p0 + r] : p0 + r) : 0;
        __syncthreads();  // previous group finished with shared memory
        if (threadIdx.x < R) s_nup[threadIdx.x] = threadIdx.x < nr ? a.cnt_up[ur[threadIdx.x]] : 0;
        for (int e = threadIdx.x; e < R * zr; e += blockDim.x) {
            const int r = e / zr, k = e - r * zr;
            if (r < nr && k < a.zmax_up) {
                const uint64_t u = a.order ? (uint64_t)a.order[p0 + r] : p0 + r;
                s_ucol[e] = a.tgt_up[(uint64_t)k * a.Du + u];
                s_uval[e] = a.val_up[(uint64_t)k * a.Du + u];
            }
        }
        if (SMEM) {
#pragma unroll
            for (int r = 0; r < R; ++r) {
                if (r >= nr) break;
                const T *xr = x + ur[r] * Dd;
                for (uint64_t d = threadIdx.x; d < Dd; d += blockDim.x) s_x[d * R + r] = xr[d];
            }
        }
        __syncthreads();
        uint32_t su[R];
#pragma unroll
        for (int r = 0; r < R; ++r) su[r] = r < nr ? a.str_up[ur[r]] : 0u;

        for (uint64_t d = threadIdx.x; d < Dd; d += blockDim.x) {
            const uint32_t sd = a.str_dn[d];
            T acc[R];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const T xv = SMEM ? s_x[d * R + r] : (r < nr ? x[ur[r] * Dd + d] : T(0));
                acc[r] = a.U * (T)__popc(su[r] & sd) * xv;
            }
            // spin-down hops: gather within the staged rows
            const int nd = a.cnt_dn[d];
            for (int k = 0; k < nd; ++k) {
                const uint64_t dk = a.tgt_dn[(uint64_t)k * Dd + d];
                const T v = a.val_dn[(uint64_t)k * Dd + d];
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const T xv = SMEM ? s_x[dk * R + r] : (r < nr ? x[ur[r] * Dd + dk] : T(0));
                    acc[r] += v * xv;
                }
            }
            // spin-up hops: rows x[u', :] read at column d (coalesced across the CTA)
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int nu = s_nup[r];
                for (int k = 0; k < nu; ++k) acc[r] += s_uval[r * zr + k] * x[(uint64_t)s_ucol[r * zr + k] * Dd + d];
            }
#pragma unroll
            for (int r = 0; r < R; ++r)
                if (r < nr) y[ur[r] * Dd + d] = acc[r];
        }
    }
}

size_t hv_smem_bytes(int R, int zmax, size_t tsize, uint64_t Dd, bool smem_rows) {
    const int zr = zmax > 0 ? zmax : 1;
    size_t off = ((size_t)R * zr * sizeof(uint32_t) + 15) & ~(size_t)15;
    off = (off + (size_t)R * zr * tsize + 15) & ~(size_t)15;
    off = (off + R * sizeof(int) + 15) & ~(size_t)15;
    if (smem_rows) off += (size_t)R * Dd * tsize;
    return off;
}

template <int R, typename T, bool SMEM>
hb_status launch_hv(hb_handle h, const HvArgs<T> &a, const T *x, T *y, cudaStream_t st, size_t smem) {
    auto kern = k_hv<R, T, SMEM>;
    PD_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int threads = 1024;
    if (a.Dd < 1024) threads = (int)std::max<uint64_t>(64, (a.Dd + 31) / 32 * 32);
    int per_sm = 0;
    PD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem));
    if (per_sm < 1) return HB_ERR_NO_MEMORY;
    const uint64_t ngroups = (a.Du + R - 1) / R;
    const uint64_t grid = std::min<uint64_t>(ngroups, (uint64_t)per_sm * h->sm_count);
    kern<<<(unsigned)grid, threads, smem, st>>>(a, x, y);
    PD_CUDA(cudaGetLastError());
    return HB_OK;
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
    a.order = h->d_row_order;
    int max_smem = 0;
    PD_CUDA(cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device));
    const size_t budget = (size_t)max_smem;
    // widest row group whose staged rows fit the shared-memory budget
    if (hv_smem_bytes(4, a.zmax_up, sizeof(T), a.Dd, true) <= budget)
        return launch_hv<4, T, true>(h, a, x, y, st, hv_smem_bytes(4, a.zmax_up, sizeof(T), a.Dd, true));
    if (hv_smem_bytes(2, a.zmax_up, sizeof(T), a.Dd, true) <= budget)
        return launch_hv<2, T, true>(h, a, x, y, st, hv_smem_bytes(2, a.zmax_up, sizeof(T), a.Dd, true));
    if (hv_smem_bytes(1, a.zmax_up, sizeof(T), a.Dd, true) <= budget)
        return launch_hv<1, T, true>(h, a, x, y, st, hv_smem_bytes(1, a.zmax_up, sizeof(T), a.Dd, true));
    return launch_hv<1, T, false>(h, a, x, y, st, hv_smem_bytes(1, a.zmax_up, sizeof(T), a.Dd, false));
}

// ---------------------------------------------------------------------------
// Fixed-point H·v (HB_FX64).  Hops are grouped per spin string into segments
// of equal amplitude class c and fermion sign; the kernel adds the raw 64-bit
// integers of each segment (exact), then applies each class's amplitude -t_c
// once per element: y = U docc x + sum_c (-t_c) (P_c - N_c), each product
// rounded once.  The float64 pipe is never used.
struct FxArgs {
    uint64_t Du, Dd;
    const uint32_t *str_up, *str_dn;
    const uint64_t *seg_up, *seg_dn;
    const uint32_t *ft_up, *ft_dn;
    const uint32_t *order;
    int zmax_up;
    int64_t Kc[PD_FX_MAXC];
    int Gc[PD_FX_MAXC];
    int64_t Kd[PD_MAXL + 1];
    int Gd[PD_MAXL + 1];
};

template <int R, int NC, bool SMEM>
__global__ void __launch_bounds__(1024) k_hv_fx(const FxArgs a, const int64_t *__restrict__ x,
                                                int64_t *__restrict__ y) {
    extern __shared__ __align__(16) unsigned char smem[];
    const uint64_t Dd = a.Dd;
    const int zr = a.zmax_up > 0 ? a.zmax_up : 1;
    // shared layout: [diag K (33 i64)][diag G (33 int)][up seg R u64][up targets R*zr u32][x rows R*Dd i64]
    int64_t *s_kd = reinterpret_cast<int64_t *>(smem);
    int *s_gd = reinterpret_cast<int *>(smem + 8 * (PD_MAXL + 1));
    size_t off = (8 * (PD_MAXL + 1) + 4 * (PD_MAXL + 1) + 15) & ~(size_t)15;
    uint64_t *s_useg = reinterpret_cast<uint64_t *>(smem + off);
    off = (off + 8 * R + 15) & ~(size_t)15;
    uint32_t *s_ucol = reinterpret_cast<uint32_t *>(smem + off);
    off = (off + (size_t)R * zr * 4 + 15) & ~(size_t)15;
    int64_t *s_x = reinterpret_cast<int64_t *>(smem + off);
    for (int k = threadIdx.x; k <= PD_MAXL; k += blockDim.x) {
        s_kd[k] = a.Kd[k];
        s_gd[k] = a.Gd[k];
    }

    const uint64_t ngroups = (a.Du + R - 1) / R;
    for (uint64_t g = blockIdx.x; g < ngroups; g += gridDim.x) {
        const uint64_t p0 = g * R;
        const uint64_t left = a.Du - p0;
        const int nr = left < (uint64_t)R ? (int)left : R;
        uint64_t ur[R];
#pragma unroll
        for (int r = 0; r < R; ++r) ur[r] = r < nr ? (a.order ? (uint64_t)a.order[p0 + r] : p0 + r) : 0;
        __syncthreads();
        if (threadIdx.x < R) s_useg[threadIdx.x] = threadIdx.x < nr ? a.seg_up[ur[threadIdx.x]] : 0ull;
        for (int e = threadIdx.x; e < R * zr; e += blockDim.x) {
            const int r = e / zr, k = e - r * zr;
            if (r < nr && k < a.zmax_up) {
                const uint64_t u = a.order ? (uint64_t)a.order[p0 + r] : p0 + r;
                s_ucol[e] = a.ft_up[(uint64_t)k * a.Du + u];
            }
        }
        if (SMEM) {
#pragma unroll
            for (int r = 0; r < R; ++r) {
                if (r >= nr) break;
                const int64_t *xr = x + ur[r] * Dd;
                for (uint64_t d = threadIdx.x; d < Dd; d += blockDim.x) s_x[d * R + r] = xr[d];
            }
        }
        __syncthreads();
        uint32_t su[R];
#pragma unroll
        for (int r = 0; r < R; ++r) su[r] = r < nr ? a.str_up[ur[r]] : 0u;

        for (uint64_t d = threadIdx.x; d < Dd; d += blockDim.x) {
            int64_t acc[R][2 * NC];
#pragma unroll
            for (int r = 0; r < R; ++r)
#pragma unroll
                for (int q = 0; q < 2 * NC; ++q) acc[r][q] = 0;
            // spin-down hops of column d: gathers within the staged rows
            const uint64_t sg = a.seg_dn[d];
            uint64_t k = 0;
#pragma unroll
            for (int q = 0; q < 2 * NC; ++q) {
                const int n = (int)((sg >> (8 * q)) & 0xFFu);
                for (int i = 0; i < n; ++i, ++k) {
                    const uint64_t dk = a.ft_dn[k * Dd + d];
#pragma unroll
                    for (int r = 0; r < R; ++r)
                        acc[r][q] += SMEM ? s_x[dk * R + r] : (r < nr ? x[ur[r] * Dd + dk] : 0);
                }
            }
            // spin-up hops of row ur[r]: rows x[u', :] at column d
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const uint64_t ug = s_useg[r];
                int kk = 0;
#pragma unroll
                for (int q = 0; q < 2 * NC; ++q) {
                    const int n = (int)((ug >> (8 * q)) & 0xFFu);
                    for (int i = 0; i < n; ++i, ++kk) acc[r][q] += x[(uint64_t)s_ucol[r * zr + kk] * Dd + d];
                }
            }
            const uint32_t sd = a.str_dn[d];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                if (r >= nr) continue;
                const int docc = __popc(su[r] & sd);
                const int64_t xd = SMEM ? s_x[d * R + r] : x[ur[r] * Dd + d];
                int64_t out = fx_mul(xd, s_kd[docc], s_gd[docc]);
#pragma unroll
                for (int c = 0; c < NC; ++c) out += fx_mul(acc[r][2 * c] - acc[r][2 * c + 1], a.Kc[c], a.Gc[c]);
                y[ur[r] * Dd + d] = out;
            }
        }
    }
}

size_t hv_fx_smem_bytes(int R, int zmax, uint64_t Dd, bool rows = true) {
    const int zr = zmax > 0 ? zmax : 1;
    size_t off = (8 * (PD_MAXL + 1) + 4 * (PD_MAXL + 1) + 15) & ~(size_t)15;
    off = (off + 8 * R + 15) & ~(size_t)15;
    off = (off + (size_t)R * zr * 4 + 15) & ~(size_t)15;
    return off + (rows ? (size_t)R * Dd * 8 : 0);
}

template <int R, int NC, bool SMEM>
hb_status launch_hv_fx(hb_handle h, const FxArgs &a, const int64_t *x, int64_t *y, cudaStream_t st) {
    auto kern = k_hv_fx<R, NC, SMEM>;
    const size_t smem = hv_fx_smem_bytes(R, a.zmax_up, a.Dd, SMEM);
    PD_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int threads = 1024;
    if (a.Dd < 1024) threads = (int)std::max<uint64_t>(64, (a.Dd + 31) / 32 * 32);
    int per_sm = 0;
    PD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem));
    if (per_sm < 1) return HB_ERR_NO_MEMORY;
    const uint64_t ngroups = (a.Du + R - 1) / R;
    const uint64_t grid = std::min<uint64_t>(ngroups, (uint64_t)per_sm * h->sm_count);
    kern<<<(unsigned)grid, threads, smem, st>>>(a, x, y);
    PD_CUDA(cudaGetLastError());
    return HB_OK;
}

template <int NC>
hb_status apply_fx_nc(hb_handle h, const FxArgs &a, const int64_t *x, int64_t *y, cudaStream_t st, size_t budget) {
    if (hv_fx_smem_bytes(2, a.zmax_up, a.Dd) <= budget) return launch_hv_fx<2, NC, true>(h, a, x, y, st);
    if (hv_fx_smem_bytes(1, a.zmax_up, a.Dd) <= budget) return launch_hv_fx<1, NC, true>(h, a, x, y, st);
    return launch_hv_fx<1, NC, false>(h, a, x, y, st);  // rows too long for shared memory: gather from L2
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
    a.order = h->d_row_order;
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
        case 1: return apply_fx_nc<1>(h, a, x, y, st, budget);
        case 2: return apply_fx_nc<2>(h, a, x, y, st, budget);
        case 3: return apply_fx_nc<3>(h, a, x, y, st, budget);
        default: return apply_fx_nc<4>(h, a, x, y, st, budget);
    }
}

}  // namespace

hb_status pd_apply(hb_handle h, hb_dtype dt, const void *x, void *y, cudaStream_t st) {
    if (dt == HB_F64) return apply_t<double>(h, static_cast<const double *>(x), static_cast<double *>(y), st);
    if (dt == HB_FX64) return apply_fx(h, static_cast<const int64_t *>(x), static_cast<int64_t *>(y), st);
    return apply_t<float>(h, static_cast<const float *>(x), static_cast<float *>(y), st);
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

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
        const uint64_t u0 = g * R;
        const uint64_t left = a.Du - u0;
        const int nr = left < (uint64_t)R ? (int)left : R;
        __syncthreads();  // previous group finished with shared memory
        if (threadIdx.x < R) s_nup[threadIdx.x] = threadIdx.x < nr ? a.cnt_up[u0 + threadIdx.x] : 0;
        for (int e = threadIdx.x; e < R * zr; e += blockDim.x) {
            const int r = e / zr, k = e - r * zr;
            if (r < nr && k < a.zmax_up) {
                s_ucol[e] = a.tgt_up[(uint64_t)k * a.Du + u0 + r];
                s_uval[e] = a.val_up[(uint64_t)k * a.Du + u0 + r];
            }
        }
        if (SMEM) {
            for (int r = 0; r < nr; ++r) {
                const T *xr = x + (u0 + r) * Dd;
                for (uint64_t d = threadIdx.x; d < Dd; d += blockDim.x) s_x[d * R + r] = xr[d];
            }
        }
        __syncthreads();
        uint32_t su[R];
#pragma unroll
        for (int r = 0; r < R; ++r) su[r] = r < nr ? a.str_up[u0 + r] : 0u;

        for (uint64_t d = threadIdx.x; d < Dd; d += blockDim.x) {
            const uint32_t sd = a.str_dn[d];
            T acc[R];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const T xv = SMEM ? s_x[d * R + r] : (r < nr ? x[(u0 + r) * Dd + d] : T(0));
                acc[r] = a.U * (T)__popc(su[r] & sd) * xv;
            }
            // spin-down hops: gather within the staged rows
            const int nd = a.cnt_dn[d];
            for (int k = 0; k < nd; ++k) {
                const uint64_t dk = a.tgt_dn[(uint64_t)k * Dd + d];
                const T v = a.val_dn[(uint64_t)k * Dd + d];
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const T xv = SMEM ? s_x[dk * R + r] : (r < nr ? x[(u0 + r) * Dd + dk] : T(0));
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
                if (r < nr) y[(u0 + r) * Dd + d] = acc[r];
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

}  // namespace

hb_status pd_apply(hb_handle h, hb_dtype dt, const void *x, void *y, cudaStream_t st) {
    if (dt == HB_F64) return apply_t<double>(h, static_cast<const double *>(x), static_cast<double *>(y), st);
    return apply_t<float>(h, static_cast<const float *>(x), static_cast<float *>(y), st);
}

extern "C" hb_status hubbard_apply(hb_handle h, hb_dtype dt, const void *x, void *y, void *stream) {
    if (!h || !x || !y || (dt != HB_F64 && dt != HB_F32)) return HB_ERR_INVALID_ARG;
    const size_t es = dt == HB_F64 ? 8 : 4;
    const uintptr_t xb = (uintptr_t)x, yb = (uintptr_t)y, n = (uintptr_t)(h->D * es);
    if (xb < yb + n && yb < xb + n) return HB_ERR_INVALID_ARG;  // overlapping vectors
    hb_status s = pd_build_tables(h);
    if (s != HB_OK) return s;
    return pd_apply(h, dt, x, y, reinterpret_cast<cudaStream_t>(stream));
}

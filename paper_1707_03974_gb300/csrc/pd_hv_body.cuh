// Per-row-group bodies of the matrix-free H·v (Eq. 1), shared by the single
// problem kernels (pd_hv.cu) and the batched kernels (pd_batch.cu).
//
// With x viewed as the row-major D_up x D_dn matrix X of the combined index
// (Sec. III), every spin-up hop changes only the row and every spin-down hop
// only the column (the other species adds no fermion sign), so
//     y[u, d] = U popcount(s_u & s_d) x[u, d]                     (Sec. II B)
//             + sum_{u' in hops(u)} h_up(u, u') x[u', d]
//             + sum_{d' in hops(d)} h_dn(d, d') x[u, d'].
// A row group is R rows of X; the CTA stages them in shared memory
// (interleaved x_s[d * R + r]) so that the spin-down gathers hit shared
// memory, while the spin-up terms read whole rows x[u', :] coalesced.
#pragma once

#include "pd_common.cuh"

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

// Shared memory of a float group: [up row offsets R*zmax u64][up vals R*zmax T][up counts R int][x rows R*Dd T]
__host__ __device__ inline size_t hv_smem_bytes(int R, int zmax, size_t tsize, uint64_t Dd, bool smem_rows) {
    const int zr = zmax > 0 ? zmax : 1;
    size_t off = ((size_t)R * zr * sizeof(uint64_t) + 15) & ~(size_t)15;
    off = (off + (size_t)R * zr * tsize + 15) & ~(size_t)15;
    off = (off + R * sizeof(int) + 15) & ~(size_t)15;
    if (smem_rows) off += (size_t)R * Dd * tsize;
    return off;
}

// y rows of group g (positions g*R .. g*R+R-1 of the visiting order).
template <int R, typename T, bool SMEM>
__device__ __forceinline__ void hv_group(const HvArgs<T> &a, const T *__restrict__ x, T *__restrict__ y, uint64_t g,
                                         unsigned char *smem) {
    const uint64_t Dd = a.Dd;
    uint64_t *s_uoff = reinterpret_cast<uint64_t *>(smem);  // spin-up hop rows as element offsets u' * D_dn
    const int zr = a.zmax_up > 0 ? a.zmax_up : 1;
    size_t off = ((size_t)R * zr * sizeof(uint64_t) + 15) & ~(size_t)15;
    T *s_uval = reinterpret_cast<T *>(smem + off);
    off = (off + (size_t)R * zr * sizeof(T) + 15) & ~(size_t)15;
    int *s_nup = reinterpret_cast<int *>(smem + off);
    off = (off + R * sizeof(int) + 15) & ~(size_t)15;
    T *s_x = reinterpret_cast<T *>(smem + off);

    const uint64_t p0 = g * R;
    const uint64_t left = a.Du - p0;
    const int nr = left < (uint64_t)R ? (int)left : R;
    uint64_t ur[R];  // the rows of this group
#pragma unroll
    for (int r = 0; r < R; ++r) ur[r] = r < nr ? (a.order ? (uint64_t)a.order[p0 + r] : p0 + r) : 0;
    __syncthreads();  // the previous group is done with shared memory
    if (threadIdx.x < R) s_nup[threadIdx.x] = threadIdx.x < nr ? a.cnt_up[ur[threadIdx.x]] : 0;
    for (int e = threadIdx.x; e < R * zr; e += blockDim.x) {
        const int r = e / zr, k = e - r * zr;
        if (r < nr && k < a.zmax_up) {
            const uint64_t u = a.order ? (uint64_t)a.order[p0 + r] : p0 + r;
            s_uoff[e] = (uint64_t)a.tgt_up[(uint64_t)k * a.Du + u] * Dd;
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
        // spin-down hops: gather within the staged rows (table loads issued in batches of 4)
        const int nd = a.cnt_dn[d];
        for (int k0 = 0; k0 < nd; k0 += 4) {
            uint32_t tk[4];
            T vk[4];
#pragma unroll
            for (int i = 0; i < 4; ++i)
                if (k0 + i < nd) {
                    tk[i] = a.tgt_dn[(uint64_t)(k0 + i) * Dd + d];
                    vk[i] = a.val_dn[(uint64_t)(k0 + i) * Dd + d];
                }
#pragma unroll
            for (int i = 0; i < 4; ++i)
                if (k0 + i < nd) {
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        const T xv = SMEM ? s_x[(uint64_t)tk[i] * R + r] : (r < nr ? x[ur[r] * Dd + tk[i]] : T(0));
                        acc[r] += vk[i] * xv;
                    }
                }
        }
        // spin-up hops: rows x[u', :] read at column d (coalesced across the CTA), 8 loads in flight
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int nu = s_nup[r];
            for (int k0 = 0; k0 < nu; k0 += 8) {
                T xv[8];
#pragma unroll
                for (int i = 0; i < 8; ++i)
                    xv[i] = (k0 + i < nu) ? x[s_uoff[r * zr + k0 + i] + d] : T(0);
#pragma unroll
                for (int i = 0; i < 8; ++i)
                    if (k0 + i < nu) acc[r] += s_uval[r * zr + k0 + i] * xv[i];
            }
        }
#pragma unroll
        for (int r = 0; r < R; ++r)
            if (r < nr) y[ur[r] * Dd + d] = acc[r];
    }
}

// ---------------------------------------------------------------------------
// Fixed-point (HB_FX64) group.  Hops come in segments of equal amplitude class
// c and fermion sign; the group forms the exact integer sums P_c (positive
// sign) and N_c (negative sign) of the 64-bit elements, then applies each
// class's amplitude -t_c once per element:
//     y = U docc x + sum_c (-t_c) (P_c - N_c),
// each product rounded once.  The float64 pipe is never used.  The spin-up
// hop list is the same for the whole CTA: its row offsets u' * D_dn are staged
// in shared memory once per group.
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

// Shared memory: [diag K (33 i64)][diag G (33 int)][up seg R u64][up row offsets R*zr u64][x rows R*Dd i64]
__host__ __device__ inline size_t hv_fx_smem_bytes(int R, int zmax, uint64_t Dd, bool rows = true) {
    const int zr = zmax > 0 ? zmax : 1;
    size_t off = (8 * (PD_MAXL + 1) + 4 * (PD_MAXL + 1) + 15) & ~(size_t)15;
    off = (off + 8 * R + 15) & ~(size_t)15;
    off = (off + (size_t)R * zr * 8 + 15) & ~(size_t)15;
    return off + (rows ? (size_t)R * Dd * 8 : 0);
}

// Loads the diagonal multipliers of a into the head of shared memory (call
// once per CTA before hv_fx_group, followed by a barrier inside the group).
__device__ __forceinline__ void hv_fx_load_diag(const FxArgs &a, unsigned char *smem) {
    int64_t *s_kd = reinterpret_cast<int64_t *>(smem);
    int *s_gd = reinterpret_cast<int *>(smem + 8 * (PD_MAXL + 1));
    for (int k = threadIdx.x; k <= PD_MAXL; k += blockDim.x) {
        s_kd[k] = a.Kd[k];
        s_gd[k] = a.Gd[k];
    }
}

template <int R, int NC, bool SMEM>
__device__ __forceinline__ void hv_fx_group(const FxArgs &a, const int64_t *__restrict__ x, int64_t *__restrict__ y,
                                            uint64_t g, unsigned char *smem) {
    const uint64_t Dd = a.Dd;
    const int zr = a.zmax_up > 0 ? a.zmax_up : 1;
    const int64_t *s_kd = reinterpret_cast<const int64_t *>(smem);
    const int *s_gd = reinterpret_cast<const int *>(smem + 8 * (PD_MAXL + 1));
    size_t off = (8 * (PD_MAXL + 1) + 4 * (PD_MAXL + 1) + 15) & ~(size_t)15;
    uint64_t *s_useg = reinterpret_cast<uint64_t *>(smem + off);
    off = (off + 8 * R + 15) & ~(size_t)15;
    uint64_t *s_uoff = reinterpret_cast<uint64_t *>(smem + off);
    off = (off + (size_t)R * zr * 8 + 15) & ~(size_t)15;
    int64_t *s_x = reinterpret_cast<int64_t *>(smem + off);

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
            s_uoff[e] = (uint64_t)a.ft_up[(uint64_t)k * a.Du + u] * Dd;
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
        // spin-down hops of column d: gathers within the staged rows, table loads in batches of 4
        const uint64_t sg = a.seg_dn[d];
        uint64_t k = 0;
#pragma unroll
        for (int q = 0; q < 2 * NC; ++q) {
            const int n = (int)((sg >> (8 * q)) & 0xFFu);
            for (int i0 = 0; i0 < n; i0 += 4) {
                uint32_t e[4];
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    if (i0 + i < n) e[i] = a.ft_dn[(k + i0 + i) * Dd + d];
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    if (i0 + i < n) {
#pragma unroll
                        for (int r = 0; r < R; ++r)
                            acc[r][q] += SMEM ? s_x[(uint64_t)e[i] * R + r] : (r < nr ? x[ur[r] * Dd + e[i]] : 0);
                    }
            }
            k += n;
        }
        // spin-up hops of row ur[r] (the same list for the whole CTA): 8 loads in flight
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const uint64_t ug = s_useg[r];
            const uint64_t *uo = s_uoff + r * zr;
            int kk = 0;
#pragma unroll
            for (int q = 0; q < 2 * NC; ++q) {
                const int n = (int)((ug >> (8 * q)) & 0xFFu);
                for (int i0 = 0; i0 < n; i0 += 8) {
                    int64_t xv[8];
#pragma unroll
                    for (int i = 0; i < 8; ++i) xv[i] = (i0 + i < n) ? x[uo[kk + i0 + i] + d] : 0;
#pragma unroll
                    for (int i = 0; i < 8; ++i) acc[r][q] += xv[i];
                }
                kk += n;
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

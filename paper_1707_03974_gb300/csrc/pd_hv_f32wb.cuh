// Float32 row pass of the split H·v on the warp-blocked spin-down table (the
// table of hv_fx_wb_group in pd_hv_body.cuh).
#pragma once

#include "pd_hv_body.cuh"

// y[u, d] = U docc x + sum_c (-t_c)(P_c - N_c), where
// P_c and N_c are float32 sums over the (class, sign) segments of the column's
// hops.  The hops of a segment are added in the table's slot order, so this
// form rounds differently from the one-kernel form (val * x hop by hop); the
// two agree to float32 rounding.  Reading 2-byte targets instead of a 4-byte
// target and a 4-byte value per hop is what it gains when few rows fit in
// shared memory.
struct FWbArgs {
    uint64_t Du, Dd;
    float U;
    const uint32_t *str_up;
    const uint32_t *order;
    float tc[PD_FX_MAXC];  // -t_c of amplitude class c
    const uint32_t *wb_perm, *wb_str, *wb_base, *wb_ent;
    const uint64_t *wb_caps;
    uint32_t wb_nblk;
};

__host__ __device__ inline size_t hv_f_wb_smem_bytes(int R, uint64_t Dd) { return (size_t)R * (Dd + 8) * 4; }

// the R staged values of column t (one 4-, 8- or 16-byte shared load)
template <int R>
__device__ __forceinline__ void f_wb_load(const float *s_x, uint32_t t, float (&v)[R]) {
    if constexpr (R == 4) {
        const float4 q = *reinterpret_cast<const float4 *>(s_x + (size_t)t * 4);
        v[0] = q.x, v[1] = q.y, v[2] = q.z, v[3] = q.w;
    } else if constexpr (R == 2) {
        const float2 q = *reinterpret_cast<const float2 *>(s_x + (size_t)t * 2);
        v[0] = q.x, v[1] = q.y;
    } else {
        v[0] = s_x[t];
    }
}

template <int R, int NC>
__device__ __forceinline__ void hv_f_wb_group(const FWbArgs &a, const float *__restrict__ x, float *__restrict__ y,
                                              uint64_t g, unsigned char *smem) {
    const uint64_t Dd = a.Dd;
    float *s_x = reinterpret_cast<float *>(smem);
    const uint64_t p0 = g * R;
    const uint64_t left = a.Du - p0;
    const int nr = left < (uint64_t)R ? (int)left : R;
    uint64_t ur[R];
#pragma unroll
    for (int r = 0; r < R; ++r) ur[r] = r < nr ? (a.order ? (uint64_t)a.order[p0 + r] : p0 + r) : 0;
    __syncthreads();  // the previous group is done with shared memory
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const float *xr = x + ur[r] * Dd;
        for (uint64_t d = threadIdx.x; d < Dd; d += blockDim.x) s_x[d * R + r] = r < nr ? xr[d] : 0.0f;
    }
    if (threadIdx.x < 8 * R) s_x[Dd * R + threadIdx.x] = 0.0f;
    __syncthreads();
    uint32_t su[R];
#pragma unroll
    for (int r = 0; r < R; ++r) su[r] = r < nr ? a.str_up[ur[r]] : 0u;
    const int lane = threadIdx.x & 31;
    for (uint32_t b = threadIdx.x >> 5; b < a.wb_nblk; b += blockDim.x >> 5) {
        const uint64_t caps = a.wb_caps[b];
        const uint32_t *ent = a.wb_ent + (uint64_t)a.wb_base[b] * 32 + lane;
        float acc[R][2 * NC];
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
            for (int q = 0; q < 2 * NC; ++q) acc[r][q] = 0.0f;
#pragma unroll
        for (int q = 0; q < 2 * NC; ++q) {
            const int np = (int)((caps >> (8 * q)) & 0xFFu);
            int s = 0;
            for (; s + 4 <= np; s += 4) {
                uint32_t e[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) e[i] = ent[(s + i) * 32];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    float v0[R], v1[R];
                    f_wb_load<R>(s_x, e[i] & 0xFFFFu, v0);
                    f_wb_load<R>(s_x, e[i] >> 16, v1);
#pragma unroll
                    for (int r = 0; r < R; ++r) acc[r][q] += v0[r] + v1[r];
                }
            }
            for (; s < np; ++s) {
                const uint32_t ev = ent[s * 32];
                float v0[R], v1[R];
                f_wb_load<R>(s_x, ev & 0xFFFFu, v0);
                f_wb_load<R>(s_x, ev >> 16, v1);
#pragma unroll
                for (int r = 0; r < R; ++r) acc[r][q] += v0[r] + v1[r];
            }
            ent += np * 32;
        }
        const uint32_t p = b * 32 + lane;
        const uint32_t col = a.wb_perm[p];
        if (col < Dd) {
            const uint32_t sd = a.wb_str[p];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                if (r >= nr) continue;
                float out = a.U * (float)__popc(su[r] & sd) * s_x[(uint64_t)col * R + r];
#pragma unroll
                for (int c = 0; c < NC; ++c) out += a.tc[c] * (acc[r][2 * c] - acc[r][2 * c + 1]);
                y[ur[r] * Dd + col] = out;
            }
        }
    }
}

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
    stage_rows_async<float, R>(s_x, x, ur, nr, Dd);
    if (threadIdx.x < 8 * R) s_x[Dd * R + threadIdx.x] = 0.0f;
    __syncthreads();
    uint32_t su[R];
#pragma unroll
    for (int r = 0; r < R; ++r) su[r] = r < nr ? a.str_up[ur[r]] : 0u;
    const int lane = threadIdx.x & 31;
    // With one staged row (one CTA per SM) a warp runs four warp blocks side by side,
    // so that four times as many table loads are in flight; a block with fewer slot
    // pairs in a segment reads the zero element s_x[D_dn] (adding +0).
    constexpr int PB = R == 1 ? 4 : 1;
    const uint32_t nw = blockDim.x >> 5;
    const uint32_t zpair = (uint32_t)Dd | ((uint32_t)Dd << 16);
    for (uint32_t b0 = (threadIdx.x >> 5) * PB; b0 < a.wb_nblk; b0 += nw * PB) {
        uint64_t caps[PB];
        const uint32_t *ent[PB];
#pragma unroll
        for (int j = 0; j < PB; ++j) {
            const bool ok = b0 + j < a.wb_nblk;
            caps[j] = ok ? a.wb_caps[b0 + j] : 0ull;
            ent[j] = a.wb_ent + (ok ? (uint64_t)a.wb_base[b0 + j] * 32 : 0ull) + lane;
        }
        float acc[PB][R][2 * NC];
#pragma unroll
        for (int j = 0; j < PB; ++j)
#pragma unroll
            for (int r = 0; r < R; ++r)
#pragma unroll
                for (int q = 0; q < 2 * NC; ++q) acc[j][r][q] = 0.0f;
#pragma unroll
        for (int q = 0; q < 2 * NC; ++q) {
            int np[PB], npm = 0;
#pragma unroll
            for (int j = 0; j < PB; ++j) {
                np[j] = (int)((caps[j] >> (8 * q)) & 0xFFu);
                npm = np[j] > npm ? np[j] : npm;
            }
            int s = 0;
            for (; s + 4 <= npm; s += 4) {
                uint32_t e[PB][4];
#pragma unroll
                for (int j = 0; j < PB; ++j)
#pragma unroll
                    for (int i = 0; i < 4; ++i) e[j][i] = s + i < np[j] ? ent[j][(s + i) * 32] : zpair;
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < PB; ++j) {
                        float v0[R], v1[R];
                        f_wb_load<R>(s_x, e[j][i] & 0xFFFFu, v0);
                        f_wb_load<R>(s_x, e[j][i] >> 16, v1);
#pragma unroll
                        for (int r = 0; r < R; ++r) acc[j][r][q] += v0[r] + v1[r];
                    }
            }
            for (; s < npm; ++s)
#pragma unroll
                for (int j = 0; j < PB; ++j) {
                    const uint32_t ev = s < np[j] ? ent[j][s * 32] : zpair;
                    float v0[R], v1[R];
                    f_wb_load<R>(s_x, ev & 0xFFFFu, v0);
                    f_wb_load<R>(s_x, ev >> 16, v1);
#pragma unroll
                    for (int r = 0; r < R; ++r) acc[j][r][q] += v0[r] + v1[r];
                }
#pragma unroll
            for (int j = 0; j < PB; ++j) ent[j] += np[j] * 32;
        }
#pragma unroll
        for (int j = 0; j < PB; ++j) {
            if (b0 + j >= a.wb_nblk) break;
            const uint32_t p = (b0 + j) * 32 + lane;
            const uint32_t col = a.wb_perm[p];
            if (col >= Dd) continue;
            const uint32_t sd = a.wb_str[p];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                if (r >= nr) continue;
                float out = a.U * (float)__popc(su[r] & sd) * s_x[(uint64_t)col * R + r];
#pragma unroll
                for (int c = 0; c < NC; ++c) out += a.tc[c] * (acc[j][r][2 * c] - acc[j][r][2 * c + 1]);
                y[ur[r] * Dd + col] = out;
            }
        }
    }
}

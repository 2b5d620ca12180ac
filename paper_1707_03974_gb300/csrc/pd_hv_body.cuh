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

#include <type_traits>

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

// Staging of R rows of x into shared memory, interleaved s_x[d * R + r]: every
// element is an asynchronous global -> shared copy (cp.async, 4 or 8 bytes), so
// a thread has all its copies in flight at once and waits once, instead of one
// global-load round trip per element.  Rows r >= nr are filled with zeros.
template <typename T, int R>
__device__ __forceinline__ void stage_rows_async(T *s_x, const T *__restrict__ x, const uint64_t (&ur)[R], int nr,
                                                 uint64_t Dd) {
    static_assert(sizeof(T) == 4 || sizeof(T) == 8, "4- or 8-byte elements");
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const T *xr = x + ur[r] * Dd;
        for (uint64_t d = threadIdx.x; d < Dd; d += blockDim.x) {
            T *dst = s_x + d * R + r;
            if (r < nr) {
                const unsigned sa = (unsigned)__cvta_generic_to_shared(dst);
                if constexpr (sizeof(T) == 8)
                    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(xr + d) : "memory");
                else
                    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(xr + d) : "memory");
            } else {
                *dst = T(0);
            }
        }
    }
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

// Shared memory of a float group: [up row offsets R*zmax u64][up vals R*zmax T][up counts R int][x rows R*Dd T]
__host__ __device__ inline size_t hv_smem_bytes(int R, int zmax, size_t tsize, uint64_t Dd, bool smem_rows) {
    const int zr = zmax > 0 ? zmax : 1;
    size_t off = ((size_t)R * zr * sizeof(uint64_t) + 15) & ~(size_t)15;
    off = (off + (size_t)R * zr * tsize + 15) & ~(size_t)15;
    off = (off + R * sizeof(int) + 15) & ~(size_t)15;
    if (smem_rows) off += (size_t)R * Dd * tsize;
    return off;
}

// y rows of group g (positions g*R .. g*R+R-1 of the visiting order).  The
// diagonal and spin-down terms are summed first and the spin-up terms in a
// separate accumulator, y = (diag + down) + up, so that the split form (this
// body with DO_A = false followed by hv_up_item) gives bit-identical results.
// Epi: optional store hook (the batched Lanczos step fuses its first vector pass
// here); with the default (void) every output is stored to y.
template <int R, typename T, bool SMEM, bool DO_A = true, class Epi = void>
__device__ __forceinline__ void hv_group(const HvArgs<T> &a, const T *__restrict__ x, T *__restrict__ y, uint64_t g,
                                         unsigned char *smem, Epi *epi = nullptr) {
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
    if (DO_A) {
        if (threadIdx.x < R) s_nup[threadIdx.x] = threadIdx.x < nr ? a.cnt_up[ur[threadIdx.x]] : 0;
        for (int e = threadIdx.x; e < R * zr; e += blockDim.x) {
            const int r = e / zr, k = e - r * zr;
            if (r < nr && k < a.zmax_up) {
                const uint64_t u = a.order ? (uint64_t)a.order[p0 + r] : p0 + r;
                s_uoff[e] = (uint64_t)a.tgt_up[(uint64_t)k * a.Du + u] * Dd;
                s_uval[e] = a.val_up[(uint64_t)k * a.Du + u];
            }
        }
    }
    if (SMEM) stage_rows_async<T, R>(s_x, x, ur, nr, Dd);
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
        if (DO_A) {
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int nu = s_nup[r];
                T accu = T(0);
                for (int k0 = 0; k0 < nu; k0 += 8) {
                    T xv[8];
#pragma unroll
                    for (int i = 0; i < 8; ++i)
                        xv[i] = (k0 + i < nu) ? x[s_uoff[r * zr + k0 + i] + d] : T(0);
#pragma unroll
                    for (int i = 0; i < 8; ++i)
                        if (k0 + i < nu) accu += s_uval[r * zr + k0 + i] * xv[i];
                }
                acc[r] += accu;
            }
        }
#pragma unroll
        for (int r = 0; r < R; ++r)
            if (r < nr) {
                if constexpr (std::is_void<Epi>::value) {
                    y[ur[r] * Dd + d] = acc[r];
                } else {
                    const T xv = SMEM ? s_x[d * R + r] : x[ur[r] * Dd + d];
                    epi->store(ur[r] * Dd + d, acc[r], xv);
                }
            }
    }
}

// ---------------------------------------------------------------------------
// Fixed-point (HB_FX64) group.  Hops come in segments of equal amplitude class
// c and fermion sign; the group forms the exact integer sums P_c (positive
// sign) and N_c (negative sign) of the 64-bit elements, separately for the
// spin-down and the spin-up hops, then applies each class's amplitude -t_c
// once per element and spin:
//     y = [U docc x] + sum_c [(-t_c) (P_c - N_c)]_down + sum_c [(-t_c) (P_c - N_c)]_up,
// each bracket one rounded 64 x 64 -> 128-bit product; the outer sum is exact,
// so any split of the terms over kernels gives the same bits.  The float64 pipe is never used.  The spin-up
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
    // warp-blocked spin-down table (row pass of the split form; see SpinTables)
    const uint32_t *wb_perm = nullptr, *wb_str = nullptr, *wb_base = nullptr, *wb_ent = nullptr;
    const uint64_t *wb_caps = nullptr;
    uint32_t wb_nblk = 0;
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

template <int R, int NC, bool SMEM, bool DO_A = true, class Epi = void>
__device__ __forceinline__ void hv_fx_group(const FxArgs &a, const int64_t *__restrict__ x, int64_t *__restrict__ y,
                                            uint64_t g, unsigned char *smem, Epi *epi = nullptr) {
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
    if (DO_A) {
        if (threadIdx.x < R) s_useg[threadIdx.x] = threadIdx.x < nr ? a.seg_up[ur[threadIdx.x]] : 0ull;
        for (int e = threadIdx.x; e < R * zr; e += blockDim.x) {
            const int r = e / zr, k = e - r * zr;
            if (r < nr && k < a.zmax_up) {
                const uint64_t u = a.order ? (uint64_t)a.order[p0 + r] : p0 + r;
                s_uoff[e] = (uint64_t)a.ft_up[(uint64_t)k * a.Du + u] * Dd;
            }
        }
    }
    if (SMEM) stage_rows_async<int64_t, R>(s_x, x, ur, nr, Dd);
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
        const uint32_t sd = a.str_dn[d];
        int64_t out[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int docc = __popc(su[r] & sd);
            const int64_t xd = SMEM ? s_x[d * R + r] : (r < nr ? x[ur[r] * Dd + d] : 0);
            out[r] = fx_mul(xd, s_kd[docc], s_gd[docc]);
#pragma unroll
            for (int c = 0; c < NC; ++c) out[r] += fx_mul(acc[r][2 * c] - acc[r][2 * c + 1], a.Kc[c], a.Gc[c]);
        }
        // spin-up hops of row ur[r] (the same list for the whole CTA): 8 loads in flight,
        // summed in the accumulators the spin-down terms have released
        if (DO_A) {
#pragma unroll
            for (int r = 0; r < R; ++r) {
#pragma unroll
                for (int q = 0; q < 2 * NC; ++q) acc[r][q] = 0;
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
#pragma unroll
                for (int c = 0; c < NC; ++c) out[r] += fx_mul(acc[r][2 * c] - acc[r][2 * c + 1], a.Kc[c], a.Gc[c]);
            }
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if (r >= nr) continue;
            if constexpr (std::is_void<Epi>::value) {
                y[ur[r] * Dd + d] = out[r];
            } else {
                const int64_t xd = SMEM ? s_x[d * R + r] : x[ur[r] * Dd + d];
                epi->store(ur[r] * Dd + d, out[r], xd);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Spin-up pass of the split H·v (the row pass above with DO_A = false has
// written y = diag + down):  y[u, d] += sum_{u' in hops(u)} h_up(u, u') x[u', d].
// Work item (j, g) covers columns j*W .. j*W+W-1 and rows g*RA .. g*RA+RA-1;
// items are handed out column-block-major, so the CTAs in flight all read the
// same D_up x W panel of x, which stays in L2 while the block lasts.  Thread
// (c, s) of a CTA of W * S threads takes column j*W + c and rows
// g*RA + s + i*S (i < RR, RA = S * RR).

// Row offsets u' * D_dn are staged as 32-bit element offsets when D < 2^32
// (IDX32), else as 64-bit ones; in the float pass each row's list starts on a
// 16-byte boundary so that groups of offsets load as vectors.  Lists (and
// fixed-point segments) run to their exact length: full batches of 8 loads,
// then 4, 2 and 1 (uniform branches, no idle slots).

// Staged row stride (elements) for hop lists of at most zmax entries in at
// most nseg segments, each segment start rounded up to a multiple of 4.
__host__ __device__ inline int up_row_stride(int zmax, int nseg) {
    const int z = (zmax > 0 ? zmax : 1) + 3 * nseg;
    return (z + 3) & ~3;
}
__host__ __device__ inline int up_pow2(int z) {
    int p = 1;
    while (p < z) p <<= 1;
    return p;
}

template <bool IDX32>
__host__ __device__ inline size_t hv_up_smem_bytes(int RA, int zmax, size_t tsize) {
    const int zs = up_row_stride(zmax, 1);
    size_t off = ((size_t)RA * zs * (IDX32 ? 4 : 8) + 15) & ~(size_t)15;
    off = (off + (size_t)RA * zs * tsize + 15) & ~(size_t)15;
    return off + (size_t)RA * 4;
}

// B offsets starting at uo[k] (k a multiple of min(B, 4)), as one or more vector loads
template <typename OFF, int B>
__device__ __forceinline__ void load_offsets(const OFF *uo, int k, OFF *o) {
    if constexpr (sizeof(OFF) == 4 && B >= 4) {
#pragma unroll
        for (int v = 0; v < B / 4; ++v) {
            const uint4 q = *reinterpret_cast<const uint4 *>(uo + k + 4 * v);
            o[4 * v] = q.x, o[4 * v + 1] = q.y, o[4 * v + 2] = q.z, o[4 * v + 3] = q.w;
        }
    } else if constexpr (sizeof(OFF) == 4 && B == 2) {
        const uint2 q = *reinterpret_cast<const uint2 *>(uo + k);
        o[0] = q.x, o[1] = q.y;
    } else {
#pragma unroll
        for (int i = 0; i < B; ++i) o[i] = uo[k + i];
    }
}

// V adjacent elements loaded or stored as one vector (V * sizeof(T) bytes, aligned).
template <typename T, int V>
struct alignas(sizeof(T) * V) Pack {
    T v[V];
};

// acc[v] += sum_{i < B} coefficient(k + i) * x[off(k + i) + d + v] in the order i = 0 .. B-1
template <typename T, typename OFF, int B, int V>
__device__ __forceinline__ void up_batch_f(const T *__restrict__ x, const OFF *uo, const T *uv, int k, OFF d,
                                           T *acc) {
    OFF o[B];
    load_offsets<OFF, B>(uo, k, o);
    Pack<T, V> xv[B];
#pragma unroll
    for (int i = 0; i < B; ++i) xv[i] = *reinterpret_cast<const Pack<T, V> *>(x + (o[i] + d));
#pragma unroll
    for (int i = 0; i < B; ++i)
#pragma unroll
        for (int v = 0; v < V; ++v) acc[v] += uv[k + i] * xv[i].v[v];
}

// Persistent walk over the items (j, g), column-block-major, without a division per item.
struct ItemWalk {
    uint64_t j, g, n_groups;
    __device__ ItemWalk(uint64_t n_groups_) : n_groups(n_groups_) {
        j = blockIdx.x / n_groups;
        g = blockIdx.x - j * n_groups;
    }
    __device__ void next() {
        g += gridDim.x;
        while (g >= n_groups) g -= n_groups, ++j;
    }
};

// Thread (c, s) takes columns (j W + c) V .. (j W + c) V + V - 1; with V = 2 the
// caller guarantees D_dn even and 2-element-aligned vectors, so pairs never
// straddle a row end.
template <int RR, typename T, bool IDX32, int V>
__device__ __forceinline__ void hv_up_item(const HvArgs<T> &a, const T *__restrict__ x, T *__restrict__ y,
                                           uint64_t j, uint64_t g, int W, int S, unsigned char *smem) {
    using OFF = typename std::conditional<IDX32, uint32_t, uint64_t>::type;
    constexpr int B0 = 8 / V;  // loads in flight per batch
    const uint64_t Dd = a.Dd;
    const int RA = S * RR;
    const int zs = up_row_stride(a.zmax_up, 1), zp = up_pow2(a.zmax_up > 0 ? a.zmax_up : 1), lz = __ffs(zp) - 1;
    OFF *s_uoff = reinterpret_cast<OFF *>(smem);
    size_t off = ((size_t)RA * zs * sizeof(OFF) + 15) & ~(size_t)15;
    T *s_uval = reinterpret_cast<T *>(smem + off);
    off = (off + (size_t)RA * zs * sizeof(T) + 15) & ~(size_t)15;
    int *s_nup = reinterpret_cast<int *>(smem + off);
    const uint64_t p0 = g * (uint64_t)RA;
    __syncthreads();  // the previous item is done with shared memory
    for (int e = threadIdx.x; e < RA * zp; e += blockDim.x) {
        const int r = e >> lz, k = e & (zp - 1);
        const uint64_t u = p0 + r;
        if (u < a.Du && k < a.zmax_up) {
            s_uoff[r * zs + k] = (OFF)((uint64_t)a.tgt_up[(uint64_t)k * a.Du + u] * Dd);
            s_uval[r * zs + k] = a.val_up[(uint64_t)k * a.Du + u];
        }
    }
    for (int r = threadIdx.x; r < RA; r += blockDim.x) s_nup[r] = p0 + r < a.Du ? (int)a.cnt_up[p0 + r] : 0;
    __syncthreads();
    const int c = threadIdx.x % W, sl = threadIdx.x / W;
    const uint64_t d = (j * (uint64_t)W + c) * V;
    if (d >= Dd || sl >= S) return;
#pragma unroll 1
    for (int i = 0; i < RR; ++i) {
        const int r = sl + i * S;
        const uint64_t u = p0 + r;
        if (u >= a.Du) break;
        const int nu = s_nup[r];
        const OFF *uo = s_uoff + r * zs;
        const T *uv = s_uval + r * zs;
        T accu[V];
#pragma unroll
        for (int v = 0; v < V; ++v) accu[v] = T(0);
        int k = 0;
        for (; k + B0 <= nu; k += B0) up_batch_f<T, OFF, B0, V>(x, uo, uv, k, (OFF)d, accu);
        if constexpr (B0 >= 8)
            if (nu - k >= 4) up_batch_f<T, OFF, 4, V>(x, uo, uv, k, (OFF)d, accu), k += 4;
        if constexpr (B0 >= 4)
            if (nu - k >= 2) up_batch_f<T, OFF, 2, V>(x, uo, uv, k, (OFF)d, accu), k += 2;
        if constexpr (B0 >= 2)
            if (nu - k >= 1) up_batch_f<T, OFF, 1, V>(x, uo, uv, k, (OFF)d, accu);
        Pack<T, V> *yp = reinterpret_cast<Pack<T, V> *>(y + u * Dd + d);
        Pack<T, V> yv = *yp;
#pragma unroll
        for (int v = 0; v < V; ++v) yv.v[v] = yv.v[v] + accu[v];
        *yp = yv;
    }
}

template <bool IDX32>
__host__ __device__ inline size_t hv_fx_up_smem_bytes(int RA, int zmax) {
    const int zr = zmax > 0 ? zmax : 1;
    return (((size_t)RA * 8 + 15) & ~(size_t)15) + (size_t)RA * zr * (IDX32 ? 4 : 8);
}

// exact integer sums acc[v] += x[off(k + i) + d + v], i < B (offsets loaded one
// by one: segment starts are not aligned in the fixed-point lists)
template <typename OFF, int B, int V>
__device__ __forceinline__ void up_batch_fx(const int64_t *__restrict__ x, const OFF *uo, int k, OFF d,
                                            int64_t *acc) {
    Pack<int64_t, V> xv[B];
#pragma unroll
    for (int i = 0; i < B; ++i) xv[i] = *reinterpret_cast<const Pack<int64_t, V> *>(x + (uo[k + i] + d));
#pragma unroll
    for (int i = 0; i < B; ++i)
#pragma unroll
        for (int v = 0; v < V; ++v) acc[v] += xv[i].v[v];
}

// one segment [k, kend) of a row's list: full batches, then the remainder by halves
template <typename OFF, int V>
__device__ __forceinline__ void up_segment_fx(const int64_t *__restrict__ x, const OFF *uo, int &k, int kend, OFF d,
                                              int64_t *acc) {
    constexpr int B0 = 8 / V;
    for (; k + B0 <= kend; k += B0) up_batch_fx<OFF, B0, V>(x, uo, k, d, acc);
    if constexpr (B0 >= 8)
        if (kend - k >= 4) up_batch_fx<OFF, 4, V>(x, uo, k, d, acc), k += 4;
    if constexpr (B0 >= 4)
        if (kend - k >= 2) up_batch_fx<OFF, 2, V>(x, uo, k, d, acc), k += 2;
    if constexpr (B0 >= 2)
        if (kend - k >= 1) up_batch_fx<OFF, 1, V>(x, uo, k, d, acc), k += 1;
}

// Epi: optional hook for the final value y_row + up of each element (the batched
// Lanczos step fuses its first vector pass there); with the default (void) the
// sum is stored back to y.
template <int RR, int NC, bool IDX32, int V, class Epi = void>
__device__ __forceinline__ void hv_fx_up_item(const FxArgs &a, const int64_t *__restrict__ x,
                                              int64_t *__restrict__ y, uint64_t j, uint64_t g, int W, int S,
                                              unsigned char *smem, Epi *epi = nullptr) {
    using OFF = typename std::conditional<IDX32, uint32_t, uint64_t>::type;
    const uint64_t Dd = a.Dd;
    const int RA = S * RR;
    const int zr = a.zmax_up > 0 ? a.zmax_up : 1, zp = up_pow2(zr), lz = __ffs(zp) - 1;
    uint64_t *s_useg = reinterpret_cast<uint64_t *>(smem);
    OFF *s_uoff = reinterpret_cast<OFF *>(smem + (((size_t)RA * 8 + 15) & ~(size_t)15));
    const uint64_t p0 = g * (uint64_t)RA;
    __syncthreads();
    for (int r = threadIdx.x; r < RA; r += blockDim.x) s_useg[r] = p0 + r < a.Du ? a.seg_up[p0 + r] : 0ull;
    for (int e = threadIdx.x; e < RA * zp; e += blockDim.x) {
        const int r = e >> lz, k = e & (zp - 1);
        const uint64_t u = p0 + r;
        if (u < a.Du && k < a.zmax_up) s_uoff[r * zr + k] = (OFF)((uint64_t)a.ft_up[(uint64_t)k * a.Du + u] * Dd);
    }
    __syncthreads();
    const int c = threadIdx.x % W, sl = threadIdx.x / W;
    const uint64_t d = (j * (uint64_t)W + c) * V;
    if (d >= Dd || sl >= S) return;
#pragma unroll 1
    for (int i = 0; i < RR; ++i) {
        const int r = sl + i * S;
        const uint64_t u = p0 + r;
        if (u >= a.Du) break;
        const uint64_t ug = s_useg[r];
        const OFF *uo = s_uoff + r * zr;
        int k = 0;
        uint64_t add[V];
#pragma unroll
        for (int v = 0; v < V; ++v) add[v] = 0;
#pragma unroll
        for (int cc = 0; cc < NC; ++cc) {
            int64_t pos[V], neg[V];
#pragma unroll
            for (int v = 0; v < V; ++v) pos[v] = neg[v] = 0;
            up_segment_fx<OFF, V>(x, uo, k, k + (int)((ug >> (16 * cc)) & 0xFFu), (OFF)d, pos);
            up_segment_fx<OFF, V>(x, uo, k, k + (int)((ug >> (16 * cc + 8)) & 0xFFu), (OFF)d, neg);
#pragma unroll
            for (int v = 0; v < V; ++v) add[v] += (uint64_t)fx_mul(pos[v] - neg[v], a.Kc[cc], a.Gc[cc]);
        }
        Pack<int64_t, V> *yp = reinterpret_cast<Pack<int64_t, V> *>(y + u * Dd + d);
        Pack<int64_t, V> yv = *yp;
#pragma unroll
        for (int v = 0; v < V; ++v) yv.v[v] = (int64_t)((uint64_t)yv.v[v] + add[v]);
        if constexpr (std::is_void<Epi>::value) {
            *yp = yv;
        } else {
#pragma unroll
            for (int v = 0; v < V; ++v) epi->store(u * Dd + d + v, yv.v[v], x[u * Dd + d + v]);
        }
    }
}

// ---------------------------------------------------------------------------
// Row pass of the split fixed-point H·v on the warp-blocked spin-down table:
// y[u, d] = [U docc x] + sum_c [(-t_c)(P_c - N_c)]_down for the R rows of group g.
// Warp w takes blocks of 32 positions; lane l of block b handles the string at
// position 32 b + l, whose column in x is wb_perm[32 b + l].  All lanes of a
// block run the same number of slot pairs per segment (empty slots point at
// one of the zero elements s_x[(D_dn + z) * R + r], z < 8), so the loop has
// no divergence.
__host__ __device__ inline size_t hv_fx_wb_smem_bytes(int R, uint64_t Dd) {
    const size_t off = (8 * (PD_MAXL + 1) + 4 * (PD_MAXL + 1) + 15) & ~(size_t)15;
    return off + (size_t)R * (Dd + 8) * 8;
}

template <int R, int NC>
__device__ __forceinline__ void hv_fx_wb_group(const FxArgs &a, const int64_t *__restrict__ x,
                                               int64_t *__restrict__ y, uint64_t g, unsigned char *smem) {
    const uint64_t Dd = a.Dd;
    const int64_t *s_kd = reinterpret_cast<const int64_t *>(smem);
    const int *s_gd = reinterpret_cast<const int *>(smem + 8 * (PD_MAXL + 1));
    int64_t *s_x = reinterpret_cast<int64_t *>(smem + ((8 * (PD_MAXL + 1) + 4 * (PD_MAXL + 1) + 15) & ~(size_t)15));
    const uint64_t p0 = g * R;
    const uint64_t left = a.Du - p0;
    const int nr = left < (uint64_t)R ? (int)left : R;
    uint64_t ur[R];
#pragma unroll
    for (int r = 0; r < R; ++r) ur[r] = r < nr ? (a.order ? (uint64_t)a.order[p0 + r] : p0 + r) : 0;
    __syncthreads();
    stage_rows_async<int64_t, R>(s_x, x, ur, nr, Dd);
    if (threadIdx.x < 8 * R) s_x[Dd * R + threadIdx.x] = 0;
    __syncthreads();
    uint32_t su[R];
#pragma unroll
    for (int r = 0; r < R; ++r) su[r] = r < nr ? a.str_up[ur[r]] : 0u;
    const int lane = threadIdx.x & 31;
    for (uint32_t b = threadIdx.x >> 5; b < a.wb_nblk; b += blockDim.x >> 5) {
        const uint64_t caps = a.wb_caps[b];
        const uint32_t *ent = a.wb_ent + (uint64_t)a.wb_base[b] * 32 + lane;
        int64_t acc[R][2 * NC];
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
            for (int q = 0; q < 2 * NC; ++q) acc[r][q] = 0;
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
                    const uint32_t t0 = e[i] & 0xFFFFu, t1 = e[i] >> 16;
#pragma unroll
                    for (int r = 0; r < R; ++r) acc[r][q] += s_x[t0 * R + r] + s_x[t1 * R + r];
                }
            }
            for (; s < np; ++s) {
                const uint32_t ev = ent[s * 32];
                const uint32_t t0 = ev & 0xFFFFu, t1 = ev >> 16;
#pragma unroll
                for (int r = 0; r < R; ++r) acc[r][q] += s_x[t0 * R + r] + s_x[t1 * R + r];
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
                const int docc = __popc(su[r] & sd);
                int64_t out = fx_mul(s_x[(uint64_t)col * R + r], s_kd[docc], s_gd[docc]);
#pragma unroll
                for (int c = 0; c < NC; ++c) out += fx_mul(acc[r][2 * c] - acc[r][2 * c + 1], a.Kc[c], a.Gc[c]);
                y[ur[r] * Dd + col] = out;
            }
        }
    }
}

// Basis handle, Paradeisos rank/unrank kernels, per-spin hop tables and the
// verification row export.
//
// Paper: Sec. II A (occupation strings, tensor-product basis), Eq. 3 and the
// forward-map procedure (rank), the backward-map procedure (unrank), Sec. III
// (combined index I = C(L, N_dn) idx_up + idx_dn), Sec. II B (hops and the
// fermion sign, double occupancy by AND).
#include <algorithm>
#include <functional>
#include <cmath>
#include <cstring>
#include <new>
#include <set>
#include <utility>
#include <vector>

#include "pd_common.cuh"
#include "pd_divmagic.h"
#include "pd_wb_sched.h"

namespace {

constexpr int kThreads = 256;

// Binomial table by Pascal's rule, C(i, m) = C(i-1, m) + C(i-1, m-1), with
// C(i, 0) = 1 and C(i, m) = 0 for m > i (the convention stated with Eq. 2).
void host_binomials(std::vector<uint32_t> &lut) {
    lut.assign(PD_LUT_W * PD_LUT_W, 0u);
    for (int i = 0; i <= PD_MAXL; ++i) {
        lut[i * PD_LUT_W + 0] = 1u;
        for (int m = 1; m <= i; ++m) {
            uint64_t v = (uint64_t)lut[(i - 1) * PD_LUT_W + m] + lut[(i - 1) * PD_LUT_W + m - 1];
            lut[i * PD_LUT_W + m] = (uint32_t)v;  // max C(32,16) = 601080390 < 2^32
        }
    }
}

__device__ __forceinline__ void load_lut(uint32_t *s_lut, const uint32_t *g_lut) {
    for (int k = threadIdx.x; k < PD_LUT_W * PD_LUT_W; k += blockDim.x) s_lut[k] = g_lut[k];
    __syncthreads();
}

__global__ void k_rank(const uint32_t *__restrict__ g_lut, const uint64_t *__restrict__ states,
                       uint64_t *__restrict__ idx, uint64_t n, int L, int N_up, int N_dn, uint64_t D_dn,
                       unsigned *err) {
    __shared__ uint32_t lut[PD_LUT_W * PD_LUT_W];
    load_lut(lut, g_lut);
    const uint64_t lmask = (L == 32) ? 0xFFFFFFFFull : ((1ull << L) - 1ull);
    for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < n; e += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t s = states[e];
        const uint64_t up = (L == 32) ? (s >> 32) : (s >> L);
        const uint64_t dn = s & lmask;
        const bool ok = (up & ~lmask) == 0 && __popcll(up) == N_up && __popcll(dn) == N_dn;
        if (!ok) {
            idx[e] = PD_INVALID;
            atomicOr(err, PD_ERRBIT(HB_ERR_INVALID_STATE));
            continue;
        }
        const uint64_t iu = pd_forward_map(lut, (uint32_t)up);
        const uint64_t id = pd_forward_map(lut, (uint32_t)dn);
        idx[e] = iu * D_dn + id;
    }
}

__global__ void k_unrank(const uint32_t *__restrict__ g_lut, const uint64_t *__restrict__ idx,
                         uint64_t *__restrict__ states, uint64_t n, int L, int N_up, int N_dn, uint64_t D_dn,
                         DivMagic by_dn, uint64_t D, unsigned *err) {
    __shared__ uint32_t lut[PD_LUT_W * PD_LUT_W];
    load_lut(lut, g_lut);
    for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < n; e += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t I = idx[e];
        if (I >= D) {
            states[e] = PD_INVALID;
            atomicOr(err, PD_ERRBIT(HB_ERR_OUT_OF_RANGE));
            continue;
        }
        const uint64_t iu = divmagic_q(I, by_dn);  // I / D_dn
        const uint64_t id = I - iu * D_dn;
        const uint64_t up = pd_backward_map(lut, (uint32_t)iu, N_up, L);
        const uint64_t dn = pd_backward_map(lut, (uint32_t)id, N_dn, L);
        states[e] = (up << L) | dn;
    }
}

// Per-spin strings by the backward map, and the number of hops of each string.
__global__ void k_spin_strings(const uint32_t *__restrict__ g_lut, uint32_t *__restrict__ str,
                               uint16_t *__restrict__ count, uint64_t D, int n, int L,
                               const int32_t *__restrict__ bonds, int n_bonds, int *zmax) {
    __shared__ uint32_t lut[PD_LUT_W * PD_LUT_W];
    load_lut(lut, g_lut);
    int local_max = 0;
    for (uint64_t r = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; r < D; r += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t s = pd_backward_map(lut, (uint32_t)r, n, L);
        str[r] = s;
        int c = 0;
        for (int b = 0; b < n_bonds; ++b) {
            const uint32_t bi = (s >> bonds[2 * b]) & 1u, bj = (s >> bonds[2 * b + 1]) & 1u;
            c += (bi != bj);
        }
        count[r] = (uint16_t)c;
        local_max = max(local_max, c);
    }
    atomicMax(zmax, local_max);
}

// Hop lists: for every string and every bond with exactly one of its two sites
// occupied, the string after the hop, its per-spin index (forward map), and
// the matrix element -t_b * (-1)^(particles strictly between the two sites).
__global__ void k_spin_hops(const uint32_t *__restrict__ g_lut, const uint32_t *__restrict__ str, uint64_t D,
                            const int32_t *__restrict__ bonds, const double *__restrict__ t, int n_bonds,
                            uint32_t *__restrict__ target, double *__restrict__ val, float *__restrict__ valf) {
    __shared__ uint32_t lut[PD_LUT_W * PD_LUT_W];
    load_lut(lut, g_lut);
    for (uint64_t r = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; r < D; r += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t s = str[r];
        int k = 0;
        for (int b = 0; b < n_bonds; ++b) {
            const int i = bonds[2 * b], j = bonds[2 * b + 1];
            if (((s >> i) & 1u) == ((s >> j) & 1u)) continue;
            const uint32_t s2 = s ^ ((1u << i) | (1u << j));
            const int lo = min(i, j), hi = max(i, j);
            const uint32_t between = ((hi >= 32 ? 0u : (1u << hi)) - 1u) & ~((2u << lo) - 1u);
            const bool neg = (__popc(s & between) & 1) != 0;
            const double v = neg ? t[b] : -t[b];
            target[(uint64_t)k * D + r] = pd_forward_map(lut, s2);
            val[(uint64_t)k * D + r] = v;
            valf[(uint64_t)k * D + r] = (float)v;
            ++k;
        }
    }
}

// The same hops re-ordered for the fixed-point path: segments of equal
// (amplitude class, fermion sign), class-major, positive sign first; seg[r]
// packs the 2*PD_FX_MAXC segment lengths as bytes (byte 2c: class c positive,
// byte 2c+1: class c negative).  The H·v then adds plain 64-bit integers per
// segment and applies each class's amplitude once per element.
__global__ void k_spin_hops_fx(const uint32_t *__restrict__ g_lut, const uint32_t *__restrict__ str, uint64_t D,
                               const int32_t *__restrict__ bonds, const int32_t *__restrict__ bond_class,
                               int n_bonds, uint32_t *__restrict__ ftarget, uint64_t *__restrict__ seg) {
    __shared__ uint32_t lut[PD_LUT_W * PD_LUT_W];
    load_lut(lut, g_lut);
    for (uint64_t r = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; r < D; r += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t s = str[r];
        int cnt[2 * PD_FX_MAXC] = {0, 0, 0, 0, 0, 0, 0, 0};
        for (int b = 0; b < n_bonds; ++b) {
            const int i = bonds[2 * b], j = bonds[2 * b + 1];
            if (((s >> i) & 1u) == ((s >> j) & 1u)) continue;
            const int lo = min(i, j), hi = max(i, j);
            const uint32_t between = ((1u << hi) - 1u) & ~((2u << lo) - 1u);
            ++cnt[2 * bond_class[b] + (__popc(s & between) & 1)];
        }
        int off[2 * PD_FX_MAXC];
        uint64_t packed = 0;
        int acc = 0;
        for (int q = 0; q < 2 * PD_FX_MAXC; ++q) {
            off[q] = acc;
            acc += cnt[q];
            packed |= (uint64_t)cnt[q] << (8 * q);
        }
        seg[r] = packed;
        for (int b = 0; b < n_bonds; ++b) {
            const int i = bonds[2 * b], j = bonds[2 * b + 1];
            if (((s >> i) & 1u) == ((s >> j) & 1u)) continue;
            const int lo = min(i, j), hi = max(i, j);
            const uint32_t between = ((1u << hi) - 1u) & ~((2u << lo) - 1u);
            const int q = 2 * bond_class[b] + (__popc(s & between) & 1);
            ftarget[(uint64_t)(off[q]++) * D + r] = pd_forward_map(lut, s ^ ((1u << i) | (1u << j)));
        }
    }
}

__global__ void k_f64_to_fx(const double *__restrict__ x, int64_t *__restrict__ y, uint64_t n, int F) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        y[i] = __double2ll_rn(ldexp(x[i], F));
}

__global__ void k_fx_to_f64(const int64_t *__restrict__ x, double *__restrict__ y, uint64_t n, int F) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        y[i] = ldexp((double)x[i], -F);
}

// One thread per exported row: diagonal, spin-up hops (u' , d), spin-down hops
// (u, d'), sorted by column (insertion sort; rows hold at most 1 + 2 n_bonds).
__global__ void k_row_entries(uint64_t row0, uint32_t nrows, uint32_t max_entries, double U, uint64_t D_dn,
                              const uint32_t *__restrict__ str_up, const uint16_t *__restrict__ cnt_up,
                              const uint32_t *__restrict__ tgt_up, const double *__restrict__ val_up, uint64_t D_up,
                              const uint32_t *__restrict__ str_dn, const uint16_t *__restrict__ cnt_dn,
                              const uint32_t *__restrict__ tgt_dn, const double *__restrict__ val_dn,
                              uint64_t *__restrict__ cols, double *__restrict__ vals, uint32_t *__restrict__ counts,
                              unsigned *err) {
    const uint32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nrows) return;
    const uint64_t I = row0 + r;
    const uint64_t u = I / D_dn, d = I - u * D_dn;
    const uint32_t nu = cnt_up[u], nd = cnt_dn[d];
    const uint32_t total = 1 + nu + nd;
    if (total > max_entries) {
        counts[r] = 0xFFFFFFFFu;
        atomicOr(err, PD_ERRBIT(HB_ERR_INVALID_ARG));
        return;
    }
    uint64_t *c = cols + (uint64_t)r * max_entries;
    double *v = vals + (uint64_t)r * max_entries;
    uint32_t m = 0;
    c[m] = I;
    v[m] = U * (double)__popc(str_up[u] & str_dn[d]);
    ++m;
    for (uint32_t k = 0; k < nu; ++k, ++m) {
        c[m] = (uint64_t)tgt_up[(uint64_t)k * D_up + u] * D_dn + d;
        v[m] = val_up[(uint64_t)k * D_up + u];
    }
    for (uint32_t k = 0; k < nd; ++k, ++m) {
        c[m] = u * D_dn + tgt_dn[(uint64_t)k * D_dn + d];
        v[m] = val_dn[(uint64_t)k * D_dn + d];
    }
    for (uint32_t a = 1; a < m; ++a) {
        const uint64_t kc = c[a];
        const double kv = v[a];
        int b = (int)a - 1;
        while (b >= 0 && c[b] > kc) {
            c[b + 1] = c[b];
            v[b + 1] = v[b];
            --b;
        }
        c[b + 1] = kc;
        v[b + 1] = kv;
    }
    counts[r] = m;
}

int grid_for(uint64_t n, int sm_count) {
    uint64_t g = (n + kThreads - 1) / kThreads;
    const uint64_t cap = (uint64_t)sm_count * 8;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (int)g;
}

uint64_t binom64(int n, int k) {
    if (k < 0 || k > n) return 0;
    uint64_t r = 1;
    for (int i = 1; i <= k; ++i) r = r * (uint64_t)(n - k + i) / (uint64_t)i;  // exact at every step
    return r;
}

void free_spin(SpinTables &s) {
    cudaFree(s.str);
    cudaFree(s.count);
    cudaFree(s.target);
    cudaFree(s.val);
    cudaFree(s.valf);
    cudaFree(s.ftarget);
    cudaFree(s.seg);
    cudaFree(s.wb_perm);
    cudaFree(s.wb_str);
    cudaFree(s.wb_base);
    cudaFree(s.wb_ent);
    cudaFree(s.wb_caps);
    s = SpinTables();
}

// Warp-blocked hop table (see SpinTables): built on the host from the
// segment-ordered fixed-point hop lists.
hb_status build_wb(SpinTables &st, int device) {
    const uint64_t D = st.D;
    if (D == 0 || D + 8 > 65535 || !st.ftarget) return HB_OK;
    const uint32_t kZeroSlot = 0xFFFFu;  // placeholder until the bank group is chosen
    const int z = st.zmax > 0 ? st.zmax : 1;
    std::vector<uint32_t> ft((uint64_t)z * D), str(D);
    std::vector<uint64_t> seg(D);
    PD_CUDA(cudaMemcpy(ft.data(), st.ftarget, ft.size() * 4, cudaMemcpyDeviceToHost));
    PD_CUDA(cudaMemcpy(seg.data(), st.seg, D * 8, cudaMemcpyDeviceToHost));
    PD_CUDA(cudaMemcpy(str.data(), st.str, D * 4, cudaMemcpyDeviceToHost));
    constexpr int NQ = 2 * PD_FX_MAXC;
    auto cnt = [&](uint64_t r, int q) { return (int)((seg[r] >> (8 * q)) & 0xFFu); };
    // bank layout of the row pass that will read this table: two staged 8-byte
    // rows (16-byte gathers) when they fit in the largest shared-memory carve-out,
    // else one staged float32 row (4-byte gathers)
    int max_smem = 0;
    PD_CUDA(cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, device));
    const bool wide = (uint64_t)2 * (D + 8) * 8 + 1024 <= (uint64_t)max_smem;
    const pd_wb::BankLayout bl = wide ? pd_wb::BankLayout{8, 8} : pd_wb::BankLayout{32, 32};
    std::vector<uint32_t> perm(D);
    for (uint64_t r = 0; r < D; ++r) perm[r] = (uint32_t)r;
    std::stable_sort(perm.begin(), perm.end(), [&](uint32_t a, uint32_t b) {
        for (int q = 0; q < NQ; ++q)
            if (cnt(a, q) != cnt(b, q)) return cnt(a, q) < cnt(b, q);
        return false;
    });
    const uint64_t nblk = (D + 31) / 32;
    std::vector<uint32_t> wperm(nblk * 32, (uint32_t)D), wstr(nblk * 32, 0u), base(nblk);
    std::vector<uint64_t> caps(nblk, 0ull);
    std::vector<uint32_t> ent;
    uint64_t rows = 0;
    for (uint64_t b = 0; b < nblk; ++b) {
        int cap[NQ] = {0};
        for (int l = 0; l < 32; ++l) {
            const uint64_t p = b * 32 + l;
            if (p >= D) break;
            wperm[p] = perm[p];
            wstr[p] = str[perm[p]];
            for (int q = 0; q < NQ; ++q) cap[q] = std::max(cap[q], cnt(perm[p], q));
        }
        base[b] = (uint32_t)rows;
        for (int q = 0; q < NQ; ++q) {
            const int pairs = (cap[q] + 1) / 2, slots = 2 * pairs;
            caps[b] |= (uint64_t)pairs << (8 * q);
            // grid[l][s]: target of lane l in slot s (-1: empty)
            std::vector<int32_t> grid((size_t)32 * slots, -1);
            for (int l = 0; l < 32; ++l) {
                const uint64_t p = b * 32 + l;
                if (p >= D) break;
                const uint32_t r = perm[p];
                int k0 = 0;
                for (int qq = 0; qq < q; ++qq) k0 += cnt(r, qq);
                for (int i = 0; i < cnt(r, q); ++i) grid[(size_t)l * slots + i] = (int32_t)ft[(uint64_t)(k0 + i) * D + r];
            }
            pd_wb::balance_banks(grid, slots, bl);
            for (int s = 0; s < pairs; ++s, ++rows)
                for (int l = 0; l < 32; ++l) {
                    uint32_t t[2];
                    for (int h = 0; h < 2; ++h) {
                        const int32_t v = grid[(size_t)l * slots + 2 * s + h];
                        t[h] = v >= 0 ? (uint32_t)v : kZeroSlot;
                    }
                    ent.push_back(t[0] | (t[1] << 16));
                }
        }
    }
    // empty slots read one of the eight zero elements s_x[D .. D+7]: one in a
    // bank group that no real target of the lanes served with it uses
    for (uint64_t b = 0, row = 0; b < nblk; ++b)
        for (int q = 0; q < NQ; ++q)
            for (uint64_t pr = 0; pr < ((caps[b] >> (8 * q)) & 0xFFu); ++pr, ++row)
                for (int h = 0; h < 2; ++h)
                    for (int l0 = 0; l0 < 32; l0 += bl.NL) {
                        bool used[32] = {false};
                        for (int l = l0; l < l0 + bl.NL; ++l) {
                            const uint32_t t = (ent[row * 32 + l] >> (16 * h)) & 0xFFFFu;
                            if (t != kZeroSlot) used[t % bl.G] = true;
                        }
                        int z = 0;
                        while (z < 7 && used[(D + z) % bl.G]) ++z;
                        const uint32_t zt = (uint32_t)D + (uint32_t)z;
                        for (int l = l0; l < l0 + bl.NL; ++l) {
                            uint32_t &e = ent[row * 32 + l];
                            if (((e >> (16 * h)) & 0xFFFFu) == kZeroSlot)
                                e = (e & ~(0xFFFFu << (16 * h))) | (zt << (16 * h));
                        }
                    }
    if (rows >= (1ull << 32) / 32) return HB_OK;
    PD_CUDA(cudaMalloc(&st.wb_perm, wperm.size() * 4));
    PD_CUDA(cudaMalloc(&st.wb_str, wstr.size() * 4));
    PD_CUDA(cudaMalloc(&st.wb_base, base.size() * 4));
    PD_CUDA(cudaMalloc(&st.wb_caps, caps.size() * 8));
    PD_CUDA(cudaMalloc(&st.wb_ent, std::max<size_t>(ent.size(), 1) * 4));
    PD_CUDA(cudaMemcpy(st.wb_perm, wperm.data(), wperm.size() * 4, cudaMemcpyHostToDevice));
    PD_CUDA(cudaMemcpy(st.wb_str, wstr.data(), wstr.size() * 4, cudaMemcpyHostToDevice));
    PD_CUDA(cudaMemcpy(st.wb_base, base.data(), base.size() * 4, cudaMemcpyHostToDevice));
    PD_CUDA(cudaMemcpy(st.wb_caps, caps.data(), caps.size() * 8, cudaMemcpyHostToDevice));
    if (!ent.empty()) PD_CUDA(cudaMemcpy(st.wb_ent, ent.data(), ent.size() * 4, cudaMemcpyHostToDevice));
    st.wb_nblk = (uint32_t)nblk;
    st.wb_ok = true;
    return HB_OK;
}

hb_status build_spin(hb_handle h, SpinTables &st, int n) {
    st.n = n;
    st.D = binom64(h->L, n);
    const uint64_t D = st.D;
    PD_CUDA(cudaMalloc(&st.str, D * sizeof(uint32_t)));
    PD_CUDA(cudaMalloc(&st.count, D * sizeof(uint16_t)));
    int *d_zmax = nullptr;
    PD_CUDA(cudaMalloc(&d_zmax, sizeof(int)));
    PD_CUDA(cudaMemset(d_zmax, 0, sizeof(int)));
    k_spin_strings<<<grid_for(D, h->sm_count), kThreads>>>(h->d_binom, st.str, st.count, D, n, h->L, h->d_bonds,
                                                           h->n_bonds, d_zmax);
    PD_CUDA(cudaGetLastError());
    int zmax = 0;
    PD_CUDA(cudaMemcpy(&zmax, d_zmax, sizeof(int), cudaMemcpyDeviceToHost));
    cudaFree(d_zmax);
    st.zmax = zmax;
    const uint64_t ne = (uint64_t)(zmax > 0 ? zmax : 1) * D;
    if (ne * (sizeof(uint32_t) + sizeof(double) + sizeof(float)) > (16ull << 30)) return HB_ERR_NO_MEMORY;
    if (cudaMalloc(&st.target, ne * sizeof(uint32_t)) != cudaSuccess) return HB_ERR_NO_MEMORY;
    if (cudaMalloc(&st.val, ne * sizeof(double)) != cudaSuccess) return HB_ERR_NO_MEMORY;
    if (cudaMalloc(&st.valf, ne * sizeof(float)) != cudaSuccess) return HB_ERR_NO_MEMORY;
    k_spin_hops<<<grid_for(D, h->sm_count), kThreads>>>(h->d_binom, st.str, D, h->d_bonds, h->d_t, h->n_bonds,
                                                        st.target, st.val, st.valf);
    PD_CUDA(cudaGetLastError());
    if (h->fx_ok) {
        if (cudaMalloc(&st.ftarget, ne * sizeof(uint32_t)) != cudaSuccess) return HB_ERR_NO_MEMORY;
        if (cudaMalloc(&st.seg, D * sizeof(uint64_t)) != cudaSuccess) return HB_ERR_NO_MEMORY;
        k_spin_hops_fx<<<grid_for(D, h->sm_count), kThreads>>>(h->d_binom, st.str, D, h->d_bonds, h->d_bond_class,
                                                               h->n_bonds, st.ftarget, st.seg);
        PD_CUDA(cudaGetLastError());
    }
    PD_CUDA(cudaDeviceSynchronize());
    if (h->fx_ok) return build_wb(st, h->device);
    return HB_OK;
}

cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

// Reverse Cuthill-McKee order of the spin-up hop graph (breadth-first from the
// lowest-degree unvisited string, neighbours in order of increasing degree,
// the whole order reversed).  Only changes the order in which rows are
// visited, never the storage order of vectors.
hb_status build_row_order(hb_handle h) {
    const uint64_t n = h->D_up;
    const int z = h->up.zmax;
    std::vector<uint16_t> cnt(n);
    std::vector<uint32_t> tgt((uint64_t)std::max(z, 1) * n);
    PD_CUDA(cudaMemcpy(cnt.data(), h->up.count, n * sizeof(uint16_t), cudaMemcpyDeviceToHost));
    if (z > 0) PD_CUDA(cudaMemcpy(tgt.data(), h->up.target, (uint64_t)z * n * sizeof(uint32_t), cudaMemcpyDeviceToHost));
    std::vector<uint32_t> by_degree(n);
    for (uint64_t i = 0; i < n; ++i) by_degree[i] = (uint32_t)i;
    std::stable_sort(by_degree.begin(), by_degree.end(), [&](uint32_t a, uint32_t b) { return cnt[a] < cnt[b]; });
    std::vector<uint8_t> seen(n, 0);
    std::vector<uint32_t> order;
    order.reserve(n);
    std::vector<uint32_t> nb;
    for (uint32_t start : by_degree) {
        if (seen[start]) continue;
        seen[start] = 1;
        uint64_t head = order.size();
        order.push_back(start);
        while (head < order.size()) {
            const uint32_t u = order[head++];
            nb.clear();
            for (int k = 0; k < cnt[u]; ++k) {
                const uint32_t v = tgt[(uint64_t)k * n + u];
                if (!seen[v]) {
                    seen[v] = 1;
                    nb.push_back(v);
                }
            }
            std::stable_sort(nb.begin(), nb.end(), [&](uint32_t a, uint32_t b) { return cnt[a] < cnt[b]; });
            order.insert(order.end(), nb.begin(), nb.end());
        }
    }
    std::reverse(order.begin(), order.end());
    if (cudaMalloc(&h->d_row_order, n * sizeof(uint32_t)) != cudaSuccess) return HB_ERR_NO_MEMORY;
    PD_CUDA(cudaMemcpy(h->d_row_order, order.data(), n * sizeof(uint32_t), cudaMemcpyHostToDevice));
    return HB_OK;
}

}  // namespace

static FxCoef fx_coef_host(double c) {
    FxCoef r;
    if (c == 0.0) return r;
    int e = 0;
    std::frexp(c, &e);
    int G = 62 - e;
    G = G < 1 ? 1 : (G > 63 ? 63 : G);
    r.G = G;
    r.K = std::llround(std::ldexp(c, G));
    return r;
}

hb_status pd_fx_coefs(hb_handle h, FxCoef *diag, FxCoef *cls) {
    if (!h->fx_ok) return HB_ERR_INVALID_ARG;
    for (int k = 0; k <= PD_MAXL; ++k) diag[k] = fx_coef_host(h->U * (double)k);
    for (int c = 0; c < PD_FX_MAXC; ++c) cls[c] = fx_coef_host(c < h->n_classes ? -h->class_t[c] : 0.0);
    return HB_OK;
}

void pd_record_error(hb_handle h, hb_status s) {
    unsigned bit = PD_ERRBIT(s);
    unsigned cur = 0;
    cudaMemcpy(&cur, h->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost);
    cur |= bit;
    cudaMemcpy(h->d_err, &cur, sizeof(unsigned), cudaMemcpyHostToDevice);
}

hb_status pd_build_tables(hb_handle h) {
    if (h->tables_built) return HB_OK;
    int dev_now = 0;
    PD_CUDA(cudaGetDevice(&dev_now));
    if (dev_now != h->device) PD_CUDA(cudaSetDevice(h->device));
    hb_status s = build_spin(h, h->up, h->N_up);
    if (s == HB_OK) {
        if (h->N_dn == h->N_up) {
            h->same_spin_tables = true;
            h->dn = h->up;
        } else {
            s = build_spin(h, h->dn, h->N_dn);
        }
    }
    if (s == HB_OK && h->D_up <= (1ull << 26)) s = build_row_order(h);
    if (dev_now != h->device) cudaSetDevice(dev_now);
    if (s != HB_OK) {
        cudaFree(h->d_row_order);
        h->d_row_order = nullptr;
        free_spin(h->up);
        if (!h->same_spin_tables) free_spin(h->dn);
        h->dn = SpinTables();
        h->same_spin_tables = false;
        return s;
    }
    h->tables_built = true;
    return HB_OK;
}

extern "C" {

const char *hb_status_string(hb_status s) {
    switch (s) {
        case HB_OK: return "HB_OK";
        case HB_ERR_INVALID_ARG: return "HB_ERR_INVALID_ARG";
        case HB_ERR_OVERFLOW: return "HB_ERR_OVERFLOW";
        case HB_ERR_INVALID_STATE: return "HB_ERR_INVALID_STATE";
        case HB_ERR_OUT_OF_RANGE: return "HB_ERR_OUT_OF_RANGE";
        case HB_ERR_NO_MEMORY: return "HB_ERR_NO_MEMORY";
        case HB_ERR_CUDA: return "HB_ERR_CUDA";
        case HB_ERR_NOT_CONVERGED: return "HB_ERR_NOT_CONVERGED";
        case HB_ERR_TIMEOUT: return "HB_ERR_TIMEOUT";
    }
    return "HB_UNKNOWN";
}

hb_status hubbard_basis_create(int L, int n_bonds, const int32_t *bonds, const double *t, double U, int N_up,
                               int N_dn, hb_handle *out) {
    if (!out) return HB_ERR_INVALID_ARG;
    *out = nullptr;
    if (L < 1 || L > PD_MAXL || N_up < 0 || N_up > L || N_dn < 0 || N_dn > L || n_bonds < 0) return HB_ERR_INVALID_ARG;
    if (n_bonds > 0 && (!bonds || !t)) return HB_ERR_INVALID_ARG;
    if (n_bonds > L * (L - 1) / 2) return HB_ERR_INVALID_ARG;
    std::set<std::pair<int, int>> seen;
    for (int b = 0; b < n_bonds; ++b) {
        const int i = bonds[2 * b], j = bonds[2 * b + 1];
        if (i < 0 || j < 0 || i >= L || j >= L || i == j) return HB_ERR_INVALID_ARG;
        if (!seen.insert({std::min(i, j), std::max(i, j)}).second) return HB_ERR_INVALID_ARG;
        if (!(t[b] == t[b])) return HB_ERR_INVALID_ARG;  // NaN amplitude
    }
    if (!(U == U)) return HB_ERR_INVALID_ARG;
    const uint64_t Du = binom64(L, N_up), Dd = binom64(L, N_dn);
    if (Du == 0 || Dd == 0) return HB_ERR_INVALID_ARG;
    if (Du > (1ull << 62) / Dd) return HB_ERR_OVERFLOW;

    hb_basis *h = new (std::nothrow) hb_basis();
    if (!h) return HB_ERR_NO_MEMORY;
    h->L = L;
    h->N_up = N_up;
    h->N_dn = N_dn;
    h->n_bonds = n_bonds;
    h->U = U;
    h->D_up = Du;
    h->D_dn = Dd;
    h->D = Du * Dd;
    auto fail = [&](hb_status s) {
        hubbard_basis_destroy(h);
        return s;
    };
    if (cudaGetDevice(&h->device) != cudaSuccess) return fail(HB_ERR_CUDA);
    if (cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess)
        return fail(HB_ERR_CUDA);
    std::vector<uint32_t> lut;
    host_binomials(lut);
    if (cudaMalloc(&h->d_binom, lut.size() * sizeof(uint32_t)) != cudaSuccess) return fail(HB_ERR_CUDA);
    if (cudaMemcpy(h->d_binom, lut.data(), lut.size() * sizeof(uint32_t), cudaMemcpyHostToDevice) != cudaSuccess)
        return fail(HB_ERR_CUDA);
    const int nb = n_bonds > 0 ? n_bonds : 1;
    h->h_bonds = new int32_t[2 * nb]();
    h->h_t = new double[nb]();
    if (n_bonds > 0) {
        std::memcpy(h->h_bonds, bonds, sizeof(int32_t) * 2 * n_bonds);
        std::memcpy(h->h_t, t, sizeof(double) * n_bonds);
    }
    if (cudaMalloc(&h->d_bonds, sizeof(int32_t) * 2 * nb) != cudaSuccess) return fail(HB_ERR_CUDA);
    if (cudaMalloc(&h->d_t, sizeof(double) * nb) != cudaSuccess) return fail(HB_ERR_CUDA);
    if (cudaMemcpy(h->d_bonds, h->h_bonds, sizeof(int32_t) * 2 * nb, cudaMemcpyHostToDevice) != cudaSuccess)
        return fail(HB_ERR_CUDA);
    if (cudaMemcpy(h->d_t, h->h_t, sizeof(double) * nb, cudaMemcpyHostToDevice) != cudaSuccess)
        return fail(HB_ERR_CUDA);
    // fixed-point format: amplitude classes (distinct t values) and fractional bits F
    {
        std::vector<int32_t> cls(nb, 0);
        int nc = 0;
        bool ok = n_bonds <= 255;
        for (int b = 0; b < n_bonds && ok; ++b) {
            int c = 0;
            while (c < nc && h->class_t[c] != t[b]) ++c;
            if (c == nc) {
                if (nc == PD_FX_MAXC) {
                    ok = false;
                    break;
                }
                h->class_t[nc++] = t[b];
            }
            cls[b] = c;
        }
        h->fx_ok = ok;
        h->n_classes = ok ? nc : 0;
        double bound = std::fabs(U) * (double)std::min(N_up, N_dn);
        double tsum = 0.0;
        for (int b = 0; b < n_bonds; ++b) tsum += std::fabs(t[b]);
        bound += 2.0 * tsum;
        int F = 60;
        const double lim1 = 3.0 * std::max(bound, 1.0);      // |w| <= 3 max row sum of |H|
        const double lim2 = 2.0 * n_bonds + 1.0;              // class sums of inputs below 1
        while (F > 8 && (std::ldexp(std::max(lim1, lim2), F) >= std::ldexp(1.0, 62))) --F;
        h->fx_frac = F;
        if (cudaMalloc(&h->d_bond_class, sizeof(int32_t) * nb) != cudaSuccess) return fail(HB_ERR_CUDA);
        if (cudaMemcpy(h->d_bond_class, cls.data(), sizeof(int32_t) * nb, cudaMemcpyHostToDevice) != cudaSuccess)
            return fail(HB_ERR_CUDA);
    }
    if (cudaMalloc(&h->d_err, sizeof(unsigned)) != cudaSuccess) return fail(HB_ERR_CUDA);
    if (cudaMemset(h->d_err, 0, sizeof(unsigned)) != cudaSuccess) return fail(HB_ERR_CUDA);
    *out = h;
    return HB_OK;
}

hb_status hubbard_basis_destroy(hb_handle h) {
    if (!h) return HB_ERR_INVALID_ARG;
    pd_k_free(h->ks);
    free_spin(h->up);
    if (!h->same_spin_tables) free_spin(h->dn);
    cudaFree(h->d_binom);
    cudaFree(h->d_bonds);
    cudaFree(h->d_t);
    cudaFree(h->d_err);
    cudaFree(h->d_bond_class);
    cudaFree(h->d_row_order);
    delete[] h->h_bonds;
    delete[] h->h_t;
    delete h;
    return HB_OK;
}

hb_status hubbard_basis_dim(hb_handle h, uint64_t *D, uint64_t *D_up, uint64_t *D_dn) {
    if (!h) return HB_ERR_INVALID_ARG;
    if (D) *D = h->D;
    if (D_up) *D_up = h->D_up;
    if (D_dn) *D_dn = h->D_dn;
    return HB_OK;
}

hb_status hubbard_fixed_point_bits(hb_handle h, int32_t *F) {
    if (!h || !F) return HB_ERR_INVALID_ARG;
    *F = h->fx_frac;
    return HB_OK;
}

hb_status hubbard_convert(hb_handle h, hb_dtype from, const void *x, hb_dtype to, void *y, uint64_t n, void *stream) {
    if (!h || (n > 0 && (!x || !y))) return HB_ERR_INVALID_ARG;
    if (n == 0) return HB_OK;
    if (from == HB_F64 && to == HB_FX64)
        k_f64_to_fx<<<grid_for(n, h->sm_count), kThreads, 0, as_stream(stream)>>>(
            static_cast<const double *>(x), static_cast<int64_t *>(y), n, h->fx_frac);
    else if (from == HB_FX64 && to == HB_F64)
        k_fx_to_f64<<<grid_for(n, h->sm_count), kThreads, 0, as_stream(stream)>>>(
            static_cast<const int64_t *>(x), static_cast<double *>(y), n, h->fx_frac);
    else
        return HB_ERR_INVALID_ARG;
    PD_CUDA(cudaGetLastError());
    return HB_OK;
}

hb_status hubbard_set_U(hb_handle h, double U) {
    if (!h || !(U == U)) return HB_ERR_INVALID_ARG;
    h->U = U;
    return HB_OK;
}

hb_status paradeisos_rank(hb_handle h, const uint64_t *states, uint64_t *idx, uint64_t n, void *stream) {
    if (!h || (n > 0 && (!states || !idx))) return HB_ERR_INVALID_ARG;
    if (n == 0) return HB_OK;
    if (h->ks) return pd_k_rank(h, states, idx, n, as_stream(stream));
    k_rank<<<grid_for(n, h->sm_count), kThreads, 0, as_stream(stream)>>>(h->d_binom, states, idx, n, h->L, h->N_up,
                                                                         h->N_dn, h->D_dn, h->d_err);
    PD_CUDA(cudaGetLastError());
    return HB_OK;
}

hb_status paradeisos_unrank(hb_handle h, const uint64_t *idx, uint64_t *states, uint64_t n, void *stream) {
    if (!h || (n > 0 && (!states || !idx))) return HB_ERR_INVALID_ARG;
    if (n == 0) return HB_OK;
    if (h->ks) return pd_k_unrank(h, idx, states, n, as_stream(stream));
    k_unrank<<<grid_for(n, h->sm_count), kThreads, 0, as_stream(stream)>>>(h->d_binom, idx, states, n, h->L,
                                                                           h->N_up, h->N_dn, h->D_dn,
                                                                           make_divmagic(h->D_dn), h->D, h->d_err);
    PD_CUDA(cudaGetLastError());
    return HB_OK;
}

hb_status hubbard_row_entries(hb_handle h, uint64_t row0, uint32_t nrows, uint32_t max_entries, uint64_t *cols,
                              double *vals, uint32_t *counts, void *stream) {
    if (!h || (nrows > 0 && (!cols || !vals || !counts)) || max_entries == 0) return HB_ERR_INVALID_ARG;
    if (row0 > h->D || nrows > h->D - row0) return HB_ERR_INVALID_ARG;
    if (nrows == 0) return HB_OK;
    if (h->ks) return pd_k_row_entries(h, row0, nrows, max_entries, cols, vals, counts, as_stream(stream));
    hb_status s = pd_build_tables(h);
    if (s != HB_OK) return s;
    const int blocks = (int)((nrows + 127) / 128);
    k_row_entries<<<blocks, 128, 0, as_stream(stream)>>>(row0, nrows, max_entries, h->U, h->D_dn, h->up.str,
                                                         h->up.count, h->up.target, h->up.val, h->D_up, h->dn.str,
                                                         h->dn.count, h->dn.target, h->dn.val, cols, vals, counts,
                                                         h->d_err);
    PD_CUDA(cudaGetLastError());
    return HB_OK;
}

hb_status hubbard_last_error(hb_handle h) {
    if (!h) return HB_ERR_INVALID_ARG;
    PD_CUDA(cudaDeviceSynchronize());
    unsigned bits = 0;
    PD_CUDA(cudaMemcpy(&bits, h->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost));
    PD_CUDA(cudaMemset(h->d_err, 0, sizeof(unsigned)));
    for (int s = 1; s <= (int)HB_ERR_TIMEOUT; ++s)
        if (bits & PD_ERRBIT(s)) return (hb_status)s;
    return HB_OK;
}

}  // extern "C"

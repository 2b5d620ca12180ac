// Momentum-space Paradeisos (Sec. IV A) and the Hubbard H·v of Eq. 4 in one
// sector of fixed total momentum K.
//
// Bit i of a spin string is the occupation of the single-particle momentum
// k_i = 2 pi (mx / Lx, my / Ly), i = mx + Lx my (Ly = 1: a ring).  Momenta add
// modulo the Brillouin zone, i.e. (mx, my) modulo (Lx, Ly).
//
// Tables (built on the host by the recursion of Sec. IV A, read by the kernels):
//   C_i^m(k)  placements of m particles on bits 0 .. i-1 with total momentum k,
//             C_i^m(k) = C_{i-1}^m(k) + C_{i-1}^{m-1}(k - k_{i-1}), C_0^0(k) = [k = 0];
//   C~_i^m(k) = sum_kd C_i^m(k - kd) C_N^{n_dn}(kd)                      (Eq. 6).
// Forward map of (up, dn): the spin-down map gives (idx_dn, K_dn); then every
// up particle (the m-th at bit i, k accumulated from K_dn) adds C~_i^m(k).  The
// backward maps scan the bits from N-1 down (Sec. IV A).
//
// The sector index splits as J = F(up) + G(dn): F is the up part of the
// forward map (it depends on the up string only, because K_dn = K - K_up) and
// G the spin-down string's index within its own momentum list.  So the sector
// is a set of rows, one per up string (F(up) its first index, C_N^{n_dn}(K -
// K_up) its length), and the interaction of Eq. 4, written as
// (U/N) sum_q rho_up(q) rho_dn(-q) with rho(q) = sum_k c^dag_{k+q} c_k, maps
// state (up, dn) to (up', dn') with up' = up moved by +q (one particle) and
// dn' = dn moved by -q, element (U/N) s_up s_dn (fermion signs as for a
// real-space hop).  Per spin string and q the moves are tabulated once (their
// F(up') or G(dn') and sign, computed by the forward map on the device); the
// H·v then gathers x[F(up') + G(dn')] for every pair of moves.
#include <algorithm>
#include <cmath>
#include <new>
#include <type_traits>
#include <vector>

#include "pd_common.cuh"

struct KSpace {
    int Lx = 0, Ly = 0, N = 0, K = 0, nu = 0, nd = 0;
    double t = 0.0, tp = 0.0;
    uint64_t Dup = 0, Ddn = 0;  // all up / down strings: C(N, n_up), C(N, n_dn)
    std::vector<uint64_t> h_doff;  // first list entry of each down momentum [N + 1]
    std::vector<uint64_t> h_mbase, h_cbase;  // move / count table bases per down momentum
    // device
    uint32_t *Cdn = nullptr;  // [(N+1) (nd+1) N]
    uint64_t *Ct = nullptr;   // [(N+1) (nu+1) N]
    double *eps = nullptr;    // [N]
    uint32_t *ustr = nullptr;  // [Dup] up strings, ascending
    uint64_t *rowF = nullptr;  // [Dup] F(up): first sector index of the row
    uint32_t *rowKd = nullptr;  // [Dup] K_dn = K - K_up of the row
    double *eu = nullptr;       // [Dup] sum of eps over the up particles
    uint64_t *upmov = nullptr;  // [Dup][N-1][nu] F(up') | sign << 63
    uint8_t *upcnt = nullptr;   // [Dup][N-1]
    uint64_t *doff = nullptr;   // [N + 1]
    uint32_t *dstr = nullptr;   // [Ddn] down strings grouped by momentum, ascending within a group
    uint32_t *dkd = nullptr;    // [Ddn] momentum of each list entry
    double *ed = nullptr;       // [Ddn]
    uint32_t *dnmov = nullptr;  // per momentum block: [(q-1) nd + slot][len] G(dn') | sign << 31
    uint8_t *dncnt = nullptr;   // per momentum block: [q-1][len]
    uint64_t *mbase = nullptr, *cbase = nullptr;  // [N]
    // rows paired by down momentum for the two-row H·v: [npairs][2] row indices,
    // second entry 0xFFFFFFFF for a row left without a partner; rows of length 0 omitted
    uint32_t *pairs = nullptr;
    uint32_t npairs = 0;
};

namespace {

constexpr int kThreads = 256;

int grid_for(uint64_t n, int sms) {
    return (int)std::max<uint64_t>(1, std::min<uint64_t>((n + kThreads - 1) / kThreads, (uint64_t)sms * 8));
}

struct KArgs {
    int Lx, Ly, N, K, nu, nd;
    const uint32_t *Cdn;
    const uint64_t *Ct;
};

__host__ __device__ inline int kadd(int Lx, int Ly, int a, int b) {
    return (a % Lx + b % Lx) % Lx + Lx * ((a / Lx + b / Lx) % Ly);
}
__host__ __device__ inline int kneg(int Lx, int Ly, int a) {
    return (Lx - a % Lx) % Lx + Lx * ((Ly - a / Lx) % Ly);
}
__host__ __device__ inline int ksub(int Lx, int Ly, int a, int b) { return kadd(Lx, Ly, a, kneg(Lx, Ly, b)); }

__device__ __forceinline__ int kmomentum(const KArgs &a, uint32_t s) {
    int k = 0;
    while (s) {
        const int i = __ffs(s) - 1;
        k = kadd(a.Lx, a.Ly, k, i);
        s &= s - 1;
    }
    return k;
}

__device__ __forceinline__ uint32_t cdn(const KArgs &a, int i, int m, int k) {
    return a.Cdn[((size_t)i * (a.nd + 1) + m) * a.N + k];
}
__device__ __forceinline__ uint64_t ct(const KArgs &a, int i, int m, int k) {
    return a.Ct[((size_t)i * (a.nu + 1) + m) * a.N + k];
}

// spin-down forward map (Sec. IV A): index within the momentum list, and the momentum
__device__ __forceinline__ uint32_t kfwd_dn(const KArgs &a, uint32_t s, int *kout) {
    uint32_t idx = 0;
    int m = 0, k = 0;
    while (s) {
        const int i = __ffs(s) - 1;
        ++m;
        k = kadd(a.Lx, a.Ly, k, i);
        idx += cdn(a, i, m, k);
        s &= s - 1;
    }
    *kout = k;
    return idx;
}

// up part of the spin-full forward map, k starting at the spin-down momentum
__device__ __forceinline__ uint64_t kfwd_up(const KArgs &a, uint32_t u, int k) {
    uint64_t idx = 0;
    int m = 0;
    while (u) {
        const int i = __ffs(u) - 1;
        ++m;
        k = kadd(a.Lx, a.Ly, k, i);
        idx += ct(a, i, m, k);
        u &= u - 1;
    }
    return idx;
}

__device__ __forceinline__ uint32_t kbwd_dn(const KArgs &a, uint64_t p, int n, int k) {
    uint32_t s = 0;
    int m = n;
    for (int i = a.N - 1; i >= 0 && m > 0; --i) {
        const uint32_t c = cdn(a, i, m, k);
        if (p >= c) {
            s |= 1u << i;
            p -= c;
            --m;
            k = ksub(a.Lx, a.Ly, k, i);
        }
    }
    return s;
}

__device__ __forceinline__ void kbwd_spin(const KArgs &a, uint64_t p, uint32_t *u_out, uint32_t *d_out) {
    uint32_t u = 0;
    int m = a.nu, k = a.K;
    for (int i = a.N - 1; i >= 0 && m > 0; --i) {
        const uint64_t c = ct(a, i, m, k);
        if (p >= c) {
            u |= 1u << i;
            p -= c;
            --m;
            k = ksub(a.Lx, a.Ly, k, i);
        }
    }
    *u_out = u;
    *d_out = kbwd_dn(a, p, a.nd, k);
}

__device__ __forceinline__ uint32_t between(int a, int b) {
    const int lo = a < b ? a : b, hi = a < b ? b : a;
    return (uint32_t)(((1ull << hi) - 1) & ~((1ull << (lo + 1)) - 1));
}

__device__ __forceinline__ double eps_sum(const double *eps, uint32_t s) {
    double e = 0.0;
    while (s) {
        e += eps[__ffs(s) - 1];
        s &= s - 1;
    }
    return e;
}

// rows: every up string (plain ascending order by the backward map of Sec. III)
__global__ void k_k_rows(KArgs a, const uint32_t *__restrict__ lut, const double *__restrict__ eps, uint64_t Dup,
                         uint32_t *ustr, uint64_t *rowF, uint32_t *rowKd, double *eu) {
    for (uint64_t r = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; r < Dup; r += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t u = pd_backward_map(lut, (uint32_t)r, a.nu, a.N);
        const int kd = ksub(a.Lx, a.Ly, a.K, kmomentum(a, u));
        ustr[r] = u;
        rowKd[r] = (uint32_t)kd;
        rowF[r] = kfwd_up(a, u, kd);
        eu[r] = eps_sum(eps, u);
    }
}

// up moves of row r: for q = 1 .. N-1, every up particle k with k+q empty, in
// ascending k: F(up') and the sign of c^dag_{k+q} c_k
__global__ void k_k_upmoves(KArgs a, const uint32_t *__restrict__ ustr, uint64_t Dup, uint64_t *upmov,
                            uint8_t *upcnt) {
    const uint64_t n = Dup * (uint64_t)(a.N - 1);
    for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < n; e += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t r = e / (a.N - 1);
        const int q = (int)(e - r * (a.N - 1)) + 1;
        const uint32_t u = ustr[r];
        const int kd2 = ksub(a.Lx, a.Ly, ksub(a.Lx, a.Ly, a.K, kmomentum(a, u)), q);  // K_dn of the target row
        int slot = 0;
        for (uint32_t s = u; s; s &= s - 1) {
            const int k = __ffs(s) - 1, kq = kadd(a.Lx, a.Ly, k, q);
            if ((u >> kq) & 1u) continue;
            const uint32_t u2 = u ^ (1u << k) ^ (1u << kq);
            const uint64_t neg = (uint64_t)(__popc(u & between(k, kq)) & 1);
            upmov[e * a.nu + slot++] = kfwd_up(a, u2, kd2) | (neg << 63);
        }
        upcnt[e] = (uint8_t)slot;
    }
}

// down lists: every down string placed at its index within its momentum list
__global__ void k_k_dlists(KArgs a, const uint32_t *__restrict__ lut, const double *__restrict__ eps, uint64_t Ddn,
                           const uint64_t *__restrict__ doff, uint32_t *dstr, uint32_t *dkd, double *ed) {
    for (uint64_t r = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; r < Ddn; r += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t d = pd_backward_map(lut, (uint32_t)r, a.nd, a.N);
        int k = 0;
        const uint32_t g = kfwd_dn(a, d, &k);
        const uint64_t e = doff[k] + g;
        dstr[e] = d;
        dkd[e] = (uint32_t)k;
        ed[e] = eps_sum(eps, d);
    }
}

// down moves of list entry e (momentum kd, position j): for q = 1 .. N-1, every
// down particle k with k-q empty: G(dn') and the sign of c^dag_{k-q} c_k
__global__ void k_k_dnmoves(KArgs a, const uint32_t *__restrict__ dstr, const uint32_t *__restrict__ dkd,
                            const uint64_t *__restrict__ doff, const uint64_t *__restrict__ mbase,
                            const uint64_t *__restrict__ cbase, uint64_t Ddn, uint32_t *dnmov, uint8_t *dncnt) {
    for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < Ddn; e += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t d = dstr[e];
        const int kd = (int)dkd[e];
        const uint64_t len = doff[kd + 1] - doff[kd], j = e - doff[kd];
        for (int q = 1; q < a.N; ++q) {
            int slot = 0;
            for (uint32_t s = d; s; s &= s - 1) {
                const int k = __ffs(s) - 1, kq = ksub(a.Lx, a.Ly, k, q);
                if ((d >> kq) & 1u) continue;
                const uint32_t d2 = d ^ (1u << k) ^ (1u << kq);
                int k2 = 0;
                const uint32_t g = kfwd_dn(a, d2, &k2);
                const uint32_t neg = (uint32_t)(__popc(d & between(k, kq)) & 1);
                dnmov[mbase[kd] + ((uint64_t)(q - 1) * a.nd + slot++) * len + j] = g | (neg << 31);
            }
            dncnt[cbase[kd] + (uint64_t)(q - 1) * len + j] = (uint8_t)slot;
        }
    }
}

struct KHv {
    KArgs a;
    uint64_t Dup;
    const uint64_t *rowF, *upmov, *doff, *mbase, *cbase;
    const uint32_t *rowKd, *dnmov;
    const uint8_t *upcnt, *dncnt;
    const double *eu, *ed;
    double U_over_N, U_diag;  // U / N, and U nu nd / N (the q = 0 terms)
    int64_t Kun;              // fixed point: U / N as K 2^-G
    int Gun;
};

// One warp per row (up string) at a time; lane j handles the row's j-th
// spin-down string.  y = diag x + (U/N) sum_q sum_{up move a} sum_{dn move b}
// s_a s_b x[F_a + G_b], the up moves of the row staged in the warp's share of
// shared memory, the gathers issued four at a time.  Fixed point: the signed
// terms are summed exactly (two non-negative running sums), then one rounded
// product each for the diagonal and for U/N.
template <typename T>
__global__ void __launch_bounds__(256) k_k_hv(KHv p, const T *__restrict__ x, T *__restrict__ y) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int N = p.a.N, nu = p.a.nu, nd = p.a.nd;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const size_t per_warp = (size_t)(N - 1) * (nu > 0 ? nu : 1);
    uint64_t *s_up = reinterpret_cast<uint64_t *>(smem) + warp * per_warp;
    uint8_t *s_cnt = reinterpret_cast<uint8_t *>(reinterpret_cast<uint64_t *>(smem) + nwarps * per_warp) + warp * 32;
    for (uint64_t r = (uint64_t)blockIdx.x * nwarps + warp; r < p.Dup; r += (uint64_t)gridDim.x * nwarps) {
        const int kd = (int)p.rowKd[r];
        const uint64_t len = p.doff[kd + 1] - p.doff[kd];
        if (len == 0) continue;  // uniform across the warp
        __syncwarp();
        for (int e = lane; e < (N - 1) * nu; e += 32) s_up[e] = p.upmov[r * (uint64_t)(N - 1) * nu + e];
        if (lane < N - 1) s_cnt[lane] = p.upcnt[r * (uint64_t)(N - 1) + lane];
        __syncwarp();
        const uint64_t F = p.rowF[r], e0 = p.doff[kd];
        const double eur = p.eu[r];
        const uint32_t *dm = p.dnmov + p.mbase[kd];
        const uint8_t *dc = p.dncnt + p.cbase[kd];
        for (uint64_t j = lane; j < len; j += 32) {
            const double diag = eur + p.ed[e0 + j] + p.U_diag;
            const T xI = x[F + j];
            int64_t pos = 0, neg = 0;
            T acc = T(0);
            for (int q = 1; q < N; ++q) {
                const int cu = s_cnt[q - 1];
                if (cu == 0) continue;
                const int cd = dc[(uint64_t)(q - 1) * len + j];
                const uint64_t *ua = s_up + (size_t)(q - 1) * nu;
                for (int b = 0; b < cd; ++b) {
                    const uint32_t ev = dm[((uint64_t)(q - 1) * nd + b) * len + j];
                    const uint64_t G = ev & 0x7FFFFFFFu;
                    const uint64_t sb = ev >> 31;
                    for (int a0 = 0; a0 < cu; a0 += 4) {
                        uint64_t m[4];
                        T v[4];
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            m[i] = a0 + i < cu ? ua[a0 + i] : 0;
                            v[i] = a0 + i < cu ? x[(m[i] & 0x7FFFFFFFFFFFFFFFull) + G] : T(0);
                        }
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            if constexpr (std::is_same<T, int64_t>::value) {
                                if ((m[i] >> 63) ^ sb) neg += v[i];
                                else pos += v[i];
                            } else {
                                acc += ((m[i] >> 63) ^ sb) ? -v[i] : v[i];
                            }
                        }
                    }
                }
            }
            if constexpr (std::is_same<T, int64_t>::value) {
                const FxCoef c = fx_coef_dev(diag);
                y[F + j] = fx_mul(xI, c.K, c.G) + fx_mul(pos - neg, p.Kun, p.Gun);
            } else {
                y[F + j] = (T)diag * xI + (T)p.U_over_N * acc;
            }
        }
    }
}

// Row-factorised form: for a row u and a momentum transfer q every up move
// lands in a row of the same length (K_dn' = K_dn - q), so
//     t_q = sum_a s_a x[row u'_a]
// is formed once per (u, q) from whole rows read coalesced and kept in shared
// memory, and each column j of row u then adds sum_b s_b t_q[G_b(j)], the
// spin-down moves of its string gathered from shared memory (the same order of
// work as the tensor-product H·v of Sec. II A).  One CTA per row; thread t
// keeps the accumulators of columns t, t + blockDim, ... (JM of them).  In
// fixed point every partial sum is an exact integer sum, so the result is the
// same integer as the pairwise form's.
template <typename T, int JM>
__global__ void __launch_bounds__(512) k_k_hv_rows(KHv p, const T *__restrict__ x, T *__restrict__ y,
                                                     uint32_t maxlen) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int N = p.a.N, nu = p.a.nu, nd = p.a.nd;
    uint64_t *s_up = reinterpret_cast<uint64_t *>(smem);
    const size_t nup = (size_t)(N - 1) * (nu > 0 ? nu : 1);
    uint8_t *s_cnt = reinterpret_cast<uint8_t *>(s_up + nup);
    // two buffers of the per-q row sums: t_q is built in buffer q % 2 while other
    // threads may still read t_{q-1} from the other one, so one barrier per q suffices
    T *s_t0 = reinterpret_cast<T *>(smem + ((nup * 8 + 32 + 15) & ~(size_t)15));
    T *s_t1 = s_t0 + maxlen;
    for (uint64_t r = blockIdx.x; r < p.Dup; r += gridDim.x) {
        const int kd = (int)p.rowKd[r];
        const uint32_t len = (uint32_t)(p.doff[kd + 1] - p.doff[kd]);
        if (len == 0) continue;  // uniform across the CTA
        __syncthreads();  // the previous row is done with shared memory
        for (int e = threadIdx.x; e < (N - 1) * nu; e += blockDim.x) s_up[e] = p.upmov[r * (uint64_t)(N - 1) * nu + e];
        if (threadIdx.x < N - 1) s_cnt[threadIdx.x] = p.upcnt[r * (uint64_t)(N - 1) + threadIdx.x];
        __syncthreads();
        const uint32_t *dm = p.dnmov + p.mbase[kd];
        const uint8_t *dc = p.dncnt + p.cbase[kd];
        int64_t acc_i[JM];
        T acc_f[JM];
#pragma unroll
        for (int i = 0; i < JM; ++i) acc_i[i] = 0, acc_f[i] = T(0);
        int buf = 0;
        for (int q = 1; q < N; ++q) {
            const int cu = s_cnt[q - 1];
            if (cu == 0) continue;  // uniform
            const int kd2 = ksub(p.a.Lx, p.a.Ly, kd, q);
            const uint32_t len2 = (uint32_t)(p.doff[kd2 + 1] - p.doff[kd2]);
            const uint64_t *ua = s_up + (size_t)(q - 1) * nu;
            T *s_t = buf ? s_t1 : s_t0;
            for (uint32_t e = threadIdx.x; e < len2; e += blockDim.x) {
                T t = T(0);
                for (int a = 0; a < cu; ++a) {
                    const uint64_t m = ua[a];
                    const T v = x[(m & 0x7FFFFFFFFFFFFFFFull) + e];
                    t = (m >> 63) ? t - v : t + v;
                }
                s_t[e] = t;
            }
            __syncthreads();
            const uint8_t *dcq = dc + (uint64_t)(q - 1) * len;
            const uint32_t *dmq = dm + (uint64_t)(q - 1) * nd * len;
#pragma unroll
            for (int i = 0; i < JM; ++i) {
                const uint32_t j = threadIdx.x + (uint32_t)i * blockDim.x;
                if (j >= len) break;
                const int cd = dcq[j];
                const uint32_t *dmj = dmq + j;
                for (int b = 0; b < cd; ++b) {
                    const uint32_t ev = dmj[(uint64_t)b * len];
                    const T v = s_t[ev & 0x7FFFFFFFu];
                    if constexpr (std::is_same<T, int64_t>::value) {
                        const int64_t mneg = -(int64_t)(ev >> 31);
                        acc_i[i] += (v ^ mneg) - mneg;
                    } else {
                        acc_f[i] += (ev >> 31) ? -v : v;
                    }
                }
            }
            buf ^= 1;
        }
        const uint64_t F = p.rowF[r], e0 = p.doff[kd];
        const double eur = p.eu[r];
#pragma unroll
        for (int i = 0; i < JM; ++i) {
            const uint32_t j = threadIdx.x + (uint32_t)i * blockDim.x;
            if (j >= len) break;
            const double diag = eur + p.ed[e0 + j] + p.U_diag;
            const T xI = x[F + j];
            if constexpr (std::is_same<T, int64_t>::value) {
                const FxCoef c = fx_coef_dev(diag);
                y[F + j] = fx_mul(xI, c.K, c.G) + fx_mul(acc_i[i], p.Kun, p.Gun);
            } else {
                y[F + j] = (T)diag * xI + (T)p.U_over_N * acc_f[i];
            }
        }
    }
}

// Two rows per CTA: rows u0, u1 of equal down momentum K_dn share the column
// count, the spin-down move lists and their per-column counts, so each move
// entry is loaded once and gathers t_q of both rows, and the two rows share
// each q's CTA barrier.  Per row the work and its order are those of
// k_k_hv_rows (t_q summed over the row's up moves in list order, then every
// column adds its spin-down moves in list order), so the results are the same
// values, bit for bit, for every vector type.
template <typename T, int JM>
__global__ void __launch_bounds__(512) k_k_hv_rows2(KHv p, const uint32_t *__restrict__ pairs, uint32_t npairs,
                                                      const T *__restrict__ x, T *__restrict__ y, uint32_t maxlen) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int N = p.a.N, nu = p.a.nu, nd = p.a.nd;
    const size_t nup = (size_t)(N - 1) * (nu > 0 ? nu : 1);
    uint64_t *s_up = reinterpret_cast<uint64_t *>(smem);           // [2][nup]
    uint8_t *s_cnt = reinterpret_cast<uint8_t *>(s_up + 2 * nup);  // [2][32]
    // per-q row sums, double-buffered as in k_k_hv_rows: [buffer][row of the pair][maxlen]
    T *s_t = reinterpret_cast<T *>(smem + ((2 * nup * 8 + 64 + 15) & ~(size_t)15));
    for (uint32_t pi = blockIdx.x; pi < npairs; pi += gridDim.x) {
        const uint32_t r0 = pairs[2 * (uint64_t)pi], r1 = pairs[2 * (uint64_t)pi + 1];
        const bool two = r1 != 0xFFFFFFFFu;
        const int kd = (int)p.rowKd[r0];
        const uint32_t len = (uint32_t)(p.doff[kd + 1] - p.doff[kd]);
        __syncthreads();  // the previous pair is done with shared memory
        for (int e = threadIdx.x; e < (N - 1) * nu; e += blockDim.x) {
            s_up[e] = p.upmov[r0 * (uint64_t)(N - 1) * nu + e];
            s_up[nup + e] = two ? p.upmov[r1 * (uint64_t)(N - 1) * nu + e] : 0ull;
        }
        if (threadIdx.x < N - 1) {
            s_cnt[threadIdx.x] = p.upcnt[r0 * (uint64_t)(N - 1) + threadIdx.x];
            s_cnt[32 + threadIdx.x] = two ? p.upcnt[r1 * (uint64_t)(N - 1) + threadIdx.x] : (uint8_t)0;
        }
        __syncthreads();
        const uint32_t *dm = p.dnmov + p.mbase[kd];
        const uint8_t *dc = p.dncnt + p.cbase[kd];
        int64_t ai0[JM], ai1[JM];
        T af0[JM], af1[JM];
#pragma unroll
        for (int i = 0; i < JM; ++i) ai0[i] = ai1[i] = 0, af0[i] = af1[i] = T(0);
        int buf = 0;
        for (int q = 1; q < N; ++q) {
            const int cu0 = s_cnt[q - 1], cu1 = s_cnt[32 + q - 1];
            if (cu0 == 0 && cu1 == 0) continue;  // uniform
            const int kd2 = ksub(p.a.Lx, p.a.Ly, kd, q);
            const uint32_t len2 = (uint32_t)(p.doff[kd2 + 1] - p.doff[kd2]);
            const uint64_t *ua0 = s_up + (size_t)(q - 1) * nu, *ua1 = ua0 + nup;
            T *st0 = s_t + (size_t)buf * 2 * maxlen, *st1 = st0 + maxlen;
            for (uint32_t e = threadIdx.x; e < len2; e += blockDim.x) {
                T t0 = T(0), t1 = T(0);
                for (int a = 0; a < cu0; ++a) {
                    const uint64_t m = ua0[a];
                    const T v = x[(m & 0x7FFFFFFFFFFFFFFFull) + e];
                    t0 = (m >> 63) ? t0 - v : t0 + v;
                }
                for (int a = 0; a < cu1; ++a) {
                    const uint64_t m = ua1[a];
                    const T v = x[(m & 0x7FFFFFFFFFFFFFFFull) + e];
                    t1 = (m >> 63) ? t1 - v : t1 + v;
                }
                st0[e] = t0;
                st1[e] = t1;
            }
            __syncthreads();
            const uint8_t *dcq = dc + (uint64_t)(q - 1) * len;
            const uint32_t *dmq = dm + (uint64_t)(q - 1) * nd * len;
#pragma unroll
            for (int i = 0; i < JM; ++i) {
                const uint32_t j = threadIdx.x + (uint32_t)i * blockDim.x;
                if (j >= len) break;
                const int cd = dcq[j];
                const uint32_t *dmj = dmq + j;
                for (int b = 0; b < cd; ++b) {
                    const uint32_t ev = dmj[(uint64_t)b * len];
                    const uint32_t g = ev & 0x7FFFFFFFu;
                    const T v0 = st0[g], v1 = st1[g];
                    if constexpr (std::is_same<T, int64_t>::value) {
                        const int64_t mneg = -(int64_t)(ev >> 31);
                        ai0[i] += (v0 ^ mneg) - mneg;
                        ai1[i] += (v1 ^ mneg) - mneg;
                    } else {
                        af0[i] += (ev >> 31) ? -v0 : v0;
                        af1[i] += (ev >> 31) ? -v1 : v1;
                    }
                }
            }
            buf ^= 1;
        }
        const uint64_t e0 = p.doff[kd];
#pragma unroll
        for (int w = 0; w < 2; ++w) {
            if (w == 1 && !two) break;
            const uint32_t r = w ? r1 : r0;
            const uint64_t F = p.rowF[r];
            const double eur = p.eu[r];
#pragma unroll
            for (int i = 0; i < JM; ++i) {
                const uint32_t j = threadIdx.x + (uint32_t)i * blockDim.x;
                if (j >= len) break;
                const double diag = eur + p.ed[e0 + j] + p.U_diag;
                const T xI = x[F + j];
                if constexpr (std::is_same<T, int64_t>::value) {
                    const FxCoef c = fx_coef_dev(diag);
                    y[F + j] = fx_mul(xI, c.K, c.G) + fx_mul(w ? ai1[i] : ai0[i], p.Kun, p.Gun);
                } else {
                    y[F + j] = (T)diag * xI + (T)p.U_over_N * (w ? af1[i] : af0[i]);
                }
            }
        }
    }
}

// Batched spin-full maps for the API: states are (up << N) | dn over the momentum bits.
__global__ void k_k_rank(KArgs a, const uint64_t *__restrict__ states, uint64_t *__restrict__ idx, uint64_t n,
                         unsigned *err) {
    const uint64_t mask = (1ull << a.N) - 1;
    for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < n; e += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t s = states[e];
        const uint32_t u = (uint32_t)((s >> a.N) & mask), d = (uint32_t)(s & mask);
        bool ok = (s >> (2 * a.N)) == 0 && __popc(u) == a.nu && __popc(d) == a.nd;
        uint64_t r = UINT64_MAX;
        if (ok) {
            int kd = 0;
            const uint32_t g = kfwd_dn(a, d, &kd);
            ok = kadd(a.Lx, a.Ly, kmomentum(a, u), kd) == a.K;
            if (ok) r = kfwd_up(a, u, kd) + g;
        }
        if (!ok) atomicOr(err, PD_ERRBIT(HB_ERR_INVALID_STATE));
        idx[e] = r;
    }
}

__global__ void k_k_unrank(KArgs a, const uint64_t *__restrict__ idx, uint64_t *__restrict__ states, uint64_t n,
                           uint64_t D, unsigned *err) {
    for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < n; e += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t i = idx[e];
        if (i >= D) {
            atomicOr(err, PD_ERRBIT(HB_ERR_OUT_OF_RANGE));
            states[e] = UINT64_MAX;
            continue;
        }
        uint32_t u = 0, d = 0;
        kbwd_spin(a, i, &u, &d);
        states[e] = ((uint64_t)u << a.N) | d;
    }
}

// Verification export: canonical rows (columns ascending, the diagonal
// included), read from the same move tables the H·v uses.
__global__ void k_k_rows_export(KHv p, const uint32_t *__restrict__ lut, uint64_t row0, uint32_t nrows, uint32_t max_entries, uint64_t *cols, double *vals,
                                uint32_t *counts, unsigned *err) {
    const int N = p.a.N, nu = p.a.nu, nd = p.a.nd;
    for (uint64_t rr = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; rr < nrows;
         rr += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t I = row0 + rr;
        uint32_t u = 0, d = 0;
        kbwd_spin(p.a, I, &u, &d);
        // row of u: its position among all up strings (forward map of Eq. 3)
        const uint64_t r = pd_forward_map(lut, u);
        const int kd = (int)p.rowKd[r];
        const uint64_t len = p.doff[kd + 1] - p.doff[kd], F = p.rowF[r];
        const uint64_t j = I - F;
        uint64_t *c = cols + rr * max_entries;
        double *v = vals + rr * max_entries;
        uint32_t n = 0;
        bool over = false;
        auto put = [&](uint64_t col, double val) {
            if (n < max_entries) {
                c[n] = col;
                v[n] = val;
            } else {
                over = true;
            }
            ++n;
        };
        put(I, p.eu[r] + p.ed[p.doff[kd] + j] + p.U_diag);
        const uint32_t *dm = p.dnmov + p.mbase[kd];
        const uint8_t *dc = p.dncnt + p.cbase[kd];
        for (int q = 1; q < N; ++q) {
            const int cu = p.upcnt[r * (uint64_t)(N - 1) + q - 1];
            const int cd = dc[(uint64_t)(q - 1) * len + j];
            for (int b = 0; b < cd; ++b) {
                const uint32_t ev = dm[((uint64_t)(q - 1) * nd + b) * len + j];
                for (int aa = 0; aa < cu; ++aa) {
                    const uint64_t m = p.upmov[(r * (uint64_t)(N - 1) + q - 1) * nu + aa];
                    const double sgn = ((m >> 63) ^ (ev >> 31)) ? -1.0 : 1.0;
                    put((m & 0x7FFFFFFFFFFFFFFFull) + (ev & 0x7FFFFFFFu), sgn * p.U_over_N);
                }
            }
        }
        if (over) {
            atomicOr(err, PD_ERRBIT(HB_ERR_INVALID_ARG));
            counts[rr] = UINT32_MAX;
            continue;
        }
        for (uint32_t a1 = 1; a1 < n; ++a1) {  // insertion sort by column
            const uint64_t ck = c[a1];
            const double vk = v[a1];
            uint32_t b1 = a1;
            while (b1 > 0 && c[b1 - 1] > ck) {
                c[b1] = c[b1 - 1];
                v[b1] = v[b1 - 1];
                --b1;
            }
            c[b1] = ck;
            v[b1] = vk;
        }
        counts[rr] = n;
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// host side

namespace {

uint64_t binom_host(int n, int k) {
    if (k < 0 || k > n) return 0;
    uint64_t r = 1;
    for (int i = 1; i <= k; ++i) r = r * (uint64_t)(n - k + i) / (uint64_t)i;
    return r;
}

// C_i^m(k) for 0 <= i <= N, 0 <= m <= n by the recursion of Sec. IV A
std::vector<uint64_t> c_table(int Lx, int Ly, int n) {
    const int N = Lx * Ly;
    std::vector<uint64_t> C((size_t)(N + 1) * (n + 1) * N, 0);
    auto at = [&](int i, int m, int k) -> uint64_t & { return C[((size_t)i * (n + 1) + m) * N + k]; };
    at(0, 0, 0) = 1;
    for (int i = 1; i <= N; ++i)
        for (int m = 0; m <= n; ++m)
            for (int k = 0; k < N; ++k) {
                uint64_t v = at(i - 1, m, k);
                if (m >= 1) v += at(i - 1, m - 1, ksub(Lx, Ly, k, i - 1));
                at(i, m, k) = v;
            }
    return C;
}

template <typename T>
hb_status upload(T **dst, const std::vector<T> &src) {
    if (cudaMalloc(dst, std::max<size_t>(src.size(), 1) * sizeof(T)) != cudaSuccess) return HB_ERR_NO_MEMORY;
    if (!src.empty() && cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess)
        return HB_ERR_CUDA;
    return HB_OK;
}

template <typename T>
hb_status alloc(T **dst, uint64_t n) {
    return cudaMalloc(dst, std::max<uint64_t>(n, 1) * sizeof(T)) == cudaSuccess ? HB_OK : HB_ERR_NO_MEMORY;
}

KArgs kargs(const KSpace &k) {
    KArgs a;
    a.Lx = k.Lx, a.Ly = k.Ly, a.N = k.N, a.K = k.K, a.nu = k.nu, a.nd = k.nd;
    a.Cdn = k.Cdn;
    a.Ct = k.Ct;
    return a;
}

KHv khv(hb_handle h) {
    const KSpace &k = *h->ks;
    KHv p;
    p.a = kargs(k);
    p.Dup = k.Dup;
    p.rowF = k.rowF, p.upmov = k.upmov, p.doff = k.doff, p.mbase = k.mbase, p.cbase = k.cbase;
    p.rowKd = k.rowKd, p.dnmov = k.dnmov, p.upcnt = k.upcnt, p.dncnt = k.dncnt, p.eu = k.eu, p.ed = k.ed;
    p.U_over_N = h->U / k.N;
    p.U_diag = h->U * k.nu * k.nd / k.N;
    // U / N as K 2^-G (same convention as the device-side conversion)
    p.Kun = 0, p.Gun = 1;
    if (p.U_over_N != 0.0) {
        int e = 0;
        std::frexp(p.U_over_N, &e);
        p.Gun = std::min(63, std::max(1, 62 - e));
        p.Kun = (int64_t)std::llrint(std::ldexp(p.U_over_N, p.Gun));
    }
    return p;
}

}  // namespace

void pd_k_free(KSpace *k) {
    if (!k) return;
    cudaFree(k->Cdn), cudaFree(k->Ct), cudaFree(k->eps), cudaFree(k->ustr), cudaFree(k->rowF), cudaFree(k->rowKd);
    cudaFree(k->eu), cudaFree(k->upmov), cudaFree(k->upcnt), cudaFree(k->doff), cudaFree(k->dstr), cudaFree(k->dkd);
    cudaFree(k->ed), cudaFree(k->dnmov), cudaFree(k->dncnt), cudaFree(k->mbase), cudaFree(k->cbase);
    cudaFree(k->pairs);
    delete k;
}

namespace {

// All sector tables: C, C~, eps on the host; rows, moves and lists by the kernels above.
hb_status build_kspace(hb_handle h, KSpace &k) {
    const int N = k.N;
    std::vector<uint64_t> Cu = c_table(k.Lx, k.Ly, k.nu), Cd = c_table(k.Lx, k.Ly, k.nd);
    std::vector<uint32_t> Cd32(Cd.size());
    for (size_t i = 0; i < Cd.size(); ++i) Cd32[i] = (uint32_t)Cd[i];  // C(N, n) < 2^32 for N <= 32
    std::vector<uint64_t> Ct((size_t)(N + 1) * (k.nu + 1) * N, 0);
    auto cd_N = [&](int kd) { return Cd[((size_t)N * (k.nd + 1) + k.nd) * N + kd]; };
    for (int i = 0; i <= N; ++i)
        for (int m = 0; m <= k.nu; ++m)
            for (int kk = 0; kk < N; ++kk) {
                uint64_t v = 0;
                for (int kd = 0; kd < N; ++kd)
                    v += Cu[((size_t)i * (k.nu + 1) + m) * N + ksub(k.Lx, k.Ly, kk, kd)] * cd_N(kd);
                Ct[((size_t)i * (k.nu + 1) + m) * N + kk] = v;
            }
    h->D = Ct[((size_t)N * (k.nu + 1) + k.nu) * N + k.K];
    std::vector<double> eps(N);
    for (int i = 0; i < N; ++i) {
        const double kx = 2.0 * M_PI * (i % k.Lx) / k.Lx, ky = 2.0 * M_PI * (i / k.Lx) / k.Ly;
        eps[i] = k.Ly == 1 ? -2.0 * k.t * std::cos(kx)
                           : -2.0 * k.t * (std::cos(kx) + std::cos(ky)) - 4.0 * k.tp * std::cos(kx) * std::cos(ky);
    }
    k.h_doff.assign(N + 1, 0);
    k.h_mbase.assign(N, 0);
    k.h_cbase.assign(N, 0);
    uint64_t mb = 0, cb = 0;
    for (int kd = 0; kd < N; ++kd) {
        const uint64_t len = cd_N(kd);
        k.h_doff[kd + 1] = k.h_doff[kd] + len;
        k.h_mbase[kd] = mb;
        k.h_cbase[kd] = cb;
        mb += (uint64_t)(N - 1) * k.nd * len;
        cb += (uint64_t)(N - 1) * len;
    }
    hb_status s;
    if ((s = upload(&k.Cdn, Cd32)) != HB_OK || (s = upload(&k.Ct, Ct)) != HB_OK || (s = upload(&k.eps, eps)) != HB_OK ||
        (s = upload(&k.doff, k.h_doff)) != HB_OK || (s = upload(&k.mbase, k.h_mbase)) != HB_OK ||
        (s = upload(&k.cbase, k.h_cbase)) != HB_OK)
        return s;
    if ((s = alloc(&k.ustr, k.Dup)) != HB_OK || (s = alloc(&k.rowF, k.Dup)) != HB_OK ||
        (s = alloc(&k.rowKd, k.Dup)) != HB_OK || (s = alloc(&k.eu, k.Dup)) != HB_OK ||
        (s = alloc(&k.upmov, k.Dup * (N - 1) * (uint64_t)std::max(k.nu, 1))) != HB_OK ||
        (s = alloc(&k.upcnt, k.Dup * (N - 1))) != HB_OK || (s = alloc(&k.dstr, k.Ddn)) != HB_OK ||
        (s = alloc(&k.dkd, k.Ddn)) != HB_OK || (s = alloc(&k.ed, k.Ddn)) != HB_OK ||
        (s = alloc(&k.dnmov, std::max<uint64_t>(mb, 1))) != HB_OK || (s = alloc(&k.dncnt, std::max<uint64_t>(cb, 1))) != HB_OK)
        return s;
    const KArgs a = kargs(k);
    k_k_rows<<<grid_for(k.Dup, h->sm_count), kThreads>>>(a, h->d_binom, k.eps, k.Dup, k.ustr, k.rowF, k.rowKd, k.eu);
    k_k_upmoves<<<grid_for(k.Dup * (N - 1), h->sm_count), kThreads>>>(a, k.ustr, k.Dup, k.upmov, k.upcnt);
    k_k_dlists<<<grid_for(k.Ddn, h->sm_count), kThreads>>>(a, h->d_binom, k.eps, k.Ddn, k.doff, k.dstr, k.dkd, k.ed);
    k_k_dnmoves<<<grid_for(k.Ddn, h->sm_count), kThreads>>>(a, k.dstr, k.dkd, k.doff, k.mbase, k.cbase, k.Ddn,
                                                           k.dnmov, k.dncnt);
    PD_CUDA(cudaGetLastError());
    PD_CUDA(cudaDeviceSynchronize());
    // rows paired by down momentum (ascending row order within each momentum) for k_k_hv_rows2
    std::vector<uint32_t> kd_of(k.Dup);
    PD_CUDA(cudaMemcpy(kd_of.data(), k.rowKd, k.Dup * sizeof(uint32_t), cudaMemcpyDeviceToHost));
    std::vector<std::vector<uint32_t>> by_kd(N);
    for (uint64_t r = 0; r < k.Dup; ++r)
        if (kd_of[r] < (uint32_t)N && k.h_doff[kd_of[r] + 1] > k.h_doff[kd_of[r]]) by_kd[kd_of[r]].push_back((uint32_t)r);
    std::vector<uint32_t> pairs;
    for (int kd = 0; kd < N; ++kd)
        for (size_t i = 0; i < by_kd[kd].size(); i += 2) {
            pairs.push_back(by_kd[kd][i]);
            pairs.push_back(i + 1 < by_kd[kd].size() ? by_kd[kd][i + 1] : 0xFFFFFFFFu);
        }
    k.npairs = (uint32_t)(pairs.size() / 2);
    if (!pairs.empty() && (s = upload(&k.pairs, pairs)) != HB_OK) return s;
    return HB_OK;
}

}  // namespace

namespace {

template <typename T, int JM>
hb_status launch_rows(hb_handle h, const KHv &p, const T *x, T *y, cudaStream_t st, uint64_t maxlen) {
    const size_t nup = (size_t)(h->ks->N - 1) * std::max(h->ks->nu, 1);
    const size_t smem = ((nup * 8 + 32 + 15) & ~(size_t)15) + 2 * (size_t)maxlen * sizeof(T);
    // threads: the fewest warps whose JM column slots cover the longest row, so no slot sits idle
    const int threads = (int)std::min<uint64_t>(512, std::max<uint64_t>(64, (maxlen + JM * 32 - 1) / (JM * 32) * 32));
    auto kern = k_k_hv_rows<T, JM>;
    PD_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    PD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem));
    if (per_sm < 1) return HB_ERR_NO_MEMORY;
    const unsigned grid = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(h->ks->Dup, (uint64_t)per_sm * h->sm_count));
    kern<<<grid, threads, smem, st>>>(p, x, y, (uint32_t)maxlen);
    PD_CUDA(cudaGetLastError());
    return HB_OK;
}

// Two rows of equal down momentum per CTA (k_k_hv_rows2); block size as in launch_rows.
template <typename T, int JM>
hb_status launch_rows2(hb_handle h, const KHv &p, const T *x, T *y, cudaStream_t st, uint64_t maxlen) {
    const KSpace &k = *h->ks;
    const size_t nup = (size_t)(k.N - 1) * std::max(k.nu, 1);
    const size_t smem = ((2 * nup * 8 + 64 + 15) & ~(size_t)15) + 4 * (size_t)maxlen * sizeof(T);
    const int threads = (int)std::min<uint64_t>(512, std::max<uint64_t>(64, (maxlen + JM * 32 - 1) / (JM * 32) * 32));
    auto kern = k_k_hv_rows2<T, JM>;
    PD_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    PD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem));
    if (per_sm < 1) return HB_ERR_NO_MEMORY;
    const unsigned grid = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(k.npairs, (uint64_t)per_sm * h->sm_count));
    kern<<<grid, threads, smem, st>>>(p, k.pairs, k.npairs, x, y, (uint32_t)maxlen);
    PD_CUDA(cudaGetLastError());
    return HB_OK;
}

template <typename T>
hb_status k_apply_t(hb_handle h, const T *x, T *y, cudaStream_t st) {
    const KHv p = khv(h);
    uint64_t maxlen = 0;
    for (int k = 0; k < h->ks->N; ++k) maxlen = std::max(maxlen, h->ks->h_doff[k + 1] - h->ks->h_doff[k]);
    // row-factorised form while a row fits the per-thread accumulators and shared memory; rows
    // in pairs of equal down momentum while both rows' double-buffered sums fit
    if (maxlen <= 4 * 512 && 4 * maxlen * sizeof(T) <= 96 * 1024 && h->ks->pairs)
        return launch_rows2<T, 4>(h, p, x, y, st, maxlen);
    if (maxlen <= 4 * 512 && 2 * maxlen * sizeof(T) <= 96 * 1024) return launch_rows<T, 4>(h, p, x, y, st, maxlen);
    if (maxlen <= 16 * 512 && 2 * maxlen * sizeof(T) <= 192 * 1024) return launch_rows<T, 16>(h, p, x, y, st, maxlen);
    constexpr int kWarps = 8;  // pairwise form, one row per warp
    const size_t smem = (size_t)kWarps * ((size_t)(h->ks->N - 1) * std::max(h->ks->nu, 1) * 8 + 32);
    const unsigned grid =
        (unsigned)std::max<uint64_t>(1, std::min<uint64_t>((h->ks->Dup + kWarps - 1) / kWarps, (uint64_t)h->sm_count * 8));
    k_k_hv<T><<<grid, 256, smem, st>>>(p, x, y);
    PD_CUDA(cudaGetLastError());
    return HB_OK;
}

}  // namespace

hb_status pd_k_apply(hb_handle h, hb_dtype dt, const void *x, void *y, cudaStream_t st) {
    if (dt == HB_F64) return k_apply_t<double>(h, static_cast<const double *>(x), static_cast<double *>(y), st);
    if (dt == HB_F32) return k_apply_t<float>(h, static_cast<const float *>(x), static_cast<float *>(y), st);
    return k_apply_t<int64_t>(h, static_cast<const int64_t *>(x), static_cast<int64_t *>(y), st);
}

hb_status pd_k_rank(hb_handle h, const uint64_t *states, uint64_t *idx, uint64_t n, cudaStream_t st) {
    k_k_rank<<<grid_for(n, h->sm_count), kThreads, 0, st>>>(kargs(*h->ks), states, idx, n, h->d_err);
    PD_CUDA(cudaGetLastError());
    return HB_OK;
}

hb_status pd_k_unrank(hb_handle h, const uint64_t *idx, uint64_t *states, uint64_t n, cudaStream_t st) {
    k_k_unrank<<<grid_for(n, h->sm_count), kThreads, 0, st>>>(kargs(*h->ks), idx, states, n, h->D, h->d_err);
    PD_CUDA(cudaGetLastError());
    return HB_OK;
}

hb_status pd_k_row_entries(hb_handle h, uint64_t row0, uint32_t nrows, uint32_t max_entries, uint64_t *cols,
                           double *vals, uint32_t *counts, cudaStream_t st) {
    k_k_rows_export<<<grid_for(nrows, h->sm_count), kThreads, 0, st>>>(khv(h), h->d_binom, row0, nrows, max_entries,
                                                                      cols, vals, counts, h->d_err);
    PD_CUDA(cudaGetLastError());
    return HB_OK;
}

extern "C" hb_status hubbard_basis_create_k(int Lx, int Ly, double t, double tp, double U, int N_up, int N_dn,
                                            int Kx, int Ky, hb_handle *out) {
    if (!out) return HB_ERR_INVALID_ARG;
    *out = nullptr;
    if (Lx < 1 || Ly < 1 || Lx * Ly < 2 || Lx * Ly > PD_MAXL || N_up < 0 || N_dn < 0 || N_up > Lx * Ly ||
        N_dn > Lx * Ly || Kx < 0 || Kx >= Lx || Ky < 0 || Ky >= Ly)
        return HB_ERR_INVALID_ARG;
    if (!(t == t) || !(tp == tp) || !(U == U)) return HB_ERR_INVALID_ARG;
    const int N = Lx * Ly;
    hb_basis *h = new (std::nothrow) hb_basis();
    if (!h) return HB_ERR_NO_MEMORY;
    KSpace *k = new (std::nothrow) KSpace();
    if (!k) {
        delete h;
        return HB_ERR_NO_MEMORY;
    }
    h->ks = k;
    k->Lx = Lx, k->Ly = Ly, k->N = N, k->K = Kx + Lx * Ky, k->nu = N_up, k->nd = N_dn, k->t = t, k->tp = tp;
    k->Dup = binom_host(N, N_up);
    k->Ddn = binom_host(N, N_dn);
    h->L = N;
    h->N_up = N_up;
    h->N_dn = N_dn;
    h->U = U;
    h->D_up = k->Dup;
    h->D_dn = k->Ddn;
    auto fail = [&](hb_status s) {
        hubbard_basis_destroy(h);
        return s;
    };
    if (cudaGetDevice(&h->device) != cudaSuccess) return fail(HB_ERR_CUDA);
    if (cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess)
        return fail(HB_ERR_CUDA);
    std::vector<uint32_t> lut((size_t)PD_LUT_W * PD_LUT_W, 0);
    for (int i = 0; i < PD_LUT_W; ++i)
        for (int m = 0; m < PD_LUT_W; ++m) lut[(size_t)i * PD_LUT_W + m] = (uint32_t)binom_host(i, m);
    if (upload(&h->d_binom, lut) != HB_OK) return fail(HB_ERR_CUDA);
    if (cudaMalloc(&h->d_err, sizeof(unsigned)) != cudaSuccess) return fail(HB_ERR_CUDA);
    if (cudaMemset(h->d_err, 0, sizeof(unsigned)) != cudaSuccess) return fail(HB_ERR_CUDA);
    hb_status s = build_kspace(h, *k);
    if (s != HB_OK) return fail(s);
    if (h->D == 0) return fail(HB_ERR_INVALID_ARG);  // empty momentum sector
    // fixed point: |w| <= 3 max row sum of |H|; the signed sums hold nu nd (N-1) terms of |x| < 1
    double emax = 0.0;
    for (int i = 0; i < N; ++i) {
        const double kx = 2.0 * M_PI * (i % Lx) / Lx, ky = 2.0 * M_PI * (i / Lx) / Ly;
        const double e = Ly == 1 ? -2.0 * t * std::cos(kx)
                                 : -2.0 * t * (std::cos(kx) + std::cos(ky)) - 4.0 * tp * std::cos(kx) * std::cos(ky);
        emax = std::max(emax, std::fabs(e));
    }
    const double bound = (N_up + N_dn) * emax + std::fabs(U) * N_up * N_dn;
    const double lim = std::max(3.0 * std::max(bound, 1.0), (double)N_up * N_dn * (N - 1) + 1.0);
    int F = 60;
    while (F > 8 && std::ldexp(lim, F) >= std::ldexp(1.0, 62)) --F;
    h->fx_frac = F;
    h->fx_ok = true;
    h->tables_built = true;
    *out = h;
    return HB_OK;
}

// ---------------------------------------------------------------------------
// Single-particle operators between momentum sectors (for the continued-
// fraction Green's function): y = c_{k s} x (op 0) or c+_{k s} x (op 1).  With
// the up creators (descending momentum index) to the left of the down
// creators, both carry (-1)^(particles of spin s above bit k) and, for s = down,
// (-1)^(N_up).  One thread per target state: its source state differs in bit k
// of spin s; the norm^2 of y is accumulated into *norm2 (if given).

namespace {

template <typename T>
__global__ void k_k_apply_c(KArgs src, KArgs dst, uint64_t Ddst, int op, int spin, int k, const T *__restrict__ x,
                            T *__restrict__ y, double *norm2) {
    double acc = 0.0;
    for (uint64_t J = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; J < Ddst; J += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t u = 0, d = 0;
        kbwd_spin(dst, J, &u, &d);
        const uint32_t part = spin == 0 ? u : d;
        const uint32_t has = (part >> k) & 1u;
        T v = T(0);
        // annihilation: the target lacks k, the source has it; creation: the reverse
        if ((op == 0 && !has) || (op == 1 && has)) {
            const uint32_t p2 = part ^ (1u << k);
            const uint32_t us = spin == 0 ? p2 : u, ds = spin == 0 ? d : p2;
            int kd = 0;
            const uint32_t g = kfwd_dn(src, ds, &kd);
            const uint64_t I = kfwd_up(src, us, kd) + g;
            int sgn = __popc(p2 >> (k + 1)) & 1;
            if (spin == 1) sgn ^= __popc(us) & 1;
            v = sgn ? -x[I] : x[I];
        }
        y[J] = v;
        acc += (double)v * (double)v;
    }
    if (norm2) {
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if ((threadIdx.x & 31) == 0 && acc != 0.0) atomicAdd(norm2, acc);
    }
}

}  // namespace

extern "C" hb_status hubbard_apply_c(hb_handle src, hb_handle dst, int op, int spin, int k, hb_dtype dt,
                                     const void *x, void *y, double *norm2, void *stream) {
    if (!src || !dst || !x || !y || !src->ks || !dst->ks || (op != 0 && op != 1) || (spin != 0 && spin != 1))
        return HB_ERR_INVALID_ARG;
    if (dt != HB_F64 && dt != HB_F32) return HB_ERR_INVALID_ARG;
    const KSpace &a = *src->ks, &b = *dst->ks;
    if (a.Lx != b.Lx || a.Ly != b.Ly || k < 0 || k >= a.N) return HB_ERR_INVALID_ARG;
    const int dn_ = op == 0 ? -1 : 1;
    const int want_nu = a.nu + (spin == 0 ? dn_ : 0), want_nd = a.nd + (spin == 1 ? dn_ : 0);
    const int want_K = op == 0 ? ksub(a.Lx, a.Ly, a.K, k) : kadd(a.Lx, a.Ly, a.K, k);
    if (b.nu != want_nu || b.nd != want_nd || b.K != want_K) return HB_ERR_INVALID_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (norm2) PD_CUDA(cudaMemsetAsync(norm2, 0, sizeof(double), st));
    if (dt == HB_F64)
        k_k_apply_c<double><<<grid_for(dst->D, dst->sm_count), kThreads, 0, st>>>(
            kargs(a), kargs(b), dst->D, op, spin, k, static_cast<const double *>(x), static_cast<double *>(y), norm2);
    else
        k_k_apply_c<float><<<grid_for(dst->D, dst->sm_count), kThreads, 0, st>>>(
            kargs(a), kargs(b), dst->D, op, spin, k, static_cast<const float *>(x), static_cast<float *>(y), norm2);
    PD_CUDA(cudaGetLastError());
    return HB_OK;
}

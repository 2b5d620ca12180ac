// Shared definitions of the Paradeisos GB300 library (internal header).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "paradeisos.h"

#define PD_MAXL 32
#define PD_LUT_W (PD_MAXL + 1)  // binomial table is PD_LUT_W x PD_LUT_W
#define PD_INVALID UINT64_MAX

#define PD_FX_MAXC 4  // distinct hopping amplitudes supported by the fixed-point path

// Sticky device error bits (one bit per hb_status code).
#define PD_ERRBIT(s) (1u << (unsigned)(s))

#define PD_CUDA(call)                                   \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) return HB_ERR_CUDA;      \
    } while (0)

// Per-spin tables of one sector: the ascending list of strings (built by the
// backward map) and the hop lists in ELL layout, entry k of string r at
// [k * D + r], so that threads handling consecutive strings read consecutive
// words.  count[r] <= zmax entries are valid; target is the per-spin index of
// the string reached through the hop, value is -t_b times the fermion sign.
struct SpinTables {
    uint64_t D = 0;
    int n = 0;
    int zmax = 0;
    uint32_t *str = nullptr;     // [D]
    uint16_t *count = nullptr;   // [D]
    uint32_t *target = nullptr;  // [zmax * D]
    double *val = nullptr;       // [zmax * D]
    float *valf = nullptr;       // [zmax * D] binary32 copy of val
    // fixed-point path: the same hops in segments of equal (amplitude class,
    // sign), ftarget[k * D + r]; seg[r] packs the 2*PD_FX_MAXC segment lengths
    // as bytes (byte 2c: class c positive sign, byte 2c+1: negative).
    uint32_t *ftarget = nullptr;
    uint64_t *seg = nullptr;
    // warp-blocked copy of the fixed-point hops for the row pass (built when
    // D + 8 < 65536): positions p are the strings sorted by their segment
    // lengths, so the 32 lanes of a warp (one block of 32 positions) share slot
    // counts.  wb_perm[p]: string at position p (D for padding); wb_str[p]: its
    // bits; wb_caps[b]: pairs of slots per segment of block b (byte q);
    // wb_base[b]: first pair row of block b in wb_ent; wb_ent[(pair row) * 32 +
    // lane]: two u16 targets (lo: even slot, hi: odd slot), D .. D+7 (a zero
    // element) for an empty slot; slots are ordered to spread each quarter
    // warp's targets over the shared-memory bank groups.
    bool wb_ok = false;
    uint32_t wb_nblk = 0;
    uint32_t *wb_perm = nullptr, *wb_str = nullptr, *wb_base = nullptr, *wb_ent = nullptr;
    uint64_t *wb_caps = nullptr;
};

// A real multiplier c in fixed point: c ~ K * 2^-G with |K| < 2^62, 1 <= G <= 63.
struct FxCoef {
    int64_t K = 0;
    int G = 1;
};

// Launch configuration of the H·v kernels (per vector type), set by
// hubbard_set_hv_config or hubbard_autotune; zeros mean "library default".
struct HvConfig {
    int rows = 0;     // rows of x staged per CTA group (1, 2 or 4)
    int threads = 0;  // threads per CTA (multiple of 32, <= 1024)
    int order = 1;    // 1: reverse Cuthill-McKee row visiting order, 0: storage order
    int split = 0;    // 1: row pass (diagonal + spin-down) then the column-blocked spin-up pass
    int up_block = 0;    // spin-up pass: columns per block (multiple of 32; 0 = 256)
    int up_threads = 0;  // spin-up pass: threads per CTA (multiple of up_block, <= 1024; 0 = 1024)
    int up_rows = 0;     // spin-up pass: rows per thread, 1, 2 or 4 (0 = 1)
};

struct KSpace;  // momentum-sector tables (pd_kspace.cu)

struct hb_basis {
    int L = 0, N_up = 0, N_dn = 0, n_bonds = 0;
    double U = 0.0;
    uint64_t D_up = 0, D_dn = 0, D = 0;
    int device = 0;
    int sm_count = 0;
    uint32_t *d_binom = nullptr;  // [PD_LUT_W * PD_LUT_W], C(i, m) at [i * PD_LUT_W + m]
    int32_t *d_bonds = nullptr;   // [n_bonds * 2]
    double *d_t = nullptr;        // [n_bonds]
    unsigned *d_err = nullptr;    // sticky error bits
    bool tables_built = false;
    bool same_spin_tables = false;  // N_up == N_dn: dn tables alias up tables
    SpinTables up, dn;
    // order in which the H·v visits the rows (spin-up strings): reverse
    // Cuthill-McKee over the spin-up hop graph, so that rows processed close in
    // time share hop neighbours and their x rows are still in L2
    uint32_t *d_row_order = nullptr;  // [D_up]
    HvConfig hv_cfg[3];               // indexed by hb_dtype
    int32_t *h_bonds = nullptr;
    double *h_t = nullptr;
    // fixed-point (HB_FX64) support
    bool fx_ok = false;          // <= PD_FX_MAXC distinct amplitudes and <= 255 bonds
    int fx_frac = 0;             // F: element q stands for q * 2^-F
    int n_classes = 0;
    double class_t[PD_FX_MAXC] = {0, 0, 0, 0};
    int32_t *d_bond_class = nullptr;  // [n_bonds]
    // momentum-space handle (Sec. IV A): L is the number of momenta, D the
    // sector dimension; H·v, ranks and rows go through pd_k_* below
    KSpace *ks = nullptr;
};

// ---- internal entry points shared between translation units ----
hb_status pd_build_tables(hb_handle h);
hb_status pd_apply(hb_handle h, hb_dtype dt, const void *x, void *y, cudaStream_t st);
// kernels one pd_apply launches under the handle's configuration for dt
int pd_hv_launches(hb_handle h, hb_dtype dt);
void pd_record_error(hb_handle h, hb_status s);
// momentum-space counterparts (pd_kspace.cu)
hb_status pd_k_apply(hb_handle h, hb_dtype dt, const void *x, void *y, cudaStream_t st);
hb_status pd_k_rank(hb_handle h, const uint64_t *states, uint64_t *idx, uint64_t n, cudaStream_t st);
hb_status pd_k_unrank(hb_handle h, const uint64_t *idx, uint64_t *states, uint64_t n, cudaStream_t st);
hb_status pd_k_row_entries(hb_handle h, uint64_t row0, uint32_t nrows, uint32_t max_entries, uint64_t *cols,
                           double *vals, uint32_t *counts, cudaStream_t st);
void pd_k_free(KSpace *ks);

hb_status pd_fx_coefs(hb_handle h, FxCoef *diag /*[PD_MAXL+1]*/, FxCoef *cls /*[PD_FX_MAXC]*/);

// Fixed-point multiply with rounding to nearest: round(a * K / 2^G), 1 <= G <= 63.
__device__ __forceinline__ int64_t fx_mul(int64_t a, int64_t K, int G) {
    int64_t hi = __mul64hi(a, K);
    const uint64_t lo = (uint64_t)a * (uint64_t)K;
    const uint64_t lo2 = lo + (1ull << (G - 1));
    hi += (lo2 < lo) ? 1 : 0;
    return (int64_t)((lo2 >> G) | ((uint64_t)hi << (64 - G)));
}

// Multiplier for a float64 value (device side, used for alpha, beta, 1/beta).
__device__ __forceinline__ FxCoef fx_coef_dev(double c) {
    FxCoef r;
    if (c == 0.0 || !(c == c)) return r;
    int e = 0;
    frexp(c, &e);
    int G = 62 - e;
    G = G < 1 ? 1 : (G > 63 ? 63 : G);
    r.G = G;
    r.K = __double2ll_rn(ldexp(c, G));
    return r;
}

// Binomial C(i, m) from a table laid out as above (0 when m > i).
__device__ __forceinline__ uint32_t pd_binom(const uint32_t *lut, int i, int m) {
    return lut[i * PD_LUT_W + m];
}

// Paradeisos forward map (Eq. 3): walk the set bits of s from the lowest,
// the k-th particle (k = 1, 2, ...) at position j contributing C(j, k).
__device__ __forceinline__ uint32_t pd_forward_map(const uint32_t *lut, uint32_t s) {
    uint32_t idx = 0;
    int m = 0;
    while (s) {
        const int j = __ffs(s) - 1;
        ++m;
        idx += pd_binom(lut, j, m);
        s &= s - 1;
    }
    return idx;
}

// Paradeisos backward map (Sec. III): scan positions from L-1 down; a particle
// sits at i when the remaining index is at least C(i, m), m the particles left.
__device__ __forceinline__ uint32_t pd_backward_map(const uint32_t *lut, uint32_t p, int n, int L) {
    uint32_t s = 0;
    int m = n;
    for (int i = L - 1; i >= 0 && m > 0; --i) {
        const uint32_t c = pd_binom(lut, i, m);
        if (p >= c) {
            s |= 1u << i;
            p -= c;
            --m;
        }
    }
    return s;
}

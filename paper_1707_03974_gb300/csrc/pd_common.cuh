// Shared definitions of the Paradeisos GB300 library (internal header).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "paradeisos.h"

#define PD_MAXL 32
#define PD_LUT_W (PD_MAXL + 1)  // binomial table is PD_LUT_W x PD_LUT_W
#define PD_INVALID UINT64_MAX

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
};

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
    int32_t *h_bonds = nullptr;
    double *h_t = nullptr;
};

// ---- internal entry points shared between translation units ----
hb_status pd_build_tables(hb_handle h);
hb_status pd_apply(hb_handle h, hb_dtype dt, const void *x, void *y, cudaStream_t st);
void pd_record_error(hb_handle h, hb_status s);

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

// Inversion-symmetric Paradeisos maps (Sec. IV B): index of the orbit
// {phi, F(phi)} of a string of n particles on an N-site chain, F(i) = N-1-i,
// in the order of the classification tree, and the representative of an index.
//
// At depth d the bits (N-1-d, d) classify a representative: (0,1) class A, a
// leaf whose inner N-2-2d bits (m-1 particles) are ranked by the standard
// forward map (Eq. 3); (0,0) class B and (1,1) class C recurse one level deeper
// (C with two particles fewer).  A precedes B precedes C at every depth, with
// counts C_{i-2}^{m-1} (the A leaf) and S_i^m = C_{i-2}^{m-1} + S_{i-2}^m +
// S_{i-2}^{m-2} (a subtree of i unclassified bits and m particles).  A string
// whose first unequal outer pair is (1, 0) is represented by its reversal.
#include <algorithm>
#include <new>
#include <vector>

#include "pd_common.cuh"
#include "paradeisos.h"

struct hb_inv {
    int N = 0, n = 0, device = 0, sm_count = 0;
    uint64_t D = 0;
    uint32_t *d_binom = nullptr;  // C(i, m) at [i * PD_LUT_W + m]
    uint64_t *d_S = nullptr;      // S(i, m) at [i * PD_LUT_W + m]
    unsigned *d_err = nullptr;
};

namespace {

constexpr int kThreads = 256;

int grid_for(uint64_t n, int sms) {
    return (int)std::max<uint64_t>(1, std::min<uint64_t>((n + kThreads - 1) / kThreads, (uint64_t)sms * 8));
}

__device__ __forceinline__ uint32_t cb(const uint32_t *lut, int i, int m) {
    return (m < 0 || i < 0) ? 0u : lut[i * PD_LUT_W + m];
}
__device__ __forceinline__ uint64_t sv(const uint64_t *S, int i, int m) {
    return (m < 0 || i < 0 || m > i) ? 0ull : S[i * PD_LUT_W + m];
}

__device__ __forceinline__ uint32_t reverse_bits(uint32_t s, int N) { return __brev(s) >> (32 - N); }

__global__ void k_inv_rank(const uint32_t *__restrict__ lut, const uint64_t *__restrict__ S, int N, int n,
                           const uint64_t *__restrict__ states, uint64_t *__restrict__ out, uint64_t cnt,
                           unsigned *err) {
    for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < cnt; e += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t s64 = states[e];
        if ((s64 >> N) != 0 || __popcll(s64) != n) {
            atomicOr(err, PD_ERRBIT(HB_ERR_INVALID_STATE));
            out[e] = UINT64_MAX;
            continue;
        }
        uint32_t s = (uint32_t)s64;
        // the representative: the first unequal outer pair must read (0, 1)
        for (int d = 0; d < N / 2; ++d) {
            const uint32_t hi = (s >> (N - 1 - d)) & 1u, lo = (s >> d) & 1u;
            if (hi != lo) {
                if (hi) s = reverse_bits(s, N);
                break;
            }
        }
        uint64_t idx = 0;
        int m = n;
        for (int d = 0; d < N / 2; ++d) {
            const int i = N - 2 * d;
            const uint32_t hi = (s >> (N - 1 - d)) & 1u, lo = (s >> d) & 1u;
            if (!hi && lo) {  // class A leaf
                const uint32_t inner = (s >> (d + 1)) & ((1u << (i - 2)) - 1u);
                idx += pd_forward_map(lut, inner);
                break;
            }
            if (!hi) {  // class B
                idx += cb(lut, i - 2, m - 1);
            } else {  // class C
                idx += cb(lut, i - 2, m - 1) + sv(S, i - 2, m);
                m -= 2;
            }
        }
        out[e] = idx;
    }
}

__global__ void k_inv_unrank(const uint32_t *__restrict__ lut, const uint64_t *__restrict__ S, int N, int n, uint64_t D,
                             const uint64_t *__restrict__ idx, uint64_t *__restrict__ out, uint64_t cnt, unsigned *err) {
    for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < cnt; e += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t p = idx[e];
        if (p >= D) {
            atomicOr(err, PD_ERRBIT(HB_ERR_OUT_OF_RANGE));
            out[e] = UINT64_MAX;
            continue;
        }
        uint32_t s = 0;
        int m = n;
        bool leaf = false;
        for (int d = 0; d < N / 2; ++d) {
            const int i = N - 2 * d;
            const uint64_t a = cb(lut, i - 2, m - 1), b = sv(S, i - 2, m);
            if (p >= a + b) {
                p -= a + b;
                s |= (1u << (N - 1 - d)) | (1u << d);
                m -= 2;
            } else if (p >= a) {
                p -= a;
            } else {
                s |= 1u << d;
                s |= pd_backward_map(lut, (uint32_t)p, m - 1, i - 2) << (d + 1);
                leaf = true;
                break;
            }
        }
        if (!leaf && (N & 1) && m == 1) s |= 1u << (N / 2);
        out[e] = s;
    }
}

}  // namespace

extern "C" {

hb_status paradeisos_inv_create(int N, int n, hb_inv_handle *out) {
    if (!out) return HB_ERR_INVALID_ARG;
    *out = nullptr;
    if (N < 1 || N > PD_MAXL || n < 0 || n > N) return HB_ERR_INVALID_ARG;
    hb_inv *h = new (std::nothrow) hb_inv();
    if (!h) return HB_ERR_NO_MEMORY;
    h->N = N;
    h->n = n;
    std::vector<uint32_t> lut((size_t)PD_LUT_W * PD_LUT_W, 0);
    for (int i = 0; i < PD_LUT_W; ++i) {
        uint64_t c = 1;
        for (int m = 0; m <= i; ++m) {
            lut[(size_t)i * PD_LUT_W + m] = (uint32_t)c;  // C(i, m) < 2^32 for i <= 32
            c = c * (uint64_t)(i - m) / (uint64_t)(m + 1);
        }
    }
    auto C = [&](int i, int m) -> uint64_t { return (m < 0 || i < 0 || m > i) ? 0 : lut[(size_t)i * PD_LUT_W + m]; };
    std::vector<uint64_t> S((size_t)PD_LUT_W * PD_LUT_W, 0);
    for (int i = 0; i <= N; ++i)
        for (int m = 0; m <= i; ++m) {
            uint64_t v;
            if (i == 0) v = m == 0;
            else if (i == 1) v = 1;
            else v = C(i - 2, m - 1) + S[(size_t)(i - 2) * PD_LUT_W + m] + (m >= 2 ? S[(size_t)(i - 2) * PD_LUT_W + m - 2] : 0);
            S[(size_t)i * PD_LUT_W + m] = v;
        }
    h->D = S[(size_t)N * PD_LUT_W + n];
    auto fail = [&](hb_status s) {
        paradeisos_inv_destroy(h);
        return s;
    };
    if (cudaGetDevice(&h->device) != cudaSuccess) return fail(HB_ERR_CUDA);
    if (cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess)
        return fail(HB_ERR_CUDA);
    if (cudaMalloc(&h->d_binom, lut.size() * 4) != cudaSuccess || cudaMalloc(&h->d_S, S.size() * 8) != cudaSuccess ||
        cudaMalloc(&h->d_err, sizeof(unsigned)) != cudaSuccess)
        return fail(HB_ERR_NO_MEMORY);
    if (cudaMemcpy(h->d_binom, lut.data(), lut.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(h->d_S, S.data(), S.size() * 8, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(h->d_err, 0, sizeof(unsigned)) != cudaSuccess)
        return fail(HB_ERR_CUDA);
    *out = h;
    return HB_OK;
}

hb_status paradeisos_inv_destroy(hb_inv_handle h) {
    if (!h) return HB_ERR_INVALID_ARG;
    cudaFree(h->d_binom);
    cudaFree(h->d_S);
    cudaFree(h->d_err);
    delete h;
    return HB_OK;
}

hb_status paradeisos_inv_dim(hb_inv_handle h, uint64_t *D) {
    if (!h || !D) return HB_ERR_INVALID_ARG;
    *D = h->D;
    return HB_OK;
}

hb_status paradeisos_inv_rank(hb_inv_handle h, const uint64_t *states, uint64_t *idx, uint64_t n, void *stream) {
    if (!h || (n > 0 && (!states || !idx))) return HB_ERR_INVALID_ARG;
    if (n == 0) return HB_OK;
    k_inv_rank<<<grid_for(n, h->sm_count), kThreads, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
        h->d_binom, h->d_S, h->N, h->n, states, idx, n, h->d_err);
    PD_CUDA(cudaGetLastError());
    return HB_OK;
}

hb_status paradeisos_inv_unrank(hb_inv_handle h, const uint64_t *idx, uint64_t *states, uint64_t n, void *stream) {
    if (!h || (n > 0 && (!states || !idx))) return HB_ERR_INVALID_ARG;
    if (n == 0) return HB_OK;
    k_inv_unrank<<<grid_for(n, h->sm_count), kThreads, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
        h->d_binom, h->d_S, h->N, h->n, h->D, idx, states, n, h->d_err);
    PD_CUDA(cudaGetLastError());
    return HB_OK;
}

hb_status paradeisos_inv_last_error(hb_inv_handle h) {
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

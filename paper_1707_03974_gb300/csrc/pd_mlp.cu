// Learned Lanczos start vector: a small multilayer perceptron over the 2L
// occupation bits of a basis state (not part of the paper; an addition that
// re-uses the method's own ground states as training data).
//
//   z1 = W1 x + b1, a1 = gelu(z1), z2 = W2 a1 + b2, a2 = gelu(z2), out = W3 a2 + b3
//   out = (log|psi|, sign logit),  hidden width 128, gelu in its tanh form
//   (Hendrycks & Gimpel 2016; tanh by the hardware's tanh.approx.f32).
//
// Weights are kept in float32 (master copy, Adam) and used as bfloat16; the two
// 128-wide matrix products of the forward pass, and the activation-gradient and
// weight-gradient products of the backward pass, run on the tensor cores
// through tcgen05.mma (bf16 x bf16 -> f32 in tensor memory, pd_tc.cuh).  The
// 2-wide output layer and the element-wise parts run on the CUDA cores.
#include <algorithm>
#include <cmath>
#include <new>
#include <type_traits>
#include <vector>

#include "pd_common.cuh"
#include "pd_tc.cuh"
#include "paradeisos_mlp.h"

namespace {

constexpr int kH = 128;    // hidden width
constexpr int kIn = 32;    // padded input width (2L <= 32)
constexpr int kBM = 128;   // GEMM tile rows (MMA M)
constexpr int kBK = 64;    // GEMM K chunk
constexpr uint32_t kWaitTries = 1u << 24;

// ---------------------------------------------------------------------------
// Generic tcgen05 GEMM:  C[M, N] (+)= A[M, K] * B[N, K]^T  (A, B bf16 row-major,
// K contiguous; C f32 row-major).  One CTA of 128 threads per 128 x BN tile and
// K range.  The K range is cut into slabs of kBK; slab i is copied to shared
// memory stage i % 2 in the core-matrix layout while the tensor core still
// runs the MMAs of slab i - 1 from the other stage (one thread issues them and
// commits them to the stage's mbarrier; a stage is refilled only after the
// MMAs that read it have completed).  The accumulator lives in tensor memory
// and the four warps read it back (warp w owns rows 32w .. 32w+31).  mode 0:
// C = acc, mode 1: atomicAdd(C, acc) (split K / accumulation).  Columns >=
// n_store are not written.  Dynamic shared memory: tc_gemm_smem(BN).
__host__ __device__ constexpr size_t tc_stage_bytes(int BN) { return (size_t)(kBM + BN) * kBK * 2; }
__host__ __device__ constexpr size_t tc_gemm_smem(int BN) { return 2 * tc_stage_bytes(BN) + 1024; }

template <int BN>
__global__ void __launch_bounds__(128) k_tc_gemm(const __nv_bfloat16 *__restrict__ A, int lda,
                                                 const __nv_bfloat16 *__restrict__ B, int ldb, float *C, int ldc,
                                                 int M, int N, int K, int k_per_cta, int n_store, int mode,
                                                 unsigned *err) {
    extern __shared__ __align__(1024) uint8_t smem_dyn[];
    // 1024-byte aligned base for the operand stages
    uint8_t *base = smem_dyn + ((1024 - (tc::smem_u32(smem_dyn) & 1023)) & 1023);
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ uint32_t tmem_slot;
    constexpr uint32_t kCols = BN < 32 ? 32 : BN;
    constexpr uint32_t kSBO = (kBK / 8) * 128;  // bytes between 8-row groups
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (warp == 0) tc::tmem_alloc(&tmem_slot, kCols);
    if (tid == 0) {
        tc::mbar_init(&bar[0], 1);
        tc::mbar_init(&bar[1], 1);
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_slot;
    const int m0 = blockIdx.x * kBM, n0 = blockIdx.y * BN;
    const int kb = blockIdx.z * k_per_cta, ke = min(K, kb + k_per_cta);
    const int nslab = ke > kb ? (ke - kb + kBK - 1) / kBK : 0;
    constexpr uint32_t idesc = tc::make_idesc_bf16(kBM, BN);
    uint32_t phase[2] = {0, 0};
    bool pending[2] = {false, false};
    bool ok = true;
    for (int i = 0; i < nslab && ok; ++i) {
        const int st = i & 1, k0 = kb + i * kBK;
        uint8_t *sA = base + st * tc_stage_bytes(BN), *sB = sA + (size_t)kBM * kBK * 2;
        if (pending[st]) {  // the MMAs of slab i - 2 read this stage: wait before refilling it
            ok = __syncthreads_and(tc::mbar_wait(&bar[st], phase[st], kWaitTries) ? 1 : 0) != 0;
            if (!ok) break;  // the stage stays pending
            phase[st] ^= 1;
            pending[st] = false;
            tc::fence_after_sync();
        }
        // 16-byte chunks: row r, K-group kc (8 elements)
        for (int c = tid; c < kBM * (kBK / 8); c += 128) {
            const int r = c / (kBK / 8), kc = c % (kBK / 8);
            const int gk = k0 + kc * 8, gr = m0 + r;
            uint4 v = make_uint4(0, 0, 0, 0);
            if (gr < M && gk + 8 <= ke) v = *reinterpret_cast<const uint4 *>(A + (size_t)gr * lda + gk);
            *reinterpret_cast<uint4 *>(sA + tc::core_off(r, kc * 8, kSBO)) = v;
        }
        for (int c = tid; c < BN * (kBK / 8); c += 128) {
            const int r = c / (kBK / 8), kc = c % (kBK / 8);
            const int gk = k0 + kc * 8, gr = n0 + r;
            uint4 v = make_uint4(0, 0, 0, 0);
            if (gr < N && gk + 8 <= ke) v = *reinterpret_cast<const uint4 *>(B + (size_t)gr * ldb + gk);
            *reinterpret_cast<uint4 *>(sB + tc::core_off(r, kc * 8, kSBO)) = v;
        }
        tc::fence_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after_sync();
            const uint32_t a0 = tc::smem_u32(sA), b0 = tc::smem_u32(sB);
#pragma unroll
            for (int ks = 0; ks < kBK / 16; ++ks) {
                const uint64_t ad = tc::make_desc(a0 + ks * 256, 128, kSBO);
                const uint64_t bd = tc::make_desc(b0 + ks * 256, 128, kSBO);
                tc::mma_bf16(tmem, ad, bd, idesc, (i > 0 || ks > 0) ? 1u : 0u);
            }
            tc::commit(&bar[st]);
        }
        pending[st] = true;
    }
    // the last commits: the accumulator is complete once every issued MMA has finished
    for (int q = 0; q < 2 && ok; ++q) {
        const int st = (nslab + q) & 1;  // older pending stage first
        if (!pending[st]) continue;
        ok = __syncthreads_and(tc::mbar_wait(&bar[st], phase[st], kWaitTries) ? 1 : 0) != 0;
        if (!ok) break;
        phase[st] ^= 1;
        pending[st] = false;
    }
    tc::fence_after_sync();
    if (!ok) {
        // a wait gave up: record it, then wait (bounded) once more on every stage still pending,
        // so that no MMA still writes the tensor memory released below
        if (tid == 0) atomicOr(err, PD_ERRBIT(HB_ERR_TIMEOUT));
        for (int st = 0; st < 2; ++st)
            if (pending[st]) tc::mbar_wait(&bar[st], phase[st], kWaitTries);
        __syncthreads();
    }
    if (ok && nslab > 0) {
        const int row = m0 + warp * 32 + lane;
#pragma unroll 1
        for (int c0 = 0; c0 < BN; c0 += 32) {
            float v[32];
            tc::tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
            if (row < M) {
                float *crow = C + (size_t)row * ldc + n0 + c0;
#pragma unroll
                for (int i = 0; i < 32; ++i) {
                    const int col = n0 + c0 + i;
                    if (col < n_store) {
                        if (mode == 0) crow[i] = v[i];
                        else atomicAdd(crow + i, v[i]);
                    }
                }
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, kCols);
}

// ---------------------------------------------------------------------------
// element-wise kernels

// GELU in its tanh form (Hendrycks & Gimpel, "Gaussian Error Linear Units",
// 2016):  gelu(x) = x/2 (1 + tanh(u)),  u = sqrt(2/pi) (x + 0.044715 x^3),
// with tanh from the SM's tanh.approx.f32 instruction (relative error about
// 2^-11, far inside the bfloat16 rounding, 2^-9 relative, that every
// activation then goes through).  Four float32 operations and one
// special-function instruction per activation.  The derivative is the exact
// derivative of the same form:
//   gelu'(x) = (1 + tanh u)/2 + x/2 (1 - tanh^2 u) sqrt(2/pi) (1 + 3 * 0.044715 x^2).
constexpr float kGeluC1 = 0.7978845608f;   // sqrt(2/pi)
constexpr float kGeluC3 = 0.0356774081f;   // 0.044715 sqrt(2/pi)
constexpr float kGeluD3 = 0.1070322244f;   // 3 * 0.044715 sqrt(2/pi)
__device__ __forceinline__ float tanh_hw(float x) {
    float y;
    asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float gelu_f(float x) {
    const float hx = 0.5f * x;
    return fmaf(hx, tanh_hw(x * fmaf(kGeluC3, x * x, kGeluC1)), hx);
}
// Blackwell's paired float32 instructions (fma/mul/add .rn.f32x2): two float32
// operations per instruction, each half rounded exactly as the scalar
// instruction rounds it.  A pair lives in one 64-bit register.
__device__ __forceinline__ unsigned long long f2_pack(float a, float b) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ float2 f2_unpack(unsigned long long r) {
    float2 v;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(v.x), "=f"(v.y) : "l"(r));
    return v;
}
__device__ __forceinline__ unsigned long long f2_add(unsigned long long a, unsigned long long b) {
    unsigned long long d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ unsigned long long f2_mul(unsigned long long a, unsigned long long b) {
    unsigned long long d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ unsigned long long f2_fma(unsigned long long a, unsigned long long b,
                                                     unsigned long long c) {
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
// gelu of both halves, each bit for bit gelu_f (the same operations in the same order)
__device__ __forceinline__ unsigned long long gelu_f2(unsigned long long x) {
    const unsigned long long u =
        f2_mul(x, f2_fma(f2_pack(kGeluC3, kGeluC3), f2_mul(x, x), f2_pack(kGeluC1, kGeluC1)));
    const float2 uu = f2_unpack(u);
    const unsigned long long hx = f2_mul(f2_pack(0.5f, 0.5f), x);
    return f2_fma(hx, f2_pack(tanh_hw(uu.x), tanh_hw(uu.y)), hx);
}
__device__ __forceinline__ float gelu_grad_f(float x) {
    const float x2 = x * x;
    const float th = tanh_hw(x * fmaf(kGeluC3, x2, kGeluC1));
    return fmaf(0.5f * x * fmaf(-th, th, 1.0f), fmaf(kGeluD3, x2, kGeluC1), 0.5f * (1.0f + th));
}

// y = gelu(x) (deriv 0) or gelu'(x) (deriv 1): the activation as the network's kernels evaluate it
__global__ void k_activation(const float *__restrict__ x, uint64_t n, float *__restrict__ y, int deriv) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        y[i] = deriv ? gelu_grad_f(x[i]) : gelu_f(x[i]);
}

// x rows: bit i of the combined state -> column i (0/1), columns >= n_bits zero.
__global__ void k_bits(const uint64_t *__restrict__ states, uint64_t n, uint64_t n_pad, int n_bits,
                       __nv_bfloat16 *__restrict__ X) {
    for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < n_pad * kIn; e += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t r = e / kIn;
        const int i = (int)(e % kIn);
        float v = 0.f;
        if (r < n && i < n_bits) v = (float)((states[r] >> i) & 1ull);
        X[e] = __float2bfloat16_rn(v);
    }
}

// Combined states of basis indices idx0 .. idx0+n-1 from the per-spin tables (backward map).
__global__ void k_states_of_range(const uint32_t *__restrict__ str_up, const uint32_t *__restrict__ str_dn,
                                  uint64_t D_dn, int L, uint64_t idx0, uint64_t n, uint64_t *__restrict__ out) {
    for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < n; e += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t I = idx0 + e;
        const uint64_t u = I / D_dn, d = I - u * D_dn;
        out[e] = ((uint64_t)str_up[u] << L) | (uint64_t)str_dn[d];
    }
}

// A1 = bf16(gelu(Z1 + b1))
__global__ void k_bias_gelu_bf16(const float *__restrict__ Z, const float *__restrict__ b, uint64_t rows,
                                 __nv_bfloat16 *__restrict__ Aout) {
    for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < rows * kH; e += (uint64_t)gridDim.x * blockDim.x)
        Aout[e] = __float2bfloat16_rn(gelu_f(Z[e] + b[e % kH]));
}

// out[r] = W3 gelu(Z2[r] + b2) + b3  (W3 used at bfloat16 precision)
__global__ void k_output(const float *__restrict__ Z2, const float *__restrict__ b2, const float *__restrict__ W3,
                         const float *__restrict__ b3, uint64_t n, float *__restrict__ out) {
    __shared__ float s_w3[2 * kH], s_b2[kH];
    for (int i = threadIdx.x; i < 2 * kH; i += blockDim.x) s_w3[i] = __bfloat162float(__float2bfloat16_rn(W3[i]));
    for (int i = threadIdx.x; i < kH; i += blockDim.x) s_b2[i] = b2[i];
    __syncthreads();
    for (uint64_t r = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; r < n; r += (uint64_t)gridDim.x * blockDim.x) {
        const float *z = Z2 + r * kH;
        float o0 = b3[0], o1 = b3[1];
        for (int h = 0; h < kH; ++h) {
            const float a = gelu_f(z[h] + s_b2[h]);
            o0 = fmaf(s_w3[h], a, o0);
            o1 = fmaf(s_w3[kH + h], a, o1);
        }
        out[2 * r] = o0;
        out[2 * r + 1] = o1;
    }
}

// Backward through the output layer.  wts are the normalised sample weights.
// Writes dZ2 (bf16, rows x 128) and its transpose (128 x n_pad), accumulates
// gW3, gb3, gb2 and the loss into grad / loss.
__global__ void k_output_back(const float *__restrict__ Z2, const float *__restrict__ b2, const float *__restrict__ W3,
                              const float *__restrict__ out, const float *__restrict__ t_log,
                              const float *__restrict__ t_sign, const float *__restrict__ wts, float lam, uint64_t n,
                              uint64_t n_pad, __nv_bfloat16 *__restrict__ dZ2, __nv_bfloat16 *__restrict__ dZ2T,
                              float *__restrict__ gW3, float *__restrict__ gb3, float *__restrict__ gb2,
                              float *__restrict__ loss) {
    __shared__ float s_w3[2 * kH], s_b2[kH], s_g[3 * kH + 2];
    for (int i = threadIdx.x; i < 2 * kH; i += blockDim.x) s_w3[i] = __bfloat162float(__float2bfloat16_rn(W3[i]));
    for (int i = threadIdx.x; i < kH; i += blockDim.x) s_b2[i] = b2[i];
    for (int i = threadIdx.x; i < 3 * kH + 2; i += blockDim.x) s_g[i] = 0.f;
    __syncthreads();
    float my_loss = 0.f;
    for (uint64_t r = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; r < n_pad; r += (uint64_t)gridDim.x * blockDim.x) {
        if (r >= n) {
            for (int h = 0; h < kH; ++h) {
                dZ2[r * kH + h] = __float2bfloat16_rn(0.f);
                dZ2T[(uint64_t)h * n_pad + r] = __float2bfloat16_rn(0.f);
            }
            continue;
        }
        const float w = wts[r];
        const float e = out[2 * r] - t_log[r];
        const float m = -t_sign[r] * out[2 * r + 1];
        my_loss += w * (e * e + lam * (m > 20.f ? m : log1pf(__expf(m))));
        const float d0 = w * 2.f * e;
        const float d1 = w * lam * (-t_sign[r]) / (1.f + __expf(-m));
        atomicAdd(&s_g[3 * kH], d0);
        atomicAdd(&s_g[3 * kH + 1], d1);
        for (int h = 0; h < kH; ++h) {
            const float z = Z2[r * kH + h] + s_b2[h];
            const float a = gelu_f(z);
            atomicAdd(&s_g[h], d0 * a);
            atomicAdd(&s_g[kH + h], d1 * a);
            const float dz = (d0 * s_w3[h] + d1 * s_w3[kH + h]) * gelu_grad_f(z);
            atomicAdd(&s_g[2 * kH + h], dz);
            const __nv_bfloat16 bz = __float2bfloat16_rn(dz);
            dZ2[r * kH + h] = bz;
            dZ2T[(uint64_t)h * n_pad + r] = bz;
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 2 * kH; i += blockDim.x) atomicAdd(&gW3[i], s_g[i]);
    for (int i = threadIdx.x; i < kH; i += blockDim.x) atomicAdd(&gb2[i], s_g[2 * kH + i]);
    if (threadIdx.x < 2) atomicAdd(&gb3[threadIdx.x], s_g[3 * kH + threadIdx.x]);
    for (int o = 16; o > 0; o >>= 1) my_loss += __shfl_down_sync(0xffffffffu, my_loss, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss, my_loss);
}

// dZ1 = dA1 * gelu'(Z1 + b1) -> transpose (128 x n_pad, bf16); gb1 += column sums.
__global__ void k_hidden_back(const float *__restrict__ dA1, const float *__restrict__ Z1, const float *__restrict__ b1,
                              uint64_t n, uint64_t n_pad, __nv_bfloat16 *__restrict__ dZ1T, float *__restrict__ gb1) {
    __shared__ float s_g[kH];
    for (int i = threadIdx.x; i < kH; i += blockDim.x) s_g[i] = 0.f;
    __syncthreads();
    for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < n_pad * kH; e += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t r = e / kH;
        const int h = (int)(e % kH);
        float dz = 0.f;
        if (r < n) {
            dz = dA1[e] * gelu_grad_f(Z1[e] + b1[h]);
            atomicAdd(&s_g[h], dz);
        }
        dZ1T[(uint64_t)h * n_pad + r] = __float2bfloat16_rn(dz);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kH; i += blockDim.x) atomicAdd(&gb1[i], s_g[i]);
}

// (rows x cols) bf16 -> (cols x rows) bf16
__global__ void k_transpose_bf16(const __nv_bfloat16 *__restrict__ a, uint64_t rows, int cols,
                                 __nv_bfloat16 *__restrict__ at) {
    for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < rows * cols; e += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t r = e / cols;
        const int c = (int)(e % cols);
        at[(uint64_t)c * rows + r] = a[e];
    }
}

// master f32 parameters -> bf16 operands (W1 padded to 128 x 32, W2 and its transpose)
__global__ void k_refresh_bf16(const float *__restrict__ W1, const float *__restrict__ W2, int n_in,
                               __nv_bfloat16 *__restrict__ W1b, __nv_bfloat16 *__restrict__ W2b,
                               __nv_bfloat16 *__restrict__ W2tb) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < kH * kH; e += gridDim.x * blockDim.x) {
        const int o = e / kH, i = e % kH;
        const __nv_bfloat16 v = __float2bfloat16_rn(W2[e]);
        W2b[e] = v;
        W2tb[i * kH + o] = v;
        if (e < kH * kIn) {
            const int oo = e / kIn, ii = e % kIn;
            W1b[e] = __float2bfloat16_rn(ii < n_in ? W1[oo * n_in + ii] : 0.f);
        }
    }
}

__global__ void k_adam(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m, float *__restrict__ v,
                       uint64_t n, float lr, float b1, float b2, float eps, float c1, float c2) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

// start vector entries: v = sign * exp(min(out0, 10) - 10)

// start value of one state: sign(out1) exp(min(out0, 10) - 10), in T (fixed
// point: scaled by 2^(F-1))
template <typename T>
__device__ __forceinline__ T start_value(float out0, float out1, int F) {
    const float a = __expf(fminf(out0, 10.f) - 10.f);
    const float s = out1 >= 0.f ? a : -a;
    if constexpr (sizeof(T) == 8 && !std::is_floating_point<T>::value)
        return (T)__double2ll_rn(ldexp((double)s, F - 1));
    else
        return (T)s;
}

// ---------------------------------------------------------------------------
// Fused inference for the start vector: one persistent CTA of 128 threads per
// 128-state tile.  Thread t builds row t of the occupation-bit tile X (from the
// per-spin strings of basis index I, i.e. the backward map's tables), thread 0
// issues Z1 = X W1^T (K = 32) into tensor-memory columns 0..127; each thread
// reads its row back, applies bias + GELU, rounds to bf16 and writes it as row
// t of the A operand of Z2 = A1 W2^T (K = 128, columns 128..255); the second
// epilogue applies bias + GELU, the 2 x 128 output layer and the start-value
// map and stores only v[I].  The weights stay in shared memory for the CTA's
// lifetime; nothing of size D but v touches HBM.  Per element the arithmetic
// is that of mlp_forward followed by the start-value map.
struct InferSmem {
    uint8_t W1[kH * kIn * 2];  // B operand of layer 1, core-matrix layout (K = 32)
    uint8_t W2[kH * kH * 2];   // B operand of layer 2 (K = 128)
    uint8_t X[kBM * kIn * 2];  // A operand of layer 1
    uint8_t A1[kBM * kH * 2];  // A operand of layer 2
    float b1[kH], b2[kH], w3[2 * kH], b3[2];
    float red[2][kBM];  // output-layer partial sums of the second column half
    uint64_t bar;
    uint32_t tmem;
};

// Threads of the fused start-vector kernel: two warpgroups.  Warp w reads the
// tensor-memory lanes 32 (w mod 4) .. + 31 (the rows of its quarter of the tile)
// and takes the hidden columns of half w / 4, so each row's 128 columns are
// split over two warps and each SM keeps twice as many warps on the epilogues.
constexpr int kStartThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kStartThreads) k_mlp_start(const __nv_bfloat16 *__restrict__ W1b,
                                                   const __nv_bfloat16 *__restrict__ W2b,
                                                   const float *__restrict__ params, uint64_t ob1, uint64_t ob2,
                                                   uint64_t oW3, uint64_t ob3, const uint32_t *__restrict__ str_up,
                                                   const uint32_t *__restrict__ str_dn, uint64_t D_dn, uint64_t D,
                                                   int L, int n_bits, T *__restrict__ v, int F, unsigned *err) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    InferSmem &S = *reinterpret_cast<InferSmem *>(smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5;
    const int row = tid & (kBM - 1), half = tid / kBM;  // tile row of this thread, hidden-column half
    constexpr uint32_t kSBO1 = (kIn / 8) * 128, kSBO2 = (kH / 8) * 128;
    constexpr int kHalfCols = kH / 2;
    // weights and biases, once per CTA
    for (int c = tid; c < kH * (kIn / 8); c += kStartThreads) {
        const int r = c / (kIn / 8), kc = c % (kIn / 8);
        *reinterpret_cast<uint4 *>(S.W1 + tc::core_off(r, kc * 8, kSBO1)) =
            *reinterpret_cast<const uint4 *>(W1b + (size_t)r * kIn + kc * 8);
    }
    for (int c = tid; c < kH * (kH / 8); c += kStartThreads) {
        const int r = c / (kH / 8), kc = c % (kH / 8);
        *reinterpret_cast<uint4 *>(S.W2 + tc::core_off(r, kc * 8, kSBO2)) =
            *reinterpret_cast<const uint4 *>(W2b + (size_t)r * kH + kc * 8);
    }
    for (int i = tid; i < kH; i += kStartThreads) {
        S.b1[i] = params[ob1 + i];
        S.b2[i] = params[ob2 + i];
        S.w3[i] = __bfloat162float(__float2bfloat16_rn(params[oW3 + i]));
        S.w3[kH + i] = __bfloat162float(__float2bfloat16_rn(params[oW3 + kH + i]));
    }
    if (tid < 2) S.b3[tid] = params[ob3 + tid];
    if (warp == 0) tc::tmem_alloc(&S.tmem, 256);
    if (tid == 0) tc::mbar_init(&S.bar, 1);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = S.tmem;
    const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
    uint32_t phase = 0;
    bool ok = true;
    const uint64_t ntiles = (D + kBM - 1) / kBM;
    for (uint64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        const int t = row;
        const uint64_t I = tile * kBM + t;
        // row t of X: the occupation bits of basis state I (zero rows past the end), built by the
        // first warpgroup
        uint64_t state = 0;
        if (half == 0 && I < D) {
            const uint64_t u = I / D_dn, d = I - u * D_dn;
            state = ((uint64_t)str_up[u] << L) | (uint64_t)str_dn[d];
        }
#pragma unroll
        for (int q = 0; q < kIn / 8; ++q) {
            if (half != 0) break;
            uint32_t w4[4];
#pragma unroll
            for (int p2 = 0; p2 < 4; ++p2) {
                const int i0 = q * 8 + 2 * p2;
                const uint32_t lo = (i0 < n_bits && ((state >> i0) & 1ull)) ? 0x3F80u : 0u;  // bf16 1.0
                const uint32_t hi = (i0 + 1 < n_bits && ((state >> (i0 + 1)) & 1ull)) ? 0x3F80u : 0u;
                w4[p2] = lo | (hi << 16);
            }
            *reinterpret_cast<uint4 *>(S.X + tc::core_off(t, q * 8, kSBO1)) = make_uint4(w4[0], w4[1], w4[2], w4[3]);
        }
        tc::fence_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after_sync();
            constexpr uint32_t idesc = tc::make_idesc_bf16(kBM, kH);
            const uint32_t x0 = tc::smem_u32(S.X), w0 = tc::smem_u32(S.W1);
#pragma unroll
            for (int ks = 0; ks < kIn / 16; ++ks)
                tc::mma_bf16(tmem, tc::make_desc(x0 + ks * 256, 128, kSBO1), tc::make_desc(w0 + ks * 256, 128, kSBO1),
                             idesc, ks > 0 ? 1u : 0u);
            tc::commit(&S.bar);
        }
        ok = __syncthreads_and(tc::mbar_wait(&S.bar, phase, kWaitTries) ? 1 : 0) != 0;
        if (!ok) break;
        phase ^= 1;
        tc::fence_after_sync();
        // epilogue 1: A1[t, :] = bf16(gelu(Z1[t, :] + b1)), this thread's column half
#pragma unroll 1
        for (int c0 = half * kHalfCols; c0 < (half + 1) * kHalfCols; c0 += 32) {
            float z[32];
            tc::tmem_ld32(tmem + lane_base + (uint32_t)c0, z);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                uint32_t w4[4];
#pragma unroll
                for (int p2 = 0; p2 < 4; ++p2) {
                    const int i = q * 8 + 2 * p2;
                    const float2 g = f2_unpack(gelu_f2(
                        f2_add(f2_pack(z[i], z[i + 1]), *reinterpret_cast<const unsigned long long *>(S.b1 + c0 + i))));
                    const __nv_bfloat16 a = __float2bfloat16_rn(g.x);
                    const __nv_bfloat16 b = __float2bfloat16_rn(g.y);
                    w4[p2] = (uint32_t)__bfloat16_as_ushort(a) | ((uint32_t)__bfloat16_as_ushort(b) << 16);
                }
                *reinterpret_cast<uint4 *>(S.A1 + tc::core_off(t, c0 + q * 8, kSBO2)) =
                    make_uint4(w4[0], w4[1], w4[2], w4[3]);
            }
        }
        tc::fence_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after_sync();
            constexpr uint32_t idesc = tc::make_idesc_bf16(kBM, kH);
            const uint32_t a0 = tc::smem_u32(S.A1), w0 = tc::smem_u32(S.W2);
#pragma unroll
            for (int ks = 0; ks < kH / 16; ++ks)
                tc::mma_bf16(tmem + kH, tc::make_desc(a0 + ks * 256, 128, kSBO2),
                             tc::make_desc(w0 + ks * 256, 128, kSBO2), idesc, ks > 0 ? 1u : 0u);
            tc::commit(&S.bar);
        }
        ok = __syncthreads_and(tc::mbar_wait(&S.bar, phase, kWaitTries) ? 1 : 0) != 0;
        if (!ok) break;
        phase ^= 1;
        tc::fence_after_sync();
        // epilogue 2: output layer (W3 at bf16 precision, as mlp_forward) and the start value;
        // paired instructions: even and odd hidden units sum in the two halves of a register
        unsigned long long p0 = 0ull, p1 = 0ull;  // (+0.0f, +0.0f)
#pragma unroll 1
        for (int c0 = half * kHalfCols; c0 < (half + 1) * kHalfCols; c0 += 32) {
            float z[32];
            tc::tmem_ld32(tmem + lane_base + (uint32_t)(kH + c0), z);
#pragma unroll
            for (int i = 0; i < 32; i += 2) {
                const unsigned long long a = gelu_f2(
                    f2_add(f2_pack(z[i], z[i + 1]), *reinterpret_cast<const unsigned long long *>(S.b2 + c0 + i)));
                p0 = f2_fma(*reinterpret_cast<const unsigned long long *>(S.w3 + c0 + i), a, p0);
                p1 = f2_fma(*reinterpret_cast<const unsigned long long *>(S.w3 + kH + c0 + i), a, p1);
            }
        }
        const float2 q0 = f2_unpack(p0), q1 = f2_unpack(p1);
        if (half == 1) {
            S.red[0][t] = q0.x + q0.y;
            S.red[1][t] = q1.x + q1.y;
        }
        tc::fence_before_sync();  // this tile's tensor-memory reads precede the next tile's MMAs
        __syncthreads();
        if (half == 0 && I < D) {
            const float o0 = S.b3[0] + ((q0.x + q0.y) + S.red[0][t]);
            const float o1 = S.b3[1] + ((q1.x + q1.y) + S.red[1][t]);
            v[I] = start_value<T>(o0, o1, F);
        }
    }
    if (!ok) {
        // gave up waiting: record it, then drain (bounded) so no MMA still writes the
        // tensor memory released below
        if (tid == 0) atomicOr(err, PD_ERRBIT(HB_ERR_TIMEOUT));
        tc::mbar_wait(&S.bar, phase, kWaitTries);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, 256);
}
int grid_of(uint64_t n, int sms) { return (int)std::max<uint64_t>(1, std::min<uint64_t>((n + 255) / 256, (uint64_t)sms * 8)); }

// ---------------------------------------------------------------------------
// Training samples: basis states drawn with probability psi^2 (inverse-CDF
// sampling over the whole basis).  psi is cut into blocks of kSampBlock
// entries; the float64 block sums of psi^2 are scanned into block offsets, a
// draw u in [0, total) picks its block by binary search and its entry by a
// warp-wide scan inside the block.  The draws are SplitMix64 outputs (Steele,
// Lea & Flood 2014), draw i = output i + 1 of the stream seeded with `seed`,
// mapped to (z >> 11) 2^-53 in [0, 1).  The global sign is fixed so that the
// entry of largest |psi| (lowest index on ties) is positive.
constexpr int kSampBlock = 1024;
constexpr uint64_t kGammaS = 0x9E3779B97F4A7C15ull;

__device__ __forceinline__ double splitmix_unit(uint64_t seed, uint64_t i) {
    uint64_t z = seed + (i + 1) * kGammaS;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z = z ^ (z >> 31);
    return (double)(z >> 11) * 0x1.0p-53;
}

// (value, index) of the larger |psi|, the lower index on ties
__device__ __forceinline__ void argmax_merge(float &a, uint64_t &ia, float b, uint64_t ib) {
    if (b > a || (b == a && ib < ia)) {
        a = b;
        ia = ib;
    }
}

// one CTA per block: sum of psi^2 in float64 (fixed tree order) and the block's argmax |psi|
__global__ void __launch_bounds__(256) k_samp_blocks(const float *__restrict__ psi, uint64_t D, double *bsum,
                                                     float *bmax, uint64_t *bidx) {
    __shared__ double s_sum[8];
    __shared__ float s_max[8];
    __shared__ uint64_t s_idx[8];
    const uint64_t b = blockIdx.x, e0 = b * kSampBlock;
    double acc = 0.0;
    float mx = -1.f;
    uint64_t mi = UINT64_MAX;
    for (int k = threadIdx.x; k < kSampBlock; k += blockDim.x) {
        const uint64_t e = e0 + k;
        if (e < D) {
            const double v = psi[e];
            acc = fma(v, v, acc);
            argmax_merge(mx, mi, fabsf(psi[e]), e);
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        acc += __shfl_down_sync(0xffffffffu, acc, o);
        const float m2 = __shfl_down_sync(0xffffffffu, mx, o);
        const uint64_t i2 = __shfl_down_sync(0xffffffffu, mi, o);
        argmax_merge(mx, mi, m2, i2);
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) {
        s_sum[w] = acc;
        s_max[w] = mx;
        s_idx[w] = mi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        float m = -1.f;
        uint64_t i = UINT64_MAX;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
            t += s_sum[k];
            argmax_merge(m, i, s_max[k], s_idx[k]);
        }
        bsum[b] = t;
        bmax[b] = m;
        bidx[b] = i;
    }
}

// one CTA: bsum -> exclusive prefix (in place), total, and the global sign of psi
__global__ void __launch_bounds__(1024) k_samp_scan(double *bsum, const float *bmax, const uint64_t *bidx,
                                                    uint64_t nblk, const float *__restrict__ psi, double *misc) {
    __shared__ double s_part[1024];
    __shared__ float s_max[1024];
    __shared__ uint64_t s_idx[1024];
    const uint64_t per = (nblk + blockDim.x - 1) / blockDim.x;
    const uint64_t b0 = min(nblk, threadIdx.x * per), b1 = min(nblk, b0 + per);
    double t = 0.0;
    float m = -1.f;
    uint64_t mi = UINT64_MAX;
    for (uint64_t b = b0; b < b1; ++b) {
        t += bsum[b];
        argmax_merge(m, mi, bmax[b], bidx[b]);
    }
    s_part[threadIdx.x] = t;
    s_max[threadIdx.x] = m;
    s_idx[threadIdx.x] = mi;
    __syncthreads();
    if (threadIdx.x == 0) {  // sequential scan of 1024 partials: fixed order
        double run = 0.0;
        float gm = -1.f;
        uint64_t gi = UINT64_MAX;
        for (int k = 0; k < (int)blockDim.x; ++k) {
            const double pk = s_part[k];
            s_part[k] = run;
            run += pk;
            argmax_merge(gm, gi, s_max[k], s_idx[k]);
        }
        misc[0] = run;                                         // total
        misc[1] = (gi != UINT64_MAX && psi[gi] < 0.f) ? -1.0 : 1.0;  // global sign
    }
    __syncthreads();
    double run = s_part[threadIdx.x];
    for (uint64_t b = b0; b < b1; ++b) {
        const double pb = bsum[b];
        bsum[b] = run;
        run += pb;
    }
}

// one warp per sample: block by binary search over the offsets, entry by a warp scan in the block
__global__ void __launch_bounds__(256) k_samp_draw(const float *__restrict__ psi, uint64_t D, const double *bpre,
                                                   uint64_t nblk, const double *misc, uint64_t n, uint64_t seed,
                                                   const uint32_t *__restrict__ str_up,
                                                   const uint32_t *__restrict__ str_dn, uint64_t D_dn, int L,
                                                   uint64_t *states, double *logs, float *t_sign) {
    const int lane = threadIdx.x & 31;
    const uint64_t warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const double total = misc[0], gsign = misc[1];
    for (uint64_t i = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5; i < n; i += warps) {
        const double u = splitmix_unit(seed, i) * total;
        uint64_t lo = 0, hi = nblk - 1;  // largest b with bpre[b] <= u
        while (lo < hi) {
            const uint64_t mid = (lo + hi + 1) >> 1;
            if (bpre[mid] <= u) lo = mid; else hi = mid - 1;
        }
        const uint64_t e0 = lo * kSampBlock;
        const double r = u - bpre[lo];
        // lane l covers entries e0 + 32 l .. e0 + 32 l + 31
        double part = 0.0;
        for (int k = 0; k < 32; ++k) {
            const uint64_t e = e0 + (uint64_t)lane * 32 + k;
            if (e < D) {
                const double v = psi[e];
                part = fma(v, v, part);
            }
        }
        double incl = part;
        for (int o = 1; o < 32; o <<= 1) {
            const double t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        const double excl = incl - part;
        const unsigned hit = __ballot_sync(0xffffffffu, incl > r);
        // the lane whose range holds r (rounding can leave r past the last sum: take the last lane)
        const int owner = hit ? __ffs(hit) - 1 : 31;
        uint64_t idx = UINT64_MAX;
        if (lane == owner) {
            double run = excl;
            uint64_t last = UINT64_MAX;
            for (int k = 0; k < 32; ++k) {
                const uint64_t e = e0 + (uint64_t)lane * 32 + k;
                if (e >= D) break;
                const double v = psi[e];
                if (v != 0.0) last = e;
                run = fma(v, v, run);
                if (run > r && v != 0.0) {
                    idx = e;
                    break;
                }
            }
            if (idx == UINT64_MAX) idx = last;
        }
        idx = __shfl_sync(0xffffffffu, idx, owner);
        if (idx == UINT64_MAX) {  // an all-zero stretch: the block's last nonzero entry below
            for (uint64_t e = min(D, e0 + kSampBlock); e > 0 && idx == UINT64_MAX; --e)
                if (psi[e - 1] != 0.f) idx = e - 1;
            if (idx == UINT64_MAX) idx = 0;
        }
        if (lane == 0) {
            const uint64_t uu = idx / D_dn, dd = idx - uu * D_dn;
            states[i] = ((uint64_t)str_up[uu] << L) | (uint64_t)str_dn[dd];
            const double amp = gsign * (double)psi[idx];
            logs[i] = log(fabs(amp) > 0.0 ? fabs(amp) : 1e-300);
            t_sign[i] = amp >= 0.0 ? 1.f : -1.f;
        }
    }
}

// t_log = logs - mean(logs), mean in float64 over a fixed order (one CTA)
__global__ void __launch_bounds__(1024) k_samp_center(const double *logs, uint64_t n, float *t_log) {
    __shared__ double s_w[32];
    __shared__ double s_mean;
    double acc = 0.0;
    for (uint64_t i = threadIdx.x; i < n; i += blockDim.x) acc += logs[i];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += s_w[k];
        s_mean = t / (double)n;
    }
    __syncthreads();
    for (uint64_t i = threadIdx.x; i < n; i += blockDim.x) t_log[i] = (float)(logs[i] - s_mean);
}

uint64_t align256u(uint64_t x) { return (x + 255) & ~255ull; }

void samp_layout(uint64_t D, uint64_t n, uint64_t *o_bmax, uint64_t *o_bidx, uint64_t *o_logs, uint64_t *o_misc,
                 uint64_t *total) {
    const uint64_t nblk = (D + kSampBlock - 1) / kSampBlock;
    *o_bmax = align256u(nblk * 8);
    *o_bidx = *o_bmax + align256u(nblk * 4);
    *o_logs = *o_bidx + align256u(nblk * 8);
    *o_misc = *o_logs + align256u(n * 8);
    *total = *o_misc + 256;
}

}  // namespace

struct hb_mlp {
    int n_in = 32, device = 0, sm_count = 0;
    uint64_t P = 0;
    float *d_p = nullptr, *d_m = nullptr, *d_v = nullptr, *d_g = nullptr, *d_loss = nullptr;
    __nv_bfloat16 *W1b = nullptr, *W2b = nullptr, *W2tb = nullptr;
    unsigned *d_err = nullptr;
    // batch workspace
    uint64_t cap = 0;
    __nv_bfloat16 *X = nullptr, *XT = nullptr, *A1 = nullptr, *A1T = nullptr, *dZ2 = nullptr, *dZ2T = nullptr,
                  *dZ1T = nullptr;
    float *Z1 = nullptr, *Z2 = nullptr, *dA1 = nullptr, *out = nullptr;
    uint64_t *states = nullptr;
    int adam_t = 0;
    // offsets of the parameter blocks (float32 master vector, oracle layout)
    uint64_t oW1 = 0, ob1 = 0, oW2 = 0, ob2 = 0, oW3 = 0, ob3 = 0;
};

namespace {

void free_ws(hb_mlp *m) {
    cudaFree(m->X); cudaFree(m->XT); cudaFree(m->A1); cudaFree(m->A1T); cudaFree(m->dZ2); cudaFree(m->dZ2T);
    cudaFree(m->dZ1T); cudaFree(m->Z1); cudaFree(m->Z2); cudaFree(m->dA1); cudaFree(m->out); cudaFree(m->states);
    m->X = m->XT = m->A1 = m->A1T = m->dZ2 = m->dZ2T = m->dZ1T = nullptr;
    m->Z1 = m->Z2 = m->dA1 = m->out = nullptr;
    m->states = nullptr;
    m->cap = 0;
}

hb_status ensure_ws(hb_mlp *m, uint64_t n_pad) {
    if (n_pad <= m->cap) return HB_OK;
    free_ws(m);
    const uint64_t b = n_pad;
    bool ok = cudaMalloc(&m->X, b * kIn * 2) == cudaSuccess && cudaMalloc(&m->XT, b * kIn * 2) == cudaSuccess &&
              cudaMalloc(&m->A1, b * kH * 2) == cudaSuccess && cudaMalloc(&m->A1T, b * kH * 2) == cudaSuccess &&
              cudaMalloc(&m->dZ2, b * kH * 2) == cudaSuccess && cudaMalloc(&m->dZ2T, b * kH * 2) == cudaSuccess &&
              cudaMalloc(&m->dZ1T, b * kH * 2) == cudaSuccess && cudaMalloc(&m->Z1, b * kH * 4) == cudaSuccess &&
              cudaMalloc(&m->Z2, b * kH * 4) == cudaSuccess && cudaMalloc(&m->dA1, b * kH * 4) == cudaSuccess &&
              cudaMalloc(&m->out, b * 2 * 4) == cudaSuccess && cudaMalloc(&m->states, b * 8) == cudaSuccess;
    if (!ok) {
        free_ws(m);
        return HB_ERR_NO_MEMORY;
    }
    m->cap = n_pad;
    return HB_OK;
}

// C = A B^T on the tensor cores; split K over `split` CTAs when mode == 1 (atomic accumulation).
hb_status gemm(hb_mlp *m, const __nv_bfloat16 *A, int lda, const __nv_bfloat16 *B, int ldb, float *C, int ldc, int M,
               int N, int K, int n_store, int mode, int split, cudaStream_t st) {
    const int kpc = ((K + split - 1) / split + kBK - 1) / kBK * kBK;
    const int zs = (K + kpc - 1) / kpc;
    if (N <= 32) {
        dim3 g((M + kBM - 1) / kBM, (N + 31) / 32, zs);
        PD_CUDA(cudaFuncSetAttribute(k_tc_gemm<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc_gemm_smem(32)));
        k_tc_gemm<32><<<g, 128, tc_gemm_smem(32), st>>>(A, lda, B, ldb, C, ldc, M, N, K, kpc, n_store, mode, m->d_err);
    } else {
        dim3 g((M + kBM - 1) / kBM, (N + 127) / 128, zs);
        PD_CUDA(cudaFuncSetAttribute(k_tc_gemm<128>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)tc_gemm_smem(128)));
        k_tc_gemm<128><<<g, 128, tc_gemm_smem(128), st>>>(A, lda, B, ldb, C, ldc, M, N, K, kpc, n_store, mode,
                                                          m->d_err);
    }
    PD_CUDA(cudaGetLastError());
    return HB_OK;
}

// forward of n_pad rows whose inputs are already in m->X; writes Z1, A1, Z2, out
hb_status forward_rows(hb_mlp *m, uint64_t n, uint64_t n_pad, cudaStream_t st) {
    hb_status s = gemm(m, m->X, kIn, m->W1b, kIn, m->Z1, kH, (int)n_pad, kH, kIn, kH, 0, 1, st);
    if (s != HB_OK) return s;
    k_bias_gelu_bf16<<<grid_of(n_pad * kH, m->sm_count), 256, 0, st>>>(m->Z1, m->d_p + m->ob1, n_pad, m->A1);
    if ((s = gemm(m, m->A1, kH, m->W2b, kH, m->Z2, kH, (int)n_pad, kH, kH, kH, 0, 1, st)) != HB_OK) return s;
    k_output<<<grid_of(n, m->sm_count), 256, 0, st>>>(m->Z2, m->d_p + m->ob2, m->d_p + m->oW3, m->d_p + m->ob3, n,
                                                      m->out);
    PD_CUDA(cudaGetLastError());
    return HB_OK;
}

void refresh(hb_mlp *m, cudaStream_t st) {
    k_refresh_bf16<<<64, 256, 0, st>>>(m->d_p + m->oW1, m->d_p + m->oW2, m->n_in, m->W1b, m->W2b, m->W2tb);
}

}  // namespace

extern "C" {

hb_status mlp_create(int n_in, uint64_t seed, hb_mlp_handle *out) {
    if (!out || n_in < 1 || n_in > kIn) return HB_ERR_INVALID_ARG;
    *out = nullptr;
    hb_mlp *m = new (std::nothrow) hb_mlp();
    if (!m) return HB_ERR_NO_MEMORY;
    m->n_in = n_in;
    m->oW1 = 0;
    m->ob1 = m->oW1 + (uint64_t)kH * n_in;
    m->oW2 = m->ob1 + kH;
    m->ob2 = m->oW2 + (uint64_t)kH * kH;
    m->oW3 = m->ob2 + kH;
    m->ob3 = m->oW3 + 2 * kH;
    m->P = m->ob3 + 2;
    cudaGetDevice(&m->device);
    cudaDeviceGetAttribute(&m->sm_count, cudaDevAttrMultiProcessorCount, m->device);
    bool ok = cudaMalloc(&m->d_p, m->P * 4) == cudaSuccess && cudaMalloc(&m->d_m, m->P * 4) == cudaSuccess &&
              cudaMalloc(&m->d_v, m->P * 4) == cudaSuccess && cudaMalloc(&m->d_g, m->P * 4) == cudaSuccess &&
              cudaMalloc(&m->d_loss, 4) == cudaSuccess && cudaMalloc(&m->W1b, kH * kIn * 2) == cudaSuccess &&
              cudaMalloc(&m->W2b, kH * kH * 2) == cudaSuccess && cudaMalloc(&m->W2tb, kH * kH * 2) == cudaSuccess &&
              cudaMalloc(&m->d_err, sizeof(unsigned)) == cudaSuccess;
    if (!ok) {
        mlp_destroy(m);
        return HB_ERR_NO_MEMORY;
    }
    // initial weights: uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) from SplitMix64(seed), zero biases
    std::vector<float> p(m->P, 0.f);
    uint64_t st = seed;
    auto uni = [&]() {
        st += 0x9E3779B97F4A7C15ull;
        uint64_t z = st;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        return (double)(z >> 11) * 0x1.0p-52 - 1.0;
    };
    for (uint64_t i = 0; i < (uint64_t)kH * n_in; ++i) p[m->oW1 + i] = (float)(uni() / std::sqrt((double)n_in));
    for (uint64_t i = 0; i < (uint64_t)kH * kH; ++i) p[m->oW2 + i] = (float)(uni() / std::sqrt((double)kH));
    for (uint64_t i = 0; i < 2ull * kH; ++i) p[m->oW3 + i] = (float)(uni() / std::sqrt((double)kH));
    cudaMemcpy(m->d_p, p.data(), m->P * 4, cudaMemcpyHostToDevice);
    cudaMemset(m->d_m, 0, m->P * 4);
    cudaMemset(m->d_v, 0, m->P * 4);
    cudaMemset(m->d_err, 0, sizeof(unsigned));
    refresh(m, 0);
    if (cudaDeviceSynchronize() != cudaSuccess) {
        mlp_destroy(m);
        return HB_ERR_CUDA;
    }
    *out = m;
    return HB_OK;
}

hb_status mlp_destroy(hb_mlp_handle m) {
    if (!m) return HB_ERR_INVALID_ARG;
    free_ws(m);
    cudaFree(m->d_p); cudaFree(m->d_m); cudaFree(m->d_v); cudaFree(m->d_g); cudaFree(m->d_loss);
    cudaFree(m->W1b); cudaFree(m->W2b); cudaFree(m->W2tb); cudaFree(m->d_err);
    delete m;
    return HB_OK;
}

hb_status mlp_param_count(hb_mlp_handle m, uint64_t *P) {
    if (!m || !P) return HB_ERR_INVALID_ARG;
    *P = m->P;
    return HB_OK;
}

hb_status mlp_get_params(hb_mlp_handle m, float *host) {
    if (!m || !host) return HB_ERR_INVALID_ARG;
    PD_CUDA(cudaMemcpy(host, m->d_p, m->P * 4, cudaMemcpyDeviceToHost));
    return HB_OK;
}

hb_status mlp_set_params(hb_mlp_handle m, const float *host) {
    if (!m || !host) return HB_ERR_INVALID_ARG;
    PD_CUDA(cudaMemcpy(m->d_p, host, m->P * 4, cudaMemcpyHostToDevice));
    refresh(m, 0);
    PD_CUDA(cudaDeviceSynchronize());
    return HB_OK;
}

hb_status mlp_forward(hb_mlp_handle m, const uint64_t *states, uint64_t n, float *out, void *stream) {
    if (!m || (n > 0 && (!states || !out))) return HB_ERR_INVALID_ARG;
    if (n == 0) return HB_OK;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const uint64_t n_pad = (n + kBM - 1) / kBM * kBM;
    hb_status s = ensure_ws(m, n_pad);
    if (s != HB_OK) return s;
    k_bits<<<grid_of(n_pad * kIn, m->sm_count), 256, 0, st>>>(states, n, n_pad, m->n_in, m->X);
    if ((s = forward_rows(m, n, n_pad, st)) != HB_OK) return s;
    PD_CUDA(cudaMemcpyAsync(out, m->out, n * 8, cudaMemcpyDeviceToDevice, st));
    return HB_OK;
}

hb_status mlp_gradient(hb_mlp_handle m, const uint64_t *states, uint64_t n, const float *t_log, const float *t_sign,
                       const float *weights, float lam, float *grad, float *loss, void *stream) {
    if (!m || !states || !t_log || !t_sign || !weights || n == 0) return HB_ERR_INVALID_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const uint64_t n_pad = (n + kBM - 1) / kBM * kBM;
    hb_status s = ensure_ws(m, n_pad);
    if (s != HB_OK) return s;
    k_bits<<<grid_of(n_pad * kIn, m->sm_count), 256, 0, st>>>(states, n, n_pad, m->n_in, m->X);
    if ((s = forward_rows(m, n, n_pad, st)) != HB_OK) return s;
    PD_CUDA(cudaMemsetAsync(m->d_g, 0, m->P * 4, st));
    PD_CUDA(cudaMemsetAsync(m->d_loss, 0, 4, st));
    k_output_back<<<grid_of(n_pad, m->sm_count), 256, 0, st>>>(
        m->Z2, m->d_p + m->ob2, m->d_p + m->oW3, m->out, t_log, t_sign, weights, lam, n, n_pad, m->dZ2, m->dZ2T,
        m->d_g + m->oW3, m->d_g + m->ob3, m->d_g + m->ob2, m->d_loss);
    // dA1 = dZ2 W2  (B = W2^T rows: [in][out])
    if ((s = gemm(m, m->dZ2, kH, m->W2tb, kH, m->dA1, kH, (int)n_pad, kH, kH, kH, 0, 1, st)) != HB_OK) return s;
    k_hidden_back<<<grid_of(n_pad * kH, m->sm_count), 256, 0, st>>>(m->dA1, m->Z1, m->d_p + m->ob1, n, n_pad, m->dZ1T,
                                                                    m->d_g + m->ob1);
    // gW2 = dZ2^T A1 and gW1 = dZ1^T X: K runs over the batch, split over CTAs, atomically accumulated
    k_transpose_bf16<<<grid_of(n_pad * kH, m->sm_count), 256, 0, st>>>(m->A1, n_pad, kH, m->A1T);
    k_transpose_bf16<<<grid_of(n_pad * kIn, m->sm_count), 256, 0, st>>>(m->X, n_pad, kIn, m->XT);
    const int split = (int)std::max<uint64_t>(1, std::min<uint64_t>(n_pad / 512, (uint64_t)m->sm_count * 2));
    if ((s = gemm(m, m->dZ2T, (int)n_pad, m->A1T, (int)n_pad, m->d_g + m->oW2, kH, kH, kH, (int)n_pad, kH, 1, split,
                  st)) != HB_OK)
        return s;
    if ((s = gemm(m, m->dZ1T, (int)n_pad, m->XT, (int)n_pad, m->d_g + m->oW1, m->n_in, kH, kIn, (int)n_pad, m->n_in, 1,
                  split, st)) != HB_OK)
        return s;
    if (grad) PD_CUDA(cudaMemcpyAsync(grad, m->d_g, m->P * 4, cudaMemcpyDeviceToDevice, st));
    if (loss) PD_CUDA(cudaMemcpyAsync(loss, m->d_loss, 4, cudaMemcpyDeviceToDevice, st));
    PD_CUDA(cudaGetLastError());
    return HB_OK;
}

hb_status mlp_adam_step(hb_mlp_handle m, float lr, void *stream) {
    if (!m || !(lr > 0)) return HB_ERR_INVALID_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    m->adam_t += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - std::pow(b1, (float)m->adam_t), c2 = 1.f - std::pow(b2, (float)m->adam_t);
    k_adam<<<grid_of(m->P, m->sm_count), 256, 0, st>>>(m->d_p, m->d_g, m->d_m, m->d_v, m->P, lr, b1, b2, 1e-8f, c1, c2);
    refresh(m, st);
    PD_CUDA(cudaGetLastError());
    return HB_OK;
}

hb_status mlp_start_vector(hb_mlp_handle m, hb_handle h, hb_dtype dt, void *v, void *stream) {
    if (!m || !h || !v || (dt != HB_F64 && dt != HB_F32 && dt != HB_FX64)) return HB_ERR_INVALID_ARG;
    if (2 * h->L != m->n_in || h->ks) return HB_ERR_INVALID_ARG;  // real-space sites only
    hb_status s = pd_build_tables(h);
    if (s != HB_OK) return s;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const size_t smem = sizeof(InferSmem);
    const uint64_t ntiles = (h->D + kBM - 1) / kBM;
    const unsigned grid = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(ntiles, 2ull * m->sm_count));
    const int F = h->fx_frac;
    constexpr int T = kStartThreads;
    if (dt == HB_F32) {
        PD_CUDA(cudaFuncSetAttribute(k_mlp_start<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_mlp_start<float><<<grid, T, smem, st>>>(m->W1b, m->W2b, m->d_p, m->ob1, m->ob2, m->oW3, m->ob3, h->up.str,
                                                   h->dn.str, h->D_dn, h->D, h->L, m->n_in,
                                                   static_cast<float *>(v), F, m->d_err);
    } else if (dt == HB_F64) {
        PD_CUDA(cudaFuncSetAttribute(k_mlp_start<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_mlp_start<double><<<grid, T, smem, st>>>(m->W1b, m->W2b, m->d_p, m->ob1, m->ob2, m->oW3, m->ob3,
                                                    h->up.str, h->dn.str, h->D_dn, h->D, h->L, m->n_in,
                                                    static_cast<double *>(v), F, m->d_err);
    } else {
        PD_CUDA(cudaFuncSetAttribute(k_mlp_start<int64_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_mlp_start<int64_t><<<grid, T, smem, st>>>(m->W1b, m->W2b, m->d_p, m->ob1, m->ob2, m->oW3, m->ob3,
                                                     h->up.str, h->dn.str, h->D_dn, h->D, h->L, m->n_in,
                                                     static_cast<int64_t *>(v), F, m->d_err);
    }
    PD_CUDA(cudaGetLastError());
    return HB_OK;
}

hb_status mlp_sample_workspace_bytes(hb_handle h, uint64_t n, uint64_t *bytes) {
    if (!h || !bytes || h->ks) return HB_ERR_INVALID_ARG;
    uint64_t a, b, c, d;
    samp_layout(h->D, n, &a, &b, &c, &d, bytes);
    return HB_OK;
}

hb_status mlp_sample_training(hb_handle h, const float *psi, uint64_t n, uint64_t seed, uint64_t *states, float *t_log,
                              float *t_sign, void *workspace, uint64_t workspace_bytes, void *stream) {
    if (!h || !psi || !states || !t_log || !t_sign || !workspace || n == 0 || h->ks) return HB_ERR_INVALID_ARG;
    if ((uintptr_t)workspace % 256 != 0) return HB_ERR_INVALID_ARG;
    uint64_t o_bmax, o_bidx, o_logs, o_misc, total;
    samp_layout(h->D, n, &o_bmax, &o_bidx, &o_logs, &o_misc, &total);
    if (workspace_bytes < total) return HB_ERR_NO_MEMORY;
    hb_status s = pd_build_tables(h);
    if (s != HB_OK) return s;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    char *ws = static_cast<char *>(workspace);
    double *bsum = reinterpret_cast<double *>(ws);
    float *bmax = reinterpret_cast<float *>(ws + o_bmax);
    uint64_t *bidx = reinterpret_cast<uint64_t *>(ws + o_bidx);
    double *logs = reinterpret_cast<double *>(ws + o_logs);
    double *misc = reinterpret_cast<double *>(ws + o_misc);
    const uint64_t nblk = (h->D + kSampBlock - 1) / kSampBlock;
    if (nblk > 0x7FFFFFFFull) return HB_ERR_OVERFLOW;
    k_samp_blocks<<<(unsigned)nblk, 256, 0, st>>>(psi, h->D, bsum, bmax, bidx);
    k_samp_scan<<<1, 1024, 0, st>>>(bsum, bmax, bidx, nblk, psi, misc);
    const unsigned grid = (unsigned)std::min<uint64_t>((n + 7) / 8, (uint64_t)h->sm_count * 16);
    k_samp_draw<<<grid, 256, 0, st>>>(psi, h->D, bsum, nblk, misc, n, seed, h->up.str, h->dn.str, h->D_dn, h->L,
                                      states, logs, t_sign);
    k_samp_center<<<1, 1024, 0, st>>>(logs, n, t_log);
    PD_CUDA(cudaGetLastError());
    return HB_OK;
}

hb_status mlp_last_error(hb_mlp_handle m) {
    if (!m) return HB_ERR_INVALID_ARG;
    PD_CUDA(cudaDeviceSynchronize());
    unsigned bits = 0;
    PD_CUDA(cudaMemcpy(&bits, m->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost));
    PD_CUDA(cudaMemset(m->d_err, 0, sizeof(unsigned)));
    for (int s = 1; s <= (int)HB_ERR_TIMEOUT; ++s)
        if (bits & PD_ERRBIT(s)) return (hb_status)s;
    return HB_OK;
}

// Failure-detection self test: one CTA waits, with the same bounded mbarrier
// wait the tensor-core kernels use, on a barrier that nothing arrives at; the
// wait gives up after max_tries polls and the kernel reports HB_ERR_TIMEOUT
// through the status word instead of hanging.
__global__ void k_wait_selftest(uint32_t max_tries, unsigned *status) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) tc::mbar_init(&bar, 1);
    __syncthreads();
    const bool ok = tc::mbar_wait(&bar, 0, max_tries);
    if (threadIdx.x == 0) *status = ok ? 0u : (unsigned)HB_ERR_TIMEOUT;
}

hb_status hb_device_wait_selftest(uint32_t max_tries) {
    unsigned *d = nullptr, h = 0;
    PD_CUDA(cudaMalloc(&d, sizeof(unsigned)));
    k_wait_selftest<<<1, 32>>>(max_tries, d);
    cudaError_t e = cudaMemcpy(&h, d, sizeof(unsigned), cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return HB_ERR_CUDA;
    return (hb_status)h;
}

// C[M, N] = A[M, K] B[N, K]^T on the tensor cores (bf16 in, f32 out), exposed for tests.
hb_status mlp_activation(const float *x, uint64_t n, float *y, int32_t deriv, void *stream) {
    if (!x || !y || (deriv != 0 && deriv != 1)) return HB_ERR_INVALID_ARG;
    if (n == 0) return HB_OK;
    int dev = 0, sms = 0;
    PD_CUDA(cudaGetDevice(&dev));
    PD_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    k_activation<<<grid_of(n, sms), 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(x, n, y, deriv);
    PD_CUDA(cudaGetLastError());
    return HB_OK;
}

hb_status mlp_tc_gemm(const void *A, const void *B, float *C, int M, int N, int K, void *stream) {
    if (!A || !B || !C || M < 1 || N < 1 || K < 1 || K % 8 != 0 || (N != 32 && N % 128 != 0)) return HB_ERR_INVALID_ARG;
    hb_mlp tmp;
    unsigned *err = nullptr;
    PD_CUDA(cudaMalloc(&err, sizeof(unsigned)));
    cudaMemset(err, 0, sizeof(unsigned));
    cudaGetDevice(&tmp.device);
    cudaDeviceGetAttribute(&tmp.sm_count, cudaDevAttrMultiProcessorCount, tmp.device);
    tmp.d_err = err;
    hb_status s = gemm(&tmp, static_cast<const __nv_bfloat16 *>(A), K, static_cast<const __nv_bfloat16 *>(B), K, C, N, M,
                       N, K, N, 0, 1, reinterpret_cast<cudaStream_t>(stream));
    cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream));
    unsigned bits = 0;
    cudaMemcpy(&bits, err, sizeof(unsigned), cudaMemcpyDeviceToHost);
    cudaFree(err);
    tmp.d_err = nullptr;
    if (s == HB_OK && bits) s = HB_ERR_TIMEOUT;
    return s;
}

}  // extern "C"

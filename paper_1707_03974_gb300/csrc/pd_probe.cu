// Measured on-chip ceilings of the GPU the library runs on (hb_measure_ceilings).
//
// The H·v of Eq. 1 moves 16 bytes per basis state through HBM but z hop
// operands per state through the SM's load path (shared memory for the
// spin-down hops of a staged row, L2 for the spin-up rows): its rooflines are
// these on-chip rates as much as HBM bandwidth.  Each probe below runs one
// unit flat out, with enough independent work per thread to hide latency, and
// is timed with CUDA events (best of three launches after a warm-up).  All
// accesses stay inside the buffers they are given; no probe waits on anything.
#include <algorithm>

#include "pd_common.cuh"

namespace {

constexpr int kProbeThreads = 256;
constexpr int kSmemBytes = 64 * 1024;  // staged buffer of the shared-memory probes (power of two)

// ---- arithmetic: eight independent dependency chains per thread ----
__global__ void __launch_bounds__(kProbeThreads) k_probe_fma64(double *out, int iters, double m, double c) {
    double a[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = threadIdx.x * 1e-3 + k;
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int k = 0; k < 8; ++k) a[k] = fma(a[k], m, c);
    double s = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += a[k];
    if (s == 1234.5678) out[0] = s;  // keeps the chains alive; never true for these inputs
}

// The float32 probe also measures the SM clock: thread 0 of CTA 0 reads the SM
// cycle counter and the global nanosecond timer before and after its loop.
__global__ void __launch_bounds__(kProbeThreads) k_probe_fma32(float *out, long long *clk, int iters, float m,
                                                               float c) {
    long long c0 = 0, t0 = 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        c0 = clock64();
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    }
    float a[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = threadIdx.x * 1e-3f + k;
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int k = 0; k < 8; ++k) a[k] = fmaf(a[k], m, c);
    float s = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += a[k];
    if (s == 1234.5678f) out[0] = s;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        long long t1;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t1));
        clk[0] = clock64() - c0;
        clk[1] = t1 - t0;
    }
}

// 32-bit and 64-bit integer adds (the fixed-point hop sums are 64-bit adds)
__global__ void __launch_bounds__(kProbeThreads) k_probe_add32(unsigned *out, int iters, unsigned inc) {
    unsigned a[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = threadIdx.x + k;
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int k = 0; k < 8; ++k) asm volatile("add.u32 %0, %0, %1;" : "+r"(a[k]) : "r"(inc));
    unsigned s = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s ^= a[k];
    if (s == 0x9E3779B9u) out[0] = s;
}

__global__ void __launch_bounds__(kProbeThreads) k_probe_add64(unsigned long long *out, int iters,
                                                               unsigned long long inc) {
    unsigned long long a[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = threadIdx.x + k;
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int k = 0; k < 8; ++k) asm volatile("add.u64 %0, %0, %1;" : "+l"(a[k]) : "l"(inc));
    unsigned long long s = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s ^= a[k];
    if (s == 0x9E3779B97F4A7C15ull) out[0] = s;
}

// ---- shared memory ----
// MODE 0: conflict-free 16-byte loads (a warp reads 512 contiguous bytes);
// MODE 1: 8-byte loads at uniformly random addresses;
// MODE 2: 16-byte loads at uniformly random addresses.
// Addresses come from a per-thread linear congruential sequence (two integer
// instructions per load), so the load path, not the address arithmetic, limits.
template <int MODE>
__global__ void __launch_bounds__(kProbeThreads) k_probe_smem(unsigned *out, int iters) {
    extern __shared__ __align__(16) unsigned char smem[];
    uint32_t *w = reinterpret_cast<uint32_t *>(smem);
    for (int i = threadIdx.x; i < kSmemBytes / 4; i += blockDim.x) w[i] = (uint32_t)i * 2654435761u;
    __syncthreads();
    uint32_t x = (blockIdx.x * blockDim.x + threadIdx.x) * 0x9E3779B9u + 12345u;
    uint32_t acc = 0;
    const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll 4
    for (int i = 0; i < iters; ++i) {
        if (MODE == 0) {
            const uint32_t idx = ((wid + (uint32_t)i * 8u) * 32u + lane) & (kSmemBytes / 16 - 1);
            const uint4 v = reinterpret_cast<const uint4 *>(smem)[idx];
            acc ^= v.x + v.y + v.z + v.w;
        } else if (MODE == 1) {
            x = x * 1664525u + 1013904223u;
            const uint2 v = reinterpret_cast<const uint2 *>(smem)[(x >> 9) & (kSmemBytes / 8 - 1)];
            acc ^= v.x + v.y;
        } else {
            x = x * 1664525u + 1013904223u;
            const uint4 v = reinterpret_cast<const uint4 *>(smem)[(x >> 9) & (kSmemBytes / 16 - 1)];
            acc ^= v.x + v.y + v.z + v.w;
        }
    }
    if (acc == 0x2545F491u) out[0] = acc;
}

// ---- global loads: coalesced 16-byte loads by whole warps ----
// LEVEL 0: every CTA re-reads its own 16 KiB window (L1 hits, ld.global.ca);
// LEVEL 1: the grid sweeps `n16` 16-byte words repeatedly (L2-resident when
//          the window fits in L2, ld.global.cg bypasses L1);
// LEVEL 2: one streaming pass over `n16` words (far larger than L2).
template <int LEVEL>
__global__ void __launch_bounds__(kProbeThreads) k_probe_load(const uint4 *__restrict__ buf, uint64_t n16, int iters,
                                                              unsigned *out) {
    uint32_t acc = 0;
    const uint64_t tid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    const uint64_t nthreads = (uint64_t)gridDim.x * blockDim.x;
    if (LEVEL == 0) {
        const uint64_t win = 1024;  // 16 KiB per CTA
        const uint64_t base = ((uint64_t)blockIdx.x * win) % (n16 - win + 1);
        for (int i = 0; i < iters; ++i)
            for (uint64_t k = threadIdx.x; k < win; k += blockDim.x) {
                uint4 v;
                asm volatile("ld.global.ca.v4.u32 {%0,%1,%2,%3}, [%4];"
                             : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                             : "l"(buf + base + k));
                acc ^= v.x + v.y + v.z + v.w;
            }
    } else {
        for (int i = 0; i < iters; ++i)
            for (uint64_t k = tid; k < n16; k += nthreads) {
                uint4 v;
                if (LEVEL == 1)
                    asm volatile("ld.global.cg.v4.u32 {%0,%1,%2,%3}, [%4];"
                                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                                 : "l"(buf + k));
                else
                    asm volatile("ld.global.cs.v4.u32 {%0,%1,%2,%3}, [%4];"
                                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                                 : "l"(buf + k));
                acc ^= v.x + v.y + v.z + v.w;
            }
    }
    if (acc == 0x2545F491u) out[0] = acc;
}

__global__ void k_probe_fill(uint4 *buf, uint64_t n16) {
    for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < n16; k += (uint64_t)gridDim.x * blockDim.x)
        buf[k] = make_uint4((unsigned)k, (unsigned)(k >> 32), 0x9E3779B9u, 0x7F4A7C15u);
}

// best of three timed launches (after one warm-up) of `launch`, in milliseconds
template <typename Fn>
hb_status best_ms(cudaStream_t st, Fn launch, float *ms) {
    cudaEvent_t e0, e1;
    PD_CUDA(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return HB_ERR_CUDA;
    }
    launch();
    float best = 3.4e38f;
    for (int r = 0; r < 3; ++r) {
        cudaEventRecord(e0, st);
        launch();
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        float t = 0.f;
        cudaEventElapsedTime(&t, e0, e1);
        best = std::min(best, t);
    }
    const cudaError_t err = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (err != cudaSuccess) return HB_ERR_CUDA;
    *ms = best;
    return HB_OK;
}

}  // namespace

extern "C" hb_status hb_measure_ceilings(void *buffer, uint64_t buffer_bytes, hb_ceilings *out, void *stream) {
    if (!buffer || !out || buffer_bytes < (64ull << 20) || (uintptr_t)buffer % 16 != 0) return HB_ERR_INVALID_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0;
    PD_CUDA(cudaGetDevice(&dev));
    PD_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    *out = hb_ceilings{};
    out->sm_count = sms;
    // scratch outputs of the probes live in the first 256 bytes of the buffer
    unsigned char *base = static_cast<unsigned char *>(buffer);
    long long *clk = reinterpret_cast<long long *>(base);
    uint4 *data = reinterpret_cast<uint4 *>(base + 256);
    const uint64_t n16_all = (buffer_bytes - 256) / 16;
    const unsigned grid = (unsigned)sms * 8;  // 8 CTAs of 256 threads per SM
    const double threads = (double)grid * kProbeThreads;
    float ms = 0.f;
    hb_status s;

    const int it64 = 2048;
    if ((s = best_ms(st, [&] { k_probe_fma64<<<grid, kProbeThreads, 0, st>>>(reinterpret_cast<double *>(base), it64, 0.999999, 1e-7); }, &ms)) != HB_OK) return s;
    out->fp64_fma_tflops = threads * 8.0 * it64 * 2.0 / (ms * 1e-3) / 1e12;

    const int it32 = 65536;
    if ((s = best_ms(st, [&] { k_probe_fma32<<<grid, kProbeThreads, 0, st>>>(reinterpret_cast<float *>(base + 64), clk, it32, 0.999999f, 1e-7f); }, &ms)) != HB_OK) return s;
    out->fp32_fma_tflops = threads * 8.0 * it32 * 2.0 / (ms * 1e-3) / 1e12;
    long long hc[2] = {0, 0};
    PD_CUDA(cudaMemcpyAsync(hc, clk, sizeof(hc), cudaMemcpyDeviceToHost, st));
    PD_CUDA(cudaStreamSynchronize(st));
    out->sm_clock_mhz = hc[1] > 0 ? (double)hc[0] / (double)hc[1] * 1e3 : 0.0;

    const int iti = 32768;
    if ((s = best_ms(st, [&] { k_probe_add32<<<grid, kProbeThreads, 0, st>>>(reinterpret_cast<unsigned *>(base + 128), iti, 3u); }, &ms)) != HB_OK) return s;
    out->int32_add_tops = threads * 8.0 * iti / (ms * 1e-3) / 1e12;
    if ((s = best_ms(st, [&] { k_probe_add64<<<grid, kProbeThreads, 0, st>>>(reinterpret_cast<unsigned long long *>(base + 192), iti, 3ull); }, &ms)) != HB_OK) return s;
    out->int64_add_tops = threads * 8.0 * iti / (ms * 1e-3) / 1e12;

    // shared memory: 3 CTAs of 64 KiB per SM
    const unsigned sgrid = (unsigned)sms * 3;
    const double swarps = (double)sgrid * (kProbeThreads / 32);
    const int its = 8192;
    PD_CUDA(cudaFuncSetAttribute(k_probe_smem<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes));
    PD_CUDA(cudaFuncSetAttribute(k_probe_smem<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes));
    PD_CUDA(cudaFuncSetAttribute(k_probe_smem<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes));
    unsigned *uo = reinterpret_cast<unsigned *>(base + 128);
    const double clk_hz = out->sm_clock_mhz * 1e6;
    if ((s = best_ms(st, [&] { k_probe_smem<0><<<sgrid, kProbeThreads, kSmemBytes, st>>>(uo, its); }, &ms)) != HB_OK) return s;
    out->smem_seq16_gbs = swarps * its * 512.0 / (ms * 1e-3) / 1e9;
    if ((s = best_ms(st, [&] { k_probe_smem<1><<<sgrid, kProbeThreads, kSmemBytes, st>>>(uo, its); }, &ms)) != HB_OK) return s;
    out->smem_gather8_gbs = swarps * its * 256.0 / (ms * 1e-3) / 1e9;
    out->smem_gather8_clk = clk_hz > 0 ? (ms * 1e-3) * clk_hz * sms / (swarps * its) : 0.0;
    if ((s = best_ms(st, [&] { k_probe_smem<2><<<sgrid, kProbeThreads, kSmemBytes, st>>>(uo, its); }, &ms)) != HB_OK) return s;
    out->smem_gather16_gbs = swarps * its * 512.0 / (ms * 1e-3) / 1e9;
    out->smem_gather16_clk = clk_hz > 0 ? (ms * 1e-3) * clk_hz * sms / (swarps * its) : 0.0;

    // global loads
    k_probe_fill<<<sms * 8, kProbeThreads, 0, st>>>(data, n16_all);
    PD_CUDA(cudaGetLastError());
    const int itl1 = 256;
    if ((s = best_ms(st, [&] { k_probe_load<0><<<grid, kProbeThreads, 0, st>>>(data, n16_all, itl1, uo); }, &ms)) != HB_OK) return s;
    out->l1_gbs = (double)grid * 1024 * 16.0 * itl1 / (ms * 1e-3) / 1e9;
    const uint64_t l2n = (32ull << 20) / 16;  // a 32 MiB window
    const int itl2 = 64;
    if ((s = best_ms(st, [&] { k_probe_load<1><<<grid, kProbeThreads, 0, st>>>(data, l2n, itl2, uo); }, &ms)) != HB_OK) return s;
    out->l2_gbs = (double)l2n * 16.0 * itl2 / (ms * 1e-3) / 1e9;
    out->l2_window_bytes = l2n * 16;
    if (buffer_bytes >= (1ull << 30)) {
        if ((s = best_ms(st, [&] { k_probe_load<2><<<grid, kProbeThreads, 0, st>>>(data, n16_all, 1, uo); }, &ms)) != HB_OK) return s;
        out->hbm_read_gbs = (double)n16_all * 16.0 / (ms * 1e-3) / 1e9;
        out->hbm_window_bytes = n16_all * 16;
    }
    PD_CUDA(cudaStreamSynchronize(st));
    return HB_OK;
}

// Pinned host buffers backed by huge pages (hb_host_alloc / hb_host_free).
//
// Host-to-device copies of page-locked memory run at the link's full rate only
// when the pages behind the buffer are large: with 4 KiB pages every DMA burst
// needs its own address translation, and the copy rate of one buffer then
// depends on how the kernel happened to back it.  These buffers are anonymous
// mappings rounded up to 2 MiB, aligned to the huge page size and advised for
// transparent huge pages, placed on the host NUMA node nearest the current
// device (where the driver names one), touched once on the host (so the pages
// exist, as huge pages where the kernel allows), then registered with the CUDA
// driver as page-locked memory.  On hosts with several CPU sockets a buffer left
// on a far node copies through the inter-socket link, at a fraction of the rate.
#include <cuda_runtime.h>
#include <sys/mman.h>
#include <sys/syscall.h>
#include <unistd.h>

#include <cstdint>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>

#include "paradeisos.h"

namespace {

constexpr uint64_t kHuge = 2ull << 20;

std::mutex g_mu;
std::map<void *, uint64_t> g_maps;  // base address -> mapped bytes

// the host's transparent huge page size (2 MiB on 4 KiB-page kernels, 512 MiB on
// 64 KiB-page Arm kernels), or 2 MiB if the kernel does not say
uint64_t thp_size() {
    uint64_t v = 0;
    if (FILE *f = std::fopen("/sys/kernel/mm/transparent_hugepage/hpage_pmd_size", "r")) {
        unsigned long long t = 0;
        if (std::fscanf(f, "%llu", &t) == 1) v = t;
        std::fclose(f);
    }
    return (v >= kHuge && v <= (1ull << 30) && (v & (v - 1)) == 0) ? v : kHuge;
}

// Preferred NUMA node of [p, p + size): the host node nearest the current device.
// Advice only (set before the first touch): without NUMA, or if the call is
// refused, the pages follow the default policy.
void prefer_device_node(void *p, uint64_t size) {
#ifdef SYS_mbind
    int dev = 0, node = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&node, cudaDevAttrHostNumaId, dev) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    constexpr int kBits = 1024, kWord = 8 * sizeof(unsigned long);
    if (node < 0 || node >= kBits) return;
    unsigned long mask[kBits / kWord] = {0};
    mask[node / kWord] |= 1ul << (node % kWord);
    constexpr int kMpolPreferred = 1;
    syscall(SYS_mbind, p, (unsigned long)size, kMpolPreferred, mask, (unsigned long)kBits + 1, 0u);
#else
    (void)p;
    (void)size;
#endif
}

}  // namespace

extern "C" hb_status hb_host_alloc(uint64_t bytes, void **ptr) {
    if (!ptr) return HB_ERR_INVALID_ARG;
    *ptr = nullptr;
    if (bytes == 0) return HB_ERR_INVALID_ARG;
    const uint64_t size = (bytes + kHuge - 1) / kHuge * kHuge, align = thp_size();
    // map align bytes more, then unmap the slack around the aligned range
    char *raw = static_cast<char *>(
        mmap(nullptr, size + align, PROT_READ | PROT_WRITE, MAP_PRIVATE | MAP_ANONYMOUS, -1, 0));
    if (raw == reinterpret_cast<char *>(MAP_FAILED)) return HB_ERR_NO_MEMORY;
    char *p = reinterpret_cast<char *>((reinterpret_cast<uintptr_t>(raw) + align - 1) & ~(uintptr_t)(align - 1));
    if (p > raw) munmap(raw, p - raw);
    if (raw + size + align > p + size) munmap(p + size, raw + size + align - (p + size));
#ifdef MADV_HUGEPAGE
    madvise(p, size, MADV_HUGEPAGE);  // advice only: without transparent huge pages the buffer still works
#endif
    prefer_device_node(p, size);
    std::memset(p, 0, size);
    if (cudaHostRegister(p, size, cudaHostRegisterDefault) != cudaSuccess) {
        cudaGetLastError();
        munmap(p, size);
        return HB_ERR_CUDA;
    }
    {
        std::lock_guard<std::mutex> lock(g_mu);
        g_maps[p] = size;
    }
    *ptr = p;
    return HB_OK;
}

extern "C" hb_status hb_host_free(void *ptr) {
    if (!ptr) return HB_OK;
    uint64_t size = 0;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        auto it = g_maps.find(ptr);
        if (it == g_maps.end()) return HB_ERR_INVALID_ARG;
        size = it->second;
        g_maps.erase(it);
    }
    const bool ok = cudaHostUnregister(ptr) == cudaSuccess;
    if (!ok) cudaGetLastError();
    munmap(ptr, size);
    return ok ? HB_OK : HB_ERR_CUDA;
}

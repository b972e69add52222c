// Page-locked host memory backed by huge pages, for the buffers that the
// host-buffer calls (pf_run_host, serving requests) upload from and write
// to.  Contract: pf_host_alloc / pf_host_free in pf.h.
//
// Why: the device translates every host address it reads or writes, and
// fewer, larger pages leave it fewer translations to make.  In one series
// of serving measurements, uploads from page-locked memory allocated buffer
// by buffer stalled more the longer the process ran (p99 at 90% load 23 to
// 40 ms), while uploads from one large region in 2 MB pages, its space
// reused, stayed steady (3.0 ms); in later series both kinds stalled at
// times, so the region helps, but does not rule the stalls out.
//
// Regions of at least 1 GB are mapped, advised for transparent huge pages
// and registered with the CUDA runtime once, and kept for the life of the
// process; blocks are carved out of them first-fit (256-byte aligned) and
// their space returns to the region's free list when freed.
#include <map>
#include <memory>
#include <mutex>
#include <vector>

#if defined(__linux__)
#include <sys/mman.h>
#endif

#include "pf_serve.h"

namespace {

constexpr size_t kHuge = size_t(2) << 20;
constexpr size_t kRegion = size_t(1) << 30;
constexpr size_t kAlign = 256;

struct Region {
    char *base = nullptr;   // 2 MB-aligned, registered
    size_t len = 0;
    void *map = nullptr;    // what the mapping call returned
    size_t map_len = 0;
    pf::Arena arena;
};

std::mutex g_mu;
std::vector<std::unique_ptr<Region>> g_regions;
std::map<void *, std::pair<Region *, size_t>> g_blocks;  // block -> (region, bytes)

// A new registered region of at least `bytes`; null on failure (*st set).
Region *new_region(size_t bytes, pf_status *st) {
    const size_t len = (std::max(bytes, kRegion) + kHuge - 1) / kHuge * kHuge;
    auto r = std::make_unique<Region>();
#if defined(__linux__)
    const size_t map_len = len + kHuge;  // slack to start on a 2 MB boundary
    void *m = mmap(nullptr, map_len, PROT_READ | PROT_WRITE, MAP_PRIVATE | MAP_ANONYMOUS, -1, 0);
    if (m == MAP_FAILED) {
        *st = PF_ENOMEM;
        return nullptr;
    }
    char *p = reinterpret_cast<char *>((reinterpret_cast<uintptr_t>(m) + kHuge - 1) &
                                       ~uintptr_t(kHuge - 1));
    madvise(p, len, MADV_HUGEPAGE);  // advice: small pages if no huge ones are free
    if (cudaHostRegister(p, len, cudaHostRegisterDefault) != cudaSuccess) {
        cudaGetLastError();
        munmap(m, map_len);
        *st = PF_ECUDA;
        return nullptr;
    }
    r->map = m;
    r->map_len = map_len;
#else
    char *p = nullptr;
    if (cudaHostAlloc(reinterpret_cast<void **>(&p), len, cudaHostAllocDefault) != cudaSuccess) {
        cudaGetLastError();
        *st = PF_ENOMEM;
        return nullptr;
    }
    r->map = p;
    r->map_len = len;
#endif
    r->base = p;
    r->len = len;
    r->arena.reset(len);
    g_regions.push_back(std::move(r));
    return g_regions.back().get();
}

}  // namespace

extern "C" pf_status pf_host_alloc(size_t bytes, void **ptr) {
    if (!ptr) return PF_EINVAL;
    *ptr = nullptr;
    if (bytes == 0) return PF_EINVAL;
    const size_t need = (bytes + kAlign - 1) / kAlign * kAlign;
    std::lock_guard<std::mutex> lk(g_mu);
    size_t off = 0;
    Region *reg = nullptr;
    for (auto &r : g_regions)
        if (r->arena.alloc(need, &off)) {
            reg = r.get();
            break;
        }
    if (!reg) {
        pf_status st = PF_OK;
        reg = new_region(need, &st);
        if (!reg) return st;
        if (!reg->arena.alloc(need, &off)) return PF_ENOMEM;
    }
    void *p = reg->base + off;
    g_blocks[p] = {reg, need};
    *ptr = p;
    return PF_OK;
}

extern "C" pf_status pf_host_free(void *ptr) {
    if (!ptr) return PF_OK;
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_blocks.find(ptr);
    if (it == g_blocks.end()) return PF_EINVAL;
    Region *r = it->second.first;
    r->arena.release((size_t)(static_cast<char *>(ptr) - r->base), it->second.second);
    g_blocks.erase(it);
    return PF_OK;
}

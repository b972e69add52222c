// Compaction for callers that cannot allocate device memory.
//
// pf_compact() takes its per-tile counters from scratch that the context
// allocates with cudaMalloc.  Some callers cannot allocate at all: code
// inside a framework whose own allocator owns every byte of device memory,
// or a latency path that cannot afford cudaMalloc's implicit device
// synchronisation.  For them, pf_compact_noalloc() runs the same three
// kernels with the tile counters in the fixed device array below, and
// allocates nothing.
#include <mutex>

#include "pf_kernels.h"

namespace {

// Counters for up to kNoallocTiles tiles of 4096 flags: n <= 134,217,728.
// Every GPU that loads the library holds these 256 KiB until the process
// exits.  All calls share the array; each call overwrites the counters it
// uses before reading them, so nothing needs clearing, but two calls whose
// kernels overlap on the GPU race on it.
constexpr int64_t kNoallocTiles = 32768;
static __device__ __align__(256) int64_t g_noalloc_tiles[kNoallocTiles];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
int64_t *g_addr[kMaxDevices] = {};

// Device address of g_noalloc_tiles on the current device.  In host code the
// array's name is only a host-side stand-in, so the address comes from
// cudaGetSymbolAddress, once per device, with that device current.  The
// address is kept for the life of the process: after a cudaDeviceReset the
// module is loaded again and the kept address may be stale (the header tells
// callers not to use this entry point across a reset).
cudaError_t tiles_on_device(int64_t **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_tiles);
        if (e != cudaSuccess) return e;
        g_addr[dev] = static_cast<int64_t *>(p);
    }
    *out = g_addr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" PF_API pf_status pf_compact_noalloc(const uint8_t *flags, int64_t n, int64_t *idx,
                                               int64_t *n_out, void *stream) {
    if (n < 0 || !n_out || (n > 0 && (!flags || !idx))) return PF_EINVAL;
    if (pf::compact_tiles(n) > kNoallocTiles) return PF_EINVAL;
    int64_t *tiles = nullptr;
    if (tiles_on_device(&tiles) != cudaSuccess) {
        cudaGetLastError();
        return PF_ECUDA;
    }
    const cudaError_t e = pf::launch_compact(flags, n, idx, n_out, tiles,
                                             static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return PF_ECUDA;
    }
    return PF_OK;
}

// a5: order-preserving compaction of the accepted pairs (the thesis sends
// only the mappings that pass the filter on to verification, Ch. 5
// Summary).  Three launches, no waits between blocks:
//   count   block b counts the set flags of its tile of kTile positions,
//   scan    one block turns the tile counts into exclusive offsets and the
//           total,
//   scatter block b re-reads its tile and writes the positions of the set
//           flags, in order, from its offset on.
// With an order array (the scheduler's grouping of the pairs by
// configuration and length) position q stands for pair order[q]: the
// indices come out in that order, so that verification runs the pairs of
// one threshold and length together.
#include "pf_internal.cuh"

namespace pf {

namespace {

constexpr int kThreads = 256;
constexpr int kPerThread = 16;                  // one 16-byte load per thread
constexpr int kTile = kThreads * kPerThread;    // 4096 positions per block

// Flags of positions [base, base + 16) as a 16-bit mask; positions >= n
// read as 0.  Uses one 16-byte load when the run is aligned and in range.
__device__ __forceinline__ unsigned load_flags16(const uint8_t *flags, int64_t base, int64_t n) {
    unsigned bits = 0;
    const uint8_t *p = flags + base;
    if (base + 16 <= n && (reinterpret_cast<uintptr_t>(p) & 15u) == 0) {
        const uint4 v = __ldg(reinterpret_cast<const uint4 *>(p));
        const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int k = 0; k < 4; ++k)
#pragma unroll
            for (int b = 0; b < 4; ++b)
                if ((w[k] >> (8 * b)) & 0xffu) bits |= 1u << (4 * k + b);
    } else {
        for (int k = 0; k < 16; ++k)
            if (base + k < n && __ldg(p + k)) bits |= 1u << k;
    }
    return bits;
}

// The same through an order array: position q's flag is flags[order[q]].
__device__ __forceinline__ unsigned load_flags16_ordered(const uint8_t *flags,
                                                         const int64_t *order, int64_t base,
                                                         int64_t n) {
    unsigned bits = 0;
#pragma unroll
    for (int k = 0; k < 16; ++k)
        if (base + k < n && __ldg(flags + __ldg(order + base + k))) bits |= 1u << k;
    return bits;
}

__device__ __forceinline__ const int64_t *active_order(const int64_t *order, const int *ident) {
    return (order && !(ident && *ident)) ? order : nullptr;
}

__device__ __forceinline__ int block_sum(int v, int *red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    v = __reduce_add_sync(0xffffffffu, v);
    if (lane == 0) red[warp] = v;
    __syncthreads();
    int t = 0;
    if (threadIdx.x < kThreads / 32) t = red[threadIdx.x];
    if (warp == 0) t = __reduce_add_sync(0xffffffffu, t);
    return t;  // valid in warp 0
}

__global__ void __launch_bounds__(kThreads)
compact_count_kernel(const uint8_t *flags, int64_t n, int64_t *tile_count,
                     const int64_t *order, const int *ident) {
    __shared__ int red[kThreads / 32];
    const int64_t base = (int64_t)blockIdx.x * kTile + (int64_t)threadIdx.x * kPerThread;
    const int64_t *ord = active_order(order, ident);
    const int c = __popc(ord ? load_flags16_ordered(flags, ord, base, n)
                             : load_flags16(flags, base, n));
    const int t = block_sum(c, red);
    if (threadIdx.x == 0) tile_count[blockIdx.x] = t;
}

// Single block: exclusive scan of ntiles counts in place, total to *n_out.
__global__ void __launch_bounds__(1024)
compact_scan_kernel(int64_t *tile_count, int64_t ntiles, int64_t *n_out) {
    __shared__ int64_t warp_tot[32];
    __shared__ int64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t b0 = 0; b0 < ntiles; b0 += blockDim.x) {
        const int64_t i = b0 + threadIdx.x;
        const int64_t v = (i < ntiles) ? tile_count[i] : 0;
        int64_t x = v;  // inclusive scan within the warp
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) warp_tot[warp] = x;
        __syncthreads();
        if (warp == 0) {
            int64_t t = (lane < (int)(blockDim.x >> 5)) ? warp_tot[lane] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int64_t y = __shfl_up_sync(0xffffffffu, t, o);
                if (lane >= o) t += y;
            }
            warp_tot[lane] = t;  // inclusive over warps
        }
        __syncthreads();
        const int64_t before = carry + (warp > 0 ? warp_tot[warp - 1] : 0);
        if (i < ntiles) tile_count[i] = before + x - v;
        __syncthreads();
        if (threadIdx.x == 0) carry += warp_tot[(blockDim.x >> 5) - 1];
        __syncthreads();
    }
    if (threadIdx.x == 0) *n_out = carry;
}

__global__ void __launch_bounds__(kThreads)
compact_scatter_kernel(const uint8_t *flags, int64_t n, const int64_t *tile_off, int64_t *idx,
                       const int64_t *order, const int *ident) {
    __shared__ int warp_tot[kThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t base = (int64_t)blockIdx.x * kTile + (int64_t)threadIdx.x * kPerThread;
    const int64_t *ord = active_order(order, ident);
    unsigned bits = ord ? load_flags16_ordered(flags, ord, base, n) : load_flags16(flags, base, n);
    const int c = __popc(bits);
    int x = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[warp] = x;
    __syncthreads();
    int before = 0;
    for (int w = 0; w < warp; ++w) before += warp_tot[w];
    int64_t out = tile_off[blockIdx.x] + before + x - c;
    while (bits) {
        const int k = __ffs(bits) - 1;
        bits &= bits - 1;
        idx[out++] = ord ? __ldg(ord + base + k) : base + k;
    }
}

}  // namespace

int64_t compact_tiles(int64_t n) { return (n + kTile - 1) / kTile; }

cudaError_t launch_compact(const uint8_t *flags, int64_t n, int64_t *idx, int64_t *n_out,
                           int64_t *tile_scratch, cudaStream_t st, const int64_t *order,
                           const int *ident) {
    const int64_t ntiles = compact_tiles(n);
    if (ntiles == 0) return cudaMemsetAsync(n_out, 0, sizeof(int64_t), st);
    compact_count_kernel<<<(unsigned)ntiles, kThreads, 0, st>>>(flags, n, tile_scratch, order,
                                                                ident);
    compact_scan_kernel<<<1, 1024, 0, st>>>(tile_scratch, ntiles, n_out);
    compact_scatter_kernel<<<(unsigned)ntiles, kThreads, 0, st>>>(flags, n, tile_scratch, idx,
                                                                  order, ident);
    return cudaGetLastError();
}

}  // namespace pf

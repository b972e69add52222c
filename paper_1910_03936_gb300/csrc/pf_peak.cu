// Integer-pipe microbenchmark: the measured peak the filter's roofline is
// taken against.  Contract: pf_peak_int in pf.h.
//
// The filter's arithmetic is 32-bit logic (LOP3), funnel shifts (SHF) and
// population counts; no floating point and no tensor cores.  Each kernel
// below keeps many independent chains of one instruction mix in flight per
// thread (written as inline PTX so that each statement is one instruction
// of the named kind) and is sized to run for tens of milliseconds per
// launch; the host times a train of launches with CUDA events.
#include <algorithm>

#include "pf_ctx.h"

namespace pf {

namespace {

constexpr int kChains = 8;      // independent dependency chains per thread
constexpr int kPeakThreads = 256;

__device__ __forceinline__ uint32_t lop3_xor3(uint32_t a, uint32_t b, uint32_t c) {
    uint32_t r;
    asm volatile("lop3.b32 %0, %1, %2, %3, 0x96;" : "=r"(r) : "r"(a), "r"(b), "r"(c));
    return r;
}
__device__ __forceinline__ uint32_t shf_r(uint32_t a, uint32_t b, uint32_t s) {
    uint32_t r;
    asm volatile("shf.r.wrap.b32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "r"(s));
    return r;
}
__device__ __forceinline__ uint32_t popc32(uint32_t a) {
    uint32_t r;
    asm volatile("popc.b32 %0, %1;" : "=r"(r) : "r"(a));
    return r;
}

// kind 0: LOP3 and SHF in equal numbers (the map's and GateKeeper's mix),
// 4 instructions per chain per iteration.
// kind 1: POPC feeding a LOP3 (popcount throughput; 2 per chain per iteration).
template <int KIND>
__global__ void __launch_bounds__(kPeakThreads) peak_kernel(uint32_t seed, int iters,
                                                            uint32_t *sink) {
    uint32_t a[kChains], b[kChains];
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
        a[c] = seed ^ (t * 0x9e3779b9u) ^ (uint32_t)c;
        b[c] = (seed + (uint32_t)c) * 0x85ebca6bu ^ t;
    }
    const uint32_t s = (seed & 15u) + 3u;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
#pragma unroll
            for (int c = 0; c < kChains; ++c) {
                if constexpr (KIND == 0) {
                    a[c] = lop3_xor3(a[c], b[c], s);
                    b[c] = shf_r(b[c], a[c], s);
                    a[c] = shf_r(a[c], b[c], s);
                    b[c] = lop3_xor3(b[c], a[c], s);
                } else {
                    a[c] = lop3_xor3(popc32(b[c]), a[c], s);
                    b[c] = lop3_xor3(popc32(a[c]), b[c], s);
                }
            }
        }
    }
    uint32_t x = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) x ^= a[c] ^ b[c];
    if (x == seed) sink[0] = x;  // keeps every chain live; practically never taken
}

// Instructions of the named kinds one thread executes per iteration.
constexpr double kOpsPerIter[2] = {4.0 * kChains * 4, 4.0 * kChains * 4};

}  // namespace

}  // namespace pf

using namespace pf;

extern "C" pf_status pf_peak_int(pf_ctx *ctx, int kind, int launches, double *ops_per_s,
                                 double *ms_per_launch) {
    if (!ctx) return PF_EINVAL;
    if (kind < 0 || kind > 1 || launches < 1 || launches > 1000 || !ops_per_s)
        return ctx->fail(PF_EINVAL, "pf_peak_int: kind 0..1, launches 1..1000, ops_per_s");
    cudaSetDevice(ctx->device);
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &per_sm, kind == 0 ? (const void *)peak_kernel<0> : (const void *)peak_kernel<1>,
        kPeakThreads, 0);
    if (e != cudaSuccess) return ctx->cuda(e, "pf_peak_int occupancy");
    const int grid = std::max(1, per_sm) * ctx->sms;
    const int iters = 1 << 14;
    uint32_t *sink = nullptr;
    if (cudaMalloc(&sink, sizeof(uint32_t)) != cudaSuccess) {
        cudaGetLastError();
        return ctx->fail(PF_ENOMEM, "pf_peak_int: sink");
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    auto launch = [&](uint32_t seed) {
        if (kind == 0) peak_kernel<0><<<grid, kPeakThreads, 0, ctx->stream>>>(seed, iters, sink);
        else peak_kernel<1><<<grid, kPeakThreads, 0, ctx->stream>>>(seed, iters, sink);
    };
    launch(1u);  // warm-up
    cudaEventRecord(e0, ctx->stream);
    for (int i = 0; i < launches; ++i) launch(2u + (uint32_t)i);
    cudaEventRecord(e1, ctx->stream);
    e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    if (e != cudaSuccess) return ctx->cuda(e, "pf_peak_int");
    const double ops = (double)grid * kPeakThreads * iters * kOpsPerIter[kind] * launches;
    *ops_per_s = ops / (ms * 1e-3);
    if (ms_per_launch) *ms_per_launch = ms / launches;
    return PF_OK;
}

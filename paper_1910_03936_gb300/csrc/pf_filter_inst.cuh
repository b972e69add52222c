// Instantiates the filter kernels for one decider set PF_DEC (1, 2 or 3).
#include <atomic>

#include "pf_filter.cuh"
#include "pf_kernels.h"

namespace pf {

#define PF_CAT2(a, b) a##b
#define PF_CAT(a, b) PF_CAT2(a, b)

template <int I>
using CfgAt = std::integral_constant<int, I>;

// The two-phase kernels take more than the default 48 KB of dynamic shared
// memory; the limit is raised once per device (a function attribute holds
// per device).
constexpr int kMaxDevices = 64;

template <int I>
static const void *batched_ptr_i() {
    constexpr KernelCfg c = kBatchCfgs[I];
    if constexpr (cfg_split(c, PF_DEC)) {
        const void *f;
        if constexpr (c.tpp == 1)
            f = reinterpret_cast<const void *>(&filter_split_kernel<PF_DEC, c.xe, c.words>);
        else
            f = reinterpret_cast<const void *>(
                &filter_split_group_kernel<PF_DEC, c.tpp, c.dpt, c.words>);
        static std::atomic<bool> raised[kMaxDevices];
        int dev = 0;
        cudaGetDevice(&dev);
        if (dev >= 0 && dev < kMaxDevices && !raised[dev].load(std::memory_order_acquire)) {
            if (cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)cfg_smem(c, PF_DEC)) == cudaSuccess)
                raised[dev].store(true, std::memory_order_release);
        }
        return f;
    } else {
        return reinterpret_cast<const void *>(&filter_batched_kernel<c.tpp, c.dpt, PF_DEC, c.xe>);
    }
}

template <int I>
static cudaError_t launch_batched_i(int grid, const BatchArgs &b, int bin, cudaStream_t st) {
    constexpr KernelCfg c = kBatchCfgs[I];
    if constexpr (cfg_split(c, PF_DEC)) {
        batched_ptr_i<I>();  // sets the shared-memory limit once
        if constexpr (c.tpp == 1)
            filter_split_kernel<PF_DEC, c.xe, c.words>
                <<<grid, cfg_threads(c, PF_DEC), cfg_smem(c, PF_DEC), st>>>(b, bin);
        else
            filter_split_group_kernel<PF_DEC, c.tpp, c.dpt, c.words>
                <<<grid, cfg_threads(c, PF_DEC), cfg_smem(c, PF_DEC), st>>>(b, bin);
    } else {
        filter_batched_kernel<c.tpp, c.dpt, PF_DEC, c.xe><<<grid, 256, 0, st>>>(b, bin);
    }
    return cudaGetLastError();
}

template <int I>
static cudaError_t launch_batched_r(int cfg, int grid, const BatchArgs &b, int bin,
                                    cudaStream_t st) {
    if (cfg == I) return launch_batched_i<I>(grid, b, bin, st);
    if constexpr (I + 1 < kNumBatchCfgs) return launch_batched_r<I + 1>(cfg, grid, b, bin, st);
    return cudaErrorInvalidValue;
}

template <int I>
static const void *batched_ptr_r(int cfg) {
    if (cfg == I) return batched_ptr_i<I>();
    if constexpr (I + 1 < kNumBatchCfgs) return batched_ptr_r<I + 1>(cfg);
    return nullptr;
}

template <int I>
static cudaError_t launch_plain_i(const FilterArgs &a, cudaStream_t st) {
    const int64_t blocks = (a.n + 255) / 256;
    filter_plain_kernel<kPlainDpt[I], PF_DEC><<<(unsigned)blocks, 256, 0, st>>>(a);
    return cudaGetLastError();
}

template <int I>
static cudaError_t launch_plain_r(int i, const FilterArgs &a, cudaStream_t st) {
    if (i == I) return launch_plain_i<I>(a, st);
    if constexpr (I + 1 < kNumPlain) return launch_plain_r<I + 1>(i, a, st);
    return cudaErrorInvalidValue;
}

template <int XE>
static cudaError_t launch_plain_exact_r(int E, const FilterArgs &a, cudaStream_t st) {
    if (E == XE) {
        const int64_t blocks = (a.n + 255) / 256;
        filter_plain_exact_kernel<XE, PF_DEC><<<(unsigned)blocks, 256, 0, st>>>(a);
        return cudaGetLastError();
    }
    if constexpr (XE + 1 <= kPlainExactMaxE) return launch_plain_exact_r<XE + 1>(E, a, st);
    return cudaErrorInvalidValue;
}

cudaError_t PF_CAT(launch_plain_exact_dec, PF_DEC)(int E, const FilterArgs &a, cudaStream_t st) {
    if (a.n <= 0) return cudaSuccess;
    return launch_plain_exact_r<0>(E, a, st);
}

cudaError_t PF_CAT(launch_batched_dec, PF_DEC)(int cfg, int grid, const BatchArgs &b, int bin,
                                               cudaStream_t st) {
    return launch_batched_r<0>(cfg, grid, b, bin, st);
}

const void *PF_CAT(batched_fn_dec, PF_DEC)(int cfg) { return batched_ptr_r<0>(cfg); }

cudaError_t PF_CAT(launch_plain_dec, PF_DEC)(int i, const FilterArgs &a, cudaStream_t st) {
    if (a.n <= 0) return cudaSuccess;
    return launch_plain_r<0>(i, a, st);
}

}  // namespace pf

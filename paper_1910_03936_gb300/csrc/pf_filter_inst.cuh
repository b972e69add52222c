// Instantiates the filter kernels for one decider set PF_DEC (1, 2 or 3).
#include "pf_filter.cuh"
#include "pf_kernels.h"

namespace pf {

#define PF_CAT2(a, b) a##b
#define PF_CAT(a, b) PF_CAT2(a, b)

template <int TPP, int DPT>
static const void *batched_ptr() {
    return reinterpret_cast<const void *>(&filter_batched_kernel<TPP, DPT, PF_DEC>);
}

template <int... I>
struct CfgList {};

template <int I>
static const void *batched_ptr_i() {
    return batched_ptr<kBatchCfgs[I].tpp, kBatchCfgs[I].dpt>();
}

template <int I>
static cudaError_t launch_batched_i(int grid, const BatchArgs &b, int bin, cudaStream_t st) {
    filter_batched_kernel<kBatchCfgs[I].tpp, kBatchCfgs[I].dpt, PF_DEC><<<grid, 256, 0, st>>>(b,
                                                                                           bin);
    return cudaGetLastError();
}

template <int I>
static cudaError_t launch_plain_i(const FilterArgs &a, cudaStream_t st) {
    const int64_t blocks = (a.n + 255) / 256;
    filter_plain_kernel<kPlainDpt[I], PF_DEC><<<(unsigned)blocks, 256, 0, st>>>(a);
    return cudaGetLastError();
}

#define PF_B(I) case I: return launch_batched_i<I>(grid, b, bin, st);
#define PF_BP(I) case I: return batched_ptr_i<I>();
#define PF_ALL(X) X(0) X(1) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11) X(12) X(13) \
    X(14) X(15) X(16) X(17) X(18) X(19)
static_assert(kNumBatchCfgs == 20, "update PF_ALL");

cudaError_t PF_CAT(launch_batched_dec, PF_DEC)(int cfg, int grid, const BatchArgs &b, int bin,
                                               cudaStream_t st) {
    switch (cfg) {
        PF_ALL(PF_B)
        default: return cudaErrorInvalidValue;
    }
}

const void *PF_CAT(batched_fn_dec, PF_DEC)(int cfg) {
    switch (cfg) {
        PF_ALL(PF_BP)
        default: return nullptr;
    }
}

cudaError_t PF_CAT(launch_plain_dec, PF_DEC)(int i, const FilterArgs &a, cudaStream_t st) {
    if (a.n <= 0) return cudaSuccess;
    switch (i) {
        case 0: return launch_plain_i<0>(a, st);
        case 1: return launch_plain_i<1>(a, st);
        case 2: return launch_plain_i<2>(a, st);
        case 3: return launch_plain_i<3>(a, st);
        case 4: return launch_plain_i<4>(a, st);
        case 5: return launch_plain_i<5>(a, st);
        default: return cudaErrorInvalidValue;
    }
}
static_assert(kNumPlain == 6, "update launch_plain_dec");

}  // namespace pf

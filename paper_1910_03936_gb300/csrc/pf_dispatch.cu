// Routes a decider set to its instantiation unit.
#include "pf_kernels.h"

namespace pf {

cudaError_t launch_batched_dec1(int, int, const BatchArgs &, int, cudaStream_t);
cudaError_t launch_batched_dec2(int, int, const BatchArgs &, int, cudaStream_t);
cudaError_t launch_batched_dec3(int, int, const BatchArgs &, int, cudaStream_t);
const void *batched_fn_dec1(int);
const void *batched_fn_dec2(int);
const void *batched_fn_dec3(int);
cudaError_t launch_plain_dec1(int, const FilterArgs &, cudaStream_t);
cudaError_t launch_plain_dec2(int, const FilterArgs &, cudaStream_t);
cudaError_t launch_plain_dec3(int, const FilterArgs &, cudaStream_t);
cudaError_t launch_plain_exact_dec1(int, const FilterArgs &, cudaStream_t);
cudaError_t launch_plain_exact_dec2(int, const FilterArgs &, cudaStream_t);
cudaError_t launch_plain_exact_dec3(int, const FilterArgs &, cudaStream_t);

cudaError_t launch_filter_plain_exact(int dec, int E, const FilterArgs &a, cudaStream_t st) {
    switch (dec) {
        case 1: return launch_plain_exact_dec1(E, a, st);
        case 2: return launch_plain_exact_dec2(E, a, st);
        case 3: return launch_plain_exact_dec3(E, a, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_filter_plain(int dec, int plain_idx, const FilterArgs &a, cudaStream_t st) {
    switch (dec) {
        case 1: return launch_plain_dec1(plain_idx, a, st);
        case 2: return launch_plain_dec2(plain_idx, a, st);
        case 3: return launch_plain_dec3(plain_idx, a, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_filter_batched(int dec, int cfg, int grid, const BatchArgs &b, int bin,
                                  cudaStream_t st) {
    switch (dec) {
        case 1: return launch_batched_dec1(cfg, grid, b, bin, st);
        case 2: return launch_batched_dec2(cfg, grid, b, bin, st);
        case 3: return launch_batched_dec3(cfg, grid, b, bin, st);
    }
    return cudaErrorInvalidValue;
}

const void *filter_batched_fn(int dec, int cfg) {
    switch (dec) {
        case 1: return batched_fn_dec1(cfg);
        case 2: return batched_fn_dec2(cfg);
        case 3: return batched_fn_dec3(cfg);
    }
    return nullptr;
}

}  // namespace pf

// a6: verification kernel, one thread per pair (device function and its
// derivation in pf_verify.cuh).
#include "pf_verify.cuh"

namespace pf {

namespace {

template <typename U>
__global__ void __launch_bounds__(256)
verify_kernel(PairsView pv, const int32_t *lens, const int16_t *Es, int E_max,
              const int64_t *idx, const int64_t *n_idx, int64_t n, int32_t *dist,
              unsigned *err) {
    const int64_t count = idx ? min(*n_idx, n) : n;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < count;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = idx ? __ldg(idx + t) : t;
        const int m = __ldg(lens + p);
        const int E = Es ? (int)__ldg(Es + p) : E_max;
        if (m < 0 || E < 0 || E > E_max) {
            dist[p] = -1;
            atomicOr(err, ERR_PAIR_ARGS);
            continue;
        }
        dist[p] = verify_pair<U>(pv, p, m, E);
    }
}

}  // namespace

cudaError_t launch_verify(const PairsView &pv, const int32_t *lens, const int16_t *E, int E_max,
                          const int64_t *idx, const int64_t *n_idx, int64_t n, int32_t *dist,
                          unsigned *err, int sms, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    int64_t blocks = (n + 255) / 256;
    const int64_t cap = (int64_t)sms * 8;
    if (blocks > cap) blocks = cap;
    if (E_max <= 15)
        verify_kernel<uint32_t><<<(unsigned)blocks, 256, 0, st>>>(pv, lens, E, E_max, idx, n_idx,
                                                                  n, dist, err);
    else
        verify_kernel<uint64_t><<<(unsigned)blocks, 256, 0, st>>>(pv, lens, E, E_max, idx, n_idx,
                                                                  n, dist, err);
    return cudaGetLastError();
}

}  // namespace pf

// a6: verification kernel, one thread per pair (device function and its
// derivation in pf_verify.cuh).
#include "pf_verify.cuh"

namespace pf {

namespace {

// SPLIT (64-bit launches whose indices come grouped by threshold): a pair
// with E <= 15 takes the 32-bit band.  Grouped, a warp's pairs take one of
// the two; in pair order a warp would run both.
template <typename U, bool SPLIT>
__device__ __forceinline__ void verify_at(const PairsView &pv, const int32_t *lens,
                                          const int16_t *Es, int E_max, const int64_t *idx,
                                          int64_t t, int32_t *dist, unsigned *err) {
    const int64_t p = idx ? __ldg(idx + t) : t;
    const int m = __ldg(lens + p);
    const int E = Es ? (int)__ldg(Es + p) : E_max;
    if (m < 0 || E < 0 || E > E_max) {
        dist[p] = -1;
        atomicOr(err, ERR_PAIR_ARGS);
        return;
    }
    if (SPLIT && E <= 15) dist[p] = verify_pair<uint32_t>(pv, p, m, E);
    else dist[p] = verify_pair<U>(pv, p, m, E);
}

// Without a work counter each thread strides over the positions.  With one
// (zeroed before the launch) warps claim 32 consecutive positions at a time:
// when the indices come grouped by threshold and length, the costly groups
// lie together, and a fixed assignment would leave them to a few blocks.
template <typename U, bool SPLIT>
__global__ void __launch_bounds__(256)
verify_kernel(PairsView pv, const int32_t *lens, const int16_t *Es, int E_max,
              const int64_t *idx, const int64_t *n_idx, int64_t n, int32_t *dist,
              unsigned *err, unsigned long long *work) {
    const int64_t count = idx ? min(*n_idx, n) : n;
    if (work) {
        const int lane = threadIdx.x & 31;
        for (;;) {
            unsigned long long item = 0;
            if (lane == 0) item = atomicAdd(work, 1ull);
            item = __shfl_sync(0xffffffffu, item, 0);
            const int64_t t0 = (int64_t)item * 32;
            if (t0 >= count) break;
            if (t0 + lane < count)
                verify_at<U, SPLIT>(pv, lens, Es, E_max, idx, t0 + lane, dist, err);
        }
        return;
    }
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < count;
         t += (int64_t)gridDim.x * blockDim.x)
        verify_at<U, SPLIT>(pv, lens, Es, E_max, idx, t, dist, err);
}

}  // namespace

cudaError_t launch_verify(const PairsView &pv, const int32_t *lens, const int16_t *E, int E_max,
                          const int64_t *idx, const int64_t *n_idx, int64_t n, int32_t *dist,
                          unsigned *err, int sms, cudaStream_t st, unsigned long long *work,
                          bool grouped) {
    if (n <= 0) return cudaSuccess;
    int64_t blocks = (n + 255) / 256;
    const int64_t cap = (int64_t)sms * 8;
    if (blocks > cap) blocks = cap;
    if (work) {
        const cudaError_t e = cudaMemsetAsync(work, 0, sizeof(unsigned long long), st);
        if (e != cudaSuccess) return e;
    }
    if (E_max <= 15)
        verify_kernel<uint32_t, false><<<(unsigned)blocks, 256, 0, st>>>(
            pv, lens, E, E_max, idx, n_idx, n, dist, err, work);
    else if (grouped && E)
        verify_kernel<uint64_t, true><<<(unsigned)blocks, 256, 0, st>>>(
            pv, lens, E, E_max, idx, n_idx, n, dist, err, work);
    else
        verify_kernel<uint64_t, false><<<(unsigned)blocks, 256, 0, st>>>(
            pv, lens, E, E_max, idx, n_idx, n, dist, err, work);
    return cudaGetLastError();
}

}  // namespace pf

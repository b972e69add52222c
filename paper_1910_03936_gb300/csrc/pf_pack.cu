// a1: pack kernels.  One thread builds one 32-bit word of each plane from
// 32 bytes (device functions in pf_pack.cuh).
#include "pf_pack.cuh"

namespace pf {

namespace {

constexpr int kSeqPerBlock = 128;
constexpr int kPackThreads = 256;

// Ragged layout: block handles sequences [s0, s0 + kSeqPerBlock); its
// threads walk the block's words, finding each word's sequence by a binary
// search over the staged word offsets.
__global__ void __launch_bounds__(kPackThreads)
pack_ragged_kernel(const uint8_t *ascii, const int64_t *byte_off, const int64_t *word_off,
                   int64_t nseq, uint32_t *lo, uint32_t *hi, uint32_t *nm, unsigned *err) {
    __shared__ int64_t woff[kSeqPerBlock + 1];
    __shared__ int64_t boff[kSeqPerBlock + 1];
    const int64_t s0 = (int64_t)blockIdx.x * kSeqPerBlock;
    const int ns = (int)min((int64_t)kSeqPerBlock, nseq - s0);
    for (int i = threadIdx.x; i <= ns; i += blockDim.x) {
        woff[i] = word_off[s0 + i];
        boff[i] = byte_off[s0 + i];
    }
    __syncthreads();
    const uint8_t *lim = ascii + __ldg(byte_off + nseq);
    const int64_t base = woff[0];
    const int total = (int)(woff[ns] - base);
    for (int j = threadIdx.x; j < total; j += blockDim.x) {
        const int64_t gw = base + j;
        int l = 0, r = ns - 1;  // last sequence with woff <= gw
        while (l < r) {
            const int mid = (l + r + 1) >> 1;
            if (woff[mid] <= gw) l = mid; else r = mid - 1;
        }
        const int w = (int)(gw - woff[l]);
        const int len = (int)(boff[l + 1] - boff[l]);
        pack_word(ascii + boff[l], len, w, lo + gw, hi + gw, nm + gw, err, lim);
    }
}

// Fixed layout: sequence s is ascii[s*len ...], words [s*W, (s+1)*W).
// Block b packs global words [512 b, 512 b + 512), two per thread (t and
// t + 256, so each half is a coalesced run); both windows are loaded before
// either is decoded.  One 64-bit division per block locates its first
// word, threads step from there.
constexpr int kPackWordsPerThread = 2;

__global__ void __launch_bounds__(kPackThreads)
pack_fixed_kernel(const uint8_t *ascii, int64_t nseq, int len, int W, uint32_t wmagic,
                  uint32_t *lo, uint32_t *hi, uint32_t *nm, unsigned *err) {
    __shared__ int64_t s_first;
    __shared__ int w_first;
    const int64_t total = nseq * (int64_t)W;
    const int64_t gw0 = (int64_t)blockIdx.x * (kPackThreads * kPackWordsPerThread);
    if (threadIdx.x == 0) {
        s_first = gw0 / W;
        w_first = (int)(gw0 - s_first * W);
    }
    __syncthreads();
    const uint8_t *lim = ascii + nseq * (int64_t)len;
    PackWindow pw[kPackWordsPerThread];
    int64_t gws[kPackWordsPerThread];
#pragma unroll
    for (int r = 0; r < kPackWordsPerThread; ++r) {
        const unsigned local = (unsigned)w_first + threadIdx.x + (unsigned)(r * kPackThreads);
        gws[r] = gw0 + threadIdx.x + r * kPackThreads;
        if (gws[r] >= total) continue;
        // local / W by multiply-high when wmagic = ceil(2^32 / W) is exact for
        // every local < W + 512 (W <= 4096), else by division
        const unsigned q = wmagic ? __umulhi(local, wmagic) : local / (unsigned)W;
        const int64_t s = s_first + q;
        const int w = (int)(local - q * (unsigned)W);
        pack_load(ascii + s * (int64_t)len, len, w, lim, pw[r]);
    }
#pragma unroll
    for (int r = 0; r < kPackWordsPerThread; ++r) {
        if (gws[r] >= total) continue;
        const int64_t gw = gws[r];
        pack_decode(pw[r], lo + gw, hi + gw, nm + gw, err);
    }
}

}  // namespace

cudaError_t launch_pack_ragged(const uint8_t *ascii, const int64_t *byte_off,
                               const int64_t *word_off, int64_t nseq, uint32_t *lo,
                               uint32_t *hi, uint32_t *nm, unsigned *err, cudaStream_t st) {
    if (nseq <= 0) return cudaSuccess;
    const int64_t blocks = (nseq + kSeqPerBlock - 1) / kSeqPerBlock;
    pack_ragged_kernel<<<(unsigned)blocks, kPackThreads, 0, st>>>(ascii, byte_off, word_off,
                                                                 nseq, lo, hi, nm, err);
    return cudaGetLastError();
}

cudaError_t launch_pack_fixed(const uint8_t *ascii, int64_t nseq, int len, uint32_t *lo,
                              uint32_t *hi, uint32_t *nm, unsigned *err, int sms,
                              cudaStream_t st) {
    const int W = (len + 31) / 32;
    const int64_t total = nseq * (int64_t)W;
    if (total <= 0) return cudaSuccess;
    (void)sms;
    const int64_t per_block = kPackThreads * kPackWordsPerThread;
    const int64_t blocks = (total + per_block - 1) / per_block;
    const uint32_t wmagic =
        (W <= 4096) ? (uint32_t)((((uint64_t)1 << 32) + (uint64_t)W - 1) / (uint64_t)W) : 0u;
    pack_fixed_kernel<<<(unsigned)blocks, kPackThreads, 0, st>>>(ascii, nseq, len, W, wmagic,
                                                                lo, hi, nm, err);
    return cudaGetLastError();
}

}  // namespace pf

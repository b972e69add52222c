// a1: pack kernels.  The fixed layout decodes the buffer as a stream of
// aligned 32-byte chunks and cuts the sequences' words out of it; the
// ragged layout (and sequences longer than 4096 words) builds each 32-bit
// word of each plane from the 32 bytes of its own window (device functions
// in pf_pack.cuh).
#include "pf_pack.cuh"

namespace pf {

namespace {

constexpr int kPackThreads = 256;

// Chunks.  Chunk j of a buffer is its 32 bytes from A + 32 j, A = an
// address rounded down to 32 bytes; decoded, it is one word per plane whose
// bit b is byte A + 32 j + b, so the word of a sequence that starts at byte
// P of that stream is the stream's 32 bits from P: one funnel shift per
// plane over two chunk words.  A block decodes up to 4 chunks per thread,
// two 16-byte loads each (coalesced across the warp, no re-reads).
constexpr int kStreamChunksPerThread = 4;
constexpr int kStreamChunks = kStreamChunksPerThread * kPackThreads;
constexpr int kStreamWords = kStreamChunks - 1;

// Decode chunks [0, nchunks) from cbase (32-byte aligned) into chunk[].
// Bytes of [vbeg, vend) are the sequences'; the 4-byte words that hold
// them are read, others count as "NNNN"; a byte outside [vbeg, vend) that
// is not a base never raises the error.
__device__ __forceinline__ void decode_chunks(uintptr_t cbase, int nchunks, uintptr_t vbeg,
                                              uintptr_t vend, uint4 *chunk, unsigned *err) {
    const uintptr_t lo4 = vbeg & ~uintptr_t(3), hi4 = (vend + 3) & ~uintptr_t(3);
    uint32_t v[kStreamChunksPerThread][8];
#pragma unroll
    for (int r = 0; r < kStreamChunksPerThread; ++r) {
        const int c = threadIdx.x + r * kPackThreads;
        if (c >= nchunks) continue;
        const uintptr_t ca = cbase + 32 * (uintptr_t)c;
        if (ca >= lo4 && ca + 32 <= hi4) {
            const uint4 x0 = __ldg(reinterpret_cast<const uint4 *>(ca));
            const uint4 x1 = __ldg(reinterpret_cast<const uint4 *>(ca + 16));
            v[r][0] = x0.x; v[r][1] = x0.y; v[r][2] = x0.z; v[r][3] = x0.w;
            v[r][4] = x1.x; v[r][5] = x1.y; v[r][6] = x1.z; v[r][7] = x1.w;
        } else {
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const uintptr_t wa = ca + 4 * k;
                v[r][k] = (wa >= lo4 && wa < hi4) ? __ldg(reinterpret_cast<const uint32_t *>(wa))
                                                  : 0x4e4e4e4eu;
            }
        }
    }
#pragma unroll
    for (int r = 0; r < kStreamChunksPerThread; ++r) {
        const int c = threadIdx.x + r * kPackThreads;
        if (c >= nchunks) continue;
        uint32_t l, h, n;
        if (decode32(v[r], l, h, n)) {
            const uintptr_t ca = cbase + 32 * (uintptr_t)c;
            const int vlo = (vbeg > ca) ? (int)(vbeg - ca) : 0;
            const int vhi = (vend < ca + 32) ? (int)((intptr_t)vend - (intptr_t)ca) : 32;
            const uint4 e = slow_chunk(make_uint4(v[r][0], v[r][1], v[r][2], v[r][3]),
                                       make_uint4(v[r][4], v[r][5], v[r][6], v[r][7]), vlo, vhi);
            if (e.w) atomicOr(err, ERR_BYTES);
            l = e.x;
            h = e.y;
            n = e.z;
        }
        chunk[c] = make_uint4(l, h, n, 0u);
    }
}

// Ragged layout: block handles sequences [s0, s0 + kSeqPerBlock); its
// threads walk the block's words, each decoding its word from its own
// 32-byte window.  A word's sequence comes from a map in shared memory
// (one byte per word, written by the sequences' threads; a block whose
// sequences hold more than kMapCap words searches the staged offsets
// instead).  (Decoding the block's bytes as one chunk stream first, as the
// fixed layout does, was slower here: the extra round of memory latency for
// the offsets left too little work per block to hide it.)  Words past
// ceil(len/32) of a sequence (a word_off with room to spare) are all N.
// With seg_of given, a byte error of sequence s is recorded in
// seg_err[seg_of[s]] instead of err (the serving batches attribute errors
// to the request a sequence came from).
//
// STARTS: word_off holds each sequence's first word, in any order (a layout
// that groups sequences by threshold and length); the block lays its
// sequences' ceil(len/32) words out locally (a prefix sum by one warp) and
// writes word w of sequence s to word_off[s] + w.
constexpr int kSeqPerBlock = 256;
constexpr int kMapCap = 16 * kSeqPerBlock;

// Six blocks per SM: at eight the kernel's 32 registers spill.
template <bool STARTS>
__global__ void __launch_bounds__(kPackThreads, 6)
pack_ragged_kernel(const uint8_t *ascii, const int64_t *byte_off, const int64_t *word_off,
                   int64_t nseq, uint32_t *lo, uint32_t *hi, uint32_t *nm, unsigned *err,
                   const int32_t *seg_of, unsigned *seg_err) {
    __shared__ int woff[kSeqPerBlock + 1];       // block-local first word, rising
    __shared__ int64_t wdst[kSeqPerBlock + 1];   // first word in the planes
    __shared__ int64_t boff[kSeqPerBlock + 1];
    __shared__ int32_t sseg[kSeqPerBlock];
    __shared__ uint8_t wseq[kMapCap];            // local word -> local sequence
    const int64_t s0 = (int64_t)blockIdx.x * kSeqPerBlock;
    const int ns = (int)min((int64_t)kSeqPerBlock, nseq - s0);
    for (int i = threadIdx.x; i <= ns; i += blockDim.x) {
        boff[i] = byte_off[s0 + i];
        if (!STARTS || i < ns) wdst[i] = word_off[s0 + i];
        if (seg_of && i < ns) sseg[i] = seg_of[s0 + i];
    }
    __syncthreads();
    if constexpr (STARTS) {
        constexpr int PER = kSeqPerBlock / 32;
        if (threadIdx.x < 32) {
            const int lane = threadIdx.x;
            int c[PER];
            int sum = 0;
#pragma unroll
            for (int k = 0; k < PER; ++k) {
                const int i = lane * PER + k;
                const int64_t len = (i < ns) ? boff[i + 1] - boff[i] : 0;
                c[k] = len > 0 ? (int)((len + 31) >> 5) : 0;
                sum += c[k];
            }
            int inc = sum;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += t;
            }
            int run = inc - sum;
#pragma unroll
            for (int k = 0; k < PER; ++k) {
                woff[lane * PER + k] = run;
                run += c[k];
            }
            if (lane == 31) woff[kSeqPerBlock] = inc;
        }
    } else {
        for (int i = threadIdx.x; i <= ns; i += blockDim.x) woff[i] = (int)(wdst[i] - wdst[0]);
    }
    __syncthreads();
    const int total = woff[ns];
    const bool direct = total <= kMapCap;
    if (direct)
        for (int i = threadIdx.x; i < ns; i += blockDim.x)
            for (int j = woff[i]; j < woff[i + 1]; ++j) wseq[j] = (uint8_t)i;
    __syncthreads();
    const uint8_t *lim = ascii + __ldg(byte_off + nseq);
    for (int j = threadIdx.x; j < total; j += blockDim.x) {
        int l;
        if (direct) {
            l = wseq[j];
        } else {  // last sequence with woff <= j
            int r = ns - 1;
            l = 0;
            while (l < r) {
                const int mid = (l + r + 1) >> 1;
                if (woff[mid] <= j) l = mid; else r = mid - 1;
            }
        }
        const int w = j - woff[l];
        const int64_t dst = STARTS ? wdst[l] + w : wdst[0] + j;
        const int len = (int)(boff[l + 1] - boff[l]);
        if (len - 32 * w <= 0) {
            lo[dst] = 0u;
            hi[dst] = 0u;
            nm[dst] = 0xffffffffu;
            continue;
        }
        pack_word(ascii + boff[l], len, w, lo + dst, hi + dst, nm + dst,
                  seg_of ? seg_err + sseg[l] : err, lim);
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

// Stream-tiled fixed layout: word w of sequence s starts at byte s*len + 32 w
// of the buffer.  A block packs kStreamWords consecutive words (s-major):
// their start bytes rise by at most 32 from one word to the next, so they
// span at most kStreamWords + 1 chunks (from A = the buffer start rounded
// down to 32 bytes), which the block decodes into shared memory first, then
// cuts out its words.
__global__ void __launch_bounds__(kPackThreads, 5)
pack_stream_kernel(const uint8_t *ascii, int64_t nseq, int len, int W, uint32_t wmagic,
                   uint32_t *lo, uint32_t *hi, uint32_t *nm, unsigned *err) {
    __shared__ uint4 chunk[kStreamWords + 1];
    __shared__ int64_t s_j0;
    __shared__ int s_wfirst, s_nchunks, s_base;
    const int64_t total = nseq * (int64_t)W;
    const int64_t g0 = (int64_t)blockIdx.x * kStreamWords;
    const uintptr_t src = reinterpret_cast<uintptr_t>(ascii);
    const uintptr_t A = src & ~uintptr_t(31);
    const int delta = (int)(src - A);
    if (threadIdx.x == 0) {
        const int64_t sf = g0 / W;
        const int wf = (int)(g0 - sf * W);
        const int64_t g1 = min(g0 + kStreamWords, total) - 1;
        const int64_t sl = g1 / W;
        const int64_t pf = sf * len + 32 * wf + delta;  // bytes from A
        const int64_t pl = sl * len + 32 * (g1 - sl * W) + delta;
        s_j0 = pf >> 5;
        s_wfirst = wf;
        s_nchunks = (int)((pl >> 5) + 2 - (pf >> 5));
        s_base = (int)((pf & 31) - 32 * wf);  // s_first*len + delta - 32*j0
    }
    __syncthreads();
    const int nchunks = s_nchunks;
    const uintptr_t cbase = A + 32 * (uintptr_t)s_j0;
    // the bytes of the buffer
    const uintptr_t vbeg = src, vend = src + (uintptr_t)(nseq * (int64_t)len);
    decode_chunks(cbase, nchunks, vbeg, vend, chunk, err);
    __syncthreads();

#pragma unroll
    for (int r = 0; r < kStreamChunksPerThread; ++r) {
        const int i = threadIdx.x + r * kPackThreads;
        const int64_t g = g0 + i;
        if (i >= kStreamWords || g >= total) continue;
        // (w_first + i) / W by multiply-high: with wmagic = ceil(2^32 / W) and
        // 2 <= W <= 4096 the quotient is exact for every numerator below 2^20
        // (ceil(2^32 / 1) does not fit 32 bits: W = 1 divides by itself)
        const unsigned local = (unsigned)s_wfirst + (unsigned)i;
        const unsigned q = (W == 1) ? local : __umulhi(local, wmagic);
        const int w = (int)(local - q * (unsigned)W);
        const int P = (int)q * len + 32 * w + s_base;  // byte of the word from chunk 0
        const int j = P >> 5;
        const unsigned sh = (unsigned)P & 31u;
        const uint4 x = chunk[j], y = chunk[j + 1];
        uint32_t l = __funnelshift_r(x.x, y.x, sh);
        uint32_t h = __funnelshift_r(x.y, y.y, sh);
        uint32_t n = __funnelshift_r(x.z, y.z, sh);
        const int vb = len - 32 * w;
        if (vb < 32) {  // bytes past the end of the sequence are N
            const uint32_t m = (1u << vb) - 1u;
            l &= m;
            h &= m;
            n |= ~m;
        }
        lo[g] = l;
        hi[g] = h;
        nm[g] = n;
    }
}

}  // namespace

cudaError_t launch_pack_ragged(const uint8_t *ascii, const int64_t *byte_off,
                               const int64_t *word_off, int64_t nseq, uint32_t *lo,
                               uint32_t *hi, uint32_t *nm, unsigned *err, cudaStream_t st,
                               const int32_t *seg_of, unsigned *seg_err) {
    if (nseq <= 0) return cudaSuccess;
    const int64_t blocks = (nseq + kSeqPerBlock - 1) / kSeqPerBlock;
    pack_ragged_kernel<false><<<(unsigned)blocks, kPackThreads, 0, st>>>(
        ascii, byte_off, word_off, nseq, lo, hi, nm, err, seg_of, seg_err);
    return cudaGetLastError();
}

cudaError_t launch_pack_starts(const uint8_t *ascii, const int64_t *byte_off,
                               const int64_t *word_start, int64_t nseq, uint32_t *lo,
                               uint32_t *hi, uint32_t *nm, unsigned *err, cudaStream_t st) {
    if (nseq <= 0) return cudaSuccess;
    const int64_t blocks = (nseq + kSeqPerBlock - 1) / kSeqPerBlock;
    pack_ragged_kernel<true><<<(unsigned)blocks, kPackThreads, 0, st>>>(
        ascii, byte_off, word_start, nseq, lo, hi, nm, err, nullptr, nullptr);
    return cudaGetLastError();
}

cudaError_t launch_pack_fixed(const uint8_t *ascii, int64_t nseq, int len, uint32_t *lo,
                              uint32_t *hi, uint32_t *nm, unsigned *err, int sms,
                              cudaStream_t st) {
    const int W = (len + 31) / 32;
    const int64_t total = nseq * (int64_t)W;
    if (total <= 0) return cudaSuccess;
    (void)sms;
    if (W <= 4096) {
        const int64_t blocks = (total + kStreamWords - 1) / kStreamWords;
        const uint32_t wmagic =
            (W == 1) ? 0u : (uint32_t)((((uint64_t)1 << 32) + (uint64_t)W - 1) / (uint64_t)W);
        pack_stream_kernel<<<(unsigned)blocks, kPackThreads, 0, st>>>(ascii, nseq, len, W, wmagic,
                                                                     lo, hi, nm, err);
        return cudaGetLastError();
    }
    const int64_t per_block = kPackThreads * kPackWordsPerThread;
    const int64_t blocks = (total + per_block - 1) / per_block;
    pack_fixed_kernel<<<(unsigned)blocks, kPackThreads, 0, st>>>(ascii, nseq, len, W, 0u, lo, hi,
                                                                nm, err);
    return cudaGetLastError();
}

}  // namespace pf

// Internal declarations shared by the CUDA sources of the library.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "pf.h"

namespace pf {

// Device-side error bits, accumulated in a context-owned word and turned
// into a status by pf_sync.
enum : unsigned {
    ERR_PAIR_ARGS = 1u,   // a pair with len < 0 or E outside [0, E_max]
    ERR_BYTES = 2u,       // a byte outside A/C/G/T/N in pf_pack
    ERR_TIMEOUT = 4u,     // a bounded device wait ran out
};

// Load policies.  LdNC: read-only data cache (data that no kernel writes
// while the reader runs).  LdCG: L2 only, for data that a long-running
// kernel reads after it was written during its lifetime (copy-engine
// uploads, words the same block just produced), where an L1 or read-only
// cache line from earlier could be stale.
struct LdNC {
    template <typename T>
    static __device__ __forceinline__ T ld(const T *p) { return __ldg(p); }
};
struct LdCG {
    template <typename T>
    static __device__ __forceinline__ T ld(const T *p) { return __ldcg(p); }
};

// Plain-old-data view of one set of packed sequences, passed by value.
struct SeqView {
    const uint32_t *lo, *hi, *nm;
    const int64_t *off;   // per-sequence first word, or null
    int64_t stride;       // words per sequence when off is null
    template <typename L = LdNC>
    __device__ __forceinline__ int64_t start(int64_t s) const {
        return off ? L::ld(off + s) : s * stride;
    }
};

struct PairsView {
    SeqView read, ref;
};

// One 32-bit word of each plane; words outside a sequence read as N.
struct Word3 {
    uint32_t lo, hi, nm;
};

template <typename L = LdNC>
__device__ __forceinline__ Word3 load_word(const SeqView &v, int64_t base, int q, int W) {
    Word3 r;
    if (q >= 0 && q < W) {
        r.lo = L::ld(v.lo + base + q);
        r.hi = L::ld(v.hi + base + q);
        r.nm = L::ld(v.nm + base + q);
    } else {
        r.lo = 0u; r.hi = 0u; r.nm = 0xffffffffu;
    }
    return r;
}

// AND of x over the TPP lanes of a lane group (TPP a power of two <= 32,
// groups aligned to TPP lanes); `gmask` names the group's lanes.
template <int TPP>
__device__ __forceinline__ uint32_t group_and(uint32_t x, unsigned gmask) {
    if constexpr (TPP == 32) {
        return __reduce_and_sync(0xffffffffu, x);
    } else {
#pragma unroll
        for (int o = 1; o < TPP; o <<= 1) x &= __shfl_xor_sync(gmask, x, o, TPP);
        return x;
    }
}

// Filter launch parameters shared by the plain and the batched kernels.
struct FilterArgs {
    PairsView pairs;
    const int32_t *lens = nullptr;
    const int16_t *E = nullptr;     // null: every pair uses E_max
    int E_max = 0;
    uint8_t *accept = nullptr;
    int16_t *count = nullptr;
    int64_t n = 0;
    unsigned *err = nullptr;
    int32_t *dist = nullptr;  // non-null: E + 1 for pairs the first decider rejects, -1 if invalid
    // Non-null (SneakySnake selected only): 1 for the SneakySnake-accepted pairs that
    // still need verification; a pair whose obstacle count equals its Hamming
    // distance gets 0 here and that count as its distance in dist.
    uint8_t *need = nullptr;
};

// Warps per block of the two-phase filter kernel.
constexpr int kSplitWarps = 4;

// Batched (scheduler) launch: pairs taken in chunks from `order` (null:
// identity) through a work counter.
struct BatchArgs {
    FilterArgs f;
    const int64_t *order;        // pair index per position, grouped by bin
    const int64_t *bin_start;    // [nbins+1] positions where bins start
    const int *bin_cfg;          // kernel configuration id per bin
    int nbins;
    int chunk;                   // pairs per work item
    unsigned long long *work;    // work-item counter (scratch, zeroed)
    const int64_t *chunk_start;  // [nbins+1] first work item of each bin
    const int *ident;            // device flag: order is the identity (one bin used)
};

}  // namespace pf

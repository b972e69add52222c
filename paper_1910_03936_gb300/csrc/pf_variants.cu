// The thesis's other deciders and knobs on the same neighbourhood map:
//   - SneakySnake on non-overlapping sub-matrices of t columns with y
//     replications per sub-matrix (§8.5, the FPGA architecture's knob);
//   - Shouji (Ch. 6): 4-column sliding windows and the Shouji bit-vector;
//   - GateKeeper with SHD's conventions (Ch. 3): vacant cells 0 instead of
//     1, and/or streak counting of the final bit-vector.
// One thread per pair over a grid-stride loop; the map is built one 32-column
// word at a time exactly as in the fused filter (pf_filter.cuh).  The largest
// threshold of a launch bounds the per-thread arrays (template EMAX).
// Contracts: pf_filter_partitioned, pf_filter_shouji, pf_filter_shd in pf.h.
#include <algorithm>

#include "pf_ctx.h"
#include "pf_filter.cuh"
#include "pf_kernels.h"

namespace pf {

namespace {

struct VariantArgs {
    PairsView pairs;
    const int32_t *lens;
    const int16_t *E;  // null: E_max for every pair
    int E_max;
    int p0, p1;        // t and y, or the SHD flags
    uint8_t *accept;
    int16_t *count;
    int64_t n;
    unsigned *err;
};

__device__ __forceinline__ bool variant_args(const VariantArgs &a, int64_t p, int *m, int *E) {
    *m = __ldg(a.lens + p);
    *E = a.E ? (int)__ldg(a.E + p) : a.E_max;
    if (*m < 0 || *E < 0 || *E > a.E_max) {
        a.count[p] = -1;
        a.accept[p] = 0;
        atomicOr(a.err, ERR_PAIR_ARGS);
        return false;
    }
    return true;
}

__device__ __forceinline__ void variant_out(const VariantArgs &a, int64_t p, int E, int c) {
    const int s = c > E + 1 ? E + 1 : c;
    a.count[p] = (int16_t)s;
    a.accept[p] = (uint8_t)(s <= E);
}

// Read words w-1, w, w+1 and reference word w of one pair, rolled a word at
// a time (words outside the sequences read as N).
struct Cursor {
    int64_t rb, fb;
    int W, w;
    Word3 Rm1, R0, Rp1, F;

    __device__ __forceinline__ void start(const PairsView &pv, int64_t p, int m) {
        W = (m + 31) >> 5;
        w = 0;
        rb = pv.read.start(p);
        fb = pv.ref.start(p);
        Rm1 = load_word(pv.read, rb, -1, W);
        R0 = load_word(pv.read, rb, 0, W);
        Rp1 = load_word(pv.read, rb, 1, W);
        F = load_word(pv.ref, fb, 0, W);
    }
    __device__ __forceinline__ void next(const PairsView &pv) {
        ++w;
        Rm1 = R0;
        R0 = Rp1;
        Rp1 = load_word(pv.read, rb, w + 1, W);
        F = load_word(pv.ref, fb, w, W);
    }
    // Mismatch word of diagonal d (cell (i, d): reference base i against
    // read base i + d); cells whose read index is outside the read, and
    // columns past the reference, are 1.
    __device__ __forceinline__ uint32_t map(int d) const {
        uint32_t slo, shi, snm;
        if (d < 0) {
            slo = shr_pair(Rm1.lo, R0.lo, d);
            shi = shr_pair(Rm1.hi, R0.hi, d);
            snm = shr_pair(Rm1.nm, R0.nm, d);
        } else {
            slo = shr_pair(R0.lo, Rp1.lo, d);
            shi = shr_pair(R0.hi, Rp1.hi, d);
            snm = shr_pair(R0.nm, Rp1.nm, d);
        }
        return (F.lo ^ slo) | (F.hi ^ shi) | F.nm | snm;
    }
};

// ---- SneakySnake on sub-matrices (§8.5) ------------------------------------
//
// Sub-matrix [b, b + t_s) with t_s = min(t, m - b) <= 32 lies in map words
// A (word b/32) and B (the next one).  Its rows are the funnel shift of the
// two words by b mod 32, with a wall of ones from bit t_s on (a pipe that
// reaches it leaves the sub-matrix).  Each replication is one SneakySnake
// step: the lowest bit of AND_d (y_d | -y_d), y_d the row from the current
// column on, is the end of the deepest pipe; below the wall it is an
// obstacle (counted, the search resumes one column further), at the wall
// the sub-matrix is done.  Its obstacles are those of its first y
// replications, min(y, t_s - sum of the pipe depths).
template <int EMAX>
__global__ void __launch_bounds__(256) partitioned_kernel(VariantArgs a) {
    constexpr int NSMAX = 2 * EMAX + 1;
    const int t = a.p0, y = a.p1;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < a.n;
         p += (int64_t)gridDim.x * blockDim.x) {
        int m, E;
        if (!variant_args(a, p, &m, &E)) continue;
        const int ns = 2 * E + 1;
        Cursor x;
        x.start(a.pairs, p, m);
        uint32_t A[NSMAX], B[NSMAX];
#pragma unroll
        for (int k = 0; k < NSMAX; ++k)
            if (k < ns) A[k] = x.map(k - E);
        x.next(a.pairs);
#pragma unroll
        for (int k = 0; k < NSMAX; ++k)
            if (k < ns) B[k] = x.map(k - E);
        int wa = 0, total = 0;
        for (int b = 0; b < m && total <= E; b += t) {
            while (wa < (b >> 5)) {  // slide the two words forward
                x.next(a.pairs);
#pragma unroll
                for (int k = 0; k < NSMAX; ++k)
                    if (k < ns) {
                        A[k] = B[k];
                        B[k] = x.map(k - E);
                    }
                ++wa;
            }
            const unsigned off = (unsigned)b & 31u;
            const int ts = min(t, m - b);
            const uint32_t wall = ts >= 32 ? 0u : (0xffffffffu << ts);
            uint32_t C = 0xffffffffu;
            for (int o = 0; o < y; ++o) {
                uint32_t T = 0xffffffffu;
#pragma unroll
                for (int k = 0; k < NSMAX; ++k)
                    if (k < ns) {
                        const uint32_t v = (__funnelshift_r(A[k], B[k], off) | wall) & C;
                        T &= v | (0u - v);
                    }
                if (T == 0u) break;          // a pipe runs to the end (t_s = 32)
                const int pos = __ffs(T) - 1;
                if (pos >= ts) break;        // the wall: sub-matrix done
                ++total;
                if (pos + 1 >= ts) break;    // the obstacle was its last column
                C = 0xfffffffeu << pos;
            }
        }
        variant_out(a, p, E, total);
    }
}

// ---- Shouji (Ch. 6) ---------------------------------------------------------
//
// Window c covers columns c..c+3.  For the 32 windows that start in word w,
// each row's window bits are the row word shifted by 0..3 (bits from the next
// word), their count of ones is added bit-sliced, and the cost 2*ones +
// (first bit) is minimised over the rows in the order d = -E..E, the first
// row winning ties: most zeros, then a leading zero, then the first row.
// The winning vectors stay as four bit-planes V0..V3.  The bit-vector is
// then updated column by column: the state is its bits c, c+1, c+2 (bit
// c+3 is still the initial 1, no earlier window reached it); the window's
// vector replaces the four bits when it has fewer ones, and bit c is final.
__device__ __forceinline__ uint32_t sel(uint32_t mask, uint32_t a, uint32_t b) {
    return (a & mask) | (b & ~mask);
}

template <int EMAX>
__global__ void __launch_bounds__(256) shouji_kernel(VariantArgs a) {
    constexpr int NSMAX = 2 * EMAX + 1;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < a.n;
         p += (int64_t)gridDim.x * blockDim.x) {
        int m, E;
        if (!variant_args(a, p, &m, &E)) continue;
        const int ns = 2 * E + 1;
        Cursor x;
        x.start(a.pairs, p, m);
        uint32_t A[NSMAX], B[NSMAX];
#pragma unroll
        for (int k = 0; k < NSMAX; ++k)
            if (k < ns) A[k] = x.map(k - E);
        x.next(a.pairs);
#pragma unroll
        for (int k = 0; k < NSMAX; ++k)
            if (k < ns) B[k] = x.map(k - E);
        unsigned state = 7u;  // bits c, c+1, c+2 of the bit-vector
        int ones = 0;
        for (int w = 0; w < x.W && ones <= E; ++w) {
            uint32_t V0 = 0, V1 = 0, V2 = 0, V3 = 0, K0 = 0, K1 = 0, K2 = 0, K3 = 0;
#pragma unroll
            for (int k = 0; k < NSMAX; ++k) {
                if (k >= ns) continue;
                const uint32_t b0 = A[k];
                const uint32_t b1 = __funnelshift_r(A[k], B[k], 1);
                const uint32_t b2 = __funnelshift_r(A[k], B[k], 2);
                const uint32_t b3 = __funnelshift_r(A[k], B[k], 3);
                // ones of the window, 0..4, as bits o2 o1 o0
                const uint32_t s01 = b0 ^ b1, c01 = b0 & b1, s23 = b2 ^ b3, c23 = b2 & b3;
                const uint32_t cc = s01 & s23;
                const uint32_t o0 = s01 ^ s23;
                const uint32_t o1 = c01 ^ c23 ^ cc;
                const uint32_t o2 = (c01 & c23) | ((c01 ^ c23) & cc);
                // cost bits k3 k2 k1 k0 = o2 o1 o0 b0
                if (k == 0) {
                    V0 = b0; V1 = b1; V2 = b2; V3 = b3;
                    K0 = b0; K1 = o0; K2 = o1; K3 = o2;
                } else {
                    // cost < K, per column, most significant bit first
                    const uint32_t eq3 = ~(o2 ^ K3), eq2 = ~(o1 ^ K2), eq1 = ~(o0 ^ K1);
                    const uint32_t lt = (~o2 & K3) |
                                        (eq3 & ((~o1 & K2) | (eq2 & ((~o0 & K1) |
                                                                      (eq1 & ~b0 & K0)))));
                    V0 = sel(lt, b0, V0); V1 = sel(lt, b1, V1);
                    V2 = sel(lt, b2, V2); V3 = sel(lt, b3, V3);
                    K0 = sel(lt, b0, K0); K1 = sel(lt, o0, K1);
                    K2 = sel(lt, o1, K2); K3 = sel(lt, o2, K3);
                }
            }
            const int ncol = min(32, m - 32 * w);
            for (int c = 0; c < ncol; ++c) {
                const unsigned v = ((V0 >> c) & 1u) | (((V1 >> c) & 1u) << 1) |
                                   (((V2 >> c) & 1u) << 2) | (((V3 >> c) & 1u) << 3);
                const unsigned cur = state | 8u;
                const unsigned nxt = (__popc(v) < __popc(cur)) ? v : cur;
                ones += (int)(nxt & 1u);
                state = nxt >> 1;
            }
            x.next(a.pairs);
#pragma unroll
            for (int k = 0; k < NSMAX; ++k)
                if (k < ns) {
                    A[k] = B[k];
                    B[k] = x.map(k - E);
                }
        }
        variant_out(a, p, E, ones);
    }
}

// ---- GateKeeper with SHD's conventions (Ch. 3) --------------------------------
//
// As GateKeeper in the fused filter: Hamming count of the d = 0 mask, word
// w-1 amended once word w is built, AND over the rows.  With vacant zero,
// cells whose read index is outside the read are cleared before the amend
// (d < 0: columns below -d; d > 0: columns from m - d on).  With streak
// counting, each maximal run of L ones of the final bit-vector costs
// ceil(L / 3); a run that reaches the end of a word continues into the next.
struct Streak {
    int run = 0, count = 0;
    // the final bits of one word; `last` closes a run that reaches its end
    __device__ __forceinline__ void add(uint32_t x, int nbits, bool last) {
        if (run > 0) {
            const int lead = (~x == 0u) ? 32 : __ffs(~x) - 1;  // ones from bit 0
            if (lead >= nbits) {
                run += nbits;
                if (last) flush();
                return;
            }
            run += lead;
            flush();
            x &= ~((lead >= 32) ? 0xffffffffu : ((1u << lead) - 1u));
        }
        while (x) {
            const int s = __ffs(x) - 1;
            const uint32_t rest = ~(x >> s);
            const int len = (rest == 0u) ? 32 - s : __ffs(rest) - 1;
            if (s + len >= nbits) {  // reaches the end of the word
                run = nbits - s;
                if (last) flush();
                return;
            }
            count += (len + 2) / 3;
            x &= ~(((len >= 32) ? 0xffffffffu : ((1u << len) - 1u)) << s);
        }
    }
    __device__ __forceinline__ void flush() {
        count += (run + 2) / 3;
        run = 0;
    }
};

template <int EMAX>
__global__ void __launch_bounds__(256) shd_kernel(VariantArgs a) {
    constexpr int NSMAX = 2 * EMAX + 1;
    const bool vacant_zero = (a.p0 & (int)PF_SHD_VACANT_ZERO) != 0;
    const bool streak = (a.p0 & (int)PF_SHD_STREAK) != 0;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < a.n;
         p += (int64_t)gridDim.x * blockDim.x) {
        int m, E;
        if (!variant_args(a, p, &m, &E)) continue;
        if (m == 0) {
            variant_out(a, p, E, 0);
            continue;
        }
        const int ns = 2 * E + 1;
        Cursor x;
        x.start(a.pairs, p, m);
        uint32_t Mp[NSMAX], Mpp[NSMAX];
#pragma unroll
        for (int k = 0; k < NSMAX; ++k) { Mp[k] = 0u; Mpp[k] = 0u; }
        int h = 0, fc = 0;
        Streak st;
        const int W = x.W;
        for (int w = 0; w <= W; ++w) {
            // mask words of word w (all 0 past the last word), columns >= m cleared
            uint32_t M[NSMAX];
            const int lo = m - 32 * w;  // columns of word w below m
            const uint32_t valid = lo >= 32 ? 0xffffffffu : (lo <= 0 ? 0u : ((1u << lo) - 1u));
#pragma unroll
            for (int k = 0; k < NSMAX; ++k) {
                if (k >= ns) continue;
                const int d = k - E;
                uint32_t v = x.map(d) & valid;
                if (vacant_zero) {
                    uint32_t vac = 0u;
                    if (d < 0 && w == 0) vac = (1u << (-d)) - 1u;
                    if (d > 0) {
                        const int from = m - d - 32 * w;  // first vacant column in this word
                        vac = from <= 0 ? 0xffffffffu : (from >= 32 ? 0u : (0xffffffffu << from));
                    }
                    v &= ~vac;
                }
                M[k] = v;
            }
            if (w < W) h += __popc(x.map(0) & valid);  // the d = 0 mask (no vacant cells)
            if (w > 0) {  // amend word w-1 and AND the rows
                uint32_t Fa = 0xffffffffu;
#pragma unroll
                for (int k = 0; k < NSMAX; ++k) {
                    if (k >= ns) continue;
                    const uint32_t H = Mp[k];
                    const uint32_t l1 = __funnelshift_l(Mpp[k], H, 1);
                    const uint32_t l2 = __funnelshift_l(Mpp[k], H, 2);
                    const uint32_t r1 = __funnelshift_r(H, M[k], 1);
                    const uint32_t r2 = __funnelshift_r(H, M[k], 2);
                    Fa &= H | (l1 & (r1 | r2)) | (l2 & r1);
                }
                const int nb = min(32, m - 32 * (w - 1));
                Fa &= nb >= 32 ? 0xffffffffu : ((1u << nb) - 1u);
                if (streak) st.add(Fa, nb, w == W);
                else fc += __popc(Fa);
                const int c = streak ? st.count + (st.run + 2) / 3 : fc;
                if (h > E && c > E) break;  // both past E: the count saturates
            }
#pragma unroll
            for (int k = 0; k < NSMAX; ++k)
                if (k < ns) {
                    Mpp[k] = Mp[k];
                    Mp[k] = M[k];
                }
            if (w < W) x.next(a.pairs);
        }
        const int c = streak ? st.count + (st.run + 2) / 3 : fc;
        variant_out(a, p, E, h <= E ? h : c);
    }
}

template <template <int> class K>
cudaError_t launch_variant(const VariantArgs &a, int sms, cudaStream_t st);

template <int EMAX>
struct PartitionedK {
    static void go(dim3 g, cudaStream_t st, const VariantArgs &a) {
        partitioned_kernel<EMAX><<<g, 256, 0, st>>>(a);
    }
};
template <int EMAX>
struct ShoujiK {
    static void go(dim3 g, cudaStream_t st, const VariantArgs &a) {
        shouji_kernel<EMAX><<<g, 256, 0, st>>>(a);
    }
};
template <int EMAX>
struct ShdK {
    static void go(dim3 g, cudaStream_t st, const VariantArgs &a) {
        shd_kernel<EMAX><<<g, 256, 0, st>>>(a);
    }
};

template <template <int> class K>
cudaError_t launch_variant(const VariantArgs &a, int sms, cudaStream_t st) {
    if (a.n <= 0) return cudaSuccess;
    const int64_t blocks = std::min<int64_t>((a.n + 255) / 256, (int64_t)sms * 8);
    const dim3 g((unsigned)blocks);
    if (a.E_max <= 7) K<7>::go(g, st, a);
    else if (a.E_max <= 15) K<15>::go(g, st, a);
    else K<31>::go(g, st, a);
    return cudaGetLastError();
}

}  // namespace

}  // namespace pf

using namespace pf;

static pf_status variant_common(pf_ctx *ctx, const pf_pairs *pairs, const int32_t *lens,
                                int E_max, uint8_t *accept, int16_t *count, int64_t n,
                                const char *who) {
    if (!ctx) return PF_EINVAL;
    if (n < 0 || E_max < 0 || E_max > PF_MAX_E)
        return ctx->fail(PF_EINVAL, "%s: bad n or E_max", who);
    if (n > 0 && (!pairs || !lens || !accept || !count))
        return ctx->fail(PF_EINVAL, "%s: null pointer argument", who);
    return PF_OK;
}

static VariantArgs variant_args_of(pf_ctx *ctx, const pf_pairs *pairs, const int32_t *lens,
                                   const int16_t *E, int E_max, int p0, int p1,
                                   uint8_t *accept, int16_t *count, int64_t n) {
    VariantArgs a;
    a.pairs.read = SeqView{pairs->read.lo, pairs->read.hi, pairs->read.nmask,
                           pairs->read.word_off, pairs->read.stride_words};
    a.pairs.ref = SeqView{pairs->ref.lo, pairs->ref.hi, pairs->ref.nmask, pairs->ref.word_off,
                          pairs->ref.stride_words};
    a.lens = lens;
    a.E = E;
    a.E_max = E_max;
    a.p0 = p0;
    a.p1 = p1;
    a.accept = accept;
    a.count = count;
    a.n = n;
    a.err = ctx->d_err;
    return a;
}

extern "C" pf_status pf_filter_partitioned(pf_ctx *ctx, const pf_pairs *pairs,
                                           const int32_t *lens, const int16_t *E, int E_max,
                                           int t, int y, uint8_t *accept, int16_t *count,
                                           int64_t n) {
    pf_status st = variant_common(ctx, pairs, lens, E_max, accept, count, n,
                                  "pf_filter_partitioned");
    if (st != PF_OK) return st;
    if (t < 1 || t > 32 || y < 1) return ctx->fail(PF_EINVAL, "pf_filter_partitioned: t or y");
    if (n == 0) return PF_OK;
    cudaSetDevice(ctx->device);
    const VariantArgs a = variant_args_of(ctx, pairs, lens, E, E_max, t, y, accept, count, n);
    return ctx->cuda(launch_variant<PartitionedK>(a, ctx->sms, ctx->stream),
                     "pf_filter_partitioned launch");
}

extern "C" pf_status pf_filter_shouji(pf_ctx *ctx, const pf_pairs *pairs, const int32_t *lens,
                                      const int16_t *E, int E_max, uint8_t *accept,
                                      int16_t *count, int64_t n) {
    pf_status st = variant_common(ctx, pairs, lens, E_max, accept, count, n, "pf_filter_shouji");
    if (st != PF_OK || n == 0) return st;
    cudaSetDevice(ctx->device);
    const VariantArgs a = variant_args_of(ctx, pairs, lens, E, E_max, 0, 0, accept, count, n);
    return ctx->cuda(launch_variant<ShoujiK>(a, ctx->sms, ctx->stream), "pf_filter_shouji launch");
}

extern "C" pf_status pf_filter_shd(pf_ctx *ctx, const pf_pairs *pairs, const int32_t *lens,
                                   const int16_t *E, int E_max, unsigned flags, uint8_t *accept,
                                   int16_t *count, int64_t n) {
    pf_status st = variant_common(ctx, pairs, lens, E_max, accept, count, n, "pf_filter_shd");
    if (st != PF_OK) return st;
    if (flags & ~(PF_SHD_VACANT_ZERO | PF_SHD_STREAK))
        return ctx->fail(PF_EINVAL, "pf_filter_shd: unknown flags");
    if (n == 0) return PF_OK;
    cudaSetDevice(ctx->device);
    const VariantArgs a =
        variant_args_of(ctx, pairs, lens, E, E_max, (int)flags, 0, accept, count, n);
    return ctx->cuda(launch_variant<ShdK>(a, ctx->sms, ctx->stream), "pf_filter_shd launch");
}

// Fused neighbourhood map + SneakySnake + GateKeeper for one pair, run by a
// group of TPP lanes one 32-column word at a time.  Included by the kernel
// instantiation units.
//
// Map (Eq. 6.1, Ch. 6 Discussion): for reference word w (columns 32w ..
// 32w+31) and diagonal d, the mismatch word is
//     M_d = (ref_lo ^ read_lo>>d) | (ref_hi ^ read_hi>>d) | ref_n | read_n>>d
// where read_x>>d is the read plane taken from bit 32w+d on (a funnel shift
// of two read words) and bits outside the read are N (vacant = mismatch).
// Columns at or past the pair length are cleared.
//
// SneakySnake (Ch. 8, Eq. 8.2, §8.4.2): from a checkpoint c the deepest
// pipe ends where every diagonal has met an obstacle.  With y_d = M_d
// restricted to columns >= c, (y_d | -y_d) marks the columns at or after
// the first obstacle of diagonal d, and the AND over d marks the columns
// where all diagonals are blocked; its lowest bit is the obstacle the snake
// passes (count + 1, checkpoint one column further).  If the AND is empty
// the deepest pipe runs on into the next word: diagonals already blocked
// are carried as dead (y = 1 makes them neutral) and the search resumes.
// The count saturates at E + 1.
//
// GateKeeper (§5.2.1-§5.2.3): h = popcount of the d = 0 mask; the amend of
// a mask word needs two bits of each neighbouring word, so word w-1 is
// amended once word w is built; amended masks are ANDed over d and
// popcounted.  count = h if h <= E, else popcount of the AND, saturated at
// E + 1; both counts can be decided early once they exceed E.
//
// Diagonal slots: with TPP == 1 one thread owns 2*DPT slots, slot k < DPT
// is d = k and slot k >= DPT is d = -(1 + k - DPT) (compile-time offsets).
// With TPP >= 2 lanes 0..TPP/2-1 own d = g + k*TPP/2 and the other lanes
// own d = -(1 + (g - TPP/2) + k*TPP/2), so every lane shifts its read
// words from one fixed pair of words (sign fixed per lane).
#pragma once
#include <type_traits>

#include "pf_internal.cuh"

namespace pf {

// XE >= 0 selects the exact-threshold form: one thread, E = XE fixed at
// compile time, slots k = 0..XE hold d = k and slots XE+1..2XE hold
// d = -(k - XE); every slot is live and every shift is a constant.
template <int TPP, int DPT, int XE = -1>
struct SlotMap {
    static constexpr int NS = (XE >= 0) ? 2 * XE + 1 : ((TPP == 1) ? 2 * DPT : DPT);
    static constexpr int HALF = (TPP == 1) ? 1 : TPP / 2;
    static constexpr int ECAP = (XE >= 0) ? XE : DPT * HALF - 1;
};

template <int TPP, int DPT, int XE = -1>
__device__ __forceinline__ int slot_d(int k, int g) {
    if constexpr (XE >= 0) {
        return k <= XE ? k : -(k - XE);
    } else if constexpr (TPP == 1) {
        return k < DPT ? k : -(1 + k - DPT);
    } else {
        constexpr int HALF = TPP / 2;
        return g < HALF ? (g + k * HALF) : -(1 + (g - HALF) + k * HALF);
    }
}

template <int TPP, int DPT, int XE>
__device__ __forceinline__ bool slot_negative(int k, int g) {
    if constexpr (XE >= 0) return k > XE;
    else if constexpr (TPP == 1) return k >= DPT;
    else return g >= TPP / 2;
}

__device__ __forceinline__ uint32_t shr_pair(uint32_t a, uint32_t b, int d) {
    // bits [r, r+32) of the 64-bit value b:a, r = d mod 32
    return __funnelshift_r(a, b, (unsigned)d & 31u);
}

__device__ __forceinline__ int imin(int a, int b) { return a < b ? a : b; }

// -1, read from memory so that the compiler cannot fold it: the SneakySnake
// step negates as y * (-1), which runs on the multiply-add pipe and leaves
// the integer ALU pipe (the filter's binding unit) to the logic operations.
static __device__ uint32_t g_minus_one = 0xffffffffu;

// The resumable state of one pair.  init() loads the first words, word()
// processes one reference word and reports whether both deciders are
// decided, finish() closes GateKeeper's last word.  Every lane of the
// group holds the same copy of the scalar state.
// SINK: every word's mask words are also stored (at sink[(w * NS + k) * 32],
// one lane's column of a per-warp array), and the words run to the end of
// the pair whatever the deciders' state: the first phase of the two-phase
// kernel below.
template <int TPP, int DPT, int DEC, int XE = -1, typename L = LdNC, bool SINK = false>
struct PairFilter {
    using SM = SlotMap<TPP, DPT, XE>;
    static constexpr int NS = SM::NS;
    static constexpr bool SS = DEC & 1;
    static constexpr bool GK = DEC & 2;

    int64_t rb, fb;
    int m, E, W, w;
    Word3 Rm1, R0, Rp1, Fw;
    // one bit per slot
    using Mask = typename std::conditional<(NS > 32), unsigned long long, uint32_t>::type;

    // Mask words of three consecutive words.  Word w's masks go into the
    // array that held word w-3's; the other two are GateKeeper's words w-1
    // and w-2.  The word loop is unrolled three times so that the roles
    // rotate by name instead of by copying (role r: w-1 in P[r], w-2 in
    // P[r+2 mod 3], new word into P[r+1 mod 3]).
    uint32_t P0[NS], P1[NS], P2[NS];
    int role;
    Mask dead;            // SneakySnake: slots blocked before the current word
    uint32_t C;           // SneakySnake: columns >= checkpoint in this word
    int kss;
    bool ss_done, gk_done, cont;
    int h, fc;
    uint32_t neg1;        // -1 (see g_minus_one)

    __device__ __forceinline__ bool live(int k, int g) const {
        if constexpr (XE >= 0) return true;
        const int d = slot_d<TPP, DPT, XE>(k, g);
        return d <= E && -d <= E;
    }

    // Lane groups with the threshold known at run time: a slot whose
    // diagonal lies outside the band holds all-ones mask words (a diagonal
    // blocked at every column).  Neither decider can tell such a diagonal
    // from none: SneakySnake's AND of (y | -y) keeps every bit at or after
    // the checkpoint of an all-ones y, GateKeeper's amend leaves an all-ones
    // word as it is.  So only the map looks at liveness (once per pair, as
    // a bit per slot), and every other loop runs all slots unconditionally.
    static constexpr bool ONES = (TPP > 1) && (XE < 0);
    uint32_t dead_bits;   // ONES: bit k set when slot k is outside the band

    __device__ __forceinline__ bool skip(int k, int g) const {
        if constexpr (ONES) return false;
        else return !live(k, g);
    }

    // the threshold, a constant in the exact-threshold form
    __device__ __forceinline__ int thr() const {
        if constexpr (XE >= 0) return XE;
        return E;
    }

    __device__ __forceinline__ void init(const PairsView &pv, int64_t p, int m_, int E_) {
        m = m_;
        E = E_;
        W = (m + 31) >> 5;
        w = 0;
        rb = pv.read.template start<L>(p);
        fb = pv.ref.template start<L>(p);
        Rm1 = load_word<L>(pv.read, rb, -1, W);
        R0 = load_word<L>(pv.read, rb, 0, W);
        Rp1 = load_word<L>(pv.read, rb, 1, W);
        Fw = load_word<L>(pv.ref, fb, 0, W);
#pragma unroll
        for (int k = 0; k < NS; ++k) { P0[k] = 0u; P2[k] = 0u; }
        role = 0;
        dead = 0u;
        C = 0xffffffffu;
        kss = 0;
        cont = false;
        ss_done = !SS;
        gk_done = !GK;
        h = 0;
        fc = 0;
        neg1 = *(volatile const uint32_t *)&g_minus_one;
    }

    uint32_t *sink;       // SINK only

    __device__ __forceinline__ bool done() const {
        if constexpr (SINK) return w >= W;
        return (ss_done && gk_done) || w >= W;
    }

    // Process every remaining word, then leave `role` for finish().
    __device__ __forceinline__ void run(const PairsView &pv, int g, unsigned gmask) {
        if constexpr (ONES) {
            dead_bits = 0u;
#pragma unroll
            for (int k = 0; k < NS; ++k)
                if (!live(k, g)) dead_bits |= 1u << k;
        }
        if constexpr (!GK) {  // no history to rotate
            while (!done()) word(pv, g, gmask, P0, P2, P1);
        } else {
            for (;;) {
                if (done()) { role = 0; return; }
                word(pv, g, gmask, P0, P2, P1);
                if (done()) { role = 1; return; }
                word(pv, g, gmask, P1, P0, P2);
                if (done()) { role = 2; return; }
                word(pv, g, gmask, P2, P1, P0);
            }
        }
    }

    // Process reference word w with GateKeeper's words w-1 (Mp) and w-2
    // (Mpp); word w's mask words are written to M.
    __device__ __forceinline__ void word(const PairsView &pv, int g, unsigned gmask,
                                         const uint32_t (&Mp)[NS], const uint32_t (&Mpp)[NS],
                                         uint32_t (&M)[NS]) {
        const Word3 F = Fw;
        Fw = load_word<L>(pv.ref, fb, w + 1, W);  // prefetch the next reference word

        // ---- map words of this lane's diagonals
        Word3 A, B;
        if constexpr (TPP > 1) {
            const bool neg = g >= SM::HALF;
            A.lo = neg ? Rm1.lo : R0.lo;  B.lo = neg ? R0.lo : Rp1.lo;
            A.hi = neg ? Rm1.hi : R0.hi;  B.hi = neg ? R0.hi : Rp1.hi;
            A.nm = neg ? Rm1.nm : R0.nm;  B.nm = neg ? R0.nm : Rp1.nm;
        }
#pragma unroll
        for (int k = 0; k < NS; ++k) {
            if (skip(k, g)) continue;
            const int d = slot_d<TPP, DPT, XE>(k, g);
            uint32_t slo, shi, snm;
            if constexpr (TPP == 1) {
                if (slot_negative<TPP, DPT, XE>(k, g)) {  // read words w-1, w
                    slo = shr_pair(Rm1.lo, R0.lo, d);
                    shi = shr_pair(Rm1.hi, R0.hi, d);
                    snm = shr_pair(Rm1.nm, R0.nm, d);
                } else {
                    slo = shr_pair(R0.lo, Rp1.lo, d);
                    shi = shr_pair(R0.hi, Rp1.hi, d);
                    snm = shr_pair(R0.nm, Rp1.nm, d);
                }
            } else {
                slo = shr_pair(A.lo, B.lo, d);
                shi = shr_pair(A.hi, B.hi, d);
                snm = shr_pair(A.nm, B.nm, d);
            }
            M[k] = (F.lo ^ slo) | (F.hi ^ shi) | F.nm | snm;
            if constexpr (ONES)  // all ones outside the band
                M[k] |= (uint32_t)((int32_t)(dead_bits << (31 - k)) >> 31);
        }
        if (w == W - 1 && (m & 31)) {  // columns >= m of the last word are not cells
            const uint32_t valid = (1u << (m & 31)) - 1u;
#pragma unroll
            for (int k = 0; k < NS; ++k)
                if (!skip(k, g)) M[k] &= valid;
        }
        if constexpr (SINK) {
#pragma unroll
            for (int k = 0; k < NS; ++k) sink[(w * NS + k) * 32] = M[k];
        }

        // ---- SneakySnake steps inside this word
        if constexpr (SS) {
            if (!ss_done) {
                bool word_done = false;
                if (cont) {  // a pipe runs on from an earlier word
                    uint32_t T = 0xffffffffu;
#pragma unroll
                    for (int k = 0; k < NS; ++k) {
                        if (skip(k, g)) continue;
                        const uint32_t y = M[k] | (uint32_t)((dead >> k) & 1u);
                        T &= (y | (y * neg1));
                    }
                    T = group_and<TPP>(T, gmask);
                    if (T == 0u) {
                        if (w == W - 1) {
                            ss_done = true;
                        } else {
#pragma unroll
                            for (int k = 0; k < NS; ++k)
                                if (!skip(k, g) && M[k]) dead |= Mask(1) << k;
                        }
                        word_done = true;
                    } else {
                        const int pbit = __ffs(T) - 1;
                        ++kss;
                        cont = false;
                        if (kss > thr()) {
                            ss_done = true;
                            word_done = true;
                        } else if (pbit == 31) {
                            C = 0xffffffffu;
                            word_done = true;
                        } else {
                            C = 0xfffffffeu << pbit;
                        }
                    }
                }
                while (!word_done) {
                    uint32_t T = 0xffffffffu;
#pragma unroll
                    for (int k = 0; k < NS; ++k) {
                        if (skip(k, g)) continue;
                        const uint32_t y = M[k] & C;
                        T &= (y | (y * neg1));
                    }
                    T = group_and<TPP>(T, gmask);
                    if (T == 0u) {
                        if (w == W - 1) {
                            ss_done = true;
                        } else {
                            Mask dd = 0u;
#pragma unroll
                            for (int k = 0; k < NS; ++k)
                                if (!skip(k, g) && (M[k] & C)) dd |= Mask(1) << k;
                            dead = dd;
                            cont = true;
                        }
                        break;
                    }
                    const int pbit = __ffs(T) - 1;
                    ++kss;
                    if (kss > thr()) {
                        ss_done = true;
                        break;
                    }
                    if (pbit == 31) {
                        C = 0xffffffffu;
                        break;
                    }
                    C = 0xfffffffeu << pbit;
                }
            }
        }

        // ---- Hamming count alone (SneakySnake without GateKeeper): lane 0
        // owns d = 0 and writes the outputs
        if constexpr (!GK && (SS || SINK)) {
            if (g == 0) h += __popc(M[0]);
        }

        // ---- GateKeeper: Hamming word, amend + AND of the previous word
        if constexpr (GK) {
            if (!gk_done) {
                int hw = 0;
                if (g == 0) hw = __popc(M[0]);
                if constexpr (TPP > 1) hw = __shfl_sync(gmask, hw, 0, TPP);
                h += hw;
                if (w > 0) {
                    uint32_t Fa = 0xffffffffu;
#pragma unroll
                    for (int k = 0; k < NS; ++k) {
                        if (skip(k, g)) continue;
                        const uint32_t H = Mp[k];
                        const uint32_t l1 = __funnelshift_l(Mpp[k], H, 1);
                        const uint32_t l2 = __funnelshift_l(Mpp[k], H, 2);
                        const uint32_t r1 = __funnelshift_r(H, M[k], 1);
                        const uint32_t r2 = __funnelshift_r(H, M[k], 2);
                        Fa &= H | (l1 & (r1 | r2)) | (l2 & r1);
                    }
                    Fa = group_and<TPP>(Fa, gmask);
                    fc += __popc(Fa);  // word w-1 is full: every bit is a column < m
                    if (h > thr() && fc > thr()) gk_done = true;
                }
            }
        }

        Rm1 = R0;
        R0 = Rp1;
        Rp1 = load_word<L>(pv.read, rb, w + 2, W);
        ++w;
    }

    // Counts once done(): SneakySnake's obstacles and GateKeeper's edits.
    __device__ __forceinline__ void finish(int g, unsigned gmask, int *ss_count, int *gk_count) {
        if (role == 0) finish_words(g, gmask, P0, P2, ss_count, gk_count);
        else if (role == 1) finish_words(g, gmask, P1, P0, ss_count, gk_count);
        else finish_words(g, gmask, P2, P1, ss_count, gk_count);
    }

    __device__ __forceinline__ void finish_words(int g, unsigned gmask, const uint32_t (&Mp)[NS],
                                                 const uint32_t (&Mpp)[NS], int *ss_count,
                                                 int *gk_count) {
        const int E = thr();
        if constexpr (SS) *ss_count = imin(kss, E + 1);
        if constexpr (GK) {
            if (gk_done) {  // decided early: both counts exceeded E
                *gk_count = E + 1;
                return;
            }
            if (W > 0) {  // amend the last word, right neighbours past the end are 0
                uint32_t Fa = 0xffffffffu;
#pragma unroll
                for (int k = 0; k < NS; ++k) {
                    if (skip(k, g)) continue;
                    const uint32_t H = Mp[k];
                    const uint32_t l1 = __funnelshift_l(Mpp[k], H, 1);
                    const uint32_t l2 = __funnelshift_l(Mpp[k], H, 2);
                    const uint32_t r1 = H >> 1;
                    const uint32_t r2 = H >> 2;
                    Fa &= H | (l1 & (r1 | r2)) | (l2 & r1);
                }
                Fa = group_and<TPP>(Fa, gmask);
                const uint32_t valid = (m & 31) ? ((1u << (m & 31)) - 1u) : 0xffffffffu;
                fc += __popc(Fa & valid);
            }
            *gk_count = (h <= E) ? h : imin(fc, E + 1);
        }
    }
};

// h: the Hamming count (the d = 0 diagonal's mismatches), exact whenever
// it is <= E and SneakySnake accepts (every word is then processed).
// SneakySnake's obstacle count never exceeds the edit distance within the
// band (each edit of a banded alignment costs the snake at most one
// obstacle, and the greedy walk needs the fewest, Ch. 8), and the Hamming
// distance never falls below it (substitutions alone align the pair on
// d = 0).  When the two agree the distance is known: with a.need set such a
// pair is written here and left out of verification.
template <int DEC>
__device__ __forceinline__ void write_outputs(const FilterArgs &a, int64_t p, int E, int ssc,
                                              int gkc, int h) {
    if (a.dist && (DEC == 2 ? gkc : ssc) > E) a.dist[p] = E + 1;  // not verified
    if constexpr (DEC & 1) {
        if (a.need) {
            const bool known = ssc <= E && h == ssc;
            a.need[p] = (uint8_t)(ssc <= E && !known);
            if (known) a.dist[p] = h;
        }
    }
    if constexpr (DEC == 3) {
        a.count[p] = (int16_t)ssc;
        a.accept[p] = (uint8_t)(ssc <= E);
        a.count[a.n + p] = (int16_t)gkc;
        a.accept[a.n + p] = (uint8_t)(gkc <= E);
    } else if constexpr (DEC == 1) {
        a.count[p] = (int16_t)ssc;
        a.accept[p] = (uint8_t)(ssc <= E);
    } else {
        a.count[p] = (int16_t)gkc;
        a.accept[p] = (uint8_t)(gkc <= E);
    }
}

template <int DEC>
__device__ __forceinline__ void write_invalid(const FilterArgs &a, int64_t p) {
    a.count[p] = -1;
    a.accept[p] = 0;
    if (a.dist) a.dist[p] = -1;
    if constexpr (DEC == 3) {
        a.count[a.n + p] = -1;
        a.accept[a.n + p] = 0;
    }
    if constexpr (DEC & 1) {
        if (a.need) a.need[p] = 0;
    }
    atomicOr(a.err, ERR_PAIR_ARGS);
}

// Reads pair p's length and threshold; false (and outputs marked) if bad.
template <int TPP, int DPT, int DEC, int XE>
__device__ __forceinline__ bool pair_args(const FilterArgs &a, int64_t p, int g, int *m, int *E) {
    *m = __ldg(a.lens + p);
    *E = a.E ? (int)__ldg(a.E + p) : a.E_max;
    if (*m < 0 || *E < 0 || *E > a.E_max || *E > SlotMap<TPP, DPT, XE>::ECAP ||
        (XE >= 0 && *E != XE)) {
        if (g == 0) write_invalid<DEC>(a, p);
        return false;
    }
    return true;
}

// Filter pair p with the group and write its outputs.
template <int TPP, int DPT, int DEC, int XE = -1>
__device__ __forceinline__ void filter_group(const FilterArgs &a, int64_t p, int g,
                                             unsigned gmask) {
    int m, E;
    if (!pair_args<TPP, DPT, DEC, XE>(a, p, g, &m, &E)) return;
    PairFilter<TPP, DPT, DEC, XE> st;
    st.init(a.pairs, p, m, E);
    st.run(a.pairs, g, gmask);
    int ssc = 0, gkc = 0;
    st.finish(g, gmask, &ssc, &gkc);
    if (g == 0) write_outputs<DEC>(a, p, E, ssc, gkc, st.h);
}

// The plain kernel: one thread per pair, every thread runs its own pair to
// the end.
template <int DPT, int DEC>
__global__ void __launch_bounds__(256) filter_plain_kernel(FilterArgs a) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= a.n) return;
    filter_group<1, DPT, DEC>(a, p, 0, 1u << (threadIdx.x & 31));
}

// Pairs per work item of a persistent launch over a bin of `bin_pairs`
// pairs: the tuned chunk, unless the bin is too short to give every warp of
// the grid one item of that size.  Then the items shrink (to a multiple of
// the pairs a warp takes at once, `step`) so that the bin spreads over the
// whole grid: a pair's latency is long (up to thousands of dependent
// instructions), and a short bin left to a few warps, each running a chain
// of pairs, would finish long after the rest of the GPU went idle.  Every
// warp computes the same value.
__device__ __forceinline__ int64_t item_pairs(int64_t bin_pairs, int tuned, int step) {
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    int64_t c = (bin_pairs + warps - 1) / warps;
    c = (c + step - 1) / step * step;
    if (c < step) c = step;
    return c < tuned ? c : (int64_t)tuned;
}

// The plain kernel with the threshold fixed at compile time (E = XE for
// every pair): one thread per pair, one launch, no scheduler; it isolates
// what specialising the threshold gains over filter_plain_kernel.
template <int XE, int DEC>
__global__ void __launch_bounds__(256) filter_plain_exact_kernel(FilterArgs a) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= a.n) return;
    filter_group<1, XE + 1, DEC, XE>(a, p, 0, 1u << (threadIdx.x & 31));
}

// The batched kernel: persistent warps take chunks of `chunk` positions of
// one bin through an atomic counter (fewer for a short bin, item_pairs); the lane groups of a warp stride
// through the chunk, one pair per group at a time, so neighbouring groups
// read neighbouring pairs' words.
template <int TPP, int DPT, int DEC, int XE>
__global__ void __launch_bounds__(256) filter_batched_kernel(BatchArgs b, int bin) {
    const int lane = threadIdx.x & 31;
    const int g = lane & (TPP - 1);
    const unsigned gmask =
        (TPP == 32) ? 0xffffffffu : (((1u << TPP) - 1u) << (lane & ~(TPP - 1)));
    constexpr int GPW = 32 / TPP;  // groups per warp
    const int gid = lane / TPP;
    const int64_t lo = b.bin_start[bin], hi = b.bin_start[bin + 1];
    const int64_t chunk = item_pairs(hi - lo, b.chunk, GPW);
    unsigned long long *counter = b.work + bin;
    const int64_t *order = (b.order && !(b.ident && *b.ident)) ? b.order : nullptr;
    for (;;) {
        unsigned long long item = 0;
        if (lane == 0) item = atomicAdd(counter, 1ull);
        item = __shfl_sync(0xffffffffu, item, 0);
        const int64_t s = lo + (int64_t)item * chunk;
        if (s >= hi) break;
        const int64_t e = min(hi, s + chunk);
        for (int64_t q = s + gid; q < e; q += GPW) {
            const int64_t p = order ? __ldg(order + q) : q;
            filter_group<TPP, DPT, DEC, XE>(b.f, p, g, gmask);
        }
    }
}

// ---- Two-phase form (exact threshold, one thread per pair) -----------------
//
// In the fused loop a warp runs, in every word, as many SneakySnake steps as
// its busiest lane needs.  Here the first phase builds the mask words of the
// whole pair (and runs GateKeeper) word by word, storing them in shared
// memory; the second runs the snake as a per-lane loop of steps over the
// stored words, so a warp runs as many steps as its busiest lane needs in
// total.  The walk is the fused loop's, word for word: the same checkpoint
// mask, the same carry of blocked diagonals into the next word.
template <int XE>
__device__ __forceinline__ int split_sneakysnake(const uint32_t *mine, int W, uint32_t neg1) {
    constexpr int NS = 2 * XE + 1;
    if (W == 0) return 0;
    uint32_t Mw[NS];
#pragma unroll
    for (int k = 0; k < NS; ++k) Mw[k] = mine[k * 32];
    int ws = 0, kss = 0;
    uint32_t C = 0xffffffffu;
    // One step shape for every lane: a pipe that runs on from the previous
    // word is the word's first step with every column open, and the
    // diagonals already blocked carry bit 0 set (blocked at once), which no
    // later step of the word looks at (they start past the first obstacle).
    // Both ways into the next word share one block, so that a warp whose
    // lanes cross words at different steps runs it once per step.
    for (;;) {
        uint32_t y[NS];
        uint32_t T = 0xffffffffu;
#pragma unroll
        for (int k = 0; k < NS; ++k) {
            y[k] = Mw[k] & C;
            T &= y[k] | (y[k] * neg1);
        }
        const int pbit = __ffs(T) - 1;  // the obstacle passed; -1 if T == 0
        if (T != 0u) {
            if (++kss > XE) break;
            if (pbit != 31) {
                C = 0xfffffffeu << pbit;
                continue;
            }
        }
        // Next word: after T == 0 the deepest pipe reaches the end of the
        // word and the diagonals blocked in the rest of it stay blocked (bit
        // 0 set, cm = 1); after an obstacle in the word's last column every
        // diagonal starts free (cm = 0).
        if (ws == W - 1) break;
        ++ws;
        const uint32_t cm = (T == 0u) ? 1u : 0u;
#pragma unroll
        for (int k = 0; k < NS; ++k) Mw[k] = mine[(ws * NS + k) * 32] | min(y[k], cm);
        C = 0xffffffffu;
    }
    return kss > XE + 1 ? XE + 1 : kss;
}

template <int DEC, int XE, int WMAX>
__device__ __forceinline__ void filter_split_pair(const FilterArgs &a, int64_t p, uint32_t *mine,
                                                  unsigned lane_mask) {
    int m, E;
    if (!pair_args<1, XE + 1, DEC, XE>(a, p, 0, &m, &E)) return;
    const int W = (m + 31) >> 5;
    if (W > WMAX) {  // longer than the shared arrays: the fused loop
        filter_group<1, XE + 1, DEC, XE>(a, p, 0, lane_mask);
        return;
    }
    PairFilter<1, XE + 1, DEC & 2, XE, LdNC, true> st;
    st.sink = mine;
    st.init(a.pairs, p, m, E);
    st.run(a.pairs, 0, lane_mask);
    int ssc = 0, gkc = 0;
    st.finish(0, lane_mask, &ssc, &gkc);
    if constexpr (DEC & 1) ssc = split_sneakysnake<XE>(mine, W, st.neg1);
    write_outputs<DEC>(a, p, E, ssc, gkc, st.h);
}

// Shared memory: kSplitWarps warps x WMAX words x (2 XE + 1) slots x 32 lanes.
// Up to E = 7 the registers are held to five blocks per SM (with 5-word
// arrays the shared memory allows them too).
template <int DEC, int XE, int WMAX>
__global__ void __launch_bounds__(kSplitWarps * 32, (XE <= 7 ? 5 : (XE <= 10 ? 4 : 3)))
    filter_split_kernel(BatchArgs b, int bin) {
    extern __shared__ uint32_t split_maps[];
    constexpr int NS = 2 * XE + 1;
    const int lane = threadIdx.x & 31;
    uint32_t *mine = split_maps + (threadIdx.x >> 5) * (WMAX * NS * 32) + lane;
    const int64_t lo = b.bin_start[bin], hi = b.bin_start[bin + 1];
    const int64_t chunk = item_pairs(hi - lo, b.chunk, 32);
    unsigned long long *counter = b.work + bin;
    const int64_t *order = (b.order && !(b.ident && *b.ident)) ? b.order : nullptr;
    for (;;) {
        unsigned long long item = 0;
        if (lane == 0) item = atomicAdd(counter, 1ull);
        item = __shfl_sync(0xffffffffu, item, 0);
        const int64_t s = lo + (int64_t)item * chunk;
        if (s >= hi) break;
        const int64_t e = min(hi, s + chunk);
        for (int64_t q = s + lane; q < e; q += 32) {
            const int64_t p = order ? __ldg(order + q) : q;
            filter_split_pair<DEC, XE, WMAX>(b.f, p, mine, 1u << lane);
        }
    }
}

// ---- Two-phase form with a lane group per pair (large thresholds) ----------
//
// For large E one thread cannot hold the 2E+1 masks of GateKeeper's three
// words in registers.  Here TPP lanes share a pair (each owns DPT diagonal
// slots, as in the fused group loop): the first phase builds the mask words
// of the whole pair and runs GateKeeper, every lane storing its own slots'
// words in its own shared-memory column; the second runs SneakySnake as a
// per-group loop of steps over the stored words, one group AND per step.
// The walk is split_sneakysnake's, with the group's lanes each folding their
// own diagonals into T.
template <int TPP, int DPT>
__device__ __forceinline__ int split_sneakysnake_group(const uint32_t *mine, int W, int E,
                                                       unsigned gmask, uint32_t neg1) {
    if (W == 0) return 0;
    // slots outside the band were stored as all ones (PairFilter::ONES):
    // neutral in the AND below, so every slot takes part
    uint32_t Mw[DPT];
#pragma unroll
    for (int k = 0; k < DPT; ++k) Mw[k] = mine[k * 32];
    int ws = 0, kss = 0;
    uint32_t C = 0xffffffffu;
    for (;;) {
        uint32_t y[DPT];
        uint32_t T = 0xffffffffu;
#pragma unroll
        for (int k = 0; k < DPT; ++k) {
            y[k] = Mw[k] & C;
            T &= y[k] | (y[k] * neg1);
        }
        T = group_and<TPP>(T, gmask);
        const int pbit = __ffs(T) - 1;  // the obstacle passed; -1 if T == 0
        if (T != 0u) {
            if (++kss > E) break;
            if (pbit != 31) {
                C = 0xfffffffeu << pbit;
                continue;
            }
        }
        if (ws == W - 1) break;
        ++ws;
        const uint32_t cm = (T == 0u) ? 1u : 0u;
#pragma unroll
        for (int k = 0; k < DPT; ++k) Mw[k] = mine[(ws * DPT + k) * 32] | min(y[k], cm);
        C = 0xffffffffu;
    }
    return kss > E + 1 ? E + 1 : kss;
}

template <int DEC, int TPP, int DPT, int WMAX>
__device__ __forceinline__ void filter_split_group_pair(const FilterArgs &a, int64_t p, int g,
                                                        unsigned gmask, uint32_t *mine) {
    int m, E;
    if (!pair_args<TPP, DPT, DEC, -1>(a, p, g, &m, &E)) return;
    const int W = (m + 31) >> 5;
    if (W > WMAX) {  // longer than the shared arrays: the fused loop
        filter_group<TPP, DPT, DEC, -1>(a, p, g, gmask);
        return;
    }
    PairFilter<TPP, DPT, DEC & 2, -1, LdNC, true> st;
    st.sink = mine;
    st.init(a.pairs, p, m, E);
    st.run(a.pairs, g, gmask);
    int ssc = 0, gkc = 0;
    st.finish(g, gmask, &ssc, &gkc);
    if constexpr (DEC & 1) ssc = split_sneakysnake_group<TPP, DPT>(mine, W, E, gmask, st.neg1);
    if (g == 0) write_outputs<DEC>(a, p, E, ssc, gkc, st.h);
}

// Shared memory: kSplitWarps warps x WMAX words x DPT slots x 32 lanes.
template <int DEC, int TPP, int DPT, int WMAX>
__global__ void __launch_bounds__(kSplitWarps * 32)
    filter_split_group_kernel(BatchArgs b, int bin) {
    extern __shared__ uint32_t split_maps[];
    const int lane = threadIdx.x & 31;
    const int g = lane & (TPP - 1);
    const unsigned gmask =
        (TPP == 32) ? 0xffffffffu : (((1u << TPP) - 1u) << (lane & ~(TPP - 1)));
    constexpr int GPW = 32 / TPP;  // groups per warp
    const int gid = lane / TPP;
    uint32_t *mine = split_maps + (threadIdx.x >> 5) * (WMAX * DPT * 32) + lane;
    const int64_t lo = b.bin_start[bin], hi = b.bin_start[bin + 1];
    const int64_t chunk = item_pairs(hi - lo, b.chunk, GPW);
    unsigned long long *counter = b.work + bin;
    const int64_t *order = (b.order && !(b.ident && *b.ident)) ? b.order : nullptr;
    for (;;) {
        unsigned long long item = 0;
        if (lane == 0) item = atomicAdd(counter, 1ull);
        item = __shfl_sync(0xffffffffu, item, 0);
        const int64_t s = lo + (int64_t)item * chunk;
        if (s >= hi) break;
        const int64_t e = min(hi, s + chunk);
        for (int64_t q = s + gid; q < e; q += GPW) {
            const int64_t p = order ? __ldg(order + q) : q;
            filter_split_group_pair<DEC, TPP, DPT, WMAX>(b.f, p, g, gmask, mine);
        }
    }
}

}  // namespace pf

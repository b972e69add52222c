// Fused neighbourhood map + SneakySnake + GateKeeper for one pair, run by a
// group of TPP lanes.  Included by the kernel instantiation units.
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
#include "pf_internal.cuh"

namespace pf {

template <int TPP, int DPT>
struct SlotMap {
    static constexpr int NS = (TPP == 1) ? 2 * DPT : DPT;
    static constexpr int HALF = (TPP == 1) ? 1 : TPP / 2;
    static constexpr int ECAP = DPT * HALF - 1;
};

template <int TPP, int DPT>
__device__ __forceinline__ int slot_d(int k, int g) {
    if constexpr (TPP == 1) {
        return k < DPT ? k : -(1 + k - DPT);
    } else {
        constexpr int HALF = TPP / 2;
        return g < HALF ? (g + k * HALF) : -(1 + (g - HALF) + k * HALF);
    }
}

__device__ __forceinline__ uint32_t shr_pair(uint32_t a, uint32_t b, int d) {
    // bits [r, r+32) of the 64-bit value b:a, r = d mod 32
    return __funnelshift_r(a, b, (unsigned)d & 31u);
}

struct Outputs {
    int ss_count, gk_count;
};

// DEC: bit 0 SneakySnake, bit 1 GateKeeper.
template <int TPP, int DPT, int DEC>
__device__ __forceinline__ Outputs filter_pair(const PairsView &pv, int64_t p, int m, int E,
                                               int g, unsigned gmask) {
    using SM = SlotMap<TPP, DPT>;
    constexpr int NS = SM::NS;
    constexpr bool SS = DEC & 1;
    constexpr bool GK = DEC & 2;

    const int W = (m + 31) >> 5;
    const int64_t rb = pv.read.start(p);
    const int64_t fb = pv.ref.start(p);

    int dd[NS];
    bool live[NS];
#pragma unroll
    for (int k = 0; k < NS; ++k) {
        dd[k] = slot_d<TPP, DPT>(k, g);
        live[k] = (dd[k] <= E) && (-dd[k] <= E);
    }
    // lanes of a multi-lane group own diagonals of one sign
    const bool lane_neg = (TPP > 1) && (g >= SM::HALF);

    uint32_t M[NS], D[NS], Mp[NS], Mpp[NS];
#pragma unroll
    for (int k = 0; k < NS; ++k) { D[k] = 0u; Mp[k] = 0u; Mpp[k] = 0u; }

    // SneakySnake state (replicated on the group's lanes)
    bool ss_done = !SS;
    int kss = 0, ss_count = 0;
    bool cont = false;
    uint32_t C = 0xffffffffu;
    // GateKeeper state
    bool gk_done = !GK;
    int h = 0, fc = 0, gk_count = 0;

    Word3 Rm1 = load_word(pv.read, rb, -1, W);
    Word3 R0 = load_word(pv.read, rb, 0, W);
    Word3 Rp1 = load_word(pv.read, rb, 1, W);

    for (int w = 0; w < W; ++w) {
        if (ss_done && gk_done) break;
        const Word3 F = load_word(pv.ref, fb, w, W);
        const uint32_t valid =
            (w == W - 1 && (m & 31)) ? ((1u << (m & 31)) - 1u) : 0xffffffffu;

        // ---- map words of this lane's diagonals
        Word3 A, B;
        if constexpr (TPP > 1) {
            A.lo = lane_neg ? Rm1.lo : R0.lo;  B.lo = lane_neg ? R0.lo : Rp1.lo;
            A.hi = lane_neg ? Rm1.hi : R0.hi;  B.hi = lane_neg ? R0.hi : Rp1.hi;
            A.nm = lane_neg ? Rm1.nm : R0.nm;  B.nm = lane_neg ? R0.nm : Rp1.nm;
        }
#pragma unroll
        for (int k = 0; k < NS; ++k) {
            if (!live[k]) continue;
            const int d = dd[k];
            uint32_t slo, shi, snm;
            if constexpr (TPP == 1) {
                if (k >= DPT) {  // negative diagonal: read words w-1, w
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
            M[k] = ((F.lo ^ slo) | (F.hi ^ shi) | F.nm | snm) & valid;
        }

        // ---- SneakySnake steps inside this word
        if constexpr (SS) {
            if (!ss_done) {
                bool word_done = false;
                if (cont) {
                    uint32_t T = 0xffffffffu;
#pragma unroll
                    for (int k = 0; k < NS; ++k) {
                        if (!live[k]) continue;
                        const uint32_t y = M[k] | D[k];
                        T &= (y | (0u - y));
                    }
                    T = group_and<TPP>(T, gmask);
                    if (T == 0u) {
                        if (w == W - 1) {
                            ss_done = true;
                            ss_count = kss;
                        } else {
#pragma unroll
                            for (int k = 0; k < NS; ++k)
                                if (live[k]) D[k] = min(D[k] | M[k], 1u);
                        }
                        word_done = true;
                    } else {
                        const int pbit = __ffs(T) - 1;
                        ++kss;
                        cont = false;
                        if (kss > E) {
                            ss_done = true;
                            ss_count = E + 1;
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
                        if (!live[k]) continue;
                        const uint32_t y = M[k] & C;
                        T &= (y | (0u - y));
                    }
                    T = group_and<TPP>(T, gmask);
                    if (T == 0u) {
                        if (w == W - 1) {
                            ss_done = true;
                            ss_count = kss;
                        } else {
#pragma unroll
                            for (int k = 0; k < NS; ++k)
                                if (live[k]) D[k] = min(M[k] & C, 1u);
                            cont = true;
                        }
                        break;
                    }
                    const int pbit = __ffs(T) - 1;
                    ++kss;
                    if (kss > E) {
                        ss_done = true;
                        ss_count = E + 1;
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

        // ---- GateKeeper: Hamming word, amend + AND of the previous word
        if constexpr (GK) {
            if (!gk_done) {
                int hw = 0;
                if (g == 0) hw = __popc(M[0]);
                if constexpr (TPP > 1) hw = __shfl_sync(gmask, hw, 0, TPP);
                h += hw;
                if (w > 0) {
                    uint32_t Fw = 0xffffffffu;
#pragma unroll
                    for (int k = 0; k < NS; ++k) {
                        if (!live[k]) continue;
                        const uint32_t H = Mp[k];
                        const uint32_t l1 = __funnelshift_l(Mpp[k], H, 1);
                        const uint32_t l2 = __funnelshift_l(Mpp[k], H, 2);
                        const uint32_t r1 = __funnelshift_r(H, M[k], 1);
                        const uint32_t r2 = __funnelshift_r(H, M[k], 2);
                        Fw &= H | (l1 & (r1 | r2)) | (l2 & r1);
                    }
                    Fw = group_and<TPP>(Fw, gmask);
                    fc += __popc(Fw);  // word w-1 is full: every bit is a column < m
                    if (h > E && fc > E) {
                        gk_done = true;
                        gk_count = E + 1;
                    }
                }
#pragma unroll
                for (int k = 0; k < NS; ++k) { Mpp[k] = Mp[k]; Mp[k] = M[k]; }
            }
        }

        Rm1 = R0;
        R0 = Rp1;
        Rp1 = load_word(pv.read, rb, w + 2, W);
    }

    if constexpr (SS) {
        if (!ss_done) ss_count = kss;  // the snake left the grid
    }
    if constexpr (GK) {
        if (!gk_done) {
            if (W > 0) {  // amend the last word, right neighbours past the end are 0
                uint32_t Fw = 0xffffffffu;
#pragma unroll
                for (int k = 0; k < NS; ++k) {
                    if (!live[k]) continue;
                    const uint32_t H = Mp[k];
                    const uint32_t l1 = __funnelshift_l(Mpp[k], H, 1);
                    const uint32_t l2 = __funnelshift_l(Mpp[k], H, 2);
                    const uint32_t r1 = H >> 1;
                    const uint32_t r2 = H >> 2;
                    Fw &= H | (l1 & (r1 | r2)) | (l2 & r1);
                }
                Fw = group_and<TPP>(Fw, gmask);
                const uint32_t valid = (m & 31) ? ((1u << (m & 31)) - 1u) : 0xffffffffu;
                fc += __popc(Fw & valid);
            }
            gk_count = (h <= E) ? h : min(fc, E + 1);
        }
    }
    return Outputs{ss_count, gk_count};
}

template <int DEC>
__device__ __forceinline__ void write_outputs(const FilterArgs &a, int64_t p, int E, Outputs o) {
    if constexpr (DEC == 3) {
        a.count[p] = (int16_t)o.ss_count;
        a.accept[p] = (uint8_t)(o.ss_count <= E);
        a.count[a.n + p] = (int16_t)o.gk_count;
        a.accept[a.n + p] = (uint8_t)(o.gk_count <= E);
    } else if constexpr (DEC == 1) {
        a.count[p] = (int16_t)o.ss_count;
        a.accept[p] = (uint8_t)(o.ss_count <= E);
    } else {
        a.count[p] = (int16_t)o.gk_count;
        a.accept[p] = (uint8_t)(o.gk_count <= E);
    }
}

template <int DEC>
__device__ __forceinline__ void write_invalid(const FilterArgs &a, int64_t p) {
    a.count[p] = -1;
    a.accept[p] = 0;
    if constexpr (DEC == 3) {
        a.count[a.n + p] = -1;
        a.accept[a.n + p] = 0;
    }
    atomicOr(a.err, ERR_PAIR_ARGS);
}

// Process pair p with the group; returns after the group wrote its outputs.
template <int TPP, int DPT, int DEC>
__device__ __forceinline__ void filter_group(const FilterArgs &a, int64_t p, int g,
                                             unsigned gmask) {
    const int m = __ldg(a.lens + p);
    const int E = a.E ? (int)__ldg(a.E + p) : a.E_max;
    if (m < 0 || E < 0 || E > a.E_max || E > SlotMap<TPP, DPT>::ECAP) {
        if (g == 0) write_invalid<DEC>(a, p);
        return;
    }
    const Outputs o = filter_pair<TPP, DPT, DEC>(a.pairs, p, m, E, g, gmask);
    if (g == 0) write_outputs<DEC>(a, p, E, o);
}

// The plain kernel: one thread per pair.
template <int DPT, int DEC>
__global__ void __launch_bounds__(256) filter_plain_kernel(FilterArgs a) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= a.n) return;
    filter_group<1, DPT, DEC>(a, p, 0, 1u << (threadIdx.x & 31));
}

// The batched kernel: persistent warps take chunks of `chunk` positions of
// one bin through an atomic counter; each group of TPP lanes filters one
// pair at a time.
template <int TPP, int DPT, int DEC>
__global__ void __launch_bounds__(256) filter_batched_kernel(BatchArgs b, int bin) {
    const int lane = threadIdx.x & 31;
    const int g = lane & (TPP - 1);
    const unsigned gmask =
        (TPP == 32) ? 0xffffffffu : (((1u << TPP) - 1u) << (lane & ~(TPP - 1)));
    constexpr int GPW = 32 / TPP;  // groups per warp
    const int gid = lane / TPP;
    const int64_t lo = b.bin_start[bin], hi = b.bin_start[bin + 1];
    unsigned long long *counter = b.work + bin;
    for (;;) {
        unsigned long long item = 0;
        if (lane == 0) item = atomicAdd(counter, 1ull);
        item = __shfl_sync(0xffffffffu, item, 0);
        const int64_t s = lo + (int64_t)item * b.chunk;
        if (s >= hi) break;
        const int64_t e = min(hi, s + (int64_t)b.chunk);
        for (int64_t q = s + gid; q < e; q += GPW) {
            const int64_t p = b.order ? __ldg(b.order + q) : q;
            filter_group<TPP, DPT, DEC>(b.f, p, g, gmask);
        }
    }
}

}  // namespace pf

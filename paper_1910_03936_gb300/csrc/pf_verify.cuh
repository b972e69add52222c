// a6: verification device function, dist = min(Levenshtein(read, ref), E + 1), exact.
//
// The thesis verifies the mappings that pass the filter with banded
// Levenshtein distance (Ch. 2, "Accelerating Read Alignment": Ukkonen's
// band of 2E+1 diagonals).  This kernel computes that band with bit
// vectors: one machine word holds the vertical differences of the 2E+1
// band cells of a DP column (Myers 1999; Hyyrö 2003), one thread per pair.
//
// Rows are read prefixes (row i = read[0..i)), columns reference prefixes.
// Column j keeps the cells of rows j-E .. j+E as
//     T  = D(j-E, j)                   (value of the top band cell)
//     VP, VN bits q-1 = +1 / -1 difference D(j-E+q) - D(j-E+q-1), q=1..2E.
// Rows above row 0 are virtual with D(i, j) = j - i, which extends the
// global boundary D(0, j) = j, D(i, 0) = i upwards; they never match.
// Step j-1 -> j runs one Myers column over rows j-E .. j+E:
//   - the vertical differences of rows j-E .. j+E-1 are those stored for
//     column j-1; row j+E (outside column j-1's band) is taken as +1,
//   - the horizontal difference entering above row j-E is taken as +1.
// Both stand-ins are upper bounds of the true values, and every DP value
// computed from upper bounds is itself an upper bound; a cell whose true
// value is <= E has an optimal path inside the band, so min(result, E+1)
// is exact.  After the column, the top row's difference updates T and the
// vectors shift down by one row.
// dist = D(m, m) = T + (sum of the first E differences) at column m.
#pragma once
#include "pf_internal.cuh"

namespace pf {

template <typename U>
struct Bits;
template <>
struct Bits<uint32_t> {
    static __device__ __forceinline__ int popc(uint32_t x) { return __popc(x); }
};
template <>
struct Bits<uint64_t> {
    static __device__ __forceinline__ int popc(uint64_t x) { return __popcll(x); }
};

// 0 or ~0: bit t of x, spread over the word.
__device__ __forceinline__ uint32_t bcast(uint32_t x, int t) {
    return (uint32_t)((int32_t)(x << (31 - t)) >> 31);
}

template <typename U>
__device__ __forceinline__ U spread(uint32_t b) {
    if constexpr (sizeof(U) == 4) return b;
    else return ((uint64_t)b << 32) | b;
}

// The read's three planes from bit 32*fw - E on: x0 covers the first 32
// bits, x1 the next 32, x2 the 32 after (used by 64-bit bands only).
struct ReadWin {
    uint32_t lo0, lo1, lo2, hi0, hi1, hi2, nm0, nm1, nm2;
};

// Bits [t, t + |U|) of the window.
template <typename U>
__device__ __forceinline__ U win(uint32_t x0, uint32_t x1, uint32_t x2, int t) {
    if constexpr (sizeof(U) == 4) {
        return __funnelshift_r(x0, x1, (unsigned)t);
    } else {
        return ((uint64_t)__funnelshift_r(x1, x2, (unsigned)t) << 32) |
               __funnelshift_r(x0, x1, (unsigned)t);
    }
}

// One DP column: reference base at bit t of the reference word f, band rows
// read from the window at offset t.  VP keeps the bottom stand-in bit set.
//
// The column's horizontal differences would enter the next row up (shift
// left, +1 entering above the top row) and the new vertical differences
// would then move down one row with the band (shift right); the two shifts
// cancel except on D0, so the new vectors come from D0 >> 1 directly.  The
// top row's new vertical difference is then never +1 and is -1 exactly when
// bit 0 of D0 is set: T grows by 1 per column, less the number of those
// bits, which go to the top of accM.
template <typename U>
__device__ __forceinline__ void column(const ReadWin &r, const Word3 &f, int t, U store_mask,
                                       U bottom, U &VP, U &VN, uint32_t &accM) {
    const U mlo = spread<U>(bcast(f.lo, t));
    const U mhi = spread<U>(bcast(f.hi, t));
    const U fn = spread<U>(bcast(f.nm, t));
    const U wlo = win<U>(r.lo0, r.lo1, r.lo2, t);
    const U whi = win<U>(r.hi0, r.hi1, r.hi2, t);
    const U wnm = win<U>(r.nm0, r.nm1, r.nm2, t);
    // Eq bit q: read base of row j-E+q equals the reference base, neither N.
    // Bits above the band (q > 2E) only ever influence higher bits (carries
    // and the left shifts run upwards), and the stored vectors drop them.
    const U Eq = ~((wlo ^ mlo) | (whi ^ mhi) | wnm | fn);
    const U X = Eq | VN;
    const U D0 = (((X & VP) + VP) ^ VP) | X;
    const U Ph = VN | ~(D0 | VP);
    const U Mh = VP & D0;
    const U D1 = D0 >> 1;
    accM = __funnelshift_r(accM, (uint32_t)D0, 1);
    VP = ((Mh | ~(D1 | Ph)) & store_mask) | bottom;
    VN = Ph & D1 & store_mask;
}

template <typename U, typename L = LdNC>
__device__ __forceinline__ int verify_pair(const PairsView &pv, int64_t p, int m, int E) {
    if (m == 0) return 0;
    const int W = (m + 31) >> 5;
    const int64_t rb = pv.read.template start<L>(p), fb = pv.ref.template start<L>(p);
    const U store_mask = (U(1) << (2 * E)) - 1;     // 2E stored differences
    const U bottom = U(1) << (2 * E);               // +1 stand-in of row j+E

    // column 0: rows -E..E hold |i|; differences -1 for rows -E+1..0,
    // +1 for rows 1..E
    U VN = (U(1) << E) - 1;
    U VP = (store_mask & ~VN) | bottom;
    int T = E;

    // Reference word fw holds columns j = 32 fw + 1 + t (t = 0..31), whose
    // band starts at read bit s = j - E - 1 = 32 fw - E + t.  Read words
    // fw-1 .. fw+2 cover every window of the word.
    const unsigned rs = 32u - (unsigned)E;
    Word3 ra = load_word<L>(pv.read, rb, -1, W);
    Word3 rb0 = load_word<L>(pv.read, rb, 0, W);
    Word3 rc = load_word<L>(pv.read, rb, 1, W);
    Word3 rd;
    if constexpr (sizeof(U) == 8) rd = load_word<L>(pv.read, rb, 2, W);
    for (int fw = 0; fw < W; ++fw) {
        const Word3 f = load_word<L>(pv.ref, fb, fw, W);
        ReadWin r;
        r.lo0 = __funnelshift_rc(ra.lo, rb0.lo, rs);
        r.hi0 = __funnelshift_rc(ra.hi, rb0.hi, rs);
        r.nm0 = __funnelshift_rc(ra.nm, rb0.nm, rs);
        r.lo1 = __funnelshift_rc(rb0.lo, rc.lo, rs);
        r.hi1 = __funnelshift_rc(rb0.hi, rc.hi, rs);
        r.nm1 = __funnelshift_rc(rb0.nm, rc.nm, rs);
        if constexpr (sizeof(U) == 8) {
            r.lo2 = __funnelshift_rc(rc.lo, rd.lo, rs);
            r.hi2 = __funnelshift_rc(rc.hi, rd.hi, rs);
            r.nm2 = __funnelshift_rc(rc.nm, rd.nm, rs);
        } else {
            r.lo2 = r.hi2 = r.nm2 = 0u;
        }
        const int ncol = min(32, m - 32 * fw);
        uint32_t accM = 0u;
        if (ncol == 32) {
#pragma unroll
            for (int t = 0; t < 32; ++t)
                column<U>(r, f, t, store_mask, bottom, VP, VN, accM);
        } else {
            for (int t = 0; t < ncol; ++t)
                column<U>(r, f, t, store_mask, bottom, VP, VN, accM);
        }
        // top cell D(j-E, j) after the word: each column adds 1 + its top
        // row's new difference (0 or -1)
        T += ncol - __popc(accM);
        // Early exit: the band's smallest value is at least T minus the
        // number of -1 differences.  Past E, every path through this column
        // costs more than E, so the distance saturates (the values that the
        // band computes are exact wherever they are <= E).
        if (T - Bits<U>::popc(VN) > E) return E + 1;
        ra = rb0;
        rb0 = rc;
        if constexpr (sizeof(U) == 8) {
            rc = rd;
            rd = load_word<L>(pv.read, rb, fw + 3, W);
        } else {
            rc = load_word<L>(pv.read, rb, fw + 2, W);
        }
    }
    const U first = (U(1) << E) - 1;
    const int dist = T + Bits<U>::popc(VP & first) - Bits<U>::popc(VN & first);
    return min(dist, E + 1);
}

}  // namespace pf

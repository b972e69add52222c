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

// Window of a read plane starting at bit s (may be negative): bits
// [s, s + 8*sizeof(U)).  wm1, w0, w1, w2 are read words q-1 .. q+2 with
// q = floor(s / 32) + 1 ... passed as the three/four words that cover it.
template <typename U>
__device__ __forceinline__ U window(uint32_t a, uint32_t b, uint32_t c, unsigned r) {
    if constexpr (sizeof(U) == 4) {
        return __funnelshift_r(a, b, r);
    } else {
        const uint64_t lo = __funnelshift_r(a, b, r);
        const uint64_t hi = __funnelshift_r(b, c, r);
        return lo | (hi << 32);
    }
}

template <typename U, typename L = LdNC>
__device__ __forceinline__ int verify_pair(const PairsView &pv, int64_t p, int m, int E) {
    if (m == 0) return 0;
    const int W = (m + 31) >> 5;
    const int64_t rb = pv.read.template start<L>(p), fb = pv.ref.template start<L>(p);
    const int BW = 2 * E + 1;                       // band width (bits used)
    const U band_mask = (BW >= (int)(8 * sizeof(U))) ? ~U(0) : ((U(1) << BW) - 1);
    const U store_mask = (U(1) << (2 * E)) - 1;     // 2E stored differences
    const U bottom = U(1) << (2 * E);

    // column 0: rows -E..E hold |i|; differences -1 for rows -E+1..0,
    // +1 for rows 1..E
    U VN = (U(1) << E) - 1;
    U VP = store_mask & ~VN;
    int T = E;

    // Read window: bits [s, s+|U|) with s = j - E - 1 at column j.  Keep the
    // read words q0 .. q0+2 where q0 = floor(s / 32).
    int s = -E;                   // s for column j = 1
    int q0 = (s >= 0) ? (s >> 5) : -1;
    Word3 r0 = load_word<L>(pv.read, rb, q0, W);
    Word3 r1 = load_word<L>(pv.read, rb, q0 + 1, W);
    Word3 r2 = load_word<L>(pv.read, rb, q0 + 2, W);
    Word3 f = load_word<L>(pv.ref, fb, 0, W);

    for (int j = 1; j <= m; ++j, ++s) {
        const int q = s >> 5;    // arithmetic shift: floor for negatives
        if (q != q0) {           // the window moved into the next word
            q0 = q;
            r0 = r1;
            r1 = r2;
            r2 = load_word<L>(pv.read, rb, q0 + 2, W);
        }
        const unsigned sh = (unsigned)s & 31u;
        const U wlo = window<U>(r0.lo, r1.lo, r2.lo, sh);
        const U whi = window<U>(r0.hi, r1.hi, r2.hi, sh);
        const U wnm = window<U>(r0.nm, r1.nm, r2.nm, sh);
        // reference base F[j-1]
        const int fbit = (j - 1) & 31;
        if (fbit == 0 && j > 1) f = load_word<L>(pv.ref, fb, (j - 1) >> 5, W);
        const U mlo = U(0) - U((f.lo >> fbit) & 1u);
        const U mhi = U(0) - U((f.hi >> fbit) & 1u);
        const U fn = U(0) - U((f.nm >> fbit) & 1u);
        // Eq bit q: read[j-E-1+q] equals F[j-1], neither N; bit 0 is the
        // row j-E, whose read base is read[j-E-1] = bit 0 of the window.
        const U Eq = ~((wlo ^ mlo) | (whi ^ mhi) | wnm | fn) & band_mask;

        const U Pv = VP | bottom;
        const U Mv = VN;
        const U X = Eq | Mv;
        const U D0 = (((X & Pv) + Pv) ^ Pv) | X;
        U Ph = Mv | ~(D0 | Pv);
        U Mh = Pv & D0;
        Ph = (Ph << 1) | U(1);   // +1 enters above the top row
        Mh = Mh << 1;
        const U nPv = Mh | ~(D0 | Ph);
        const U nMv = Ph & D0;
        T += 1 + (int)(nPv & U(1)) - (int)(nMv & U(1));
        VP = (nPv >> 1) & store_mask;
        VN = (nMv >> 1) & store_mask;
    }
    const U first = (U(1) << E) - 1;
    const int dist = T + Bits<U>::popc(VP & first) - Bits<U>::popc(VN & first);
    return min(dist, E + 1);
}

}  // namespace pf

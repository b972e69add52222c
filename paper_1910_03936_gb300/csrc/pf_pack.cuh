// Device functions of the packer (a1), shared by the pack kernels and the
// serving loop: ASCII -> bit-planes with the two-bit code of §5.2.3
// (A=00 C=01 G=10 T=11, N in its own plane, bytes past the end of a
// sequence in its last word are N, bytes other than A/C/G/T/N pack as N and
// raise an error bit), four bytes classified per 32-bit register.
#pragma once
#include "pf_internal.cuh"

namespace pf {

// Code bits of an ASCII base sit in bits 1..3 and ignore case:
//   a/A 0x61/0x41 -> 000, c 0x63 -> 001, t 0x74 -> 010, g 0x67 -> 011,
//   n 0x6e -> 111 (bit 1, bit 2, bit 3).
// low code bit = bit1 ^ bit2, high code bit = bit2, N = bit3.
//
// Eight bytes are handled per step.  With a = bytes 0..3 and b = bytes
// 4..7 of the step, Y keeps the low nibble of byte j of a in nibble 2j and
// the low nibble of byte j of b in nibble 2j+1, so a flag bit at bit S of
// every byte of a and b sits at bits S + 8j (a) and S + 8j + 4 (b) of Y.
// Multiplying the masked flags by sum_j 2^(24 - 7j - S) sends both flags of
// byte j (the a one and the b one) to bits 24 + j and 28 + j; every other
// partial product lands on a distinct bit below 24 or beyond bit 31, so no
// carry reaches bits 24..31, which then hold the 8 flags in byte order.
__device__ __forceinline__ uint32_t interleave_nibbles(uint32_t a, uint32_t b) {
    return (a & 0x0f0f0f0fu) | ((b << 4) & 0xf0f0f0f0u);
}

template <int S>
__device__ __forceinline__ uint32_t gather8(uint32_t y) {
    return (y & (0x11111111u << S)) * (0x01020408u >> S);
}

// Canonical lower-case letter per 3-bit pattern (bits 1..3 of the byte),
// as an 8-byte table for byte_perm: patterns 0,1,2,3,7 -> a,c,t,g,n;
// 4,5,6 -> 0, which no lower-cased byte equals.
constexpr uint32_t kCanonLo = 0x67746361u;  // g t c a
constexpr uint32_t kCanonHi = 0x6e000000u;  // n . . .

// Nonzero iff one of the 8 bytes of (a, b) is not A/C/G/T/N (either case).
// The patterns of Y, one per nibble, select the canonical letters of bytes
// (a0 b0 a1 b1) and (a2 b2 a3 b3); the bytes are interleaved the same way.
__device__ __forceinline__ uint32_t invalid8(uint32_t a, uint32_t b, uint32_t y) {
    const uint32_t z = (y >> 1) & 0x77777777u;
    const uint32_t c0 = __byte_perm(kCanonLo, kCanonHi, z);
    const uint32_t c1 = __byte_perm(kCanonLo, kCanonHi, z >> 16);
    const uint32_t i0 = __byte_perm(a, b, 0x5140u);
    const uint32_t i1 = __byte_perm(a, b, 0x7362u);
    return (c0 ^ (i0 | 0x20202020u)) | (c1 ^ (i1 | 0x20202020u));
}

// Per-byte exact classification of the first vb bytes, for words in which
// the fast test saw a byte outside A/C/G/T/N.  Returns whether such a byte
// lies among the first vb (bytes past vb are N and never an error).
__device__ __forceinline__ bool slow_word(const uint32_t *vals, int vb, uint32_t *lo,
                                          uint32_t *hi, uint32_t *nm) {
    uint32_t olo = 0u, ohi = 0u, onm = 0u;
    bool found = false;
    for (int b = 0; b < 32; ++b) {
        const uint32_t c = (vals[b >> 2] >> (8 * (b & 3))) & 0xffu;
        const uint32_t l = c | 0x20u;
        int code;
        if (b >= vb) code = 4;
        else if (l == 0x61u) code = 0;
        else if (l == 0x63u) code = 1;
        else if (l == 0x67u) code = 2;
        else if (l == 0x74u) code = 3;
        else {
            code = 4;
            found |= (l != 0x6eu);
        }
        if (code == 4) onm |= 1u << b;
        else {
            if (code & 1) olo |= 1u << b;
            if (code & 2) ohi |= 1u << b;
        }
    }
    *lo = olo;
    *hi = ohi;
    *nm = onm;
    return found;
}

// The 36 bytes that word w of a sequence needs, and where its bases start.
struct PackWindow {
    uint32_t u[9];  // aligned 4-byte words from the word's first base on
    unsigned sh;    // bit offset of the first base in u[0]
    int vb;         // valid bytes in the word, 1..32
};

// Load word w of a sequence whose bytes start at `src` (len bytes).  All 32
// byte slots go through the fast path, including those past the end, which
// are then forced to N.  `lim` is one past the last byte of the whole input
// buffer: a word whose 36-byte window lies below it (rounded up to 4 bytes)
// reads its window unguarded, so bytes past the end of the sequence are the
// next sequence's; otherwise 4-byte words wholly past the end are not read
// and count as "NNNN".  A byte past the end that is not a base only sends
// the word to the exact path.
template <typename L = LdNC>
__device__ __forceinline__ void pack_load(const uint8_t *src, int len, int w, const uint8_t *lim,
                                          PackWindow &pw) {
    const int b0 = 32 * w;
    pw.vb = min(32, len - b0);
    const uintptr_t a = reinterpret_cast<uintptr_t>(src + b0);
    const uint32_t *aw = reinterpret_cast<const uint32_t *>(a & ~uintptr_t(3));
    pw.sh = 8u * unsigned(a & 3u);
    if (reinterpret_cast<uintptr_t>(aw + 9) <= ((reinterpret_cast<uintptr_t>(lim) + 3u) & ~uintptr_t(3))) {
#pragma unroll
        for (int k = 0; k < 9; ++k) pw.u[k] = L::ld(aw + k);
    } else {
        const uintptr_t end = a + (uintptr_t)pw.vb;  // one past the last valid byte
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            const uintptr_t wa = reinterpret_cast<uintptr_t>(aw + k);
            pw.u[k] = (wa < end) ? L::ld(aw + k) : 0x4e4e4e4eu;
        }
    }
}

// The three plane words of a loaded window.
__device__ __forceinline__ void pack_decode(const PackWindow &pw, uint32_t *lo, uint32_t *hi,
                                            uint32_t *nm, unsigned *err) {
    uint32_t v[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = __funnelshift_r(pw.u[i], pw.u[i + 1], pw.sh);
    uint32_t olo = 0u, ohi = 0u, onm = 0u, bad = 0u;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const uint32_t y = interleave_nibbles(v[2 * i], v[2 * i + 1]);
        bad |= invalid8(v[2 * i], v[2 * i + 1], y);
        const uint32_t t = y ^ (y >> 1);  // bit 1 of each nibble: bit1 ^ bit2
        const uint32_t keep = 0xffu << (8 * i);
        olo |= (gather8<1>(t) >> (24 - 8 * i)) & keep;
        ohi |= (gather8<2>(y) >> (24 - 8 * i)) & keep;
        onm |= (gather8<3>(y) >> (24 - 8 * i)) & keep;
    }
    if (bad) {
        if (slow_word(v, pw.vb, lo, hi, nm)) atomicOr(err, ERR_BYTES);
        return;
    }
    const uint32_t vmask = (pw.vb >= 32) ? 0xffffffffu : ((1u << pw.vb) - 1u);
    onm |= ~vmask;      // bytes past the end are N
    *lo = olo & ~onm;   // N carries code 00
    *hi = ohi & ~onm;
    *nm = onm;
}

template <typename L = LdNC>
__device__ __forceinline__ void pack_word(const uint8_t *src, int len, int w, uint32_t *lo,
                                          uint32_t *hi, uint32_t *nm, unsigned *err,
                                          const uint8_t *lim) {
    PackWindow pw;
    pack_load<L>(src, len, w, lim, pw);
    pack_decode(pw, lo, hi, nm, err);
}

}  // namespace pf

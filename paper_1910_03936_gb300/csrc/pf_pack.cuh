// Device functions of the packer (a1), shared by the pack kernels and the
// serving loop: ASCII -> bit-planes with the two-bit code of §5.2.3
// (A=00 C=01 G=10 T=11, N in its own plane, bytes past the end of a
// sequence in its last word are N, bytes other than A/C/G/T/N pack as N and
// raise an error bit), four bytes classified per 32-bit register.
#pragma once
#include "pf_internal.cuh"

namespace pf {

// Code bits of an ASCII base sit in bits 1..3 and ignore case:
//   a/A 0x61/0x41 -> 000, c 0x63 -> 100, g 0x67 -> 110, t 0x74 -> 010,
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

// Canonical lower-case letter per 3-bit pattern of bits 0..2, as an 8-byte
// table for byte_perm: patterns 1,3,4,6,7 -> a,c,t,n,g (the five letters
// differ there); 0,2,5 -> 0, which no lower-cased byte equals.  A byte is
// a base or N exactly when, lower-cased, it equals the entry of its own
// pattern.
constexpr uint32_t kCanonLo = 0x63006100u;  // c . a .
constexpr uint32_t kCanonHi = 0x676e0074u;  // g n . t

// Nonzero iff one of the 8 bytes of (a, b) is not A/C/G/T/N (either case).
// The nibbles of Y select the canonical letters of bytes (a0 b0 a1 b1) and
// (a2 b2 a3 b3); the bytes are interleaved the same way.
__device__ __forceinline__ uint32_t invalid8(uint32_t a, uint32_t b, uint32_t y) {
    const uint32_t z = y & 0x77777777u;
    const uint32_t c0 = __byte_perm(kCanonLo, kCanonHi, z);
    const uint32_t c1 = __byte_perm(kCanonLo, kCanonHi, z >> 16);
    const uint32_t i0 = __byte_perm(a, b, 0x5140u);
    const uint32_t i1 = __byte_perm(a, b, 0x7362u);
    return (c0 ^ (i0 | 0x20202020u)) | (c1 ^ (i1 | 0x20202020u));
}

// Bits 24..31 of g0..g3 (the flags of bytes 0..7, 8..15, 16..23, 24..31)
// as one word.
__device__ __forceinline__ uint32_t join4(uint32_t g0, uint32_t g1, uint32_t g2, uint32_t g3) {
    return __byte_perm(__byte_perm(g0, g1, 0x0073u), __byte_perm(g2, g3, 0x0073u), 0x5410u);
}

// The three plane words of 32 bytes (byte b in byte b%4 of v[b/4]), N
// carrying code 00.  Returns nonzero if a byte is not A/C/G/T/N; the words
// are then not meaningful.
__device__ __forceinline__ uint32_t decode32(const uint32_t *v, uint32_t &lo, uint32_t &hi,
                                             uint32_t &nm) {
    uint32_t g1[4], g2[4], g3[4], bad = 0u;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const uint32_t y = interleave_nibbles(v[2 * i], v[2 * i + 1]);
        bad |= invalid8(v[2 * i], v[2 * i + 1], y);
        g1[i] = gather8<1>(y);
        g2[i] = gather8<2>(y);
        g3[i] = gather8<3>(y);
    }
    const uint32_t h = join4(g2[0], g2[1], g2[2], g2[3]);
    nm = join4(g3[0], g3[1], g3[2], g3[3]);
    lo = join4(g1[0], g1[1], g1[2], g1[3]) ^ h;  // N: bit1 = bit2 = 1 -> 0
    hi = h & ~nm;
    return bad;
}

// Per-byte exact classification of 32 bytes (bytes 0..15 in x, 16..31 in
// y), for chunks in which the fast test saw a byte outside A/C/G/T/N.
// Bytes outside [vlo, vhi) are N and never an error.  Returns the lo, hi
// and N words and, in w, whether a byte inside is neither a base nor N
// (such a byte packs as N).
static __device__ __noinline__ uint4 slow_chunk(uint4 x, uint4 y, int vlo, int vhi) {
    const uint32_t vals[8] = {x.x, x.y, x.z, x.w, y.x, y.y, y.z, y.w};
    uint32_t olo = 0u, ohi = 0u, onm = 0u, found = 0u;
    for (int b = 0; b < 32; ++b) {
        const uint32_t c = (vals[b >> 2] >> (8 * (b & 3))) & 0xffu;
        const uint32_t l = c | 0x20u;
        int code;
        if (b < vlo || b >= vhi) code = 4;
        else if (l == 0x61u) code = 0;
        else if (l == 0x63u) code = 1;
        else if (l == 0x67u) code = 2;
        else if (l == 0x74u) code = 3;
        else {
            code = 4;
            found |= (l != 0x6eu) ? 1u : 0u;
        }
        if (code == 4) onm |= 1u << b;
        else {
            if (code & 1) olo |= 1u << b;
            if (code & 2) ohi |= 1u << b;
        }
    }
    return make_uint4(olo, ohi, onm, found);
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
    uint32_t olo, ohi, onm;
    if (decode32(v, olo, ohi, onm)) {
        const uint4 r = slow_chunk(make_uint4(v[0], v[1], v[2], v[3]),
                                   make_uint4(v[4], v[5], v[6], v[7]), 0, pw.vb);
        if (r.w) atomicOr(err, ERR_BYTES);
        *lo = r.x;
        *hi = r.y;
        *nm = r.z;
        return;
    }
    const uint32_t vmask = (pw.vb >= 32) ? 0xffffffffu : ((1u << pw.vb) - 1u);
    *lo = olo & vmask;  // bytes past the end are N
    *hi = ohi & vmask;
    *nm = onm | ~vmask;
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

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
// Gather: for x with one flag bit at bit s of each byte, x * (0x10204080 >>
// s) puts the flag of byte i at bit 28 + i and every other partial product
// on a distinct lower bit or above bit 31, so bits 28..31 are the 4 flags.
template <int S>
__device__ __forceinline__ uint32_t gather4(uint32_t x) {
    return (x & (0x01010101u << S)) * (0x10204080u >> S);
}

// Canonical lower-case letter per 3-bit pattern (bits 1..3 of the byte),
// as an 8-byte table for byte_perm: patterns 0,1,2,3,7 -> a,c,t,g,n;
// 4,5,6 -> 0, which no lower-cased byte equals.
constexpr uint32_t kCanonLo = 0x67746361u;  // g t c a
constexpr uint32_t kCanonHi = 0x6e000000u;  // n . . .

// Per-byte classification of four bytes against the canonical table:
// returns a nonzero word iff some byte outside `pad` is not A/C/G/T/N.
__device__ __forceinline__ uint32_t invalid4(uint32_t v, uint32_t pad) {
    const uint32_t x = (v >> 1) & 0x07070707u;          // pattern per byte
    const uint32_t y = x | (x >> 4);                    // byte0 = p0|p1<<4, byte2 = p2|p3<<4
    const uint32_t sel = __byte_perm(y, 0u, 0x0020u);   // nibbles p0 p1 p2 p3
    const uint32_t canon = __byte_perm(kCanonLo, kCanonHi, sel);
    return (canon ^ (v | 0x20202020u)) & ~pad;
}

// Per-byte exact classification, for words that hold an invalid byte.
__device__ __forceinline__ void slow_word(const uint32_t *vals, int vb, uint32_t *lo,
                                          uint32_t *hi, uint32_t *nm) {
    uint32_t olo = 0u, ohi = 0u, onm = 0u;
    for (int b = 0; b < 32; ++b) {
        const uint32_t c = (vals[b >> 2] >> (8 * (b & 3))) & 0xffu;
        const uint32_t l = c | 0x20u;
        int code;
        if (b >= vb) code = 4;
        else if (l == 0x61u) code = 0;
        else if (l == 0x63u) code = 1;
        else if (l == 0x67u) code = 2;
        else if (l == 0x74u) code = 3;
        else code = 4;  // N and every invalid byte
        if (code == 4) onm |= 1u << b;
        else {
            if (code & 1) olo |= 1u << b;
            if (code & 2) ohi |= 1u << b;
        }
    }
    *lo = olo;
    *hi = ohi;
    *nm = onm;
}

// Pack word w of a sequence whose bytes start at `src` (len bytes).
template <typename L = LdNC>
__device__ __forceinline__ void pack_word(const uint8_t *src, int len, int w, uint32_t *lo,
                                          uint32_t *hi, uint32_t *nm, unsigned *err) {
    const int b0 = 32 * w;
    const int vb = min(32, len - b0);  // valid bytes in this word, >= 1
    const uintptr_t a = reinterpret_cast<uintptr_t>(src + b0);
    const uint32_t *aw = reinterpret_cast<const uint32_t *>(a & ~uintptr_t(3));
    const unsigned sh = 8u * unsigned(a & 3u);
    const uintptr_t end = a + (uintptr_t)vb;  // one past the last valid byte
    uint32_t u[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        const uintptr_t wa = reinterpret_cast<uintptr_t>(aw + k);
        u[k] = (wa < end) ? L::ld(aw + k) : 0u;
    }
    uint32_t v[8];
    uint32_t olo = 0u, ohi = 0u, onm = 0u, bad = 0u;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        v[i] = __funnelshift_r(u[i], u[i + 1], sh);
        const int first = 4 * i;
        uint32_t pad;
        if (first + 4 <= vb) pad = 0u;
        else if (first >= vb) pad = 0xffffffffu;
        else pad = 0xffffffffu << (8 * (vb - first));
        bad |= invalid4(v[i], pad);
        const uint32_t t = v[i] ^ (v[i] >> 1);  // bit 1 = bit1 ^ bit2
        const int up = 28 - first;          // flags of bytes first..first+3
        const uint32_t keep = 0xfu << first;
        olo |= (gather4<1>(t) >> up) & keep;
        ohi |= (gather4<2>(v[i]) >> up) & keep;
        onm |= (gather4<3>(v[i]) >> up) & keep;
    }
    if (bad) {
        slow_word(v, vb, lo, hi, nm);
        atomicOr(err, ERR_BYTES);
        return;
    }
    const uint32_t vmask = (vb >= 32) ? 0xffffffffu : ((1u << vb) - 1u);
    onm = (onm & vmask) | ~vmask;  // bytes past the end are N
    *lo = olo & ~onm;              // N carries code 00
    *hi = ohi & ~onm;
    *nm = onm;
}

}  // namespace pf

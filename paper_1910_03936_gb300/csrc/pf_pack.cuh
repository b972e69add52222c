// Device functions of the packer (a1), shared by the pack kernels and the
// serving loop: ASCII -> bit-planes with the two-bit code of §5.2.3
// (A=00 C=01 G=10 T=11, N in its own plane, bytes past the end of a
// sequence in its last word are N), four bytes classified per register.
#pragma once
#include "pf_internal.cuh"

namespace pf {

// Bits at byte positions 0, 8, 16, 24 of x gathered into bits 28..31.
__device__ __forceinline__ uint32_t gather_byte_lsbs(uint32_t x) {
    return x * 0x10204080u;
}

struct Planes4 {
    uint32_t lo, hi, nm;  // per-byte LSBs (bit 0 of each byte)
    uint32_t bad;         // per-byte LSB set where the byte is not A/C/G/T/N
};

// Classify four ASCII bytes.  Lower-casing (| 0x20) maps A/C/G/T/N onto
// a (0x61) c (0x63) g (0x67) t (0x74) n (0x6e): bit 2 is the high code bit,
// bit 1 ^ bit 2 the low code bit, bit 3 flags n.  A byte is valid exactly
// when it equals the canonical letter rebuilt from those bits.
// `pad` has 0xff in the bytes past the end of the sequence: they become N.
__device__ __forceinline__ Planes4 classify4(uint32_t v, uint32_t pad) {
    const uint32_t y = v | 0x20202020u;
    const uint32_t s2 = y >> 2;
    const uint32_t hb = s2 & 0x01010101u;
    const uint32_t lb = ((y >> 1) ^ s2) & 0x01010101u;
    const uint32_t nb = (y >> 3) & 0x01010101u;
    const uint32_t lh = lb & hb;
    const uint32_t acgt = 0x61616161u + lb * 2u + hb * 6u + lh * 11u;
    const uint32_t nbytes = nb * 0xffu;
    const uint32_t canon = (acgt & ~nbytes) | (0x6e6e6e6eu & nbytes);
    const uint32_t diff = (canon ^ y) & ~pad;
    uint32_t badb = 0u;
    if (diff) {
        const uint32_t nz = (((diff & 0x7f7f7f7fu) + 0x7f7f7f7fu) | diff) & 0x80808080u;
        badb = nz >> 7;
    }
    const uint32_t padb = pad & 0x01010101u;
    const uint32_t asn = badb | padb;  // bytes forced to N
    const uint32_t nall = nb | asn;    // N bytes carry code 00
    Planes4 r;
    r.lo = lb & ~nall;
    r.hi = hb & ~nall;
    r.nm = nall;
    r.bad = badb;
    return r;
}

// Pack word w of a sequence whose bytes start at `src` (len bytes).
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
        u[k] = (wa < end) ? __ldg(aw + k) : 0u;
    }
    uint32_t olo = 0u, ohi = 0u, onm = 0u, obad = 0u;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const uint32_t v = __funnelshift_r(u[i], u[i + 1], sh);
        const int first = 4 * i;
        uint32_t pad;
        if (first + 4 <= vb) pad = 0u;
        else if (first >= vb) pad = 0xffffffffu;
        else pad = 0xffffffffu << (8 * (vb - first));
        const Planes4 c = classify4(v, pad);
        olo |= (gather_byte_lsbs(c.lo) >> 28) << first;
        ohi |= (gather_byte_lsbs(c.hi) >> 28) << first;
        onm |= (gather_byte_lsbs(c.nm) >> 28) << first;
        obad |= c.bad;
    }
    *lo = olo;
    *hi = ohi;
    *nm = onm;
    if (obad) atomicOr(err, ERR_BYTES);
}

}  // namespace pf

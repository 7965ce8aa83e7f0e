// pack_bits.cuh -- the packing kernels' inner step: 32 ASCII bases -> one
// word of each of the hi, lo and N planes.  Compiles for the host as well
// (g++), so a CPU test checks it against the byte-wise rule on every byte
// value at every position.
#pragma once
#include <cstdint>

#ifdef __CUDACC__
#define IFA_PACK_FN __host__ __device__ __forceinline__
#else
#define IFA_PACK_FN inline
#endif

namespace ifa {
namespace packbits {

// Byte k of the result is byte (s >> 4k) & 7 of {y:x} (x bytes 0-3, y 4-7).
IFA_PACK_FN uint32_t byte_perm(uint32_t x, uint32_t y, uint32_t s) {
#ifdef __CUDA_ARCH__
    return __byte_perm(x, y, s);
#else
    const uint64_t v = (static_cast<uint64_t>(y) << 32) | x;
    uint32_t r = 0;
    for (int k = 0; k < 4; k++) r |= static_cast<uint32_t>((v >> (8 * ((s >> (4 * k)) & 7u))) & 0xffu) << (8 * k);
    return r;
#endif
}

// Two words' selected bits -- bits 0, 8, 16, 24 (word a) and 4, 12, 20,
// 28 (word b) of t -- gathered into bits 24..31 of the product by one
// multiply: the partial products of 2^24, 2^17, 2^10, 2^3 put the
// selected bits on 24..31 in base order and every other bit on a distinct
// position below 24 or past 31, so no carry reaches the top byte.
IFA_PACK_FN uint32_t gather_pair(uint32_t t) { return t * 0x01020408u; }

// The top bytes of four gathered products as one word (byte p from p).
IFA_PACK_FN uint32_t top_bytes(uint32_t p0, uint32_t p1, uint32_t p2, uint32_t p3) {
    return byte_perm(byte_perm(p0, p1, 0x0073u), byte_perm(p2, p3, 0x0073u), 0x5410u);
}

// Per byte of u, zero exactly when the byte is A, C, G or T in either case.
// m = u & 0x06060606 holds the code bits (1, 2).  With the code and case
// bits masked off (0xD9), a, c and g leave 0x41 and t leaves 0x50, so the
// byte is compared with 0x41 + 15 [code == 2].
IFA_PACK_FN uint32_t letter_miss(uint32_t u, uint32_t m) {
    const uint32_t t2 = (m >> 2) & ~(m >> 1) & 0x01010101u;
    return (u & 0xD9D9D9D9u) ^ (t2 * 15u + 0x41414141u);
}

// 32 ASCII bytes (byte j of u[i] = base 4 i + j) -> the hi, lo and N planes
// of one word.  The 2-bit code is (byte >> 1) & 3 (A 0, C 1, T 2, G 3).
// Words are taken in pairs: their code bits are merged into one word
// (word b's shifted up a nibble) and each plane's 8 bits gathered by one
// multiply.  The N plane is built only when some byte is not a base; the
// code bits of non-bases are cleared.
IFA_PACK_FN void pack32(const uint32_t *u, uint32_t &hi, uint32_t &lo, uint32_t &nn) {
    uint32_t pl[4], ph[4], miss = 0;
#ifdef __CUDACC__
#pragma unroll
#endif
    for (int p = 0; p < 4; p++) {
        const uint32_t a = u[2 * p], b = u[2 * p + 1];
        const uint32_t ma = a & 0x06060606u, mb = b & 0x06060606u;
        const uint32_t v = mb * 16u + ma;   // bits 1, 2 (word a) and 5, 6 (word b) of each byte
        pl[p] = gather_pair((v >> 1) & 0x11111111u);
        ph[p] = gather_pair((v >> 2) & 0x11111111u);
        miss |= letter_miss(a, ma) | letter_miss(b, mb);
    }
    lo = top_bytes(pl[0], pl[1], pl[2], pl[3]);
    hi = top_bytes(ph[0], ph[1], ph[2], ph[3]);
    nn = 0;
    if (miss) {
        uint32_t pn[4];
#ifdef __CUDACC__
#pragma unroll
#endif
        for (int p = 0; p < 4; p++) {
            const uint32_t a = u[2 * p], b = u[2 * p + 1];
            const uint32_t xa = letter_miss(a, a & 0x06060606u), xb = letter_miss(b, b & 0x06060606u);
            // high bit of each byte: the byte is not a base
            const uint32_t za = (((xa & 0x7f7f7f7fu) + 0x7f7f7f7fu) | xa) & 0x80808080u;
            const uint32_t zb = (((xb & 0x7f7f7f7fu) + 0x7f7f7f7fu) | xb) & 0x80808080u;
            pn[p] = gather_pair((za >> 7) | (zb >> 3));
        }
        nn = top_bytes(pn[0], pn[1], pn[2], pn[3]);
        hi &= ~nn;
        lo &= ~nn;
    }
}

}  // namespace packbits
}  // namespace ifa

// pack.cu -- reference packing on the device (ASCII -> 2-bit planes + N + piece starts).
//
// The reference is streamed as ASCII and never pre-indexed (Methods,
// "Algorithm Design"); each pushed segment is packed here, in HBM, right
// before it is scanned.  A batch is a halo region of H bases (H a multiple
// of 32: 'N' padding, then the last <= L_max - 1 bases of a contig that
// continues from the previous segment) followed by the new segment, which
// therefore starts on a word boundary and is read with aligned vectors.
#include "ifa_internal.cuh"

namespace ifa {

namespace {

constexpr int kPackThreads = 256;  // one output word (32 bases) per thread

__device__ __forceinline__ void pack_byte(uint32_t c, uint32_t bit, uint32_t &hi, uint32_t &lo,
                                          uint32_t &nn) {
    const uint32_t ok = is_base(c) ? 1u : 0u;
    const uint32_t code = base_code(c) * ok;
    hi |= (code >> 1) << bit;
    lo |= (code & 1u) << bit;
    nn |= (ok ^ 1u) << bit;
}

// Bits 0, 8, 16, 24 of m gathered into bits 24..27 by one multiply: the
// partial products of 2^24, 2^17, 2^10, 2^3 land on distinct bits, so no
// carries occur and bits 24..27 hold exactly the four selected bits.
__device__ __forceinline__ uint32_t gather_nibble(uint32_t m) { return (m * 0x01020408u) >> 24; }

// Four ASCII bytes (byte j of u = base j) -> bits 0..3 of the hi, lo and N
// planes.  The 2-bit code is (byte >> 1) & 3 (A 0, C 1, T 2, G 3); a byte is
// a base exactly when, with the case bit set, it equals the lower-case
// letter its code bits name, tested for all four bytes at once with an
// exact zero-byte test.  Code bits of non-bases are cleared by the caller.
__device__ __forceinline__ void pack4(uint32_t u, uint32_t &h4, uint32_t &l4, uint32_t &n4) {
    const uint32_t l = (u >> 1) & 0x01010101u;
    const uint32_t h = (u >> 2) & 0x01010101u;
    // per byte 0x61 + 2 l + 19 h - 15 l h: 'a' 'c' 't' 'g' for codes 0..3 (no carries)
    const uint32_t letter = 0x61616161u + 2u * l + 19u * h - 15u * (l & h);
    const uint32_t x = (u | 0x20202020u) ^ letter;
    const uint32_t nz = (((x & 0x7f7f7f7fu) + 0x7f7f7f7fu) | x) & 0x80808080u;  // high bit: byte != 0
    l4 = gather_nibble(l);
    h4 = gather_nibble(h);
    n4 = gather_nibble(nz >> 7);
}

// Word w of the batch.  Words below H/32 hold the halo region: 'N' padding
// up to H - hlen, then the hlen halo bases.  Word H/32 + i holds segment
// bytes [32 i, 32 i + 32), read as two 16-byte vectors when the segment is
// 16-byte aligned; bytes past the segment end are N.
template <bool ALIGNED>
__global__ void __launch_bounds__(kPackThreads)
k_pack(const uint8_t *__restrict__ halo, uint32_t hlen, uint32_t H, const uint8_t *__restrict__ seg,
       uint64_t slen, uint4 *__restrict__ words, uint64_t nwords) {
    const uint64_t w = static_cast<uint64_t>(blockIdx.x) * kPackThreads + threadIdx.x;
    if (w >= nwords) return;
    uint32_t hi = 0, lo = 0, nn = 0;
    const uint64_t hw = H >> 5;
    if (w < hw) {
        const uint32_t pad = H - hlen;
        for (uint32_t b = 0; b < 32; b++) {
            const uint32_t i = static_cast<uint32_t>(w) * 32 + b;
            pack_byte(i < pad ? 'N' : halo[i - pad], b, hi, lo, nn);
        }
    } else {
        const uint64_t o = (w - hw) * 32;
        if (ALIGNED && o + 32 <= slen) {
            const uint4 *v = reinterpret_cast<const uint4 *>(seg + o);
            const uint4 a = __ldg(v), c = __ldg(v + 1);
            const uint32_t u[8] = {a.x, a.y, a.z, a.w, c.x, c.y, c.z, c.w};
#pragma unroll
            for (int j = 0; j < 8; j++) {
                uint32_t h4, l4, n4;
                pack4(u[j], h4, l4, n4);
                hi |= h4 << (4 * j);
                lo |= l4 << (4 * j);
                nn |= n4 << (4 * j);
            }
            hi &= ~nn;
            lo &= ~nn;
        } else {
            for (uint32_t b = 0; b < 32; b++)
                pack_byte(o + b < slen ? seg[o + b] : 'N', b, hi, lo, nn);
        }
    }
    words[w] = make_uint4(hi, lo, nn, 0u);
}

// B plane: a bit at the first base of every piece that does not start the batch.
__global__ void k_mark_pieces(const DevPiece *__restrict__ pc, uint32_t n, uint4 *__restrict__ words) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint64_t p = pc[i].start;
    if (p == 0) return;
    uint32_t *w = reinterpret_cast<uint32_t *>(words + (p >> 5)) + 3;
    atomicOr(w, 1u << (p & 31));
}

__global__ void k_halo_update(const uint8_t *__restrict__ old_halo, uint32_t old_len,
                              const uint8_t *__restrict__ seg, uint64_t slen, uint32_t new_len,
                              uint8_t *__restrict__ new_halo) {
    const uint64_t total = old_len + slen;
    for (uint32_t i = threadIdx.x; i < new_len; i += blockDim.x) {
        uint64_t g = total - new_len + i;
        new_halo[i] = g < old_len ? old_halo[g] : seg[g - old_len];
    }
}

}  // namespace

cudaError_t launch_pack(const uint8_t *halo, uint32_t hlen, uint32_t H, const uint8_t *seg,
                        uint64_t slen, uint4 *words, uint64_t nwords_padded, cudaStream_t st) {
    if (nwords_padded == 0) return cudaSuccess;
    const uint64_t grid = (nwords_padded + kPackThreads - 1) / kPackThreads;
    if ((reinterpret_cast<uintptr_t>(seg) & 15u) == 0)
        k_pack<true><<<static_cast<unsigned>(grid), kPackThreads, 0, st>>>(halo, hlen, H, seg, slen, words,
                                                                           nwords_padded);
    else
        k_pack<false><<<static_cast<unsigned>(grid), kPackThreads, 0, st>>>(halo, hlen, H, seg, slen, words,
                                                                            nwords_padded);
    return cudaGetLastError();
}

cudaError_t launch_mark_pieces(const DevPiece *pieces, uint32_t n, uint4 *words, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    unsigned grid = (n + 255) / 256;
    k_mark_pieces<<<grid, 256, 0, st>>>(pieces, n, words);
    return cudaGetLastError();
}

cudaError_t launch_halo_update(const uint8_t *old_halo, uint32_t old_len, const uint8_t *seg,
                               uint64_t slen, uint32_t new_len, uint8_t *new_halo, cudaStream_t st) {
    if (new_len == 0) return cudaSuccess;
    k_halo_update<<<1, 256, 0, st>>>(old_halo, old_len, seg, slen, new_len, new_halo);
    return cudaGetLastError();
}

}  // namespace ifa

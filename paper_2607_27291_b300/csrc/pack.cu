// pack.cu -- reference packing on the device (ASCII -> 2-bit planes + N + piece starts).
//
// The reference is streamed as ASCII and never pre-indexed (Methods,
// "Algorithm Design"); each pushed segment is packed here, in HBM, right
// before it is scanned.  A batch is the previous segment's halo (the last
// L_max - 1 bases of a contig that continues) followed by the new segment.
#include "ifa_internal.cuh"

namespace ifa {

namespace {

constexpr int kPackThreads = 256;                 // one output word per thread
constexpr int kPackBases = kPackThreads * 32;     // bases per CTA

__global__ void __launch_bounds__(kPackThreads)
k_pack(const uint8_t *__restrict__ halo, uint32_t hlen, const uint8_t *__restrict__ seg,
       uint64_t slen, uint4 *__restrict__ words, uint64_t nwords) {
    __shared__ uint32_t sbuf[kPackBases / 4];
    uint8_t *sb = reinterpret_cast<uint8_t *>(sbuf);
    const uint64_t base0 = static_cast<uint64_t>(blockIdx.x) * kPackBases;
    const uint64_t total = hlen + slen;
    // coalesced byte loads: a warp reads 32 consecutive bytes per step
    for (int i = threadIdx.x; i < kPackBases; i += kPackThreads) {
        uint64_t g = base0 + i;
        uint8_t c = 'N';
        if (g < hlen) c = halo[g];
        else if (g < total) c = seg[g - hlen];
        sb[i] = c;
    }
    __syncthreads();
    const uint64_t w = static_cast<uint64_t>(blockIdx.x) * kPackThreads + threadIdx.x;
    if (w >= nwords) return;
    uint32_t hi = 0, lo = 0, nn = 0;
    const uint32_t t = threadIdx.x;
#pragma unroll
    for (int jj = 0; jj < 8; jj++) {
        // rotated order: lanes t = a + 4m read banks 8a + (jj + t + t/8) mod 8,
        // which are distinct over the warp, so the reads are conflict-free
        const uint32_t j = (jj + t + (t >> 3)) & 7u;
        const uint32_t v = sbuf[t * 8 + j];
#pragma unroll
        for (int b = 0; b < 4; b++) {
            const uint32_t c = (v >> (8 * b)) & 0xFFu;
            const uint32_t bit = j * 4 + b;
            const uint32_t ok = is_base(c) ? 1u : 0u;
            const uint32_t code = base_code(c) * ok;
            hi |= (code >> 1) << bit;
            lo |= (code & 1u) << bit;
            nn |= (ok ^ 1u) << bit;
        }
    }
    words[w] = make_uint4(hi, lo, nn, 0u);
}

__global__ void k_mark_pieces(const DevPiece *__restrict__ pc, uint32_t n, uint4 *__restrict__ words) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x + 1;  // piece 0 starts the batch
    if (i >= n) return;
    uint64_t p = pc[i].start;
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

cudaError_t launch_pack(const uint8_t *halo, uint32_t hlen, const uint8_t *seg, uint64_t slen,
                        uint4 *words, uint64_t nwords_padded, cudaStream_t st) {
    if (nwords_padded == 0) return cudaSuccess;
    uint64_t grid = (nwords_padded + kPackThreads - 1) / kPackThreads;
    k_pack<<<static_cast<unsigned>(grid), kPackThreads, 0, st>>>(halo, hlen, seg, slen, words,
                                                                 nwords_padded);
    return cudaGetLastError();
}

cudaError_t launch_mark_pieces(const DevPiece *pieces, uint32_t n, uint4 *words, cudaStream_t st) {
    if (n <= 1) return cudaSuccess;
    unsigned grid = (n - 1 + 255) / 256;
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

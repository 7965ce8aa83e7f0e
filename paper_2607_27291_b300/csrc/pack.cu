// pack.cu -- reference packing on the device (ASCII -> 2-bit planes, and a
// sparse table of the words holding an N or a piece start).
//
// The reference is streamed as ASCII and never pre-indexed (Methods,
// "Algorithm Design"); each pushed segment is packed here, in HBM, right
// before it is scanned.  A batch is a halo region of H bases (H a multiple
// of 32: 'N' padding, then the last <= L_max - 1 bases of a contig that
// continues from the previous segment) followed by the new segment, which
// therefore starts on a word boundary and is read with aligned vectors.
//
// Appends to the resident store take three steps: k_pack writes the hi/lo
// words and every word's N mask into a scratch array; k_mark_pieces adds
// the piece-start (B) bits there; k_build_dir turns the scratch into the
// directory (one bitmap per 32 words) and the exception entries of the
// special words (see ifa_internal.cuh), continuing a partly filled group.
// Streamed batches, which always start at word 0, take one fused pass,
// k_pack_dir, with no scratch.
#include "ifa_internal.cuh"
#include "pack_bits.cuh"

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

using packbits::pack32;   // 32 bases -> hi, lo and N plane words (pack_bits.cuh)

// Word w of the batch.  Words below H/32 hold the halo region: 'N' padding
// up to H - hlen, then the hlen halo bases.  Word H/32 + i holds segment
// bytes [32 i, 32 i + 32), read as two 16-byte vectors when the segment is
// 16-byte aligned; bytes past the segment end are N.
template <bool ALIGNED>
__global__ void __launch_bounds__(kPackThreads)
k_pack(const uint8_t *__restrict__ halo, uint32_t hlen, uint32_t H, const uint8_t *__restrict__ seg,
       uint64_t slen, uint2 *__restrict__ hl, uint2 *__restrict__ nb, uint64_t nwords) {
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
            pack32(u, hi, lo, nn);
        } else {
            for (uint32_t b = 0; b < 32; b++)
                pack_byte(o + b < slen ? seg[o + b] : 'N', b, hi, lo, nn);
        }
    }
    hl[w] = make_uint2(hi, lo);
    nb[w] = make_uint2(nn, 0u);
}

// B plane: a bit at the first base of every piece that does not start the
// batch, for the pieces starting among the nwords words from base `first`.
__global__ void k_mark_pieces(const DevPiece *__restrict__ pc, uint32_t n, uint64_t first, uint64_t nwords,
                              uint2 *__restrict__ nb) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint64_t p = pc[i].start;
    if (p == 0 || p < first || p - first >= 32 * nwords) return;
    atomicOr(&nb[(p - first) >> 5].y, 1u << ((p - first) & 31));
}

// One warp per group of 32 words: ballot of the special words, one range of
// exception entries per group (taken from exc_n[0]), the group's entries in
// word order.  Words of the first group below w0 keep their old masks,
// read through the old directory entry.  The last group written is one past
// the words' last group (all zero), so that a reader of two neighbouring
// entries never meets an unwritten one.
__global__ void __launch_bounds__(256)
k_build_dir(const uint2 *__restrict__ nb, uint64_t w0, uint64_t n, uint2 *__restrict__ dir, uint2 *__restrict__ exc,
            uint64_t exc_cap, unsigned long long *__restrict__ exc_n) {
    const uint32_t lane = threadIdx.x & 31u;
    const uint64_t g0 = w0 >> 5, g_end = ((w0 + n - 1) >> 5) + 2;
    const uint64_t g = g0 + (static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x) / 32;
    if (g >= g_end) return;  // whole warps: 256 threads = 8 groups
    const uint64_t w = (g << 5) + lane;
    uint2 m = make_uint2(0u, 0u);
    if (w >= w0 && w < w0 + n) {
        m = nb[w - w0];
    } else if (w < w0) {
        const uint2 d = dir[g];
        if ((d.x >> lane) & 1u) m = exc[d.y + __popc(d.x & ((1u << lane) - 1u))];
    }
    __syncwarp();
    const bool special = (m.x | m.y) != 0u;
    const uint32_t bits = __ballot_sync(0xffffffffu, special);
    const uint32_t cnt = __popc(bits);
    unsigned long long base = 0;
    if (lane == 0 && cnt) base = atomicAdd(exc_n, static_cast<unsigned long long>(cnt));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (base + cnt > exc_cap) {
        if (lane == 0) exc_n[1] = 1ull;
        return;
    }
    if (special) exc[base + __popc(bits & ((1u << lane) - 1u))] = m;
    if (lane == 0) dir[g] = make_uint2(bits, static_cast<uint32_t>(base));
}

// The first of the n pieces (sorted by start) that starts at or after base
// x, or n; all lanes of a warp call it and get the answer.  A 32-way
// search: each round probes 32 evenly spaced pieces of the range [lo, hi)
// that holds the answer, and the probes below x (a prefix of the lanes)
// narrow it to one gap between probes; three rounds cover 40,000 pieces.
__device__ __forceinline__ uint32_t first_piece_at(const DevPiece *__restrict__ pc, uint32_t n, uint64_t x,
                                                   uint32_t lane) {
    uint32_t lo = 0, hi = n;
    while (hi - lo > 32u) {
        const uint32_t step = (hi - lo + 31u) / 32u;
        const uint32_t i = lo + lane * step;
        const bool below = i < hi && pc[i].start < x;
        const uint32_t c = __popc(__ballot_sync(0xffffffffu, below));
        const uint32_t nlo = c ? lo + (c - 1u) * step + 1u : lo;
        hi = min(hi, lo + c * step);
        lo = nlo;
    }
    const uint32_t i = lo + lane;
    const bool below = i < hi && pc[i].start < x;
    return lo + __popc(__ballot_sync(0xffffffffu, below));
}

// Streamed batches in one pass: k_pack's words, the piece-start bits and
// k_build_dir's directory, with no mask scratch.  A warp packs kPackGroups
// consecutive directory groups of 32 words, lane l word l of each: it
// issues its ASCII loads for all of them first (8 x 16 bytes per lane in
// flight), finds the first group's first piece start once (first_piece_at)
// and walks the piece starts forward across its groups.  The grid covers
// one group past the words' last one, written as an empty entry (see
// k_build_dir).  exc holds at least nwords entries, so the claims cannot
// run out; a claim past exc_cap sets exc_n[1] like k_build_dir.
constexpr int kPackGroups = 4;

template <bool ALIGNED>
__global__ void __launch_bounds__(kPackThreads)
k_pack_dir(const uint8_t *__restrict__ halo, uint32_t hlen, uint32_t H, const uint8_t *__restrict__ seg,
           uint64_t slen, uint2 *__restrict__ hl, uint64_t nwords, const DevPiece *__restrict__ pc, uint32_t npieces,
           bool mark, uint2 *__restrict__ dir, uint2 *__restrict__ exc, uint64_t exc_cap,
           unsigned long long *__restrict__ exc_n) {
    const uint32_t lane = threadIdx.x & 31u;
    const uint64_t g0 = ((static_cast<uint64_t>(blockIdx.x) * kPackThreads + threadIdx.x) >> 5) * kPackGroups;
    const uint64_t last_g = ((nwords - 1) >> 5) + 1;   // one group past the last word's
    if (g0 > last_g) return;                           // whole warps
    const uint64_t hw = H >> 5;
    uint4 va[kPackGroups], vc[kPackGroups];
#pragma unroll
    for (int t = 0; t < kPackGroups; t++) {
        va[t] = vc[t] = make_uint4(0u, 0u, 0u, 0u);
        const uint64_t w = (g0 + t) * 32 + lane;
        if (ALIGNED && w < nwords && w >= hw && (w - hw) * 32 + 32 <= slen) {
            const uint4 *v = reinterpret_cast<const uint4 *>(seg + (w - hw) * 32);
            va[t] = __ldg(v);
            vc[t] = __ldg(v + 1);
        }
    }
    uint32_t pi = mark && npieces ? first_piece_at(pc, npieces, g0 << 10, lane) : 0u;
#pragma unroll
    for (int t = 0; t < kPackGroups; t++) {
        const uint64_t g = g0 + t;
        if (g > last_g) break;   // warp-uniform
        const uint64_t w = g * 32 + lane;
        uint32_t hi = 0, lo = 0, nn = 0, bb = 0;
        const bool live = w < nwords;
        if (live) {
            if (w < hw) {
                const uint32_t pad = H - hlen;
                for (uint32_t b = 0; b < 32; b++) {
                    const uint32_t i = static_cast<uint32_t>(w) * 32 + b;
                    pack_byte(i < pad ? 'N' : halo[i - pad], b, hi, lo, nn);
                }
            } else {
                const uint64_t o = (w - hw) * 32;
                if (ALIGNED && o + 32 <= slen) {
                    const uint32_t u[8] = {va[t].x, va[t].y, va[t].z, va[t].w, vc[t].x, vc[t].y, vc[t].z, vc[t].w};
                    pack32(u, hi, lo, nn);
                } else {
                    for (uint32_t b = 0; b < 32; b++)
                        pack_byte(o + b < slen ? seg[o + b] : 'N', b, hi, lo, nn);
                }
            }
            hl[w] = make_uint2(hi, lo);
        }
        if (mark && npieces) {
            // the starts in this group; pi ends at the first start of the next
            const uint64_t ge = (g + 1) << 10;
            for (; pi < npieces; pi++) {
                const uint64_t p = pc[pi].start;   // warp-uniform
                if (p >= ge) break;
                if (p != 0 && (p >> 5) == w) bb |= 1u << (p & 31);
            }
            if (!live) bb = 0;
        }
        const bool special = (nn | bb) != 0u;
        const uint32_t bits = __ballot_sync(0xffffffffu, special);
        const uint32_t cnt = __popc(bits);
        unsigned long long base = 0;
        if (lane == 0 && cnt) base = atomicAdd(exc_n, static_cast<unsigned long long>(cnt));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (base + cnt > exc_cap) {
            if (lane == 0) exc_n[1] = 1ull;
            return;
        }
        if (special) exc[base + __popc(bits & ((1u << lane) - 1u))] = make_uint2(nn, bb);
        if (lane == 0) dir[g] = make_uint2(bits, static_cast<uint32_t>(base));
    }
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
                        uint64_t slen, uint2 *hl, uint2 *nb, uint64_t nwords_padded, cudaStream_t st) {
    if (nwords_padded == 0) return cudaSuccess;
    const uint64_t grid = (nwords_padded + kPackThreads - 1) / kPackThreads;
    if ((reinterpret_cast<uintptr_t>(seg) & 15u) == 0)
        k_pack<true><<<static_cast<unsigned>(grid), kPackThreads, 0, st>>>(halo, hlen, H, seg, slen, hl, nb,
                                                                           nwords_padded);
    else
        k_pack<false><<<static_cast<unsigned>(grid), kPackThreads, 0, st>>>(halo, hlen, H, seg, slen, hl, nb,
                                                                            nwords_padded);
    return cudaGetLastError();
}

cudaError_t launch_mark_pieces(const DevPiece *pieces, uint32_t n, uint64_t first, uint64_t nwords, uint2 *nb,
                               cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    unsigned grid = (n + 255) / 256;
    k_mark_pieces<<<grid, 256, 0, st>>>(pieces, n, first, nwords, nb);
    return cudaGetLastError();
}

cudaError_t launch_build_dir(const uint2 *nb, uint64_t w0, uint64_t n, uint2 *dir, uint2 *exc, uint64_t exc_cap,
                             unsigned long long *exc_n, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    const uint64_t groups = ((w0 + n - 1) >> 5) + 2 - (w0 >> 5);
    const uint64_t grid = (groups + 7) / 8;
    k_build_dir<<<static_cast<unsigned>(grid), 256, 0, st>>>(nb, w0, n, dir, exc, exc_cap, exc_n);
    return cudaGetLastError();
}

cudaError_t refbufs_alloc(RefBufs &R, uint64_t words, uint64_t nb_words, uint64_t exc_entries) {
    cudaError_t e = cudaSuccess;
    auto get = [&](uint2 *&p, uint64_t n) {
        if (e == cudaSuccess) e = cudaMalloc(&p, (n ? n : 1) * sizeof(uint2));
    };
    get(R.hl, words);
    get(R.nb, nb_words);
    get(R.dir, dir_entries(words));
    get(R.exc, exc_entries);
    if (e == cudaSuccess) e = cudaMalloc(&R.exc_n, 2 * sizeof(unsigned long long));
    if (e == cudaSuccess) {
        R.words_cap = words;
        R.nb_cap = nb_words;
        R.exc_cap = exc_entries;
    }
    return e;
}

void refbufs_free(RefBufs &R) {
    cudaFree(R.hl);
    cudaFree(R.nb);
    cudaFree(R.dir);
    cudaFree(R.exc);
    cudaFree(R.exc_n);
    R = RefBufs{};
}

cudaError_t pack_batch(const RefBufs &R, const uint8_t *halo, uint32_t hlen, uint32_t H, const uint8_t *seg,
                       uint64_t slen, uint64_t nwords, const DevPiece *pieces, uint32_t npieces, bool mark,
                       cudaStream_t st, int *launches) {
    // every word takes at most one entry, so exc (nwords entries) cannot run out
    if (nwords == 0 || nwords > R.words_cap || nwords > R.exc_cap) return cudaErrorInvalidValue;
    cudaError_t e = cudaMemsetAsync(R.exc_n, 0, 2 * sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    const uint64_t groups = ((nwords - 1) >> 5) + 2;   // one group past the last word's
    const uint64_t threads = (groups + kPackGroups - 1) / kPackGroups * 32;
    const unsigned grid = static_cast<unsigned>((threads + kPackThreads - 1) / kPackThreads);
    if ((reinterpret_cast<uintptr_t>(seg) & 15u) == 0)
        k_pack_dir<true><<<grid, kPackThreads, 0, st>>>(halo, hlen, H, seg, slen, R.hl, nwords, pieces, npieces, mark,
                                                        R.dir, R.exc, R.exc_cap, R.exc_n);
    else
        k_pack_dir<false><<<grid, kPackThreads, 0, st>>>(halo, hlen, H, seg, slen, R.hl, nwords, pieces, npieces,
                                                         mark, R.dir, R.exc, R.exc_cap, R.exc_n);
    if (launches) *launches += 1;
    return cudaGetLastError();
}

Batch make_batch(const RefBufs &R, uint64_t nbases, uint32_t halo, const DevPiece *pieces, uint32_t npieces) {
    Batch b;
    b.hl = R.hl;
    b.dir = R.dir;
    b.exc = R.exc;
    b.nbases = nbases;
    b.halo = halo;
    b.pieces = pieces;
    b.npieces = npieces;
    b.nwords = R.words_cap;
    b.ndir = R.words_cap ? dir_entries(R.words_cap) : 0;
    b.nexc = R.exc_cap;
    b.bounds = bounds_word();
    return b;
}

#ifdef IFA_BOUNDS_CHECK
namespace {
__device__ unsigned long long g_bounds_word;   // zero-initialised when the module loads
}

unsigned long long *bounds_word() {
    static unsigned long long *word[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    if (!word[dev & 63]) {
        void *a = nullptr;
        if (cudaGetSymbolAddress(&a, g_bounds_word) == cudaSuccess) word[dev & 63] = static_cast<unsigned long long *>(a);
        else (void)cudaGetLastError();
    }
    return word[dev & 63];
}
#else
unsigned long long *bounds_word() { return nullptr; }
#endif

cudaError_t launch_halo_update(const uint8_t *old_halo, uint32_t old_len, const uint8_t *seg,
                               uint64_t slen, uint32_t new_len, uint8_t *new_halo, cudaStream_t st) {
    if (new_len == 0) return cudaSuccess;
    k_halo_update<<<1, 256, 0, st>>>(old_halo, old_len, seg, slen, new_len, new_halo);
    return cudaGetLastError();
}

}  // namespace ifa

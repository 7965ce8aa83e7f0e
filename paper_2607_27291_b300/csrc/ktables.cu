// ktables.cu -- query k-mer tables of indexed mode, built on the device.
//
// Indexed mode looks every reference k-mer up among the query k-mers
// (Methods, indexed mode: seeds of length k taken every `step` bases of
// each query, both strands).  A table maps a k-mer key (planar hi/lo bits
// of its counted positions, the same key the seed scan forms from the
// reference) to the postings (entry << 8 | offset) that carry it:
//  - k <= 12: offsets addressed by the key directly (4^k + 1 words);
//  - k > 12: a presence bitmap of 4^k bits with a rank directory (per
//    32-bit bitmap word, the number of keys before it), and offsets
//    addressed by the key's rank among the present keys.
// Both are built from the posting list alone, with atomics and scans:
// count postings per key (or rank), scan the counts into the ends of the
// key ranges, then place every posting by decrementing its key's end
// (which leaves each key's start behind).  Posting order inside a key is
// therefore arbitrary; the seed scan does not depend on it.
#include "indexed.cuh"

namespace ifa {

namespace {

constexpr int kTThreads = 256;
constexpr int kTItems = 32;
constexpr uint64_t kTile = static_cast<uint64_t>(kTThreads) * kTItems;  // items per scanned tile

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t x, uint32_t lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= static_cast<uint32_t>(o)) x += y;
    }
    return x;
}

// Exclusive scan of one value per thread over the block; *total gets the sum.
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t *wsum, uint32_t *total) {
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    constexpr uint32_t nw = kTThreads / 32;
    const uint32_t x = warp_incl_scan(v, lane);
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
        const uint32_t w = lane < nw ? wsum[lane] : 0u;
        const uint32_t wi = warp_incl_scan(w, lane);
        if (lane < nw) wsum[lane] = wi;
    }
    __syncthreads();
    const uint32_t off = warp ? wsum[warp - 1] : 0u;
    *total = wsum[nw - 1];
    __syncthreads();
    return off + x - v;
}

template <bool POPC>
__device__ __forceinline__ uint32_t item(const uint32_t *in, uint64_t i, uint64_t n) {
    if (i >= n) return 0u;
    const uint32_t v = in[i];
    return POPC ? static_cast<uint32_t>(__popc(v)) : v;
}

// Phase 1: the sum of every tile.
template <bool POPC>
__global__ void __launch_bounds__(kTThreads) k_tile_sums(const uint32_t *__restrict__ in, uint64_t n,
                                                         uint32_t *__restrict__ sums) {
    __shared__ uint32_t wsum[kTThreads / 32];
    const uint64_t base = static_cast<uint64_t>(blockIdx.x) * kTile;
    uint32_t acc = 0;
#pragma unroll 4
    for (int i = 0; i < kTItems; i++) acc += item<POPC>(in, base + static_cast<uint64_t>(i) * kTThreads + threadIdx.x, n);
    uint32_t total;
    block_excl_scan(acc, wsum, &total);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

// Phase 2: exclusive scan of the nb tile sums, in one block (thread t takes
// a run of ceil(nb / threads) of them).
__global__ void __launch_bounds__(kTThreads) k_scan_sums(uint32_t *sums, uint32_t nb) {
    __shared__ uint32_t wsum[kTThreads / 32];
    const uint32_t per = (nb + kTThreads - 1) / kTThreads;
    const uint32_t first = threadIdx.x * per;
    const uint32_t last = first + per < nb ? first + per : nb;
    uint32_t acc = 0;
    for (uint32_t i = first; i < last; i++) acc += sums[i];
    uint32_t total;
    uint32_t run = block_excl_scan(acc, wsum, &total);
    for (uint32_t i = first; i < last; i++) {
        const uint32_t v = sums[i];
        sums[i] = run;
        run += v;
    }
}

// Phase 3: scan every tile (inclusive or exclusive) and add its offset.
// The tile passes through shared memory (padded by one word per 32 so that
// each thread's run of 32 consecutive items is free of bank conflicts), so
// global loads and stores stay coalesced.  `in` may equal `out` unless POPC.
template <bool POPC, bool EXCL>
__global__ void __launch_bounds__(kTThreads) k_tile_scan(const uint32_t *in, uint32_t *out, uint64_t n,
                                                         const uint32_t *__restrict__ sums) {
    __shared__ uint32_t t[kTile + kTile / 32];
    __shared__ uint32_t wsum[kTThreads / 32];
    const uint64_t base = static_cast<uint64_t>(blockIdx.x) * kTile;
    for (int i = 0; i < kTItems; i++) {
        const uint32_t j = static_cast<uint32_t>(i) * kTThreads + threadIdx.x;
        t[j + j / 32] = item<POPC>(in, base + j, n);
    }
    __syncthreads();
    const uint32_t first = threadIdx.x * kTItems;
    uint32_t acc = 0;
#pragma unroll 8
    for (int i = 0; i < kTItems; i++) acc += t[first + i + (first + i) / 32];
    uint32_t total;
    uint32_t run = block_excl_scan(acc, wsum, &total) + sums[blockIdx.x];
#pragma unroll 8
    for (int i = 0; i < kTItems; i++) {
        const uint32_t j = first + i + (first + i) / 32;
        const uint32_t v = t[j];
        t[j] = EXCL ? run : run + v;
        run += v;
    }
    __syncthreads();
    for (int i = 0; i < kTItems; i++) {
        const uint32_t j = static_cast<uint32_t>(i) * kTThreads + threadIdx.x;
        if (base + j < n) out[base + j] = t[j + j / 32];
    }
}

// Postings of `nents` entries for one table: warp w expands entry ents[w]
// into its offsets 0, step, ... (first[w + 1] - first[w] of them) and forms
// each k-mer's key from the entry's packed words (bit i = base i).
__global__ void k_postings(const uint4 *__restrict__ words, uint32_t wmax, const uint32_t *__restrict__ ents,
                           const uint32_t *__restrict__ first, uint32_t nents, uint32_t k, uint32_t care,
                           uint32_t step, uint32_t *__restrict__ keys, uint32_t *__restrict__ pv) {
    const uint32_t w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t lane = threadIdx.x & 31u;
    if (w >= nents) return;
    const uint32_t e = ents[w];
    const uint32_t base = first[w], cnt = first[w + 1] - base;
    const uint4 *qw = words + static_cast<size_t>(e) * wmax;
    for (uint32_t i = lane; i < cnt; i += 32) {
        const uint32_t o = i * step;
        const uint32_t wi = o >> 5, sh = o & 31u;
        const uint4 a = qw[wi];
        // the next word exists whenever the k-mer reaches into it (o + k <= L <= 32 wmax)
        const uint4 c = sh + k > 32u ? qw[wi + 1] : make_uint4(0u, 0u, 0u, 0u);
        const uint32_t hi = __funnelshift_r(a.x, c.x, sh), lo = __funnelshift_r(a.y, c.y, sh);
        keys[base + i] = ((hi & care) << k) | (lo & care);
        pv[base + i] = (e << 8) | o;
    }
}

__global__ void k_count(const uint32_t *__restrict__ keys, uint32_t np, uint32_t *__restrict__ off) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < np) atomicAdd(off + keys[i] + 2, 1u);
}

// Each posting carries its entry's meta word, so verification reads no
// second random word per candidate.
__global__ void k_place(const uint32_t *__restrict__ keys, const uint32_t *__restrict__ pv,
                        const uint32_t *__restrict__ meta, uint32_t np, uint32_t *__restrict__ off,
                        uint2 *__restrict__ post) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < np) post[atomicSub(off + keys[i] + 2, 1u) - 1u] = make_uint2(pv[i], meta[pv[i] >> 8]);
}

__global__ void k_set_bits(const uint32_t *__restrict__ keys, uint32_t np, uint32_t *__restrict__ bits) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < np) atomicOr(bits + (keys[i] >> 5), 1u << (keys[i] & 31u));
}

// keys -> their ranks among the present keys (in place)
__global__ void k_rank(uint32_t *__restrict__ keys, uint32_t np, const uint32_t *__restrict__ bits,
                       const uint32_t *__restrict__ rank) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np) return;
    const uint32_t key = keys[i], w = key >> 5;
    keys[i] = rank[w] + __popc(bits[w] & ((1u << (key & 31u)) - 1u));
}

unsigned grid_for(uint64_t n, int threads) { return static_cast<unsigned>((n + threads - 1) / threads); }

}  // namespace

uint64_t device_scan_sums_words(uint64_t n) { return (n + kTile - 1) / kTile; }

cudaError_t device_scan(const uint32_t *in, uint32_t *out, uint64_t n, bool popc, bool exclusive,
                        uint32_t *sums, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    const uint64_t nb = device_scan_sums_words(n);
    if (nb > 0x7fffffffull) return cudaErrorInvalidValue;
    const unsigned g = static_cast<unsigned>(nb);
    if (popc) k_tile_sums<true><<<g, kTThreads, 0, st>>>(in, n, sums);
    else k_tile_sums<false><<<g, kTThreads, 0, st>>>(in, n, sums);
    k_scan_sums<<<1, kTThreads, 0, st>>>(sums, g);
    if (popc && exclusive) k_tile_scan<true, true><<<g, kTThreads, 0, st>>>(in, out, n, sums);
    else if (popc) k_tile_scan<true, false><<<g, kTThreads, 0, st>>>(in, out, n, sums);
    else if (exclusive) k_tile_scan<false, true><<<g, kTThreads, 0, st>>>(in, out, n, sums);
    else k_tile_scan<false, false><<<g, kTThreads, 0, st>>>(in, out, n, sums);
    return cudaGetLastError();
}

cudaError_t launch_postings(const uint4 *words, uint32_t wmax, const uint32_t *ents, const uint32_t *first,
                            uint32_t nents, uint32_t k, uint32_t care, uint32_t step, uint32_t *keys,
                            uint32_t *pv, cudaStream_t st) {
    if (nents == 0) return cudaSuccess;
    k_postings<<<grid_for(static_cast<uint64_t>(nents) * 32, 256), 256, 0, st>>>(words, wmax, ents, first, nents,
                                                                                 k, care, step, keys, pv);
    return cudaGetLastError();
}

// Offsets and postings of one table from np (key, posting) pairs; meta:
// the query table's meta words, copied into each posting.
// off: 4^k + 3 words (direct) or np + 3 words (ranked); bits and rank:
// 4^k / 32 words each (ranked only); sums: device_scan_sums_words(largest
// scanned length) words.  Lookups then read offsets from off + 2.
cudaError_t build_table(uint32_t k, bool direct, uint32_t *keys, const uint32_t *pv, const uint32_t *meta, uint32_t np,
                        uint32_t *off, uint32_t *bits, uint32_t *rank, uint2 *post, uint32_t *sums, cudaStream_t st) {
    cudaError_t e = cudaSuccess;
    const uint64_t nkeys = 1ull << (2 * k);
    uint64_t noff;
    if (direct) {
        noff = nkeys + 3;
    } else {
        const uint64_t nw = nkeys / 32;
        e = cudaMemsetAsync(bits, 0, nw * sizeof(uint32_t), st);
        if (e == cudaSuccess && np) k_set_bits<<<grid_for(np, 256), 256, 0, st>>>(keys, np, bits);
        if (e == cudaSuccess) e = device_scan(bits, rank, nw, true, true, sums, st);
        if (e == cudaSuccess && np) k_rank<<<grid_for(np, 256), 256, 0, st>>>(keys, np, bits, rank);
        noff = static_cast<uint64_t>(np) + 3;
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(off, 0, noff * sizeof(uint32_t), st);
    if (e == cudaSuccess && np) k_count<<<grid_for(np, 256), 256, 0, st>>>(keys, np, off);
    if (e == cudaSuccess) e = device_scan(off, off, noff, false, false, sums, st);
    if (e == cudaSuccess && np) k_place<<<grid_for(np, 256), 256, 0, st>>>(keys, pv, meta, np, off, post);
    if (e == cudaSuccess) e = cudaGetLastError();
    return e;
}

}  // namespace ifa

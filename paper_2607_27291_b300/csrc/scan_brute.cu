// scan_brute.cu -- brute-force Hamming scan (Methods, "Algorithm Design",
// brute-force mode; "SIMD Optimization").
//
// The paper's CPU kernel broadcasts each query base against 32 consecutive
// reference positions and counts mismatches per lane, stopping early once
// every lane is over the threshold.  Here a warp owns 128 consecutive
// windows (four per lane) and compares 32-base words bit-parallel:
//   x  = ((R_hi ^ Q_hi) | (R_lo ^ Q_lo)) & care        one word, 32 bases
//   mm = nN + sum over words of popc(x)
// R_* is the lane's window word, cut from two packed words by a funnel
// shift; Q_* the query word (reverse complement precomputed) in shared
// memory.  The hi/lo words of the warp's next block and the two directory
// entries covering them are prefetched into a per-warp shared double buffer
// with cp.async while the current one is scanned.
//
// Early termination, batched: for maxSubs < 32 the first word alone
// rejects almost every window (E[mm] = 24 of 32 on random sequence), so
// the hot loop computes only word 0 for 4 entries x 4 windows, packs each
// entry's four counts into one word whose byte high bits say "over the
// threshold" (see packed_counts), and one warp vote per 4 entries decides
// whether the exact path (all words, hit emission) runs for any of them
// (then a vote per entry picks which).  Entries whose first word is fully
// counted and that hold no N ("class F") need no care mask, so a window
// costs 2 LOP3 + 1 POPC on the ALU/POPC pipes plus 1 IMAD on the FMA
// pipe -- the POPC pipe (16 lanes/clk/SM) is the binding unit.  Other
// entries ("class M") also AND a care mask and use the threshold
// maxSubs - nN.
//
// Blocks of windows that touch a special word (an N or a contig-piece
// start), the batch end or the halo take a generic path that rebuilds the N
// and piece-start planes and checks each window stays inside one piece and
// is owned by this batch.
//
// Deferred hits (streaming, indexed mode's exhaustive entries, the rate
// measurement): the scan writes each window event (entry, lane, block, the
// windows' counts and hit bits) straight to a device event buffer, and a
// second kernel expands the events into hits -- piece lookup, query id,
// digest, one ring claim per warp range, per-entry counts.  The scan loop
// then holds none of that code, which alone made the hot loop 3 % slower
// at maxSubs 0 where hits are rare, and the expansion of dense hits
// (maxSubs 16: 8e7 hits per 4 Gbp pass) runs converged in its own kernel.
// A launch whose events overflow the buffer is scanned again by the
// second kernel with the hits expanded in the loop.  That one-kernel form
// (k_scan_brute) also serves the callers without an event buffer: the
// per-set batch baseline and the allocation-free entry point; the
// persistent batch kernel expands in its loop the same way.
#include "scan_brute.cuh"

namespace ifa {

namespace {

using namespace brute;

// Resident CTAs per SM the register allocation must allow: 4 (64 registers)
// fits queries up to 128 bases without spilling; the 256-base build needs 96
// registers and gets 2.
#ifndef IFA_SCAN_MIN_CTAS
#define IFA_SCAN_MIN_CTAS 4
#endif
template <int WMAX>
constexpr int kScanMinCtas = WMAX <= 4 ? IFA_SCAN_MIN_CTAS : (IFA_SCAN_MIN_CTAS > 2 ? 2 : IFA_SCAN_MIN_CTAS);

// The scan with hits expanded in the loop: this warp's blocks, hits staged
// and flushed per warp, then the per-entry counts.
template <int WMAX>
__device__ __forceinline__ void scan_inline(const Batch &b, const QueryTable &qt, uint32_t e0, uint32_t e1,
                                            uint32_t s, uint32_t lmin, uint32_t lmax, const HitSink &sink,
                                            uint4 *smem4, ifa_hit (*wbuf)[32],
                                            uint2 (*stage)[2][Stage<WMAX>::kSlots], uint16_t (*cq)[kQRows][32],
                                            uint32_t *s_nF, uint32_t *s_nM) {
    const uint32_t nent = e1 - e0;
    const Smem m = load_chunk<WMAX>(qt, e0, e1, s, smem4, s_nF, s_nM);
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t warp = threadIdx.x >> 5;
    WarpHits wh;
    wh.init(wbuf[warp]);
    uint32_t mul[kWin];
    lane_multipliers(mul);
    const uint64_t nblk = (b.nbases + 32 * kWin - 1) / (32 * kWin);
    scan_blocks<WMAX>(b, qt, m, nent, *s_nF, *s_nM, e0, s, lmin, lmax, sink, wh, stage[warp], mul, 0, nblk,
                      blockIdx.x * kScanWarps + warp, gridDim.x * kScanWarps, lane, cq[warp]);
    wh.finish(sink, lane);
    __syncthreads();
    flush_counts(qt, m, nent, e0, sink);
}

// One kernel, hits expanded in the loop.
template <int WMAX>
__global__ void __launch_bounds__(kScanThreads, kScanMinCtas<WMAX>)
k_scan_brute(Batch b, QueryTable qt, uint32_t e0, uint32_t e1, uint32_t s, uint32_t lmin,
             uint32_t lmax, HitSink sink) {
    extern __shared__ uint4 smem4[];
    __shared__ __align__(16) ifa_hit wbuf[kScanWarps][32];
    __shared__ __align__(8) uint2 stage[kScanWarps][2][Stage<WMAX>::kSlots];
    __shared__ uint16_t cq[kScanWarps][kQRows][32];
    __shared__ uint32_t s_nF, s_nM;
    scan_inline<WMAX>(b, qt, e0, e1, s, lmin, lmax, sink, smem4, wbuf, stage, cq, &s_nF, &s_nM);
}

// Deferred hits, first kernel: the same scan, each window event written to
// the event buffer (WarpEvents).  Nothing is counted here.
template <int WMAX>
__global__ void __launch_bounds__(kScanThreads, kScanMinCtas<WMAX>)
k_scan_brute_events(Batch b, QueryTable qt, uint32_t e0, uint32_t e1, uint32_t s, uint32_t lmin,
                    uint32_t lmax, HitSink sink, EventSink es) {
    extern __shared__ uint4 smem4[];
    __shared__ __align__(8) uint2 stage[kScanWarps][2][Stage<WMAX>::kSlots];
    __shared__ uint16_t cq[kScanWarps][kQRows][32];
    __shared__ uint32_t s_nF, s_nM;
    const uint32_t nent = e1 - e0;
    const Smem m = load_chunk<WMAX>(qt, e0, e1, s, smem4, &s_nF, &s_nM);
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t warp = threadIdx.x >> 5;
    WarpEvents we;
    we.init(es);
    uint32_t mul[kWin];
    lane_multipliers(mul);
    const uint64_t nblk = (b.nbases + 32 * kWin - 1) / (32 * kWin);
    scan_blocks<WMAX>(b, qt, m, nent, s_nF, s_nM, e0, s, lmin, lmax, sink, we, stage[warp], mul, 0, nblk,
                      blockIdx.x * kScanWarps + warp, gridDim.x * kScanWarps, lane, cq[warp]);
}

// Deferred hits, second kernel (same grid and shared memory).  When every
// event fit: warp w takes a contiguous range of event records, counts its
// hits (one bit per window in each record's mask), claims ring slots for
// all of them with one atomic, then expands 32 records per step -- lane i
// record i, its slots at the lane's prefix offset -- into hits: piece,
// query id, digest terms, ring store, per-entry count.  Empty records
// (unused chunk slots) carry no window bit.  When some did not fit: the
// range is scanned again with the hits expanded in line.
template <int WMAX>
__global__ void __launch_bounds__(kScanThreads, kScanMinCtas<WMAX>)
k_expand_events(Batch b, QueryTable qt, uint32_t e0, uint32_t e1, uint32_t s, uint32_t lmin,
                uint32_t lmax, HitSink sink, EventSink es) {
    extern __shared__ uint4 smem4[];
    __shared__ __align__(16) ifa_hit wbuf[kScanWarps][32];
    __shared__ __align__(8) uint2 stage[kScanWarps][2][Stage<WMAX>::kSlots];
    __shared__ uint16_t cq[kScanWarps][kQRows][32];
    __shared__ uint32_t s_nF, s_nM;
    const unsigned long long nev = *es.head;
    if (nev > es.cap) {
        scan_inline<WMAX>(b, qt, e0, e1, s, lmin, lmax, sink, smem4, wbuf, stage, cq, &s_nF, &s_nM);
        return;
    }
    const uint32_t nent = e1 - e0;
    uint32_t *cnt = reinterpret_cast<uint32_t *>(smem4);   // nent counters (the chunk's smem is larger)
    for (uint32_t i = threadIdx.x; i < nent; i += blockDim.x) cnt[i] = 0;
    __syncthreads();
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t warp = threadIdx.x >> 5;
    const unsigned long long nw = static_cast<unsigned long long>(gridDim.x) * kScanWarps;
    const unsigned long long per = ((nev + nw - 1) / nw + 31) / 32 * 32;
    const unsigned long long a = min(nev, (static_cast<unsigned long long>(blockIdx.x) * kScanWarps + warp) * per);
    const unsigned long long z = min(nev, a + per);
    unsigned long long dcount = 0, dsum = 0, dxor = 0;
    if (a < z) {
        uint32_t tot = 0;
        for (unsigned long long i = a + lane; i < z; i += 32) tot += __popc(es.buf[i].w & 0x80808080u);
        tot = __reduce_add_sync(0xffffffffu, tot);
        // one claim for the range (as the warp staging claims per flush)
        unsigned long long base = 0, pos = 0, room = 0;
        if (!sink.count_only && lane == 0 && tot) {
            base = atomicAdd(sink.head, static_cast<unsigned long long>(tot));
            const Claim c = claim_room(sink, base);
            pos = c.pos;
            room = c.room;
        }
        base = __shfl_sync(0xffffffffu, base, 0);
        pos = __shfl_sync(0xffffffffu, pos, 0);
        room = __shfl_sync(0xffffffffu, room, 0);
        if (!sink.count_only && tot && room < tot && lane == 0) drop_claim(sink, base + room);
        uint32_t off0 = 0;          // claims used by earlier steps (warp-uniform)
        uint32_t pidx = 0xffffffffu;
        for (unsigned long long i0 = a; i0 < z; i0 += 32) {
            uint4 ev = make_uint4(0u, 0u, 0u, 0u);
            if (i0 + lane < z) ev = es.buf[i0 + lane];
            uint32_t hm = ev.w & 0x80808080u;
            const uint32_t nh = __popc(hm);
            uint32_t inc = nh;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= static_cast<uint32_t>(o)) inc += y;
            }
            uint32_t off = off0 + inc - nh;
            off0 += __shfl_sync(0xffffffffu, inc, 31);
            if (!nh) continue;
            const uint32_t e = ev.x & 0xffffu, el = ev.x >> 16;
            const uint32_t id = qt.ids ? qt.ids[e0 + e] : e0 + e;
            const uint32_t q = id >> 1, strand = id & 1u;
            atomicAdd(cnt + e, nh);
            const uint64_t p0 = static_cast<uint64_t>(ev.z) * kEventBlock + el;
            unsigned long long at = pos + off;
            if (!sink.count_only && at >= sink.capacity) at %= sink.capacity;
            while (hm) {
                const uint32_t bit = static_cast<uint32_t>(__ffs(hm) - 1);  // 8 k + 7 for window k
                hm &= hm - 1u;
                const uint64_t p = p0 + 4u * (bit - 7u);                     // = p0 + 32 k
                pidx = find_piece_from(b.pieces, b.npieces, p, pidx);
                const DevPiece pc = b.pieces[pidx];
                const uint32_t hpos = static_cast<uint32_t>(pc.contig_off + (p - pc.start));
                const uint32_t mm = (ev.y >> (bit - 7u)) & 0xffu;
                const uint64_t v = hit_digest_item(q, pc.contig, hpos, strand, mm);
                dcount += 1;
                dsum += v;
                dxor ^= v;
                if (!sink.count_only) {
                    if (off < room) {
                        ifa_hit h;
                        h.query = q;
                        h.contig = pc.contig;
                        h.pos = hpos;
                        h.strand = static_cast<uint8_t>(strand);
                        h.mismatches = static_cast<uint8_t>(mm);
                        h.clips = 0;
                        sink.ring[at] = h;
                    }
                    off++;
                    if (++at == sink.capacity) at = 0;
                }
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        dcount += __shfl_xor_sync(0xffffffffu, dcount, o);
        dsum += __shfl_xor_sync(0xffffffffu, dsum, o);
        dxor ^= __shfl_xor_sync(0xffffffffu, dxor, o);
    }
    if (lane == 0 && dcount) {
        atomicAdd(&sink.digest[0], dcount);
        atomicAdd(&sink.digest[1], dsum);
        atomicXor(&sink.digest[2], dxor);
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < nent; i += blockDim.x)
        if (cnt[i]) {
            const uint32_t id = qt.ids ? qt.ids[e0 + i] : e0 + i;
            atomicAdd(&sink.qcount[id >> 1], static_cast<unsigned long long>(cnt[i]));
        }
}

template <int WMAX>
cudaError_t launch_t(const Batch &b, const QueryTable &qt, uint32_t e0, uint32_t e1, uint32_t s,
                     uint32_t lmin, uint32_t lmax, const HitSink &sink, cudaStream_t st, const EventSink *es) {
    const size_t smem = static_cast<size_t>(e1 - e0) * entry_smem(WMAX);
    static int grids[64] = {0};  // per device and template instance: SMs x resident CTAs
    int dev = 0;
    cudaGetDevice(&dev);
    int &grid = grids[dev & 63];
    if (grid == 0) {
        int sms = 0, per_sm = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_scan_brute<WMAX>, kScanThreads,
                                                      kScanSmemBudget);
        grid = sms * (per_sm > 0 ? per_sm : 1);
    }
    const uint64_t nblk = (b.nbases + 32 * kWin - 1) / (32 * kWin);
    const uint64_t need = (nblk + kScanWarps - 1) / kScanWarps;
    int g = static_cast<int>(need < static_cast<uint64_t>(grid) ? need : grid);
    if (g < 1) g = 1;
    if (!es) {
        k_scan_brute<WMAX><<<g, kScanThreads, smem, st>>>(b, qt, e0, e1, s, lmin, lmax, sink);
        return cudaGetLastError();
    }
    cudaError_t e = cudaMemsetAsync(es->head, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    k_scan_brute_events<WMAX><<<g, kScanThreads, smem, st>>>(b, qt, e0, e1, s, lmin, lmax, sink, *es);
    k_expand_events<WMAX><<<g, kScanThreads, smem, st>>>(b, qt, e0, e1, s, lmin, lmax, sink, *es);
    return cudaGetLastError();
}

}  // namespace

uint32_t scan_brute_chunk_entries(uint32_t wmax) {
    const uint32_t n = chunk_cap(static_cast<int>(wmax));
    return n < 65535u ? n : 65535u;
}

cudaError_t launch_scan_brute(const Batch &b, const QueryTable &qt, uint32_t e0, uint32_t e1,
                              uint32_t max_subs, uint32_t lmin, uint32_t lmax, const HitSink &sink,
                              cudaStream_t st, int *launches, const EventSink *es) {
    if (e1 <= e0 || b.nbases == 0) return cudaSuccess;
    if (launches) *launches += es ? 2 : 1;
    switch (qt.wmax) {
    case 1: return launch_t<1>(b, qt, e0, e1, max_subs, lmin, lmax, sink, st, es);
    case 2: return launch_t<2>(b, qt, e0, e1, max_subs, lmin, lmax, sink, st, es);
    case 4: return launch_t<4>(b, qt, e0, e1, max_subs, lmin, lmax, sink, st, es);
    case 8: return launch_t<8>(b, qt, e0, e1, max_subs, lmin, lmax, sink, st, es);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace ifa

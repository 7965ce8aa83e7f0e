// scan_brute.cuh -- device code of the brute-force scan, shared by the
// streaming kernel (scan_brute.cu) and the persistent multi-set kernel
// (batch.cu).
//
//
// The paper's CPU kernel broadcasts each query base against 32 consecutive
// reference positions and counts mismatches per lane, stopping early once
// every lane is over the threshold.  Here a warp owns 128 consecutive
// windows (four per lane) and compares 32-base words bit-parallel:
//   x  = ((R_hi ^ Q_hi) | (R_lo ^ Q_lo)) & care        one word, 32 bases
//   mm = nN + sum over words of popc(x)
// R_* is the lane's window word, cut from two packed words by a funnel
// shift; Q_* the query word (reverse complement precomputed) in shared
// memory.  The hi/lo words of the warp's next block (8 bytes per 32 bases)
// and the two directory entries that cover them are prefetched into a
// per-warp shared double buffer with cp.async while the current one is
// scanned.
//
// Early termination, batched: for maxSubs < 32 the first word alone
// rejects almost every window (E[mm] = 24 of 32 on random sequence), so
// the hot loop computes only word 0 for 4 entries x 4 windows, packs each
// entry's four counts into one word whose byte high bits say "over the
// threshold" (see packed_counts), and one warp vote per 4 entries decides
// whether any of them passed.  Entries that passed in a lane wait in that
// lane's column of a small shared queue until the block ends; then every
// lane recounts its own candidates (all words, hit events) at once
// (drain_queue).  Entries whose first word is fully
// counted and that hold no N ("class F") need no care mask, so a window
// costs 2 LOP3 + 1 POPC on the ALU/POPC pipes plus 1 IMAD on the FMA
// pipe -- the POPC pipe (16 lanes/clk/SM) is the binding unit.  Other
// entries ("class M") also AND a care mask and use the threshold
// maxSubs - nN.
//
// Blocks of windows that touch a special word (an N or a contig-piece
// start, per the directory), the batch end or the halo take a generic path
// that rebuilds the N and piece-start planes (ref_word) and checks each
// window stays inside one piece and is owned by this batch.
#pragma once
#include "hits.cuh"

namespace ifa {
namespace brute {


constexpr int kScanThreads = 256;
constexpr int kScanWarps = kScanThreads / kWarp;
#ifndef IFA_SCAN_GROUP
#define IFA_SCAN_GROUP 4
#endif
constexpr int kGroup = IFA_SCAN_GROUP;          // entries per warp vote in the hot loop
constexpr int kWin = 4;                         // windows per lane (32 * kWin per warp step)
// Candidate queue (per warp, one column per lane): entries whose word 0
// passes in a lane wait there as 16-bit record indices until the block ends
// (or a column is nearly full), then every lane recounts its own candidates
// at once.  0 = the warp-wide exact path per fired entry instead.
#ifndef IFA_SCAN_QUEUE
#define IFA_SCAN_QUEUE 8
#endif
constexpr int kQDepth = IFA_SCAN_QUEUE;
constexpr uint32_t kQClassM = 0x8000u;          // queued index of a class-M record
static_assert(kQDepth == 0 || kQDepth >= kGroup, "a queue column holds at least one group");
constexpr int kQRows = kQDepth > 0 ? kQDepth : 1;  // shared rows per warp

// Static shared memory of a scan kernel (streaming or persistent, 8 warps)
// at the widest entries: hit staging, word staging (kWin + 8 words and two
// directory entries, double buffered), the candidate queue, a few counters.
// The dynamic query chunk gets the rest of 48 KB, whole kilobytes.
constexpr size_t kScanStaticSmem = kScanWarps * (32 * 16 + 2 * (kWin + 8 + 2) * 8 + kQRows * 32 * 2) + 64;
constexpr size_t kScanSmemBudget = (48 * 1024 - kScanStaticSmem) / 1024 * 1024;

// Per-entry shared memory: WMAX uint4 words, a class-M word-0 record, a
// class-F word-0 record, meta, count, and two 16-bit index slots.
__host__ __device__ constexpr size_t entry_smem(int wmax) {
    return wmax * sizeof(uint4) + 2 * sizeof(uint4) + 2 * sizeof(uint32_t) + 2 * sizeof(uint16_t);
}

// The most entries of one chunk that fit the shared-memory budget.
__host__ __device__ constexpr uint32_t chunk_cap(int wmax) {
    return static_cast<uint32_t>(kScanSmemBudget / entry_smem(wmax));
}

struct Smem {
    uint4 *sq;         // entries x WMAX full words
    uint4 *sM;         // class M: {hi0, lo0, care0, threshold}
    uint4 *sF;         // class F: {hi0, lo0, threshold, 0}
    uint32_t *meta;
    uint32_t *cnt;
    uint16_t *fidx;
    uint16_t *midx;
};

__device__ inline Smem carve(uint4 *base, uint32_t nent, int wmax) {
    Smem m;
    m.sq = base;
    m.sM = m.sq + static_cast<size_t>(nent) * wmax;
    m.sF = m.sM + nent;
    m.meta = reinterpret_cast<uint32_t *>(m.sF + nent);
    m.cnt = m.meta + nent;
    m.fidx = reinterpret_cast<uint16_t *>(m.cnt + nent);
    m.midx = m.fidx + nent;
    return m;
}

// Words of a block are staged per warp in shared memory; a block is
// WIN x 32 windows: lane l owns windows p0 + 32 k + l, k < WIN, and window
// k's word j is cut from staged words k + j, k + j + 1.  After the kWords
// hi/lo words come the directory entries of their group and the next.
template <int WMAX>
struct Stage {
    static constexpr int kWords = kWin + WMAX;  // staged hi/lo words per block
    static constexpr int kSlots = kWords + 2;   // + two directory entries
};

// Generic evaluation of every entry for one window per lane (p = p0 + lane)
// whose block may hold N, piece boundaries, the batch end or the halo.
template <int WMAX, class WH>
__device__ void generic_window(const Batch &b, const QueryTable &qt, const Smem &m, uint32_t nent,
                               uint32_t e0, uint64_t p0, uint32_t lane, uint32_t s,
                               const HitSink &sink, WH &wh) {
    const uint64_t w0 = p0 >> 5;
    uint32_t hi[WMAX], lo[WMAX], nw[WMAX], bw[WMAX];
    uint4 cur = ref_word(b, w0);
#pragma unroll
    for (int j = 0; j < WMAX; j++) {
        const uint4 nx = ref_word(b, w0 + j + 1);
        hi[j] = __funnelshift_r(cur.x, nx.x, lane);
        lo[j] = __funnelshift_r(cur.y, nx.y, lane);
        nw[j] = __funnelshift_r(cur.z, nx.z, lane);
        bw[j] = __funnelshift_r(cur.w, nx.w, lane);
        cur = nx;
    }
    bw[0] &= ~1u;  // a piece may start at the window's first base
    const uint64_t p = p0 + lane;
    for (uint32_t e = 0; e < nent; e++) {
        const uint32_t meta = m.meta[e];
        const uint32_t L = meta_L(meta);
        const uint32_t W = meta_W(meta);
        const uint4 *qw = m.sq + static_cast<size_t>(e) * WMAX;
        uint32_t mm = meta_nN(meta);
        uint32_t bnd = 0;
#pragma unroll
        for (int j = 0; j < WMAX; j++) {
            if (j < static_cast<int>(W)) {
                const uint4 q = qw[j];
                mm += __popc(((hi[j] ^ q.x) | (lo[j] ^ q.y) | nw[j]) & q.z);
                bnd |= bw[j] & q.w;
            }
        }
        const bool valid = (p + L <= b.nbases) && (p + L >= static_cast<uint64_t>(b.halo) + 1) && bnd == 0u;
        const bool hit = valid && mm <= entry_s(meta, s);
        // this call's window is window k of block p0 / 128 (mm <= 255 fits a byte)
        const uint32_t k = static_cast<uint32_t>(p0 >> 5) & (kWin - 1);
        wh.event(b, qt.ids, e0, m.cnt, sink, lane, hit, e, mm << (8 * k), static_cast<uint32_t>(p0 / (32 * kWin)),
                 hit ? 0x80u << (8 * k) : 0u);
    }
}

// Byte-lane threshold test.  The four windows' word-0 counts p_k (<= 32)
// are packed as v = C + p0 + p1 << 8 + p2 << 16 + p3 << 24 with
// C = 0x80808080 - (T + 1) * 0x01010101 for the entry's threshold T in
// [-1, 127]: byte k is 128 - (T + 1) + p_k, in [0, 160], so no carry crosses
// bytes and its high bit is clear exactly when p_k <= T.  The packing runs
// as IMADs on the FMA pipe (multipliers held in registers), keeping the ALU
// pipe for the two LOP3 per window.
__host__ __device__ inline uint32_t byte_bias(int T) {
    if (T < -1) T = -1;
    if (T > 127) T = 127;
    return 0x80808080u - static_cast<uint32_t>(T + 1) * 0x01010101u;
}

__device__ __forceinline__ uint32_t mad(uint32_t a, uint32_t b, uint32_t c) {
    uint32_t d;
    asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}

// Exact evaluation of one entry for the lane's kWin windows of a block
// without N, piece boundary or ownership limits, then one hit event per
// lane.  Counts stay packed one byte per window.  Word j of window k is word
// 0 of window k + j, so it is taken from the hot loop's registers where
// k + j < kWin and cut from the staged words otherwise.
//  - Queries of up to 64 bases (WMAX <= 2): word-1 counts are added straight
//    onto v, whose bytes are 128 - (T + 1) + count for the word-0 threshold
//    T (see packed_counts).  T already is the whole window's threshold
//    (maxSubs less the query's Ns), and a byte stays below 256 (count <= 64),
//    so a byte's high bit is clear exactly when its window hits.
//  - Longer queries: d = v - bias holds the counts themselves, the Ns are
//    added to every byte, then words 1.. by IMAD, and d is tested against
//    maxSubs.  No byte can carry: a count is at most the query length.
template <int WMAX, class WH>
__device__ __forceinline__ void exact_fast(const Batch &b, const QueryTable &qt, const Smem &m,
                                           const uint2 *R, const uint32_t *hw, const uint32_t *lw,
                                           const uint32_t *mul, uint32_t e, uint32_t e0, uint32_t blk,
                                           uint32_t lane, uint32_t s, const HitSink &sink, WH &wh, uint32_t v,
                                           uint32_t bias, bool act = true) {
    const uint32_t meta = m.meta[e];
    const uint4 *qw = m.sq + static_cast<size_t>(e) * WMAX;
    uint32_t hm, d;
    if constexpr (WMAX <= 2) {
        uint32_t vf = v;
        if (WMAX == 2 && meta_W(meta) > 1u) {
            const uint4 q = qw[WMAX - 1];
#pragma unroll
            for (int k = 0; k < kWin; k++) {
                uint32_t h, l;
                if (k + 1 < kWin) {
                    h = hw[k + 1];
                    l = lw[k + 1];
                } else {
                    const uint2 a = R[k + 1], c = R[k + 2];
                    h = __funnelshift_r(a.x, c.x, lane);
                    l = __funnelshift_r(a.y, c.y, lane);
                }
                vf = mad(__popc(((h ^ q.x) | (l ^ q.y)) & q.z), mul[k], vf);
            }
        }
        hm = ~vf & 0x80808080u;
        d = vf - bias + meta_nN(meta) * 0x01010101u;
    } else {
        const uint32_t W = meta_W(meta);
        const uint32_t se = entry_s(meta, s);
        d = v - bias + meta_nN(meta) * 0x01010101u;
#pragma unroll
        for (int j = 1; j < WMAX; j++) {
            if (j < static_cast<int>(W)) {
                const uint4 q = qw[j];
#pragma unroll
                for (int k = 0; k < kWin; k++) {
                    uint32_t h, l;
                    if (k + j < kWin) {
                        h = hw[k + j];
                        l = lw[k + j];
                    } else {
                        const uint2 a = R[k + j], c = R[k + j + 1];
                        h = __funnelshift_r(a.x, c.x, lane);
                        l = __funnelshift_r(a.y, c.y, lane);
                    }
                    d = mad(__popc(((h ^ q.x) | (l ^ q.y)) & q.z), mul[k], d);
                }
            }
        }
        if constexpr (WMAX <= 4) {
            // counts <= 128 (queries up to 128 bases), so for se <= 127 the
            // byte-lane test applies (128 - (se + 1) + count stays below 256);
            // se >= 128 passes every window
            hm = se >= 128u ? 0x80808080u : ~(d + byte_bias(static_cast<int>(se))) & 0x80808080u;
        } else {
            hm = 0;
#pragma unroll
            for (int k = 0; k < kWin; k++) hm |= (((d >> (8 * k)) & 0xffu) <= se ? 0x80u : 0u) << (8 * k);
        }
    }
    wh.event(b, qt.ids, e0, m.cnt, sink, lane, act && hm != 0u, e, d, blk, hm);
}

// Entry word-0 records: {hi0, lo0, bias, -} (class F) or
// {hi0, lo0, care0, bias} (class M, MASKED).
template <bool MASKED>
__device__ __forceinline__ uint32_t packed_counts(const uint4 &q, const uint32_t *hw, const uint32_t *lw,
                                                  const uint32_t *mul) {
    uint32_t p[kWin];
#pragma unroll
    for (int w = 0; w < kWin; w++) {
        uint32_t x = (hw[w] ^ q.x) | (lw[w] ^ q.y);
        if (MASKED) x &= q.z;
        p[w] = __popc(x);
    }
    uint32_t v = (MASKED ? q.w : q.z) + p[0];
#pragma unroll
    for (int w = 1; w < kWin; w++) v = mad(p[w], mul[w], v);
    return v;
}

// Recount the queued candidates of the lane's windows in this block: row r
// of every column at once, each lane its own (entry, class), then one event
// per lane.  Leaves the queue empty (all lanes, warp converged).
template <int WMAX, class WH>
__device__ __forceinline__ void drain_queue(const Batch &b, const QueryTable &qt, const Smem &m, uint16_t (*cq)[32],
                                            uint32_t &qn, const uint32_t *hw, const uint32_t *lw,
                                            const uint32_t *mul, const uint2 *R, uint32_t e0, uint32_t blk,
                                            uint32_t lane, uint32_t s, const HitSink &sink, WH &wh) {
    const uint32_t rows = __reduce_max_sync(0xffffffffu, qn);
#pragma unroll 1
    for (uint32_t r = 0; r < rows; r++) {
        // a lane without an r-th candidate reads no record (a class may be
        // empty) and runs the path on entry 0 of the chunk, emitting nothing
        const bool act = r < qn;
        uint4 q = make_uint4(0u, 0u, 0u, 0u);
        uint32_t e = 0, bias = 0, care = 0;
        if (act) {
            const uint32_t c = cq[r][lane];
            const uint32_t k = c & (kQClassM - 1u);
            if (c & kQClassM) {
                q = m.sM[k];   // {hi0, lo0, care0, bias}
                e = m.midx[k];
                care = q.z;
                bias = q.w;
            } else {
                q = m.sF[k];   // {hi0, lo0, bias, -}: care all ones
                e = m.fidx[k];
                care = 0xffffffffu;
                bias = q.z;
            }
        }
        const uint32_t v = packed_counts<true>(make_uint4(q.x, q.y, care, bias), hw, lw, mul);
        exact_fast<WMAX>(b, qt, m, R, hw, lw, mul, e, e0, blk, lane, s, sink, wh, v, bias, act);
    }
    qn = 0;
}

template <int WMAX, bool MASKED, class WH>
__device__ __forceinline__ void scan_class(const Batch &b, const QueryTable &qt, const Smem &m,
                                           const uint4 *rec, const uint16_t *idx, uint32_t n,
                                           const uint32_t *hw, const uint32_t *lw, const uint32_t *mul,
                                           const uint2 *R, uint32_t e0, uint32_t blk, uint32_t lane,
                                           uint32_t s, const HitSink &sink, WH &wh, uint16_t (*cq)[32],
                                           uint32_t &qn, bool &queued) {
    constexpr uint32_t kHigh = 0x80808080u;
    constexpr uint32_t cls = MASKED ? kQClassM : 0u;
    uint32_t k = 0;
    for (; k + kGroup <= n; k += kGroup) {
        uint32_t v[kGroup];
#pragma unroll
        for (int i = 0; i < kGroup; i++) v[i] = packed_counts<MASKED>(rec[k + i], hw, lw, mul);
        uint32_t acc = v[0];
#pragma unroll
        for (int i = 1; i < kGroup; i++) acc &= v[i];
        if constexpr (kQDepth > 0) {
            if (__any_sync(0xffffffffu, (acc & kHigh) != kHigh)) {
                // queue the lane's passing entries; drain while a column
                // could not take another group
                queued = true;   // warp-uniform: the block ends with a drain
#pragma unroll
                for (int i = 0; i < kGroup; i++)
                    if ((v[i] & kHigh) != kHigh) cq[qn++][lane] = static_cast<uint16_t>((k + i) | cls);
                if (__any_sync(0xffffffffu, qn > static_cast<uint32_t>(kQDepth - kGroup)))
                    drain_queue<WMAX>(b, qt, m, cq, qn, hw, lw, mul, R, e0, blk, lane, s, sink, wh);
            }
        } else if (__any_sync(0xffffffffu, (acc & kHigh) != kHigh)) {
            // which of the group's entries fired in any lane; one (not
            // unrolled) copy of the exact path walks them
            uint32_t fired = 0;
#pragma unroll
            for (int i = 0; i < kGroup; i++) fired |= ((v[i] & kHigh) != kHigh ? 1u : 0u) << i;
            fired = __reduce_or_sync(0xffffffffu, fired);
#pragma unroll 1
            while (fired) {
                const int i = __ffs(fired) - 1;
                fired &= fired - 1;
                // v[i] by a select chain (no local array); the bias from the record
                uint32_t vi = v[0];
#pragma unroll
                for (int t = 1; t < kGroup; t++) vi = i == t ? v[t] : vi;
                const uint4 q = rec[k + i];
                exact_fast<WMAX>(b, qt, m, R, hw, lw, mul, idx[k + i], e0, blk, lane, s, sink, wh, vi,
                                 MASKED ? q.w : q.z);
            }
        }
    }
    for (; k < n; k++) {
        const uint4 q = rec[k];
        const uint32_t v = packed_counts<MASKED>(q, hw, lw, mul);
        if (__any_sync(0xffffffffu, (v & kHigh) != kHigh)) {
            if constexpr (kQDepth > 0) {
                queued = true;
                if ((v & kHigh) != kHigh) cq[qn++][lane] = static_cast<uint16_t>(k | cls);
                if (__any_sync(0xffffffffu, qn > static_cast<uint32_t>(kQDepth - kGroup)))
                    drain_queue<WMAX>(b, qt, m, cq, qn, hw, lw, mul, R, e0, blk, lane, s, sink, wh);
            } else {
                exact_fast<WMAX>(b, qt, m, R, hw, lw, mul, idx[k], e0, blk, lane, s, sink, wh, v,
                                 MASKED ? q.w : q.z);
            }
        }
    }
}

// Stage block `blk` into `dst` (shared) with cp.async: lane i < NW copies
// hi/lo word blk * kWin + i (8 bytes), lanes NW and NW + 1 the directory
// entries of that word's group and the next.
template <int NW>
__device__ __forceinline__ void stage_block(const Batch &b, uint64_t blk, uint2 *dst, uint32_t lane) {
    if (lane < NW + 2) {
        const uint64_t i = lane < NW ? blk * kWin + lane : ((blk * kWin) >> 5) + (lane - NW);
        if (lane < NW ? in_range(b, kBoundsWord, i, b.nwords) : in_range(b, kBoundsDir, i, b.ndir)) {
            const uint2 *src = lane < NW ? b.hl + i : b.dir + i;
            const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(dst + lane));
            asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
        } else {
            // out of range (checked builds): a directory entry marking every
            // word special sends the block down the generic path
            dst[lane] = make_uint2(lane < NW ? 0u : 0xffffffffu, 0u);
        }
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}

// Load entries [e0, e1) of the table into shared memory and split them into
// class F and class M (all threads of the CTA; ends with a barrier).
template <int WMAX>
__device__ __forceinline__ Smem load_chunk(const QueryTable &qt, uint32_t e0, uint32_t e1, uint32_t s,
                                           uint4 *smem_base, uint32_t *s_nF, uint32_t *s_nM) {
    const uint32_t nent = e1 - e0;
    const Smem m = carve(smem_base, nent, WMAX);
    for (uint32_t i = threadIdx.x; i < nent * WMAX; i += blockDim.x)
        m.sq[i] = qt.words[static_cast<size_t>(e0) * WMAX + i];
    for (uint32_t i = threadIdx.x; i < nent; i += blockDim.x) {
        m.meta[i] = qt.meta[e0 + i];
        m.cnt[i] = 0;
    }
    __syncthreads();
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t warp = threadIdx.x >> 5;
    if (warp == 0) {
        // split entries into class F (word 0 fully counted, no N) and class M
        uint32_t nF = 0, nM = 0;
        for (uint32_t base = 0; base < nent; base += 32) {
            const uint32_t e = base + lane;
            bool isF = false, isM = false;
            uint4 w0 = make_uint4(0, 0, 0, 0);
            uint32_t meta = 0;
            if (e < nent) {
                meta = m.meta[e];
                w0 = m.sq[static_cast<size_t>(e) * WMAX];
                isF = meta_nN(meta) == 0u && w0.z == 0xffffffffu;
                isM = !isF;
            }
            const uint32_t se = entry_s(meta, s);
            const uint32_t bf = __ballot_sync(0xffffffffu, isF);
            const uint32_t bm = __ballot_sync(0xffffffffu, isM);
            const uint32_t below = (1u << lane) - 1u;
            if (isF) {
                const uint32_t k = nF + __popc(bf & below);
                m.sF[k] = make_uint4(w0.x, w0.y, byte_bias(se > 127u ? 127 : static_cast<int>(se)), 0u);
                m.fidx[k] = static_cast<uint16_t>(e);
            }
            if (isM) {
                const uint32_t k = nM + __popc(bm & below);
                const uint32_t nN = meta_nN(meta);
                // threshold for word 0 alone: popc(word 0) <= s - nN is necessary
                // for a hit; -1 (as int) when the query's Ns alone exceed s
                const int thr = se >= nN ? static_cast<int>(se - nN > 127u ? 127u : se - nN) : -1;
                m.sM[k] = make_uint4(w0.x, w0.y, w0.z, byte_bias(thr));
                m.midx[k] = static_cast<uint16_t>(e);
            }
            nF += __popc(bf);
            nM += __popc(bm);
        }
        if (lane == 0) {
            *s_nF = nF;
            *s_nM = nM;
        }
    }
    __syncthreads();
    return m;
}

// Per-entry counts of the chunk into the per-query counters (all threads,
// after the last scan of the chunk and a barrier).
__device__ __forceinline__ void flush_counts(const QueryTable &qt, const Smem &m, uint32_t nent, uint32_t e0,
                                             const HitSink &sink) {
    for (uint32_t i = threadIdx.x; i < nent; i += blockDim.x)
        if (m.cnt[i]) {
            const uint32_t id = qt.ids ? qt.ids[e0 + i] : e0 + i;
            atomicAdd(&sink.qcount[id >> 1], static_cast<unsigned long long>(m.cnt[i]));
            m.cnt[i] = 0;
        }
}

// Byte-lane multipliers 1, 2^8, 2^16, 2^24 in registers (opaque to the
// compiler, so the count packing stays IMAD on the FMA pipe).
__device__ __forceinline__ void lane_multipliers(uint32_t *mul) {
#pragma unroll
    for (int w = 0; w < kWin; w++) asm volatile("mov.u32 %0, %1;" : "=r"(mul[w]) : "r"(1u << (8 * w)));
}

// Blocks (of 32 * kWin windows) are dealt to the nw warps of a range in
// chunks of kChunk consecutive blocks, round robin: warp w scans blocks
// base + w * kChunk + j * nw * kChunk + i (i < kChunk) below blk_end.  The
// warps together sweep the range front to back, so their reads share DRAM
// pages, while each warp still moves forward through the pieces.  Words are
// staged through stage[2][NW] (this warp's buffers), one block ahead.
#ifndef IFA_SCAN_CHUNK
#define IFA_SCAN_CHUNK 1  // measured on B300: 1 beats 4, 8 and 32 at maxSubs 4 and 16
#endif
constexpr uint32_t kChunk = IFA_SCAN_CHUNK;
template <int WMAX, class WH>
__device__ __forceinline__ void scan_blocks(const Batch &b, const QueryTable &qt, const Smem &m, uint32_t nent,
                                            uint32_t nF, uint32_t nM, uint32_t e0, uint32_t s, uint32_t lmin,
                                            uint32_t lmax, const HitSink &sink, WH &wh,
                                            uint2 (*stage)[Stage<WMAX>::kSlots], const uint32_t *mul,
                                            uint64_t base, uint64_t blk_end, uint32_t w, uint32_t nw,
                                            uint32_t lane, uint16_t (*cq)[32]) {
    constexpr int NW = Stage<WMAX>::kWords;
    static_assert(32 * kWin == kEventBlock, "events address blocks of 32 x kWin windows");
    wh.flush(sink, lane);  // the staging buffer now takes events
    const uint64_t jump = static_cast<uint64_t>(nw - 1) * kChunk;
    uint64_t blk = base + static_cast<uint64_t>(w) * kChunk;
    uint32_t in_chunk = 0;
    uint64_t nxt = blk;
    if (blk < blk_end) stage_block<NW>(b, blk, stage[0], lane);
    for (uint32_t it = 0; blk < blk_end; it++, blk = nxt) {
        const bool chunk_end = in_chunk + 1 == kChunk;
        nxt = chunk_end ? blk + 1 + jump : blk + 1;
        in_chunk = chunk_end ? 0u : in_chunk + 1;
        if (nxt < blk_end) stage_block<NW>(b, nxt, stage[(it + 1) & 1], lane);
        else asm volatile("cp.async.commit_group;\n" ::: "memory");
        asm volatile("cp.async.wait_group 1;\n" ::: "memory");
        __syncwarp();
        const uint2 *R = stage[it & 1];
        const uint64_t p0 = blk * (32 * kWin);
        const uint32_t flags = special_bits(R[NW].x, R[NW + 1].x, blk * kWin, NW);
        // a uniform maxSubs >= 32 makes word 0 useless as a filter: scan generically
        const bool special = (s != kSPerEntry && s >= 32u) || flags != 0u ||
                             p0 + 32 * kWin - 1 + lmax - 1 >= b.nbases ||
                             p0 + lmin < static_cast<uint64_t>(b.halo) + 1;
        if (special) {
#pragma unroll 1
            for (int k = 0; k < kWin; k++)
                generic_window<WMAX>(b, qt, m, nent, e0, p0 + 32 * k, lane, s, sink, wh);
            __syncwarp();
            continue;
        }
        // word 0 of the lane's windows
        uint32_t hw[kWin], lw[kWin];
#pragma unroll
        for (int k = 0; k < kWin; k++) {
            hw[k] = __funnelshift_r(R[k].x, R[k + 1].x, lane);
            lw[k] = __funnelshift_r(R[k].y, R[k + 1].y, lane);
        }
        const uint32_t bi = static_cast<uint32_t>(blk);
        uint32_t qn = 0;       // this lane's queued candidates
        bool queued = false;   // some group fired in this block (warp-uniform)
        scan_class<WMAX, false>(b, qt, m, m.sF, m.fidx, nF, hw, lw, mul, R, e0, bi, lane, s, sink, wh, cq, qn,
                                queued);
        scan_class<WMAX, true>(b, qt, m, m.sM, m.midx, nM, hw, lw, mul, R, e0, bi, lane, s, sink, wh, cq, qn,
                               queued);
        if constexpr (kQDepth > 0) {
            if (queued) drain_queue<WMAX>(b, qt, m, cq, qn, hw, lw, mul, R, e0, bi, lane, s, sink, wh);
        }
        __syncwarp();
    }
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    wh.flush_events(b, qt.ids, e0, m.cnt, sink, lane);
}

}  // namespace brute
}  // namespace ifa

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
// memory.  The packed words of the warp's next block are prefetched into a
// per-warp shared double buffer with cp.async while the current one is
// scanned.
//
// Early termination, batched: for maxSubs < 32 the first word alone
// rejects almost every window (E[mm] = 24 of 32 on random sequence), so
// the hot loop computes only word 0 for 4 entries x 4 windows, keeps the
// minimum count per entry, and one warp vote per 4 entries decides whether
// the exact path (all words, hit emission) runs for any of them (then a vote
// per entry picks which).  Entries
// whose first word is fully counted and that hold no N ("class F") need no
// care mask and share the threshold maxSubs, so their word costs
// 2 LOP3 + 1 POPC + 1 IMNMX per window -- the POPC pipe (16 lanes/clk/SM)
// is the binding unit.  Other entries ("class M") also AND a care mask and
// use their own threshold maxSubs - nN.
//
// Blocks of windows that touch an N, a contig-piece boundary, the batch end
// or the halo take a generic path that folds in the reference N plane and
// checks each window stays inside one piece and is owned by this batch.
#include "hits.cuh"

namespace ifa {

namespace {

constexpr int kScanThreads = 256;
constexpr int kScanWarps = kScanThreads / kWarp;
constexpr size_t kScanSmemBudget = 40 * 1024;  // dynamic; + static (hit staging, word staging) < 48 KB
constexpr int kGroup = 4;                       // entries per warp vote in the hot loop
constexpr int kWin = 4;                         // windows per lane (32 * kWin per warp step)

// Per-entry shared memory: WMAX uint4 words, a class-M word-0 record, a
// class-F word-0 record, meta, count, and two 16-bit index slots.
__host__ __device__ constexpr size_t entry_smem(int wmax) {
    return wmax * sizeof(uint4) + sizeof(uint4) + sizeof(uint2) + 2 * sizeof(uint32_t) +
           2 * sizeof(uint16_t);
}

struct Smem {
    uint4 *sq;         // entries x WMAX full words
    uint4 *sM;         // class M: {hi0, lo0, care0, threshold}
    uint2 *sF;         // class F: {hi0, lo0}
    uint32_t *meta;
    uint32_t *cnt;
    uint16_t *fidx;
    uint16_t *midx;
};

__device__ inline Smem carve(uint4 *base, uint32_t nent, int wmax) {
    Smem m;
    m.sq = base;
    m.sM = m.sq + static_cast<size_t>(nent) * wmax;
    m.sF = reinterpret_cast<uint2 *>(m.sM + nent);
    m.meta = reinterpret_cast<uint32_t *>(m.sF + nent);
    m.cnt = m.meta + nent;
    m.fidx = reinterpret_cast<uint16_t *>(m.cnt + nent);
    m.midx = m.fidx + nent;
    return m;
}

// Words of the block starting at word 2*? are staged per warp in shared
// memory; a block is WIN x 32 windows: lane l owns windows p0 + 32 k + l,
// k < WIN, and window k's word j is cut from staged words k + j, k + j + 1.
template <int WMAX>
struct Stage {
    static constexpr int kWords = kWin + WMAX;  // staged words per block
};

// Exact evaluation of one entry for the lane's WIN windows of a block without
// N, piece boundary or ownership limits, then hit emission.
template <int WMAX>
__device__ __forceinline__ void exact_fast(const Batch &b, const QueryTable &qt, const Smem &m,
                                           const uint4 *R, uint32_t e, uint32_t e0, uint64_t p0,
                                           uint32_t lane, uint32_t s, const HitSink &sink,
                                           WarpHits &wh, uint32_t &pidx) {
    const uint32_t meta = m.meta[e];
    const uint32_t W = (meta >> 8) & 0xffu;
    const uint4 *qw = m.sq + static_cast<size_t>(e) * WMAX;
    uint32_t mm[kWin];
#pragma unroll
    for (int k = 0; k < kWin; k++) mm[k] = meta >> 16;
#pragma unroll
    for (int j = 0; j < WMAX; j++) {
        if (j < static_cast<int>(W)) {
            const uint4 q = qw[j];
#pragma unroll
            for (int k = 0; k < kWin; k++) {
                const uint4 a = R[k + j], c = R[k + j + 1];
                const uint32_t h = __funnelshift_r(a.x, c.x, lane), l = __funnelshift_r(a.y, c.y, lane);
                mm[k] += __popc(((h ^ q.x) | (l ^ q.y)) & q.z);
            }
        }
    }
    bool any = false;
#pragma unroll
    for (int k = 0; k < kWin; k++) any |= mm[k] <= s;
    if (!__any_sync(0xffffffffu, any)) return;
    if (pidx == 0xffffffffu) pidx = find_piece(b.pieces, b.npieces, p0);
    const DevPiece pc = b.pieces[pidx];
    const uint32_t id = qt.ids ? qt.ids[e0 + e] : e0 + e;
    const uint32_t pos0 = static_cast<uint32_t>(pc.contig_off + (p0 + lane - pc.start));
#pragma unroll
    for (int k = 0; k < kWin; k++)
        wh.emit(sink, lane, mm[k] <= s, id >> 1, pc.contig, pos0 + 32 * k, id & 1u, mm[k], m.cnt + e);
}

// Generic evaluation of every entry for one window per lane (p = p0 + lane)
// whose block may hold N, piece boundaries, the batch end or the halo.
template <int WMAX>
__device__ void generic_window(const Batch &b, const QueryTable &qt, const Smem &m, uint32_t nent,
                               uint32_t e0, uint64_t p0, uint32_t lane, uint32_t s,
                               const HitSink &sink, WarpHits &wh) {
    const uint64_t w0 = p0 >> 5;
    uint32_t hi[WMAX], lo[WMAX], nw[WMAX], bw[WMAX];
    uint4 cur = __ldg(b.words + w0);
#pragma unroll
    for (int j = 0; j < WMAX; j++) {
        const uint4 nx = __ldg(b.words + w0 + j + 1);
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
        const uint32_t L = meta & 0xffu;
        const uint32_t W = (meta >> 8) & 0xffu;
        const uint4 *qw = m.sq + static_cast<size_t>(e) * WMAX;
        uint32_t mm = meta >> 16;
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
        const bool hit = valid && mm <= s;
        if (__any_sync(0xffffffffu, hit)) {
            uint32_t contig = 0, pos = 0;
            if (hit) {
                const DevPiece pc = b.pieces[find_piece(b.pieces, b.npieces, p)];
                contig = pc.contig;
                pos = static_cast<uint32_t>(pc.contig_off + (p - pc.start));
            }
            const uint32_t id = qt.ids ? qt.ids[e0 + e] : e0 + e;
            wh.emit(sink, lane, hit, id >> 1, contig, pos, id & 1u, mm, m.cnt + e);
        }
    }
}

// Stage the words of block `blk` into `dst` (shared) with cp.async: lane i
// copies word i (16 bytes).
template <int NW>
__device__ __forceinline__ void stage_block(const Batch &b, uint64_t blk, uint4 *dst, uint32_t lane) {
    if (lane < NW) {
        const uint4 *src = b.words + blk * kWin + lane;
        const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(dst + lane));
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}

template <int WMAX>
__global__ void __launch_bounds__(kScanThreads)
k_scan_brute(Batch b, QueryTable qt, uint32_t e0, uint32_t e1, uint32_t s, uint32_t lmin,
             uint32_t lmax, HitSink sink) {
    constexpr int NW = Stage<WMAX>::kWords;
    extern __shared__ uint4 smem4[];
    __shared__ ifa_hit wbuf[kScanWarps][32];
    __shared__ uint4 stage[kScanWarps][2][NW];
    __shared__ uint32_t s_nF, s_nM;
    const uint32_t nent = e1 - e0;
    const Smem m = carve(smem4, nent, WMAX);

    for (uint32_t i = threadIdx.x; i < nent * WMAX; i += kScanThreads)
        m.sq[i] = qt.words[static_cast<size_t>(e0) * WMAX + i];
    for (uint32_t i = threadIdx.x; i < nent; i += kScanThreads) {
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
                isF = (meta >> 16) == 0u && w0.z == 0xffffffffu;
                isM = !isF;
            }
            const uint32_t bf = __ballot_sync(0xffffffffu, isF);
            const uint32_t bm = __ballot_sync(0xffffffffu, isM);
            const uint32_t below = (1u << lane) - 1u;
            if (isF) {
                const uint32_t k = nF + __popc(bf & below);
                m.sF[k] = make_uint2(w0.x, w0.y);
                m.fidx[k] = static_cast<uint16_t>(e);
            }
            if (isM) {
                const uint32_t k = nM + __popc(bm & below);
                const uint32_t nN = meta >> 16;
                // threshold for word 0 alone: popc(word 0) <= s - nN is necessary
                // for a hit; -1 (as int) when the query's Ns alone exceed s
                const uint32_t thr = s >= nN ? s - nN : 0xffffffffu;
                m.sM[k] = make_uint4(w0.x, w0.y, w0.z, thr);
                m.midx[k] = static_cast<uint16_t>(e);
            }
            nF += __popc(bf);
            nM += __popc(bm);
        }
        if (lane == 0) {
            s_nF = nF;
            s_nM = nM;
        }
    }
    __syncthreads();
    const uint32_t nF = s_nF, nM = s_nM;
    const int thrF = static_cast<int>(s);

    WarpHits wh;
    wh.init(wbuf[warp]);

    const uint64_t nblk = (b.nbases + 32 * kWin - 1) / (32 * kWin);
    const uint64_t stride = static_cast<uint64_t>(gridDim.x) * kScanWarps;
    uint64_t blk = static_cast<uint64_t>(blockIdx.x) * kScanWarps + warp;
    if (blk < nblk) stage_block<NW>(b, blk, stage[warp][0], lane);
    for (uint32_t it = 0; blk < nblk; it++, blk += stride) {
        const uint64_t nxt = blk + stride;
        if (nxt < nblk) stage_block<NW>(b, nxt, stage[warp][(it + 1) & 1], lane);
        else asm volatile("cp.async.commit_group;\n" ::: "memory");
        asm volatile("cp.async.wait_group 1;\n" ::: "memory");
        __syncwarp();
        const uint4 *R = stage[warp][it & 1];
        const uint64_t p0 = blk * (32 * kWin);
        uint32_t flags = R[0].z | (R[0].w & ~1u);
#pragma unroll
        for (int i = 1; i < NW; i++) flags |= R[i].z | R[i].w;
        const bool special = s >= 32u || flags != 0u || p0 + 32 * kWin - 1 + lmax - 1 >= b.nbases ||
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
        uint32_t pidx = 0xffffffffu;
        uint32_t k = 0;
        for (; k + kGroup <= nF; k += kGroup) {
            bool need[kGroup];
#pragma unroll
            for (int i = 0; i < kGroup; i++) {
                const uint2 q = m.sF[k + i];
                int mn = __popc((hw[0] ^ q.x) | (lw[0] ^ q.y));
#pragma unroll
                for (int w = 1; w < kWin; w++) mn = min(mn, __popc((hw[w] ^ q.x) | (lw[w] ^ q.y)));
                need[i] = mn <= thrF;
            }
            if (__any_sync(0xffffffffu, need[0] || need[1] || need[2] || need[3])) {
#pragma unroll 1
                for (int i = 0; i < kGroup; i++)
                    if (__any_sync(0xffffffffu, need[i]))
                        exact_fast<WMAX>(b, qt, m, R, m.fidx[k + i], e0, p0, lane, s, sink, wh, pidx);
            }
        }
        for (; k < nF; k++) {
            const uint2 q = m.sF[k];
            int mn = __popc((hw[0] ^ q.x) | (lw[0] ^ q.y));
#pragma unroll
            for (int w = 1; w < kWin; w++) mn = min(mn, __popc((hw[w] ^ q.x) | (lw[w] ^ q.y)));
            if (__any_sync(0xffffffffu, mn <= thrF))
                exact_fast<WMAX>(b, qt, m, R, m.fidx[k], e0, p0, lane, s, sink, wh, pidx);
        }
        for (k = 0; k < nM; k++) {
            const uint4 q = m.sM[k];
            int mn = __popc(((hw[0] ^ q.x) | (lw[0] ^ q.y)) & q.z);
#pragma unroll
            for (int w = 1; w < kWin; w++) mn = min(mn, __popc(((hw[w] ^ q.x) | (lw[w] ^ q.y)) & q.z));
            if (__any_sync(0xffffffffu, mn <= static_cast<int>(q.w)))
                exact_fast<WMAX>(b, qt, m, R, m.midx[k], e0, p0, lane, s, sink, wh, pidx);
        }
        __syncwarp();
    }
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    wh.finish(sink, lane);
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < nent; i += kScanThreads)
        if (m.cnt[i]) {
            const uint32_t id = qt.ids ? qt.ids[e0 + i] : e0 + i;
            atomicAdd(&sink.qcount[id >> 1], static_cast<unsigned long long>(m.cnt[i]));
        }
}

template <int WMAX>
cudaError_t launch_t(const Batch &b, const QueryTable &qt, uint32_t e0, uint32_t e1, uint32_t s,
                     uint32_t lmin, uint32_t lmax, const HitSink &sink, cudaStream_t st) {
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
    k_scan_brute<WMAX><<<g, kScanThreads, smem, st>>>(b, qt, e0, e1, s, lmin, lmax, sink);
    return cudaGetLastError();
}

}  // namespace

uint32_t scan_brute_chunk_entries(uint32_t wmax) {
    const size_t n = kScanSmemBudget / entry_smem(static_cast<int>(wmax));
    return static_cast<uint32_t>(n < 65535 ? n : 65535);
}

cudaError_t launch_scan_brute(const Batch &b, const QueryTable &qt, uint32_t e0, uint32_t e1,
                              uint32_t max_subs, uint32_t lmin, uint32_t lmax, const HitSink &sink,
                              cudaStream_t st, int *launches) {
    if (e1 <= e0 || b.nbases == 0) return cudaSuccess;
    if (launches) (*launches)++;
    switch (qt.wmax) {
    case 1: return launch_t<1>(b, qt, e0, e1, max_subs, lmin, lmax, sink, st);
    case 2: return launch_t<2>(b, qt, e0, e1, max_subs, lmin, lmax, sink, st);
    case 4: return launch_t<4>(b, qt, e0, e1, max_subs, lmin, lmax, sink, st);
    case 8: return launch_t<8>(b, qt, e0, e1, max_subs, lmin, lmax, sink, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace ifa

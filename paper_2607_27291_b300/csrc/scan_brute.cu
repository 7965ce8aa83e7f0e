// scan_brute.cu -- brute-force Hamming scan (Methods, "Algorithm Design",
// brute-force mode; "SIMD Optimization").
//
// The paper's CPU kernel broadcasts each query base against 32 consecutive
// reference positions and counts mismatches per lane with early
// termination.  Here a warp owns 32 consecutive windows (lane = window
// offset) and compares whole 32-base words with bit-parallel logic:
//   x  = ((R_hi ^ Q_hi) | (R_lo ^ Q_lo)) & care        one word, 32 bases
//   mm = nN + sum popc(x)
// where R_* is the reference window word of the lane, extracted from two
// packed words by a funnel shift, and Q_* the query word (reverse
// complement precomputed) held in shared memory.  Early termination: when
// no lane of the warp can still reach mm <= maxSubs after a word, the
// remaining words of that query are skipped (warp vote).
//
// Windows that touch an N, a contig-piece boundary, the batch end or the
// halo take a slow path that also folds in the reference N plane and
// checks the window stays inside one piece and is owned by this batch.
#include "hits.cuh"

namespace ifa {

namespace {

constexpr int kScanThreads = 256;
constexpr int kScanWarps = kScanThreads / kWarp;
constexpr size_t kScanSmemBudget = 40 * 1024;  // dynamic; + 4 KB static stays under 48 KB

template <int WMAX>
__global__ void __launch_bounds__(kScanThreads)
k_scan_brute(Batch b, QueryTable qt, uint32_t e0, uint32_t e1, uint32_t s, uint32_t lmin,
             uint32_t lmax, HitSink sink) {
    extern __shared__ uint4 smem4[];
    __shared__ ifa_hit wbuf[kScanWarps][32];
    const uint32_t nent = e1 - e0;
    uint4 *sq = smem4;
    uint32_t *smeta = reinterpret_cast<uint32_t *>(sq + static_cast<size_t>(nent) * WMAX);
    uint32_t *scnt = smeta + nent;

    for (uint32_t i = threadIdx.x; i < nent * WMAX; i += kScanThreads)
        sq[i] = qt.words[static_cast<size_t>(e0) * WMAX + i];
    for (uint32_t i = threadIdx.x; i < nent; i += kScanThreads) {
        smeta[i] = qt.meta[e0 + i];
        scnt[i] = 0;
    }
    __syncthreads();

    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t warp = threadIdx.x >> 5;
    WarpHits wh;
    wh.init(wbuf[warp]);

    const uint64_t nblocks = (b.nbases + 31) >> 5;
    const uint64_t stride = static_cast<uint64_t>(gridDim.x) * kScanWarps;
    for (uint64_t blk = static_cast<uint64_t>(blockIdx.x) * kScanWarps + warp; blk < nblocks;
         blk += stride) {
        const uint64_t p0 = blk << 5;
        uint4 R[WMAX + 1];
#pragma unroll
        for (int i = 0; i <= WMAX; i++) R[i] = __ldg(b.words + blk + i);
        uint32_t hi[WMAX], lo[WMAX];
#pragma unroll
        for (int j = 0; j < WMAX; j++) {
            hi[j] = __funnelshift_r(R[j].x, R[j + 1].x, lane);
            lo[j] = __funnelshift_r(R[j].y, R[j + 1].y, lane);
        }
        uint32_t flags = R[0].z | (R[0].w & ~1u);
#pragma unroll
        for (int i = 1; i <= WMAX; i++) flags |= R[i].z | R[i].w;
        const bool special = flags != 0u || p0 + 31 + lmax - 1 >= b.nbases ||
                             p0 + lmin < static_cast<uint64_t>(b.halo) + 1;

        if (!special) {
            // fast path: every (lane, entry) window is inside one piece, N-free, owned
            uint32_t pidx = 0xffffffffu;
            for (uint32_t e = 0; e < nent; e++) {
                const uint32_t meta = smeta[e];
                const uint32_t W = (meta >> 8) & 0xffu;
                const uint4 *qw = sq + static_cast<size_t>(e) * WMAX;
                uint4 q = qw[0];
                uint32_t mm = (meta >> 16) + __popc(((hi[0] ^ q.x) | (lo[0] ^ q.y)) & q.z);
#pragma unroll
                for (int j = 1; j < WMAX; j++) {
                    if (j < static_cast<int>(W)) {
                        if (!__any_sync(0xffffffffu, mm <= s)) break;  // early termination
                        q = qw[j];
                        mm += __popc(((hi[j] ^ q.x) | (lo[j] ^ q.y)) & q.z);
                    }
                }
                const bool hit = mm <= s;
                if (__any_sync(0xffffffffu, hit)) {
                    if (pidx == 0xffffffffu) pidx = find_piece(b.pieces, b.npieces, p0);
                    const DevPiece pc = b.pieces[pidx];
                    const uint64_t p = p0 + lane;
                    const uint32_t id = qt.ids ? qt.ids[e0 + e] : e0 + e;
                    wh.emit(sink, lane, hit, id >> 1, pc.contig,
                            static_cast<uint32_t>(pc.contig_off + (p - pc.start)), id & 1u, mm,
                            scnt + e);
                }
            }
        } else {
            const uint64_t p = p0 + lane;
            uint32_t nw[WMAX], bw[WMAX];
#pragma unroll
            for (int j = 0; j < WMAX; j++) {
                nw[j] = __funnelshift_r(R[j].z, R[j + 1].z, lane);
                bw[j] = __funnelshift_r(R[j].w, R[j + 1].w, lane);
            }
            bw[0] &= ~1u;  // a piece may start at the window's first base
            for (uint32_t e = 0; e < nent; e++) {
                const uint32_t meta = smeta[e];
                const uint32_t L = meta & 0xffu;
                const uint32_t W = (meta >> 8) & 0xffu;
                const uint4 *qw = sq + static_cast<size_t>(e) * WMAX;
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
                const bool valid = (p + L <= b.nbases) && (p + L >= static_cast<uint64_t>(b.halo) + 1) &&
                                   bnd == 0u;
                const bool hit = valid && mm <= s;
                if (__any_sync(0xffffffffu, hit)) {
                    uint32_t contig = 0, pos = 0;
                    if (hit) {
                        const DevPiece pc = b.pieces[find_piece(b.pieces, b.npieces, p)];
                        contig = pc.contig;
                        pos = static_cast<uint32_t>(pc.contig_off + (p - pc.start));
                    }
                    const uint32_t id = qt.ids ? qt.ids[e0 + e] : e0 + e;
                    wh.emit(sink, lane, hit, id >> 1, contig, pos, id & 1u, mm, scnt + e);
                }
            }
        }
    }
    wh.finish(sink, lane);
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < nent; i += kScanThreads)
        if (scnt[i]) {
            const uint32_t id = qt.ids ? qt.ids[e0 + i] : e0 + i;
            atomicAdd(&sink.qcount[id >> 1], static_cast<unsigned long long>(scnt[i]));
        }
}

template <int WMAX>
cudaError_t launch_t(const Batch &b, const QueryTable &qt, uint32_t e0, uint32_t e1, uint32_t s,
                     uint32_t lmin, uint32_t lmax, const HitSink &sink, cudaStream_t st) {
    const size_t smem = static_cast<size_t>(e1 - e0) * (WMAX * sizeof(uint4) + 2 * sizeof(uint32_t));
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
    uint64_t nblocks = (b.nbases + 31) >> 5;
    uint64_t need = (nblocks + kScanWarps - 1) / kScanWarps;
    int g = static_cast<int>(need < static_cast<uint64_t>(grid) ? need : grid);
    if (g < 1) g = 1;
    k_scan_brute<WMAX><<<g, kScanThreads, smem, st>>>(b, qt, e0, e1, s, lmin, lmax, sink);
    return cudaGetLastError();
}

}  // namespace

uint32_t scan_brute_chunk_entries(uint32_t wmax) {
    return static_cast<uint32_t>(kScanSmemBudget / (wmax * sizeof(uint4) + 2 * sizeof(uint32_t)));
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

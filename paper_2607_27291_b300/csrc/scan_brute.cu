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

template <int WMAX>
__global__ void __launch_bounds__(kScanThreads, kScanMinCtas<WMAX>)
k_scan_brute(Batch b, QueryTable qt, uint32_t e0, uint32_t e1, uint32_t s, uint32_t lmin,
             uint32_t lmax, HitSink sink) {
    extern __shared__ uint4 smem4[];
    __shared__ __align__(16) ifa_hit wbuf[kScanWarps][32];
    __shared__ __align__(8) uint2 stage[kScanWarps][2][Stage<WMAX>::kSlots];
    __shared__ uint16_t cq[kScanWarps][kQRows][32];
    __shared__ uint32_t s_nF, s_nM;
    const uint32_t nent = e1 - e0;
    const Smem m = load_chunk<WMAX>(qt, e0, e1, s, smem4, &s_nF, &s_nM);
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t warp = threadIdx.x >> 5;
    WarpHits wh;
    wh.init(wbuf[warp]);
    uint32_t mul[kWin];
    lane_multipliers(mul);
    const uint64_t nblk = (b.nbases + 32 * kWin - 1) / (32 * kWin);
    scan_blocks<WMAX>(b, qt, m, nent, s_nF, s_nM, e0, s, lmin, lmax, sink, wh, stage[warp], mul, 0, nblk,
                      blockIdx.x * kScanWarps + warp, gridDim.x * kScanWarps, lane, cq[warp]);
    wh.finish(sink, lane);
    __syncthreads();
    flush_counts(qt, m, nent, e0, sink);
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
    const uint32_t n = chunk_cap(static_cast<int>(wmax));
    return n < 65535u ? n : 65535u;
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

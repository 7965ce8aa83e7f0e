// clip.cu -- soft-clipped windows at contig ends (Methods, Algorithm Design).
//
// With soft clipping an alignment may overhang an end of its contig by up
// to C = floor(clip_pct * L / 100) bases; the overhang counts as clips, not
// mismatches, and the window is a hit when its aligned bases have at most
// maxSubs mismatches (N mismatching everything, as everywhere).  The whole-
// window scans never leave a contig, so the clipped windows are a separate,
// small set: per contig and entry, the C windows that start before the
// contig (left clips) and the C that end after it (right clips), found
// exhaustively in both modes.  pos of such a hit is the contig coordinate
// of its first aligned base; ifa_hit.clips = left | right << 8.
//
// A batch evaluates the clipped windows whose last aligned base is one of
// its new bases (the rule for every window): left windows of contigs that
// start in the batch's visible bases, right windows of contigs that end in
// it.  The aligned bases then always lie in the batch (halo included).
// The serving loop scans the whole store as one batch, a range of its
// pieces per slice, and sends each hit to its request's own ring (MULTI).
#include "hits.cuh"

namespace ifa {

namespace {

constexpr int kClipThreads = 256;

// The 32 bases of the batch starting at x (which may be negative: bases
// before the batch read as zero words; they are masked by the caller).
__device__ __forceinline__ uint4 bases32(const Batch &b, int64_t x) {
    if (x <= -32) return make_uint4(0u, 0u, 0u, 0u);
    if (x < 0) {
        const uint4 w = ref_word(b, 0);
        const uint32_t sh = static_cast<uint32_t>(-x);
        return make_uint4(w.x << sh, w.y << sh, w.z << sh, 0u);
    }
    const uint64_t wi = static_cast<uint64_t>(x) >> 5;
    const uint32_t sh = static_cast<uint32_t>(x & 31);
    const uint4 a = ref_word(b, wi), c = ref_word(b, wi + 1);
    return make_uint4(__funnelshift_r(a.x, c.x, sh), __funnelshift_r(a.y, c.y, sh), __funnelshift_r(a.z, c.z, sh),
                      0u);
}

// Mismatches of entry qw (wmax words, bit i = base i) at window p over the
// aligned positions [lo, hi): a query N (care bit 0), a reference N or
// differing codes.
__device__ __forceinline__ uint32_t clipped_mismatches(const Batch &b, const uint4 *qw, uint32_t wmax, int64_t p,
                                                      uint32_t lo, uint32_t hi) {
    uint32_t mm = 0;
    for (uint32_t j = 0; j < wmax && 32u * j < hi; j++) {
        const uint32_t j0 = 32u * j;
        uint32_t amask = 0xffffffffu;
        if (lo > j0) amask &= lo - j0 >= 32u ? 0u : ~((1u << (lo - j0)) - 1u);
        if (hi < j0 + 32u) amask &= (1u << (hi - j0)) - 1u;
        if (!amask) continue;
        const uint4 q = qw[j];
        const uint4 r = bases32(b, p + j0);
        mm += __popc(amask & (~q.z | r.z | (r.x ^ q.x) | (r.y ^ q.y)));
    }
    return mm;
}

// Pairs (piece, entry) for pieces [p_lo, p_hi) of b and entries
// [e_base, e_base + nent) of qt.
template <bool MULTI>
__global__ void __launch_bounds__(kClipThreads)
k_clip_scan(Batch b, QueryTable qt, uint32_t e_base, uint32_t nent, uint32_t p_lo, uint32_t p_hi,
            uint32_t clip_pct, uint32_t s, uint32_t cmax, HitSink sink) {
    __shared__ __align__(16) ifa_hit wbuf[kClipThreads / 32][32];
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    WarpHitsT<MULTI> wh;
    wh.init(wbuf[warp]);
    const uint64_t npairs = static_cast<uint64_t>(p_hi - p_lo) * nent;
    const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
    // every lane of a warp runs the same number of rounds (emit is warp-wide)
    const uint64_t first = static_cast<uint64_t>(blockIdx.x) * blockDim.x + (threadIdx.x & ~31u);
    for (uint64_t base = first; base < npairs; base += stride) {
        const uint64_t pair = base + lane;
        const bool live = pair < npairs;
        uint32_t piece = 0, e = 0, L = 0, C = 0, se = 0;
        int64_t cs = 0, ce = 0;
        bool has_start = false, has_end = false;
        if (live) {
            piece = p_lo + static_cast<uint32_t>(pair / nent);
            e = e_base + static_cast<uint32_t>(pair % nent);
            const uint32_t m = qt.meta[e];
            L = meta_L(m);
            C = clip_pct * L / 100u;
            se = entry_s(m, s);
            const DevPiece pc = b.pieces[piece];
            const uint64_t pend = piece + 1 < b.npieces ? b.pieces[piece + 1].start : b.nbases;
            cs = static_cast<int64_t>(pc.start) - static_cast<int64_t>(pc.contig_off);
            ce = static_cast<int64_t>(pend);
            has_start = pc.contig_off == 0;   // the contig's first base is in this batch
            has_end = pc.last != 0;           // and its last base
            if (!has_end) ce = INT64_MAX;
        }
        // rounds: w < cmax left windows p = cs - 1 - w; then right windows
        // p = ce - L + 1 + (w - cmax) that start inside the contig
        for (uint32_t w = 0; w < 2u * cmax; w++) {
            bool hit = false;
            int64_t p = 0;
            uint32_t left = 0, right = 0, mm = 0;
            if (live && C) {
                bool cand;
                if (w < cmax) {
                    cand = has_start && w < C;
                    p = cs - 1 - static_cast<int64_t>(w);
                } else {
                    const uint32_t o = w - cmax;
                    cand = has_end && o < C;
                    p = ce - static_cast<int64_t>(L) + 1 + static_cast<int64_t>(o);
                    cand = cand && p >= cs;
                }
                if (cand) {
                    left = p < cs ? static_cast<uint32_t>(cs - p) : 0u;
                    right = p + static_cast<int64_t>(L) > ce ? static_cast<uint32_t>(p + L - ce) : 0u;
                    const uint32_t clips = left + right;
                    // owned by the batch holding the last aligned base as a new base
                    const int64_t last = (p + static_cast<int64_t>(L) < ce ? p + static_cast<int64_t>(L) : ce) - 1;
                    cand = clips >= 1 && clips <= C && clips < L && last >= static_cast<int64_t>(b.halo) &&
                           last < static_cast<int64_t>(b.nbases);
                }
                if (cand) {
                    mm = clipped_mismatches(b, qt.words + static_cast<size_t>(e) * qt.wmax, qt.wmax, p, left,
                                            L - right);
                    hit = mm <= se;
                }
            }
            uint32_t pos = 0, contig = 0;
            if (hit) {
                const DevPiece pc = b.pieces[piece];
                contig = pc.contig;
                pos = static_cast<uint32_t>(p + left - cs);
            }
            const uint32_t id = qt.ids ? (live ? qt.ids[e] : 0u) : e;
            wh.emit(sink, lane, hit, id >> 1, contig, pos, id & 1u, mm, nullptr, left | (right << 8));
        }
    }
    wh.finish(sink, lane);
}

}  // namespace

cudaError_t launch_clip_scan(const Batch &b, const QueryTable &qt, uint32_t nent, uint32_t clip_pct, uint32_t s,
                             uint32_t lmax, const HitSink &sink, cudaStream_t st, uint32_t e_base, uint32_t p_lo,
                             uint32_t p_hi) {
    const uint32_t cmax = clip_pct * lmax / 100u;
    if (p_hi > b.npieces) p_hi = b.npieces;
    if (nent == 0 || p_lo >= p_hi || cmax == 0) return cudaSuccess;
    const uint64_t npairs = static_cast<uint64_t>(p_hi - p_lo) * nent;
    uint64_t grid = (npairs + kClipThreads - 1) / kClipThreads;
    if (grid > 148ull * 16) grid = 148ull * 16;
    if (sink.rings)
        k_clip_scan<true><<<static_cast<unsigned>(grid), kClipThreads, 0, st>>>(b, qt, e_base, nent, p_lo, p_hi,
                                                                               clip_pct, s, cmax, sink);
    else
        k_clip_scan<false><<<static_cast<unsigned>(grid), kClipThreads, 0, st>>>(b, qt, e_base, nent, p_lo, p_hi,
                                                                                clip_pct, s, cmax, sink);
    return cudaGetLastError();
}

}  // namespace ifa

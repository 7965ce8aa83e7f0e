// seed_scan.cuh -- device code of the indexed-mode seed scan, shared by the
// streaming kernel (indexed.cu) and the persistent multi-set kernel
// (batch.cu).  See indexed.cu for the method.
#pragma once
#include "hits.cuh"
#include "indexed.cuh"

namespace ifa {
namespace seed {

// Scan 32-position blocks blk, blk + stride, ... < blk_end with this warp:
// look every position's k-mer up in each table, verify the window each
// posting names, and emit it from its first seed when its seed count
// reaches the entry's threshold.  Adds verified candidates to ncand.
template <int WMAX, class WH>
__device__ __forceinline__ void seed_blocks(const Batch &b, const QueryTable &qt, const KTablesArg &tabs,
                                            const uint32_t *__restrict__ entry_minhits, uint32_t step,
                                            uint32_t s, const HitSink &sink, WH &wh, uint64_t blk,
                                            uint64_t blk_end, uint64_t stride, uint32_t lane,
                                            unsigned long long &ncand) {
    uint32_t pidx = 0xffffffffu;   // the lane's last hit's piece
    for (; blk < blk_end; blk += stride) {
        const uint64_t j = (blk << 5) + lane;
        const uint4 A = ref_word(b, blk), B = ref_word(b, blk + 1);
        const uint32_t hiw = __funnelshift_r(A.x, B.x, lane);
        const uint32_t low = __funnelshift_r(A.y, B.y, lane);
        const uint32_t nw = __funnelshift_r(A.z, B.z, lane);
        const uint32_t bw = __funnelshift_r(A.w, B.w, lane);
        for (uint32_t ti = 0; ti < tabs.n; ti++) {
            const KTableDev &T = tabs.t[ti];
            const uint32_t k = T.k;
            const uint32_t full = (k >= 32) ? 0xffffffffu : ((1u << k) - 1u);
            uint32_t beg = 0, end = 0;
            if (j + k <= b.nbases && (nw & full) == 0u && ((bw >> 1) & (full >> 1)) == 0u) {
                const uint32_t key = ((hiw & T.care) << k) | (low & T.care);
                if (T.direct) {
                    beg = __ldg(T.off + key);
                    end = __ldg(T.off + key + 1);
                } else {
                    // ranked: bitmap word and the rank of its first bit, then
                    // the key's rank among the present keys
                    const uint32_t w = key >> 5, bw = __ldg(T.bits + w);
                    if ((bw >> (key & 31u)) & 1u) {
                        const uint32_t r = __ldg(T.rank + w) + __popc(bw & ((1u << (key & 31u)) - 1u));
                        beg = __ldg(T.off + r);
                        end = __ldg(T.off + r + 1);
                    }
                }
            }
            // The warp's postings, flattened: lane l owns [exc_l, exc_l + cnt_l)
            // of the warp's total; each round every lane verifies one posting
            // (its owner found by a 5-step search over the lanes' offsets), so
            // lanes stay busy however unevenly the k-mers hit, and the warp
            // stays converged for ballot compaction of the hits.
            const uint32_t cnt = end - beg;
            uint32_t inc = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t v = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= static_cast<uint32_t>(o)) inc += v;
            }
            const uint32_t total = __shfl_sync(0xffffffffu, inc, 31);
            const uint32_t exc = inc - cnt;
            for (uint32_t base = 0; base < total; base += 32) {
                const uint32_t f = base + lane;
                // owner: the largest lane whose first flat index is <= f
                uint32_t own = 0;
#pragma unroll
                for (int stp = 16; stp > 0; stp >>= 1) {
                    const uint32_t c = own + stp;
                    if (__shfl_sync(0xffffffffu, exc, c) <= f) own = c;
                }
                const uint32_t own_beg = __shfl_sync(0xffffffffu, beg, own);
                const uint32_t own_exc = __shfl_sync(0xffffffffu, exc, own);
                bool hit = false;
                uint32_t id = 0, contig = 0, pos = 0, mm = 0;
                if (f < total) {
                    const uint64_t j = (blk << 5) + own;
                    const uint2 pm = __ldg(T.post + own_beg + (f - own_exc));   // posting and entry meta
                    const uint32_t e = pm.x >> 8, o = pm.x & 0xffu;
                    const uint32_t meta = pm.y;
                    // Issued together, since none depends on another: the
                    // entry's first word, and the directory entries and first
                    // two hi/lo words of the window the posting names.  The
                    // window starts at or before position j, so these reads
                    // stay in the batch (checked builds: an out-of-range
                    // directory entry reads as all special, and ref_word
                    // checks the words).
                    const uint64_t wa = (o <= j ? j - o : j) >> 5;
                    const uint4 q0 = __ldg(qt.words + static_cast<size_t>(e) * WMAX);
                    const bool dok = in_range(b, kBoundsDir, (wa >> 5) + 1, b.ndir);
                    const uint2 d0 = dok ? __ldg(b.dir + (wa >> 5)) : make_uint2(0xffffffffu, 0u);
                    const uint2 d1 = dok ? __ldg(b.dir + (wa >> 5) + 1) : make_uint2(0xffffffffu, 0u);
                    const bool hok = in_range(b, kBoundsWord, wa + 1, b.nwords);
                    const uint2 ha = hok ? __ldg(b.hl + wa) : make_uint2(0u, 0u);
                    const uint2 hb = hok ? __ldg(b.hl + wa + 1) : make_uint2(0u, 0u);
                    const uint32_t L = meta_L(meta), W = meta_W(meta);
                    const uint32_t se = entry_s(meta, s);
                    if (o <= j) {
                        const uint64_t p = j - o;
                        if (p + L <= b.nbases && p + L >= static_cast<uint64_t>(b.halo) + 1) {
                            ncand++;
                            const uint64_t w0 = p >> 5;
                            const uint32_t sh = static_cast<uint32_t>(p & 31);
                            uint32_t x[WMAX + 1];
                            uint32_t bnd = 0;
                            mm = 0;
                            // the window's words w0 .. w0 + W: hi/lo words, and
                            // the N / piece-start masks only when the directory
                            // marks one of them special
                            const bool spec = !hok || special_bits(d0.x, d1.x, w0, W + 1) != 0u;
                            uint4 cur = spec ? ref_word(b, w0) : make_uint4(ha.x, ha.y, 0u, 0u);
#pragma unroll
                            for (int w = 0; w < WMAX; w++) {
                                x[w] = 0;
                                if (w < static_cast<int>(W)) {
                                    uint4 nx;
                                    if (spec) {
                                        nx = ref_word(b, w0 + w + 1);
                                    } else if (w == 0) {
                                        nx = make_uint4(hb.x, hb.y, 0u, 0u);
                                    } else {
                                        const uint2 h2 = __ldg(b.hl + w0 + w + 1);
                                        nx = make_uint4(h2.x, h2.y, 0u, 0u);
                                    }
                                    const uint32_t rh = __funnelshift_r(cur.x, nx.x, sh);
                                    const uint32_t rl = __funnelshift_r(cur.y, nx.y, sh);
                                    const uint32_t rn = __funnelshift_r(cur.z, nx.z, sh);
                                    uint32_t rb = __funnelshift_r(cur.w, nx.w, sh);
                                    if (w == 0) rb &= ~1u;
                                    const uint4 q = w == 0 ? q0 : __ldg(qt.words + static_cast<size_t>(e) * WMAX + w);
                                    x[w] = ((rh ^ q.x) | (rl ^ q.y) | rn) & q.w;
                                    mm += __popc(x[w]);
                                    bnd |= rb & q.w;
                                    cur = nx;
                                    if (mm > se) break;  // over maxSubs already
                                }
                            }
                            x[WMAX] = 0;
                            if (bnd == 0u && mm <= se) {
                                // error-free k-mer offsets from the mismatch mask
                                const uint32_t last = L - k;  // largest offset
                                uint32_t nseed = 0, first = 0xffffffffu;
#pragma unroll
                                for (int w = 0; w < WMAX; w++) {
                                    if (w < static_cast<int>(W) && static_cast<uint32_t>(w) * 32 <= last) {
                                        // c bit i: a mismatch among the k-mer's cared
                                        // positions starting at offset base + i
                                        uint32_t c = 0;
                                        if (T.care == full) {
                                            // OR of the k shifts by doubling: after the loop
                                            // the shifts [0, span) are in; one more shift by
                                            // k - span <= span adds [k - span, k)
                                            uint64_t cc = x[w] | (static_cast<uint64_t>(x[w + 1]) << 32);
                                            uint32_t span = 1;
                                            while (2 * span <= k) {
                                                cc |= cc >> span;
                                                span *= 2;
                                            }
                                            if (span < k) cc |= cc >> (k - span);
                                            c = static_cast<uint32_t>(cc);
                                        } else {
                                            for (uint32_t i = 0; i < k; i++)
                                                if ((T.care >> i) & 1u) c |= __funnelshift_r(x[w], x[w + 1], i);
                                        }
                                        uint32_t valid = 0xffffffffu;
                                        const uint32_t base = static_cast<uint32_t>(w) * 32;
                                        if (last - base < 31) valid = (2u << (last - base)) - 1u;
                                        uint32_t S = ~c & valid;
                                        if (step > 1) {
                                            uint32_t sm = 0;
                                            for (uint32_t bi = 0; bi < 32; bi++)
                                                if ((base + bi) % step == 0) sm |= 1u << bi;
                                            S &= sm;
                                        }
                                        nseed += __popc(S);
                                        if (first == 0xffffffffu && S) first = base + __ffs(S) - 1;
                                    }
                                }
                                if (first == o && nseed >= __ldg(entry_minhits + e)) {
                                    hit = true;
                                    pidx = find_piece_from(b.pieces, b.npieces, p, pidx);
                                    const DevPiece pc = b.pieces[pidx];
                                    contig = pc.contig;
                                    pos = static_cast<uint32_t>(pc.contig_off + (p - pc.start));
                                    id = e;
                                }
                            }
                        }
                    }
                }
                wh.emit(sink, lane, hit, id >> 1, contig, pos, id & 1u, mm, nullptr);
            }
        }
    }
}

}  // namespace seed
}  // namespace ifa

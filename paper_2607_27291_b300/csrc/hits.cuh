// hits.cuh -- warp-ballot hit compaction into the device hit buffer.
//
// Hits are rare but can reach 10^8 per pass at high maxSubs, so no hit
// touches a global atomic on its own:
//  - a warp stages its hits in a private 32-entry shared-memory buffer
//    (slots assigned by ballot rank) and claims global slots with one
//    atomicAdd per 32 hits;
//  - the digest terms (count, sum, xor) are taken when a full or final
//    buffer is flushed, one staged hit per lane, so the hash runs with the
//    warp converged rather than once per hitting lane in divergent code;
//    each lane keeps its terms in registers, reduced over the warp once at
//    the end of the kernel;
//  - per-entry counts go to a per-CTA shared array, flushed once.
// The staging runs in count-only mode too (it feeds the digest); only the
// global writes are skipped there.
#pragma once
#include "ifa_internal.cuh"

namespace ifa {

// MULTI: hits go to per-request rings (serving); otherwise to the shared
// hit buffer with warp staging.  A compile-time choice, so the streaming and
// batch kernels carry no serving code.
template <bool MULTI>
struct WarpHitsT {
    ifa_hit *buf;          // this warp's 32 staged hits (shared memory)
    uint32_t n;            // staged count (warp-uniform)
    unsigned long long dcount, dsum, dxor;  // this lane's digest terms

    __device__ void init(ifa_hit *b) {
        buf = b;
        n = 0;
        dcount = dsum = dxor = 0;
    }

    __device__ void flush(const HitSink &s, uint32_t lane) {
        __syncwarp();
        if (n == 0) return;
        if (lane < n) {
            const ifa_hit h = buf[lane];
            const uint64_t v = hit_digest_item(h.query, h.contig, h.pos, h.strand, h.mismatches);
            dcount += 1;
            dsum += v;
            dxor ^= v;
        }
        if (s.count_only) {
            n = 0;
            __syncwarp();
            return;
        }
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(s.head, static_cast<unsigned long long>(n));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (lane < n) {
            unsigned long long idx = base + lane;
            if (idx < s.capacity) {
                const uint4 v = reinterpret_cast<const uint4 *>(buf)[lane];
                reinterpret_cast<uint4 *>(s.ring)[idx] = v;
            } else {
                *s.overflow = 1u;
            }
        }
        n = 0;
        __syncwarp();
    }

    // Called by the whole warp; lanes with `hit` report (q, contig, pos, strand, mm).
    // `entry_count` is a per-CTA shared counter that takes the warp's hit count
    // when all hitting lanes share one entry; otherwise (null) each hit adds one
    // to the query's global counter.
    __device__ void emit(const HitSink &s, uint32_t lane, bool hit, uint32_t q, uint32_t contig,
                         uint32_t pos, uint32_t strand, uint32_t mm, uint32_t *entry_count) {
        const uint32_t ballot = __ballot_sync(0xffffffffu, hit);
        if (ballot == 0) return;
        const uint32_t cnt = __popc(ballot);
        if constexpr (MULTI) {
            // each hit goes straight to its request's own ring and digest
            if (hit) {
                const RingDesc R = s.rings[s.q2r[q]];
                const uint32_t rq = q - R.qfirst;
                const uint64_t v = hit_digest_item(rq, contig, pos, strand, mm);
                atomicAdd(&R.counters[2], 1ull);
                atomicAdd(&R.counters[3], static_cast<unsigned long long>(v));
                atomicXor(&R.counters[4], static_cast<unsigned long long>(v));
                const unsigned long long idx = atomicAdd(&R.counters[0], 1ull);
                if (idx < R.cap) {
                    ifa_hit h;
                    h.query = rq;
                    h.contig = contig;
                    h.pos = pos;
                    h.strand = static_cast<uint8_t>(strand);
                    h.mismatches = static_cast<uint8_t>(mm > 255 ? 255 : mm);
                    h.reserved = 0;
                    R.ring[idx] = h;
                } else {
                    R.counters[1] = 1ull;
                }
                if (!entry_count) atomicAdd(&s.qcount[q], 1ull);
            }
            if (entry_count && lane == static_cast<uint32_t>(__ffs(ballot) - 1)) atomicAdd(entry_count, cnt);
            return;
        }
        if (hit && !entry_count) atomicAdd(&s.qcount[q], 1ull);
        if (entry_count && lane == static_cast<uint32_t>(__ffs(ballot) - 1))
            atomicAdd(entry_count, cnt);
        if (n + cnt > 32) flush(s, lane);
        if (hit) {
            const uint32_t r = __popc(ballot & ((1u << lane) - 1u));
            ifa_hit h;
            h.query = q;
            h.contig = contig;
            h.pos = pos;
            h.strand = static_cast<uint8_t>(strand);
            h.mismatches = static_cast<uint8_t>(mm > 255 ? 255 : mm);
            h.reserved = 0;
            buf[n + r] = h;
        }
        n += cnt;
        __syncwarp();
    }

    // End of kernel: flush staged hits and fold the digest terms of the warp.
    __device__ void finish(const HitSink &s, uint32_t lane) {
        flush(s, lane);
        unsigned long long c = dcount, su = dsum, x = dxor;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            c += __shfl_xor_sync(0xffffffffu, c, o);
            su += __shfl_xor_sync(0xffffffffu, su, o);
            x ^= __shfl_xor_sync(0xffffffffu, x, o);
        }
        if (lane == 0 && c) {
            atomicAdd(&s.digest[0], c);
            atomicAdd(&s.digest[1], su);
            atomicXor(&s.digest[2], x);
        }
    }
};

using WarpHits = WarpHitsT<false>;

}  // namespace ifa

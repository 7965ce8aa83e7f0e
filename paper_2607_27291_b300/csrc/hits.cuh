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

// Windows per brute-force block (32 lanes x 4 windows); an event's block
// index times this is the block's first window.
constexpr uint32_t kEventBlock = 128;

// MULTI: hits go to per-request rings (serving); otherwise to the shared
// hit buffer with warp staging.  A compile-time choice, so the streaming and
// batch kernels carry no serving code.
//
// Two ways in, sharing the warp's 32-slot buffer (never mixed: a brute-force
// block range starts by flushing hits and ends by flushing events):
//  - emit(): one hit per lane (seed scan), staged as ifa_hit;
//  - event(): the brute-force scan's (entry, lane, block) with a byte mask of
//    its hitting windows and their mismatch counts, staged as 16 bytes.  The
//    flush expands events into hits with the warp converged: piece lookup,
//    query id, digest, one slot claim per flush.
//
// Claims [base, base + n) of the shared buffer (warp-uniform): the first
// claim's position in the buffer, and the room left before the first claim
// that must be dropped (see HitSink).
struct Claim {
    unsigned long long pos;   // buffer position of claim `base`
    unsigned long long room;  // claims base .. base + room - 1 may be stored
};

__device__ __forceinline__ Claim claim_room(const HitSink &s, unsigned long long base) {
    Claim c;
    if (s.tail) {
        const unsigned long long t = *reinterpret_cast<const volatile unsigned long long *>(s.tail);
        c.room = base - t < s.capacity ? s.capacity - (base - t) : 0ull;
        c.pos = base % s.capacity;
    } else {
        c.room = base < s.capacity ? s.capacity - base : 0ull;
        c.pos = base;
    }
    return c;
}

// Record a dropped claim (any lane).
__device__ __forceinline__ void drop_claim(const HitSink &s, unsigned long long idx) {
    *s.overflow = 1u;
    if (s.ovf_at) atomicMin(s.ovf_at, idx);
}

template <bool MULTI>
struct WarpHitsT {
    ifa_hit *buf;          // this warp's 32 staged hits (shared memory, 16-byte aligned:
                           // hits and events move through it as uint4)
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
            const uint64_t v = hit_digest_item(h.query, h.contig, h.pos, h.strand, h.mismatches, h.clips);
            dcount += 1;
            dsum += v;
            dxor ^= v;
        }
        if (s.count_only) {
            n = 0;
            __syncwarp();
            return;
        }
        unsigned long long base = 0, pos = 0, room = 0;
        if (lane == 0) {
            base = atomicAdd(s.head, static_cast<unsigned long long>(n));
            const Claim c = claim_room(s, base);
            pos = c.pos;
            room = c.room;
        }
        base = __shfl_sync(0xffffffffu, base, 0);
        pos = __shfl_sync(0xffffffffu, pos, 0);
        room = __shfl_sync(0xffffffffu, room, 0);
        if (lane < n) {
            if (lane < room) {
                unsigned long long at = pos + lane;
                if (at >= s.capacity) at %= s.capacity;   // ring wrap (room <= capacity)
                const uint4 v = reinterpret_cast<const uint4 *>(buf)[lane];
                reinterpret_cast<uint4 *>(s.ring)[at] = v;
            } else if (lane == room) {
                drop_claim(s, base + lane);   // the first dropped claim of this flush
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
                         uint32_t pos, uint32_t strand, uint32_t mm, uint32_t *entry_count, uint32_t clips = 0) {
        const uint32_t ballot = __ballot_sync(0xffffffffu, hit);
        if (ballot == 0) return;
        const uint32_t cnt = __popc(ballot);
        if constexpr (MULTI) {
            // each hit goes straight to its request's own ring and digest
            if (hit) {
                ring_put(s, q, contig, pos, strand, mm, clips);
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
            h.clips = static_cast<uint16_t>(clips);
            buf[n + r] = h;
        }
        n += cnt;
        __syncwarp();
    }

    // One hit to a request's own ring and digest (serving).
    __device__ static void ring_put(const HitSink &s, uint32_t q, uint32_t contig, uint32_t pos, uint32_t strand,
                                    uint32_t mm, uint32_t clips = 0) {
        const RingDesc R = s.rings[s.q2r[q]];
        const uint32_t rq = q - R.qfirst;
        const uint64_t v = hit_digest_item(rq, contig, pos, strand, mm, clips);
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
            h.clips = static_cast<uint16_t>(clips);
            R.ring[idx] = h;
        } else {
            R.counters[1] = 1ull;
        }
    }

    // Stage one event per lane with has != 0: chunk-local entry e (< 2^16),
    // block index blk, hm = high bit of byte k set when window k of the lane
    // hits, d = byte k the window's mismatch count.
    __device__ void event(const Batch &b, const uint32_t *ids, uint32_t e0, uint32_t *cnt, const HitSink &s,
                          uint32_t lane, bool has, uint32_t e, uint32_t d, uint32_t blk, uint32_t hm) {
        const uint32_t ballot = __ballot_sync(0xffffffffu, has);
        if (ballot == 0) return;
        const uint32_t c = __popc(ballot);
        if (n + c > 32) flush_events(b, ids, e0, cnt, s, lane);
        if (has) {
            const uint32_t r = __popc(ballot & ((1u << lane) - 1u));
            reinterpret_cast<uint4 *>(buf)[n + r] = make_uint4(e | (lane << 16), d, blk, hm);
        }
        n += c;
        __syncwarp();
    }

    // Expand the staged events into hits (all lanes; lane i takes event i).
    __device__ void flush_events(const Batch &b, const uint32_t *ids, uint32_t e0, uint32_t *cnt,
                                 const HitSink &s, uint32_t lane) {
        __syncwarp();
        if (n == 0) return;
        uint4 ev = make_uint4(0u, 0u, 0u, 0u);
        if (lane < n) ev = reinterpret_cast<const uint4 *>(buf)[lane];
        n = 0;
        __syncwarp();
        uint32_t hm = ev.w & 0x80808080u;
        const uint32_t nh = __popc(hm);
        // this lane's claims are offsets off .. off + nh - 1 of the warp's
        // claim; offsets below `room` are stored, from buffer position `at`
        unsigned long long at = 0, room = 0;
        uint32_t off = 0;
        if (!MULTI && !s.count_only) {
            // one claim of global slots for the warp's hits
            uint32_t inc = nh;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= static_cast<uint32_t>(o)) inc += y;
            }
            const uint32_t total = __shfl_sync(0xffffffffu, inc, 31);
            unsigned long long base = 0, pos = 0;
            if (lane == 31 && total) {
                base = atomicAdd(s.head, static_cast<unsigned long long>(total));
                const Claim c = claim_room(s, base);
                pos = c.pos;
                room = c.room;
            }
            base = __shfl_sync(0xffffffffu, base, 31);
            pos = __shfl_sync(0xffffffffu, pos, 31);
            room = __shfl_sync(0xffffffffu, room, 31);
            off = inc - nh;
            at = pos + off;
            if (at >= s.capacity) at %= s.capacity;
            // the lane holding the warp's first claim without room reports it
            if (room < total && room >= off && room < off + nh) drop_claim(s, base + room);
        }
        if (nh) {
            const uint32_t e = ev.x & 0xffffu, el = ev.x >> 16;
            const uint32_t id = ids ? ids[e0 + e] : e0 + e;
            const uint32_t q = id >> 1, strand = id & 1u;
            atomicAdd(cnt + e, nh);
            const uint64_t p0 = static_cast<uint64_t>(ev.z) * kEventBlock + el;
            uint32_t pidx = 0xffffffffu;
            while (hm) {
                const uint32_t bit = static_cast<uint32_t>(__ffs(hm) - 1);  // 8 k + 7 for window k
                hm &= hm - 1u;
                const uint64_t p = p0 + 4u * (bit - 7u);                     // = p0 + 32 k
                if (pidx == 0xffffffffu) {
                    pidx = find_piece(b.pieces, b.npieces, p);
                } else {
                    while (pidx + 1 < b.npieces && b.pieces[pidx + 1].start <= p) pidx++;
                }
                const DevPiece pc = b.pieces[pidx];
                const uint32_t pos = static_cast<uint32_t>(pc.contig_off + (p - pc.start));
                const uint32_t mm = (ev.y >> (bit - 7u)) & 0xffu;
                if constexpr (MULTI) {
                    ring_put(s, q, pc.contig, pos, strand, mm);
                } else {
                    const uint64_t v = hit_digest_item(q, pc.contig, pos, strand, mm);
                    dcount += 1;
                    dsum += v;
                    dxor ^= v;
                    if (!s.count_only) {
                        if (off < room) {
                            ifa_hit h;
                            h.query = q;
                            h.contig = pc.contig;
                            h.pos = pos;
                            h.strand = static_cast<uint8_t>(strand);
                            h.mismatches = static_cast<uint8_t>(mm);
                            h.clips = 0;
                            s.ring[at] = h;
                        }
                        off++;
                        if (++at == s.capacity) at = 0;
                    }
                }
            }
        }
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

// The scan side of deferred hits (EventSink).  The same event() call as
// WarpHits, but the lanes with an event store it straight into the warp's
// open chunk of kEventChunk slots of the buffer, at their ballot ranks: no
// shared staging, no piece lookup, digest or ring claim in the scan loop,
// so the loop carries none of that code either.  A chunk is claimed with
// one atomic; the slots a warp leaves unused are zeroed (no window bit
// set), and the expansion skips them.  Slots at or past the capacity are
// not written (head then tells the expansion to rescan).
constexpr uint32_t kEventChunk = 128;   // > 32: one claim always fits a call's events

struct WarpEvents {
    EventSink es;
    unsigned long long at, end;   // the warp's open chunk [at, end) (warp-uniform)

    __device__ void init(const EventSink &s) {
        es = s;
        at = end = 0;
    }

    // nothing is staged for emit() (the brute-force loop only makes events)
    __device__ void flush(const HitSink &, uint32_t) {}

    __device__ __forceinline__ void event(const Batch &, const uint32_t *, uint32_t, uint32_t *, const HitSink &,
                                          uint32_t lane, bool has, uint32_t e, uint32_t d, uint32_t blk, uint32_t hm) {
        const uint32_t ballot = __ballot_sync(0xffffffffu, has);
        if (ballot == 0) return;
        const uint32_t c = __popc(ballot);
        if (at + c > end) claim(lane);
        if (has) {
            const unsigned long long i = at + __popc(ballot & ((1u << lane) - 1u));
            if (i < es.cap) es.buf[i] = make_uint4(e | (lane << 16), d, blk, hm);
        }
        at += c;
    }

    // Zero the open chunk's unused slots (all lanes).
    __device__ void close(uint32_t lane) {
        for (unsigned long long i = at + lane; i < end; i += 32)
            if (i < es.cap) es.buf[i] = make_uint4(0u, 0u, 0u, 0u);
        at = end;
    }

    __device__ void claim(uint32_t lane) {
        close(lane);
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(es.head, static_cast<unsigned long long>(kEventChunk));
        base = __shfl_sync(0xffffffffu, base, 0);
        at = base;
        end = base + kEventChunk;
    }

    // End of a block range.
    __device__ void flush_events(const Batch &, const uint32_t *, uint32_t, uint32_t *, const HitSink &,
                                 uint32_t lane) {
        close(lane);
    }
};

}  // namespace ifa

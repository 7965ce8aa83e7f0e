// ifa_internal.cuh -- device-side layouts shared by the kernels and the host engine.
//
// Reference layout in HBM ("2-bit store"): base i of a batch lives in bit
// (i & 31) of word i >> 5 of two planes, stored interleaved as one uint2 per
// 32 bases,
//   hl[w] = {hi plane (code >> 1), lo plane (code & 1)},
// with code A=0, C=1, T=2, G=3 (the byte's bits 1..2), so the complement of
// a base is code ^ 2.  That is 0.25 byte per base.  Two more planes exist
// only where they are not zero, in a sparse table:
//   N plane  1 where the byte is not A/C/G/T (its hi/lo bits are 0),
//   B plane  1 at the first base of every contig piece not at base 0.
// A word with a bit in either ("special": N runs and contig starts, a
// fraction of a percent of the words) has an entry {N mask, B mask} in exc;
// dir holds one {bitmap, base} per group of 32 words: bit j of the bitmap
// says word 32 g + j is special, and its entry is
//   exc[base + popc(bitmap & ((1 << j) - 1))].
// ref_word() rebuilds the four planes of any word; the scans stage only hl
// and read dir to send the few blocks with special words down their
// generic paths.
//
// Query table ("entries"): entry e = 2*q + t holds query q on strand t
// (t = 1: reverse complement, precomputed) as WMAX uint4 words
//   .x hi, .y lo,
//   .z care mask: 1 where position < L and the query base is A/C/G/T,
//   .w length mask: 1 where position < L,
// and a meta word L | W << 8 | nN << 16 | s_e << 24 (W = words used, nN =
// query Ns, which always count as mismatches, s_e = the entry's own maxSubs,
// capped at 255, used when a launch asks for per-entry thresholds).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include <utility>
#include <vector>

#include "ifa.h"

#include <nvtx3/nvToolsExt.h>

namespace ifa {

// An NVTX range over a host call (segment push, drain, batch run, serving
// step), so that a timeline (Nsight Systems, ncu's NVTX filters) shows the
// library's steps; header-only, no cost without a tool attached.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

constexpr int kWarp = 32;
constexpr uint32_t kSPerEntry = 0xffffffffu;  // launch threshold: use each entry's own s_e

__host__ __device__ inline uint32_t meta_L(uint32_t m) { return m & 0xffu; }
__host__ __device__ inline uint32_t meta_W(uint32_t m) { return (m >> 8) & 0xffu; }
__host__ __device__ inline uint32_t meta_nN(uint32_t m) { return (m >> 16) & 0xffu; }
// maxSubs of an entry under launch threshold s
__host__ __device__ inline uint32_t entry_s(uint32_t m, uint32_t s) { return s == kSPerEntry ? (m >> 24) : s; }

struct DevPiece {
    uint64_t start;        // first base of the piece in batch coordinates
    uint64_t contig_off;   // contig coordinate of `start`
    uint32_t contig;       // caller's contig id
    uint32_t last;         // 1: the contig ends with this piece (its end is the next piece's start)
};

// One request's own hit ring (serving): counters = {head, overflow, digest
// count, digest sum, digest xor}; hits carry query ids relative to qfirst.
struct RingDesc {
    ifa_hit *ring;
    unsigned long long *counters;
    unsigned long long cap;
    uint32_t qfirst;
    uint32_t pad;
};

// Grow-only device buffers addressed by slot, kept across rebuilds of a
// plan so that a rebuild allocates nothing once sizes have settled.  Reuse
// is ordered by the stream the plan's work runs on; growing frees the old
// buffer (cudaFree waits for the device).
struct DevBufs {
    std::vector<std::pair<void *, size_t>> b;

    void *get(size_t slot, size_t bytes, cudaError_t &e) {
        if (e != cudaSuccess) return nullptr;
        if (b.size() <= slot) b.resize(slot + 1, {nullptr, 0});
        auto &x = b[slot];
        if (x.second < bytes || !x.first) {
            const bool grew = x.first != nullptr;
            cudaFree(x.first);
            x = {nullptr, 0};
            // exact on first use; a quarter of headroom once a slot has had to grow
            size_t want = grew ? bytes + bytes / 4 : bytes;
            if (want < 256) want = 256;
            e = cudaMalloc(&x.first, want);
            if (e != cudaSuccess) return nullptr;
            x.second = want;
        }
        return x.first;
    }
    void release() {
        for (auto &x : b) cudaFree(x.first);
        b.clear();
    }
};

// Where hits go.  With `tail` set the buffer is a ring: claim idx (from
// `head`, which only grows) is stored at idx % capacity while
// idx - *tail < capacity, *tail being the count the host has drained; a
// claim that finds no room is dropped, raises `overflow` and lowers
// *ovf_at (the first dropped claim) so the host never drains past a hole.
// Without `tail` the buffer is linear: claims below capacity are stored.
struct HitSink {
    ifa_hit *ring;                 // hit buffer (may be null in count-only mode)
    unsigned long long *head;      // total hits claimed (can exceed capacity)
    unsigned long long capacity;
    unsigned long long *digest;    // [count, sum, xor]
    unsigned long long *qcount;    // per query
    uint32_t *overflow;            // set to 1 when a hit is dropped
    int count_only;
    // serving: query -> request slot and the slots' rings (null: one shared ring)
    const uint32_t *q2r = nullptr;
    const RingDesc *rings = nullptr;
    const unsigned long long *tail = nullptr;  // ring mode: hits drained so far (host-written)
    unsigned long long *ovf_at = nullptr;      // ring mode: first dropped claim (~0 when none)
};

// Deferred brute-force hits (streaming scan): the scan writes its window
// events -- one 16-byte record per (entry, lane, block) with a hit, the
// record the warp staging uses -- into this buffer, and a second kernel
// expands them into hits.  Slots are claimed a chunk per warp; `head`
// counts the slots claimed and exceeds `cap` when some did not fit, in
// which case the second kernel scans the launch's range again with the
// hits expanded in line.
struct EventSink {
    uint4 *buf;
    unsigned long long *head;
    unsigned long long cap;
};

struct QueryTable {
    const uint4 *words;      // entries x wmax
    const uint32_t *meta;    // entries
    const uint32_t *ids;     // optional: original entry id of each entry (null = identity)
    uint32_t n_entries;      // 2 * queries
    uint32_t wmax;
};

struct Batch {
    const uint2 *hl;          // hi/lo planes, >= nbases/32 + 16 words (padding words are N)
    const uint2 *dir;         // one {special bitmap, exc base} per 32 words, >= hl's words/32 + 2 groups
    const uint2 *exc;         // {N mask, B mask} of each special word
    uint64_t nbases;          // halo region + segment
    uint32_t halo;            // halo region length H; windows must end at or after base H
    const DevPiece *pieces;
    uint32_t npieces;
    // allocated sizes of hl, dir and exc, and the device word that records
    // the first out-of-range read (read only by IFA_BOUNDS_CHECK builds)
    uint64_t nwords, ndir, nexc;
    unsigned long long *bounds;
};

// Bounds-checked builds (-DIFA_BOUNDS_CHECK): every read of the packed
// reference checks its index; the first one out of range is recorded as
// kind << 56 | index in b.bounds (kinds below) and reads as an all-N word,
// so no window through it hits.  The host reports the word
// (ifa_bounds_check); nothing traps.  Default builds compile no check.
enum BoundsKind : uint32_t { kBoundsWord = 1, kBoundsDir = 2, kBoundsExc = 3 };
#ifdef IFA_BOUNDS_CHECK
__device__ __forceinline__ bool in_range(const Batch &b, uint32_t kind, uint64_t i, uint64_t n) {
    if (i < n) return true;
    if (b.bounds)
        atomicCAS(b.bounds, 0ull, (static_cast<unsigned long long>(kind) << 56) | (i & ((1ull << 56) - 1)));
    return false;
}
#else
__device__ __forceinline__ constexpr bool in_range(const Batch &, uint32_t, uint64_t, uint64_t) { return true; }
#endif

// The four planes {hi, lo, N, B} of word w.
__device__ __forceinline__ uint4 ref_word(const Batch &b, uint64_t w) {
    if (!in_range(b, kBoundsWord, w, b.nwords) || !in_range(b, kBoundsDir, w >> 5, b.ndir))
        return make_uint4(0u, 0u, 0xffffffffu, 0u);
    const uint2 a = __ldg(b.hl + w);
    const uint2 d = __ldg(b.dir + (w >> 5));
    const uint32_t bit = 1u << (w & 31u);
    uint32_t n = 0, s = 0;
    if (d.x & bit) {
        const uint64_t xi = d.y + __popc(d.x & (bit - 1u));
        if (!in_range(b, kBoundsExc, xi, b.nexc)) return make_uint4(0u, 0u, 0xffffffffu, 0u);
        const uint2 x = __ldg(b.exc + xi);
        n = x.x;
        s = x.y;
    }
    return make_uint4(a.x, a.y, n, s);
}

// Special bits of words w .. w + n - 1 (n <= 32) from two directory
// entries g = w >> 5 and g + 1; nonzero when any of them holds an N or a
// piece start.
__device__ __forceinline__ uint32_t special_bits(uint32_t d0, uint32_t d1, uint64_t w, uint32_t n) {
    const uint64_t both = static_cast<uint64_t>(d0) | (static_cast<uint64_t>(d1) << 32);
    const uint32_t x = static_cast<uint32_t>(both >> (w & 31u));
    return n >= 32u ? x : x & ((1u << n) - 1u);
}

// Device buffers of one packed reference (a streamed batch or the store).
struct RefBufs {
    uint2 *hl = nullptr;
    uint2 *nb = nullptr;      // scratch: {N, B} masks of the words being packed
    uint2 *dir = nullptr;
    uint2 *exc = nullptr;
    unsigned long long *exc_n = nullptr;  // [0] entries used, [1] set when an append ran out of room
    uint64_t words_cap = 0;   // hl words
    uint64_t nb_cap = 0;      // nb words
    uint64_t exc_cap = 0;     // exc entries
};

__host__ __device__ inline uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__host__ __device__ inline uint64_t hit_digest_item(uint32_t q, uint32_t contig, uint32_t pos,
                                                    uint32_t strand, uint32_t mm, uint32_t clips = 0) {
    uint64_t a = (static_cast<uint64_t>(q) << 32) | contig;
    uint64_t b = (static_cast<uint64_t>(pos) << 32) | (static_cast<uint64_t>(clips) << 16) | (strand << 8) | mm;
    return mix64(a ^ mix64(b));
}

// 2-bit code of an ASCII byte and whether it is a base.
__host__ __device__ inline uint32_t base_code(uint32_t c) { return (c >> 1) & 3u; }
__host__ __device__ inline bool is_base(uint32_t c) {
    uint32_t u = c & 0xDFu;
    return u == 'A' || u == 'C' || u == 'G' || u == 'T';
}

// Last piece whose start is <= p (pieces sorted by start, pieces[0].start == 0).
__device__ inline uint32_t find_piece(const DevPiece *pc, uint32_t n, uint64_t p) {
    uint32_t lo = 0, hi = n;  // answer in [lo, hi)
    while (hi - lo > 1) {
        uint32_t mid = (lo + hi) >> 1;
        if (pc[mid].start <= p) lo = mid; else hi = mid;
    }
    return lo;
}

// find_piece starting from a previous answer `hint` (a lane's last piece;
// ~0 for none): the hint itself when p lies inside it, else the search.
// Scans move forward through the pieces, so the hint usually holds.
__device__ inline uint32_t find_piece_from(const DevPiece *pc, uint32_t n, uint64_t p, uint32_t hint) {
    if (hint < n && pc[hint].start <= p && (hint + 1 == n || pc[hint + 1].start > p)) return hint;
    return find_piece(pc, n, p);
}

// ---------------------------------------------------------------- launchers
// (defined in the .cu files; all enqueue on `st`)

// Soft-clipped windows at contig ends (clip.cu), for entries [e_base, e_base + nent) of qt
// and pieces [p_lo, min(p_hi, b.npieces)) of b; a sink with rings sends each
// hit to its request's ring (serving).
cudaError_t launch_clip_scan(const Batch &b, const QueryTable &qt, uint32_t nent, uint32_t clip_pct, uint32_t s,
                             uint32_t lmax, const HitSink &sink, cudaStream_t st, uint32_t e_base = 0,
                             uint32_t p_lo = 0, uint32_t p_hi = 0xffffffffu);

// Tensor-core brute-force scan (scan_tc.cu): queries up to 64 bases.
uint32_t tc_lpad(uint32_t lmax);
bool tc_eligible(uint32_t lmax);
// Set the tensor-core kernel's attributes on the current device (once;
// before a stream capture that launches it).
cudaError_t tc_prepare();
// ids (may be null: identity) maps operand row e to the entry id it scans;
// rows of length 0 (padding) never hit.
cudaError_t launch_scan_tc(const Batch &b, const uint8_t *tcA, const uint32_t *meta, uint32_t nent, uint32_t lpad,
                           uint32_t s, const HitSink &sink, unsigned int *status, cudaStream_t st,
                           uint32_t withhold_first = 0, const uint32_t *ids = nullptr);

// ASCII -> hl words [0, nwords_padded) and their {N, B = 0} masks in nb.
cudaError_t launch_pack(const uint8_t *halo, uint32_t hlen, uint32_t H, const uint8_t *seg,
                        uint64_t slen, uint2 *hl, uint2 *nb, uint64_t nwords_padded, cudaStream_t st);
// B bits of the pieces starting among nb's nwords words (nb[0] holds base `first`).
cudaError_t launch_mark_pieces(const DevPiece *pieces, uint32_t n, uint64_t first, uint64_t nwords, uint2 *nb,
                               cudaStream_t st);
// Directory and exception entries of words [w0, w0 + n) from their masks nb[0 .. n); words of
// w0's group below w0 keep theirs (read back through the old directory entry).  Entries are
// taken from exc_n[0]; when they would pass exc_cap nothing of a group is written and exc_n[1]
// is set (grow exc, then run it again: the call is idempotent).
cudaError_t launch_build_dir(const uint2 *nb, uint64_t w0, uint64_t n, uint2 *dir, uint2 *exc, uint64_t exc_cap,
                             unsigned long long *exc_n, cudaStream_t st);
// Directory entries a reference of `words` hi/lo words needs (its groups,
// the group after the last that k_build_dir and k_pack_dir write, and one more that a
// reader of two neighbouring entries may touch).
inline uint64_t dir_entries(uint64_t words) { return (words + 31) / 32 + 3; }
// Allocate hl (words), nb (nb_words), dir and exc (exc_entries) and the
// two-word entry counter.
cudaError_t refbufs_alloc(RefBufs &R, uint64_t words, uint64_t nb_words, uint64_t exc_entries);
void refbufs_free(RefBufs &R);
// Pack one streamed batch into R: halo region + segment -> words [0, nwords),
// piece starts marked when `mark`, directory and exceptions built (R.exc_cap
// >= nwords).  Adds its kernel launches to *launches.
cudaError_t pack_batch(const RefBufs &R, const uint8_t *halo, uint32_t hlen, uint32_t H, const uint8_t *seg,
                       uint64_t slen, uint64_t nwords, const DevPiece *pieces, uint32_t npieces, bool mark,
                       cudaStream_t st, int *launches);
Batch make_batch(const RefBufs &R, uint64_t nbases, uint32_t halo, const DevPiece *pieces, uint32_t npieces);
// The device word of the first out-of-range read on the current device
// (IFA_BOUNDS_CHECK builds; nullptr otherwise).
unsigned long long *bounds_word();
cudaError_t launch_halo_update(const uint8_t *old_halo, uint32_t old_len, const uint8_t *seg,
                               uint64_t slen, uint32_t new_len, uint8_t *new_halo, cudaStream_t st);

// Brute-force scan of entries [e0, e1) of qt.  With an event sink the hits
// are deferred (two kernels, see EventSink); without one they are expanded
// in the scan loop (one kernel).
cudaError_t launch_scan_brute(const Batch &b, const QueryTable &qt, uint32_t e0, uint32_t e1,
                              uint32_t max_subs, uint32_t lmin, uint32_t lmax, const HitSink &sink,
                              cudaStream_t st, int *launches, const EventSink *es = nullptr);
uint32_t scan_brute_chunk_entries(uint32_t wmax);

cudaError_t launch_minhits(const uint32_t *dL, const uint32_t *dsubs, const uint32_t *dk,
                           uint32_t nbins, uint32_t step, uint32_t mask_w, uint32_t max_clips,
                           uint32_t num, uint32_t den, uint32_t trials, uint64_t seed,
                           uint32_t *dhist_scratch, uint32_t hist_stride, uint32_t *dout,
                           cudaStream_t st);

}  // namespace ifa

// noalloc.cu -- brute-force scan of one reference chunk without allocating.
//
// Some callers cannot call cudaMalloc: code that runs where a framework's
// caching allocator already owns the device memory and any allocation
// outside it fails, or a host that must not allocate at a given point (a
// serving loop with a fixed memory plan).  For them this file offers one
// entry point that takes the caller's input and output buffers and keeps
// all of its scratch -- the packed reference planes, the encoded query
// table, the piece table and the per-query counts -- in a file-scope
// device array of fixed size (about 18 MB).
//
// When the array takes its device memory: the array belongs to this file's
// CUDA module, and the runtime loads a module into a context when it is
// first used (lazy loading, CUDA's default), so on each device the array is
// placed by the first call here -- its cudaGetSymbolAddress -- and then stays
// until the process exits.  A call with nq = 0 does only that set-up; make it
// once per device at start-up, before a caching allocator reserves the
// device's memory and before any stream capture.  (With
// CUDA_MODULE_LOADING=EAGER the array is placed when the context is made.)
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "ifa_internal.cuh"

namespace ifa {
void set_global_error(const std::string &msg);
}

using namespace ifa;

namespace {

constexpr uint64_t kNaMaxBases = 32ull << 20;  // reference bytes per call
constexpr uint32_t kNaMaxQueries = 256;        // queries per call
constexpr uint32_t kNaMaxPieces = 1u << 15;    // contigs per call
constexpr uint32_t kNaWmax = 8;                // words per query entry (255 bp)
constexpr uint64_t kNaWords = kNaMaxBases / 32 + 16;

// Byte offsets of the parts inside the scratch array (256-aligned each):
// the packed reference (2-bit words, directory, exception entries and
// their counter; a streamed batch packs in one pass, with no mask
// scratch), the query table, the piece table and the per-query counts.
constexpr uint64_t align256(uint64_t x) { return (x + 255) & ~uint64_t(255); }
constexpr uint64_t kOffHl = 0;
constexpr uint64_t kOffDir = align256(kOffHl + kNaWords * sizeof(uint2));
constexpr uint64_t kOffExc = align256(kOffDir + ((kNaWords + 31) / 32 + 3) * sizeof(uint2));
constexpr uint64_t kOffExcN = align256(kOffExc + kNaWords * sizeof(uint2));
constexpr uint64_t kOffQWords = align256(kOffExcN + 2 * sizeof(unsigned long long));
constexpr uint64_t kOffQMeta = align256(kOffQWords + 2ull * kNaMaxQueries * kNaWmax * sizeof(uint4));
constexpr uint64_t kOffPieces = align256(kOffQMeta + 2ull * kNaMaxQueries * sizeof(uint32_t));
constexpr uint64_t kOffQCount = align256(kOffPieces + uint64_t(kNaMaxPieces) * sizeof(DevPiece));
constexpr uint64_t kScratchBytes = align256(kOffQCount + kNaMaxQueries * sizeof(unsigned long long));

// The scratch: one array, shared by every call on a device.
static __device__ __align__(256) unsigned char g_na_scratch[kScratchBytes];

// Device address of g_na_scratch per device (host code cannot use the
// symbol itself: on the host it names a stand-in, not device memory).
std::mutex g_na_mutex;
unsigned char *g_na_addr[64] = {nullptr};

ifa_status na_fail(ifa_status st, const std::string &msg) {
    set_global_error(msg);
    return st;
}

void na_encode(const uint8_t *q, uint32_t L, bool rc, uint32_t wmax, uint4 *out, uint32_t *meta) {
    for (uint32_t j = 0; j < wmax; j++) out[j] = make_uint4(0, 0, 0, 0);
    uint32_t nN = 0;
    for (uint32_t i = 0; i < L; i++) {
        const uint32_t c = rc ? q[L - 1 - i] : q[i];
        const uint32_t w = i >> 5, bit = 1u << (i & 31);
        if (is_base(c)) {
            uint32_t code = base_code(c);
            if (rc) code ^= 2u;
            if (code >> 1) out[w].x |= bit;
            if (code & 1u) out[w].y |= bit;
            out[w].z |= bit;
        } else {
            nN++;
        }
        out[w].w |= bit;
    }
    *meta = L | (((L + 31) / 32) << 8) | (nN << 16);
}

}  // namespace

extern "C" ifa_status ifa_scan_brute_noalloc(int32_t device, const uint8_t *const *queries,
                                             const uint32_t *qlens, uint32_t nq,
                                             const uint8_t *ref_device, uint64_t len,
                                             const ifa_piece *pieces, uint32_t n_pieces,
                                             uint32_t max_subs, ifa_hit *hits_device,
                                             uint64_t hit_capacity, uint64_t *counters_device,
                                             uint64_t *per_query_counts_device, void *stream) {
    if (device < 0 || device >= 64) return na_fail(IFA_ERR_INVALID_ARG, "ifa_scan_brute_noalloc: device ordinal");
    // ---- arguments (host only; nothing is enqueued before they pass)
    const bool setup_only = nq == 0;
    if (nq > kNaMaxQueries)
        return na_fail(IFA_ERR_INVALID_ARG, "ifa_scan_brute_noalloc: at most 256 queries per call (0: set-up only)");
    if (!setup_only && (!queries || !qlens))
        return na_fail(IFA_ERR_INVALID_ARG, "ifa_scan_brute_noalloc: queries/qlens is NULL");
    for (uint32_t i = 0; i < nq; i++)
        if (!queries[i] || qlens[i] == 0 || qlens[i] > IFA_MAX_QUERY_LEN)
            return na_fail(IFA_ERR_INVALID_ARG, "ifa_scan_brute_noalloc: query length must be in 1..255");
    if (!setup_only && (len == 0 || len > kNaMaxBases))
        return na_fail(IFA_ERR_INVALID_ARG,
                       "ifa_scan_brute_noalloc: reference length must be in 1..33554432 bytes (32 MiB)");
    if (!setup_only && (n_pieces == 0 || n_pieces > kNaMaxPieces))
        return na_fail(IFA_ERR_INVALID_ARG, "ifa_scan_brute_noalloc: 1 to 32768 contigs per call");
    if (!setup_only && (!ref_device || !pieces || !hits_device || !counters_device || hit_capacity == 0))
        return na_fail(IFA_ERR_INVALID_ARG, "ifa_scan_brute_noalloc: NULL buffer or zero hit capacity");
    // hits are written 16 bytes at a time and the counters take 64-bit atomics
    if (reinterpret_cast<uintptr_t>(hits_device) % 16 != 0 || reinterpret_cast<uintptr_t>(counters_device) % 8 != 0 ||
        reinterpret_cast<uintptr_t>(per_query_counts_device) % 8 != 0)
        return na_fail(IFA_ERR_INVALID_ARG,
                       "ifa_scan_brute_noalloc: hits_device must be 16-byte aligned, counters_device and "
                       "per_query_counts_device 8-byte aligned");
    uint64_t at = 0;
    for (uint32_t i = 0; i < (setup_only ? 0u : n_pieces); i++) {
        const ifa_piece &p = pieces[i];
        if (p.start != at || p.len == 0 || !p.last || p.offset_in_contig != 0 || p.len > 0xffffffffull)
            return na_fail(IFA_ERR_INVALID_ARG,
                           "ifa_scan_brute_noalloc: pieces must be whole contigs, contiguous from 0");
        if (i > 0 && p.contig <= pieces[i - 1].contig)
            return na_fail(IFA_ERR_INVALID_ARG, "ifa_scan_brute_noalloc: contig ids must increase");
        at += p.len;
    }
    if (!setup_only && at != len)
        return na_fail(IFA_ERR_INVALID_ARG, "ifa_scan_brute_noalloc: pieces must cover the reference");
    // a window has at most 255 bases, so any maxSubs of 255 or more reports every
    // window; clamping keeps the value clear of the per-entry launch sentinel
    const uint32_t s_launch = max_subs < 255u ? max_subs : 255u;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // work on `device`; the calling thread's current device is put back on return
    int prev = 0;
    cudaError_t e = cudaGetDevice(&prev);
    if (e != cudaSuccess) return na_fail(IFA_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (prev != device) {
        e = cudaSetDevice(device);
        if (e != cudaSuccess) return na_fail(IFA_ERR_CUDA, std::string("cudaSetDevice: ") + cudaGetErrorString(e));
    }
    struct RestoreDevice {
        int dev;
        bool on;
        ~RestoreDevice() {
            if (on) cudaSetDevice(dev);
        }
    } restore{prev, prev != device};
    if (!setup_only) {
        // the call copies from host memory that is freed on return, so a
        // captured graph could not replay it
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        const cudaError_t ce = cudaStreamIsCapturing(st, &cap);
        if (ce != cudaSuccess || cap != cudaStreamCaptureStatusNone) {
            if (ce != cudaSuccess) cudaGetLastError();
            return na_fail(IFA_ERR_INVALID_ARG,
                           "ifa_scan_brute_noalloc: the stream is being captured; calls cannot be captured");
        }
    }

    // ---- set-up, once per device, with that device current
    unsigned char *base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_na_mutex);
        if (!g_na_addr[device]) {
            void *ptr = nullptr;
            e = cudaGetSymbolAddress(&ptr, g_na_scratch);
            if (e != cudaSuccess)
                return na_fail(IFA_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            g_na_addr[device] = static_cast<unsigned char *>(ptr);
        }
        base = g_na_addr[device];
    }
    if (setup_only) return IFA_OK;
    RefBufs ref;
    ref.hl = reinterpret_cast<uint2 *>(base + kOffHl);
    ref.nb = nullptr;
    ref.dir = reinterpret_cast<uint2 *>(base + kOffDir);
    ref.exc = reinterpret_cast<uint2 *>(base + kOffExc);
    ref.exc_n = reinterpret_cast<unsigned long long *>(base + kOffExcN);
    ref.words_cap = ref.exc_cap = kNaWords;
    ref.nb_cap = 0;
    uint4 *qwords = reinterpret_cast<uint4 *>(base + kOffQWords);
    uint32_t *qmeta = reinterpret_cast<uint32_t *>(base + kOffQMeta);
    DevPiece *dpieces = reinterpret_cast<DevPiece *>(base + kOffPieces);
    unsigned long long *qcount = reinterpret_cast<unsigned long long *>(base + kOffQCount);

    // ---- host-side encoding of the queries and the piece table
    uint32_t lmax = 0;
    for (uint32_t i = 0; i < nq; i++) lmax = qlens[i] > lmax ? qlens[i] : lmax;
    uint32_t wmax = 1;
    while (wmax * 32 < lmax) wmax <<= 1;
    const uint32_t ne = 2 * nq;
    std::vector<uint4> hw(static_cast<size_t>(ne) * wmax);
    std::vector<uint32_t> hm(ne);
    for (uint32_t q = 0; q < nq; q++)
        for (uint32_t t = 0; t < 2; t++)
            na_encode(queries[q], qlens[q], t == 1, wmax, &hw[static_cast<size_t>(2 * q + t) * wmax], &hm[2 * q + t]);
    std::vector<DevPiece> hp(n_pieces);
    for (uint32_t i = 0; i < n_pieces; i++) {
        hp[i].start = pieces[i].start;
        hp[i].contig_off = 0;
        hp[i].contig = pieces[i].contig;
        hp[i].last = 1;
    }

    // ---- enqueue: copies into the scratch, zeroing, pack, scan
    auto ck = [&](cudaError_t r) {
        if (e == cudaSuccess && r != cudaSuccess) e = r;
    };
    ck(cudaMemcpyAsync(qwords, hw.data(), hw.size() * sizeof(uint4), cudaMemcpyHostToDevice, st));
    ck(cudaMemcpyAsync(qmeta, hm.data(), hm.size() * sizeof(uint32_t), cudaMemcpyHostToDevice, st));
    ck(cudaMemcpyAsync(dpieces, hp.data(), hp.size() * sizeof(DevPiece), cudaMemcpyHostToDevice, st));
    unsigned long long *qc = per_query_counts_device ? reinterpret_cast<unsigned long long *>(per_query_counts_device)
                                                     : qcount;
    ck(cudaMemsetAsync(qc, 0, nq * sizeof(unsigned long long), st));
    ck(cudaMemsetAsync(counters_device, 0, 5 * sizeof(uint64_t), st));
    const uint64_t nwords = (len + 31) / 32 + 16;
    if (e == cudaSuccess) e = pack_batch(ref, nullptr, 0, 0, ref_device, len, nwords, dpieces, n_pieces, true, st, nullptr);
    const Batch b = make_batch(ref, len, 0, dpieces, n_pieces);
    QueryTable qt;
    qt.words = qwords;
    qt.meta = qmeta;
    qt.ids = nullptr;
    qt.n_entries = ne;
    qt.wmax = wmax;
    HitSink sink;
    sink.ring = hits_device;
    sink.head = reinterpret_cast<unsigned long long *>(counters_device);
    sink.capacity = hit_capacity;
    sink.overflow = reinterpret_cast<uint32_t *>(counters_device + 1);
    sink.digest = reinterpret_cast<unsigned long long *>(counters_device + 2);
    sink.qcount = qc;
    sink.count_only = 0;
    uint32_t cap = scan_brute_chunk_entries(wmax) & ~1u;
    if (cap < 2) cap = 2;
    for (uint32_t e0 = 0; e0 < ne && e == cudaSuccess; e0 += cap) {
        const uint32_t e1 = e0 + cap < ne ? e0 + cap : ne;
        uint32_t lo = 0xffffffffu, hi = 0;
        for (uint32_t i = e0; i < e1; i++) {
            const uint32_t L = hm[i] & 0xffu;
            lo = L < lo ? L : lo;
            hi = L > hi ? L : hi;
        }
        ck(launch_scan_brute(b, qt, e0, e1, s_launch, lo, hi, sink, st, nullptr));
    }
    if (e != cudaSuccess)
        return na_fail(IFA_ERR_CUDA, std::string("ifa_scan_brute_noalloc: ") + cudaGetErrorString(e));
    return IFA_OK;
}

// capi.cu -- the handle-based C ABI (include/ifa.h) and its streaming engine.
//
// One handle = one device, one query set, one streamed reference pass at a
// time.  Segments are double-buffered: while the compute stream packs and
// scans segment k, the copy stream moves segment k+1 from host to device;
// a slot is reused only after the compute that read it has finished
// (event per slot).  Memory on the device is bounded by the segment size,
// not by the reference size (Methods, "Memory Management").
#include <algorithm>
#include <cstdio>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "handle.cuh"

using namespace ifa;

namespace {

thread_local std::string g_err = "no error";

constexpr uint32_t kHaloCap = 256;   // >= halo region H = 32 * ceil((IFA_MAX_QUERY_LEN - 1) / 32)
constexpr uint64_t kWordPad = 16;    // padding words after the last packed word (packed as N)

}  // namespace

namespace {

ifa_status fail(ifa_handle *h, ifa_status st, const std::string &msg) {
    if (h) h->err = msg; else g_err = msg;
    return st;
}

ifa_status fail_cuda(ifa_handle *h, const char *what, cudaError_t e) {
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    return fail(h, cuda_status(e), m);
}

#define CK(h, call)                                           \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return fail_cuda((h), #call, e_); \
    } while (0)

}  // namespace

namespace ifa {

void encode_entry(const std::string &q, bool rc, uint32_t wmax, uint32_t s_e, uint4 *out, uint32_t *meta) {
    const uint32_t L = static_cast<uint32_t>(q.size());
    for (uint32_t j = 0; j < wmax; j++) out[j] = make_uint4(0, 0, 0, 0);
    uint32_t nN = 0;
    for (uint32_t i = 0; i < L; i++) {
        const uint32_t c = static_cast<uint8_t>(rc ? q[L - 1 - i] : q[i]);
        const uint32_t w = i >> 5, bit = 1u << (i & 31);
        if (is_base(c)) {
            uint32_t code = base_code(c);
            if (rc) code ^= 2u;  // complement: A<->T, C<->G
            if (code >> 1) out[w].x |= bit;
            if (code & 1u) out[w].y |= bit;
            out[w].z |= bit;
        } else {
            nN++;
        }
        out[w].w |= bit;
    }
    *meta = L | (((L + 31) / 32) << 8) | (nN << 16) | ((s_e > 255u ? 255u : s_e) << 24);
}

ifa_status upload_queries(ifa_handle *h) {
    if (!h->qdirty) return IFA_OK;
    const uint32_t nq = static_cast<uint32_t>(h->qs.size());
    uint32_t wneed = (h->lmax + 31) / 32;
    uint32_t w = 1;
    while (w < wneed) w <<= 1;
    h->wmax = w;
    const uint32_t ne = 2 * nq;
    std::vector<uint4> &words = h->qwords_host;
    words.assign(static_cast<size_t>(ne) * w, make_uint4(0, 0, 0, 0));
    h->qmeta_host.assign(ne, 0);
    for (uint32_t q = 0; q < nq; q++)
        for (uint32_t t = 0; t < 2; t++)
            encode_entry(h->qs[q], t == 1, w, q < h->qs_s.size() ? h->qs_s[q] : 0u,
                         &words[static_cast<size_t>(2 * q + t) * w], &h->qmeta_host[2 * q + t]);
    cudaFree(h->d_qwords);
    cudaFree(h->d_qmeta);
    h->d_qwords = nullptr;
    h->d_qmeta = nullptr;
    CK(h, cudaMalloc(&h->d_qwords, words.size() * sizeof(uint4)));
    CK(h, cudaMalloc(&h->d_qmeta, ne * sizeof(uint32_t)));
    CK(h, cudaMemcpyAsync(h->d_qwords, words.data(), words.size() * sizeof(uint4), cudaMemcpyHostToDevice, h->stream));
    CK(h, cudaMemcpyAsync(h->d_qmeta, h->qmeta_host.data(), ne * sizeof(uint32_t), cudaMemcpyHostToDevice, h->stream));
    // entry chunks that fit the scan kernel's shared-memory budget
    uint32_t cap = scan_brute_chunk_entries(w) & ~1u;
    if (cap < 2) cap = 2;
    h->chunks.clear();
    for (uint32_t e0 = 0; e0 < ne; e0 += cap) {
        Chunk c{e0, std::min(ne, e0 + cap), 0xffffffffu, 0};
        for (uint32_t e = c.e0; e < c.e1; e++) {
            uint32_t L = h->qmeta_host[e] & 0xffu;
            c.lmin = std::min(c.lmin, L);
            c.lmax = std::max(c.lmax, L);
        }
        h->chunks.push_back(c);
    }
    // tensor-core operand when the brute-force kernel may use it
    cudaFree(h->d_tcA);
    h->d_tcA = nullptr;
    h->tc_lpad = 0;
    if (h->cfg.brute_kernel != IFA_BRUTE_POPC && tc_eligible(h->lmax)) {
        std::vector<uint8_t> op;
        h->tc_lpad = tc_lpad(h->lmax);
        tc_operand(h->qs, h->tc_lpad, op);
        CK(h, cudaMalloc(&h->d_tcA, op.size()));
        CK(h, cudaMemcpyAsync(h->d_tcA, op.data(), op.size(), cudaMemcpyHostToDevice, h->stream));
    }
    h->qdirty = false;
    h->idx.invalidate();
    h->batch.plan_valid = false;
    return IFA_OK;
}

}  // namespace ifa

namespace {

ifa_status ensure_pieces(ifa_handle *h, int slot, uint32_t n) {
    if (n <= h->pieces_cap[slot]) return IFA_OK;
    uint32_t cap = std::max<uint32_t>(n, 2 * h->pieces_cap[slot]);
    cudaFree(h->d_pieces[slot]);
    cudaFreeHost(h->h_pieces[slot]);
    h->d_pieces[slot] = nullptr;
    h->h_pieces[slot] = nullptr;
    h->pieces_cap[slot] = 0;
    CK(h, cudaMalloc(&h->d_pieces[slot], static_cast<size_t>(cap) * sizeof(DevPiece)));
    CK(h, cudaHostAlloc(&h->h_pieces[slot], static_cast<size_t>(cap) * sizeof(DevPiece), cudaHostAllocDefault));
    h->pieces_cap[slot] = cap;
    return IFA_OK;
}

// The mode of the streaming pass: the explicit one; for IFA_MODE_AUTO the
// paper's rule by query count when auto_crossover > 0, else the measured-
// rate model (rates taken once per handle and maxSubs on the calibration
// sequence, before the stream's first segment is scanned).
ifa_status resolve_mode(ifa_handle *h, ifa_mode *out) {
    if (h->mode != IFA_MODE_AUTO) {
        *out = h->mode;
        return IFA_OK;
    }
    if (h->cfg.auto_crossover) {
        *out = h->qs.size() >= h->cfg.auto_crossover ? IFA_MODE_INDEXED : IFA_MODE_BRUTE;
        return IFA_OK;
    }
    const uint32_t s_key = h->per_query_s ? kSPerEntry : h->max_subs;
    if (h->auto_mode == IFA_MODE_AUTO || h->auto_s != s_key) {
        const std::vector<uint32_t> svec =
            h->per_query_s ? h->qs_s : std::vector<uint32_t>(h->qs.size(), h->max_subs);
        Rates r;
        ifa_status st = rates_on_random(h, h->qs, svec, r);
        if (st != IFA_OK) return st;
        ifa_mode m = IFA_MODE_BRUTE;
        st = choose_mode(h, r, h->qs, svec, &m);
        if (st != IFA_OK) return st;
        h->auto_rates = r;
        h->auto_s = s_key;
        h->auto_mode = m;
    }
    *out = h->auto_mode;
    return IFA_OK;
}

HitSink make_sink(const ifa_handle *h) {
    HitSink s;
    s.ring = h->d_ring;
    s.head = h->d_head;
    s.capacity = h->cfg.count_only ? 0 : h->cfg.hit_capacity;
    s.digest = h->d_digest;
    s.qcount = h->d_qcount;
    s.overflow = h->d_overflow;
    s.count_only = h->cfg.count_only ? 1 : 0;
    s.ovf_at = h->d_head + 1;
    s.tail = h->d_head + 2;
    return s;
}

// Fold the completed segment marks, oldest first (all of them, waiting, when
// `wait`).
ifa_status collect_marks(ifa_handle *h, bool wait) {
    size_t i = 0;
    for (; i < h->marks_pending.size(); i++) {
        const int k = h->marks_pending[i];
        cudaError_t e = wait ? cudaEventSynchronize(h->ev_mark[k]) : cudaEventQuery(h->ev_mark[k]);
        if (e == cudaErrorNotReady) break;
        if (e != cudaSuccess) return fail_cuda(h, "segment mark", e);
        h->done_head = h->h_marks[2 * k];
        h->done_ovf = h->h_marks[2 * k + 1];
    }
    h->marks_pending.erase(h->marks_pending.begin(), h->marks_pending.begin() + i);
    return IFA_OK;
}

// Copy ring claims [tail, min(end, tail + cap)) to out (host) on the drain
// stream, then advance the device tail (after the copies, same stream) so
// producers may reuse the slots.  Waits for the drain stream only.
ifa_status drain_span(ifa_handle *h, ifa_hit *out, uint64_t cap, uint64_t end, uint64_t *n_out) {
    *n_out = 0;
    if (end <= h->tail || cap == 0) return IFA_OK;
    const uint64_t C = h->cfg.hit_capacity;
    const uint64_t take = std::min<uint64_t>(end - h->tail, cap);
    const uint64_t pos = h->tail % C;
    const uint64_t n1 = std::min<uint64_t>(take, C - pos);
    CK(h, cudaMemcpyAsync(out, h->d_ring + pos, n1 * sizeof(ifa_hit), cudaMemcpyDeviceToHost, h->drain_stream));
    if (take > n1)
        CK(h, cudaMemcpyAsync(out + n1, h->d_ring, (take - n1) * sizeof(ifa_hit), cudaMemcpyDeviceToHost,
                              h->drain_stream));
    h->tail += take;
    unsigned long long *ht = h->h_marks + 2 * ifa_handle::kMarks;
    *ht = h->tail;
    CK(h, cudaMemcpyAsync(h->d_head + 2, ht, sizeof(unsigned long long), cudaMemcpyHostToDevice, h->drain_stream));
    CK(h, cudaStreamSynchronize(h->drain_stream));
    *n_out = take;
    return IFA_OK;
}

// Reset the ring counters on the compute stream (head 0, none dropped, tail 0).
ifa_status reset_ring(ifa_handle *h) {
    CK(h, cudaMemsetAsync(h->d_head, 0, 3 * sizeof(unsigned long long), h->stream));
    CK(h, cudaMemsetAsync(h->d_head + 1, 0xff, sizeof(unsigned long long), h->stream));
    h->tail = 0;
    h->done_head = 0;
    h->done_ovf = ~0ull;
    h->marks_pending.clear();
    return IFA_OK;
}

ifa_status sync_all(ifa_handle *h) {
    CK(h, cudaStreamSynchronize(h->copy_stream));
    CK(h, cudaStreamSynchronize(h->stream));
    return IFA_OK;
}

// Start/stop a timed region around scan kernels on the compute stream.
ifa_status prof_begin(ifa_handle *h, cudaEvent_t *stop_out) {
    *stop_out = nullptr;
    if (!h->cfg.profile) return IFA_OK;
    std::pair<cudaEvent_t, cudaEvent_t> ev{nullptr, nullptr};
    if (!h->ev_free.empty()) {
        ev = h->ev_free.back();
        h->ev_free.pop_back();
    } else {
        CK(h, cudaEventCreate(&ev.first));
        CK(h, cudaEventCreate(&ev.second));
    }
    CK(h, cudaEventRecord(ev.first, h->stream));
    h->ev_pending.push_back(ev);
    *stop_out = ev.second;
    return IFA_OK;
}

ifa_status prof_end(ifa_handle *h, cudaEvent_t stop, int launches) {
    if (!stop) return IFA_OK;
    CK(h, cudaEventRecord(stop, h->stream));
    h->stats.scan_launches += launches;
    return IFA_OK;
}

// Fold finished timed regions into the statistics (after a stream sync).
ifa_status prof_collect(ifa_handle *h) {
    for (auto &ev : h->ev_pending) {
        float ms = 0.f;
        CK(h, cudaEventElapsedTime(&ms, ev.first, ev.second));
        h->stats.scan_ns += static_cast<uint64_t>(ms * 1e6);
        h->ev_free.push_back(ev);
    }
    h->ev_pending.clear();
    return IFA_OK;
}

}  // namespace

namespace ifa {
// Record a failure for ifa_last_error(NULL) from entry points in other files.
void set_global_error(const std::string &msg) { g_err = msg; }
}  // namespace ifa

namespace {

// The brute-force kernel of a pass: the tensor cores when forced, or (auto)
// from 64 entries (32 queries) on, where one half-filled 128-entry tile
// already matches the popcount kernel (measured on B300: 1.04x at 32
// queries, 2.0x from 64 queries on, 256 Mbp, maxSubs 4), as long as hits
// are sparse (below).
constexpr uint32_t kTcAutoEntries = 64;
constexpr uint32_t kTcMaxQueryBases = 64;  // the tensor-core operand holds queries up to 64 bases

// The tensor-core kernel tests whole 64-window chunks and takes every hit of
// a flagged chunk one by one, so it suits sparse hits.  Probability that a
// random window of a query of L bases (independent uniform bases, a base
// matching with probability 1/4) has at most s mismatches.
double random_window_hit_rate(uint32_t L, uint32_t s) {
    if (s >= L) return 1.0;
    double term = std::pow(0.25, static_cast<double>(L));  // i = 0 mismatches
    double sum = term;
    for (uint32_t i = 1; i <= s; i++) {
        term *= 3.0 * static_cast<double>(L - i + 1) / static_cast<double>(i);
        sum += term;
    }
    return sum;
}

// Above this mean hit rate the popcount kernel's per-hit path wins
// (256 Mbp, 2048 queries: tensor cores 1.35-1.6x faster at a mean rate of
// 0.7-0.8e-4, 0.6x at 1.3e-3).
constexpr double kTcAutoMaxHitRate = 2e-4;

bool use_tensor_cores(const ifa_handle *h) {
    if (!h->d_tcA) return false;
    if (h->cfg.brute_kernel == IFA_BRUTE_TENSOR) return true;
    // per-query thresholds: judged at the largest (the densest hits)
    uint32_t s = h->max_subs;
    if (h->per_query_s)
        s = h->qs_s.empty() ? 0u : *std::max_element(h->qs_s.begin(), h->qs_s.end());
    return h->cfg.brute_kernel == IFA_BRUTE_AUTO && tc_auto_choice(h->qs, 0, static_cast<uint32_t>(h->qs.size()), s);
}

// The streaming indexed plan and tables for the current thresholds: one
// maxSubs for all queries, or each query's own (ifa_set_query_max_subs).
ifa_status stream_indexed_prepare(ifa_handle *h) {
    if (!h->per_query_s)
        return indexed_prepare(h->idx, h->qs, h->qmeta_host, h->qwords_host, h->wmax, h->cfg, h->max_subs,
                               h->stream, h->err);
    IndexedState &S = h->idx;
    if (!(S.plan_valid && !S.plan_uniform && S.plan_s == kSPerEntry)) {
        const ifa_status st = indexed_plan_q(S, h->qs, h->qs_s, std::vector<uint8_t>(h->qs.size(), 1), h->cfg,
                                             h->stream, h->err);
        if (st != IFA_OK) return st;
        S.plan_uniform = false;
        S.plan_s = kSPerEntry;
    }
    if (S.tables_valid && S.tables_s == kSPerEntry && S.wmax == h->wmax) return IFA_OK;
    const ifa_status st = indexed_tables(S, h->qs, h->qmeta_host, h->qwords_host, h->wmax, h->cfg, h->stream, h->err);
    if (st != IFA_OK) return st;
    S.tables_s = kSPerEntry;
    return IFA_OK;
}

}  // namespace

namespace ifa {
// Mean of that probability over the queries: the expected share of (entry,
// window) pairs that are hits on a random reference.
double mean_window_hit_rate(const std::vector<std::string> &qs, uint32_t first, uint32_t n, uint32_t s) {
    if (n == 0) return 0.0;
    double rate[kTcMaxQueryBases + 1];
    for (uint32_t L = 0; L <= kTcMaxQueryBases; L++) rate[L] = random_window_hit_rate(L, s);
    double sum = 0.0;
    for (uint32_t q = first; q < first + n; q++)
        sum += qs[q].size() <= kTcMaxQueryBases ? rate[qs[q].size()] : 1.0;
    return sum / static_cast<double>(n);
}

bool tc_auto_choice(const std::vector<std::string> &qs, uint32_t first, uint32_t n, uint32_t s) {
    uint32_t lmax = 0;
    for (uint32_t q = first; q < first + n; q++) lmax = std::max<uint32_t>(lmax, static_cast<uint32_t>(qs[q].size()));
    return tc_eligible(lmax) && 2 * n >= kTcAutoEntries && mean_window_hit_rate(qs, first, n, s) <= kTcAutoMaxHitRate;
}
}  // namespace ifa

// ------------------------------------------------------------------------ API

extern "C" {

ifa_status ifa_config_default(ifa_config *cfg) {
    if (!cfg) return fail(nullptr, IFA_ERR_INVALID_ARG, "cfg is NULL");
    std::memset(cfg, 0, sizeof(*cfg));
    cfg->device = 0;
    cfg->count_only = 0;
    cfg->hit_capacity = 1ull << 26;
    cfg->segment_bytes = 256ull << 20;
    const uint32_t ks[5] = {8, 9, 10, 12, 14};  // paper default k list
    for (int i = 0; i < 5; i++) cfg->k_list[i] = ks[i];
    cfg->n_k = 5;
    cfg->kmer_step = 1;
    cfg->mask_width = 0;
    cfg->minhits_num = 999;   // 99.9%, paper default
    cfg->minhits_den = 1000;
    cfg->minhits_trials = 200000;  // paper default iterations
    cfg->minhits_seed = 1;
    cfg->clip_pct = 0;
    cfg->exhaustive_fallback = 0;
    cfg->auto_crossover = 0;    // measured rates (the paper's count rule: 150, between its 100 and 200)
    return IFA_OK;
}

ifa_status ifa_create(const ifa_config *cfg, ifa_handle **out) {
    if (!out) return fail(nullptr, IFA_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!cfg) return fail(nullptr, IFA_ERR_INVALID_ARG, "cfg is NULL");
    if (cfg->clip_pct > 50)
        return fail(nullptr, IFA_ERR_INVALID_ARG, "clip_pct must be at most 50 (percent of the query length)");
    if (cfg->brute_kernel > IFA_BRUTE_TENSOR)
        return fail(nullptr, IFA_ERR_INVALID_ARG, "brute_kernel must be 0 (auto), 1 (popcount) or 2 (tensor cores)");
    if (cfg->n_k == 0 || cfg->n_k > IFA_MAX_KLIST)
        return fail(nullptr, IFA_ERR_INVALID_ARG, "n_k must be in 1..8");
    for (uint32_t i = 0; i < cfg->n_k; i++)
        if (cfg->k_list[i] == 0 || cfg->k_list[i] > 16 || cfg->k_list[i] <= cfg->mask_width)
            return fail(nullptr, IFA_ERR_INVALID_ARG, "k_list entries must be in (mask_width, 16]");
    if (cfg->kmer_step == 0 || cfg->minhits_den == 0)
        return fail(nullptr, IFA_ERR_INVALID_ARG, "kmer_step and minhits_den must be > 0");
    if (cfg->segment_bytes == 0 || cfg->segment_bytes > (1ull << 36))
        return fail(nullptr, IFA_ERR_INVALID_ARG, "segment_bytes out of range");
    if (!cfg->count_only && cfg->hit_capacity == 0)
        return fail(nullptr, IFA_ERR_INVALID_ARG, "hit_capacity must be > 0 unless count_only");
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess) return fail_cuda(nullptr, "cudaGetDeviceCount", e);
    if (cfg->device < 0 || cfg->device >= ndev)
        return fail(nullptr, IFA_ERR_CUDA, "no such CUDA device");
    ifa_handle *h = new ifa_handle();
    h->cfg = *cfg;
    h->dev = cfg->device;
    auto bail = [&](ifa_status st) {
        g_err = h->err;
        ifa_destroy(h);
        return st;
    };
#define CKC(call)                                                     \
    do {                                                              \
        cudaError_t e_ = (call);                                      \
        if (e_ != cudaSuccess) return bail(fail_cuda(h, #call, e_));  \
    } while (0)
    CKC(cudaSetDevice(h->dev));
    CKC(cudaStreamCreateWithFlags(&h->own_stream, cudaStreamNonBlocking));
    CKC(cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking));
    h->stream = h->own_stream;
    const uint64_t sb = cfg->segment_bytes;
    const uint64_t words = (sb + kHaloCap + 31) / 32 + kWordPad;
    CKC(refbufs_alloc(h->ref, words, 0, words));   // streamed batches pack with no mask scratch
    for (int i = 0; i < 2; i++) {
        CKC(cudaMalloc(&h->d_seg[i], sb));
        CKC(cudaMalloc(&h->d_halo[i], kHaloCap));
        CKC(cudaEventCreateWithFlags(&h->ev_copied[i], cudaEventDisableTiming));
        CKC(cudaEventCreateWithFlags(&h->ev_consumed[i], cudaEventDisableTiming));
    }
    if (!cfg->count_only) CKC(cudaMalloc(&h->d_ring, cfg->hit_capacity * sizeof(ifa_hit)));
    h->ev.cap = cfg->event_capacity ? cfg->event_capacity : std::max<uint64_t>(1ull << 20, sb / 32);
    CKC(cudaMalloc(&h->ev.buf, h->ev.cap * sizeof(uint4)));
    CKC(cudaMalloc(&h->ev.head, sizeof(unsigned long long)));
    CKC(cudaMalloc(&h->d_head, 3 * sizeof(unsigned long long)));
    CKC(cudaMalloc(&h->d_overflow, sizeof(uint32_t)));
    CKC(cudaMalloc(&h->d_digest, 3 * sizeof(unsigned long long)));
    CKC(cudaStreamCreateWithFlags(&h->drain_stream, cudaStreamNonBlocking));
    CKC(cudaHostAlloc(&h->h_marks, (2 * ifa_handle::kMarks + 1) * sizeof(unsigned long long), cudaHostAllocDefault));
    for (int i = 0; i < ifa_handle::kMarks; i++)
        CKC(cudaEventCreateWithFlags(&h->ev_mark[i], cudaEventDisableTiming));
    if (reset_ring(h) != IFA_OK) return bail(IFA_ERR_CUDA);
    CKC(cudaMemsetAsync(h->d_overflow, 0, sizeof(uint32_t), h->stream));
    CKC(cudaMemsetAsync(h->d_digest, 0, 3 * sizeof(unsigned long long), h->stream));
#undef CKC
    ifa_status st = ensure_pieces(h, 0, 1024);
    if (st == IFA_OK) st = ensure_pieces(h, 1, 1024);
    if (st != IFA_OK) return bail(st);
    *out = h;
    return IFA_OK;
}

void ifa_destroy(ifa_handle *h) {
    if (!h) return;
    cudaSetDevice(h->dev);
    if (h->copy_stream) cudaStreamSynchronize(h->copy_stream);
    if (h->stream) cudaStreamSynchronize(h->stream);
    h->idx.release();
    ifa::serve_release(h);
    ifa::batch_release(h);
    for (int i = 0; i < 2; i++) {
        cudaFree(h->d_seg[i]);
        cudaFreeHost(h->h_stage[i]);
        cudaFree(h->d_pieces[i]);
        cudaFreeHost(h->h_pieces[i]);
        cudaFree(h->d_halo[i]);
        if (h->ev_copied[i]) cudaEventDestroy(h->ev_copied[i]);
        if (h->ev_consumed[i]) cudaEventDestroy(h->ev_consumed[i]);
    }
    for (auto *v : {&h->ev_pending, &h->ev_free})
        for (auto &ev : *v) {
            cudaEventDestroy(ev.first);
            cudaEventDestroy(ev.second);
        }
    refbufs_free(h->ref);
    cudaFree(h->d_qwords);
    cudaFree(h->d_qmeta);
    cudaFree(h->d_tcA);
    cudaFree(h->d_tc_status);
    cudaFree(h->d_ring);
    cudaFree(h->ev.buf);
    cudaFree(h->ev.head);
    cudaFree(h->d_head);
    if (h->drain_stream) cudaStreamSynchronize(h->drain_stream);
    cudaFreeHost(h->h_marks);
    for (int i = 0; i < ifa_handle::kMarks; i++)
        if (h->ev_mark[i]) cudaEventDestroy(h->ev_mark[i]);
    if (h->drain_stream) cudaStreamDestroy(h->drain_stream);
    cudaFree(h->d_overflow);
    cudaFree(h->d_digest);
    cudaFree(h->d_qcount);
    if (h->copy_stream) cudaStreamDestroy(h->copy_stream);
    if (h->own_stream) cudaStreamDestroy(h->own_stream);
    delete h;
}

ifa_status ifa_set_stream(ifa_handle *h, void *stream) {
    if (!h) return fail(nullptr, IFA_ERR_INVALID_ARG, "handle is NULL");
    CK(h, cudaSetDevice(h->dev));
    ifa_status st = sync_all(h);
    if (st != IFA_OK) return st;
    h->stream = stream ? static_cast<cudaStream_t>(stream) : h->own_stream;
    return IFA_OK;
}

ifa_status ifa_load_queries(ifa_handle *h, const uint8_t *const *seqs, const uint32_t *lens, uint32_t n,
                            uint32_t *first_id) {
    if (!h) return fail(nullptr, IFA_ERR_INVALID_ARG, "handle is NULL");
    if (h->pushed) return fail(h, IFA_ERR_BAD_STATE, "queries must be loaded before the first segment");
    if (n && (!seqs || !lens)) return fail(h, IFA_ERR_INVALID_ARG, "seqs/lens is NULL");
    for (uint32_t i = 0; i < n; i++) {
        if (lens[i] == 0 || lens[i] > IFA_MAX_QUERY_LEN)
            return fail(h, IFA_ERR_INVALID_ARG, "query length must be in 1..255");
        if (!seqs[i]) return fail(h, IFA_ERR_INVALID_ARG, "query pointer is NULL");
    }
    if (h->qs.size() + n > (1u << 24))
        return fail(h, IFA_ERR_INVALID_ARG, "at most 2^24 queries");
    if (first_id) *first_id = static_cast<uint32_t>(h->qs.size());
    CK(h, cudaSetDevice(h->dev));
    for (uint32_t i = 0; i < n; i++) {
        h->qs.emplace_back(reinterpret_cast<const char *>(seqs[i]), lens[i]);
        h->lmin = h->qs.size() == 1 ? lens[i] : std::min(h->lmin, lens[i]);
        h->lmax = std::max(h->lmax, lens[i]);
    }
    h->qdirty = true;
    h->per_query_s = false;         // the new queries have no value of their own yet
    h->auto_mode = IFA_MODE_AUTO;   // the automatic choice is redone for the new set
    cudaFree(h->d_qcount);
    h->d_qcount = nullptr;
    CK(h, cudaMalloc(&h->d_qcount, std::max<size_t>(1, h->qs.size()) * sizeof(unsigned long long)));
    CK(h, cudaMemsetAsync(h->d_qcount, 0, std::max<size_t>(1, h->qs.size()) * sizeof(unsigned long long), h->stream));
    return IFA_OK;
}

ifa_status ifa_set_max_subs(ifa_handle *h, uint32_t s) {
    if (!h) return fail(nullptr, IFA_ERR_INVALID_ARG, "handle is NULL");
    // A window has at most IFA_MAX_QUERY_LEN = 255 bases, so every value of
    // 255 or more reports every window (and plans MinHits bins with s >= L);
    // the clamp keeps launches clear of the per-entry threshold sentinel.
    h->max_subs = s < 255u ? s : 255u;
    h->per_query_s = false;
    return IFA_OK;
}

ifa_status ifa_set_query_max_subs(ifa_handle *h, const uint32_t *max_subs, uint32_t n) {
    if (!h) return fail(nullptr, IFA_ERR_INVALID_ARG, "handle is NULL");
    if (!max_subs && n == 0) {
        h->per_query_s = false;
        return IFA_OK;
    }
    if (!max_subs) return fail(h, IFA_ERR_INVALID_ARG, "max_subs is NULL");
    // query sets keep their own maxSubs in the same per-query table
    if (!h->batch.sets.empty())
        return fail(h, IFA_ERR_BAD_STATE, "per-query maxSubs is for streaming; query sets carry their own");
    if (n != h->qs.size()) return fail(h, IFA_ERR_INVALID_ARG, "one maxSubs per loaded query");
    CK(h, cudaSetDevice(h->dev));
    // in-flight scans read the query table that the next push re-uploads
    const ifa_status st = sync_all(h);
    if (st != IFA_OK) return st;
    // each value lives in its entries' meta word (bits 24-31), which the
    // kernels read when the launch threshold is the per-entry sentinel
    h->qs_s.assign(max_subs, max_subs + n);
    for (uint32_t &v : h->qs_s) v = std::min<uint32_t>(v, 255u);
    h->per_query_s = true;
    h->qdirty = true;
    h->auto_mode = IFA_MODE_AUTO;
    h->batch.plan_valid = false;
    return IFA_OK;
}

ifa_status ifa_set_mode(ifa_handle *h, ifa_mode m) {
    if (!h) return fail(nullptr, IFA_ERR_INVALID_ARG, "handle is NULL");
    if (m != IFA_MODE_AUTO && m != IFA_MODE_BRUTE && m != IFA_MODE_INDEXED)
        return fail(h, IFA_ERR_INVALID_ARG, "unknown mode");
    h->mode = m;
    return IFA_OK;
}

ifa_status ifa_push_segment(ifa_handle *h, const uint8_t *ascii, uint64_t len, const ifa_piece *pieces,
                            uint32_t n, ifa_mem mem) {
    if (!h) return fail(nullptr, IFA_ERR_INVALID_ARG, "handle is NULL");
    if (len == 0 && n == 0) return IFA_OK;
    if (len == 0 || n == 0 || !ascii || !pieces)
        return fail(h, IFA_ERR_INVALID_ARG, "a segment needs bytes and at least one piece");
    if (len > h->cfg.segment_bytes) return fail(h, IFA_ERR_INVALID_ARG, "segment longer than segment_bytes");
    const NvtxRange nvtx("ifa_push_segment");
    if (mem != IFA_MEM_HOST && mem != IFA_MEM_HOST_PINNED && mem != IFA_MEM_DEVICE &&
        mem != IFA_MEM_HOST_PINNED_ASYNC)
        return fail(h, IFA_ERR_INVALID_ARG, "unknown memory kind");
    if (h->qs.empty()) return fail(h, IFA_ERR_BAD_STATE, "no queries loaded");
    // piece table checks
    uint64_t at = 0;
    for (uint32_t i = 0; i < n; i++) {
        const ifa_piece &p = pieces[i];
        if (p.start != at || p.len == 0) return fail(h, IFA_ERR_INVALID_ARG, "pieces must be contiguous, non-empty and start at 0");
        at += p.len;
        if (!p.last && i + 1 != n) return fail(h, IFA_ERR_INVALID_ARG, "only a segment's last piece may continue");
        if (i == 0 && h->open) {
            if (p.contig != h->open_contig || p.offset_in_contig != h->open_next)
                return fail(h, IFA_ERR_INVALID_ARG, "segment must continue the open contig");
        } else {
            if (p.offset_in_contig != 0) return fail(h, IFA_ERR_INVALID_ARG, "a new contig must start at offset 0");
            const bool have_prev = i > 0 || h->any_contig;
            const uint32_t prev = i > 0 ? pieces[i - 1].contig : h->last_contig;
            if (have_prev && p.contig <= prev) return fail(h, IFA_ERR_INVALID_ARG, "contig ids must increase");
        }
        if (p.offset_in_contig + p.len > 0xffffffffull)
            return fail(h, IFA_ERR_INVALID_ARG, "contig longer than 2^32 - 1 bases");
    }
    if (at != len) return fail(h, IFA_ERR_INVALID_ARG, "pieces must cover the segment exactly");

    CK(h, cudaSetDevice(h->dev));
    ifa_status st = upload_queries(h);
    if (st != IFA_OK) return st;
    ifa_mode mode = IFA_MODE_BRUTE;
    st = resolve_mode(h, &mode);
    if (st != IFA_OK) return st;
    h->mode_run = mode;
    if (mode == IFA_MODE_INDEXED) {
        st = stream_indexed_prepare(h);
        if (st != IFA_OK) return st;
    }

    const int slot = h->slot;
    h->slot ^= 1;
    if (h->slot_used[slot]) CK(h, cudaEventSynchronize(h->ev_consumed[slot]));
    st = ensure_pieces(h, slot, n);
    if (st != IFA_OK) return st;

    // halo region: H bases (a multiple of 32), the continuing contig's last
    // hlen bases at its end, 'N' padding before them
    const uint32_t hlen = h->open ? h->halo_len : 0u;
    const uint32_t H = h->open ? ((h->lmax + 30u) / 32u) * 32u : 0u;
    DevPiece *hp = h->h_pieces[slot];
    for (uint32_t i = 0; i < n; i++) {
        hp[i].start = i == 0 ? H - hlen : H + pieces[i].start;
        hp[i].contig_off = pieces[i].offset_in_contig - (i == 0 ? hlen : 0);
        hp[i].contig = pieces[i].contig;
        hp[i].last = pieces[i].last ? 1u : 0u;
    }
    CK(h, cudaMemcpyAsync(h->d_pieces[slot], hp, n * sizeof(DevPiece), cudaMemcpyHostToDevice, h->copy_stream));
    const uint8_t *dsrc = ascii;
    if (mem == IFA_MEM_HOST) {
        if (!h->h_stage[slot]) CK(h, cudaHostAlloc(&h->h_stage[slot], h->cfg.segment_bytes, cudaHostAllocDefault));
        std::memcpy(h->h_stage[slot], ascii, len);
        CK(h, cudaMemcpyAsync(h->d_seg[slot], h->h_stage[slot], len, cudaMemcpyHostToDevice, h->copy_stream));
        dsrc = h->d_seg[slot];
        h->stats.h2d_bytes += len;
    } else if (mem == IFA_MEM_HOST_PINNED || mem == IFA_MEM_HOST_PINNED_ASYNC) {
        CK(h, cudaMemcpyAsync(h->d_seg[slot], ascii, len, cudaMemcpyHostToDevice, h->copy_stream));
        dsrc = h->d_seg[slot];
        h->stats.h2d_bytes += len;
    }
    CK(h, cudaEventRecord(h->ev_copied[slot], h->copy_stream));
    CK(h, cudaStreamWaitEvent(h->stream, h->ev_copied[slot], 0));

    const uint64_t nbases = H + len;
    const uint64_t nwords = (nbases + 31) / 32 + kWordPad;
    int launches = 0;
    CK(h, pack_batch(h->ref, h->d_halo[h->halo_cur], hlen, H, dsrc, len, nwords, h->d_pieces[slot], n,
                     n > 1 || H > hlen, h->stream, &launches));
    const Batch b = make_batch(h->ref, nbases, H, h->d_pieces[slot], n);
    QueryTable qt;
    qt.words = h->d_qwords;
    qt.meta = h->d_qmeta;
    qt.ids = nullptr;
    qt.n_entries = 2 * static_cast<uint32_t>(h->qs.size());
    qt.wmax = h->wmax;
    // one threshold for all entries, or each entry's own from its meta word
    const uint32_t s_run = h->per_query_s ? kSPerEntry : h->max_subs;
    const HitSink sink = make_sink(h);
    cudaEvent_t prof_stop = nullptr;
    st = prof_begin(h, &prof_stop);
    if (st != IFA_OK) return st;
    const int before_scan = launches;
    if (mode == IFA_MODE_INDEXED) {
        st = indexed_scan(h->idx, b, qt, s_run, sink, h->stream, &launches, h->err, &h->ev);
        if (st != IFA_OK) return st;
    }
    if (mode == IFA_MODE_BRUTE) {
        if (h->cfg.brute_kernel == IFA_BRUTE_TENSOR && !h->d_tcA)
            return fail(h, IFA_ERR_INVALID_ARG, "brute_kernel 2 (tensor cores) takes queries of at most 64 bases");
        if (use_tensor_cores(h)) {
            if (!h->d_tc_status) {
                CK(h, cudaMalloc(&h->d_tc_status, 2 * sizeof(unsigned int)));
                CK(h, cudaMemsetAsync(h->d_tc_status, 0, 2 * sizeof(unsigned int), h->stream));
            }
            CK(h, launch_scan_tc(b, h->d_tcA, h->d_qmeta, qt.n_entries, h->tc_lpad, s_run, sink,
                                 h->d_tc_status, h->stream, h->cfg.test_stall));
            h->tc_used = true;
            launches++;
        } else {
            for (const Chunk &c : h->chunks)
                CK(h, launch_scan_brute(b, qt, c.e0, c.e1, s_run, c.lmin, c.lmax, sink, h->stream, &launches,
                                        &h->ev));
        }
    }
    if (h->cfg.clip_pct) {
        // windows overhanging contig ends, exhaustively in either mode
        CK(h, launch_clip_scan(b, qt, qt.n_entries, h->cfg.clip_pct, s_run, h->lmax, sink, h->stream));
        launches++;
    }
    st = prof_end(h, prof_stop, launches - before_scan);
    if (st != IFA_OK) return st;
    // halo for the next segment when the last piece continues
    const ifa_piece &lp = pieces[n - 1];
    if (!lp.last) {
        const uint64_t avail = lp.len + (n == 1 ? hlen : 0);
        const uint32_t new_len = static_cast<uint32_t>(std::min<uint64_t>(avail, h->lmax > 0 ? h->lmax - 1 : 0));
        CK(h, launch_halo_update(h->d_halo[h->halo_cur], hlen, dsrc, len, new_len, h->d_halo[h->halo_cur ^ 1], h->stream));
        if (new_len) launches++;
        h->halo_cur ^= 1;
        h->halo_len = new_len;
        h->open = true;
        h->open_contig = lp.contig;
        h->open_next = lp.offset_in_contig + lp.len;
    } else {
        h->open = false;
        h->halo_len = 0;
    }
    h->any_contig = true;
    h->last_contig = lp.contig;
    h->pushed = true;
    if (!h->cfg.count_only) {
        // the ring's head after this segment's scan, for ifa_poll_hits
        if (static_cast<int>(h->marks_pending.size()) == ifa_handle::kMarks) {
            st = collect_marks(h, false);
            if (st != IFA_OK) return st;
            if (static_cast<int>(h->marks_pending.size()) == ifa_handle::kMarks) {
                CK(h, cudaEventSynchronize(h->ev_mark[h->marks_pending.front()]));
                st = collect_marks(h, false);
                if (st != IFA_OK) return st;
            }
        }
        const int k = h->mark_next;
        h->mark_next = (k + 1) % ifa_handle::kMarks;
        CK(h, cudaMemcpyAsync(h->h_marks + 2 * k, h->d_head, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                              h->stream));
        CK(h, cudaEventRecord(h->ev_mark[k], h->stream));
        h->marks_pending.push_back(k);
    }
    CK(h, cudaEventRecord(h->ev_consumed[slot], h->stream));
    h->slot_used[slot] = true;
    if (mem == IFA_MEM_HOST_PINNED) CK(h, cudaEventSynchronize(h->ev_copied[slot]));  // the caller may reuse it

    // nominal work counters: windows owned by this batch
    h->stats.segments++;
    h->stats.bases += len;
    h->stats.kernel_launches += launches;
    for (uint32_t i = 0; i < n; i++) {
        const uint64_t plen = pieces[i].len + (i == 0 ? hlen : 0);
        const uint64_t first_new = (i == 0 ? hlen : 0);
        for (uint32_t q = 0; q < h->qs.size(); q++) {
            const uint64_t L = h->qs[q].size();
            if (plen < L) continue;
            // windows whose last base is new: ends in [max(L-1, first_new), plen)
            const uint64_t lo = std::max<uint64_t>(L - 1, first_new);
            if (plen > lo) {
                h->stats.windows += 2 * (plen - lo);
                h->stats.query_bases += 2 * (plen - lo) * L;
            }
        }
    }
    return IFA_OK;
}

ifa_status ifa_prime_halo(ifa_handle *h, uint32_t contig, uint64_t offset_in_contig, const uint8_t *ascii,
                          uint64_t len, ifa_mem mem) {
    if (!h) return fail(nullptr, IFA_ERR_INVALID_ARG, "handle is NULL");
    if (len == 0 || !ascii) return fail(h, IFA_ERR_INVALID_ARG, "the halo needs at least one base");
    if (mem != IFA_MEM_HOST && mem != IFA_MEM_HOST_PINNED && mem != IFA_MEM_DEVICE &&
        mem != IFA_MEM_HOST_PINNED_ASYNC)
        return fail(h, IFA_ERR_INVALID_ARG, "unknown memory kind");
    if (h->qs.empty()) return fail(h, IFA_ERR_BAD_STATE, "no queries loaded");
    if (h->open) return fail(h, IFA_ERR_BAD_STATE, "a contig is still open; the halo must come first");
    if (h->any_contig && contig <= h->last_contig) return fail(h, IFA_ERR_INVALID_ARG, "contig ids must increase");
    if (offset_in_contig + len > 0xffffffffull) return fail(h, IFA_ERR_INVALID_ARG, "contig longer than 2^32 - 1 bases");
    CK(h, cudaSetDevice(h->dev));
    // the same halo a preceding segment of this contig would have left: its
    // last min(len, L_max - 1) bases
    const uint32_t keep = static_cast<uint32_t>(std::min<uint64_t>(len, h->lmax > 0 ? h->lmax - 1 : 0));
    const int nxt = h->halo_cur ^ 1;
    if (keep)
        CK(h, cudaMemcpyAsync(h->d_halo[nxt], ascii + (len - keep), keep, cudaMemcpyDefault, h->stream));
    h->halo_cur = nxt;
    h->halo_len = keep;
    h->open = true;
    h->open_contig = contig;
    h->open_next = offset_in_contig + len;
    h->any_contig = true;
    h->last_contig = contig;
    h->pushed = true;
    if (mem != IFA_MEM_DEVICE && mem != IFA_MEM_HOST_PINNED_ASYNC) CK(h, cudaStreamSynchronize(h->stream));
    return IFA_OK;
}

ifa_status ifa_flush(ifa_handle *h) {
    if (!h) return fail(nullptr, IFA_ERR_INVALID_ARG, "handle is NULL");
    CK(h, cudaSetDevice(h->dev));
    ifa_status st = sync_all(h);
    if (st != IFA_OK) return st;
    st = prof_collect(h);
    if (st != IFA_OK) return st;
    if (h->tc_used) {
        unsigned int tcs = 0;
        CK(h, cudaMemcpy(&tcs, h->d_tc_status, sizeof(tcs), cudaMemcpyDeviceToHost));
        if (tcs) return fail(h, IFA_ERR_TIMEOUT, "tensor-core scan: a pipeline wait gave up; results incomplete");
    }
#ifdef IFA_BOUNDS_CHECK
    if (unsigned long long *bw = bounds_word()) {
        unsigned long long v = 0;
        CK(h, cudaMemcpy(&v, bw, sizeof(v), cudaMemcpyDeviceToHost));
        if (v) {
            char m[128];
            std::snprintf(m, sizeof m, "bounds check: read of kind %llu at index %llu out of range; results invalid",
                          v >> 56, v & ((1ull << 56) - 1));
            return fail(h, IFA_ERR_CUDA, m);
        }
    }
#endif
    uint32_t ov = 0;
    CK(h, cudaMemcpy(&ov, h->d_overflow, sizeof(ov), cudaMemcpyDeviceToHost));
    if (ov) return fail(h, IFA_ERR_HIT_OVERFLOW, "hit buffer overflowed; some hit tuples were dropped");
    return IFA_OK;
}

ifa_status ifa_bounds_check(int device, uint64_t *first, uint32_t *enabled, int reset) {
    if (!first || !enabled) return fail(nullptr, IFA_ERR_INVALID_ARG, "NULL argument");
    *first = 0;
#ifdef IFA_BOUNDS_CHECK
    *enabled = 1;
    cudaError_t e = cudaSetDevice(device);
    unsigned long long *bw = e == cudaSuccess ? bounds_word() : nullptr;
    if (e == cudaSuccess && !bw) e = cudaErrorSymbolNotFound;
    unsigned long long v = 0;
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(&v, bw, sizeof(v), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && reset) e = cudaMemset(bw, 0, sizeof(v));
    if (e != cudaSuccess) return fail_cuda(nullptr, "ifa_bounds_check", e);
    *first = v;
#else
    (void)device;
    (void)reset;
    *enabled = 0;
#endif
    return IFA_OK;
}

ifa_status ifa_drain_hits(ifa_handle *h, ifa_hit *out, uint64_t cap, uint64_t *n_out, int *more) {
    if (!h) return fail(nullptr, IFA_ERR_INVALID_ARG, "handle is NULL");
    if (!n_out || (cap && !out)) return fail(h, IFA_ERR_INVALID_ARG, "out/n_out is NULL");
    *n_out = 0;
    if (more) *more = 0;
    const NvtxRange nvtx("ifa_drain_hits");
    ifa_status st = ifa_flush(h);
    if (st != IFA_OK && st != IFA_ERR_HIT_OVERFLOW) return st;
    const ifa_status ret = st;
    if (h->cfg.count_only) return ret;
    // the device is idle: every claim is written
    unsigned long long ctr[2] = {0, 0};
    CK(h, cudaMemcpy(ctr, h->d_head, sizeof(ctr), cudaMemcpyDeviceToHost));
    h->marks_pending.clear();
    h->done_head = ctr[0];
    h->done_ovf = ctr[1];
    const uint64_t end = std::min<uint64_t>(ctr[0], ctr[1]);
    st = drain_span(h, out, cap, end, n_out);
    if (st != IFA_OK) return st;
    const bool left = h->tail < end;
    if (more) *more = left ? 1 : 0;
    if (!left && ctr[1] != ~0ull) {
        // everything before the first dropped claim is out: skip the claims
        // after it (dropped or not, they are part of the overflow) and
        // re-arm the ring
        h->tail = ctr[0];
        h->done_ovf = ~0ull;
        const unsigned long long rearm[2] = {~0ull, ctr[0]};
        CK(h, cudaMemcpy(h->d_head + 1, rearm, sizeof(rearm), cudaMemcpyHostToDevice));
    }
    return ret;
}

ifa_status ifa_poll_hits(ifa_handle *h, ifa_hit *out, uint64_t cap, uint64_t *n_out, int *more) {
    if (!h) return fail(nullptr, IFA_ERR_INVALID_ARG, "handle is NULL");
    if (!n_out || (cap && !out)) return fail(h, IFA_ERR_INVALID_ARG, "out/n_out is NULL");
    *n_out = 0;
    if (more) *more = 0;
    if (h->cfg.count_only) return IFA_OK;
    const NvtxRange nvtx("ifa_poll_hits");
    CK(h, cudaSetDevice(h->dev));
    ifa_status st = collect_marks(h, false);
    if (st != IFA_OK) return st;
    const uint64_t end = std::min<uint64_t>(h->done_head, h->done_ovf);
    st = drain_span(h, out, cap, end, n_out);
    if (st != IFA_OK) return st;
    if (more) *more = h->tail < end ? 1 : 0;
    return h->done_ovf != ~0ull ? fail(h, IFA_ERR_HIT_OVERFLOW, "hit ring overflowed; some hit tuples were dropped")
                                : IFA_OK;
}

ifa_status ifa_get_digest(ifa_handle *h, ifa_digest *d, uint64_t *per_query_counts) {
    if (!h) return fail(nullptr, IFA_ERR_INVALID_ARG, "handle is NULL");
    ifa_status st = ifa_flush(h);
    if (st != IFA_OK && st != IFA_ERR_HIT_OVERFLOW) return st;
    if (d) {
        unsigned long long v[3];
        CK(h, cudaMemcpy(v, h->d_digest, sizeof(v), cudaMemcpyDeviceToHost));
        d->count = v[0];
        d->sum = v[1];
        d->xr = v[2];
    }
    if (per_query_counts && !h->qs.empty())
        CK(h, cudaMemcpy(per_query_counts, h->d_qcount, h->qs.size() * sizeof(uint64_t), cudaMemcpyDeviceToHost));
    return IFA_OK;
}

ifa_status ifa_reset_results(ifa_handle *h) {
    if (!h) return fail(nullptr, IFA_ERR_INVALID_ARG, "handle is NULL");
    CK(h, cudaSetDevice(h->dev));
    ifa_status st = sync_all(h);
    if (st != IFA_OK) return st;
    // on the compute stream, so the next pass's kernels see the zeros
    st = reset_ring(h);
    if (st != IFA_OK) return st;
    CK(h, cudaMemsetAsync(h->d_overflow, 0, sizeof(uint32_t), h->stream));
    CK(h, cudaMemsetAsync(h->d_digest, 0, 3 * sizeof(unsigned long long), h->stream));
    if (h->d_qcount)
        CK(h, cudaMemsetAsync(h->d_qcount, 0, std::max<size_t>(1, h->qs.size()) * sizeof(unsigned long long),
                              h->stream));
    h->open = false;
    h->halo_len = 0;
    h->any_contig = false;
    h->pushed = false;
    st = prof_collect(h);
    if (st != IFA_OK) return st;
    h->stats = ifa_stats{};
    if (h->idx.d_candidates) CK(h, cudaMemsetAsync(h->idx.d_candidates, 0, sizeof(unsigned long long), h->stream));
    if (h->batch.d_cand) CK(h, cudaMemsetAsync(h->batch.d_cand, 0, sizeof(unsigned long long), h->stream));
    if (h->d_tc_status) CK(h, cudaMemsetAsync(h->d_tc_status, 0, 2 * sizeof(unsigned int), h->stream));
    h->tc_used = false;
    return IFA_OK;
}

ifa_status ifa_get_stats(ifa_handle *h, ifa_stats *s) {
    if (!h || !s) return fail(h, IFA_ERR_INVALID_ARG, "NULL argument");
    CK(h, cudaSetDevice(h->dev));
    ifa_status st = sync_all(h);
    if (st != IFA_OK) return st;
    st = prof_collect(h);
    if (st != IFA_OK) return st;
    *s = h->stats;
    s->candidates = h->idx.candidates_host(h->stream);
    s->mode = h->mode_run;
    return IFA_OK;
}

ifa_status ifa_get_query_plan(ifa_handle *h, uint32_t *k, uint32_t *minhits, uint8_t *exhaustive) {
    if (!h) return fail(nullptr, IFA_ERR_INVALID_ARG, "handle is NULL");
    if (h->qs.empty()) return fail(h, IFA_ERR_BAD_STATE, "no queries loaded");
    CK(h, cudaSetDevice(h->dev));
    ifa_status st = upload_queries(h);
    if (st != IFA_OK) return st;
    st = h->per_query_s ? stream_indexed_prepare(h)
                        : indexed_plan(h->idx, h->qs, h->cfg, h->max_subs, h->stream, h->err);
    if (st != IFA_OK) return st;
    for (size_t q = 0; q < h->qs.size(); q++) {
        if (k) k[q] = h->idx.plan_k[q];
        if (minhits) minhits[q] = h->idx.plan_minhits[q];
        if (exhaustive) exhaustive[q] = h->idx.plan_exhaustive[q];
    }
    return IFA_OK;
}

ifa_status ifa_minhits(int32_t device, const uint32_t *L, const uint32_t *subs, const uint32_t *k, uint32_t n,
                       uint32_t step, uint32_t mask_width, uint32_t max_clips, uint32_t num, uint32_t den,
                       uint32_t trials, uint64_t seed, uint32_t *out) {
    if (n == 0) return IFA_OK;
    if (!L || !subs || !k || !out) return fail(nullptr, IFA_ERR_INVALID_ARG, "NULL array");
    if (step == 0 || den == 0) return fail(nullptr, IFA_ERR_INVALID_ARG, "step and den must be > 0");
    uint32_t maxK = 1;
    for (uint32_t i = 0; i < n; i++) {
        if (L[i] == 0 || L[i] > IFA_MAX_QUERY_LEN || k[i] == 0 || k[i] > 64 || k[i] <= mask_width)
            return fail(nullptr, IFA_ERR_INVALID_ARG, "bins need 1 <= L <= 255 and mask_width < k <= 64");
        if (k[i] <= L[i]) maxK = std::max(maxK, (L[i] - k[i]) / step + 2);
    }
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) return fail_cuda(nullptr, "cudaSetDevice", e);
    std::string err;
    ifa_status st = minhits_device(L, subs, k, n, step, mask_width, max_clips, num, den, trials, seed, out,
                                   nullptr, maxK, err);
    if (st != IFA_OK) g_err = err;
    return st;
}

const char *ifa_last_error(const ifa_handle *h) { return h ? h->err.c_str() : g_err.c_str(); }

}  // extern "C"

// serve.cu -- continuous-batching serving over the device-resident store.
//
// Requests (query sets with their own maxSubs) arrive at any time.  The
// store is cut into n_slices slices and scanned cyclically, one slice per
// ifa_serve_step: at every slice boundary the waiting requests that fit the
// HBM budget (their hit ring plus their share of the merged plan) are
// admitted, then the persistent multi-set kernel scans the slice for every
// active request at once -- one reference read and, in indexed mode, one
// k-mer lookup per position shared by all of them.  A request that joined
// at slice t is complete when the scan has covered every slice once, i.e.
// when it wraps back to t; its hit ring stays on the device until drained.
// A request's hits do not depend on what else is active: windows are
// owned by the slice of their start (brute force) or of their first seed
// (indexed), soft-clipped windows by the slice holding their piece's first
// base, and every slice is scanned once per request.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <string>
#include <vector>

#include "handle.cuh"
#include "scan_brute.cuh"

using namespace ifa;

namespace {

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

ifa_status sfail(ifa_handle *h, ifa_status st, const std::string &msg) {
    h->err = msg;
    return st;
}

#define SCK(h, call)                                                                       \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return sfail((h), cuda_status(e_),                                               \
                         std::string(#call) + ": " + cudaGetErrorString(e_));              \
    } while (0)

// The plan's device arrays live in S.pool (grow-only, one slot per array)
// and the merged k-mer tables in S.merged's own buffers, so a rebuild at a
// slice boundary allocates nothing once sizes have settled.
enum PlanSlot : size_t { kPWords, kPMeta, kPBw, kPBm, kPIds, kPC0, kPC1, kPCl, kPCh, kPQ2r, kPRings, kPQc };

void free_serve_plan(ServeState &S) { S.merged.free_tables(); }

template <typename T>
T *salloc(ServeState &S, PlanSlot slot, size_t n, cudaError_t &e) {
    return static_cast<T *>(S.pool.get(slot, std::max<size_t>(1, n) * sizeof(T), e));
}

// Stream-ordered upload (pageable source: staged before the call returns).
template <typename T>
void sput(T *d, const std::vector<T> &v, cudaStream_t st, cudaError_t &e) {
    if (e == cudaSuccess && !v.empty())
        e = cudaMemcpyAsync(d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, st);
}

// Bytes a request is charged against the HBM budget: its ring and counters
// plus its entries in the merged plan (query words, postings, counts).
uint64_t request_bytes(const ServeState &S, const Request &r) {
    uint64_t b = S.ring_cap * sizeof(ifa_hit) + 5 * sizeof(unsigned long long);
    for (const auto &q : r.qs) b += 2 * (8 * sizeof(uint4) + 16) + 2 * 4 * q.size() + 8;
    return b;
}

// Encoding and (indexed requests) per-query plan of one request, made once.
ifa_status prepare_request(ifa_handle *h, Request &r) {
    if (r.prepared) return IFA_OK;
    if (r.mode == IFA_MODE_AUTO) {
        // rates measured once per session on the store, with the first
        // automatic request's queries
        ServeState &S = h->serve;
        if (!S.rates.valid()) {
            const BatchState &B = h->batch;
            const Batch b = make_batch(B.ref, B.nbases, 0, B.d_pieces, B.d_pieces_n);
            const ifa_status st = rates_on_store(h, b, r.qs, std::vector<uint32_t>(r.qs.size(), r.s), S.rates);
            if (st != IFA_OK) return st;
        }
        const ifa_status st = choose_mode(h, S.rates, r.qs, std::vector<uint32_t>(r.qs.size(), r.s), &r.mode);
        if (st != IFA_OK) return st;
    }
    uint32_t lmax = 1;
    for (const auto &q : r.qs) lmax = std::max<uint32_t>(lmax, static_cast<uint32_t>(q.size()));
    r.w = 1;
    while (r.w * 32 < lmax) r.w <<= 1;
    const size_t nq = r.qs.size();
    r.words.assign(2 * nq * r.w, make_uint4(0, 0, 0, 0));
    r.meta.assign(2 * nq, 0);
    for (size_t q = 0; q < nq; q++)
        for (uint32_t t = 0; t < 2; t++)
            encode_entry(r.qs[q], t == 1, r.w, r.s, &r.words[(2 * q + t) * r.w], &r.meta[2 * q + t]);
    if (r.mode == IFA_MODE_INDEXED) {
        IndexedState plan;
        const ifa_status st = indexed_plan_q(plan, r.qs, std::vector<uint32_t>(nq, r.s),
                                             std::vector<uint8_t>(nq, 1), h->cfg, h->stream, h->err);
        if (st != IFA_OK) return st;
        r.plan_k = plan.plan_k;
        r.plan_minhits = plan.plan_minhits;
        r.plan_exhaustive = plan.plan_exhaustive;
    }
    r.prepared = true;
    return IFA_OK;
}

// Merged plan of the active requests: their cached encodings and plans,
// concatenated (entries padded to the widest request), then the merged
// seed tables and the compact brute-force table.
ifa_status build_serve_plan(ifa_handle *h) {
    ServeState &S = h->serve;
    free_serve_plan(S);
    std::vector<uint32_t> q2r, rfirst, qlen;
    uint32_t wmax = 1;
    size_t nqs = 0;
    for (uint32_t id : S.active) {
        wmax = std::max(wmax, S.reqs[id].w);
        nqs += S.reqs[id].qs.size();
    }
    const uint32_t nq = static_cast<uint32_t>(nqs);
    S.wmax = wmax;
    S.nq = nq;
    S.lmax = 0;
    std::vector<uint4> words(static_cast<size_t>(2) * nq * wmax, make_uint4(0, 0, 0, 0));
    std::vector<uint32_t> meta(2 * static_cast<size_t>(nq));
    std::vector<uint8_t> seeded(nq, 0);
    IndexedState &M = S.merged;
    M.plan_k.assign(nq, 0);
    M.plan_minhits.assign(nq, 0);
    M.plan_exhaustive.assign(nq, 0);
    qlen.reserve(nq);
    uint32_t q0 = 0;
    for (size_t slot = 0; slot < S.active.size(); slot++) {
        const Request &r = S.reqs[S.active[slot]];
        rfirst.push_back(q0);
        const uint32_t n = static_cast<uint32_t>(r.qs.size());
        for (uint32_t i = 0; i < n; i++) {
            const uint32_t q = q0 + i;
            q2r.push_back(static_cast<uint32_t>(slot));
            qlen.push_back(static_cast<uint32_t>(r.qs[i].size()));
            S.lmax = std::max<uint32_t>(S.lmax, qlen.back());
            for (uint32_t t = 0; t < 2; t++) {
                const size_t src = (2 * static_cast<size_t>(i) + t) * r.w, dst = (2 * static_cast<size_t>(q) + t) * wmax;
                std::copy(r.words.begin() + src, r.words.begin() + src + r.w, words.begin() + dst);
                meta[2 * q + t] = r.meta[2 * i + t];
            }
            if (r.mode == IFA_MODE_INDEXED) {
                M.plan_k[q] = r.plan_k[i];
                M.plan_minhits[q] = r.plan_minhits[i];
                M.plan_exhaustive[q] = r.plan_exhaustive[i];
                seeded[q] = r.plan_exhaustive[i] ? 0 : 1;
            }
        }
        q0 += n;
    }
    ifa_status st = IFA_OK;
    if (std::any_of(seeded.begin(), seeded.end(), [](uint8_t x) { return x != 0; })) {
        M.plan_in = seeded;
        M.plan_valid = true;
        M.plan_uniform = false;
        st = indexed_tables_len(M, qlen, meta, words, wmax, h->cfg, h->stream, h->err);
        if (st != IFA_OK) return st;
    }
    // compact brute table (brute requests and exhaustive indexed queries)
    std::vector<uint32_t> ids;
    for (uint32_t q = 0; q < nq; q++)
        if (!seeded[q]) {
            ids.push_back(2 * q);
            ids.push_back(2 * q + 1);
        }
    uint32_t cap = brute::chunk_cap(static_cast<int>(wmax));
    cap = std::min<uint32_t>(cap, 65535) & ~1u;
    std::vector<uint32_t> c0, c1, cl, ch;
    for (uint32_t a = 0; a < ids.size(); a += cap) {
        const uint32_t z = std::min<uint32_t>(static_cast<uint32_t>(ids.size()), a + cap);
        uint32_t lo = 255, hi = 0;
        for (uint32_t i = a; i < z; i++) {
            lo = std::min(lo, meta_L(meta[ids[i]]));
            hi = std::max(hi, meta_L(meta[ids[i]]));
        }
        c0.push_back(a);
        c1.push_back(z);
        cl.push_back(lo);
        ch.push_back(hi);
    }
    std::vector<uint4> bw(std::max<size_t>(1, ids.size()) * wmax, make_uint4(0, 0, 0, 0));
    std::vector<uint32_t> bm(std::max<size_t>(1, ids.size()), 0);
    for (size_t i = 0; i < ids.size(); i++) {
        bm[i] = meta[ids[i]];
        for (uint32_t j = 0; j < wmax; j++) bw[i * wmax + j] = words[static_cast<size_t>(ids[i]) * wmax + j];
    }
    // rings of the active slots
    std::vector<RingDesc> rings(std::max<size_t>(1, S.active.size()));
    for (size_t slot = 0; slot < S.active.size(); slot++) {
        const Request &r = S.reqs[S.active[slot]];
        rings[slot].ring = r.d_ring;
        rings[slot].counters = r.d_counters;
        rings[slot].cap = r.cap;
        rings[slot].qfirst = rfirst[slot];
        rings[slot].pad = 0;
    }
    cudaError_t e = cudaSuccess;
    const cudaStream_t st_ = h->stream;
    uint4 *d_words = salloc<uint4>(S, kPWords, words.size(), e);
    uint32_t *d_meta = salloc<uint32_t>(S, kPMeta, meta.size(), e);
    uint4 *d_bw = salloc<uint4>(S, kPBw, bw.size(), e);
    uint32_t *d_bm = salloc<uint32_t>(S, kPBm, bm.size(), e);
    uint32_t *d_ids = salloc<uint32_t>(S, kPIds, ids.size(), e);
    uint32_t *d_c0 = salloc<uint32_t>(S, kPC0, c0.size(), e), *d_c1 = salloc<uint32_t>(S, kPC1, c1.size(), e);
    uint32_t *d_cl = salloc<uint32_t>(S, kPCl, cl.size(), e), *d_ch = salloc<uint32_t>(S, kPCh, ch.size(), e);
    uint32_t *d_q2r = salloc<uint32_t>(S, kPQ2r, q2r.size(), e);
    RingDesc *d_rings = salloc<RingDesc>(S, kPRings, rings.size(), e);
    unsigned long long *d_qc = salloc<unsigned long long>(S, kPQc, nq, e);
    sput(d_words, words, st_, e);
    sput(d_meta, meta, st_, e);
    sput(d_bw, bw, st_, e);
    sput(d_bm, bm, st_, e);
    sput(d_ids, ids, st_, e);
    sput(d_c0, c0, st_, e);
    sput(d_c1, c1, st_, e);
    sput(d_cl, cl, st_, e);
    sput(d_ch, ch, st_, e);
    sput(d_q2r, q2r, st_, e);
    sput(d_rings, rings, st_, e);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_qc, 0, std::max<size_t>(1, nq) * sizeof(unsigned long long), st_);
    if (e != cudaSuccess) return sfail(h, IFA_ERR_CUDA, std::string("serve plan: ") + cudaGetErrorString(e));
    S.ft = QueryTable{d_words, d_meta, nullptr, 2 * nq, wmax};
    S.bt = QueryTable{d_bw, d_bm, d_ids, static_cast<uint32_t>(ids.size()), wmax};
    S.b_entries = static_cast<uint32_t>(ids.size());
    S.chunk_e0 = c0;
    BatchWork &W = S.work;
    W = BatchWork{};
    W.bwords = d_bw;
    W.bmeta = d_bm;
    W.bids = d_ids;
    W.chunk_e0 = d_c0;
    W.chunk_e1 = d_c1;
    W.chunk_lmin = d_cl;
    W.chunk_lmax = d_ch;
    W.nchunks = static_cast<uint32_t>(c0.size());
    W.tabs = S.merged.tables_valid ? S.merged.targ : KTablesArg{};
    W.emh = S.merged.d_entry_minhits;
    W.step = h->cfg.kmer_step;
    W.qwords = d_words;
    W.qmeta = d_meta;
    HitSink &k = S.sink;
    k = HitSink{};
    k.ring = nullptr;
    k.head = nullptr;
    k.capacity = 0;
    k.digest = nullptr;
    k.overflow = nullptr;
    k.qcount = d_qc;
    k.count_only = 0;
    k.q2r = d_q2r;
    k.rings = d_rings;
    S.grid = batch_kernel_grid(wmax);
    S.dirty = false;
    return IFA_OK;
}

}  // namespace

namespace ifa {
void serve_release(ifa_handle *h) {
    ServeState &S = h->serve;
    free_serve_plan(S);
    S.merged.release();
    S.pool.release();
    for (Request &r : S.reqs) {
        cudaFree(r.d_ring);
        cudaFree(r.d_counters);
        r.d_ring = nullptr;
        r.d_counters = nullptr;
    }
    cudaFree(S.d_queue);
    cudaFree(S.d_cand);
    S.d_queue = nullptr;
    S.d_cand = nullptr;
    S.reqs.clear();
    S.pending.clear();
    S.active.clear();
    S.on = false;
}
}  // namespace ifa

extern "C" {

ifa_status ifa_serve_start(ifa_handle *h, uint32_t n_slices, uint64_t hbm_budget_bytes, uint64_t ring_hits) {
    if (!h) return IFA_ERR_INVALID_ARG;
    if (n_slices == 0 || ring_hits == 0) return sfail(h, IFA_ERR_INVALID_ARG, "ifa_serve_start: n_slices and ring_hits must be > 0");
    if (h->batch.nbases == 0) return sfail(h, IFA_ERR_BAD_STATE, "ifa_serve_start: the reference store is empty");
    SCK(h, cudaSetDevice(h->dev));
    serve_release(h);
    ServeState &S = h->serve;
    S.on = true;
    S.clip_pct = h->cfg.clip_pct;
    S.n_slices = n_slices;
    S.budget = hbm_budget_bytes;
    S.used = 0;
    S.ring_cap = ring_hits;
    S.t0 = now_s();
    S.slice = 0;
    S.dirty = true;
    S.slices_run = 0;
    S.scanned_query_bases = 0;
    S.plan_s = 0;
    S.scan_s = 0;
    SCK(h, cudaMalloc(&S.d_queue, 2 * sizeof(unsigned int)));   // brute-force and seed items
    SCK(h, cudaMalloc(&S.d_cand, sizeof(unsigned long long)));
    SCK(h, cudaMemsetAsync(S.d_cand, 0, sizeof(unsigned long long), h->stream));
    // the store's piece table on the device
    BatchState &B = h->batch;
    if (B.pieces_dirty) {
        cudaFree(B.d_pieces);
        B.d_pieces = nullptr;
        SCK(h, cudaMalloc(&B.d_pieces, std::max<size_t>(1, B.pieces.size()) * sizeof(DevPiece)));
        if (!B.pieces.empty())
            SCK(h, cudaMemcpyAsync(B.d_pieces, B.pieces.data(), B.pieces.size() * sizeof(DevPiece),
                                   cudaMemcpyHostToDevice, h->stream));
        B.d_pieces_n = static_cast<uint32_t>(B.pieces.size());
        B.pieces_dirty = false;
    }
    return IFA_OK;
}

ifa_status ifa_serve_submit(ifa_handle *h, const uint8_t *const *seqs, const uint32_t *lens, uint32_t n,
                            uint32_t max_subs, ifa_mode mode, uint32_t *request_id) {
    if (!h) return IFA_ERR_INVALID_ARG;
    ServeState &S = h->serve;
    if (!S.on) return sfail(h, IFA_ERR_BAD_STATE, "ifa_serve_submit: call ifa_serve_start first");
    if (n == 0 || !seqs || !lens) return sfail(h, IFA_ERR_INVALID_ARG, "ifa_serve_submit: empty request");
    if (mode != IFA_MODE_AUTO && mode != IFA_MODE_BRUTE && mode != IFA_MODE_INDEXED)
        return sfail(h, IFA_ERR_INVALID_ARG, "ifa_serve_submit: unknown mode");
    Request r;
    for (uint32_t i = 0; i < n; i++) {
        if (!seqs[i] || lens[i] == 0 || lens[i] > IFA_MAX_QUERY_LEN)
            return sfail(h, IFA_ERR_INVALID_ARG, "ifa_serve_submit: query length must be in 1..255");
        r.qs.emplace_back(reinterpret_cast<const char *>(seqs[i]), lens[i]);
    }
    r.s = std::min<uint32_t>(max_subs, 255);
    // automatic mode: the paper's rule by query count (Discussion) when a
    // crossover is configured, else measured rates at admission
    r.mode = mode;
    if (mode == IFA_MODE_AUTO && h->cfg.auto_crossover)
        r.mode = n >= h->cfg.auto_crossover ? IFA_MODE_INDEXED : IFA_MODE_BRUTE;
    r.t_submit = now_s() - S.t0;
    r.cap = S.ring_cap;
    r.bytes = request_bytes(S, r);
    S.reqs.push_back(std::move(r));
    S.pending.push_back(static_cast<uint32_t>(S.reqs.size() - 1));
    if (request_id) *request_id = static_cast<uint32_t>(S.reqs.size() - 1);
    return IFA_OK;
}

ifa_status ifa_serve_step(ifa_handle *h, uint32_t *n_active, uint32_t *n_completed) {
    const NvtxRange nvtx("ifa_serve_step");
    if (!h) return IFA_ERR_INVALID_ARG;
    ServeState &S = h->serve;
    if (!S.on) return sfail(h, IFA_ERR_BAD_STATE, "ifa_serve_step: call ifa_serve_start first");
    SCK(h, cudaSetDevice(h->dev));
    // admission at the slice boundary, in arrival order, within the budget
    size_t admitted = 0;
    while (admitted < S.pending.size()) {
        Request &r = S.reqs[S.pending[admitted]];
        if (S.used + r.bytes > S.budget && !S.active.empty()) break;
        {
            // a failed allocation leaves the request queued with nothing held
            // (the ones admitted before it stay admitted)
            const auto unwind = [&]() {
                cudaFree(r.d_ring);
                cudaFree(r.d_counters);
                r.d_ring = nullptr;
                r.d_counters = nullptr;
                S.pending.erase(S.pending.begin(), S.pending.begin() + admitted);
            };
            cudaError_t e = cudaMalloc(&r.d_ring, r.cap * sizeof(ifa_hit));
            if (e == cudaSuccess) e = cudaMalloc(&r.d_counters, 5 * sizeof(unsigned long long));
            if (e == cudaSuccess) e = cudaMemsetAsync(r.d_counters, 0, 5 * sizeof(unsigned long long), h->stream);
            if (e != cudaSuccess) {
                unwind();
                return sfail(h, cuda_status(e),
                             std::string("ifa_serve_step: request ring: ") + cudaGetErrorString(e));
            }
            const double tp = now_s();
            const ifa_status pst = prepare_request(h, r);
            S.plan_s += now_s() - tp;
            if (pst != IFA_OK) {
                unwind();
                return pst;
            }
        }
        r.state = 1;
        r.t_admit = now_s() - S.t0;
        r.slices_done = 0;
        S.used += r.bytes;
        S.active.push_back(S.pending[admitted]);
        S.dirty = true;
        admitted++;
    }
    S.pending.erase(S.pending.begin(), S.pending.begin() + admitted);
    uint32_t done = 0;
    if (!S.active.empty()) {
        if (S.dirty) {
            const double t0 = now_s();
            const ifa_status st = build_serve_plan(h);
            S.plan_s += now_s() - t0;
            if (st != IFA_OK) return st;
        }
        // this slice's block ranges and tiles
        const BatchState &B = h->batch;
        const uint64_t nbblk = (B.nbases + 32 * brute::kWin - 1) / (32 * brute::kWin);
        const uint64_t per = (nbblk + S.n_slices - 1) / S.n_slices;
        BatchWork w = S.work;
        w.b_block0 = std::min<uint64_t>(nbblk, per * S.slice);
        w.b_block_end = std::min<uint64_t>(nbblk, w.b_block0 + per);
        const uint64_t nsblk = (B.nbases + 31) / 32;
        w.s_block0 = std::min<uint64_t>(nsblk, w.b_block0 * brute::kWin);
        w.s_block_end = S.slice + 1 == S.n_slices ? nsblk : std::min<uint64_t>(nsblk, w.b_block_end * brute::kWin);
        const uint64_t nb = w.b_block_end - w.b_block0, ns = w.s_block_end - w.s_block0;
        const uint64_t want = static_cast<uint64_t>(8) * S.grid;
        const uint64_t tpc = w.nchunks ? std::max<uint64_t>(1, want / w.nchunks) : 1;
        w.tile_bblocks = std::max<uint64_t>(32, (nb + tpc - 1) / tpc);
        w.n_btiles = static_cast<uint32_t>((nb + w.tile_bblocks - 1) / w.tile_bblocks);
        w.tile_sblocks = std::max<uint64_t>(64, (ns + want - 1) / want);
        w.n_stiles = w.tabs.n ? static_cast<uint32_t>((ns + w.tile_sblocks - 1) / w.tile_sblocks) : 0;
        w.n_brute_items = w.nchunks * w.n_btiles;
        w.n_items = w.n_brute_items + w.n_stiles;
        w.queue = S.d_queue;
        w.candidates = S.d_cand;
        const Batch b = make_batch(B.ref, B.nbases, 0, B.d_pieces, B.d_pieces_n);
        const double t1 = now_s();
        SCK(h, cudaMemsetAsync(S.d_queue, 0, 2 * sizeof(unsigned int), h->stream));
        int nl = 0;
        SCK(h, launch_batch_kernels(S.wmax, b, w, S.bt, S.ft, S.sink, h->stream, &nl));
        h->stats.kernel_launches += nl;
        if (S.clip_pct) {
            // soft-clipped windows of the pieces whose first base is in this
            // slice, every active entry exhaustively at its own maxSubs
            const auto first_at = [&B](uint64_t x) {
                return static_cast<uint32_t>(
                    std::lower_bound(B.pieces.begin(), B.pieces.end(), x,
                                     [](const DevPiece &p, uint64_t v) { return p.start < v; }) -
                    B.pieces.begin());
            };
            const uint32_t p_lo = first_at(w.s_block0 * 32);
            const uint32_t p_hi = S.slice + 1 == S.n_slices ? static_cast<uint32_t>(B.pieces.size())
                                                             : first_at(w.s_block_end * 32);
            if (p_lo < p_hi) {
                SCK(h, launch_clip_scan(b, S.ft, S.ft.n_entries, S.clip_pct, kSPerEntry, S.lmax, S.sink, h->stream, 0,
                                        p_lo, p_hi));
                h->stats.kernel_launches += 1;
            }
        }
        SCK(h, cudaStreamSynchronize(h->stream));
        S.scan_s += now_s() - t1;
        S.slices_run++;
        const double slice_bases = static_cast<double>(ns) * 32.0;
        // retire the requests that have now seen every slice
        std::vector<uint32_t> still;
        const double t = now_s() - S.t0;
        for (uint32_t id : S.active) {
            Request &r = S.reqs[id];
            for (const auto &q : r.qs) S.scanned_query_bases += 2.0 * q.size() * slice_bases;
            if (++r.slices_done == S.n_slices) {
                SCK(h, cudaMemcpy(r.final_counters, r.d_counters, sizeof(r.final_counters), cudaMemcpyDeviceToHost));
                r.state = 2;
                r.t_done = t;
                S.dirty = true;
                done++;
            } else {
                still.push_back(id);
            }
        }
        S.active.swap(still);
        S.slice = (S.slice + 1) % S.n_slices;
    }
    if (n_active) *n_active = static_cast<uint32_t>(S.active.size());
    if (n_completed) *n_completed = done;
    return IFA_OK;
}

ifa_status ifa_serve_poll(ifa_handle *h, uint32_t id, ifa_request_info *info) {
    if (!h || !info) return IFA_ERR_INVALID_ARG;
    ServeState &S = h->serve;
    if (id >= S.reqs.size()) return sfail(h, IFA_ERR_INVALID_ARG, "ifa_serve_poll: unknown request");
    const Request &r = S.reqs[id];
    info->state = static_cast<uint32_t>(r.state);
    info->mode = r.mode;
    info->queries = static_cast<uint32_t>(r.qs.size());
    info->slices_done = r.slices_done;
    info->hits = r.final_counters[2];
    info->overflowed = r.final_counters[1] ? 1 : 0;
    info->submit_s = r.t_submit;
    info->admit_s = r.t_admit;
    info->done_s = r.t_done;
    info->digest.count = r.final_counters[2];
    info->digest.sum = r.final_counters[3];
    info->digest.xr = r.final_counters[4];
    return IFA_OK;
}

ifa_status ifa_serve_drain(ifa_handle *h, uint32_t id, ifa_hit *out, uint64_t cap, uint64_t *n_out) {
    if (!h || !n_out || (cap && !out)) return IFA_ERR_INVALID_ARG;
    ServeState &S = h->serve;
    if (id >= S.reqs.size()) return sfail(h, IFA_ERR_INVALID_ARG, "ifa_serve_drain: unknown request");
    Request &r = S.reqs[id];
    if (r.state != 2) return sfail(h, IFA_ERR_BAD_STATE, "ifa_serve_drain: request not complete (or drained)");
    SCK(h, cudaSetDevice(h->dev));
    const uint64_t have = std::min<uint64_t>(r.final_counters[0], r.cap);
    const uint64_t take = std::min<uint64_t>(have, cap);
    if (take) SCK(h, cudaMemcpy(out, r.d_ring, take * sizeof(ifa_hit), cudaMemcpyDeviceToHost));
    *n_out = take;
    cudaFree(r.d_ring);
    cudaFree(r.d_counters);
    r.d_ring = nullptr;
    r.d_counters = nullptr;
    S.used -= r.bytes;
    r.state = 3;
    return r.final_counters[1] ? IFA_ERR_HIT_OVERFLOW : IFA_OK;
}

ifa_status ifa_serve_cancel(ifa_handle *h, uint32_t id) {
    if (!h) return IFA_ERR_INVALID_ARG;
    ServeState &S = h->serve;
    if (!S.on) return sfail(h, IFA_ERR_BAD_STATE, "ifa_serve_cancel: call ifa_serve_start first");
    if (id >= S.reqs.size()) return sfail(h, IFA_ERR_INVALID_ARG, "ifa_serve_cancel: unknown request");
    Request &r = S.reqs[id];
    if (r.state >= 3) return sfail(h, IFA_ERR_BAD_STATE, "ifa_serve_cancel: request already drained or cancelled");
    SCK(h, cudaSetDevice(h->dev));
    if (r.state == 0) {
        S.pending.erase(std::find(S.pending.begin(), S.pending.end(), id));
    } else {
        if (r.state == 1) {
            S.active.erase(std::find(S.active.begin(), S.active.end(), id));
            S.dirty = true;   // the merged plan drops its entries
        }
        // the stream is idle between steps; free only after any queued work
        SCK(h, cudaStreamSynchronize(h->stream));
        cudaFree(r.d_ring);
        cudaFree(r.d_counters);
        r.d_ring = nullptr;
        r.d_counters = nullptr;
        S.used -= r.bytes;
    }
    r.state = 4;
    r.t_done = now_s() - S.t0;
    return IFA_OK;
}

ifa_status ifa_serve_stats(ifa_handle *h, uint64_t *slices_run, double *query_bases, double *plan_seconds,
                           double *scan_seconds) {
    if (!h) return IFA_ERR_INVALID_ARG;
    if (slices_run) *slices_run = h->serve.slices_run;
    if (query_bases) *query_bases = h->serve.scanned_query_bases;
    if (plan_seconds) *plan_seconds = h->serve.plan_s;
    if (scan_seconds) *scan_seconds = h->serve.scan_s;
    return IFA_OK;
}

ifa_status ifa_serve_stop(ifa_handle *h) {
    if (!h) return IFA_ERR_INVALID_ARG;
    cudaSetDevice(h->dev);
    cudaStreamSynchronize(h->stream);
    serve_release(h);
    return IFA_OK;
}

}  // extern "C"

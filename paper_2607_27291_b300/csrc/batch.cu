// batch.cu -- many query sets against a device-resident reference.
//
// The paper picks brute force or indexed mode per run by query count
// (Discussion; crossover 100-200 queries on RefSeq) and streams the
// reference once per run.  Here the reference is packed once into a store
// in HBM, query sets of uneven sizes -- each with its own maxSubs -- are
// registered, and one call scans all of them:
//
//  * the autotuner decides brute force or indexed for every IFA_MODE_AUTO
//    set from rates it measures on a slice of the store (brute-force
//    entry x base evaluations per second, seed-scan positions per second,
//    verified candidates per second), comparing the set's brute-force cost
//    with the cost of scanning it alone in indexed mode -- the per-set
//    crossover -- and sizes the work tiles;
//  * brute-force sets share one compact entry table cut into shared-memory
//    chunks; indexed sets share one set of merged k-mer tables (a window's
//    threshold and maxSubs are per query, carried in the entry's meta word);
//  * IFA_BATCH_PERSISTENT runs everything in one persistent kernel whose
//    CTAs pull (chunk, tile) and (seed, tile) items from a device work
//    queue; the launch and its queue reset are captured once in a CUDA graph
//    and replayed;
//  * IFA_BATCH_PER_SET is the baseline: every set is scanned by its own
//    launches over the whole store (its own tables in indexed mode), one set
//    after another.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "handle.cuh"
#include "scan_brute.cuh"
#include "seed_scan.cuh"

using namespace ifa;

namespace {

constexpr int kBThreads = 256;
constexpr int kBWarps = kBThreads / kWarp;
// Resident CTAs per SM the brute-force persistent kernel's registers are
// held to: 4 (62-64 registers, no spills up to 128-base queries).  When one
// kernel took both kinds of item it measured (128 sets vs 5 Gbp): no bound
// (64 registers, 124 bytes spilled) 3.96 s; 4 CTAs (64 registers, 16-32
// bytes spilled) 3.76 s; 3 CTAs (80 registers, none spilled) 4.21 s.
#ifndef IFA_BATCH_MIN_CTAS
#define IFA_BATCH_MIN_CTAS 4
#endif
constexpr uint64_t kStorePad = 16;  // padding words after the last packed word (packed as N)

ifa_status bfail(ifa_handle *h, ifa_status st, const std::string &msg) {
    h->err = msg;
    return st;
}

#define BCK(h, call)                                                                       \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return bfail((h), cuda_status(e_),                                               \
                         std::string(#call) + ": " + cudaGetErrorString(e_));              \
    } while (0)

// Resident CTAs per SM of the seed-only persistent kernel: the seed scan's
// own bound (48 registers at 5; see k_seed_scan).
#ifndef IFA_BATCH_SEED_MIN_CTAS
#define IFA_BATCH_SEED_MIN_CTAS 5
#endif

// Which items a persistent launch takes.  The batch and serving calls run
// one kernel per kind back to back, each held to the register budget its
// own scan wants: one kernel for both kinds had to fit both in 64
// registers and spilled (256 sets vs 16 Gbp: 27.1 s fused, 19.1 s split).
enum BatchPart { kSeedOnly = 1, kBruteOnly = 2 };

// One persistent launch: CTAs pull items of their kind from a device queue
// until it runs dry.  Items [0, n_items - n_brute_items) are seed tiles
// (counted in w.queue[0]), the rest brute-force (chunk, tile) items in
// chunk-major order, so a CTA reloads its shared query chunk rarely
// (counted in w.queue[1], from the first brute-force item).
template <int WMAX, bool MULTI, int PART>
__global__ void __launch_bounds__(kBThreads, PART == kSeedOnly ? IFA_BATCH_SEED_MIN_CTAS : IFA_BATCH_MIN_CTAS)
k_batch(Batch b, BatchWork w, QueryTable bt, QueryTable ft, HitSink sink) {
    using namespace brute;
    extern __shared__ uint4 smem4[];
    __shared__ __align__(16) ifa_hit wbuf[kBWarps][32];
    __shared__ __align__(8) uint2 stage[kBWarps][2][Stage<WMAX>::kSlots];
    __shared__ uint16_t cq[kBWarps][kQRows][32];
    __shared__ uint32_t s_nF, s_nM, s_item;
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t warp = threadIdx.x >> 5;
    WarpHitsT<MULTI> wh;
    wh.init(wbuf[warp]);
    uint32_t mul[kWin];
    lane_multipliers(mul);
    unsigned long long ncand = 0;
    int loaded = -1;
    Smem m{};
    uint32_t nent = 0, e0 = 0, lmin = 0, lmax = 0;
    const uint32_t n_seed = w.n_items - w.n_brute_items;
    const uint32_t item_end = PART == kSeedOnly ? n_seed : w.n_items;
    for (;;) {
        if (threadIdx.x == 0)
            s_item = PART == kBruteOnly ? n_seed + atomicAdd(w.queue + 1, 1u) : atomicAdd(w.queue, 1u);
        __syncthreads();
        const uint32_t item = s_item;
        if (item >= item_end) break;
        if (PART == kSeedOnly) {
            const uint64_t lo = w.s_block0 + static_cast<uint64_t>(item) * w.tile_sblocks;
            const uint64_t hi = lo + w.tile_sblocks < w.s_block_end ? lo + w.tile_sblocks : w.s_block_end;
            seed::seed_blocks<WMAX>(b, ft, w.tabs, w.emh, w.step, kSPerEntry, sink, wh, lo + warp, hi,
                                    kBWarps, lane, ncand);
        } else {
            const uint32_t bi = item - n_seed;
            const uint32_t chunk = bi / w.n_btiles, tile = bi % w.n_btiles;
            if (static_cast<int>(chunk) != loaded) {
                if (loaded >= 0) {
                    flush_counts(bt, m, nent, e0, sink);
                    __syncthreads();
                }
                e0 = w.chunk_e0[chunk];
                const uint32_t e1 = w.chunk_e1[chunk];
                lmin = w.chunk_lmin[chunk];
                lmax = w.chunk_lmax[chunk];
                m = load_chunk<WMAX>(bt, e0, e1, kSPerEntry, smem4, &s_nF, &s_nM);
                nent = e1 - e0;
                loaded = static_cast<int>(chunk);
            }
            const uint64_t lo = w.b_block0 + static_cast<uint64_t>(tile) * w.tile_bblocks;
            const uint64_t hi = lo + w.tile_bblocks < w.b_block_end ? lo + w.tile_bblocks : w.b_block_end;
            scan_blocks<WMAX>(b, bt, m, nent, s_nF, s_nM, e0, kSPerEntry, lmin, lmax, sink, wh, stage[warp], mul,
                              lo, hi, warp, kBWarps, lane, cq[warp]);
        }
        __syncthreads();
    }
    if (loaded >= 0) flush_counts(bt, m, nent, e0, sink);
    wh.finish(sink, lane);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ncand += __shfl_xor_sync(0xffffffffu, ncand, o);
    if (lane == 0 && ncand) atomicAdd(w.candidates, ncand);
}

template <int WMAX, int PART>
cudaError_t launch_batch_t(const Batch &b, const BatchWork &w, const QueryTable &bt, const QueryTable &ft,
                           const HitSink &sink, int grid, size_t smem, cudaStream_t st) {
    if (sink.q2r)
        k_batch<WMAX, true, PART><<<grid, kBThreads, smem, st>>>(b, w, bt, ft, sink);
    else
        k_batch<WMAX, false, PART><<<grid, kBThreads, smem, st>>>(b, w, bt, ft, sink);
    return cudaGetLastError();
}

template <int PART>
cudaError_t launch_batch_p(uint32_t wmax, const Batch &b, const BatchWork &w, const QueryTable &bt,
                           const QueryTable &ft, const HitSink &sink, int grid, size_t smem, cudaStream_t st) {
    switch (wmax) {
    case 1: return launch_batch_t<1, PART>(b, w, bt, ft, sink, grid, smem, st);
    case 2: return launch_batch_t<2, PART>(b, w, bt, ft, sink, grid, smem, st);
    case 4: return launch_batch_t<4, PART>(b, w, bt, ft, sink, grid, smem, st);
    case 8: return launch_batch_t<8, PART>(b, w, bt, ft, sink, grid, smem, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_batch(uint32_t wmax, const Batch &b, const BatchWork &w, const QueryTable &bt,
                         const QueryTable &ft, const HitSink &sink, int grid, size_t smem, cudaStream_t st,
                         int part) {
    if (part == kSeedOnly) return launch_batch_p<kSeedOnly>(wmax, b, w, bt, ft, sink, grid, smem, st);
    return launch_batch_p<kBruteOnly>(wmax, b, w, bt, ft, sink, grid, smem, st);
}

template <int PART>
int batch_grid_p(uint32_t wmax, size_t smem) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t e = cudaSuccess;
    switch (wmax) {
    case 1: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_batch<1, false, PART>, kBThreads, smem); break;
    case 2: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_batch<2, false, PART>, kBThreads, smem); break;
    case 4: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_batch<4, false, PART>, kBThreads, smem); break;
    default: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_batch<8, false, PART>, kBThreads, smem); break;
    }
    if (e != cudaSuccess || per < 1) per = 1;
    return sms * per;
}

// SMs x resident CTAs of the persistent kernel for `part` (the seed-only
// kernel takes no dynamic shared memory).  Tiles are sized for the
// brute-force kernel's grid.
int batch_grid(uint32_t wmax, int part = kBruteOnly) {
    if (part == kSeedOnly) return batch_grid_p<kSeedOnly>(wmax, 0);
    return batch_grid_p<kBruteOnly>(wmax, brute::kScanSmemBudget);
}

}  // namespace

namespace ifa {
cudaError_t launch_batch_kernels(uint32_t wmax, const Batch &b, const BatchWork &w, const QueryTable &bt,
                                 const QueryTable &ft, const HitSink &sink, cudaStream_t st, int *launches) {
    cudaError_t e = cudaSuccess;
    if (w.n_brute_items) {
        e = launch_batch(wmax, b, w, bt, ft, sink, batch_grid(wmax, kBruteOnly), brute::kScanSmemBudget, st,
                         kBruteOnly);
        if (launches) (*launches)++;
    }
    if (e == cudaSuccess && w.n_items > w.n_brute_items) {
        e = launch_batch(wmax, b, w, bt, ft, sink, batch_grid(wmax, kSeedOnly), 0, st, kSeedOnly);
        if (launches) (*launches)++;
    }
    return e;
}
int batch_kernel_grid(uint32_t wmax) { return batch_grid(wmax); }
}  // namespace ifa

namespace {

Batch store_batch(const BatchState &B) { return make_batch(B.ref, B.nbases, 0, B.d_pieces, B.d_pieces_n); }

// Grow a device array to `want` elements, keeping its first `keep` (the
// copy is finished before the old array is freed).
template <class T>
cudaError_t grow(T *&p, uint64_t &cap, uint64_t want, uint64_t keep, cudaStream_t st) {
    if (want <= cap && p) return cudaSuccess;
    T *n = nullptr;
    cudaError_t e = cudaMalloc(&n, want * sizeof(T));
    if (e != cudaSuccess) return e;
    if (p && keep) {
        e = cudaMemcpyAsync(n, p, keep * sizeof(T), cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) {
            cudaFree(n);
            return e;
        }
    }
    cudaFree(p);
    p = n;
    cap = want;
    return cudaSuccess;
}

HitSink handle_sink(const ifa_handle *h) {
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

ifa_status sync_pieces(ifa_handle *h) {
    BatchState &B = h->batch;
    if (!B.pieces_dirty) return IFA_OK;
    cudaFree(B.d_pieces);
    B.d_pieces = nullptr;
    BCK(h, cudaMalloc(&B.d_pieces, std::max<size_t>(1, B.pieces.size()) * sizeof(DevPiece)));
    if (!B.pieces.empty())
        BCK(h, cudaMemcpyAsync(B.d_pieces, B.pieces.data(), B.pieces.size() * sizeof(DevPiece), cudaMemcpyHostToDevice,
                               h->stream));
    B.d_pieces_n = static_cast<uint32_t>(B.pieces.size());
    B.pieces_dirty = false;
    return IFA_OK;
}

void free_plan(BatchState &B) {
    for (void *p : B.allocs) cudaFree(p);
    B.allocs.clear();
    B.merged.release();
    for (auto &p : B.per_set)
        if (p) p->release();
    B.per_set.clear();
    if (B.graph) cudaGraphExecDestroy(B.graph);
    B.graph = nullptr;
    B.graph_stream = nullptr;
    B.plan_valid = false;
    B.tc_rows = 0;
    B.d_tcA = nullptr;
    B.d_tcmeta = nullptr;
    B.d_tcids = nullptr;
    B.d_tcstatus = nullptr;
}

template <typename T>
T *plan_alloc(ifa_handle *h, size_t n, cudaError_t &e) {
    void *p = nullptr;
    cudaError_t r = cudaMalloc(&p, std::max<size_t>(1, n) * sizeof(T));
    if (r != cudaSuccess) {
        if (e == cudaSuccess) e = r;
        return nullptr;
    }
    h->batch.allocs.push_back(p);
    return static_cast<T *>(p);
}


}  // namespace

// ------------------------------------------------------------------ plan

namespace {

// Build the merged plan: modes of AUTO sets (autotuner), the compact brute
// table with its chunks, merged and per-set k-mer tables, work descriptor.
ifa_status build_plan(ifa_handle *h) {
    BatchState &B = h->batch;
    if (B.plan_valid) return IFA_OK;
    free_plan(B);
    ifa_status st = upload_queries(h);
    if (st != IFA_OK) return st;
    st = sync_pieces(h);
    if (st != IFA_OK) return st;
    const uint32_t nq = static_cast<uint32_t>(h->qs.size());
    const uint32_t wmax = h->wmax;
    B.wmax = wmax;
    std::vector<uint32_t> svec(nq, 0);
    for (uint32_t q = 0; q < nq; q++) svec[q] = q < h->qs_s.size() ? h->qs_s[q] : 0u;

    // indexed plan over every set that may run indexed (AUTO or INDEXED)
    std::vector<uint8_t> cand_in(nq, 0);
    for (const QuerySet &S : B.sets)
        if (S.mode != IFA_MODE_BRUTE)
            for (uint32_t q = S.first; q < S.first + S.n; q++) cand_in[q] = 1;
    IndexedState plan_all;
    if (std::any_of(cand_in.begin(), cand_in.end(), [](uint8_t x) { return x != 0; })) {
        st = indexed_plan_q(plan_all, h->qs, svec, cand_in, h->cfg, h->stream, h->err);
        if (st != IFA_OK) return st;
    }

    // autotuner: brute force or indexed per AUTO set, from measured rates
    for (QuerySet &S : B.sets) {
        if (S.mode == IFA_MODE_BRUTE) { S.chosen = IFA_MODE_BRUTE; continue; }
        if (S.mode == IFA_MODE_INDEXED) { S.chosen = IFA_MODE_INDEXED; continue; }
        const ModeCost c = predict_cost(B.rates, h->qs, S.first, S.n, plan_all, h->cfg.kmer_step);
        S.chosen = (!c.seeded || c.brute_s <= c.idx_s) ? IFA_MODE_BRUTE : IFA_MODE_INDEXED;
    }

    // queries that run indexed (seeded ones go to the merged tables; their
    // exhaustive ones to the compact brute table)
    std::vector<uint8_t> idx_in(nq, 0);
    for (const QuerySet &S : B.sets)
        if (S.chosen == IFA_MODE_INDEXED)
            for (uint32_t q = S.first; q < S.first + S.n; q++) idx_in[q] = 1;

    // brute-force sets the tensor cores scan: the streaming rule per set
    // (queries of at most 64 bases, 32 queries or more, sparse hits), or
    // every eligible one when the config forces the tensor cores
    std::vector<uint8_t> on_tc(B.sets.size(), 0);
    uint32_t tc_lmax = 0;
    for (size_t si = 0; si < B.sets.size(); si++) {
        const QuerySet &S = B.sets[si];
        if (S.chosen != IFA_MODE_BRUTE || h->cfg.brute_kernel == IFA_BRUTE_POPC) continue;
        uint32_t lmax = 0;
        for (uint32_t q = S.first; q < S.first + S.n; q++) lmax = std::max<uint32_t>(lmax, h->qs[q].size());
        const bool pick = h->cfg.brute_kernel == IFA_BRUTE_TENSOR ? tc_eligible(lmax)
                                                                  : tc_auto_choice(h->qs, S.first, S.n, S.s);
        if (pick) {
            on_tc[si] = 1;
            tc_lmax = std::max(tc_lmax, lmax);
        }
    }
    // the tensor-core operand: each such set's queries, padded with empty
    // ones to whole 128-row tiles (2 rows per query)
    std::vector<std::string> tc_qs;
    std::vector<uint32_t> tc_ids, tc_meta;
    B.set_tc_row0.assign(B.sets.size(), 0);
    B.set_tc_rows.assign(B.sets.size(), 0);
    for (size_t si = 0; si < B.sets.size(); si++) {
        if (!on_tc[si]) continue;
        const QuerySet &S = B.sets[si];
        B.set_tc_row0[si] = static_cast<uint32_t>(tc_ids.size());
        for (uint32_t q = S.first; q < S.first + S.n; q++) {
            tc_qs.push_back(h->qs[q]);
            for (uint32_t t = 0; t < 2; t++) {
                tc_ids.push_back(2 * q + t);
                tc_meta.push_back(h->qmeta_host[2 * q + t]);
            }
        }
        while (tc_ids.size() % 128) {
            tc_qs.emplace_back();
            tc_ids.insert(tc_ids.end(), {0u, 0u});
            tc_meta.insert(tc_meta.end(), {0u, 0u});
        }
        B.set_tc_rows[si] = static_cast<uint32_t>(tc_ids.size()) - B.set_tc_row0[si];
    }
    B.tc_rows = static_cast<uint32_t>(tc_ids.size());
    B.tc_lpad = B.tc_rows ? tc_lpad(tc_lmax) : 0;

    // compact brute table, set by set so each set's entries are contiguous
    std::vector<uint32_t> ids;
    B.set_bchunk_lo.assign(B.sets.size(), 0);
    B.set_bchunk_hi.assign(B.sets.size(), 0);
    B.bchunk_e0.clear();
    B.bchunk_e1.clear();
    B.bchunk_lmin.clear();
    B.bchunk_lmax.clear();
    uint32_t cap = brute::chunk_cap(static_cast<int>(wmax));
    cap = std::min<uint32_t>(cap, 65535) & ~1u;
    if (cap < 2) cap = 2;
    bool any_idx = false;
    for (size_t si = 0; si < B.sets.size(); si++) {
        const QuerySet &S = B.sets[si];
        const uint32_t start = static_cast<uint32_t>(ids.size());
        for (uint32_t q = S.first; q < S.first + S.n && !on_tc[si]; q++) {
            const bool brute = S.chosen == IFA_MODE_BRUTE || plan_all.plan_exhaustive[q];
            if (S.chosen == IFA_MODE_INDEXED && !plan_all.plan_exhaustive[q]) any_idx = true;
            if (!brute) continue;
            ids.push_back(2 * q);
            ids.push_back(2 * q + 1);
        }
        const uint32_t end = static_cast<uint32_t>(ids.size());
        B.set_bchunk_lo[si] = static_cast<uint32_t>(B.bchunk_e0.size());
        for (uint32_t a = start; a < end; a += cap) {
            const uint32_t z = std::min(end, a + cap);
            uint32_t lo = 0xffffffffu, hi = 0;
            for (uint32_t i = a; i < z; i++) {
                const uint32_t L = meta_L(h->qmeta_host[ids[i]]);
                lo = std::min(lo, L);
                hi = std::max(hi, L);
            }
            B.bchunk_e0.push_back(a);
            B.bchunk_e1.push_back(z);
            B.bchunk_lmin.push_back(lo);
            B.bchunk_lmax.push_back(hi);
        }
        B.set_bchunk_hi[si] = static_cast<uint32_t>(B.bchunk_e0.size());
    }
    B.b_entries = static_cast<uint32_t>(ids.size());
    cudaError_t e = cudaSuccess;
    const uint32_t nbe = std::max<uint32_t>(1, B.b_entries);
    std::vector<uint4> bw(static_cast<size_t>(nbe) * wmax, make_uint4(0, 0, 0, 0));
    std::vector<uint32_t> bm(nbe, 0);
    for (uint32_t i = 0; i < B.b_entries; i++) {
        bm[i] = h->qmeta_host[ids[i]];
        for (uint32_t j = 0; j < wmax; j++) bw[static_cast<size_t>(i) * wmax + j] = h->qwords_host[static_cast<size_t>(ids[i]) * wmax + j];
    }
    uint4 *d_bw = plan_alloc<uint4>(h, bw.size(), e);
    uint32_t *d_bm = plan_alloc<uint32_t>(h, nbe, e);
    uint32_t *d_bids = plan_alloc<uint32_t>(h, nbe, e);
    const size_t nch = std::max<size_t>(1, B.bchunk_e0.size());
    uint32_t *d_c0 = plan_alloc<uint32_t>(h, nch, e), *d_c1 = plan_alloc<uint32_t>(h, nch, e);
    uint32_t *d_cl = plan_alloc<uint32_t>(h, nch, e), *d_ch = plan_alloc<uint32_t>(h, nch, e);
    if (e == cudaSuccess) {
        // on the compute stream, ahead of the kernels that read them (pageable
        // sources are staged before each call returns)
        const cudaMemcpyKind hd = cudaMemcpyHostToDevice;
        e = cudaMemcpyAsync(d_bw, bw.data(), bw.size() * sizeof(uint4), hd, h->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(d_bm, bm.data(), nbe * sizeof(uint32_t), hd, h->stream);
        if (e == cudaSuccess && !ids.empty())
            e = cudaMemcpyAsync(d_bids, ids.data(), ids.size() * sizeof(uint32_t), hd, h->stream);
        if (e == cudaSuccess && !B.bchunk_e0.empty()) {
            const size_t nb = B.bchunk_e0.size() * sizeof(uint32_t);
            e = cudaMemcpyAsync(d_c0, B.bchunk_e0.data(), nb, hd, h->stream);
            if (e == cudaSuccess) e = cudaMemcpyAsync(d_c1, B.bchunk_e1.data(), nb, hd, h->stream);
            if (e == cudaSuccess) e = cudaMemcpyAsync(d_cl, B.bchunk_lmin.data(), nb, hd, h->stream);
            if (e == cudaSuccess) e = cudaMemcpyAsync(d_ch, B.bchunk_lmax.data(), nb, hd, h->stream);
        }
    }
    if (e == cudaSuccess && B.tc_rows) {
        std::vector<uint8_t> op;
        tc_operand(tc_qs, B.tc_lpad, op);
        B.d_tcA = plan_alloc<uint8_t>(h, op.size(), e);
        B.d_tcmeta = plan_alloc<uint32_t>(h, B.tc_rows, e);
        B.d_tcids = plan_alloc<uint32_t>(h, B.tc_rows, e);
        B.d_tcstatus = plan_alloc<unsigned int>(h, 2, e);
        const cudaMemcpyKind hd = cudaMemcpyHostToDevice;
        if (e == cudaSuccess) e = cudaMemcpyAsync(B.d_tcA, op.data(), op.size(), hd, h->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(B.d_tcmeta, tc_meta.data(), B.tc_rows * sizeof(uint32_t), hd, h->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(B.d_tcids, tc_ids.data(), B.tc_rows * sizeof(uint32_t), hd, h->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(B.d_tcstatus, 0, 2 * sizeof(unsigned int), h->stream);
        if (e == cudaSuccess) e = tc_prepare();   // kernel attributes, outside any stream capture
    }
    if (e != cudaSuccess) return bfail(h, IFA_ERR_CUDA, std::string("batch plan: ") + cudaGetErrorString(e));

    // merged tables of the indexed sets (seeded queries only)
    if (any_idx) {
        std::vector<uint8_t> seeded(nq, 0);
        for (uint32_t q = 0; q < nq; q++) seeded[q] = idx_in[q] && !plan_all.plan_exhaustive[q];
        st = indexed_plan_q(B.merged, h->qs, svec, seeded, h->cfg, h->stream, h->err);
        if (st != IFA_OK) return st;
        st = indexed_tables(B.merged, h->qs, h->qmeta_host, h->qwords_host, wmax, h->cfg, h->stream, h->err);
        if (st != IFA_OK) return st;
    }
    // per-set tables for the per-set baseline
    B.per_set.clear();
    for (const QuerySet &S : B.sets) {
        B.per_set.emplace_back(new IndexedState());
        if (S.chosen != IFA_MODE_INDEXED) continue;
        std::vector<uint8_t> mine(nq, 0);
        for (uint32_t q = S.first; q < S.first + S.n; q++) mine[q] = !plan_all.plan_exhaustive[q];
        if (std::none_of(mine.begin(), mine.end(), [](uint8_t x) { return x != 0; })) continue;
        st = indexed_plan_q(*B.per_set.back(), h->qs, svec, mine, h->cfg, h->stream, h->err);
        if (st != IFA_OK) return st;
        st = indexed_tables(*B.per_set.back(), h->qs, h->qmeta_host, h->qwords_host, wmax, h->cfg, h->stream, h->err);
        if (st != IFA_OK) return st;
        cudaMalloc(&B.per_set.back()->d_candidates, sizeof(unsigned long long));
    }

    // work descriptor and tiles
    if (!B.d_queue) BCK(h, cudaMalloc(&B.d_queue, 2 * sizeof(unsigned int)));   // seed and brute-force items
    if (!B.d_cand) BCK(h, cudaMalloc(&B.d_cand, sizeof(unsigned long long)));
    B.grid = batch_grid(wmax);
    BatchWork &W = B.work;
    W = BatchWork{};
    W.bwords = d_bw;
    W.bmeta = d_bm;
    W.bids = d_bids;
    W.chunk_e0 = d_c0;
    W.chunk_e1 = d_c1;
    W.chunk_lmin = d_cl;
    W.chunk_lmax = d_ch;
    W.nchunks = static_cast<uint32_t>(B.bchunk_e0.size());
    W.tabs = B.merged.tables_valid ? B.merged.targ : KTablesArg{};
    W.emh = B.merged.d_entry_minhits;
    W.step = h->cfg.kmer_step;
    W.qwords = h->d_qwords;
    W.qmeta = h->d_qmeta;
    const uint64_t nbblk = (B.nbases + 32 * brute::kWin - 1) / (32 * brute::kWin);
    const uint64_t nsblk = (B.nbases + 31) / 32;
    // tiles: about 16 items per CTA slot over all chunks, at least 32 blocks per tile
    const uint64_t want_b = static_cast<uint64_t>(16) * B.grid;
    const uint64_t tiles_per_chunk = W.nchunks ? std::max<uint64_t>(1, want_b / W.nchunks) : 1;
    W.b_block0 = 0;
    W.b_block_end = nbblk;
    W.s_block0 = 0;
    W.s_block_end = nsblk;
    W.tile_bblocks = std::max<uint64_t>(32, (nbblk + tiles_per_chunk - 1) / tiles_per_chunk);
    W.n_btiles = static_cast<uint32_t>((nbblk + W.tile_bblocks - 1) / W.tile_bblocks);
    W.tile_sblocks = std::max<uint64_t>(64, (nsblk + 8 * B.grid - 1) / (8 * B.grid));
    W.n_stiles = W.tabs.n ? static_cast<uint32_t>((nsblk + W.tile_sblocks - 1) / W.tile_sblocks) : 0;
    W.n_brute_items = W.nchunks * W.n_btiles;
    W.n_items = W.n_brute_items + W.n_stiles;
    W.queue = B.d_queue;
    W.candidates = B.d_cand;
    B.plan_valid = true;
    return IFA_OK;
}

// Measure the autotuner's three rates on a slice of the store (once per
// handle), with count-only sinks so no result is touched.
ifa_status calibrate(ifa_handle *h) {
    BatchState &B = h->batch;
    if (B.rates.valid()) return IFA_OK;
    ifa_status st = sync_pieces(h);
    if (st != IFA_OK) return st;
    std::vector<uint32_t> svec(h->qs.size(), 0);
    for (size_t q = 0; q < svec.size(); q++) svec[q] = q < h->qs_s.size() ? h->qs_s[q] : 0u;
    return rates_on_store(h, store_batch(B), h->qs, svec, B.rates);
}

}  // namespace

namespace ifa {
// Free the store and the plan of a handle (at ifa_destroy).
void batch_release(ifa_handle *h) {
    BatchState &B = h->batch;
    free_plan(B);
    refbufs_free(B.ref);
    B.exc_used = 0;
    cudaFree(B.d_pieces);
    cudaFree(B.d_queue);
    cudaFree(B.d_cand);
    B.d_pieces = nullptr;
    B.d_queue = nullptr;
    B.d_cand = nullptr;
}
}  // namespace ifa

// ------------------------------------------------------------------ ABI

extern "C" {

ifa_status ifa_ref_append(ifa_handle *h, const uint8_t *ascii, uint64_t len, const ifa_piece *pieces,
                          uint32_t n, ifa_mem mem) {
    if (!h) return IFA_ERR_INVALID_ARG;
    if (len == 0 && n == 0) return IFA_OK;
    if (!ascii || !pieces || len == 0 || n == 0)
        return bfail(h, IFA_ERR_INVALID_ARG, "ifa_ref_append: bytes and at least one piece needed");
    if (mem != IFA_MEM_HOST && mem != IFA_MEM_HOST_PINNED && mem != IFA_MEM_DEVICE &&
        mem != IFA_MEM_HOST_PINNED_ASYNC)
        return bfail(h, IFA_ERR_INVALID_ARG, "ifa_ref_append: unknown memory kind");
    BatchState &B = h->batch;
    if (B.nbases % 32 != 0)
        return bfail(h, IFA_ERR_INVALID_ARG, "ifa_ref_append: the previous append was not a multiple of 32 bases");
    uint64_t at = 0;
    for (uint32_t i = 0; i < n; i++) {
        const ifa_piece &p = pieces[i];
        if (p.start != at || p.len == 0)
            return bfail(h, IFA_ERR_INVALID_ARG, "ifa_ref_append: pieces must be contiguous, non-empty, from 0");
        at += p.len;
        if (!p.last && i + 1 != n) return bfail(h, IFA_ERR_INVALID_ARG, "ifa_ref_append: only the last piece may continue");
        if (i == 0 && B.open) {
            if (p.contig != B.open_contig || p.offset_in_contig != B.open_next)
                return bfail(h, IFA_ERR_INVALID_ARG, "ifa_ref_append: must continue the open contig");
        } else {
            if (p.offset_in_contig != 0) return bfail(h, IFA_ERR_INVALID_ARG, "ifa_ref_append: a new contig starts at 0");
            const bool have_prev = i > 0 || B.any_contig;
            const uint32_t prev = i > 0 ? pieces[i - 1].contig : B.last_contig;
            if (have_prev && p.contig <= prev) return bfail(h, IFA_ERR_INVALID_ARG, "ifa_ref_append: contig ids must increase");
        }
        if (p.offset_in_contig + p.len > 0xffffffffull)
            return bfail(h, IFA_ERR_INVALID_ARG, "ifa_ref_append: contig longer than 2^32 - 1 bases");
    }
    if (at != len) return bfail(h, IFA_ERR_INVALID_ARG, "ifa_ref_append: pieces must cover the bytes");
    const NvtxRange nvtx("ifa_ref_append");
    BCK(h, cudaSetDevice(h->dev));
    BCK(h, cudaStreamSynchronize(h->stream));
    // grow the store (geometric), keeping the packed words and directory
    const uint64_t seg = h->cfg.segment_bytes & ~uint64_t(31);
    const uint64_t old_words = B.nbases / 32;
    const uint64_t need = (B.nbases + len + 31) / 32 + kStorePad;
    if (need > B.ref.words_cap || !B.ref.hl) {
        const uint64_t cap = std::max<uint64_t>(need, B.ref.words_cap + B.ref.words_cap / 2);
        uint64_t hc = B.ref.words_cap, dc = B.ref.words_cap ? dir_entries(B.ref.words_cap) : 0;
        BCK(h, grow(B.ref.hl, hc, cap, old_words, h->stream));
        BCK(h, grow(B.ref.dir, dc, dir_entries(cap), dir_entries(old_words + 1), h->stream));
        B.ref.words_cap = cap;
    }
    const uint64_t chunk_words = (std::min<uint64_t>(seg, len) + 31) / 32 + kStorePad;
    if (chunk_words > B.ref.nb_cap) {
        cudaFree(B.ref.nb);
        B.ref.nb = nullptr;
        B.ref.nb_cap = 0;
        BCK(h, cudaMalloc(&B.ref.nb, chunk_words * sizeof(uint2)));
        B.ref.nb_cap = chunk_words;
    }
    if (!B.ref.exc) {
        uint64_t c = 0;
        BCK(h, grow(B.ref.exc, c, std::max<uint64_t>(1u << 16, need / 64), 0, h->stream));
        B.ref.exc_cap = c;
        BCK(h, cudaMalloc(&B.ref.exc_n, 2 * sizeof(unsigned long long)));
    }
    // the new pieces (a continuation extends the open piece); their start bits
    // go into each chunk's masks
    std::vector<DevPiece> fresh;
    for (uint32_t i = 0; i < n; i++) {
        if (i == 0 && B.open) continue;
        DevPiece d;
        d.start = B.nbases + pieces[i].start;
        d.contig_off = 0;
        d.contig = pieces[i].contig;
        d.last = pieces[i].last ? 1u : 0u;
        fresh.push_back(d);
    }
    DevPiece *dfresh = nullptr;
    struct FreeLater {
        DevPiece *&p;
        ~FreeLater() { cudaFree(p); }
    } free_later{dfresh};
    if (!fresh.empty()) {
        BCK(h, cudaMalloc(&dfresh, fresh.size() * sizeof(DevPiece)));
        BCK(h, cudaMemcpyAsync(dfresh, fresh.data(), fresh.size() * sizeof(DevPiece), cudaMemcpyHostToDevice,
                               h->stream));
    }
    // copy (via the handle's segment buffer) and pack, one segment at a time
    for (uint64_t off = 0; off < len; off += seg) {
        const uint64_t c = std::min<uint64_t>(seg, len - off);
        const uint8_t *src = ascii + off;
        if (mem != IFA_MEM_DEVICE) {
            BCK(h, cudaMemcpyAsync(h->d_seg[0], src, c, cudaMemcpyHostToDevice, h->stream));
            src = h->d_seg[0];
        }
        const uint64_t w0 = (B.nbases + off) / 32;
        const uint64_t nw = (c + 31) / 32 + kStorePad;
        BCK(h, launch_pack(nullptr, 0, 0, src, c, B.ref.hl + w0, B.ref.nb, nw, h->stream));
        if (!fresh.empty())
            BCK(h, launch_mark_pieces(dfresh, static_cast<uint32_t>(fresh.size()), 32 * w0, nw, B.ref.nb, h->stream));
        // directory and exceptions; when the exception table runs out it
        // grows and the build runs again (it is idempotent)
        for (;;) {
            const unsigned long long cnt[2] = {B.exc_used, 0ull};
            BCK(h, cudaMemcpyAsync(B.ref.exc_n, cnt, sizeof(cnt), cudaMemcpyHostToDevice, h->stream));
            BCK(h, launch_build_dir(B.ref.nb, w0, nw, B.ref.dir, B.ref.exc, B.ref.exc_cap, B.ref.exc_n, h->stream));
            unsigned long long got[2] = {0, 0};
            BCK(h, cudaMemcpyAsync(got, B.ref.exc_n, sizeof(got), cudaMemcpyDeviceToHost, h->stream));
            BCK(h, cudaStreamSynchronize(h->stream));
            if (!got[1]) {
                B.exc_used = got[0];
                break;
            }
            // directory bases are 32-bit
            const uint64_t want = std::min<uint64_t>(std::max<uint64_t>(2 * B.ref.exc_cap, got[0] + nw), 0xffffffffull);
            if (want <= B.ref.exc_cap)
                return bfail(h, IFA_ERR_INVALID_ARG, "ifa_ref_append: more than 2^32 - 1 words hold an N or a contig start");
            BCK(h, grow(B.ref.exc, B.ref.exc_cap, want, B.exc_used, h->stream));
        }
    }
    if (!fresh.empty()) B.pieces.insert(B.pieces.end(), fresh.begin(), fresh.end());
    // a contig continued from the previous append ends here: its piece is now its last
    if (B.open && pieces[0].last && !B.pieces.empty()) B.pieces[B.pieces.size() - fresh.size() - 1].last = 1u;
    const ifa_piece &lp = pieces[n - 1];
    B.open = !lp.last;
    B.open_contig = lp.contig;
    B.open_next = lp.offset_in_contig + lp.len;
    B.any_contig = true;
    B.last_contig = lp.contig;
    B.nbases += len;
    B.pieces_dirty = true;
    B.plan_valid = false;
    B.rates = Rates{};
    return IFA_OK;
}

ifa_status ifa_ref_reserve(ifa_handle *h, uint64_t bases) {
    if (!h) return IFA_ERR_INVALID_ARG;
    BCK(h, cudaSetDevice(h->dev));
    BCK(h, cudaStreamSynchronize(h->stream));
    BatchState &B = h->batch;
    const uint64_t want = (std::max<uint64_t>(bases, B.nbases) + 31) / 32 + kStorePad;
    if (want <= B.ref.words_cap && B.ref.hl) return IFA_OK;
    const uint64_t old_words = B.nbases / 32;
    uint64_t hc = B.ref.words_cap, dc = B.ref.words_cap ? dir_entries(B.ref.words_cap) : 0;
    BCK(h, grow(B.ref.hl, hc, want, old_words, h->stream));
    BCK(h, grow(B.ref.dir, dc, dir_entries(want), dir_entries(old_words + 1), h->stream));
    B.ref.words_cap = want;
    return IFA_OK;
}

ifa_status ifa_ref_reset(ifa_handle *h) {
    if (!h) return IFA_ERR_INVALID_ARG;
    BCK(h, cudaSetDevice(h->dev));
    BCK(h, cudaStreamSynchronize(h->stream));
    BatchState &B = h->batch;
    free_plan(B);
    refbufs_free(B.ref);
    B.exc_used = 0;
    cudaFree(B.d_pieces);
    B.d_pieces = nullptr;
    B.nbases = 0;
    B.pieces.clear();
    B.d_pieces_n = 0;
    B.pieces_dirty = true;
    B.open = false;
    B.any_contig = false;
    B.rates = Rates{};
    return IFA_OK;
}

ifa_status ifa_set_add(ifa_handle *h, const uint8_t *const *seqs, const uint32_t *lens, uint32_t n,
                       uint32_t max_subs, ifa_mode mode, uint32_t *set_id, uint32_t *first_query) {
    if (!h) return IFA_ERR_INVALID_ARG;
    if (mode != IFA_MODE_AUTO && mode != IFA_MODE_BRUTE && mode != IFA_MODE_INDEXED)
        return bfail(h, IFA_ERR_INVALID_ARG, "ifa_set_add: unknown mode");
    if (n == 0) return bfail(h, IFA_ERR_INVALID_ARG, "ifa_set_add: empty set");
    if (h->pushed) return bfail(h, IFA_ERR_BAD_STATE, "ifa_set_add: the handle is streaming segments");
    const uint32_t first = static_cast<uint32_t>(h->qs.size());
    ifa_status st = ifa_load_queries(h, seqs, lens, n, nullptr);
    if (st != IFA_OK) return st;
    h->qs_s.resize(first, 0);
    h->qs_s.resize(first + n, std::min<uint32_t>(max_subs, 255));
    QuerySet S;
    S.first = first;
    S.n = n;
    S.s = std::min<uint32_t>(max_subs, 255);
    S.mode = mode;
    h->batch.sets.push_back(S);
    h->batch.plan_valid = false;
    if (set_id) *set_id = static_cast<uint32_t>(h->batch.sets.size() - 1);
    if (first_query) *first_query = first;
    return IFA_OK;
}

ifa_status ifa_batch_run(ifa_handle *h, ifa_batch_kind kind, ifa_set_result *per_set) {
    if (!h) return IFA_ERR_INVALID_ARG;
    BatchState &B = h->batch;
    if (B.nbases == 0 || B.sets.empty()) return bfail(h, IFA_ERR_BAD_STATE, "ifa_batch_run: empty store or no sets");
    if (kind != IFA_BATCH_PERSISTENT && kind != IFA_BATCH_PER_SET)
        return bfail(h, IFA_ERR_INVALID_ARG, "ifa_batch_run: unknown kind");
    const NvtxRange nvtx(kind == IFA_BATCH_PERSISTENT ? "ifa_batch_run persistent" : "ifa_batch_run per set");
    BCK(h, cudaSetDevice(h->dev));
    ifa_status st = calibrate(h);
    if (st != IFA_OK) return st;
    st = build_plan(h);
    if (st != IFA_OK) return st;
    const Batch b = store_batch(B);
    const HitSink sink = handle_sink(h);
    QueryTable bt;
    bt.words = B.work.bwords;
    bt.meta = B.work.bmeta;
    bt.ids = B.work.bids;
    bt.n_entries = B.b_entries;
    bt.wmax = B.wmax;
    QueryTable ft;
    ft.words = h->d_qwords;
    ft.meta = h->d_qmeta;
    ft.ids = nullptr;
    ft.n_entries = 2 * static_cast<uint32_t>(h->qs.size());
    ft.wmax = B.wmax;
    cudaEvent_t start, stop;
    BCK(h, cudaEventCreate(&start));
    BCK(h, cudaEventCreate(&stop));
    std::vector<cudaEvent_t> done(B.sets.size(), nullptr);
    cudaError_t e = cudaEventRecord(start, h->stream);
    if (kind == IFA_BATCH_PERSISTENT) {
        if (!B.graph || B.graph_stream != h->stream) {
            if (B.graph) cudaGraphExecDestroy(B.graph);
            B.graph = nullptr;
            cudaGraph_t g = nullptr;
            const size_t smem = brute::kScanSmemBudget;
            e = cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                cudaError_t e1 = cudaMemsetAsync(B.d_queue, 0, 2 * sizeof(unsigned int), h->stream);
                // one persistent kernel per kind of item, each at its own
                // register budget, back to back
                cudaError_t e2 = cudaSuccess;
                if (B.work.n_brute_items)
                    e2 = launch_batch(B.wmax, b, B.work, bt, ft, sink, batch_grid(B.wmax, kBruteOnly), smem,
                                      h->stream, kBruteOnly);
                if (e2 == cudaSuccess && B.work.n_items > B.work.n_brute_items)
                    e2 = launch_batch(B.wmax, b, B.work, bt, ft, sink, batch_grid(B.wmax, kSeedOnly), 0, h->stream,
                                      kSeedOnly);
                // the tensor-core sets, every row at its own maxSubs
                if (e2 == cudaSuccess && B.tc_rows)
                    e2 = launch_scan_tc(b, B.d_tcA, B.d_tcmeta, B.tc_rows, B.tc_lpad, kSPerEntry, sink,
                                        B.d_tcstatus, h->stream, 0, B.d_tcids);
                // soft-clipped windows at the store's contig ends, every set's
                // entries at their own maxSubs, exhaustively in both modes
                if (e2 == cudaSuccess && h->cfg.clip_pct)
                    e2 = launch_clip_scan(b, ft, ft.n_entries, h->cfg.clip_pct, kSPerEntry, h->lmax, sink, h->stream);
                e = cudaStreamEndCapture(h->stream, &g);
                if (e == cudaSuccess) e = e1 != cudaSuccess ? e1 : e2;
            }
            if (e == cudaSuccess) e = cudaGraphInstantiate(&B.graph, g, 0);
            if (g) cudaGraphDestroy(g);
            B.graph_stream = h->stream;
        }
        if (e == cudaSuccess) e = cudaGraphLaunch(B.graph, h->stream);
        h->stats.kernel_launches += 1;
    } else {
        for (size_t si = 0; si < B.sets.size() && e == cudaSuccess; si++) {
            const QuerySet &S = B.sets[si];
            if (B.set_tc_rows[si]) {
                const size_t r0 = B.set_tc_row0[si];
                e = launch_scan_tc(b, B.d_tcA + r0 * 4u * B.tc_lpad, B.d_tcmeta + r0, B.set_tc_rows[si], B.tc_lpad,
                                   kSPerEntry, sink, B.d_tcstatus, h->stream, 0, B.d_tcids + r0);
                h->stats.kernel_launches += 1;
            }
            for (uint32_t c = B.set_bchunk_lo[si]; c < B.set_bchunk_hi[si] && e == cudaSuccess; c++) {
                int launches = 0;
                e = launch_scan_brute(b, bt, B.bchunk_e0[c], B.bchunk_e1[c], kSPerEntry, B.bchunk_lmin[c],
                                      B.bchunk_lmax[c], sink, h->stream, &launches);
                h->stats.kernel_launches += launches;
            }
            IndexedState &I = *B.per_set[si];
            if (e == cudaSuccess && S.chosen == IFA_MODE_INDEXED && I.tables_valid && I.targ.n) {
                e = launch_seed_scan(b, ft, I.targ, I.d_entry_minhits, h->cfg.kmer_step, kSPerEntry, sink,
                                     I.d_candidates ? I.d_candidates : B.d_cand, h->stream);
                h->stats.kernel_launches += 1;
            }
            if (e == cudaSuccess && h->cfg.clip_pct) {
                uint32_t lmax = 0;
                for (uint32_t q = S.first; q < S.first + S.n; q++)
                    lmax = std::max<uint32_t>(lmax, static_cast<uint32_t>(h->qs[q].size()));
                e = launch_clip_scan(b, ft, 2 * S.n, h->cfg.clip_pct, kSPerEntry, lmax, sink, h->stream, 2 * S.first);
                h->stats.kernel_launches += 1;
            }
            if (e == cudaSuccess) e = cudaEventCreate(&done[si]);
            if (e == cudaSuccess) e = cudaEventRecord(done[si], h->stream);
        }
    }
    if (e == cudaSuccess) e = cudaEventRecord(stop, h->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(stop);
    float total = 0;
    if (e == cudaSuccess) cudaEventElapsedTime(&total, start, stop);
    if (e == cudaSuccess && per_set) {
        std::vector<unsigned long long> qc(h->qs.size(), 0);
        e = cudaMemcpy(qc.data(), h->d_qcount, qc.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost);
        for (size_t si = 0; si < B.sets.size() && e == cudaSuccess; si++) {
            const QuerySet &S = B.sets[si];
            ifa_set_result &r = per_set[si];
            r.mode = S.chosen;
            r.queries = S.n;
            r.hits = 0;
            for (uint32_t q = S.first; q < S.first + S.n; q++) r.hits += qc[q];
            r.done_ms = total;
            if (done[si]) cudaEventElapsedTime(&r.done_ms, start, done[si]);
            r.pad = 0;
        }
    }
    for (cudaEvent_t d : done)
        if (d) cudaEventDestroy(d);
    cudaEventDestroy(start);
    cudaEventDestroy(stop);
    if (e != cudaSuccess) return bfail(h, IFA_ERR_CUDA, std::string("ifa_batch_run: ") + cudaGetErrorString(e));
    if (B.tc_rows) {
        unsigned int tcs = 0;
        BCK(h, cudaMemcpy(&tcs, B.d_tcstatus, sizeof(tcs), cudaMemcpyDeviceToHost));
        if (tcs) return bfail(h, IFA_ERR_TIMEOUT, "ifa_batch_run: a tensor-core pipeline wait gave up; results incomplete");
    }
    return IFA_OK;
}

}  // extern "C"

// indexed.cu -- indexed mode (Methods, indexed mode).
//
// The paper indexes each reference contig (PackedIndex) and looks the query
// seeds up in it, counting seed hits per diagonal before verifying
// candidates.  On the GPU the roles are inverted: the query k-mers are
// tabulated once, and every reference position's k-mer is looked up in
// that table as the segment streams past.  The set of (query, strand,
// window) candidates is the same either way.
//
// Per-diagonal counting without counters: each seed hit (query entry e,
// offset o, reference position j) names the window p = j - o, which is
// verified at once.  Verification builds the window's mismatch bitmask x;
// the k-mer at offset o' is error-free exactly when x has no set bit among
// its counted positions, so the window's full seed count S and its first
// seed come out of x.  The window is reported by the seed hit whose offset
// is that first seed (so exactly once), when mm <= maxSubs and
// |S| >= minHits.  This equals "seed count on the diagonal reaches the
// threshold, then Hamming verification".
//
// Queries that contain N, or that get no usable seed length, are scanned
// exhaustively by the brute-force kernel (compacted table).
#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>

#include "hits.cuh"
#include "indexed.cuh"
#include "seed_scan.cuh"
#include "status.cuh"

namespace ifa {

namespace {

constexpr int kSeedThreads = 256;
constexpr int kSeedWarps = kSeedThreads / kWarp;
// Resident CTAs per SM the register allocation is held to: the scan waits
// on chains of dependent L2 reads, so more resident warps hide more of them.
// Measured on B300 (1 Gbp, 10,000 queries, maxSubs 4 / 8 / 16): 4 CTAs
// (64 registers) 59.5 / 85.0 / 149.6 ms; 5 (48, a few spilled words)
// 59.2 / 81.9 / 146.5 ms; 6 (40) 59.7 / 81.3 / 148.9 ms.
#ifndef IFA_SEED_MIN_CTAS
#define IFA_SEED_MIN_CTAS 5
#endif

template <int WMAX>
__global__ void __launch_bounds__(kSeedThreads, IFA_SEED_MIN_CTAS)
k_seed_scan(Batch b, QueryTable qt, KTablesArg tabs, const uint32_t *__restrict__ entry_minhits,
            uint32_t step, uint32_t s, HitSink sink, unsigned long long *candidates) {
    __shared__ __align__(16) ifa_hit wbuf[kSeedWarps][32];
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t warp = threadIdx.x >> 5;
    WarpHits wh;
    wh.init(wbuf[warp]);
    unsigned long long ncand = 0;
    const uint64_t nblocks = (b.nbases + 31) >> 5;
    const uint64_t stride = static_cast<uint64_t>(gridDim.x) * kSeedWarps;
    seed::seed_blocks<WMAX>(b, qt, tabs, entry_minhits, step, s, sink, wh,
                            static_cast<uint64_t>(blockIdx.x) * kSeedWarps + warp, nblocks, stride, lane, ncand);
    wh.finish(sink, lane);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ncand += __shfl_xor_sync(0xffffffffu, ncand, o);
    if (lane == 0 && ncand) atomicAdd(candidates, ncand);
}

template <int WMAX>
cudaError_t seed_launch_t(const Batch &b, const QueryTable &qt, const KTablesArg &tabs,
                          const uint32_t *emh, uint32_t step, uint32_t s, const HitSink &sink,
                          unsigned long long *cand, cudaStream_t st) {
    static int grids[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    int &grid = grids[dev & 63];
    if (grid == 0) {
        int sms = 0, per_sm = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_seed_scan<WMAX>, kSeedThreads, 0);
        grid = sms * (per_sm > 0 ? per_sm : 1);
    }
    const uint64_t nblocks = (b.nbases + 31) >> 5;
    const uint64_t need = (nblocks + kSeedWarps - 1) / kSeedWarps;
    int g = static_cast<int>(need < static_cast<uint64_t>(grid) ? need : grid);
    if (g < 1) g = 1;
    k_seed_scan<WMAX><<<g, kSeedThreads, 0, st>>>(b, qt, tabs, emh, step, s, sink, cand);
    return cudaGetLastError();
}

bool has_n(const std::string &q) {
    for (char c : q)
        if (!is_base(static_cast<uint8_t>(c))) return true;
    return false;
}

uint32_t care_mask(uint32_t k, uint32_t mask_w) {
    uint32_t full = (k >= 32) ? 0xffffffffu : ((1u << k) - 1u);
    if (!mask_w) return full;
    const uint32_t mlo = (k - mask_w) / 2;
    return full & ~(((1u << mask_w) - 1u) << mlo);
}

}  // namespace

cudaError_t launch_seed_scan(const Batch &b, const QueryTable &qt, const KTablesArg &tabs,
                             const uint32_t *emh, uint32_t step, uint32_t s, const HitSink &sink,
                             unsigned long long *cand, cudaStream_t st) {
    switch (qt.wmax) {
    case 1: return seed_launch_t<1>(b, qt, tabs, emh, step, s, sink, cand, st);
    case 2: return seed_launch_t<2>(b, qt, tabs, emh, step, s, sink, cand, st);
    case 4: return seed_launch_t<4>(b, qt, tabs, emh, step, s, sink, cand, st);
    case 8: return seed_launch_t<8>(b, qt, tabs, emh, step, s, sink, cand, st);
    default: return cudaErrorInvalidValue;
    }
}

void IndexedState::free_tables() {
    // the buffers stay for the next build; only the plan's view is dropped
    targ = KTablesArg{};
    d_entry_minhits = nullptr;
    d_ex_words = nullptr;
    d_ex_meta = nullptr;
    d_ex_ids = nullptr;
    ex_entries = 0;
    ex_chunks.clear();
    any_exhaustive = false;
    tables_valid = false;
}

void IndexedState::release() {
    free_tables();
    bufs.release();
    cudaFree(d_candidates);
    d_candidates = nullptr;
}

uint64_t IndexedState::candidates_host(cudaStream_t st) const {
    if (!d_candidates) return 0;
    unsigned long long v = 0;
    cudaStreamSynchronize(st);
    cudaMemcpy(&v, d_candidates, sizeof(v), cudaMemcpyDeviceToHost);
    return v;
}

namespace {

// Thresholds are a pure function of the bin and the Monte Carlo settings, so
// they are remembered for the life of the process (query sets that come and
// go reuse the same bins).
struct BinKey {
    uint32_t L, s, k, step, mask, clips, num, den, trials;
    uint64_t seed;
    bool operator<(const BinKey &o) const {
        return std::tie(L, s, k, step, mask, clips, num, den, trials, seed) <
               std::tie(o.L, o.s, o.k, o.step, o.mask, o.clips, o.num, o.den, o.trials, o.seed);
    }
};
std::mutex g_bin_mutex;
std::map<BinKey, uint32_t> g_bin_cache;

}  // namespace

ifa_status minhits_device(const uint32_t *L, const uint32_t *subs, const uint32_t *k, uint32_t n,
                          uint32_t step, uint32_t mask_w, uint32_t max_clips, uint32_t num, uint32_t den,
                          uint32_t trials, uint64_t seed, uint32_t *out, cudaStream_t st,
                          uint32_t stride, std::string &err) {
    if (n == 0) return IFA_OK;
    // answer remembered bins, compute the rest on the device
    std::vector<uint32_t> mL, mS, mK, where;
    {
        std::lock_guard<std::mutex> lock(g_bin_mutex);
        for (uint32_t i = 0; i < n; i++) {
            auto it = g_bin_cache.find(BinKey{L[i], subs[i], k[i], step, mask_w, max_clips, num, den, trials, seed});
            if (it != g_bin_cache.end()) {
                out[i] = it->second;
            } else {
                mL.push_back(L[i]);
                mS.push_back(subs[i]);
                mK.push_back(k[i]);
                where.push_back(i);
            }
        }
    }
    if (mL.empty()) return IFA_OK;
    std::vector<uint32_t> mo(mL.size());
    ifa_status r = minhits_compute(mL.data(), mS.data(), mK.data(), static_cast<uint32_t>(mL.size()), step, mask_w,
                                   max_clips, num, den, trials, seed, mo.data(), st, stride, err);
    if (r != IFA_OK) return r;
    std::lock_guard<std::mutex> lock(g_bin_mutex);
    for (size_t j = 0; j < mL.size(); j++) {
        out[where[j]] = mo[j];
        g_bin_cache[BinKey{mL[j], mS[j], mK[j], step, mask_w, max_clips, num, den, trials, seed}] = mo[j];
    }
    return IFA_OK;
}

ifa_status minhits_compute(const uint32_t *L, const uint32_t *subs, const uint32_t *k, uint32_t n,
                           uint32_t step, uint32_t mask_w, uint32_t max_clips, uint32_t num, uint32_t den,
                           uint32_t trials, uint64_t seed, uint32_t *out, cudaStream_t st,
                           uint32_t stride, std::string &err) {
    if (n == 0) return IFA_OK;
    uint32_t *dL = nullptr, *dS = nullptr, *dK = nullptr, *dH = nullptr, *dO = nullptr;
    const size_t nb = static_cast<size_t>(n) * sizeof(uint32_t);
    cudaError_t e = cudaSuccess;
    auto ck = [&](cudaError_t r) {
        if (e == cudaSuccess && r != cudaSuccess) e = r;
    };
    ck(cudaMalloc(&dL, nb));
    ck(cudaMalloc(&dS, nb));
    ck(cudaMalloc(&dK, nb));
    ck(cudaMalloc(&dO, nb));
    ck(cudaMalloc(&dH, static_cast<size_t>(n) * stride * sizeof(uint32_t)));
    if (e == cudaSuccess) {
        ck(cudaMemcpyAsync(dL, L, nb, cudaMemcpyHostToDevice, st));
        ck(cudaMemcpyAsync(dS, subs, nb, cudaMemcpyHostToDevice, st));
        ck(cudaMemcpyAsync(dK, k, nb, cudaMemcpyHostToDevice, st));
        ck(launch_minhits(dL, dS, dK, n, step, mask_w, max_clips, num, den, trials, seed, dH, stride, dO, st));
        ck(cudaMemcpyAsync(out, dO, nb, cudaMemcpyDeviceToHost, st));
        ck(cudaStreamSynchronize(st));
    }
    cudaFree(dL);
    cudaFree(dS);
    cudaFree(dK);
    cudaFree(dH);
    cudaFree(dO);
    if (e != cudaSuccess) {
        err = std::string("MinHits on the device: ") + cudaGetErrorString(e);
        return cuda_status(e);
    }
    return IFA_OK;
}

ifa_status indexed_plan_q(IndexedState &S, const std::vector<std::string> &qs,
                          const std::vector<uint32_t> &svec, const std::vector<uint8_t> &include,
                          const ifa_config &cfg, cudaStream_t st, std::string &err) {
    const uint32_t nq = static_cast<uint32_t>(qs.size());
    // MinHits bins: distinct (L, s) of the included queries x listed k
    std::vector<std::pair<uint32_t, uint32_t>> ls;
    for (uint32_t q = 0; q < nq; q++)
        if (include[q]) ls.push_back({static_cast<uint32_t>(qs[q].size()), svec[q]});
    std::sort(ls.begin(), ls.end());
    ls.erase(std::unique(ls.begin(), ls.end()), ls.end());
    std::vector<uint32_t> bL, bS, bK;
    uint32_t stride = 2;
    for (const auto &p : ls)
        for (uint32_t i = 0; i < cfg.n_k; i++) {
            const uint32_t k = cfg.k_list[i];
            if (k > p.first || k <= cfg.mask_width) continue;
            bL.push_back(p.first);
            bS.push_back(p.second);
            bK.push_back(k);
            stride = std::max(stride, (p.first - k) / cfg.kmer_step + 2);
        }
    std::vector<uint32_t> bm(bL.size());
    ifa_status r = minhits_device(bL.data(), bS.data(), bK.data(), static_cast<uint32_t>(bL.size()),
                                  cfg.kmer_step, cfg.mask_width, 0u /* clipped windows are scanned exhaustively */, cfg.minhits_num,
                                  cfg.minhits_den, cfg.minhits_trials, cfg.minhits_seed, bm.data(), st,
                                  stride, err);
    if (r != IFA_OK) return r;
    // per (L, s): the longest k with threshold >= 1, else the smallest k clamped to 1
    std::map<std::pair<uint32_t, uint32_t>, std::pair<int, std::pair<uint32_t, uint32_t>>> choice;
    for (const auto &p : ls) choice[p] = {-1, {0, 0}};
    for (size_t i = 0; i < bL.size(); i++) {
        auto &c = choice[{bL[i], bS[i]}];
        if (bm[i] >= 1 && (c.first != 1 || bK[i] > c.second.first)) c = {1, {bK[i], bm[i]}};
    }
    for (size_t i = 0; i < bL.size(); i++) {
        auto &c = choice[{bL[i], bS[i]}];
        if (c.first == 1) continue;
        if (c.first == -1 || bK[i] < c.second.first) c = {0, {bK[i], 1u}};
    }
    S.plan_k.assign(nq, 0);
    S.plan_minhits.assign(nq, 0);
    S.plan_exhaustive.assign(nq, 0);
    S.plan_in = include;
    for (uint32_t q = 0; q < nq; q++) {
        if (!include[q]) continue;
        const auto &c = choice[{static_cast<uint32_t>(qs[q].size()), svec[q]}];
        S.plan_k[q] = c.second.first;
        S.plan_minhits[q] = c.second.second;
        const bool ex = c.first < 0 || (c.first == 0 && cfg.exhaustive_fallback) || has_n(qs[q]);
        S.plan_exhaustive[q] = ex ? 1 : 0;
    }
    S.plan_valid = true;
    S.tables_valid = false;
    return IFA_OK;
}

ifa_status indexed_plan(IndexedState &S, const std::vector<std::string> &qs, const ifa_config &cfg,
                        uint32_t s, cudaStream_t st, std::string &err) {
    if (S.plan_valid && S.plan_s == s && S.plan_uniform) return IFA_OK;
    ifa_status r = indexed_plan_q(S, qs, std::vector<uint32_t>(qs.size(), s),
                                  std::vector<uint8_t>(qs.size(), 1), cfg, st, err);
    if (r != IFA_OK) return r;
    S.plan_s = s;
    S.plan_uniform = true;
    return IFA_OK;
}

ifa_status indexed_tables(IndexedState &S, const std::vector<std::string> &qs,
                          const std::vector<uint32_t> &qmeta, const std::vector<uint4> &qwords,
                          uint32_t wmax, const ifa_config &cfg, cudaStream_t st, std::string &err) {
    std::vector<uint32_t> qlen(qs.size());
    for (size_t q = 0; q < qs.size(); q++) qlen[q] = static_cast<uint32_t>(qs[q].size());
    return indexed_tables_len(S, qlen, qmeta, qwords, wmax, cfg, st, err);
}

ifa_status indexed_tables_len(IndexedState &S, const std::vector<uint32_t> &qlen,
                              const std::vector<uint32_t> &qmeta, const std::vector<uint4> &qwords,
                              uint32_t wmax, const ifa_config &cfg, cudaStream_t st, std::string &err) {
    enum : size_t { kWords, kEmh, kEnts, kFirst, kKeys, kPv, kSums, kExWords, kExMeta, kExIds, kMeta, kTab0 };
    S.free_tables();
    S.wmax = wmax;
    S.step = cfg.kmer_step;
    cudaError_t e = cudaSuccess;
    auto ck = [&](cudaError_t x) {
        if (e == cudaSuccess && x != cudaSuccess) e = x;
    };
    // host -> device on st; pageable sources are staged by the driver before
    // the call returns, so the host vectors may go right after
    auto put = [&](void *d, const void *h, size_t bytes) {
        if (e == cudaSuccess && bytes) ck(cudaMemcpyAsync(d, h, bytes, cudaMemcpyHostToDevice, st));
    };
    const uint32_t nq = static_cast<uint32_t>(qlen.size());
    if (!S.d_candidates) {
        ck(cudaMalloc(&S.d_candidates, sizeof(unsigned long long)));
        ck(cudaMemsetAsync(S.d_candidates, 0, sizeof(unsigned long long), st));
    }
    // per-entry thresholds
    std::vector<uint32_t> emh(2 * static_cast<size_t>(nq));
    for (uint32_t q = 0; q < nq; q++) emh[2 * q] = emh[2 * q + 1] = S.plan_minhits[q];
    S.d_entry_minhits = static_cast<uint32_t *>(S.bufs.get(kEmh, emh.size() * sizeof(uint32_t), e));
    put(S.d_entry_minhits, emh.data(), emh.size() * sizeof(uint32_t));
    // tables per distinct k among seeded queries
    std::vector<uint32_t> ks;
    for (uint32_t q = 0; q < nq; q++)
        if (S.plan_in[q] && !S.plan_exhaustive[q]) ks.push_back(S.plan_k[q]);
    std::sort(ks.begin(), ks.end());
    ks.erase(std::unique(ks.begin(), ks.end()), ks.end());
    if (!ks.empty()) {
        const uint4 *d_words = static_cast<const uint4 *>(S.bufs.get(kWords, qwords.size() * sizeof(uint4), e));
        put(const_cast<uint4 *>(d_words), qwords.data(), qwords.size() * sizeof(uint4));
        uint32_t *d_meta = static_cast<uint32_t *>(S.bufs.get(kMeta, qmeta.size() * sizeof(uint32_t), e));
        put(d_meta, qmeta.data(), qmeta.size() * sizeof(uint32_t));
        S.targ.n = static_cast<uint32_t>(ks.size());
        for (size_t ti = 0; ti < ks.size() && e == cudaSuccess; ti++) {
            const uint32_t k = ks[ti];
            const uint32_t care = care_mask(k, cfg.mask_width);
            // entries of this table and their first posting
            std::vector<uint32_t> ents, first{0};
            for (uint32_t q = 0; q < nq; q++) {
                if (!S.plan_in[q] || S.plan_exhaustive[q] || S.plan_k[q] != k) continue;
                const uint32_t L = qlen[q];
                const uint32_t n_off = L >= k ? (L - k) / cfg.kmer_step + 1 : 0;
                for (uint32_t t = 0; t < 2; t++) {
                    ents.push_back(2 * q + t);
                    first.push_back(first.back() + n_off);
                }
            }
            const uint32_t np = first.back();
            const bool direct = k <= kDirectMaxK;
            const uint64_t nkeys = 1ull << (2 * k);
            const uint64_t noff = direct ? nkeys + 3 : static_cast<uint64_t>(np) + 3;
            const uint64_t nbw = direct ? 0 : nkeys / 32;
            uint32_t *d_ents = static_cast<uint32_t *>(S.bufs.get(kEnts, ents.size() * sizeof(uint32_t), e));
            uint32_t *d_first = static_cast<uint32_t *>(S.bufs.get(kFirst, first.size() * sizeof(uint32_t), e));
            uint32_t *d_keys = static_cast<uint32_t *>(S.bufs.get(kKeys, std::max<size_t>(np, 1) * sizeof(uint32_t), e));
            uint32_t *d_pv = static_cast<uint32_t *>(S.bufs.get(kPv, std::max<size_t>(np, 1) * sizeof(uint32_t), e));
            uint32_t *d_sums = static_cast<uint32_t *>(
                S.bufs.get(kSums, device_scan_sums_words(std::max(noff, nbw)) * sizeof(uint32_t), e));
            uint32_t *d_off = static_cast<uint32_t *>(S.bufs.get(kTab0 + 4 * ti, noff * sizeof(uint32_t), e));
            uint32_t *d_bits = direct ? nullptr
                                      : static_cast<uint32_t *>(S.bufs.get(kTab0 + 4 * ti + 1, nbw * sizeof(uint32_t), e));
            uint32_t *d_rank = direct ? nullptr
                                      : static_cast<uint32_t *>(S.bufs.get(kTab0 + 4 * ti + 2, nbw * sizeof(uint32_t), e));
            uint2 *d_post = static_cast<uint2 *>(S.bufs.get(kTab0 + 4 * ti + 3, std::max<size_t>(np, 1) * sizeof(uint2), e));
            put(d_ents, ents.data(), ents.size() * sizeof(uint32_t));
            put(d_first, first.data(), first.size() * sizeof(uint32_t));
            if (e == cudaSuccess)
                ck(launch_postings(d_words, wmax, d_ents, d_first, static_cast<uint32_t>(ents.size()), k, care,
                                   cfg.kmer_step, d_keys, d_pv, st));
            if (e == cudaSuccess)
                ck(build_table(k, direct, d_keys, d_pv, d_meta, np, d_off, d_bits, d_rank, d_post, d_sums, st));
            KTableDev &T = S.targ.t[ti];
            T.k = k;
            T.care = care;
            T.direct = direct ? 1u : 0u;
            T.pad = 0;
            T.off = d_off ? d_off + 2 : nullptr;
            T.rank = d_rank;
            T.bits = d_bits;
            T.post = d_post;
        }
    }
    // exhaustive queries: compact table for the brute-force kernel
    std::vector<uint32_t> exq;
    for (uint32_t q = 0; q < nq; q++)
        if (S.plan_in[q] && S.plan_exhaustive[q]) exq.push_back(q);
    S.any_exhaustive = !exq.empty();
    if (S.any_exhaustive && e == cudaSuccess) {
        const uint32_t ne = 2 * static_cast<uint32_t>(exq.size());
        std::vector<uint32_t> ids(ne), meta(ne);
        std::vector<uint4> words(static_cast<size_t>(ne) * wmax);
        S.ex_entries = ne;
        S.d_ex_words = static_cast<uint4 *>(S.bufs.get(kExWords, words.size() * sizeof(uint4), e));
        S.d_ex_meta = static_cast<uint32_t *>(S.bufs.get(kExMeta, ne * sizeof(uint32_t), e));
        S.d_ex_ids = static_cast<uint32_t *>(S.bufs.get(kExIds, ne * sizeof(uint32_t), e));
        for (uint32_t i = 0; i < ne; i++) {
            const uint32_t src = 2 * exq[i / 2] + (i & 1);
            ids[i] = src;
            meta[i] = qmeta[src];
            for (uint32_t w = 0; w < wmax; w++) words[static_cast<size_t>(i) * wmax + w] = qwords[static_cast<size_t>(src) * wmax + w];
        }
        put(S.d_ex_words, words.data(), words.size() * sizeof(uint4));
        put(S.d_ex_meta, meta.data(), ne * sizeof(uint32_t));
        put(S.d_ex_ids, ids.data(), ne * sizeof(uint32_t));
        uint32_t cap = scan_brute_chunk_entries(wmax) & ~1u;
        if (cap < 2) cap = 2;
        for (uint32_t e0 = 0; e0 < ne; e0 += cap) {
            IndexedState::ExChunk c{e0, std::min(ne, e0 + cap), 0xffffffffu, 0};
            for (uint32_t i = c.e0; i < c.e1; i++) {
                c.lmin = std::min(c.lmin, meta[i] & 0xffu);
                c.lmax = std::max(c.lmax, meta[i] & 0xffu);
            }
            S.ex_chunks.push_back(c);
        }
    }
    if (e != cudaSuccess) {
        err = std::string("indexed tables: ") + cudaGetErrorString(e);
        S.free_tables();
        return cuda_status(e);
    }
    S.tables_valid = true;
    return IFA_OK;
}

ifa_status indexed_prepare(IndexedState &S, const std::vector<std::string> &qs,
                           const std::vector<uint32_t> &qmeta, const std::vector<uint4> &qwords,
                           uint32_t wmax, const ifa_config &cfg, uint32_t s, cudaStream_t st,
                           std::string &err) {
    ifa_status r = indexed_plan(S, qs, cfg, s, st, err);
    if (r != IFA_OK) return r;
    if (S.tables_valid && S.tables_s == s && S.wmax == wmax) return IFA_OK;
    r = indexed_tables(S, qs, qmeta, qwords, wmax, cfg, st, err);
    if (r != IFA_OK) return r;
    S.tables_s = s;
    return IFA_OK;
}

ifa_status indexed_scan(IndexedState &S, const Batch &b, const QueryTable &qt, uint32_t s,
                        const HitSink &sink, cudaStream_t st, int *launches, std::string &err,
                        const EventSink *es) {
    cudaError_t e = cudaSuccess;
    if (S.targ.n) {
        e = launch_seed_scan(b, qt, S.targ, S.d_entry_minhits, S.step, s, sink, S.d_candidates, st);
        if (launches) (*launches)++;
    }
    if (e == cudaSuccess && S.any_exhaustive) {
        QueryTable ex;
        ex.words = S.d_ex_words;
        ex.meta = S.d_ex_meta;
        ex.ids = S.d_ex_ids;
        ex.n_entries = S.ex_entries;
        ex.wmax = qt.wmax;
        for (const auto &c : S.ex_chunks) {
            e = launch_scan_brute(b, ex, c.e0, c.e1, s, c.lmin, c.lmax, sink, st, launches, es);
            if (e != cudaSuccess) break;
        }
    }
    if (e != cudaSuccess) {
        err = std::string("indexed scan: ") + cudaGetErrorString(e);
        return IFA_ERR_CUDA;
    }
    return IFA_OK;
}

}  // namespace ifa

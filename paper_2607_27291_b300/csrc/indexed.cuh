// indexed.cuh -- indexed mode (Methods, indexed mode): per-query seed length
// and min-hits threshold from the MinHitsCalculator, query k-mer tables on
// the device, and the seed scan with verification.
#pragma once
#include <string>
#include <utility>
#include <vector>

#include "ifa_internal.cuh"

namespace ifa {

constexpr int kMaxTables = IFA_MAX_KLIST;
constexpr uint32_t kDirectMaxK = 12;   // k <= 12: direct-address offsets (4^k + 1 words)

// One seed length's query k-mer table.  Keys are "planar": the k hi-plane
// bits of the k-mer above its k lo-plane bits (masked positions zeroed), an
// injective code of the unmasked bases.  Postings are (entry << 8 | offset);
// the postings of a key are post[off[x] .. off[x + 1]) with x the key
// (direct) or the key's rank among the present keys (ranked).
struct KTableDev {
    uint32_t k;
    uint32_t care;         // k-bit mask of the positions that count
    uint32_t direct;       // 1: off[] indexed by key
    uint32_t pad;
    const uint32_t *off;   // direct: 4^k + 1 words; ranked: present keys + 1
    const uint32_t *rank;  // ranked: keys present before each bitmap word
    const uint32_t *bits;  // ranked: presence bitmap of 4^k bits
    const uint2 *post;     // postings grouped by key: {entry << 8 | offset, the entry's meta word}
};

struct KTablesArg {
    KTableDev t[kMaxTables];
    uint32_t n;
};

struct IndexedState {
    // plan (per query) for plan_s
    bool plan_valid = false;
    bool plan_uniform = false;   // plan made for one maxSubs (plan_s) over all queries
    uint32_t plan_s = 0;
    std::vector<uint32_t> plan_k, plan_minhits;
    std::vector<uint8_t> plan_exhaustive;
    std::vector<uint8_t> plan_in;  // query is part of this plan

    // device tables for tables_s, in grow-only buffers kept across rebuilds
    // (slot -> (pointer, bytes)); released by release()
    bool tables_valid = false;
    uint32_t tables_s = 0;
    KTablesArg targ{};
    DevBufs bufs;
    uint32_t *d_entry_minhits = nullptr;
    unsigned long long *d_candidates = nullptr;
    uint32_t wmax = 1;
    uint32_t step = 1;

    // exhaustive queries: compacted table scanned by the brute kernel
    bool any_exhaustive = false;
    uint4 *d_ex_words = nullptr;
    uint32_t *d_ex_meta = nullptr;
    uint32_t *d_ex_ids = nullptr;
    uint32_t ex_entries = 0;
    struct ExChunk { uint32_t e0, e1, lmin, lmax; };
    std::vector<ExChunk> ex_chunks;

    void invalidate() {
        plan_valid = false;
        plan_uniform = false;
        tables_valid = false;
    }
    void free_tables();
    void release();
    uint64_t candidates_host(cudaStream_t st) const;
};

// MinHits thresholds on the device (remembered per bin for the process).
ifa_status minhits_compute(const uint32_t *L, const uint32_t *subs, const uint32_t *k, uint32_t n,
                           uint32_t step, uint32_t mask_w, uint32_t max_clips, uint32_t num,
                           uint32_t den, uint32_t trials, uint64_t seed, uint32_t *out,
                           cudaStream_t st, uint32_t hist_stride, std::string &err);
ifa_status minhits_device(const uint32_t *L, const uint32_t *subs, const uint32_t *k, uint32_t n,
                          uint32_t step, uint32_t mask_w, uint32_t max_clips, uint32_t num,
                          uint32_t den, uint32_t trials, uint64_t seed, uint32_t *out,
                          cudaStream_t st, uint32_t hist_stride, std::string &err);

ifa_status indexed_plan(IndexedState &S, const std::vector<std::string> &qs, const ifa_config &cfg,
                        uint32_t max_subs, cudaStream_t st, std::string &err);

// Plan for the included queries, each with its own maxSubs.
ifa_status indexed_plan_q(IndexedState &S, const std::vector<std::string> &qs,
                          const std::vector<uint32_t> &svec, const std::vector<uint8_t> &include,
                          const ifa_config &cfg, cudaStream_t st, std::string &err);

// Device tables of the current plan (seeded queries) and the compact table of
// its exhaustive queries, built on stream st (ordered before later work on
// st; the host does not wait).
ifa_status indexed_tables(IndexedState &S, const std::vector<std::string> &qs,
                          const std::vector<uint32_t> &qmeta, const std::vector<uint4> &qwords,
                          uint32_t wmax, const ifa_config &cfg, cudaStream_t st, std::string &err);

// The same from query lengths alone (the only property of the queries the
// tables need besides their encoded words).
ifa_status indexed_tables_len(IndexedState &S, const std::vector<uint32_t> &qlen,
                              const std::vector<uint32_t> &qmeta, const std::vector<uint4> &qwords,
                              uint32_t wmax, const ifa_config &cfg, cudaStream_t st, std::string &err);

// Device table construction (ktables.cu).
uint64_t device_scan_sums_words(uint64_t n);
cudaError_t device_scan(const uint32_t *in, uint32_t *out, uint64_t n, bool popc, bool exclusive,
                        uint32_t *sums, cudaStream_t st);
cudaError_t launch_postings(const uint4 *words, uint32_t wmax, const uint32_t *ents, const uint32_t *first,
                            uint32_t nents, uint32_t k, uint32_t care, uint32_t step, uint32_t *keys,
                            uint32_t *pv, cudaStream_t st);
cudaError_t build_table(uint32_t k, bool direct, uint32_t *keys, const uint32_t *pv, const uint32_t *meta, uint32_t np,
                        uint32_t *off, uint32_t *bits, uint32_t *rank, uint2 *post, uint32_t *sums, cudaStream_t st);

ifa_status indexed_prepare(IndexedState &S, const std::vector<std::string> &qs,
                           const std::vector<uint32_t> &qmeta, const std::vector<uint4> &qwords,
                           uint32_t wmax, const ifa_config &cfg, uint32_t max_subs, cudaStream_t st,
                           std::string &err);

// The seed scan, then the exhaustive entries by brute force (their hits
// deferred through es when given).
ifa_status indexed_scan(IndexedState &S, const Batch &b, const QueryTable &qt, uint32_t max_subs,
                        const HitSink &sink, cudaStream_t st, int *launches, std::string &err,
                        const EventSink *es = nullptr);

cudaError_t launch_seed_scan(const Batch &b, const QueryTable &qt, const KTablesArg &tabs,
                             const uint32_t *entry_minhits, uint32_t step, uint32_t max_subs,
                             const HitSink &sink, unsigned long long *candidates, cudaStream_t st);

}  // namespace ifa

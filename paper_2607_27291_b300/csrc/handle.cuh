// handle.cuh -- the ifa_handle state shared by the C ABI files.
#pragma once
#include <string>
#include <utility>
#include <vector>

#include "batch_state.cuh"
#include "ifa_internal.cuh"
#include "indexed.cuh"
#include "status.cuh"

namespace ifa {
struct Chunk {
    uint32_t e0, e1, lmin, lmax;
};

}  // namespace ifa

using ifa::Chunk;
using ifa::DevPiece;
using ifa::IndexedState;
using ifa::BatchState;

struct ifa_handle {
    ifa_config cfg{};
    int dev = 0;
    cudaStream_t own_stream = nullptr;
    cudaStream_t stream = nullptr;
    cudaStream_t copy_stream = nullptr;
    std::string err = "no error";

    // queries
    std::vector<std::string> qs;
    uint32_t lmin = 0, lmax = 0, wmax = 1;
    bool qdirty = true;
    uint4 *d_qwords = nullptr;
    uint32_t *d_qmeta = nullptr;
    // tensor-core operand of the entries (queries up to 64 bases), its row
    // width in bases, and the kernel's status words (bit 0 of the first: a
    // wait gave up; the second: the launch's work counter)
    uint8_t *d_tcA = nullptr;
    uint32_t tc_lpad = 0;
    unsigned int *d_tc_status = nullptr;
    bool tc_used = false;
    std::vector<Chunk> chunks;
    std::vector<uint32_t> qmeta_host;
    std::vector<uint4> qwords_host;

    // segment slots
    uint8_t *d_seg[2] = {nullptr, nullptr};
    uint8_t *h_stage[2] = {nullptr, nullptr};
    DevPiece *d_pieces[2] = {nullptr, nullptr};
    DevPiece *h_pieces[2] = {nullptr, nullptr};
    uint32_t pieces_cap[2] = {0, 0};
    cudaEvent_t ev_copied[2] = {nullptr, nullptr};
    cudaEvent_t ev_consumed[2] = {nullptr, nullptr};
    bool slot_used[2] = {false, false};
    int slot = 0;

    uint8_t *d_halo[2] = {nullptr, nullptr};
    int halo_cur = 0;
    uint32_t halo_len = 0;

    ifa::RefBufs ref;  // the packed batch (2-bit words, directory, exceptions)

    // results: the device hit ring and its counters d_head = {head (claims),
    // first dropped claim (~0 when none), tail (drained, written by the host)}
    ifa_hit *d_ring = nullptr;
    unsigned long long *d_head = nullptr;
    uint32_t *d_overflow = nullptr;
    unsigned long long *d_digest = nullptr;
    unsigned long long *d_qcount = nullptr;
    ifa::EventSink ev{nullptr, nullptr, 0};  // deferred hits of the brute-force scan
    uint64_t tail = 0;                       // hits drained from the ring
    // per pushed segment, a pinned copy of {head, first dropped claim} taken
    // on the compute stream after its scan, and an event: once the event has
    // completed, every claim below that head is written
    static constexpr int kMarks = 8;
    unsigned long long *h_marks = nullptr;   // pinned: kMarks x 2, then the tail word for uploads
    cudaEvent_t ev_mark[kMarks] = {};
    std::vector<int> marks_pending;          // oldest first
    int mark_next = 0;
    uint64_t done_head = 0, done_ovf = ~0ull;  // from the latest completed mark
    cudaStream_t drain_stream = nullptr;     // ring-to-host copies and tail uploads

    // stream position
    bool open = false;
    uint32_t open_contig = 0;
    uint64_t open_next = 0;
    bool any_contig = false;
    uint32_t last_contig = 0;
    bool pushed = false;

    uint32_t max_subs = 0;
    bool per_query_s = false;   // qs_s holds each query's own maxSubs (ifa_set_query_max_subs)
    ifa_mode mode = IFA_MODE_BRUTE;
    // IFA_MODE_AUTO by measured rates: rates on the calibration sequence
    // (per maxSubs, auto_s) and the mode they gave for the loaded queries
    ifa::Rates auto_rates;
    uint32_t auto_s = 0xffffffffu;
    ifa_mode auto_mode = IFA_MODE_AUTO;
    ifa_mode mode_run = IFA_MODE_AUTO;   // the mode the current pass runs in
    ifa_stats stats{};

    // optional per-launch timing of the scan kernels (config.profile)
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_pending, ev_free;

    IndexedState idx;

    // per-query maxSubs of queries added by ifa_set_add (0 for ifa_load_queries)
    std::vector<uint32_t> qs_s;
    BatchState batch;
    ifa::ServeState serve;
};


namespace ifa {
// Encode the handle's queries into the device query table (no-op when clean).
ifa_status upload_queries(ifa_handle *h);
// Free the multi-set store and plan.
void batch_release(ifa_handle *h);
// The persistent multi-set kernels (batch.cu), for the serving loop: the
// brute-force items, then the seed items, each kind in its own persistent
// launch (w.queue: two counters, zeroed by the caller).  *launches gets
// the kernels launched.
cudaError_t launch_batch_kernels(uint32_t wmax, const Batch &b, const BatchWork &w, const QueryTable &bt,
                                 const QueryTable &ft, const HitSink &sink, cudaStream_t st, int *launches);
int batch_kernel_grid(uint32_t wmax);
void encode_entry(const std::string &q, bool rc, uint32_t wmax, uint32_t s_e, uint4 *out, uint32_t *meta);
void tc_operand(const std::vector<std::string> &qs, uint32_t lpad, std::vector<uint8_t> &out);
// Mean over queries [first, first + n) of the probability that a random
// window (uniform bases) hits at maxSubs s; and whether the tensor-core
// kernel should scan such a brute-force query set (the automatic rule).
double mean_window_hit_rate(const std::vector<std::string> &qs, uint32_t first, uint32_t n, uint32_t s);
bool tc_auto_choice(const std::vector<std::string> &qs, uint32_t first, uint32_t n, uint32_t s);

// The measured-rate choice of IFA_MODE_AUTO (autotune.cu).
// Expected random seed hits per reference base of one entry of length L.
double seed_hits_per_base(uint32_t L, uint32_t k, uint32_t step);
// Cost of queries [first, first + n) of qs under rates r and seed plan
// `plan` (indexed by query; plan_exhaustive empty = no plan).
ModeCost predict_cost(const Rates &r, const std::vector<std::string> &qs, uint32_t first, uint32_t n,
                      const IndexedState &plan, uint32_t step);
// Measure the rates on batch b with (up to 128 of) the queries qs at
// maxSubs svec; count-only sinks, so no result of the handle changes.
ifa_status measure_rates(ifa_handle *h, const Batch &b, const std::vector<std::string> &qs,
                         const std::vector<uint32_t> &svec, Rates &out);
// The mode with the smaller predicted time for qs at maxSubs svec.
ifa_status choose_mode(ifa_handle *h, const Rates &r, const std::vector<std::string> &qs,
                       const std::vector<uint32_t> &svec, ifa_mode *mode);
// Rates measured on 16 Mbp of uniform random bases packed on the device
// (the streaming calls, and stores smaller than that), or on a slice of
// the store.
ifa_status rates_on_random(ifa_handle *h, const std::vector<std::string> &qs, const std::vector<uint32_t> &svec,
                           Rates &out);
ifa_status rates_on_store(ifa_handle *h, const Batch &store, const std::vector<std::string> &qs,
                          const std::vector<uint32_t> &svec, Rates &out);
// Free the serving state.
void serve_release(ifa_handle *h);
}  // namespace ifa

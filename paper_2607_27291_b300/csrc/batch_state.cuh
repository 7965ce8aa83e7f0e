// batch_state.cuh -- state of the multi-set scan (device-resident reference
// store, query sets, merged plan, persistent-launch graph).
#pragma once
#include <cstdint>
#include <memory>
#include <string>
#include <vector>

#include "ifa_internal.cuh"
#include "indexed.cuh"

namespace ifa {

// Measured rates of the two modes' work (autotune.cu).
struct Rates {
    double brute = 0;   // brute-force entry x base evaluations per second
    double pos = 0;     // seed scan: reference positions x tables per second
    double cand = 0;    // verified candidates per second
    bool valid() const { return brute > 0; }
};

// Predicted seconds per reference base of a query set in each mode.
struct ModeCost {
    double brute_s = 0, idx_s = 0;
    bool seeded = false;   // some query has a seed plan (else indexed = brute force)
};

struct QuerySet {
    uint32_t first = 0, n = 0;      // global query ids [first, first + n)
    uint32_t s = 0;                 // maxSubs (capped at 255)
    ifa_mode mode = IFA_MODE_AUTO;  // as requested
    ifa_mode chosen = IFA_MODE_BRUTE;
};

// Device work descriptor of one persistent multi-set launch.
struct BatchWork {
    // brute-force part: compact entry table and its chunks
    const uint4 *bwords;
    const uint32_t *bmeta;
    const uint32_t *bids;
    const uint32_t *chunk_e0, *chunk_e1, *chunk_lmin, *chunk_lmax;
    uint32_t nchunks;
    // indexed part: merged k-mer tables over the full query table
    KTablesArg tabs;
    const uint32_t *emh;
    uint32_t step;
    const uint4 *qwords;
    const uint32_t *qmeta;
    // tiles over block ranges [b_block0, b_block_end) and [s_block0, s_block_end)
    uint64_t b_block0, b_block_end;  // blocks of 128 windows
    uint64_t s_block0, s_block_end;  // blocks of 32 positions
    uint64_t tile_bblocks;   // brute tile, in blocks of 128 windows
    uint64_t tile_sblocks;   // seed tile, in blocks of 32 positions
    uint32_t n_btiles, n_stiles;
    uint32_t n_brute_items, n_items;
    unsigned int *queue;
    unsigned long long *candidates;
};

struct BatchState {
    // reference store
    RefBufs ref;               // the store: 2-bit words, directory, exceptions (nb: one chunk's scratch)
    uint64_t exc_used = 0;     // exception entries in use
    uint64_t nbases = 0;
    std::vector<DevPiece> pieces;
    DevPiece *d_pieces = nullptr;
    uint32_t d_pieces_n = 0;
    bool pieces_dirty = true;
    bool open = false;
    uint32_t open_contig = 0;
    uint64_t open_next = 0;
    bool any_contig = false;
    uint32_t last_contig = 0;

    // query sets
    std::vector<QuerySet> sets;

    // merged plan (valid until sets change)
    bool plan_valid = false;
    uint32_t wmax = 1;
    std::vector<void *> allocs;           // plan buffers
    uint32_t b_entries = 0;
    std::vector<uint32_t> bchunk_e0, bchunk_e1, bchunk_lmin, bchunk_lmax;
    std::vector<uint32_t> set_bchunk_lo, set_bchunk_hi;  // per set: its brute chunks
    // brute-force sets on the tensor cores: one one-hot operand of every such
    // set's entries, each set padded to whole 128-row tiles (rows of length
    // 0), with the rows' metas and entry ids
    uint32_t tc_rows = 0, tc_lpad = 0;
    std::vector<uint32_t> set_tc_row0, set_tc_rows;    // per set: its rows (0 rows: popcount kernel)
    uint8_t *d_tcA = nullptr;
    uint32_t *d_tcmeta = nullptr, *d_tcids = nullptr;
    unsigned int *d_tcstatus = nullptr;                // [0] a wait gave up, [1] work counter
    IndexedState merged;                  // all indexed sets together
    std::vector<std::unique_ptr<IndexedState>> per_set;  // each indexed set alone (per-set runs)
    BatchWork work{};
    unsigned int *d_queue = nullptr;
    unsigned long long *d_cand = nullptr;
    int grid = 0;

    // persistent launch captured as a CUDA graph
    cudaGraphExec_t graph = nullptr;
    cudaStream_t graph_stream = nullptr;

    // autotuner measurements (per handle)
    Rates rates;
};

}  // namespace ifa

namespace ifa {

// One served request (a query set) and its device hit ring.
struct Request {
    std::vector<std::string> qs;
    uint32_t s = 0;
    ifa_mode mode = IFA_MODE_BRUTE;  // as run (AUTO resolved at submission)
    int state = 0;                   // 0 queued, 1 active, 2 done, 3 drained
    double t_submit = 0, t_admit = 0, t_done = 0;  // seconds since ifa_serve_start
    uint32_t slices_done = 0;
    ifa_hit *d_ring = nullptr;
    unsigned long long *d_counters = nullptr;  // head, overflow, count, sum, xor
    uint64_t cap = 0;
    uint64_t bytes = 0;                        // charged to the budget
    unsigned long long final_counters[5] = {0, 0, 0, 0, 0};
    // computed once when admitted: entries encoded with w words each, and
    // for indexed requests each query's seed length, threshold and whether
    // it is scanned exhaustively
    bool prepared = false;
    uint32_t w = 1;
    std::vector<uint4> words;
    std::vector<uint32_t> meta;
    std::vector<uint32_t> plan_k, plan_minhits;
    std::vector<uint8_t> plan_exhaustive;
};

// Continuous-batching serving over the reference store.
struct ServeState {
    bool on = false;
    uint32_t n_slices = 1;
    uint64_t budget = 0, used = 0;
    uint64_t ring_cap = 0;
    double t0 = 0;
    std::vector<Request> reqs;
    std::vector<uint32_t> pending;   // FIFO of request ids
    std::vector<uint32_t> active;    // request ids being scanned
    uint32_t slice = 0;
    bool dirty = true;
    // plan of the active set
    DevBufs pool;
    uint32_t wmax = 1;
    uint32_t nq = 0;
    uint32_t lmax = 0;               // longest active query (soft-clip count bound)
    uint32_t clip_pct = 0;           // soft clipping, fixed at ifa_serve_start
    QueryTable ft{};
    QueryTable bt{};
    uint32_t b_entries = 0;
    std::vector<uint32_t> chunk_e0;
    IndexedState merged;
    BatchWork work{};
    HitSink sink{};
    int grid = 0;
    unsigned int *d_queue = nullptr;
    unsigned long long *d_cand = nullptr;
    uint64_t slices_run = 0;
    double scanned_query_bases = 0;   // nominal comparisons done by completed slices
    double plan_s = 0, scan_s = 0;    // host time building plans, time waiting for slices
    Rates rates;                      // measured on the store at the first automatic request
};

}  // namespace ifa

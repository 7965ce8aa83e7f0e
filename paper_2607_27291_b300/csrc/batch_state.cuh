// batch_state.cuh -- state of the multi-set scan (device-resident reference
// store, query sets, merged plan, persistent-launch graph).
#pragma once
#include <cstdint>
#include <memory>
#include <vector>

#include "ifa_internal.cuh"
#include "indexed.cuh"

namespace ifa {

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
    // tiles
    uint64_t tile_bblocks;   // brute tile, in blocks of 128 windows
    uint64_t tile_sblocks;   // seed tile, in blocks of 32 positions
    uint32_t n_btiles, n_stiles;
    uint32_t n_brute_items, n_items;
    unsigned int *queue;
    unsigned long long *candidates;
};

struct BatchState {
    // reference store
    uint4 *d_words = nullptr;
    uint64_t words_cap = 0;
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
    double brute_entry_bases_per_s = 0;  // entry x base evaluations per second
    double seed_pos_per_s = 0;           // positions x tables per second
    double cand_per_s = 0;               // verified candidates per second
};

}  // namespace ifa

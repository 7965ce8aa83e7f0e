/*
 * ifa.h -- C ABI of the B300 indel-free (Hamming) aligner.
 *
 * The calls follow the paper's statement of the problem (IndelFreeAligner,
 * Methods, "Algorithm Design" and "Memory Management"): the query set is
 * loaded once, a maxSubs threshold with no upper limit is set, the mode is
 * chosen explicitly or automatically, the reference is streamed past the
 * queries segment by segment and never indexed, and hits come out as the
 * stream goes (Methods, "Output Format").
 *
 * Conventions shared by every call:
 *  - Every call returns an ifa_status; none aborts the process.  On failure
 *    ifa_last_error() describes the cause.
 *  - A handle is used by one host thread at a time.
 *  - Pointers are host pointers unless a parameter says otherwise.  The
 *    library copies what it needs before returning unless stated otherwise;
 *    the caller keeps ownership of every buffer it passes.
 *  - Sequences are ASCII.  A, C, G, T in either case are bases; every other
 *    byte is N, and N mismatches everything on either side (a reading: the
 *    paper only says reference Ns are tracked apart from substitutions,
 *    Methods, "Algorithm Design").
 *  - Positions are 0-based.  Strand 0 is '+', strand 1 is '-'; a '-' hit at
 *    pos means the reverse complement of the query lies at
 *    ref[pos .. pos+L-1] with `mismatches` substitutions.  A window stays
 *    inside its contig unless soft clipping is on (ifa_config.clip_pct);
 *    without it a contig shorter than a query gives that query no hit.
 *  - Query ids are dense in load order.  Contig ids are the caller's; each
 *    new contig's id must be larger than the previous one's.
 *  - Device work runs on the handle's compute stream (ifa_set_stream) and
 *    a private copy stream; results are complete after ifa_flush().
 */
#ifndef IFA_H
#define IFA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define IFA_ABI_VERSION 1
#define IFA_MAX_QUERY_LEN 255u   /* longest query, in bases */
#define IFA_MAX_KLIST 8u

typedef struct ifa_handle ifa_handle;

typedef enum {
    IFA_OK = 0,
    IFA_ERR_INVALID_ARG = 1,   /* bad pointer, size, id order or piece table */
    IFA_ERR_OOM = 2,           /* a host or device allocation failed */
    IFA_ERR_CUDA = 3,          /* a CUDA call failed (no device, launch error) */
    IFA_ERR_BAD_STATE = 4,     /* call not allowed now (e.g. queries after segments) */
    IFA_ERR_HIT_OVERFLOW = 5,  /* the device hit buffer filled; see ifa_drain_hits */
    IFA_ERR_TIMEOUT = 6        /* a bounded device wait gave up */
} ifa_status;

typedef enum {
    IFA_MODE_AUTO = 0,     /* the mode with the smaller predicted time (see ifa_config.auto_crossover) */
    IFA_MODE_BRUTE = 1,    /* every window of every contig, both strands */
    IFA_MODE_INDEXED = 2   /* query k-mer seeds + min-hits threshold + verification */
} ifa_mode;

typedef enum {
    IFA_BRUTE_AUTO = 0,    /* tensor cores from 32 queries on when eligible (queries of at most 64 bases) and
                              hits are sparse: the set's mean probability that a random window hits, over
                              its queries (uniform bases, Binomial(L, 3/4) <= maxSubs; with per-query
                              values, the largest), is at most 2e-4 */
    IFA_BRUTE_POPC = 1,    /* bit-plane XOR/OR/popcount kernel */
    IFA_BRUTE_TENSOR = 2   /* one-hot GEMM on the tensor cores; queries of at most 64 bases */
} ifa_brute_kernel;

typedef enum {
    IFA_MEM_HOST = 0,               /* pageable host memory: copied through pinned staging */
    IFA_MEM_HOST_PINNED = 1,        /* page-locked host memory: DMA'd directly */
    IFA_MEM_DEVICE = 2,             /* device memory on the handle's device */
    IFA_MEM_HOST_PINNED_ASYNC = 3   /* page-locked host memory, DMA'd directly; ifa_push_segment and
                                       ifa_prime_halo return once the copy is enqueued, so the next
                                       segment's copy follows with no host round trip: the buffer must
                                       stay unchanged until ifa_flush (or a drain) returns.  Store
                                       appends treat it as IFA_MEM_HOST_PINNED. */
} ifa_mem;

/* One reported alignment (16 bytes). */
typedef struct {
    uint32_t query;       /* query id */
    uint32_t contig;      /* caller's contig id */
    uint32_t pos;         /* leftmost forward coordinate in the contig */
    uint8_t strand;       /* 0 '+', 1 '-' */
    uint8_t mismatches;   /* Hamming distance of the window */
    uint16_t clips;       /* soft clips at a contig end: left | right << 8 (0 inside a contig);
                             pos is then the first aligned base */
} ifa_hit;

/* Order-independent digest of every hit produced so far: the count, and
 * the sum (mod 2^64) and xor of mix(a ^ mix(b)) over hits, where
 * a = query << 32 | contig, b = pos << 32 | clips << 16 | strand << 8 |
 * mismatches and
 * mix is the splitmix64 output function.  Kept apart from the hit buffer,
 * so it stays exact when that buffer overflows or is disabled. */
typedef struct {
    uint64_t count;
    uint64_t sum;
    uint64_t xr;
} ifa_digest;

/* One contig piece inside a pushed segment.  Pieces of one segment are
 * given in order, are contiguous and cover the segment exactly
 * (start_0 = 0, start_{i+1} = start_i + len_i, sum len = segment length).
 * A piece whose `last` is 0 continues in the next segment; the next
 * segment's first piece then carries the same contig id with
 * offset_in_contig advanced by len.  Only a segment's last piece may have
 * last = 0. */
typedef struct {
    uint32_t contig;
    uint32_t last;
    uint64_t offset_in_contig;
    uint64_t start;
    uint64_t len;
} ifa_piece;

typedef struct {
    int32_t device;                /* CUDA device ordinal */
    uint32_t count_only;           /* 1: keep digest/counts only, write no hit tuples */
    uint64_t hit_capacity;         /* device hit ring entries (16 bytes each) */
    uint64_t segment_bytes;        /* largest segment accepted by ifa_push_segment */
    /* indexed mode (Methods, indexed mode) */
    uint32_t k_list[IFA_MAX_KLIST];/* candidate seed lengths, paper default 8,9,10,12,14 */
    uint32_t n_k;
    uint32_t kmer_step;            /* query k-mer offset step (reading: 1) */
    uint32_t mask_width;           /* masked middle bases of each k-mer (reading: 0) */
    uint32_t minhits_num;          /* detection probability num/den, paper default 99.9% */
    uint32_t minhits_den;
    uint32_t minhits_trials;       /* Monte Carlo trials, paper default 200,000 */
    uint64_t minhits_seed;         /* Philox key of the Monte Carlo */
    uint32_t clip_pct;             /* soft clipping at contig ends (Methods, Algorithm Design): a window may
                                      overhang its contig by up to floor(clip_pct * L / 100) bases, which
                                      count as clips, not mismatches; 0 = off, at most 50 (paper: 25);
                                      streaming, batched and serving calls (serving takes the value
                                      current at ifa_serve_start) */
    uint32_t exhaustive_fallback;  /* 1: queries with no qualifying k are scanned exhaustively */
    uint32_t auto_crossover;       /* IFA_MODE_AUTO in the streaming and serving calls: 0 (default) picks
                                      the mode with the smaller predicted time from rates measured on the
                                      device (once per handle and maxSubs on 16 Mbp of random sequence when
                                      streaming; once per session on the store when serving); n > 0 picks
                                      indexed from n queries on (the paper's rule; its crossover lies
                                      between 100 and 200).  Batches always use measured rates. */
    uint32_t profile;              /* 1: time every scan kernel with CUDA events (ifa_stats.scan_ns) */
    uint32_t brute_kernel;         /* brute-force kernel: 0 automatic, 1 popcount, 2 tensor cores
                                      (one-hot e4m3 GEMM; queries of at most 64 bases) */
    uint32_t test_stall;           /* testing only (keep 0): 1 makes each tensor-core CTA withhold its
                                      first tile, so a pipeline wait runs out after its 4 s limit and
                                      ifa_flush reports TIMEOUT -- the bounded-wait path, without a fault */
    uint32_t event_capacity;       /* streaming brute force defers hit expansion: the scan writes one
                                      16-byte record per (query strand, 32-window group) with a hit into a
                                      device buffer of this many records (0: max(2^20, segment_bytes / 32)),
                                      and a second kernel turns them into hits; a launch whose records do
                                      not fit is scanned again with the hits expanded in line (same
                                      results, slower) */
    uint32_t reserved[3];
} ifa_config;

typedef struct {
    uint64_t segments;        /* segments pushed */
    uint64_t bases;           /* reference bases pushed (one strand) */
    uint64_t h2d_bytes;       /* bytes copied host -> device for segments */
    uint64_t windows;         /* (query, strand, window) evaluations, nominal */
    uint64_t query_bases;     /* query-base comparisons, nominal */
    uint64_t kernel_launches; /* device kernels launched */
    uint64_t candidates;      /* indexed mode: candidate windows verified */
    uint64_t scan_launches;   /* scan kernels timed (config.profile = 1) */
    uint64_t scan_ns;         /* their summed device time, from CUDA events on the compute stream */
    uint32_t mode;            /* the streaming pass's mode: IFA_MODE_BRUTE or IFA_MODE_INDEXED
                                 (IFA_MODE_AUTO before the first segment) */
    uint32_t reserved;
} ifa_stats;

/* Fill *cfg with the defaults (paper defaults where it gives one).
 * INVALID_ARG if cfg is NULL. */
ifa_status ifa_config_default(ifa_config *cfg);

/* Create a handle on cfg->device; allocates device buffers for one segment
 * pair, the hit buffer and the digest.  *out is NULL on failure.
 * Errors: INVALID_ARG (NULL, clip_pct > 50, bad k list), CUDA (no such
 * device), OOM. */
ifa_status ifa_create(const ifa_config *cfg, ifa_handle **out);

/* Free everything the handle owns (waits for its device work).  NULL is a
 * no-op. */
void ifa_destroy(ifa_handle *h);

/* Use `stream` (a cudaStream_t of the handle's device, or NULL for the
 * library's own stream) as the compute stream for later calls. */
ifa_status ifa_set_stream(ifa_handle *h, void *stream);

/* Append n queries (the query set is loaded once at startup, Methods,
 * "Memory Management").  seqs[i] points at lens[i] ASCII bytes,
 * 1 <= lens[i] <= IFA_MAX_QUERY_LEN.  *first_id (may be NULL) receives the
 * id of the first appended query.  Copies the sequences.
 * BAD_STATE once a segment has been pushed since the last reset. */
ifa_status ifa_load_queries(ifa_handle *h, const uint8_t *const *seqs, const uint32_t *lens,
                            uint32_t n, uint32_t *first_id);

/* maxSubs for segments pushed from now on; any value (no upper limit,
 * Methods; a value >= L reports every window).  Applies to every query and
 * clears the per-query values of ifa_set_query_max_subs. */
ifa_status ifa_set_max_subs(ifa_handle *h, uint32_t max_subs);

/* Each query's own maxSubs for segments pushed from now on: max_subs[i] is
 * query i's (the paper fixes one maxSubs per run, Methods; a window of query
 * i is reported when its substitutions are <= max_subs[i]).  n must equal
 * the number of loaded queries; values of 255 or more report every window.
 * The array is copied.  Every streaming path honours it: popcount and
 * tensor-core brute force, the clip pass, indexed mode (one k and MinHits
 * plan per query for its own value) and the automatic mode choice, which
 * is redone.  max_subs == NULL with n == 0 goes back to the single value
 * of ifa_set_max_subs.  ifa_load_queries also goes back to it (the new
 * queries have no value yet).  Hits already reported are unchanged.
 * Errors: INVALID_ARG (NULL handle, n != loaded query count, NULL array
 * with n > 0); BAD_STATE when query sets are registered (ifa_set_add: each
 * set carries its own maxSubs); CUDA/OOM from re-uploading the query table. */
ifa_status ifa_set_query_max_subs(ifa_handle *h, const uint32_t *max_subs, uint32_t n);

/* Brute force, indexed, or automatic (Discussion): by rates measured on
 * this GPU unless ifa_config.auto_crossover sets a query-count rule. */
ifa_status ifa_set_mode(ifa_handle *h, ifa_mode mode);

/* Stream one reference segment past the queries (Methods, "Algorithm
 * Design": reference processed on demand, no preprocessing).  `ascii`
 * holds len bytes in memory of kind `mem`; `pieces` (host memory) maps it
 * onto contigs as described at ifa_piece.  Windows that straddle two
 * segments of one contig are found through a halo of the previous
 * segment's last bases.
 * IFA_MEM_HOST / IFA_MEM_HOST_PINNED: returns once the bytes are on the
 * device (the caller may then reuse its buffer); the scan continues
 * asynchronously.  IFA_MEM_DEVICE and IFA_MEM_HOST_PINNED_ASYNC: returns
 * once the work is enqueued; the buffer must stay unchanged until
 * ifa_flush() returns.
 * Errors: INVALID_ARG (len > segment_bytes, bad piece table, contig order),
 * BAD_STATE (no queries), CUDA. */
ifa_status ifa_push_segment(ifa_handle *h, const uint8_t *ascii, uint64_t len,
                            const ifa_piece *pieces, uint32_t n_pieces, ifa_mem mem);

/* Start the stream in the middle of a contig, as if the segments before
 * had been pushed: the next segment continues contig `contig` at offset
 * offset_in_contig + len, and `ascii` (len bytes, memory of kind `mem`)
 * holds that contig's bases just before it, from offset_in_contig on.  The
 * last min(len, L_max - 1) of them become the halo (L_max = the longest
 * loaded query), so windows (and soft-clipped windows) that straddle the
 * boundary are found, while windows lying wholly inside these bases are not
 * reported: they belong to whoever scans that part of the reference.  This
 * is how one reference is split by range over several handles or GPUs (the
 * paper splits its work by contig over threads, Methods, "Memory
 * Management"): each range's handle primes its halo and streams its range,
 * and the ranges' hits together are exactly one pass's hits.
 * Call it after ifa_load_queries and before the range's first segment, with
 * no contig open.  Host buffers may be reused on return; a device buffer
 * must stay unchanged until the next ifa_flush().
 * Errors: INVALID_ARG (len 0, contig order), BAD_STATE (no queries, a
 * contig open), CUDA. */
ifa_status ifa_prime_halo(ifa_handle *h, uint32_t contig, uint64_t offset_in_contig, const uint8_t *ascii,
                          uint64_t len, ifa_mem mem);

/* Wait until every pushed segment is scanned.  Returns HIT_OVERFLOW if the
 * hit buffer filled since the last ifa_reset_results (hits already written
 * stay valid; digest and counts stay exact), and TIMEOUT if a tensor-core
 * scan's pipeline wait gave up (its results are incomplete; the context
 * stays usable and ifa_reset_results clears the status). */
ifa_status ifa_flush(ifa_handle *h);

/* Hits wait in a ring of hit_capacity entries in device memory (Methods,
 * "Output Format": hits leave as the stream goes).  A hit that finds the
 * ring full is dropped: the digest and per-query counts still count it,
 * HIT_OVERFLOW is reported, and hits claimed after the first dropped one are
 * not drained (they are part of the overflow).
 *
 * Copy up to cap buffered hits into out (host memory) and release their
 * ring slots; *n_out gets the number copied, *more (may be NULL) whether
 * buffered hits remain.  Order is unspecified (compare as sets).  Implies
 * ifa_flush().  Returns HIT_OVERFLOW (with the data) if hits were dropped;
 * once everything before the drop is drained the ring takes hits again. */
ifa_status ifa_drain_hits(ifa_handle *h, ifa_hit *out, uint64_t cap, uint64_t *n_out, int *more);

/* Like ifa_drain_hits, without waiting: copies (up to cap) the hits of the
 * segments whose scans have already finished, on a stream of its own, while
 * later segments are still being scanned, and frees their ring slots.  Call
 * it between ifa_push_segment calls to stream hits out of a ring smaller
 * than a pass's hits.  *more: finished hits remain.  Returns HIT_OVERFLOW
 * (with the data) once a hit was dropped. */
ifa_status ifa_poll_hits(ifa_handle *h, ifa_hit *out, uint64_t cap, uint64_t *n_out, int *more);

/* Digest of all hits since the last reset; per_query_counts (may be NULL)
 * receives one count per loaded query.  Implies ifa_flush(). */
ifa_status ifa_get_digest(ifa_handle *h, ifa_digest *d, uint64_t *per_query_counts);

/* Forget hits, digest, counts, overflow, a tensor-core timeout status,
 * statistics and the stream position (the next segment may start any
 * contig); keeps the queries, maxSubs (one or per query) and mode. */
ifa_status ifa_reset_results(ifa_handle *h);

/* Counters since the last reset. */
ifa_status ifa_get_stats(ifa_handle *h, ifa_stats *s);

/* Indexed-mode plan of each loaded query under the current maxSubs: its
 * seed length k, min-hits threshold and whether it is scanned exhaustively
 * (no listed k fits, or none qualifies and exhaustive_fallback is set, or
 * the query holds an N).  Arrays hold one entry per query; any may be NULL.
 * Computed on the device (MinHitsCalculator, Methods, indexed mode). */
ifa_status ifa_get_query_plan(ifa_handle *h, uint32_t *k, uint32_t *minhits, uint8_t *exhaustive);

/* MinHitsCalculator on the device for n bins (Methods, indexed mode): for
 * bin i, the query length L[i], substitutions subs[i] and seed length
 * k[i]; step, mask width, clip count, probability num/den, trials and seed
 * are shared.  out[i] receives the threshold (the largest m such that
 * at least num/den of the trials keep >= m error-free k-mers; the
 * deterministic bound when num >= den).  Host arrays.  Stateless apart from
 * the device choice. */
ifa_status ifa_minhits(int32_t device, const uint32_t *L, const uint32_t *subs, const uint32_t *k,
                       uint32_t n, uint32_t step, uint32_t mask_width, uint32_t max_clips,
                       uint32_t num, uint32_t den, uint32_t trials, uint64_t seed, uint32_t *out);

/* ---- Many query sets against a device-resident reference ------------
 *
 * Batching and serving (the paper's mode choice by query count,
 * Discussion, generalised): the reference is packed once into a store on
 * the device, any number of query sets -- each with its own maxSubs and
 * mode -- are registered, and one call scans all of them.  Hits, digest
 * and per-query counts go to the handle's usual outputs (ifa_drain_hits,
 * ifa_get_digest); query ids are global, a set's queries being the range
 * [first_query, first_query + n). */

/* Append len reference bytes to the store (packed on the device: 2 bits
 * per base, plus the sparse table of the words holding an N or a contig
 * start).  pieces: as for ifa_push_segment, in this chunk's coordinates;
 * a contig may continue into the next append (its piece has last = 0).
 * Every append except the last must hold a multiple of 32 bytes.
 * Errors: INVALID_ARG (pieces, alignment, contig order), OOM, CUDA. */
ifa_status ifa_ref_append(ifa_handle *h, const uint8_t *ascii, uint64_t len, const ifa_piece *pieces,
                          uint32_t n_pieces, ifa_mem mem);

/* Make room in the store for `bases` bases in total (bytes already appended
 * included), so that appends up to that size allocate nothing more; without
 * it the store grows by half its size whenever an append does not fit.
 * Errors: OOM, CUDA. */
ifa_status ifa_ref_reserve(ifa_handle *h, uint64_t bases);

/* Drop the store (frees its device memory). */
ifa_status ifa_ref_reset(ifa_handle *h);

/* Register n queries as one set with its own maxSubs (0..255 used as is;
 * larger values act as 255) and mode (IFA_MODE_AUTO: the autotuner picks
 * brute force or indexed).  *set_id and *first_query (may be NULL) receive
 * the set's id and its first global query id.  BAD_STATE after
 * ifa_push_segment (streaming and batching do not share a handle). */
ifa_status ifa_set_add(ifa_handle *h, const uint8_t *const *seqs, const uint32_t *lens, uint32_t n,
                       uint32_t max_subs, ifa_mode mode, uint32_t *set_id, uint32_t *first_query);

typedef enum {
    IFA_BATCH_PERSISTENT = 0,  /* one persistent launch over a device work queue, replayed from a CUDA graph */
    IFA_BATCH_PER_SET = 1      /* each set scanned by its own launches, one set after the other */
} ifa_batch_kind;

typedef struct {
    uint32_t mode;        /* IFA_MODE_BRUTE or IFA_MODE_INDEXED as run */
    uint32_t queries;     /* queries in the set */
    uint64_t hits;        /* hits of the set's queries in this run */
    float done_ms;        /* device time from the run's start to the set's completion */
    float pad;
} ifa_set_result;

/* Scan every registered set against the store; per_set (may be NULL)
 * receives one ifa_set_result per set.  Results add to the handle's
 * outputs (call ifa_reset_results between runs).  Waits for completion.
 * Errors: BAD_STATE (empty store or no sets), OOM, CUDA. */
ifa_status ifa_batch_run(ifa_handle *h, ifa_batch_kind kind, ifa_set_result *per_set);

/* ---- Serving: continuous batching over the store -------------------
 *
 * Requests (query sets) arrive at any time.  The store is cut into
 * n_slices slices scanned cyclically, one per ifa_serve_step: at each slice
 * boundary the waiting requests that fit the HBM budget are admitted (in
 * arrival order; one request is always admitted when none is active), then
 * one persistent launch scans the slice for every active request at once.
 * A request is complete once every slice has been scanned for it (one full
 * cycle from its admission); its hits wait in its own device ring until
 * ifa_serve_drain.  A request's results do not depend on the others
 * active with it.  Hit query ids are relative to the request. */

typedef struct {
    uint32_t state;        /* 0 queued, 1 active, 2 complete, 3 drained, 4 cancelled */
    uint32_t mode;         /* IFA_MODE_BRUTE or IFA_MODE_INDEXED as run */
    uint32_t queries;
    uint32_t slices_done;
    uint64_t hits;         /* hits found (may exceed the ring) */
    uint64_t overflowed;   /* 1 when the ring dropped hits */
    double submit_s;       /* seconds since ifa_serve_start */
    double admit_s;
    double done_s;
    ifa_digest digest;     /* over the request's hits, request-relative ids */
} ifa_request_info;

/* Start serving over the store: n_slices slices, an HBM budget (bytes) for
 * admitted requests' rings and plan entries, ring_hits hits per request.
 * The handle's clip_pct at this call applies to the whole session: the
 * clipped windows of a contig are scanned in the slice holding the contig's
 * first piece, for every request active there.
 * BAD_STATE when the store is empty.  Ends any previous serving session. */
ifa_status ifa_serve_start(ifa_handle *h, uint32_t n_slices, uint64_t hbm_budget_bytes, uint64_t ring_hits);

/* Queue one request.  IFA_MODE_AUTO is resolved when the request is
 * admitted (ifa_request_info.mode reads IFA_MODE_AUTO until then): by the
 * measured-rate model when auto_crossover is 0, else indexed from
 * auto_crossover queries on.  *request_id may be NULL. */
ifa_status ifa_serve_submit(ifa_handle *h, const uint8_t *const *seqs, const uint32_t *lens, uint32_t n,
                            uint32_t max_subs, ifa_mode mode, uint32_t *request_id);

/* Admit what fits, scan the next slice for all active requests, retire
 * the ones that are complete.  Waits for the slice.  *n_active and
 * *n_completed (may be NULL) receive the counts after the step.
 * OOM when a request's ring cannot be allocated: that request and the ones
 * after it stay queued holding nothing (cancel it, or retry the step). */
ifa_status ifa_serve_step(ifa_handle *h, uint32_t *n_active, uint32_t *n_completed);

/* State, timing and digest of one request. */
ifa_status ifa_serve_poll(ifa_handle *h, uint32_t request_id, ifa_request_info *info);

/* Copy a complete request's hits (up to cap) to out and free its ring;
 * HIT_OVERFLOW (with the data) when its ring dropped hits. */
ifa_status ifa_serve_drain(ifa_handle *h, uint32_t request_id, ifa_hit *out, uint64_t cap, uint64_t *n_out);

/* Bounds-checked builds.  A library compiled with -DIFA_BOUNDS_CHECK
 * (libifa_bc.so beside libifa.so) checks the index of every read of the
 * packed reference (hi/lo words, directory, exception table) against its
 * allocation.  The first read out of range on a device is recorded in a
 * device word as kind << 56 | index (kind 1 word, 2 directory entry,
 * 3 exception entry), the read returns an all-N word and nothing traps;
 * ifa_flush then fails with IFA_ERR_CUDA naming it.  This call waits for
 * the device, stores that word in *first (0: none) and *enabled = 1; with
 * reset != 0 it clears the word.  Default builds store *enabled = 0 and
 * *first = 0 and touch no device. */
ifa_status ifa_bounds_check(int device, uint64_t *first, uint32_t *enabled, int reset);

/* Cancel a queued, active or complete request: its ring is freed, its
 * budget returned and its hits discarded (state 4).  An active request
 * leaves the scan from the next ifa_serve_step on; the others active with
 * it are unaffected.  Nothing of it is in flight: ifa_serve_step waits for
 * its slice.  BAD_STATE for a drained or already cancelled request,
 * INVALID_ARG for an unknown id. */
ifa_status ifa_serve_cancel(ifa_handle *h, uint32_t request_id);

/* Slices scanned, nominal query-base comparisons done, host seconds spent
 * building plans and seconds spent waiting for slices, since
 * ifa_serve_start.  Any pointer may be NULL. */
ifa_status ifa_serve_stats(ifa_handle *h, uint64_t *slices_run, double *query_bases, double *plan_seconds,
                           double *scan_seconds);

/* End serving and free every request's ring. */
ifa_status ifa_serve_stop(ifa_handle *h);

/* Brute-force scan of one reference chunk that allocates no memory.
 *
 * The paper has no counterpart: this entry point exists for callers that
 * cannot call cudaMalloc at the point where they scan -- for example code
 * inside a framework whose caching allocator already holds the device
 * memory, where any allocation outside it fails, or a serving loop with a
 * fixed memory plan.  The caller passes every input and output buffer; the
 * library's own scratch (packed reference words, encoded queries, piece
 * table, per-query counts when per_query_counts_device is NULL) lives in one
 * file-scope device array of about 18 MB.  No call allocates device or
 * pinned memory itself (torch's allocator included).
 *
 * When that array takes device memory: the CUDA runtime loads the library's
 * device code into a context module by module, on first use (lazy loading,
 * its default), so on each device the array is placed by the first call of
 * this function there and stays until the process exits.  A call with
 * nq = 0 does only that set-up (every other argument but device is then
 * ignored) and returns IFA_OK: make it once per device at start-up, before
 * a caching allocator reserves the device's memory and before any stream
 * capture.  Later calls need no new device memory.  (With the environment
 * variable CUDA_MODULE_LOADING=EAGER the array is placed when the context
 * is created.)
 *
 * Limits: 1..256 queries (1..255 bp each), 1..32 MiB of reference, 1..32768
 * whole contigs (every piece has last = 1 and offset_in_contig = 0; no
 * halo is carried between calls).  Larger sizes return
 * IFA_ERR_INVALID_ARG with a message naming the limit, before anything is
 * enqueued.  max_subs takes any value (255 or more reports every window).
 *
 * queries/qlens: host ASCII, as for ifa_load_queries.  ref_device: len
 * ASCII bytes in device memory.  pieces: host, as for ifa_push_segment.
 * hits_device: room for hit_capacity ifa_hit (device, 16-byte aligned:
 * hits are stored 16 bytes at a time).  counters_device: 5 uint64 on the
 * device (8-byte aligned), set to {hits claimed (may exceed hit_capacity),
 * overflow flag, digest count, digest sum, digest xor}.
 * per_query_counts_device: nq uint64 on the device (8-byte aligned), or
 * NULL.  A misaligned buffer returns IFA_ERR_INVALID_ARG.  stream: the
 * cudaStream_t to enqueue on (NULL = legacy default stream).  Results are
 * in the caller's buffers once the stream has passed this call's work; hit
 * order is unspecified.
 *
 * The work is enqueued on `device` (a device ordinal); the calling
 * thread's current device is the same after the call as before it.
 *
 * The call copies queries and the piece table from host memory that it
 * frees on return, so it cannot be captured into a CUDA graph: on a stream
 * that is being captured it returns IFA_ERR_INVALID_ARG before enqueuing
 * anything.
 * Every call on a device shares the one scratch array and leaves its
 * contents behind; each call clears what must start at zero (the counters
 * and per-query counts) itself.  Calls whose device work overlaps -- two
 * streams, or two threads -- race on the scratch and give wrong results. */
ifa_status ifa_scan_brute_noalloc(int32_t device, const uint8_t *const *queries,
                                  const uint32_t *qlens, uint32_t nq, const uint8_t *ref_device,
                                  uint64_t len, const ifa_piece *pieces, uint32_t n_pieces,
                                  uint32_t max_subs, ifa_hit *hits_device, uint64_t hit_capacity,
                                  uint64_t *counters_device, uint64_t *per_query_counts_device,
                                  void *stream);

/* ---- SAM text (Methods, "Output Format"; host-side, needs no device) ----
 *
 * The paper writes headerless SAM records as the stream goes, because the
 * full contig list is only known at the end, and a separate header file
 * (its outh= flag) to be concatenated in front.  The primary alignment of a
 * query is the first valid one in reference order (Results, accuracy
 * validation).
 *
 * Readings where the paper is silent: FLAG is 16 for strand '-' plus 256
 * for a secondary record; POS is pos + 1; MAPQ is 255 (not available);
 * CIGAR is "<L>M", or "<left>S<L - left - right>M<right>S" for a hit with
 * soft clips (ifa_hit.clips); RNEXT/PNEXT/TLEN are * 0 0; SEQ is the
 * query on the reference's forward strand (the reverse complement for
 * '-'), upper case, every non-ACGT byte written as N; QUAL is *; the one
 * tag is NM:i:<mismatches>. */
typedef struct {
    const uint8_t *const *query_seqs;   /* n_queries ASCII queries, as loaded */
    const uint32_t *query_lens;
    const char *const *query_names;     /* n_queries NUL-terminated names, or NULL: "q<id>" */
    uint32_t n_queries;
    const char *const *contig_names;    /* indexed by contig id, or NULL: "c<id>" */
    uint32_t n_contig_names;            /* entries of contig_names (ids beyond get "c<id>") */
} ifa_sam_info;

/* SAM records for n hits, one line each, no header.  hits (host) is sorted
 * in place into reference order (contig id, pos, strand, query,
 * mismatches, clips).  primary_seen (host, n_queries bytes, zeroed by the caller
 * once per pass over the reference) marks queries whose primary was already
 * written: a hit is primary when its query's byte is 0, which this call then
 * sets.  Calls must follow the stream order (drain after ifa_flush).
 * out (host, cap bytes) receives the text, not NUL-terminated; *n_out is
 * its length.  If cap is too small nothing is written, primary_seen is not
 * changed, *n_out is the length needed and the status is
 * IFA_ERR_INVALID_ARG.  A hit naming a query >= n_queries or a strand
 * other than 0/1 is IFA_ERR_INVALID_ARG, before anything is written. */
ifa_status ifa_sam_records(ifa_hit *hits, uint64_t n, const ifa_sam_info *info, uint8_t *primary_seen,
                           char *out, uint64_t cap, uint64_t *n_out);

/* The separate SAM header: "@HD VN:1.6 SO:unsorted" and one "@SQ SN LN"
 * line per contig, tab-separated, in the order given.  contig_ids[i] names
 * contig i ("c<id>") when contig_names is NULL.  Buffer rules as for
 * ifa_sam_records. */
ifa_status ifa_sam_header(const char *const *contig_names, const uint32_t *contig_ids,
                          const uint64_t *contig_lens, uint32_t n, char *out, uint64_t cap, uint64_t *n_out);

/* Human-readable description of the last failure on h (or of the last
 * failed ifa_create/ifa_minhits/ifa_scan_brute_noalloc/ifa_sam_* when h is NULL).
 * Never NULL. */
const char *ifa_last_error(const ifa_handle *h);

#ifdef __cplusplus
}
#endif

#endif /* IFA_H */

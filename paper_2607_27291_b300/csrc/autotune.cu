// autotune.cu -- the measured-rate choice behind IFA_MODE_AUTO.
//
// The paper finds that the crossover between brute force and indexed mode
// depends on the workload: on its RefSeq runs it lies between 100 and 200
// queries (Results, Terabase-Scale Performance; Discussion).  Here the
// crossover is computed instead.  The rates of the modes' three kinds of
// work are measured once on the device with count-only sinks:
//   R_brute  entry x base evaluations / s of the brute-force scan,
//   R_pos    reference positions x seed tables / s of the seed scan,
//   R_cand   verified candidates / s.
// A query set then takes the mode with the smaller predicted time per
// reference base:
//   brute   = 2 n / R_brute
//   indexed = T / R_pos + C / R_cand + 2 n_exh / R_brute
// where n is the number of queries, T the number of distinct seed lengths
// (one table each), C the expected random seed hits per base of the seeded
// entries ((L - k) / step + 1 k-mers, each hitting with probability 4^-k),
// and n_exh the queries the plan scans exhaustively.
//
// The rates are measured on at least 16 Mbp, so that launch overheads do
// not decide, and with at least 16 queries (the given ones, then random
// ones of their lengths), so that R_brute is the rate one more query costs.
// Batches measure on the store (once per handle), serving on the store once
// per session, streaming once per handle and maxSubs -- each on a 16 Mbp
// uniform random sequence packed on the device when the store is smaller or
// absent (a stream's reference has not arrived when its mode is needed).
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "handle.cuh"

namespace ifa {

namespace {

constexpr uint32_t kRateQueries = 128;          // queries the rates are measured with, at most
constexpr uint32_t kRateQueriesMin = 16;        // and at least (padded with random ones)
constexpr uint64_t kCalibBases = 16ull << 20;   // streaming calibration sequence
constexpr uint64_t kCalibPad = 16;              // words packed (as N) after it, read ahead by the scans

ifa_status afail(ifa_handle *h, ifa_status st, const std::string &msg) {
    h->err = msg;
    return st;
}

// Uniform random ACGT, one base per byte, from a counter hash.
__global__ void k_fill_random_bases(uint8_t *a, uint64_t n, uint64_t seed) {
    const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
    for (uint64_t i = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride)
        a[i] = "ACGT"[mix64(i + seed) & 3u];
}

// Device buffers of one measurement, freed on every return path.
struct Scratch {
    std::vector<void *> p;
    template <class T>
    cudaError_t get(T *&out, size_t n) {
        void *q = nullptr;
        const cudaError_t e = cudaMalloc(&q, std::max<size_t>(1, n) * sizeof(T));
        if (e == cudaSuccess) p.push_back(q);
        out = static_cast<T *>(q);
        return e;
    }
    ~Scratch() {
        for (void *q : p) cudaFree(q);
    }
};

// Time of the last of `reps` back-to-back runs of f on stream st (ms).
template <class F>
cudaError_t time_ms(cudaStream_t st, int reps, F f, float &ms) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    for (int r = 0; r < reps && e == cudaSuccess; r++) {
        e = cudaEventRecord(e0, st);
        if (e == cudaSuccess) e = f();
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    }
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    return e;
}

}  // namespace

double seed_hits_per_base(uint32_t L, uint32_t k, uint32_t step) {
    if (k == 0 || k > L || step == 0) return 0;
    return static_cast<double>((L - k) / step + 1) / std::pow(4.0, static_cast<double>(k));
}

ModeCost predict_cost(const Rates &r, const std::vector<std::string> &qs, uint32_t first, uint32_t n,
                      const IndexedState &plan, uint32_t step) {
    ModeCost c;
    c.brute_s = 2.0 * n / std::max(1.0, r.brute);
    double cand = 0, exh = 0;
    std::vector<uint32_t> ks;
    for (uint32_t q = first; q < first + n; q++) {
        if (plan.plan_exhaustive.size() <= q || plan.plan_exhaustive[q]) {
            exh += 2.0;
            continue;
        }
        c.seeded = true;
        cand += 2.0 * seed_hits_per_base(static_cast<uint32_t>(qs[q].size()), plan.plan_k[q], step);
        ks.push_back(plan.plan_k[q]);
    }
    std::sort(ks.begin(), ks.end());
    ks.erase(std::unique(ks.begin(), ks.end()), ks.end());
    c.idx_s = ks.size() / std::max(1.0, r.pos) + cand / std::max(1.0, r.cand) + exh / std::max(1.0, r.brute);
    return c;
}

ifa_status measure_rates(ifa_handle *h, const Batch &b, const std::vector<std::string> &qs_in,
                         const std::vector<uint32_t> &s_in, Rates &out) {
    const uint32_t ngiven = static_cast<uint32_t>(std::min<size_t>(qs_in.size(), kRateQueries));
    if (ngiven == 0 || b.nbases == 0) return afail(h, IFA_ERR_BAD_STATE, "rate measurement: no queries or no reference");
    std::vector<std::string> qs(qs_in.begin(), qs_in.begin() + ngiven);
    std::vector<uint32_t> svec(s_in.begin(), s_in.begin() + ngiven);
    for (uint32_t i = 0; qs.size() < kRateQueriesMin; i++) {
        // random queries of the given lengths and maxSubs, in turn
        std::string q(qs[i % ngiven].size(), 'A');
        for (size_t j = 0; j < q.size(); j++) q[j] = "ACGT"[mix64((static_cast<uint64_t>(i) << 32) + j) & 3u];
        qs.push_back(q);
        svec.push_back(svec[i % ngiven]);
    }
    const uint32_t nq = static_cast<uint32_t>(qs.size());
    uint32_t lmax = 1;
    for (const auto &q : qs) lmax = std::max<uint32_t>(lmax, static_cast<uint32_t>(q.size()));
    uint32_t w = 1;
    while (w * 32 < lmax) w <<= 1;
    std::vector<uint4> words(static_cast<size_t>(2) * nq * w, make_uint4(0, 0, 0, 0));
    std::vector<uint32_t> meta(2 * nq, 0);
    for (uint32_t q = 0; q < nq; q++)
        for (uint32_t t = 0; t < 2; t++)
            encode_entry(qs[q], t == 1, w, svec[q], &words[static_cast<size_t>(2 * q + t) * w], &meta[2 * q + t]);
    const cudaStream_t st = h->stream;
    Scratch sc;
    uint4 *d_words = nullptr;
    uint32_t *d_meta = nullptr;
    unsigned long long *scratch = nullptr, *d_cand = nullptr;
    cudaError_t e = sc.get(d_words, words.size());
    if (e == cudaSuccess) e = sc.get(d_meta, meta.size());
    if (e == cudaSuccess) e = sc.get(scratch, 4 + nq);
    if (e == cudaSuccess) e = sc.get(d_cand, 1);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_words, words.data(), words.size() * sizeof(uint4), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_meta, meta.data(), meta.size() * sizeof(uint32_t), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(scratch, 0, (4 + nq) * sizeof(unsigned long long), st);
    if (e != cudaSuccess) return afail(h, cuda_status(e), std::string("rate measurement: ") + cudaGetErrorString(e));
    HitSink sink;
    sink.ring = nullptr;
    sink.head = scratch;
    sink.capacity = 0;
    sink.digest = scratch + 1;
    sink.overflow = reinterpret_cast<uint32_t *>(scratch + 3);
    sink.qcount = scratch + 4;
    sink.count_only = 1;
    QueryTable qt{d_words, d_meta, nullptr, 2 * nq, w};

    // brute force: the entries of one shared-memory chunk at their own maxSubs
    const uint32_t ne = std::max<uint32_t>(2, std::min<uint32_t>(2 * nq, scan_brute_chunk_entries(w) & ~1u));
    uint32_t lo = 255, hi = 0;
    for (uint32_t i = 0; i < ne; i++) {
        lo = std::min(lo, meta_L(meta[i]));
        hi = std::max(hi, meta_L(meta[i]));
    }
    float ms = 0;
    // the one-kernel scan: what batches run, and within 3 % of the streaming
    // scan + expansion pair on full segments, whose extra launch would weigh
    // about 15 % on this short calibration range
    e = time_ms(st, 2, [&] { return launch_scan_brute(b, qt, 0, ne, kSPerEntry, lo, hi, sink, st, nullptr); }, ms);
    if (e != cudaSuccess) return afail(h, cuda_status(e), std::string("rate measurement: ") + cudaGetErrorString(e));
    Rates r;
    r.brute = ne * static_cast<double>(b.nbases) / std::max(1e-6, ms * 1e-3);
    r.pos = 1e11;
    r.cand = 1e10;

    // seed scan with one query's tables: positions x tables per second
    uint32_t pick = 0;
    while (pick < nq && qs[pick].size() < 8) pick++;
    if (pick < nq) {
        IndexedState one;
        std::vector<uint8_t> in(nq, 0);
        in[pick] = 1;
        ifa_status s2 = indexed_plan_q(one, qs, svec, in, h->cfg, st, h->err);
        if (s2 == IFA_OK) s2 = indexed_tables(one, qs, meta, words, w, h->cfg, st, h->err);
        if (s2 != IFA_OK) return s2;
        if (one.targ.n) {
            e = cudaMemsetAsync(d_cand, 0, sizeof(unsigned long long), st);
            if (e == cudaSuccess)
                e = time_ms(st, 2, [&] {
                    return launch_seed_scan(b, qt, one.targ, one.d_entry_minhits, h->cfg.kmer_step, kSPerEntry, sink,
                                            d_cand, st);
                }, ms);
            if (e == cudaSuccess) r.pos = b.nbases / std::max(1e-6, ms * 1e-3);
        }
        one.release();
        // candidates: a dense plan (every query at k = 8, threshold 1, no
        // Monte Carlo), less the lookup time just measured
        IndexedState dense;
        std::vector<uint8_t> all(nq, 0);
        for (uint32_t q = 0; q < nq; q++) all[q] = qs[q].size() >= 8;
        ifa_config c8 = h->cfg;
        c8.k_list[0] = 8;
        c8.n_k = 1;
        c8.minhits_num = 1;
        c8.minhits_den = 1;
        s2 = e == cudaSuccess ? indexed_plan_q(dense, qs, svec, all, c8, st, h->err) : IFA_OK;
        if (s2 == IFA_OK && e == cudaSuccess) s2 = indexed_tables(dense, qs, meta, words, w, c8, st, h->err);
        if (s2 != IFA_OK) return s2;
        if (e == cudaSuccess && dense.targ.n) {
            e = cudaMemsetAsync(d_cand, 0, sizeof(unsigned long long), st);
            if (e == cudaSuccess)
                e = time_ms(st, 1, [&] {
                    return launch_seed_scan(b, qt, dense.targ, dense.d_entry_minhits, 1, kSPerEntry, sink, d_cand, st);
                }, ms);
            unsigned long long nc = 0;
            if (e == cudaSuccess) e = cudaMemcpy(&nc, d_cand, sizeof(nc), cudaMemcpyDeviceToHost);
            const double t = ms * 1e-3 - b.nbases / r.pos;
            if (e == cudaSuccess && nc > 1000 && t > 0) r.cand = nc / t;
        }
        dense.release();
        if (e != cudaSuccess) return afail(h, cuda_status(e), std::string("rate measurement: ") + cudaGetErrorString(e));
    }
    out = r;
    return IFA_OK;
}

ifa_status choose_mode(ifa_handle *h, const Rates &r, const std::vector<std::string> &qs,
                       const std::vector<uint32_t> &svec, ifa_mode *mode) {
    const uint32_t nq = static_cast<uint32_t>(qs.size());
    IndexedState plan;
    const ifa_status st = indexed_plan_q(plan, qs, svec, std::vector<uint8_t>(nq, 1), h->cfg, h->stream, h->err);
    if (st != IFA_OK) return st;
    const ModeCost c = predict_cost(r, qs, 0, nq, plan, h->cfg.kmer_step);
    *mode = c.seeded && c.idx_s < c.brute_s ? IFA_MODE_INDEXED : IFA_MODE_BRUTE;
    return IFA_OK;
}

ifa_status rates_on_random(ifa_handle *h, const std::vector<std::string> &qs, const std::vector<uint32_t> &svec,
                           Rates &out) {
    const cudaStream_t st = h->stream;
    const uint64_t nwords = kCalibBases / 32 + kCalibPad;
    Scratch sc;
    uint8_t *d_ascii = nullptr;
    DevPiece *d_piece = nullptr;
    RefBufs R;
    cudaError_t e = sc.get(d_ascii, kCalibBases);
    if (e == cudaSuccess) e = sc.get(d_piece, 1);
    if (e == cudaSuccess) e = refbufs_alloc(R, nwords, 0, nwords);
    const DevPiece piece{0, 0, 0, 1};
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_piece, &piece, sizeof(piece), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) {
        k_fill_random_bases<<<148 * 4, 256, 0, st>>>(d_ascii, kCalibBases, 0x5eed5eedull);
        e = cudaGetLastError();
    }
    int launches = 0;
    if (e == cudaSuccess)
        e = pack_batch(R, d_ascii, 0, 0, d_ascii, kCalibBases, nwords, d_piece, 1, false, st, &launches);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    ifa_status status = IFA_OK;
    if (e != cudaSuccess) {
        status = afail(h, cuda_status(e), std::string("calibration sequence: ") + cudaGetErrorString(e));
    } else {
        const Batch b = make_batch(R, kCalibBases, 0, d_piece, 1);
        status = measure_rates(h, b, qs, svec, out);
    }
    refbufs_free(R);
    return status;
}

ifa_status rates_on_store(ifa_handle *h, const Batch &store, const std::vector<std::string> &qs,
                          const std::vector<uint32_t> &svec, Rates &out) {
    if (store.nbases < kCalibBases) return rates_on_random(h, qs, svec, out);
    Batch b = store;
    b.nbases = std::min<uint64_t>(store.nbases, 2 * kCalibBases);
    return measure_rates(h, b, qs, svec, out);
}

}  // namespace ifa

/*
 * ifa_oracle.c -- plain, slow CPU oracle for the indel-free scan.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the timed
 * CPU baseline of the benchmark may load this file's library.  It shares no
 * code, header, table or constant with the CUDA path.
 *
 * What it computes (each function cites the paper passage it follows):
 *
 *  oracle_brute    every (query, strand, contig, window) whose Hamming
 *                  distance is <= maxSubs (Methods, "Algorithm Design",
 *                  brute-force mode: alignment tested at every start
 *                  position; the introduction fixes Hamming distance as the
 *                  metric).  A byte that is not A/C/G/T (either case) is N
 *                  and mismatches everything, on both sides.
 *  oracle_indexed  the brute hits whose seed count reaches the query's
 *                  min-hits threshold (Methods, indexed mode: query k-mer
 *                  seeds, per-query MinHitsCalculator threshold).
 *  oracle_minhits  the MinHitsCalculator Monte Carlo threshold, and its
 *                  P = 100% deterministic bound (Methods, indexed mode).
 *  oracle_philox4x32_10  the counter-based generator of Salmon et al.,
 *                  "Parallel random numbers: as easy as 1, 2, 3" (SC'11).
 *  oracle_digest   order-independent digest of a hit list (count, sum and
 *                  xor of a 64-bit mix of each tuple; the mix is Vigna's
 *                  splitmix64 finaliser).
 *
 * Readings where the paper is silent (kept in the design notes as well):
 *  - N on either side counts as one mismatch;
 *  - a '-' hit at pos means revcomp(query) equals ref[pos .. pos+L-1] up to
 *    the mismatches, pos being the leftmost forward coordinate;
 *  - soft clipping at contig ends (Methods, "Algorithm Design": alignments
 *    may overhang a contig end by up to a share of the query length, 25 %
 *    by default): with clip_pct > 0 a window may start up to
 *    C = floor(clip_pct * L / 100) bases before its contig or end up to C
 *    bases after it.  Its overhanging bases are clips, not mismatches; it
 *    is a hit when clips <= C, at least one base is aligned and the
 *    mismatches of the aligned bases are <= maxSubs.  pos is the contig
 *    coordinate of the first aligned base and `clips` holds the clips
 *    (left | right << 8).  With clip_pct = 0 windows never leave a contig,
 *    so a contig shorter than the query gives no hit;
 *  - palindromic queries report both strands.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    uint32_t query, contig, pos;
    uint8_t strand, mismatches;
    uint16_t clips;
} oracle_hit;

/* ------------------------------------------------------------------ bases */

/* Upper-case A/C/G/T for a base, 'N' for anything else. */
static uint8_t fold_base(uint8_t c)
{
    switch (c) {
    case 'A': case 'a': return 'A';
    case 'C': case 'c': return 'C';
    case 'G': case 'g': return 'G';
    case 'T': case 't': return 'T';
    default: return 'N';
    }
}

static uint8_t complement_base(uint8_t c)
{
    switch (fold_base(c)) {
    case 'A': return 'T';
    case 'C': return 'G';
    case 'G': return 'C';
    case 'T': return 'A';
    default: return 'N';
    }
}

/* Reverse complement of q[0..L) into out (folded; non-bases become 'N'). */
void oracle_revcomp(const uint8_t *q, uint32_t L, uint8_t *out)
{
    for (uint32_t i = 0; i < L; i++)
        out[i] = complement_base(q[L - 1 - i]);
}

/* Number of positions i < L where a[i] != b[i] or either is N.
 * Stops counting once the count exceeds `limit` (the result is then
 * only known to be > limit, which is all a caller with threshold `limit`
 * needs). */
static uint32_t window_mismatches(const uint8_t *a, const uint8_t *b, uint32_t L, uint32_t limit)
{
    uint32_t mm = 0;
    for (uint32_t i = 0; i < L; i++) {
        uint8_t x = fold_base(a[i]);
        uint8_t y = fold_base(b[i]);
        if (x == 'N' || y == 'N' || x != y) {
            mm++;
            if (mm > limit)
                return mm;
        }
    }
    return mm;
}

/* Mismatch count of query q (strand t) at window pos of a contig, in full
 * (no early stop).  Exposed so tests can recompute single hits. */
uint32_t oracle_window_mismatches(const uint8_t *q, uint32_t L, uint8_t strand,
                                  const uint8_t *contig, uint64_t pos)
{
    uint8_t *qq = (uint8_t *)malloc(L ? L : 1);
    if (strand)
        oracle_revcomp(q, L, qq);
    else
        for (uint32_t i = 0; i < L; i++) qq[i] = fold_base(q[i]);
    uint32_t mm = window_mismatches(qq, contig + pos, L, 0xffffffffu);
    free(qq);
    return mm;
}

static void put_hit(oracle_hit *out, int64_t cap, int64_t n, uint32_t q, uint32_t c,
                    uint64_t p, uint8_t t, uint32_t mm, uint16_t clips)
{
    if (n < cap) {
        out[n].query = q;
        out[n].contig = c;
        out[n].pos = (uint32_t)p;
        out[n].strand = t;
        out[n].mismatches = (uint8_t)(mm > 255 ? 255 : mm);
        out[n].clips = clips;
    }
}

/*
 * Clipped windows of one (query, strand, contig) (Methods, "Algorithm
 * Design", soft clipping): every start p in [-C, n - L + C] whose window
 * overhangs the contig (p < 0 or p + L > n) by 1..C bases in total and
 * keeps at least one base inside it.  Writes the hits from index n on and
 * returns the new count.
 */
static int64_t clipped_windows(const uint8_t *qq, uint32_t L, const uint8_t *r, uint64_t rn, uint32_t clip_pct,
                               uint32_t max_subs, uint32_t j, uint32_t cid, uint8_t t, oracle_hit *out,
                               int64_t cap, int64_t n)
{
    const int64_t C = (int64_t)((uint64_t)clip_pct * L / 100u);
    const int64_t len = (int64_t)rn;
    for (int64_t p = -C; p <= len - (int64_t)L + C; p++) {
        const int64_t left = p < 0 ? -p : 0;
        const int64_t right = p + (int64_t)L > len ? p + (int64_t)L - len : 0;
        const int64_t clips = left + right;
        if (clips == 0 || clips > C || clips >= (int64_t)L)
            continue;
        const uint32_t aligned = L - (uint32_t)clips;
        uint32_t mm = window_mismatches(qq + left, r + p + left, aligned, max_subs);
        if (mm <= max_subs) {
            put_hit(out, cap, n, j, cid, (uint64_t)(p + left), t, mm, (uint16_t)(left | (right << 8)));
            n++;
        }
    }
    return n;
}

/*
 * Brute-force mode (Methods, "Algorithm Design"): every start position of
 * every contig, both strands, every query.
 *
 * queries: concatenated ASCII, query j is qcat[qoff[j] .. qoff[j]+qlen[j]).
 * contigs: concatenated ASCII, contig i is rcat[roff[i] .. roff[i]+rlen[i]),
 *          reported with id rid[i].
 * Writes at most `cap` hits to `out` in loop order and returns the total
 * number of hits (call again with a larger buffer if it exceeds cap).
 */
int64_t oracle_brute(const uint8_t *qcat, const uint64_t *qoff, const uint32_t *qlen, uint32_t nq,
                     const uint8_t *rcat, const uint64_t *roff, const uint64_t *rlen,
                     const uint32_t *rid, uint32_t nc, uint32_t max_subs, uint32_t clip_pct,
                     oracle_hit *out, int64_t cap)
{
    int64_t n = 0;
    for (uint32_t j = 0; j < nq; j++) {
        uint32_t L = qlen[j];
        if (L == 0)
            continue;
        uint8_t *fwd = (uint8_t *)malloc(L);
        uint8_t *rev = (uint8_t *)malloc(L);
        for (uint32_t i = 0; i < L; i++)
            fwd[i] = fold_base(qcat[qoff[j] + i]);
        oracle_revcomp(qcat + qoff[j], L, rev);
        for (uint8_t t = 0; t < 2; t++) {
            const uint8_t *qq = t ? rev : fwd;
            for (uint32_t c = 0; c < nc; c++) {
                const uint8_t *r = rcat + roff[c];
                if (clip_pct)
                    n = clipped_windows(qq, L, r, rlen[c], clip_pct, max_subs, j, rid[c], t, out, cap, n);
                if (rlen[c] < L)
                    continue;
                for (uint64_t p = 0; p + L <= rlen[c]; p++) {
                    uint32_t mm = window_mismatches(qq, r + p, L, max_subs);
                    if (mm <= max_subs) {
                        put_hit(out, cap, n, j, rid[c], p, t, mm, 0);
                        n++;
                    }
                }
            }
        }
        free(fwd);
        free(rev);
    }
    return n;
}

/*
 * Seed count of one window (Methods, indexed mode).  The query k-mers are
 * taken at offsets 0, step, 2*step, ... with o + k <= L.  Position j of a
 * k-mer is ignored when it lies in the masked middle [mlo, mlo + mask_w),
 * mlo = (k - mask_w) / 2 (the paper's XXXXX-NNN-XXXXX example).  A k-mer is
 * a seed hit when every unmasked position holds the same A/C/G/T base on
 * the query and the reference.
 */
static uint32_t window_seeds(const uint8_t *qq, const uint8_t *r, uint32_t L, uint32_t k,
                             uint32_t step, uint32_t mask_w)
{
    uint32_t seeds = 0;
    uint32_t mlo = (k - mask_w) / 2;
    for (uint32_t o = 0; o + k <= L; o += step) {
        int ok = 1;
        for (uint32_t j = 0; j < k && ok; j++) {
            if (mask_w && j >= mlo && j < mlo + mask_w)
                continue;
            uint8_t a = fold_base(qq[o + j]);
            uint8_t b = fold_base(r[o + j]);
            if (a == 'N' || b == 'N' || a != b)
                ok = 0;
        }
        seeds += (uint32_t)ok;
    }
    return seeds;
}

/*
 * Indexed mode result: the brute-force hits whose seed count reaches the
 * query's threshold.  Per query j: k[j] is its seed length and minhits[j]
 * its threshold; exhaustive[j] != 0 keeps every brute hit of that query
 * (queries with no usable seed length, e.g. ones that contain N).
 * Clipped windows (clip_pct > 0) are kept exhaustively, as in brute-force
 * mode: the seed threshold is planned for whole windows (a reading; the
 * paper does not say how clips enter the Monte Carlo).
 */
int64_t oracle_indexed(const uint8_t *qcat, const uint64_t *qoff, const uint32_t *qlen, uint32_t nq,
                       const uint8_t *rcat, const uint64_t *roff, const uint64_t *rlen,
                       const uint32_t *rid, uint32_t nc, uint32_t max_subs,
                       const uint32_t *kq, const uint32_t *minhits, const uint8_t *exhaustive,
                       uint32_t step, uint32_t mask_w, uint32_t clip_pct, oracle_hit *out, int64_t cap)
{
    int64_t n = 0;
    for (uint32_t j = 0; j < nq; j++) {
        uint32_t L = qlen[j];
        if (L == 0)
            continue;
        uint8_t *fwd = (uint8_t *)malloc(L);
        uint8_t *rev = (uint8_t *)malloc(L);
        for (uint32_t i = 0; i < L; i++)
            fwd[i] = fold_base(qcat[qoff[j] + i]);
        oracle_revcomp(qcat + qoff[j], L, rev);
        for (uint8_t t = 0; t < 2; t++) {
            const uint8_t *qq = t ? rev : fwd;
            for (uint32_t c = 0; c < nc; c++) {
                const uint8_t *r = rcat + roff[c];
                if (clip_pct)
                    n = clipped_windows(qq, L, r, rlen[c], clip_pct, max_subs, j, rid[c], t, out, cap, n);
                if (rlen[c] < L)
                    continue;
                for (uint64_t p = 0; p + L <= rlen[c]; p++) {
                    uint32_t mm = window_mismatches(qq, r + p, L, max_subs);
                    if (mm > max_subs)
                        continue;
                    if (!exhaustive[j]) {
                        uint32_t sd = window_seeds(qq, r + p, L, kq[j], step, mask_w);
                        if (sd < minhits[j])
                            continue;
                    }
                    put_hit(out, cap, n, j, rid[c], p, t, mm, 0);
                    n++;
                }
            }
        }
        free(fwd);
        free(rev);
    }
    return n;
}

/* Seed count of one (query, strand, window); exposed for tests. */
uint32_t oracle_window_seeds(const uint8_t *q, uint32_t L, uint8_t strand, const uint8_t *contig,
                             uint64_t pos, uint32_t k, uint32_t step, uint32_t mask_w)
{
    uint8_t *qq = (uint8_t *)malloc(L ? L : 1);
    if (strand)
        oracle_revcomp(q, L, qq);
    else
        for (uint32_t i = 0; i < L; i++) qq[i] = fold_base(q[i]);
    uint32_t sd = window_seeds(qq, contig + pos, L, k, step, mask_w);
    free(qq);
    return sd;
}

/* ------------------------------------------------------------- Philox */

/*
 * Philox4x32 with 10 rounds (Salmon, Moraes, Dror, Shaw, SC'11).  One round
 * multiplies words 0 and 2 by the two round multipliers, keeps both halves
 * of each 64-bit product, and mixes the high halves with words 1 and 3 and
 * the round key; the key is bumped by the two Weyl constants between
 * rounds.  The multipliers and Weyl constants are the ones given in that
 * paper.
 */
void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; r++) {
        uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* A stream of 32-bit words for one Monte Carlo trial: counter
 * (trial, block, bin, step) with key (seed low, seed high); the four
 * words of a block are used in order, then the block index advances. */
typedef struct {
    uint32_t ctr[4];
    uint32_t key[2];
    uint32_t buf[4];
    int used;
} word_stream;

static void ws_init(word_stream *ws, uint32_t trial, uint32_t bin, uint32_t step, uint64_t seed)
{
    ws->ctr[0] = trial;
    ws->ctr[1] = 0;
    ws->ctr[2] = bin;
    ws->ctr[3] = step;
    ws->key[0] = (uint32_t)seed;
    ws->key[1] = (uint32_t)(seed >> 32);
    ws->used = 4;
}

static uint32_t ws_next(word_stream *ws)
{
    if (ws->used == 4) {
        oracle_philox4x32_10(ws->ctr, ws->key, ws->buf);
        ws->ctr[1]++;
        ws->used = 0;
    }
    return ws->buf[ws->used++];
}

/* Uniform integer in [0, m), m >= 1: Lemire's multiply-shift with
 * rejection ("Fast random integer generation in an interval", 2019). */
static uint32_t ws_below(word_stream *ws, uint32_t m)
{
    uint64_t prod = (uint64_t)ws_next(ws) * m;
    uint32_t low = (uint32_t)prod;
    if (low < m) {
        uint32_t thresh = (uint32_t)(-m) % m;
        while (low < thresh) {
            prod = (uint64_t)ws_next(ws) * m;
            low = (uint32_t)prod;
        }
    }
    return (uint32_t)(prod >> 32);
}

/* Number of k-mer offsets (0, step, ... with o + k <= L). */
uint32_t oracle_kmer_count(uint32_t L, uint32_t k, uint32_t step)
{
    if (k == 0 || k > L || step == 0)
        return 0;
    return (L - k) / step + 1;
}

/*
 * The threshold a survivor histogram h[0..K] of `trials` trials gives: the
 * largest m such that at least num/den of the trials kept m or more
 * error-free k-mers, i.e. #{trials with >= m} * den >= num * trials
 * (Methods, indexed mode: the count needed to find an alignment "with a
 * user-defined probability").  m = 0 always qualifies.
 */
uint32_t oracle_minhits_quantile(const uint64_t *h, uint32_t K, uint32_t num, uint32_t den,
                                 uint64_t trials)
{
    unsigned __int128 need = (unsigned __int128)num * trials;
    uint64_t tail = 0;
    for (int64_t m = K; m >= 0; m--) {
        tail += h[m];
        if ((unsigned __int128)tail * den >= need)
            return (uint32_t)m;
    }
    return 0;
}

/*
 * MinHitsCalculator (Methods, indexed mode): the minimum number of seed
 * hits that an alignment with `subs` substitutions still shows with
 * probability >= num/den, for a query of length L, seed length k, offset
 * step `step` and a masked middle of width mask_w.
 *
 * Monte Carlo: each of `trials` trials places `subs` substitutions at
 * distinct uniform positions of [0, L) (a partial Fisher-Yates shuffle) and
 * counts the k-mers that keep every unmasked position free of them.  The
 * survivor counts are histogrammed (hist[0 .. K], K = k-mer count, may be
 * NULL) and the threshold is the largest m with
 *     #{trials with survivors >= m} * den >= num * trials.
 * With num == den (P = 100%) the deterministic bound
 *     max(0, K - (k - mask_w) * subs - max_clips)
 * is returned instead (no trials run, hist untouched).
 *
 * Randomness: trial t draws words from Philox4x32-10 with key (seed low,
 * seed high) and counter (t, block, L | subs << 8 | k << 16 | mask_w << 24,
 * step), consuming the four words of each block in order.
 */
uint32_t oracle_minhits(uint32_t L, uint32_t subs, uint32_t k, uint32_t step, uint32_t mask_w,
                        uint32_t max_clips, uint32_t num, uint32_t den, uint32_t trials,
                        uint64_t seed, uint64_t *hist)
{
    uint32_t K = oracle_kmer_count(L, k, step);
    if (K == 0)
        return 0;
    if (num >= den) {
        int64_t b = (int64_t)K - (int64_t)(k - mask_w) * (int64_t)subs - (int64_t)max_clips;
        return b > 0 ? (uint32_t)b : 0;
    }
    uint64_t *h = (uint64_t *)calloc(K + 1, sizeof(uint64_t));
    uint32_t *perm = (uint32_t *)malloc(L * sizeof(uint32_t));
    uint8_t *hitpos = (uint8_t *)malloc(L);
    uint32_t bin = (L & 0xff) | ((subs & 0xff) << 8) | ((k & 0xff) << 16) | ((mask_w & 0xff) << 24);
    uint32_t mlo = (k - mask_w) / 2;
    uint32_t ns = subs < L ? subs : L;
    for (uint32_t t = 0; t < trials; t++) {
        word_stream ws;
        ws_init(&ws, t, bin, step, seed);
        for (uint32_t i = 0; i < L; i++) {
            perm[i] = i;
            hitpos[i] = 0;
        }
        for (uint32_t i = 0; i < ns; i++) {
            uint32_t j = i + ws_below(&ws, L - i);
            uint32_t tmp = perm[i];
            perm[i] = perm[j];
            perm[j] = tmp;
            hitpos[perm[i]] = 1;
        }
        uint32_t surv = 0;
        for (uint32_t o = 0; o + k <= L; o += step) {
            int ok = 1;
            for (uint32_t j = 0; j < k; j++) {
                if (mask_w && j >= mlo && j < mlo + mask_w)
                    continue;
                if (hitpos[o + j]) {
                    ok = 0;
                    break;
                }
            }
            surv += (uint32_t)ok;
        }
        h[surv]++;
    }
    uint32_t best = oracle_minhits_quantile(h, K, num, den, trials);
    if (hist)
        memcpy(hist, h, (K + 1) * sizeof(uint64_t));
    free(h);
    free(perm);
    free(hitpos);
    return best;
}

/*
 * Seed length choice (Methods, indexed mode: the longest k of the list for
 * which enough seed hits are expected).  Reading: "enough" means a
 * threshold of at least 1.  Returns 1 and sets k/minhits when some k <= L
 * qualifies; otherwise sets k to the smallest listed k <= L with minhits
 * clamped to 1 and returns 0; returns -1 when no listed k fits in L.
 */
int oracle_choose_k(uint32_t L, uint32_t subs, const uint32_t *klist, uint32_t nk, uint32_t step,
                    uint32_t mask_w, uint32_t max_clips, uint32_t num, uint32_t den,
                    uint32_t trials, uint64_t seed, uint32_t *k_out, uint32_t *minhits_out)
{
    uint32_t best_k = 0, best_m = 0, small_k = 0;
    for (uint32_t i = 0; i < nk; i++) {
        uint32_t k = klist[i];
        if (k > L || k <= mask_w)
            continue;
        if (small_k == 0 || k < small_k)
            small_k = k;
        uint32_t m = oracle_minhits(L, subs, k, step, mask_w, max_clips, num, den, trials, seed, NULL);
        if (m >= 1 && k > best_k) {
            best_k = k;
            best_m = m;
        }
    }
    if (best_k) {
        *k_out = best_k;
        *minhits_out = best_m;
        return 1;
    }
    if (small_k) {
        *k_out = small_k;
        *minhits_out = 1;
        return 0;
    }
    *k_out = 0;
    *minhits_out = 0;
    return -1;
}

/* ------------------------------------------------------------- digest */

/* Vigna's splitmix64 output function (a variant of Stafford's Mix13). */
static uint64_t mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* Digest of a hit list: count, sum (mod 2^64) and xor of
 * mix64(a ^ mix64(b)) with a = query << 32 | contig and
 * b = pos << 32 | clips << 16 | strand << 8 | mismatches (clips is 0 for
 * a window inside its contig). */
void oracle_digest(const oracle_hit *h, int64_t n, uint64_t out[3])
{
    uint64_t sum = 0, xr = 0;
    for (int64_t i = 0; i < n; i++) {
        uint64_t a = ((uint64_t)h[i].query << 32) | h[i].contig;
        uint64_t b = ((uint64_t)h[i].pos << 32) | ((uint64_t)h[i].clips << 16) | ((uint64_t)h[i].strand << 8) |
                     h[i].mismatches;
        uint64_t v = mix64(a ^ mix64(b));
        sum += v;
        xr ^= v;
    }
    out[0] = (uint64_t)n;
    out[1] = sum;
    out[2] = xr;
}

// scan_tc.cu -- brute-force scan on the tensor cores (tcgen05, one-hot e4m3).
//
// The Hamming count of the paper's brute-force mode (Methods, Algorithm
// Design and SIMD Optimization) is L minus the number of matching bases, and
// the matches of every (query entry, window) pair form a matrix product:
// with each base written as a one-hot 4-vector (all zero for N, so an N on
// either side never matches),
//     matches(e, p) = sum_i sum_c Q[e][4 i + c] * R[p + i][c].
// Q is an M x K operand (entries x 4 L), R a K x N operand whose column for
// window p is the one-hot reference from p on.  The values are 0/1, exact in
// e4m3, and the sums (<= 64) exact in the f16 accumulator.
//
// The reference operand needs no Toeplitz matrix: in the K-major layout
// without swizzle, the 8 rows of a core matrix lie 16 bytes apart, and the
// one-hot string of windows 4 bases apart is exactly that -- window p + 4
// starts 16 bytes after window p.  So the N = 256 rows of one MMA are the
// windows p0 + phase + 4 n (n < 256) read straight from one one-hot string
// with leading offset 16 bytes (next 4 bases) and stride offset 128 bytes
// (next 8 windows); four phase-shifted strings cover 1024 consecutive
// windows.  A CTA keeps one 128-entry tile of Q in shared memory and sweeps
// its share of the reference:
//   warp 0      allocates the 512 TMEM columns; one lane issues the MMAs
//               (K / 32 per phase) into one of two 256-column accumulators
//               and commits them to mbarriers;
//   warp 1      builds the four one-hot strings of the next tile from the
//               2-bit words and their N / piece-start masks (double-buffered);
//   warps 2..9  read the accumulator (tcgen05.ld; a warp reads its 32 lanes
//               = 32 entries and half of the columns, two warps per lane
//               quarter so that two TMEM loads are in flight per quarter),
//               compare each entry's row with L - maxSubs and emit the hits
//               after checking that the window lies inside one piece and
//               belongs to this batch.
// Every mbarrier wait is bounded (4 s); a wait that gives up sets a status
// bit and makes every role skip its remaining work, so the CTA still reaches
// its barriers and frees the TMEM, and the host reads the status.
#include <cstring>
#include <string>
#include <vector>

#include <cuda_fp16.h>

#include "hits.cuh"

namespace ifa {

namespace {

constexpr int kTcEpiWarps = 8;                  // two per TMEM lane quarter, each half the columns
constexpr int kTcThreads = 32 * (2 + kTcEpiWarps);
constexpr int kTcM = 128;                       // entries per tile (MMA M)
constexpr int kTcN = 256;                       // windows per MMA (MMA N), 4 bases apart
constexpr int kTcPhases = 4;
constexpr int kTcTile = kTcN * kTcPhases;       // consecutive windows per reference tile
constexpr uint32_t kOneE4M3 = 0x38u;            // 1.0 in e4m3
constexpr uint32_t kTcMaxLpad = 64;             // queries up to 64 bases
constexpr size_t kTcHead = 8192;                // barriers, per-row data, hit staging
constexpr size_t kTcScratch = kTcEpiWarps * 32 * 33 * sizeof(float);
constexpr size_t kTcSmem = 120 * 1024;          // above half of an SM's shared memory: one CTA per SM
constexpr uint64_t kWaitLimitNs = 4000000000ull;  // a pipeline wait gives up after 4 s

struct TcHead {
    unsigned long long full_b[2], empty_b[2], full_acc[2], empty_acc[2];
    uint32_t tmem;
    uint32_t abort;
    uint32_t item;      // the item this CTA works on (taken from the work counter)
    uint32_t pad;
    float thr[kTcM];
    uint32_t len[kTcM];
    uint4 words[40];    // the builder's packed words of the current tile
    uint32_t tile_clean[2];  // per B buffer: 1 when every window of the tile lies in one piece and in this batch
    uint32_t tile_piece[2];  // per B buffer: that piece (valid when clean)
    uint32_t discard;        // takes the per-call hit counts of the clean-tile path (counted per lane instead)
    alignas(16) ifa_hit stage[kTcEpiWarps][32];  // read and written as uint4
};
static_assert(sizeof(TcHead) <= kTcHead, "tensor-core scan header");
static_assert(offsetof(TcHead, stage) % 16 == 0, "hit staging is moved as uint4");
// header + Q tile (128 x 256 B) + strings (2 x 4 x 4 (1024 + 64) B) + scratch
static_assert(kTcHead + 128 * 256 + 2 * 4 * 4 * (1024 + 64) + kTcScratch <= kTcSmem, "tensor-core scan smem");

__host__ __device__ constexpr uint32_t string_bytes(uint32_t lpad) { return 4u * (kTcTile + lpad); }

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor, K-major without swizzle: start address,
// leading byte offset (next core matrix along K), stride byte offset (next 8
// rows), descriptor version 1 at bit 46.
__device__ __forceinline__ uint64_t mdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return static_cast<uint64_t>((addr >> 4) & 0x3FFFu) | (static_cast<uint64_t>((lbo >> 4) & 0x3FFFu) << 16) |
           (static_cast<uint64_t>((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor: f16 accumulator (counts <= 64 are exact; each
// value still takes one 32-bit TMEM column, in its low half), e4m3 x e4m3,
// both K-major, N, M.
constexpr uint32_t kIdesc = (0u << 4) | (static_cast<uint32_t>(kTcN >> 3) << 17) |
                            (static_cast<uint32_t>(kTcM >> 4) << 24);

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for the barrier's phase `parity`; false when another role gave up or
// this wait passed its time limit (then the CTA's abort flag is set).
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile uint32_t *abort) {
    uint64_t t0 = 0;
    for (uint32_t i = 0;; i++) {
        uint32_t ok;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok) return true;
        if ((i & 63u) == 63u) {
            if (*abort) return false;
            const uint64_t t = global_ns();
            if (t0 == 0) {
                t0 = t;
            } else if (t - t0 > kWaitLimitNs) {
                *abort = 1;
                return false;
            }
        }
    }
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("{\n.reg .b64 st;\nmbarrier.arrive.shared::cta.b64 st, [%0];\n}" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tc_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t accumulate) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.u32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}" ::"r"(d),
        "l"(a), "l"(b), "r"(kIdesc), "r"(accumulate)
        : "memory");
}

// Issue a 64-column TMEM load of f16 values, two columns per register (the
// even column in the low half); the registers are valid after
// tc_wait_ld_regs().
__device__ __forceinline__ void tc_ld64h(uint32_t taddr, uint32_t *r) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.pack::16b.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
}

// Wait for outstanding TMEM loads; r's registers are operands, so their
// uses cannot move above the wait.
__device__ __forceinline__ void tc_wait_ld_regs(uint32_t *r) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                   "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]),
                   "+r"(r[22]), "+r"(r[23]), "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]),
                   "+r"(r[29]), "+r"(r[30]), "+r"(r[31])
                 :
                 : "memory");
}

// Largest of the 64 f16 counts held two per register.
__device__ __forceinline__ float max64h(const uint32_t *r) {
    __half2 m[16];
#pragma unroll
    for (int j = 0; j < 16; j++)
        m[j] = __hmax2(*reinterpret_cast<const __half2 *>(&r[j]), *reinterpret_cast<const __half2 *>(&r[j + 16]));
#pragma unroll
    for (int w = 8; w > 0; w >>= 1)
#pragma unroll
        for (int j = 0; j < w; j++) m[j] = __hmax2(m[j], m[j + w]);
    return fmaxf(__low2float(m[0]), __high2float(m[0]));
}

// Whether a piece other than the window's own starts inside [p + 1, p + L).
__device__ __forceinline__ bool crosses_piece(const Batch &b, uint64_t p, uint32_t L) {
    for (uint64_t q = p + 1; q < p + L;) {
        const uint64_t w = q >> 5;
        const uint32_t lo = static_cast<uint32_t>(q & 31u);
        const uint64_t end = (w + 1) << 5 < p + L ? (w + 1) << 5 : p + L;
        const uint32_t n = static_cast<uint32_t>(end - q);
        const uint32_t mask = (n >= 32u ? 0xffffffffu : ((1u << n) - 1u)) << lo;
        if (ref_word(b, w).w & mask) return true;
        q = end;
    }
    return false;
}

// Hits of one flagged chunk with every check: 64 counts of this lane's row
// (two f16 per word of mine2, even column low), windows p0 + 4 j; window
// bounds, piece crossing and piece lookup per hit (all lanes of the warp).
__device__ __noinline__ void emit_chunk(const Batch &b, const HitSink &sink, WarpHits &wh, const uint32_t *mine2,
                                        float thr, uint32_t L, uint32_t e, uint64_t p0, uint32_t lane) {
    for (int j = 0; j < 64; j++) {
        const __half2 v2 = *reinterpret_cast<const __half2 *>(&mine2[j >> 1]);
        const float mt_j = (j & 1) ? __high2float(v2) : __low2float(v2);
        const uint64_t p = p0 + 4u * static_cast<uint32_t>(j);
        bool hit = mt_j >= thr && p + L <= b.nbases && p + L >= static_cast<uint64_t>(b.halo) + 1;
        if (hit) hit = !crosses_piece(b, p, L);
        uint32_t contig = 0, pos = 0;
        if (hit) {
            const DevPiece pc = b.pieces[find_piece(b.pieces, b.npieces, p)];
            contig = pc.contig;
            pos = static_cast<uint32_t>(pc.contig_off + (p - pc.start));
        }
        wh.emit(sink, lane, hit, e >> 1, contig, pos, e & 1u, L - static_cast<uint32_t>(mt_j), nullptr);
    }
}

__global__ void __launch_bounds__(kTcThreads, 1)
k_scan_tc(Batch b, const uint8_t *__restrict__ tcA, const uint32_t *__restrict__ meta,
          const uint32_t *__restrict__ ids, uint32_t nent,
          uint32_t lpad, uint32_t s, uint32_t n_rt, uint32_t rt_per_item, uint32_t n_rchunks, uint32_t n_items,
          HitSink sink, unsigned int *status, unsigned int *work, uint32_t withhold_first) {
    extern __shared__ __align__(1024) uint8_t smem[];
    TcHead &H = *reinterpret_cast<TcHead *>(smem);
    const uint32_t K = 4u * lpad;                   // bytes per operand row
    uint8_t *sA = smem + kTcHead;                   // kTcM x K, core matrices of 8 rows x 16 B
    uint8_t *sB = sA + kTcM * K;                    // [2 buffers][4 phases][string_bytes]
    const uint32_t SB = string_bytes(lpad);
    // per epilogue warp: a flagged chunk of 32 x 32 counts (row = lane, padded)
    float *scratch = reinterpret_cast<float *>(sB + 2u * kTcPhases * SB);
    const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
    volatile uint32_t *abort = &H.abort;

    if (threadIdx.x == 0) {
        for (int i = 0; i < 2; i++) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&H.full_b[i])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&H.empty_b[i])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&H.full_acc[i])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&H.empty_acc[i])), "r"(kTcEpiWarps));
        }
        H.abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(&H.tmem)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = H.tmem;

    WarpHits wh;
    wh.init(warp >= 2 ? H.stage[warp - 2] : H.stage[0]);
    uint32_t gtile = 0;  // tiles processed by this CTA (barrier phases)

    for (;;) {
        // next item from the launch's work counter (balances the CTAs' shares)
        if (threadIdx.x == 0) H.item = atomicAdd(work, 1u);
        __syncthreads();
        const uint32_t item = H.item;
        if (item >= n_items) break;
        const uint32_t mt = item / n_rchunks;
        const uint32_t rt0 = (item % n_rchunks) * rt_per_item;
        const uint32_t rt1 = rt0 + rt_per_item < n_rt ? rt0 + rt_per_item : n_rt;
        // this item's entry tile and per-row thresholds
        {
            const uint4 *src = reinterpret_cast<const uint4 *>(tcA + static_cast<size_t>(mt) * kTcM * K);
            uint4 *dst = reinterpret_cast<uint4 *>(sA);
            for (uint32_t i = threadIdx.x; i < kTcM * K / 16; i += kTcThreads) dst[i] = __ldg(src + i);
            for (uint32_t r = threadIdx.x; r < kTcM; r += kTcThreads) {
                const uint32_t e = mt * kTcM + r;
                float t = 3.0e38f;
                uint32_t L = 0;
                if (e < nent) {
                    const uint32_t m = __ldg(meta + e);
                    L = meta_L(m);
                    // a row of length 0 pads a tile (batched sets): it never hits
                    t = L ? static_cast<float>(L) - static_cast<float>(entry_s(m, s)) : 3.0e38f;
                }
                H.thr[r] = t;
                H.len[r] = L;
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncthreads();
        }
        const uint32_t ntiles = rt1 > rt0 ? rt1 - rt0 : 0;
        if (warp == 0) {
            // ---- MMA issue (one lane)
            if (lane == 0 && !*abort) {
                const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
                for (uint32_t ti = 0; ti < ntiles; ti++) {
                    const uint32_t g = gtile + ti, sbuf = g & 1u, v = g >> 1;
                    if (!mbar_wait(smem_u32(&H.full_b[sbuf]), v & 1u, abort)) break;
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    bool ok = true;
                    for (uint32_t ph = 0; ph < kTcPhases && ok; ph++) {
                        const uint32_t u = 4u * g + ph, a = u & 1u, w = u >> 1;
                        if (w >= 1 && !mbar_wait(smem_u32(&H.empty_acc[a]), (w - 1) & 1u, abort)) {
                            ok = false;
                            break;
                        }
                        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                        const uint32_t bs = b0 + (sbuf * kTcPhases + ph) * SB;
                        for (uint32_t kk = 0; kk < K / 32; kk++) {
                            // A: next 16 B of K at +128 B, next 8 entries at +8 K; B: next 4 bases at
                            // +16 B, next 8 windows (32 bases) at +128 B
                            tc_mma(tmem + a * kTcN, mdesc(a0 + kk * 256u, 128u, 8u * K), mdesc(bs + kk * 32u, 16u, 128u),
                                   kk > 0);
                        }
                        tc_commit(smem_u32(&H.full_acc[a]));
                    }
                    if (!ok) break;
                    tc_commit(smem_u32(&H.empty_b[sbuf]));
                }
            }
            __syncwarp();
        } else if (warp == 1) {
            // ---- one-hot strings of each tile: string ph holds bases
            // pt + ph + i, i < 1024 + lpad, as 4 bytes each.  A lane takes the
            // 16-byte chunk q of every string (bases pt + 4 q + ph .. + 3): it
            // cuts the one-hots of bases 4 q .. 4 q + 7 from the packed words
            // and writes each string's chunk with one 16-byte store.
            const uint32_t nq4 = (kTcTile + lpad) / 4;   // chunks per string
            const uint64_t nwords = (b.nbases + 31) / 32;
            const uint32_t nw = (kTcTile + lpad + 31) / 32 + 1;  // words per tile (<= 35)
            // the piece holding the current tile's first window: one search per
            // item, then advanced tile by tile (the item's tiles are consecutive)
            uint32_t pi = lane == 0 && ntiles && b.npieces
                              ? find_piece(b.pieces, b.npieces, static_cast<uint64_t>(rt0) * kTcTile)
                              : 0u;
            for (uint32_t ti = 0; ti < ntiles && !*abort; ti++) {
                const uint32_t g = gtile + ti, sbuf = g & 1u, v = g >> 1;
                const uint64_t pt = static_cast<uint64_t>(rt0 + ti) * kTcTile;
                // the tile's words, loaded lane-parallel before the wait (N past the batch)
                const uint4 nword = make_uint4(0u, 0u, 0xffffffffu, 0u);
                const uint4 w0 = (pt >> 5) + lane < nwords ? ref_word(b, (pt >> 5) + lane) : nword;
                const uint4 w1 = 32u + lane < nw && (pt >> 5) + 32u + lane < nwords
                                     ? ref_word(b, (pt >> 5) + 32u + lane) : nword;
                if (lane == 0)
                    while (pi + 1 < b.npieces && b.pieces[pi + 1].start <= pt) pi++;
                if (v >= 1 && !mbar_wait(smem_u32(&H.empty_b[sbuf]), (v - 1) & 1u, abort)) break;
                H.words[lane] = w0;
                if (32u + lane < nw) H.words[32u + lane] = w1;
                __syncwarp();
                uint8_t *bb = sB + sbuf * kTcPhases * SB;
#pragma unroll 3
                for (uint32_t q = lane; q < nq4; q += 32u) {
                    const uint32_t k = q >> 3;                      // word of bases 4 q .. 4 q + 3
                    const uint32_t sh = (4u * q) & 31u;             // 0, 4, .., 28
                    const uint4 W0 = H.words[k];
                    const uint4 W1 = sh > 24u ? H.words[k + 1] : W0;
                    const uint32_t hi = __funnelshift_r(W0.x, W1.x, sh), lo = __funnelshift_r(W0.y, W1.y, sh);
                    const uint32_t nn = __funnelshift_r(W0.z, W1.z, sh);
                    uint32_t oh[8];
#pragma unroll
                    for (int k = 0; k < 8; k++) {
                        const uint32_t code = (((hi >> k) & 1u) << 1) | ((lo >> k) & 1u);
                        oh[k] = ((nn >> k) & 1u) ? 0u : (kOneE4M3 << (8u * code));
                    }
#pragma unroll
                    for (int ph = 0; ph < kTcPhases; ph++)
                        *reinterpret_cast<uint4 *>(bb + ph * SB + 16u * q) =
                            make_uint4(oh[ph], oh[ph + 1], oh[ph + 2], oh[ph + 3]);
                }
                // whether every window of the tile stays in one piece and in the batch
                // (no piece starts after its first base; halo and batch end clear)
                {
                    uint32_t starts = lane < nw ? H.words[lane].w : 0u;
                    if (lane == 0) starts &= ~1u;
                    if (32u + lane < nw) starts |= H.words[32u + lane].w;
                    const bool inside = pt >= b.halo && pt + kTcTile + lpad + 3 <= b.nbases;
                    const bool clean = inside && !__any_sync(0xffffffffu, starts != 0u);
                    if (lane == 0) {
                        H.tile_clean[sbuf] = clean && b.npieces > 0 ? 1u : 0u;
                        H.tile_piece[sbuf] = pi;
                    }
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncwarp();
                // (testing: withhold the CTA's first tile so that the MMA's wait runs out)
                if (lane == 0 && !(withhold_first && g == 0)) mbar_arrive(smem_u32(&H.full_b[sbuf]));
            }
        } else {
            // ---- epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31, columns
            // half * 128 .. + 127 of the accumulator
            const uint32_t quarter = warp & 3u;
            const uint32_t half = (warp - 2u) / 4u;
            const uint32_t row = 32u * quarter + lane;
            const uint32_t e = mt * kTcM + row;
            // the row's entry id (its query and strand): ids map the operand's
            // rows to the handle's entries when the operand holds a subset
            const uint32_t id = ids && e < nent ? __ldg(ids + e) : e;
            const float thr = H.thr[row];
            const __half2 thr2 = __float2half2_rn(thr < 60000.0f ? thr : 60000.0f);
            const uint32_t L = H.len[row];
            uint32_t row_hits = 0;  // this lane's hits in clean tiles (counted once per item)
            for (uint32_t ti = 0; ti < ntiles && !*abort; ti++) {
                const uint32_t g = gtile + ti;
                const uint64_t pt = static_cast<uint64_t>(rt0 + ti) * kTcTile;
                uint32_t clean = 0;
                uint32_t tpi = 0;         // the tile's piece (builder's record)
                bool have_piece = false;  // tpc loaded (first flagged chunk of a clean tile)
                DevPiece tpc{};
                bool ok = true;
                for (uint32_t ph = 0; ph < kTcPhases; ph++) {
                    const uint32_t u = 4u * g + ph, a = u & 1u, w = u >> 1;
                    if (!mbar_wait(smem_u32(&H.full_acc[a]), w & 1u, abort)) {
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    if (ph == 0) {
                        // the builder's clean flag: the tile's full_b phase has completed
                        // (acquire; returns at once), and the flag is not rewritten before
                        // this phase's readout lets the MMAs of phases 2 and 3 run, after
                        // which empty_b frees the buffer
                        if (!mbar_wait(smem_u32(&H.full_b[g & 1u]), (g >> 1) & 1u, abort)) {
                            ok = false;
                            break;
                        }
                        clean = H.tile_clean[g & 1u];
                        tpi = H.tile_piece[g & 1u];
                    }
                    // the warp's 128 columns in two packed loads; the accumulator is
                    // handed back to the MMAs as soon as they are in registers, so
                    // the tests and hits below overlap the next MMAs into it
                    const uint32_t tbase = tmem + ((32u * quarter) << 16) + a * kTcN + half * (kTcN / 2);
                    uint32_t ra[32], rb[32];
                    tc_ld64h(tbase, ra);
                    tc_ld64h(tbase + 64u, rb);
                    tc_wait_ld_regs(ra);
                    tc_wait_ld_regs(rb);
                    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                    __syncwarp();
                    if (lane == 0) mbar_arrive(smem_u32(&H.empty_acc[a]));
#pragma unroll
                    for (uint32_t c = 0; c < 2; c++) {
                        uint32_t *cur = c ? rb : ra;
                        const float mx = max64h(cur);
                        if (__any_sync(0xffffffffu, mx >= thr)) {
                            uint32_t *mine2 = reinterpret_cast<uint32_t *>(scratch) + ((warp - 2u) * 32u + lane) * 33u;
                            uint64_t bits = 0;
#pragma unroll
                            for (int j = 0; j < 32; j++) {
                                mine2[j] = cur[j];
                                const uint32_t m = __hge2_mask(*reinterpret_cast<const __half2 *>(&cur[j]), thr2);
                                bits |= static_cast<uint64_t>((m & 1u) | ((m >> 15) & 2u)) << (2 * j);
                            }
                            const uint64_t p0 = pt + ph + 4u * (half * (kTcN / 2) + 64u * c);
                            if (clean) {
                                // every window of the tile is valid and in one piece: emit
                                // the set bits only, the piece looked up once per tile
                                if (!have_piece) {
                                    tpc = b.pieces[tpi];
                                    have_piece = true;
                                }
                                const uint32_t rounds = __reduce_max_sync(0xffffffffu, __popcll(bits));
                                for (uint32_t r = 0; r < rounds; r++) {
                                    const bool has = bits != 0;
                                    const uint32_t col = has ? static_cast<uint32_t>(__ffsll(bits) - 1) : 0u;
                                    bits &= bits - 1;
                                    const __half2 v2 = *reinterpret_cast<const __half2 *>(&mine2[col >> 1]);
                                    const float mt_c = (col & 1u) ? __high2float(v2) : __low2float(v2);
                                    const uint32_t pos =
                                        static_cast<uint32_t>(tpc.contig_off + (p0 + 4u * col - tpc.start));
                                    wh.emit(sink, lane, has, id >> 1, tpc.contig, pos, id & 1u,
                                            L - static_cast<uint32_t>(mt_c), &H.discard);
                                    row_hits += has ? 1u : 0u;
                                }
                            } else {
                                emit_chunk(b, sink, wh, mine2, thr, L, id, p0, lane);
                            }
                        }
                    }
                }
                if (!ok) break;
            }
            if (row_hits && e < nent) atomicAdd(&sink.qcount[id >> 1], static_cast<unsigned long long>(row_hits));
        }
        gtile += ntiles;
        __syncthreads();
    }
    if (warp >= 2) wh.finish(sink, lane);
    if (threadIdx.x == 0 && H.abort) atomicOr(status, 1u);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem));
}

}  // namespace

uint32_t tc_lpad(uint32_t lmax) { return (lmax + 7u) & ~7u; }

bool tc_eligible(uint32_t lmax) { return lmax >= 1 && tc_lpad(lmax) <= kTcMaxLpad; }

// Q operand of the tensor-core scan: entry tiles of 128 rows x K = 4 lpad
// bytes in the K-major core-matrix order (8 rows x 16 B blocks; blocks along
// K 128 B apart, 8-row groups 8 K apart); row e is the one-hot e4m3 of the
// entry's bases (query, or its reverse complement for odd e), zero for N and
// past the query's end.
void tc_operand(const std::vector<std::string> &qs, uint32_t lpad, std::vector<uint8_t> &out) {
    const uint32_t K = 4u * lpad;
    const uint32_t ne = 2u * static_cast<uint32_t>(qs.size());
    const uint32_t ntile = (ne + kTcM - 1) / kTcM;
    out.assign(static_cast<size_t>(ntile) * kTcM * K, 0);
    for (uint32_t e = 0; e < ne; e++) {
        const std::string &q = qs[e >> 1];
        const uint32_t L = static_cast<uint32_t>(q.size());
        const size_t tile = static_cast<size_t>(e / kTcM) * kTcM * K;
        const uint32_t row = e % kTcM;
        for (uint32_t i = 0; i < L && i < lpad; i++) {
            const uint8_t ch = static_cast<uint8_t>((e & 1u) ? q[L - 1 - i] : q[i]);
            if (!is_base(ch)) continue;
            uint32_t code = base_code(ch);
            if (e & 1u) code ^= 2u;  // complement
            const uint32_t k = 4u * i + code;
            out[tile + (row / 8) * 8 * K + (k / 16) * 128 + (row % 8) * 16 + k % 16] = static_cast<uint8_t>(kOneE4M3);
        }
    }
}

namespace {
int g_tc_sms[64] = {0};   // per device: SMs, once the kernel's attributes are set
}

cudaError_t tc_prepare() {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || g_tc_sms[dev & 63]) return e;
    e = cudaFuncSetAttribute(k_scan_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(kTcSmem));
    if (e != cudaSuccess) return e;
    return cudaDeviceGetAttribute(&g_tc_sms[dev & 63], cudaDevAttrMultiProcessorCount, dev);
}

cudaError_t launch_scan_tc(const Batch &b, const uint8_t *tcA, const uint32_t *meta, uint32_t nent, uint32_t lpad,
                           uint32_t s, const HitSink &sink, unsigned int *status, cudaStream_t st,
                           uint32_t withhold_first, const uint32_t *ids) {
    // status[0]: wait gave up (bit 0); status[1]: the launch's work counter
    if (nent == 0 || b.nbases == 0) return cudaSuccess;
    if (lpad == 0 || lpad > kTcMaxLpad || (lpad & 7u)) return cudaErrorInvalidValue;
    cudaError_t pe = tc_prepare();
    if (pe != cudaSuccess) return pe;
    int dev = 0;
    cudaGetDevice(&dev);
    const uint32_t grid_max = static_cast<uint32_t>(g_tc_sms[dev & 63]);
    const uint32_t n_mt = (nent + kTcM - 1) / kTcM;
    const uint32_t n_rt = static_cast<uint32_t>((b.nbases + kTcTile - 1) / kTcTile);
    // about 24 items per CTA, each a run of reference tiles for one entry tile,
    // taken from a counter so that uneven items even out
    const uint64_t want = static_cast<uint64_t>(grid_max) * 24u;
    uint64_t per = (static_cast<uint64_t>(n_mt) * n_rt + want - 1) / want;
    if (per < 1) per = 1;
    if (per > n_rt) per = n_rt;
    const uint32_t rt_per_item = static_cast<uint32_t>(per);
    const uint32_t n_rchunks = (n_rt + rt_per_item - 1) / rt_per_item;
    const uint32_t n_items = n_mt * n_rchunks;
    const uint32_t grid = n_items < grid_max ? n_items : grid_max;
    cudaError_t e = cudaMemsetAsync(status + 1, 0, sizeof(unsigned int), st);
    if (e != cudaSuccess) return e;
    k_scan_tc<<<grid, kTcThreads, kTcSmem, st>>>(b, tcA, meta, ids, nent, lpad, s, n_rt, rt_per_item, n_rchunks,
                                                 n_items, sink, status, status + 1, withhold_first);
    return cudaGetLastError();
}

}  // namespace ifa

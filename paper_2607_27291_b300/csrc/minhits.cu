// minhits.cu -- MinHitsCalculator on the device (Methods, indexed mode).
//
// For a bin (query length L, substitutions s, seed length k) the paper
// estimates by Monte Carlo the smallest number of error-free seed k-mers a
// true alignment still shows with probability P, and switches to the
// deterministic bound validKmers - kEffective * maxSubs - maxClips at
// P = 100%.  Every trial here is one thread:
//   1. draw s distinct positions of [0, L) by a partial Fisher-Yates shuffle
//      whose uniform draws come from Philox4x32-10 words (Salmon et al.,
//      SC'11) mapped to [0, m) by Lemire's multiply-shift with rejection;
//   2. count the k-mer offsets (0, step, 2 step, ...) whose unmasked
//      positions hold none of the drawn positions;
//   3. add one to that bin's histogram cell.
// A second kernel turns each histogram into the threshold: the largest m
// with #{trials with >= m survivors} * den >= num * trials.
//
// Trial t of a bin uses counter (t, block, L | s<<8 | k<<16 | mask<<24,
// step) and key (seed low, seed high), consuming each block's four words in
// order, so the thresholds are a pure function of the bin and the seed.
#include "ifa_internal.cuh"

namespace ifa {

namespace {

struct Philox {
    uint32_t c[4];
    uint32_t k[2];
    uint32_t w[4];
    int used;

    __device__ void block() {
        uint32_t c0 = c[0], c1 = c[1], c2 = c[2], c3 = c[3];
        uint32_t k0 = k[0], k1 = k[1];
#pragma unroll
        for (int r = 0; r < 10; r++) {
            const uint32_t m0 = 0xD2511F53u, m1 = 0xCD9E8D57u;
            const uint32_t h0 = __umulhi(m0, c0), l0 = m0 * c0;
            const uint32_t h1 = __umulhi(m1, c2), l1 = m1 * c2;
            c0 = h1 ^ c1 ^ k0;
            c1 = l1;
            c2 = h0 ^ c3 ^ k1;
            c3 = l0;
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        w[0] = c0; w[1] = c1; w[2] = c2; w[3] = c3;
    }
    __device__ uint32_t next() {
        if (used == 4) {
            block();
            c[1]++;
            used = 0;
        }
        return w[used++];
    }
    // uniform in [0, m), m >= 1 (Lemire 2019, multiply-shift with rejection)
    __device__ uint32_t below(uint32_t m) {
        uint64_t prod = static_cast<uint64_t>(next()) * m;
        uint32_t low = static_cast<uint32_t>(prod);
        if (low < m) {
            const uint32_t thresh = (0u - m) % m;
            while (low < thresh) {
                prod = static_cast<uint64_t>(next()) * m;
                low = static_cast<uint32_t>(prod);
            }
        }
        return static_cast<uint32_t>(prod >> 32);
    }
};

__device__ inline uint32_t n_offsets(uint32_t L, uint32_t k, uint32_t step) {
    return (k == 0 || k > L || step == 0) ? 0u : (L - k) / step + 1;
}

// bits [o, o+64) of a 256-bit mask held as four words
__device__ inline uint64_t bits64(const uint64_t m[5], uint32_t o) {
    const uint32_t wi = o >> 6, sh = o & 63;
    return sh ? (m[wi] >> sh) | (m[wi + 1] << (64 - sh)) : m[wi];
}

__global__ void __launch_bounds__(256)
k_minhits_trials(const uint32_t *__restrict__ dL, const uint32_t *__restrict__ dsubs,
                 const uint32_t *__restrict__ dk, uint32_t step, uint32_t mask_w, uint32_t trials,
                 uint64_t seed, uint32_t *__restrict__ hist, uint32_t stride) {
    const uint32_t bin = blockIdx.y;
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= trials) return;
    const uint32_t L = dL[bin], s = dsubs[bin], k = dk[bin];
    const uint32_t K = n_offsets(L, k, step);
    if (K == 0) return;
    Philox ph;
    ph.c[0] = t;
    ph.c[1] = 0;
    ph.c[2] = (L & 0xffu) | ((s & 0xffu) << 8) | ((k & 0xffu) << 16) | ((mask_w & 0xffu) << 24);
    ph.c[3] = step;
    ph.k[0] = static_cast<uint32_t>(seed);
    ph.k[1] = static_cast<uint32_t>(seed >> 32);
    ph.used = 4;
    uint8_t perm[256];
    for (uint32_t i = 0; i < L; i++) perm[i] = static_cast<uint8_t>(i);
    uint64_t drawn[5] = {0, 0, 0, 0, 0};
    const uint32_t ns = s < L ? s : L;
    for (uint32_t i = 0; i < ns; i++) {
        const uint32_t j = i + ph.below(L - i);
        const uint8_t tmp = perm[i];
        perm[i] = perm[j];
        perm[j] = tmp;
        drawn[perm[i] >> 6] |= 1ull << (perm[i] & 63);
    }
    // positions of a k-mer that count: all k minus the centred mask
    const uint64_t kmask = (k >= 64 ? ~0ull : ((1ull << k) - 1));
    const uint32_t mlo = (k - mask_w) / 2;
    const uint64_t mmask = mask_w ? (((1ull << mask_w) - 1) << mlo) : 0ull;
    const uint64_t care = kmask & ~mmask;
    uint32_t surv = 0;
    for (uint32_t o = 0; o + k <= L; o += step) surv += (bits64(drawn, o) & care) == 0ull;
    atomicAdd(&hist[static_cast<size_t>(bin) * stride + surv], 1u);
}

__global__ void k_minhits_threshold(const uint32_t *__restrict__ dL, const uint32_t *__restrict__ dsubs,
                                    const uint32_t *__restrict__ dk, uint32_t nbins, uint32_t step,
                                    uint32_t mask_w, uint32_t max_clips, uint32_t num, uint32_t den,
                                    uint32_t trials, const uint32_t *__restrict__ hist,
                                    uint32_t stride, uint32_t *__restrict__ out) {
    const uint32_t bin = blockIdx.x * blockDim.x + threadIdx.x;
    if (bin >= nbins) return;
    const uint32_t L = dL[bin], s = dsubs[bin], k = dk[bin];
    const uint32_t K = n_offsets(L, k, step);
    if (K == 0) {
        out[bin] = 0;
        return;
    }
    if (num >= den) {  // P = 100%: deterministic bound
        const int64_t v = static_cast<int64_t>(K) - static_cast<int64_t>(k - mask_w) * s -
                          static_cast<int64_t>(max_clips);
        out[bin] = v > 0 ? static_cast<uint32_t>(v) : 0u;
        return;
    }
    // need: tail * den >= num * trials, compared as 128-bit products
    const uint64_t need_lo = static_cast<uint64_t>(num) * trials;  // < 2^64
    uint64_t tail = 0;
    uint32_t best = 0;
    for (int64_t m = K; m >= 0; m--) {
        tail += hist[static_cast<size_t>(bin) * stride + m];
        const uint64_t lo = tail * den;
        const uint64_t hi = __umul64hi(tail, static_cast<uint64_t>(den));
        if (hi > 0 || lo >= need_lo) {
            best = static_cast<uint32_t>(m);
            break;
        }
    }
    out[bin] = best;
}

}  // namespace

cudaError_t launch_minhits(const uint32_t *dL, const uint32_t *dsubs, const uint32_t *dk,
                           uint32_t nbins, uint32_t step, uint32_t mask_w, uint32_t max_clips,
                           uint32_t num, uint32_t den, uint32_t trials, uint64_t seed,
                           uint32_t *dhist, uint32_t stride, uint32_t *dout, cudaStream_t st) {
    if (nbins == 0) return cudaSuccess;
    if (num < den && trials > 0) {
        cudaError_t e = cudaMemsetAsync(dhist, 0, static_cast<size_t>(nbins) * stride * sizeof(uint32_t), st);
        if (e != cudaSuccess) return e;
        dim3 grid((trials + 255) / 256, nbins);
        k_minhits_trials<<<grid, 256, 0, st>>>(dL, dsubs, dk, step, mask_w, trials, seed, dhist, stride);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    k_minhits_threshold<<<(nbins + 127) / 128, 128, 0, st>>>(dL, dsubs, dk, nbins, step, mask_w,
                                                             max_clips, num, den, trials, dhist,
                                                             stride, dout);
    return cudaGetLastError();
}

}  // namespace ifa

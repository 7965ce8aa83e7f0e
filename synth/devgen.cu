// devgen.cu -- the device twin of synth.counter_bases: seeded synthetic
// reference bases generated straight into device memory, for references too
// large to stage from the host (200 Gbp).  Input generation only: nothing of
// the aligner's arithmetic is here.
//
// Base i (a position of the whole concatenated reference) is drawn from
// u = high 32 bits of mix(i + seed * 0x9E3779B97F4A7C15), mix being the
// splitmix64 output function (Steele, Lea, Flood, OOPSLA 2014): A if
// u < t1, C if u < t2, G if u < t3, else T, with t1 = floor((1 - gc) / 2 * 2^32),
// t2 = 2^31, t3 = floor((1 + gc) / 2 * 2^32) passed in.  N-runs are then
// written over the bases from a list of (start, length) runs.
#include <cstdint>
#include <cuda_runtime.h>

namespace {

__device__ __forceinline__ uint64_t splitmix_out(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// One thread writes 16 bases (one 16-byte store) at out + 16 t.
__global__ void k_bases(uint8_t *__restrict__ out, uint64_t first, uint64_t n, uint64_t key, uint32_t t1,
                        uint32_t t2, uint32_t t3) {
    const uint64_t t = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    const uint64_t o = t * 16;
    if (o >= n) return;
    uint32_t w[4] = {0, 0, 0, 0};
    const uint32_t cnt = n - o < 16 ? static_cast<uint32_t>(n - o) : 16u;
    for (uint32_t j = 0; j < 16; j++) {
        const uint32_t u = static_cast<uint32_t>(splitmix_out(first + o + j + key) >> 32);
        const uint32_t c = (u >= t1 ? 1u : 0u) + (u >= t2 ? 1u : 0u) + (u >= t3 ? 1u : 0u);
        const uint32_t b = c == 0 ? 'A' : c == 1 ? 'C' : c == 2 ? 'G' : 'T';
        w[j >> 2] |= b << (8 * (j & 3));
    }
    if (cnt == 16 && (reinterpret_cast<uintptr_t>(out + o) & 15u) == 0) {
        *reinterpret_cast<uint4 *>(out + o) = make_uint4(w[0], w[1], w[2], w[3]);
    } else {
        for (uint32_t j = 0; j < cnt; j++) out[o + j] = static_cast<uint8_t>(w[j >> 2] >> (8 * (j & 3)));
    }
}

// Runs (start, length) in whole-reference coordinates, clipped to
// [first, first + n): one block per run.
__global__ void k_runs(uint8_t *__restrict__ out, uint64_t first, uint64_t n, const uint64_t *__restrict__ rs,
                       const uint32_t *__restrict__ rl, uint32_t nruns) {
    const uint32_t r = blockIdx.x;
    if (r >= nruns) return;
    const uint64_t a = rs[r], b = rs[r] + rl[r];
    const uint64_t lo = a > first ? a : first, hi = b < first + n ? b : first + n;
    for (uint64_t p = lo + threadIdx.x; p < hi; p += blockDim.x) out[p - first] = 'N';
}

}  // namespace

// Bases [first, first + n) of the reference into out (device, n bytes) on
// `stream`; runs (device arrays, nruns entries) are written as N where they
// overlap.  Returns a cudaError_t.
extern "C" int synth_dev_bases(uint8_t *out, uint64_t first, uint64_t n, uint64_t seed, uint32_t t1, uint32_t t2,
                               uint32_t t3, const uint64_t *run_start, const uint32_t *run_len, uint32_t nruns,
                               void *stream) {
    if (n == 0) return 0;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const uint64_t threads = (n + 15) / 16;
    const uint64_t key = seed * 0x9E3779B97F4A7C15ull;
    k_bases<<<static_cast<unsigned>((threads + 255) / 256), 256, 0, st>>>(out, first, n, key, t1, t2, t3);
    if (nruns) k_runs<<<nruns, 256, 0, st>>>(out, first, n, run_start, run_len, nruns);
    return static_cast<int>(cudaGetLastError());
}

// pipe_rates.cu -- issue-rate microbenchmark of the integer pipes the scan
// kernels use (population count, three-input logic, funnel shift, integer
// multiply-add), per SM per clock.
//
// Not part of the aligner: a measurement tool, built into its own library
// (libifa_probe.so) and called by the benchmark, whose roofline for the
// brute-force scan is SMs x (measured POPC results per SM per clock) x the
// SM clock sampled during the timed region.
//
// Method.  Every thread runs kChains independent dependency chains of one
// instruction kind, unrolled kUnroll times per loop trip, so that enough
// independent instructions are in flight on every scheduler to hide the
// pipe's latency.  Each chain step takes fresh operands from a rotating set
// of registers loaded from memory, so that ptxas can neither fold two steps
// into one instruction (two three-input logic steps over five inputs are not
// one LOP3) nor evaluate them at compile time.  Each block records its SM
// (%smid) and clock64() at start and end; the rate on an SM is the
// instructions its blocks issued divided by the clock cycles between its
// first start and its last end, so the result is per clock, independent of
// the clock frequency.  The CUDA-event duration and the cycles give the SM
// clock as well.
#include <cstdint>
#include <cstring>
#include <cuda_runtime.h>
#include <vector>
#include <algorithm>

namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 16;
constexpr int kThreads = 256;

enum Kind { kPopc = 0, kLop3 = 1, kShf = 2, kImad = 3, kKinds = 4 };

template <int K>
__device__ __forceinline__ uint32_t step(uint32_t a, uint32_t b, uint32_t c) {
    uint32_t d;
    if constexpr (K == kPopc) {
        asm volatile("popc.b32 %0, %1;" : "=r"(d) : "r"(a));
    } else if constexpr (K == kLop3) {
        asm volatile("lop3.b32 %0, %1, %2, %3, 0xE8;" : "=r"(d) : "r"(a), "r"(b), "r"(c));  // majority
    } else if constexpr (K == kShf) {
        asm volatile("shf.r.wrap.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    } else {
        asm volatile("mad.lo.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    }
    return d;
}

template <int K>
__global__ void __launch_bounds__(kThreads) k_pipe(const uint32_t *__restrict__ in, uint64_t trips,
                                                   uint32_t *__restrict__ out, unsigned long long *__restrict__ clk,
                                                   uint32_t *__restrict__ smid) {
    uint32_t x[kChains], r[8];
#pragma unroll
    for (int i = 0; i < kChains; i++) x[i] = in[(threadIdx.x + i) & 63];
#pragma unroll
    for (int i = 0; i < 8; i++) r[i] = in[64 + ((threadIdx.x * 3 + i) & 63)];
    __syncthreads();
    const unsigned long long t0 = clock64();
    for (uint64_t t = 0; t < trips; t++) {
#pragma unroll
        for (int u = 0; u < kUnroll; u++) {
#pragma unroll
            for (int i = 0; i < kChains; i++) x[i] = step<K>(x[i], r[(u + i) & 7], r[(u + 3 * i + 1) & 7]);
        }
    }
    __syncthreads();
    const unsigned long long t1 = clock64();
    uint32_t acc = 0;
#pragma unroll
    for (int i = 0; i < kChains; i++) acc ^= x[i];
    out[blockIdx.x * blockDim.x + threadIdx.x] = acc;
    if (threadIdx.x == 0) {
        clk[2 * blockIdx.x] = t0;
        clk[2 * blockIdx.x + 1] = t1;
        uint32_t s;
        asm volatile("mov.u32 %0, %%smid;" : "=r"(s));
        smid[blockIdx.x] = s;
    }
}

template <int K>
cudaError_t launch(int grid, const uint32_t *in, uint64_t trips, uint32_t *out, unsigned long long *clk,
                   uint32_t *smid, cudaStream_t st) {
    k_pipe<K><<<grid, kThreads, 0, st>>>(in, trips, out, clk, smid);
    return cudaGetLastError();
}

// Random gathers: every thread loads `per_thread` 32-bit words at
// independent pseudo-random offsets (a multiplicative hash of its index) of
// a table of `words` words, summing them so that no load is dead.  The rate
// of such loads bounds a table lookup per reference position (the seed
// scan's k-mer offsets).
__global__ void __launch_bounds__(256) k_gather(const uint32_t *__restrict__ table, uint64_t words,
                                                uint32_t per_thread, uint32_t *__restrict__ out) {
    const uint64_t t = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    uint32_t acc = 0;
    uint64_t x = t * 0x9E3779B97F4A7C15ull + 1;
    for (uint32_t i = 0; i < per_thread; i++) {
        x = x * 6364136223846793005ull + 1442695040888963407ull;   // Knuth's MMIX LCG step
        acc += __ldg(table + ((x >> 20) % words));
    }
    out[t] = acc;
}

}  // namespace

// Random 32-bit gathers per second from a device table of `table_bytes`
// (filled once), `per_thread` loads per thread over a grid of 148 x 8
// blocks; outputs the rate (loads/s) and the kernel's event time.
extern "C" int ifa_probe_gather_rate(int device, uint64_t table_bytes, uint32_t per_thread, double *loads_per_s,
                                     double *ms) {
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) return e;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    const uint64_t words = table_bytes / 4;
    if (words == 0 || per_thread == 0) return 1;
    const int grid = sms * 8;
    uint32_t *table = nullptr, *out = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    e = cudaMalloc(&table, words * 4);
    if (e == cudaSuccess) e = cudaMalloc(&out, static_cast<size_t>(grid) * 256 * 4);
    if (e == cudaSuccess) e = cudaMemset(table, 1, words * 4);
    if (e == cudaSuccess) e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    if (e == cudaSuccess) {
        k_gather<<<grid, 256>>>(table, words, per_thread < 64 ? per_thread : 64, out);  // warm-up
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(a);
    if (e == cudaSuccess) {
        k_gather<<<grid, 256>>>(table, words, per_thread, out);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(b);
    if (e == cudaSuccess) e = cudaEventSynchronize(b);
    float t = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, a, b);
    if (e == cudaSuccess) {
        *ms = t;
        *loads_per_s = static_cast<double>(grid) * 256.0 * per_thread / (t * 1e-3);
    }
    cudaFree(table);
    cudaFree(out);
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    return e;
}

// Measure one instruction kind (0 popc, 1 lop3, 2 shf, 3 imad) with
// `blocks_per_sm` resident blocks of 256 threads on every SM for `trips`
// loop trips (each trip is 16 x 8 instructions per thread).  Outputs: the
// median over SMs of instructions per SM per clock (thread-level results,
// so a pipe that completes one warp instruction per clock counts 32), the
// kernel's CUDA-event time in ms, and the mean SM clock in MHz (cycles of
// the busiest SM divided by that time).  Returns 0, or a cudaError_t.
extern "C" int ifa_probe_pipe_rate(int device, int kind, int blocks_per_sm, uint64_t trips,
                                   double *per_clk_sm, double *ms, double *sm_mhz) {
    if (kind < 0 || kind >= kKinds || blocks_per_sm < 1 || blocks_per_sm > 8 || trips == 0) return 1;
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) return e;
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    if (e != cudaSuccess) return e;
    const int grid = sms * blocks_per_sm;
    uint32_t *in = nullptr, *out = nullptr, *smid = nullptr;
    unsigned long long *clk = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    std::vector<uint32_t> hin(128);
    for (int i = 0; i < 128; i++) hin[i] = 0x9E3779B9u * (i + 1) ^ (0x7F4A7C15u >> (i & 7));
    auto cleanup = [&]() {
        cudaFree(in);
        cudaFree(out);
        cudaFree(smid);
        cudaFree(clk);
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
    };
#define PCK(x)                     \
    do {                           \
        e = (x);                   \
        if (e != cudaSuccess) {    \
            cleanup();             \
            return e;              \
        }                          \
    } while (0)
    PCK(cudaMalloc(&in, 128 * sizeof(uint32_t)));
    PCK(cudaMalloc(&out, static_cast<size_t>(grid) * kThreads * sizeof(uint32_t)));
    PCK(cudaMalloc(&smid, grid * sizeof(uint32_t)));
    PCK(cudaMalloc(&clk, 2 * static_cast<size_t>(grid) * sizeof(unsigned long long)));
    PCK(cudaMemcpy(in, hin.data(), 128 * sizeof(uint32_t), cudaMemcpyHostToDevice));
    PCK(cudaEventCreate(&a));
    PCK(cudaEventCreate(&b));
    auto run = [&](uint64_t t) -> cudaError_t {
        switch (kind) {
        case kPopc: return launch<kPopc>(grid, in, t, out, clk, smid, nullptr);
        case kLop3: return launch<kLop3>(grid, in, t, out, clk, smid, nullptr);
        case kShf: return launch<kShf>(grid, in, t, out, clk, smid, nullptr);
        default: return launch<kImad>(grid, in, t, out, clk, smid, nullptr);
        }
    };
    PCK(run(trips < 16 ? trips : 16));  // warm-up
    PCK(cudaDeviceSynchronize());
    PCK(cudaEventRecord(a));
    PCK(run(trips));
    PCK(cudaEventRecord(b));
    PCK(cudaEventSynchronize(b));
    float t_ms = 0.f;
    PCK(cudaEventElapsedTime(&t_ms, a, b));
    std::vector<unsigned long long> hc(2 * static_cast<size_t>(grid));
    std::vector<uint32_t> hs(grid);
    PCK(cudaMemcpy(hc.data(), clk, hc.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost));
    PCK(cudaMemcpy(hs.data(), smid, hs.size() * sizeof(uint32_t), cudaMemcpyDeviceToHost));
    cleanup();
#undef PCK
    // per SM: blocks, first start, last end
    std::vector<double> nblk(1024, 0.0);
    std::vector<unsigned long long> lo(1024, ~0ull), hi(1024, 0ull);
    for (int i = 0; i < grid; i++) {
        const uint32_t s = hs[i] & 1023u;
        nblk[s] += 1.0;
        lo[s] = std::min(lo[s], hc[2 * i]);
        hi[s] = std::max(hi[s], hc[2 * i + 1]);
    }
    const double per_block = static_cast<double>(kThreads) * kChains * kUnroll * static_cast<double>(trips);
    std::vector<double> rates;
    unsigned long long busiest = 0;
    for (int s = 0; s < 1024; s++)
        if (nblk[s] > 0 && hi[s] > lo[s]) {
            rates.push_back(nblk[s] * per_block / static_cast<double>(hi[s] - lo[s]));
            busiest = std::max(busiest, hi[s] - lo[s]);
        }
    if (rates.empty()) return 1;
    std::sort(rates.begin(), rates.end());
    *per_clk_sm = rates[rates.size() / 2];
    *ms = t_ms;
    *sm_mhz = t_ms > 0.f ? static_cast<double>(busiest) / (t_ms * 1e3) : 0.0;
    return 0;
}

// Pinned host <-> device copy rate with cudaMemcpyAsync (the call the
// library streams segments with): `bytes` per copy between cudaHostAlloc
// memory and device memory, to_device selecting the direction; outputs the
// best of `reps` single copies and the rate of `reps` copies back to back on
// one stream, in GB/s.
extern "C" int ifa_probe_copy_rate(int device, uint64_t bytes, int to_device, int reps, double *best_gbps,
                                   double *b2b_gbps) {
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) return e;
    if (bytes == 0 || reps < 1) return 1;
    void *hbuf = nullptr, *dbuf = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    e = cudaHostAlloc(&hbuf, bytes, cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaMalloc(&dbuf, bytes);
    if (e == cudaSuccess) e = cudaMemset(dbuf, 0, bytes);
    if (e == cudaSuccess) std::memset(hbuf, 1, bytes);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    const cudaMemcpyKind kind = to_device ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToHost;
    void *dst = to_device ? dbuf : hbuf;
    const void *src = to_device ? hbuf : dbuf;
    float best = 1e30f, t = 0.f;
    for (int i = 0; i <= reps && e == cudaSuccess; i++) {  // the first copy is a warm-up
        e = cudaEventRecord(a, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dst, src, bytes, kind, st);
        if (e == cudaSuccess) e = cudaEventRecord(b, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(b);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, a, b);
        if (e == cudaSuccess && i > 0 && t < best) best = t;
    }
    if (e == cudaSuccess) e = cudaEventRecord(a, st);
    for (int i = 0; i < reps && e == cudaSuccess; i++) e = cudaMemcpyAsync(dst, src, bytes, kind, st);
    if (e == cudaSuccess) e = cudaEventRecord(b, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(b);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, a, b);
    if (e == cudaSuccess) {
        *best_gbps = static_cast<double>(bytes) / (best * 1e-3) / 1e9;
        *b2b_gbps = static_cast<double>(bytes) * reps / (t * 1e-3) / 1e9;
    }
    cudaFreeHost(hbuf);
    cudaFree(dbuf);
    if (st) cudaStreamDestroy(st);
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    return e;
}

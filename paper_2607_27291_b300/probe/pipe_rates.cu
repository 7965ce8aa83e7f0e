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

}  // namespace

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

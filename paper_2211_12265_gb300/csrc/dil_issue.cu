// Test-only probes.  dil_test_issue_rate: sustained rate of one integer
// instruction class, in thread-operations per SM clock, over independent
// dependency chains at full occupancy.  dil_test_keccak_rate: SM clocks per
// state per round of the four Keccak-f[1600] forms the kernels use, 32 warps
// per SM.
//
// Timing: every block records its SM (%smid) and clock64() after a barrier
// at its start and end; an SM's time is the span from the first start to the
// last end of the blocks it ran (clock64 counts that SM's clock), and its work
// is the sum of theirs.  Blocks of one SM need not run at the same time, so a
// block's own window is not the SM's time.
#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <vector>

#include "dil_keccak16.cuh"
#include "dil_keccak6.cuh"
#include "dil_launch.h"

namespace dil {

constexpr int PROBE_ITERS = 4096;

__device__ __forceinline__ unsigned sm_id() {
    unsigned id;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(id));
    return id;
}

// rec: 3 entries per block (SM id, start clock, end clock)
__device__ __forceinline__ void record(long long *rec, long long t0, long long t1) {
    if (threadIdx.x == 0) {
        rec[3 * blockIdx.x] = sm_id();
        rec[3 * blockIdx.x + 1] = t0;
        rec[3 * blockIdx.x + 2] = t1;
    }
}

// Per-SM work / per-SM span (first start to last end), averaged over SMs;
// work_per_block in the caller's unit.
double per_sm_rate(const std::vector<long long> &rec, int blocks, double work_per_block) {
    std::map<long long, std::pair<long long, long long>> span;
    std::map<long long, int> count;
    for (int b = 0; b < blocks; ++b) {
        const long long sm = rec[3 * b], t0 = rec[3 * b + 1], t1 = rec[3 * b + 2];
        auto it = span.find(sm);
        if (it == span.end()) {
            span[sm] = {t0, t1};
        } else {
            it->second.first = std::min(it->second.first, t0);
            it->second.second = std::max(it->second.second, t1);
        }
        ++count[sm];
    }
    double sum = 0;
    for (auto &kv : span) sum += count[kv.first] * work_per_block / (double)(kv.second.second - kv.second.first);
    return span.empty() ? 0.0 : sum / span.size();
}

template <int OP>
__device__ __forceinline__ uint32_t probe_op(uint32_t a, uint32_t b, uint32_t c) {
    uint32_t r;
    if (OP == 0) asm volatile("lop3.b32 %0, %1, %2, %3, 0x96;" : "=r"(r) : "r"(a), "r"(b), "r"(c));
    if (OP == 1) asm volatile("shf.l.wrap.b32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "r"(c));
    if (OP == 2) asm volatile("mul.lo.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
    if (OP == 3) asm volatile("mul.hi.s32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
    if (OP == 4) r = __shfl_sync(0xffffffffu, a, b & 31);
    return r;
}

template <int OP>
__global__ void __launch_bounds__(1024) k_probe(uint32_t *out, long long *cyc) {
    uint32_t a0 = threadIdx.x, a1 = a0 * 3 + 1, a2 = a0 * 5 + 2, a3 = a0 * 7 + 3;
    uint32_t a4 = a0 ^ 9, a5 = a0 + 11, a6 = a0 * 13, a7 = a0 + 17, c = blockIdx.x | 1;
    __syncthreads();
    long long t0 = clock64();
#pragma unroll 4
    for (int i = 0; i < PROBE_ITERS; ++i) {
        a0 = probe_op<OP>(a0, a1, c); a1 = probe_op<OP>(a1, a2, c);
        a2 = probe_op<OP>(a2, a3, c); a3 = probe_op<OP>(a3, a4, c);
        a4 = probe_op<OP>(a4, a5, c); a5 = probe_op<OP>(a5, a6, c);
        a6 = probe_op<OP>(a6, a7, c); a7 = probe_op<OP>(a7, a0, c);
    }
    __syncthreads();
    long long t1 = clock64();
    record(cyc, t0, t1);
    out[blockIdx.x * blockDim.x + threadIdx.x] = a0 ^ a1 ^ a2 ^ a3 ^ a4 ^ a5 ^ a6 ^ a7;
}

cudaError_t measure_issue_rate(int op, double *rate) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int blocks = 2 * sms, threads = 1024;   // two resident 1024-thread blocks per SM
    uint32_t *out = nullptr;
    long long *cyc = nullptr;
    cudaError_t e = cudaMalloc(&out, (size_t)blocks * threads * 4);
    if (e != cudaSuccess) return e;
    e = cudaMalloc(&cyc, (size_t)blocks * 3 * 8);
    if (e != cudaSuccess) {
        cudaFree(out);
        return e;
    }
    for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {
        switch (op) {
            case 0: k_probe<0><<<blocks, threads>>>(out, cyc); break;
            case 1: k_probe<1><<<blocks, threads>>>(out, cyc); break;
            case 2: k_probe<2><<<blocks, threads>>>(out, cyc); break;
            case 3: k_probe<3><<<blocks, threads>>>(out, cyc); break;
            default: k_probe<4><<<blocks, threads>>>(out, cyc); break;
        }
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
    }
    std::vector<long long> h(3 * (size_t)blocks);
    if (e == cudaSuccess) e = cudaMemcpy(h.data(), cyc, (size_t)blocks * 3 * 8, cudaMemcpyDeviceToHost);
    cudaFree(out);
    cudaFree(cyc);
    if (e != cudaSuccess) return e;
    *rate = per_sm_rate(h, blocks, (double)threads * PROBE_ITERS * 8);
    return cudaSuccess;
}

constexpr int KPROBE_PERMS = 64;
constexpr int KPROBE_WARPS = 8;
constexpr int KPROBE_CTAS_PER_SM = 4;

// Every warp permutes its FORM states (1: 25-lane form, 2: two interleaved
// states, 6: six-state row form, 16: two-thread-per-state form)
// KPROBE_PERMS times.
template <int FORM>
__global__ void __launch_bounds__(KPROBE_WARPS * 32, KPROBE_CTAS_PER_SM) k_keccak_probe(uint32_t *out,
                                                                                       long long *cyc) {
    __shared__ __align__(16) uint32_t sm[KPROBE_WARPS][K16_WORDS];   // six states + exchange, or sixteen states
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint32_t *kst = sm[warp], *kpi = kst + K6_STATES * K6_WORDS;
    uint32_t lo = lane * 0x9E3779B9u + blockIdx.x, hi = lo ^ 0x5BD1E995u, lo1 = lo + 1, hi1 = hi + 1;
    if (FORM == 6 || FORM == 16) {
        for (int w = lane; w < K16_WORDS; w += 32) kst[w] = w * 2654435761u + blockIdx.x;
    }
    __syncthreads();
    const long long t0 = clock64();
    for (int i = 0; i < KPROBE_PERMS; ++i) {
        if (FORM == 1) keccak_f(lo, hi);
        if (FORM == 2) keccak_f2(lo, hi, lo1, hi1);
        if (FORM == 6) keccak6_permute(kst, kpi);
        if (FORM == 16) keccak16_permute(kst);
    }
    __syncthreads();
    const long long t1 = clock64();
    record(cyc, t0, t1);
    out[blockIdx.x * blockDim.x + threadIdx.x] = lo ^ hi ^ lo1 ^ hi1 ^ (FORM >= 6 ? kst[lane] : 0u);
}

cudaError_t measure_keccak_rate(int form, double *clk_per_state_round) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int blocks = KPROBE_CTAS_PER_SM * sms, threads = KPROBE_WARPS * 32;
    uint32_t *out = nullptr;
    long long *cyc = nullptr;
    cudaError_t e = cudaMalloc(&out, (size_t)blocks * threads * 4);
    if (e != cudaSuccess) return e;
    e = cudaMalloc(&cyc, (size_t)blocks * 3 * 8);
    if (e != cudaSuccess) {
        cudaFree(out);
        return e;
    }
    for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {
        if (form == 1) k_keccak_probe<1><<<blocks, threads>>>(out, cyc);
        if (form == 2) k_keccak_probe<2><<<blocks, threads>>>(out, cyc);
        if (form == 6) k_keccak_probe<6><<<blocks, threads>>>(out, cyc);
        if (form == 16) k_keccak_probe<16><<<blocks, threads>>>(out, cyc);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
    }
    std::vector<long long> h(3 * (size_t)blocks);
    if (e == cudaSuccess) e = cudaMemcpy(h.data(), cyc, (size_t)blocks * 3 * 8, cudaMemcpyDeviceToHost);
    cudaFree(out);
    cudaFree(cyc);
    if (e != cudaSuccess) return e;
    // state-rounds per SM clock, inverted
    const double rate = per_sm_rate(h, blocks, (double)KPROBE_WARPS * form * KPROBE_PERMS * 24);
    *clk_per_state_round = rate > 0 ? 1.0 / rate : 0.0;
    return cudaSuccess;
}

}  // namespace dil

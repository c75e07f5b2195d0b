// Plain one-launch-per-batch kernels (section 4.2 single-warp fusion): one warp
// runs one whole Gen, Sign or Verify task; a CTA holds `warps` tasks and shares
// the twiddle tables in shared memory.
#include "dil_launch.h"
#include "dil_procs.cuh"

namespace dil {

size_t cta_smem_bytes(int warps) { return CTA_TABLE_BYTES + (size_t)warps * sizeof(WarpSmem); }

template <int LEVEL>
static size_t polys_for(int op) {
    using S = Scratch<LEVEL>;
    return op == OP_KEYGEN ? S::GEN_POLYS : op == OP_SIGN ? S::SIGN_POLYS : S::VERIFY_POLYS;
}

size_t scratch_polys(int op, int level) {
    switch (level) {
        case 2: return polys_for<2>(op);
        case 3: return polys_for<3>(op);
        case 5: return polys_for<5>(op);
    }
    return 0;
}

#define DIL_CTA_PROLOGUE                                                          \
    extern __shared__ __align__(16) uint8_t smem[];                               \
    int32_t *zt = reinterpret_cast<int32_t *>(smem);                              \
    int32_t *izt = zt + 256;                                                      \
    WarpSmem *wsa = reinterpret_cast<WarpSmem *>(smem + CTA_TABLE_BYTES);         \
    load_zetas(zt, izt);                                                          \
    __syncthreads();                                                              \
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;                   \
    const int task = blockIdx.x * (blockDim.x >> 5) + warp;                       \
    if (task >= n) return;                                                        \
    WarpSmem &ws = wsa[warp];                                                     \
    const KLane k = klane_init(lane);

template <int LEVEL>
__global__ void __launch_bounds__(256) k_keygen(int n, const uint8_t *__restrict__ seeds, uint8_t *pk,
                                                uint8_t *sk, int32_t *scratch) {
    DIL_CTA_PROLOGUE
    using V = Lv<LEVEL>;
    gen_task<LEVEL>(seeds + (size_t)task * 32, pk + (size_t)task * V::PK, sk + (size_t)task * V::SK,
                    scratch + (size_t)task * Scratch<LEVEL>::GEN_POLYS * N, ws, zt, izt, k, lane);
}

template <int LEVEL>
__global__ void __launch_bounds__(256) k_sign(int n, const uint8_t *__restrict__ sk, const uint8_t *__restrict__ msg,
                                              const uint64_t *__restrict__ off, uint8_t *sig, int32_t *status,
                                              int32_t *iters, int32_t *scratch, int max_iter) {
    DIL_CTA_PROLOGUE
    using V = Lv<LEVEL>;
    int32_t *scr = scratch + (size_t)task * Scratch<LEVEL>::SIGN_POLYS * N;
    const uint64_t m0 = off[task], m1 = off[task + 1];
    sign_prepare<LEVEL>(sk + (size_t)task * V::SK, msg + m0, (size_t)(m1 - m0), scr, ws, zt, k, lane);
    int it = 0;
    bool ok = false;
    while (it < max_iter) {
        ok = sign_attempt<LEVEL>(it * V::L, scr, ws, zt, izt, k, lane);
        ++it;
        if (ok) break;
    }
    uint8_t *tsig = sig + (size_t)task * V::SIG;
    if (ok)
        sign_pack<LEVEL>(tsig, scr, ws, lane);
    else
        sign_zero<LEVEL>(tsig, lane);
    if (lane == 0) {
        if (status) status[task] = ok ? 0 : -5;
        if (iters) iters[task] = it;
    }
}

template <int LEVEL>
__global__ void __launch_bounds__(256) k_verify(int n, const uint8_t *__restrict__ pk,
                                                const uint8_t *__restrict__ msg, const uint64_t *__restrict__ off,
                                                const uint8_t *__restrict__ sig, uint8_t *ok, int32_t *scratch) {
    DIL_CTA_PROLOGUE
    using V = Lv<LEVEL>;
    const uint64_t m0 = off[task], m1 = off[task + 1];
    int r = verify_task<LEVEL>(pk + (size_t)task * V::PK, msg + m0, (size_t)(m1 - m0), sig + (size_t)task * V::SIG,
                               scratch + (size_t)task * Scratch<LEVEL>::VERIFY_POLYS * N, ws, zt, izt, k, lane);
    if (lane == 0) ok[task] = (uint8_t)r;
}

template <class Kern, class... Args>
static cudaError_t launch(Kern kern, int n, int warps, cudaStream_t s, Args... args) {
    if (n <= 0) return cudaSuccess;
    size_t smem = cta_smem_bytes(warps);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int grid = (n + warps - 1) / warps;
    kern<<<grid, warps * 32, smem, s>>>(n, args...);
    return cudaGetLastError();
}

cudaError_t launch_keygen(int level, int n, const uint8_t *seeds, uint8_t *pk, uint8_t *sk, int32_t *scratch,
                          int warps, cudaStream_t s) {
    switch (level) {
        case 2: return launch(k_keygen<2>, n, warps, s, seeds, pk, sk, scratch);
        case 3: return launch(k_keygen<3>, n, warps, s, seeds, pk, sk, scratch);
        case 5: return launch(k_keygen<5>, n, warps, s, seeds, pk, sk, scratch);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_sign(int level, int n, const uint8_t *sk, const uint8_t *msg, const uint64_t *off,
                        uint8_t *sig, int32_t *status, int32_t *iters, int32_t *scratch, int max_iter,
                        int warps, cudaStream_t s) {
    switch (level) {
        case 2: return launch(k_sign<2>, n, warps, s, sk, msg, off, sig, status, iters, scratch, max_iter);
        case 3: return launch(k_sign<3>, n, warps, s, sk, msg, off, sig, status, iters, scratch, max_iter);
        case 5: return launch(k_sign<5>, n, warps, s, sk, msg, off, sig, status, iters, scratch, max_iter);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_verify(int level, int n, const uint8_t *pk, const uint8_t *msg, const uint64_t *off,
                          const uint8_t *sig, uint8_t *ok, int32_t *scratch, int warps, cudaStream_t s) {
    switch (level) {
        case 2: return launch(k_verify<2>, n, warps, s, pk, msg, off, sig, ok, scratch);
        case 3: return launch(k_verify<3>, n, warps, s, pk, msg, off, sig, ok, scratch);
        case 5: return launch(k_verify<5>, n, warps, s, pk, msg, off, sig, ok, scratch);
    }
    return cudaErrorInvalidValue;
}

}  // namespace dil

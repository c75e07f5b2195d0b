// Shared prologue and launch helper of the plain one-launch-per-batch kernels
// (section 4.2 fusion: one kernel runs whole Gen, Sign or Verify tasks).  A CTA
// holds W warps = W / P task groups of P warps; the CTA shares the NTT twiddle
// tables in shared memory, each group its GroupSmem, each warp its WarpSmem.
#pragma once
#include "../../include/dil.h"
#include "dil_launch.h"
#include "dil_procs.cuh"

namespace dil {

__host__ __device__ constexpr size_t cta_bytes(int warps, int p) {
    return CTA_TABLE_BYTES + (size_t)(warps / p) * sizeof(GroupSmem) + (size_t)warps * sizeof(WarpSmem);
}

struct CtaView {
    int32_t *zt, *izt;
    GroupSmem *gs;
    WarpSmem *ws;
    int g, bar, lane, group, groups;
};

// Carves the dynamic shared memory, loads the twiddles (whole CTA) and locates
// this warp's group.
template <int P>
__device__ __forceinline__ CtaView cta_setup(uint8_t *smem) {
    CtaView v;
    const int warps = blockDim.x >> 5;
    v.groups = warps / P;
    v.zt = reinterpret_cast<int32_t *>(smem);
    v.izt = v.zt + 256;
    GroupSmem *gsa = reinterpret_cast<GroupSmem *>(smem + CTA_TABLE_BYTES);
    WarpSmem *wsa = reinterpret_cast<WarpSmem *>(smem + CTA_TABLE_BYTES + v.groups * sizeof(GroupSmem));
    load_zetas(v.zt, v.izt);
    __syncthreads();
    const int warp = threadIdx.x >> 5;
    v.lane = threadIdx.x & 31;
    v.group = warp / P;
    v.g = warp % P;
    v.bar = 1 + v.group;   // named barrier 0 is __syncthreads
    v.gs = gsa + v.group;
    v.ws = wsa + warp;
    return v;
}

template <class Kern, class... Args>
static cudaError_t launch_plain(Kern kern, int n, int warps, int p, cudaStream_t s, Args... args) {
    if (n <= 0) return cudaSuccess;
    const size_t smem = cta_bytes(warps, p);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int groups = warps / p;
    kern<<<(n + groups - 1) / groups, warps * 32, smem, s>>>(n, args...);
    return cudaGetLastError();
}

// Dispatch on (level, warps per task) to kernel template K<LEVEL, P>.
#define DIL_DISPATCH(KERN, ...)                                                                  \
    switch (level * 10 + p) {                                                                    \
        case 21: return launch_plain(KERN<2, 1>, n, warps, p, s, __VA_ARGS__);                   \
        case 22: return launch_plain(KERN<2, 2>, n, warps, p, s, __VA_ARGS__);                   \
        case 24: return launch_plain(KERN<2, 4>, n, warps, p, s, __VA_ARGS__);                   \
        case 31: return launch_plain(KERN<3, 1>, n, warps, p, s, __VA_ARGS__);                   \
        case 32: return launch_plain(KERN<3, 2>, n, warps, p, s, __VA_ARGS__);                   \
        case 34: return launch_plain(KERN<3, 4>, n, warps, p, s, __VA_ARGS__);                   \
        case 51: return launch_plain(KERN<5, 1>, n, warps, p, s, __VA_ARGS__);                   \
        case 52: return launch_plain(KERN<5, 2>, n, warps, p, s, __VA_ARGS__);                   \
        case 54: return launch_plain(KERN<5, 4>, n, warps, p, s, __VA_ARGS__);                   \
    }                                                                                            \
    return cudaErrorInvalidValue;

}  // namespace dil

// dil_sign_noalloc: Sign without any device allocation.
//
// Some callers cannot call cudaMalloc when they sign: a service that has
// already handed all device memory to its own allocator, a latency-critical
// path that must not pay for cudaMalloc/cudaFree (both may synchronise the
// device), or code that must not fail with out-of-memory in the middle of a
// request.  For them this entry point runs the same Sign kernel as dil_sign on
// a fixed scratch area that lives in this library's device image: a file-scope
// array of NOALLOC_SCRATCH_BYTES, which every GPU that loads the library holds
// until the process exits.
//
// Set-up: the first call on a device (with that device current; a call with
// n = 0 does only this) looks up the array's device address with
// cudaGetSymbolAddress, caches it per device, loads the Sign kernels of the
// three levels and runs each once on no tasks, so that their code and their
// local-memory reservation are in place before the first real request.  That
// first call synchronises its stream and should come before any stream
// capture.  Every later call reuses the cached address and allocates nothing.
// The cache is per device ordinal: after cudaDeviceReset the array may move,
// so this entry point must not be used on a device that was reset.
//
// Launch shape: 4 warps per CTA, one warp per task (every level), whatever
// the context tuning says; the autotuned plain Sign shapes also use one warp
// per task and lie within about 1% of it.
//
// The array is shared by every call and keeps the previous call's contents.
// The Sign kernel writes every scratch word of a task before it reads it, so
// nothing has to be cleared between calls.  Calls that overlap on the GPU (for
// example on two streams) use the same scratch and race: serialise them.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/dil.h"
#include "dil_launch.h"

namespace {

constexpr size_t NOALLOC_SCRATCH_BYTES = (size_t)64 << 20;   // 64 MiB
constexpr int MAX_DEVICES = 64;

__device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

constexpr int NOALLOC_WARPS = 4;   // warps per CTA; one warp per task

std::mutex g_setup_mu;
void *g_scratch_addr[MAX_DEVICES] = {};

// Device address of g_noalloc_scratch on the current device; the first use on
// a device also warms the three Sign kernels on stream s.
int scratch_address(void **out, cudaStream_t s) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) {
        cudaGetLastError();
        return DIL_ECUDA;
    }
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        for (int level : {2, 3, 5})
            if (e == cudaSuccess) e = dil::warm_sign(level, NOALLOC_WARPS, 1, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return DIL_ECUDA;
        }
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return DIL_OK;
}

}  // namespace

extern "C" int dil_sign_noalloc(int level, size_t n, const uint8_t *sk, const uint8_t *msg,
                                const uint64_t *msg_off, uint8_t *sig, int32_t *task_status, void *stream) {
    if (level != 2 && level != 3 && level != 5) return DIL_EINVAL;
    const size_t per_task = dil::scratch_polys(dil::OP_SIGN, level) * 256 * sizeof(int32_t);
    if (n > NOALLOC_SCRATCH_BYTES / per_task) return DIL_EINVAL;   // beyond the static scratch
    void *scratch = nullptr;
    int rc = scratch_address(&scratch, (cudaStream_t)stream);   // set-up on a device's first call
    if (rc != DIL_OK || n == 0) return rc;
    if (!sk || !msg_off || !sig) return DIL_EINVAL;
    const int l = level == 2 ? 4 : level == 3 ? 5 : 7;
    const int max_iter = (65536 - l) / l + 1;   // cap implied by the 16-bit nonce
    cudaError_t e = dil::launch_sign(level, (int)n, sk, msg, msg_off, sig, task_status, nullptr,
                                     static_cast<int32_t *>(scratch), max_iter, NOALLOC_WARPS, 1,
                                     (cudaStream_t)stream);
    if (e != cudaSuccess) return DIL_ECUDA;
    return DIL_OK;
}

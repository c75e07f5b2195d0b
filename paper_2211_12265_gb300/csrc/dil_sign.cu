// Plain Sign kernel (Alg 2): one task per group of P warps, whole rejection
// loop in one launch (section 4.2 single-kernel fusion with early evaluation).
#include "dil_kern.cuh"

namespace dil {

template <int LEVEL, int P>
__global__ void __launch_bounds__(256, 4) k_sign(int n, const uint8_t *__restrict__ sk,
                                                 const uint8_t *__restrict__ msg, const uint64_t *__restrict__ off,
                                                 uint8_t *sig, int32_t *status, int32_t *iters, int32_t *scratch,
                                                 int max_iter) {
    extern __shared__ __align__(16) uint8_t smem[];
    const CtaView v = cta_setup<P>(smem);
    const int task = blockIdx.x * v.groups + v.group;
    if (task >= n) return;
    using V = Lv<LEVEL>;
    int32_t *scr = scratch + (size_t)task * Scratch<LEVEL>::SIGN_POLYS * N;
    uint64_t m0;
    size_t mlen;
    if (!message_of(off, task, m0, mlen)) {   // decreasing offsets: reject the task
        sign_zero<LEVEL, P>(sig + (size_t)task * V::SIG, v.g, v.lane);
        if (v.g == 0 && v.lane == 0) {
            if (status) status[task] = DIL_EINVAL;
            if (iters) iters[task] = 0;
        }
        return;
    }
    sign_prepare<LEVEL, P>(sk + (size_t)task * V::SK, msg + m0, mlen, scr, *v.gs, *v.ws, v.zt, v.g, v.bar, v.lane);
    int it = 0;
    bool ok = false;
    MaskStream ms{0, 0};
    while (it < max_iter) {
        ok = sign_attempt<LEVEL, P>(it * V::L, scr, scr + Scratch<LEVEL>::PRE_POLYS * N, ms, *v.gs, *v.ws, v.zt,
                                    v.izt, v.g, v.bar, v.lane);
        ++it;
        if (ok) break;
    }
    uint8_t *tsig = sig + (size_t)task * V::SIG;
    if (ok)
        sign_pack<LEVEL, P>(tsig, scr + Scratch<LEVEL>::PRE_POLYS * N, *v.gs, v.g, v.lane);
    else
        sign_zero<LEVEL, P>(tsig, v.g, v.lane);
    if (v.g == 0 && v.lane == 0) {
        if (status) status[task] = ok ? DIL_OK : DIL_EITER;
        if (iters) iters[task] = it;
    }
}

cudaError_t launch_sign(int level, int n, const uint8_t *sk, const uint8_t *msg, const uint64_t *off,
                        uint8_t *sig, int32_t *status, int32_t *iters, int32_t *scratch, int max_iter, int warps,
                        int p, cudaStream_t s) {
    DIL_DISPATCH(k_sign, sk, msg, off, sig, status, iters, scratch, max_iter)
}

namespace {
template <class Kern>
cudaError_t warm(Kern kern, int warps, int p, cudaStream_t s) {
    const size_t smem = cta_bytes(warps, p);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    // n = 0: every group returns before it touches a pointer
    kern<<<1, warps * 32, smem, s>>>(0, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, 0);
    return cudaGetLastError();
}
}  // namespace

cudaError_t warm_sign(int level, int warps, int p, cudaStream_t s) {
    switch (level * 10 + p) {
        case 21: return warm(k_sign<2, 1>, warps, p, s);
        case 31: return warm(k_sign<3, 1>, warps, p, s);
        case 51: return warm(k_sign<5, 1>, warps, p, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace dil

// Resident-A^ forms of the plain kernels: A^ = ExpandA(rho) written to a
// caller's buffer (Alg 4; the matrix Alg 1 samples and Alg 2 / Alg 3 use in the
// NTT domain), and Sign / Verify reading that A^ instead of sampling it.  A
// task runs on one warp, as in the plain kernels' tuned shapes; the task
// bodies are the plain ones (dil_procs.cuh) with the A^ source switched.
#include "dil_kern.cuh"

namespace dil {

// A^ of task `task` at ahat + task k l N, polynomial (i, j) at index i l + j,
// coefficients in index order, each in [0, q).
template <int LEVEL>
__global__ void __launch_bounds__(256, 4) k_expand_a(int n, const uint8_t *__restrict__ rho, size_t rho_stride,
                                                     int32_t *ahat) {
    extern __shared__ __align__(16) uint8_t smem[];
    const CtaView v = cta_setup<1>(smem);
    const int task = blockIdx.x * v.groups + v.group;
    if (task >= n) return;
    using V = Lv<LEVEL>;
    constexpr int KL = V::K * V::L;
    stage_bytes(v.gs->rho, rho + (size_t)task * rho_stride, 32, v.lane);
    __syncwarp();
    expand_a_range<LEVEL>(v.gs->rho, 0, KL, ahat + (size_t)task * KL * N, *v.ws, v.lane);
}

template <int LEVEL>
__global__ void __launch_bounds__(256, 4) k_sign_a(int n, const uint8_t *__restrict__ sk,
                                                   const uint8_t *__restrict__ msg, const uint64_t *__restrict__ off,
                                                   const int32_t *__restrict__ ahat, uint8_t *sig, int32_t *status,
                                                   int32_t *iters, int32_t *scratch, int max_iter) {
    extern __shared__ __align__(16) uint8_t smem[];
    const CtaView v = cta_setup<1>(smem);
    const int task = blockIdx.x * v.groups + v.group;
    if (task >= n) return;
    using V = Lv<LEVEL>;
    int32_t *scr = scratch + (size_t)task * Scratch<LEVEL>::SIGN_POLYS * N;
    uint64_t m0;
    size_t mlen;
    uint8_t *tsig = sig + (size_t)task * V::SIG;
    if (!message_of(off, task, m0, mlen)) {   // decreasing offsets: reject the task
        sign_zero<LEVEL, 1>(tsig, 0, v.lane);
        if (v.lane == 0) {
            if (status) status[task] = DIL_EINVAL;
            if (iters) iters[task] = 0;
        }
        return;
    }
    sign_prepare<LEVEL, 1, true>(sk + (size_t)task * V::SK, msg + m0, mlen, scr, *v.gs, *v.ws, v.zt, 0, v.bar,
                                 v.lane, ahat + (size_t)task * V::K * V::L * N);
    int it = 0;
    bool ok = false;
    MaskStream ms{0, 0};
    while (it < max_iter) {
        ok = sign_attempt<LEVEL, 1>(it * V::L, scr, scr + Scratch<LEVEL>::PRE_POLYS * N, ms, *v.gs, *v.ws, v.zt,
                                    v.izt, 0, v.bar, v.lane);
        ++it;
        if (ok) break;
    }
    if (ok)
        sign_pack<LEVEL, 1>(tsig, scr + Scratch<LEVEL>::PRE_POLYS * N, *v.gs, 0, v.lane);
    else
        sign_zero<LEVEL, 1>(tsig, 0, v.lane);
    if (v.lane == 0) {
        if (status) status[task] = ok ? DIL_OK : DIL_EITER;
        if (iters) iters[task] = it;
    }
}

template <int LEVEL>
__global__ void __launch_bounds__(256, 4) k_verify_a(int n, const uint8_t *__restrict__ pk,
                                                     const uint8_t *__restrict__ msg,
                                                     const uint64_t *__restrict__ off,
                                                     const uint8_t *__restrict__ sig, const int32_t *__restrict__ ahat,
                                                     uint8_t *ok, int32_t *scratch) {
    extern __shared__ __align__(16) uint8_t smem[];
    const CtaView v = cta_setup<1>(smem);
    const int task = blockIdx.x * v.groups + v.group;
    if (task >= n) return;
    using V = Lv<LEVEL>;
    uint64_t m0;
    size_t mlen;
    if (!message_of(off, task, m0, mlen)) {   // decreasing offsets: reject
        if (v.lane == 0) ok[task] = 0;
        return;
    }
    const int r = verify_task<LEVEL, 1, false, true>(
        pk + (size_t)task * V::PK, msg + m0, mlen, sig + (size_t)task * V::SIG,
        scratch + (size_t)task * Scratch<LEVEL>::VERIFY_POLYS * N, *v.gs, *v.ws, v.zt, v.izt, 0, v.bar, v.lane,
        ahat + (size_t)task * V::K * V::L * N);
    if (v.lane == 0) ok[task] = (uint8_t)r;
}

cudaError_t launch_expand_a(int level, int n, const uint8_t *rho, size_t rho_stride, int32_t *ahat, int warps,
                            cudaStream_t s) {
    switch (level) {
        case 2: return launch_plain(k_expand_a<2>, n, warps, 1, s, rho, rho_stride, ahat);
        case 3: return launch_plain(k_expand_a<3>, n, warps, 1, s, rho, rho_stride, ahat);
        case 5: return launch_plain(k_expand_a<5>, n, warps, 1, s, rho, rho_stride, ahat);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_sign_a(int level, int n, const uint8_t *sk, const uint8_t *msg, const uint64_t *off,
                          const int32_t *ahat, uint8_t *sig, int32_t *status, int32_t *iters, int32_t *scratch,
                          int max_iter, int warps, cudaStream_t s) {
    switch (level) {
        case 2: return launch_plain(k_sign_a<2>, n, warps, 1, s, sk, msg, off, ahat, sig, status, iters, scratch, max_iter);
        case 3: return launch_plain(k_sign_a<3>, n, warps, 1, s, sk, msg, off, ahat, sig, status, iters, scratch, max_iter);
        case 5: return launch_plain(k_sign_a<5>, n, warps, 1, s, sk, msg, off, ahat, sig, status, iters, scratch, max_iter);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_verify_a(int level, int n, const uint8_t *pk, const uint8_t *msg, const uint64_t *off,
                            const uint8_t *sig, const int32_t *ahat, uint8_t *ok, int32_t *scratch, int warps,
                            cudaStream_t s) {
    switch (level) {
        case 2: return launch_plain(k_verify_a<2>, n, warps, 1, s, pk, msg, off, sig, ahat, ok, scratch);
        case 3: return launch_plain(k_verify_a<3>, n, warps, 1, s, pk, msg, off, sig, ahat, ok, scratch);
        case 5: return launch_plain(k_verify_a<5>, n, warps, 1, s, pk, msg, off, sig, ahat, ok, scratch);
    }
    return cudaErrorInvalidValue;
}

}  // namespace dil

// Resident-key kernels: preparing a key store (A^, s^1, s^2, t^0, NTT(t1 2^d),
// tr per key) and Sign / Verify of tasks that name a resident key.  With the
// key's precomputation resident, Sign only hashes mu and rho' per message
// before its rejection loop, and Verify skips ExpandA and H(pk).
#include "dil_kern.cuh"

namespace dil {

template <int LEVEL, int P>
__global__ void __launch_bounds__(256, 4) k_key_prepare(int n, const uint8_t *__restrict__ pk,
                                                        const uint8_t *__restrict__ sk, int32_t *keys, uint8_t *tr) {
    extern __shared__ __align__(16) uint8_t smem[];
    const CtaView v = cta_setup<P>(smem);
    const int task = blockIdx.x * v.groups + v.group;
    if (task >= n) return;
    using V = Lv<LEVEL>;
    key_prepare<LEVEL, P>(pk + (size_t)task * V::PK, sk ? sk + (size_t)task * V::SK : nullptr,
                          keys + (size_t)task * Scratch<LEVEL>::KEY_POLYS * N, tr + (size_t)task * 32, *v.gs, *v.ws,
                          v.zt, v.g, v.bar, v.lane);
}

template <int LEVEL, int P>
__global__ void __launch_bounds__(256, 4) k_sign_keyed(int n, int n_keys, const int32_t *__restrict__ key_idx,
                                                       const uint8_t *__restrict__ sk, const int32_t *keys,
                                                       const uint8_t *__restrict__ msg,
                                                       const uint64_t *__restrict__ off, uint8_t *sig,
                                                       int32_t *status, int32_t *iters, int32_t *scratch,
                                                       int max_iter) {
    extern __shared__ __align__(16) uint8_t smem[];
    const CtaView v = cta_setup<P>(smem);
    const int task = blockIdx.x * v.groups + v.group;
    if (task >= n) return;
    using V = Lv<LEVEL>;
    using S = Scratch<LEVEL>;
    const int key = key_idx[task];
    uint64_t m0;
    size_t mlen;
    if (key < 0 || key >= n_keys || !message_of(off, task, m0, mlen)) {   // unknown key or bad offsets: reject
        sign_zero<LEVEL, P>(sig + (size_t)task * V::SIG, v.g, v.lane);
        if (v.g == 0 && v.lane == 0) {
            if (status) status[task] = DIL_EINVAL;
            if (iters) iters[task] = 0;
        }
        return;
    }
    const int32_t *pre = keys + (size_t)key * S::KEY_POLYS * N;
    int32_t *itr = scratch + (size_t)task * S::ITR_POLYS * N;
    sign_prepare_keyed<LEVEL, P>(sk + (size_t)key * V::SK, msg + m0, mlen, *v.gs, v.g, v.bar, v.lane);
    int it = 0;
    bool ok = false;
    MaskStream ms{0, 0};
    while (it < max_iter) {
        ok = sign_attempt<LEVEL, P>(it * V::L, pre, itr, ms, *v.gs, *v.ws, v.zt, v.izt, v.g, v.bar, v.lane);
        ++it;
        if (ok) break;
    }
    uint8_t *tsig = sig + (size_t)task * V::SIG;
    if (ok)
        sign_pack<LEVEL, P>(tsig, itr, *v.gs, v.g, v.lane);
    else
        sign_zero<LEVEL, P>(tsig, v.g, v.lane);
    if (v.g == 0 && v.lane == 0) {
        if (status) status[task] = ok ? DIL_OK : DIL_EITER;
        if (iters) iters[task] = it;
    }
}

template <int LEVEL, int P>
__global__ void __launch_bounds__(256, 4) k_verify_keyed(int n, int n_keys, const int32_t *__restrict__ key_idx,
                                                         const uint8_t *__restrict__ pk, const int32_t *keys,
                                                         const uint8_t *__restrict__ tr,
                                                         const uint8_t *__restrict__ msg,
                                                         const uint64_t *__restrict__ off,
                                                         const uint8_t *__restrict__ sig, uint8_t *ok,
                                                         int32_t *scratch) {
    extern __shared__ __align__(16) uint8_t smem[];
    const CtaView v = cta_setup<P>(smem);
    const int task = blockIdx.x * v.groups + v.group;
    if (task >= n) return;
    using V = Lv<LEVEL>;
    using S = Scratch<LEVEL>;
    const int key = key_idx[task];
    uint64_t m0;
    size_t mlen;
    if (key < 0 || key >= n_keys || !message_of(off, task, m0, mlen)) {   // unknown key or bad offsets: reject
        if (v.g == 0 && v.lane == 0) ok[task] = 0;
        return;
    }
    int r = verify_task<LEVEL, P, true>(pk + (size_t)key * V::PK, msg + m0, mlen,
                                        sig + (size_t)task * V::SIG, scratch + (size_t)task * S::KEYED_VERIFY_POLYS * N,
                                        *v.gs, *v.ws, v.zt, v.izt, v.g, v.bar, v.lane,
                                        keys + (size_t)key * S::KEY_POLYS * N, tr + (size_t)key * 32);
    if (v.g == 0 && v.lane == 0) ok[task] = (uint8_t)r;
}

cudaError_t launch_key_prepare(int level, int n, const uint8_t *pk, const uint8_t *sk, int32_t *keys, uint8_t *tr,
                               int warps, int p, cudaStream_t s) {
    DIL_DISPATCH(k_key_prepare, pk, sk, keys, tr)
}

cudaError_t launch_sign_keyed(int level, int n, int n_keys, const int32_t *key_idx, const uint8_t *sk,
                              const int32_t *keys, const uint8_t *msg, const uint64_t *off, uint8_t *sig,
                              int32_t *status, int32_t *iters, int32_t *scratch, int max_iter, int warps, int p,
                              cudaStream_t s) {
    DIL_DISPATCH(k_sign_keyed, n_keys, key_idx, sk, keys, msg, off, sig, status, iters, scratch, max_iter)
}

cudaError_t launch_verify_keyed(int level, int n, int n_keys, const int32_t *key_idx, const uint8_t *pk,
                                const int32_t *keys, const uint8_t *tr, const uint8_t *msg, const uint64_t *off,
                                const uint8_t *sig, uint8_t *ok, int32_t *scratch, int warps, int p, cudaStream_t s) {
    DIL_DISPATCH(k_verify_keyed, n_keys, key_idx, pk, keys, tr, msg, off, sig, ok, scratch)
}

template <int LEVEL>
static size_t key_polys_of() { return Scratch<LEVEL>::KEY_POLYS; }
template <int LEVEL>
static size_t itr_polys_of() { return Scratch<LEVEL>::ITR_POLYS; }
template <int LEVEL>
static size_t keyed_verify_polys_of() { return Scratch<LEVEL>::KEYED_VERIFY_POLYS; }

size_t key_polys(int level) {
    return level == 2 ? key_polys_of<2>() : level == 3 ? key_polys_of<3>() : level == 5 ? key_polys_of<5>() : 0;
}

size_t keyed_verify_polys(int level) {
    return level == 2   ? keyed_verify_polys_of<2>()
           : level == 3 ? keyed_verify_polys_of<3>()
           : level == 5 ? keyed_verify_polys_of<5>()
                        : 0;
}

size_t keyed_sign_polys(int level) {
    return level == 2 ? itr_polys_of<2>() : level == 3 ? itr_polys_of<3>() : level == 5 ? itr_polys_of<5>() : 0;
}

}  // namespace dil

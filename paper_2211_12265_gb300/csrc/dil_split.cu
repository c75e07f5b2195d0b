// Split Sign: the fusion ablation of the paper's section 4.2 (one fused
// kernel per Sign against a split into several kernels).  A precompute kernel
// prepares every task (mu, rho', A^, s^1, s^2, t^0); then each repetition
// round is two kernels over all pending tasks — the first half (y, w, w1,
// c~) and the second half (c^, z, r0, hint, and the signature on acceptance)
// — with the per-task state in global memory between them.  The host repeats
// rounds until no task is pending.  Same outputs as the fused kernel.
#include "../../include/dil.h"
#include "dil_kern.cuh"

namespace dil {

// Per-task state carried between the split kernels (global memory).
struct __align__(16) SplitState {
    uint8_t mu[64];
    uint8_t rhop[64];
    uint8_t ctilde[32];
    int rep;      // current repetition index (nonce kappa = l rep)
    int done;     // 1 once signed or capped
    int ms_lo;    // the one-warp mask stream: nonces [ms_lo, ms_hi) sampled
    int ms_hi;    // into the task's y ring by earlier rounds
    int pad[4];
};

template <int LEVEL, int P>
__global__ void __launch_bounds__(256, 4) k_split_prepare(int n, const uint8_t *__restrict__ sk,
                                                          const uint8_t *__restrict__ msg,
                                                          const uint64_t *__restrict__ off, int32_t *scratch,
                                                          SplitState *state, uint8_t *sig, int32_t *status,
                                                          int32_t *iters, int *pending) {
    extern __shared__ __align__(16) uint8_t smem[];
    const CtaView v = cta_setup<P>(smem);
    const int task = blockIdx.x * v.groups + v.group;
    if (task >= n) return;
    using V = Lv<LEVEL>;
    GroupSmem &gs = *v.gs;
    int32_t *scr = scratch + (size_t)task * Scratch<LEVEL>::SIGN_POLYS * N;
    uint64_t m0;
    size_t mlen;
    if (!message_of(off, task, m0, mlen)) {   // decreasing offsets: reject now
        sign_zero<LEVEL, P>(sig + (size_t)task * V::SIG, v.g, v.lane);
        if (v.g == 0 && v.lane == 0) {
            state[task].done = 1;
            if (status) status[task] = DIL_EINVAL;
            if (iters) iters[task] = 0;
            atomicSub(pending, 1);
        }
        return;
    }
    sign_prepare<LEVEL, P>(sk + (size_t)task * V::SK, msg + m0, mlen, scr, gs, *v.ws, v.zt, v.g, v.bar, v.lane);
    if (v.g == 0) {
        SplitState &st = state[task];
        st.mu[v.lane] = gs.hb[HB_MU + v.lane];
        st.mu[32 + v.lane] = gs.hb[HB_MU + 32 + v.lane];
        st.rhop[v.lane] = gs.rhop[v.lane];
        st.rhop[32 + v.lane] = gs.rhop[32 + v.lane];
        if (v.lane == 0) {
            st.rep = 0;
            st.done = 0;
            st.ms_lo = 0;
            st.ms_hi = 0;
        }
    }
}

template <int LEVEL, int P>
__global__ void __launch_bounds__(256, 4) k_split_front(int n, int32_t *scratch, SplitState *state) {
    extern __shared__ __align__(16) uint8_t smem[];
    const CtaView v = cta_setup<P>(smem);
    const int task = blockIdx.x * v.groups + v.group;
    if (task >= n) return;
    SplitState &st = state[task];
    if (st.done) return;
    GroupSmem &gs = *v.gs;
    using S = Scratch<LEVEL>;
    if (v.g == 0) {
        gs.hb[HB_MU + v.lane] = st.mu[v.lane];
        gs.hb[HB_MU + 32 + v.lane] = st.mu[32 + v.lane];
        gs.rhop[v.lane] = st.rhop[v.lane];
        gs.rhop[32 + v.lane] = st.rhop[32 + v.lane];
    }
    group_sync<P>(v.bar);
    int32_t *scr = scratch + (size_t)task * S::SIGN_POLYS * N;
    MaskStream ms{st.ms_lo, st.ms_hi};   // continues across rounds like the fused loop's
    const int kappa = Lv<LEVEL>::L * st.rep;
    sign_front<LEVEL, P>(kappa, scr, scr + S::PRE_POLYS * N, ms, gs, *v.ws, v.zt, v.izt, v.g, v.bar, v.lane);
    if (v.g == 0) {
        st.ctilde[v.lane] = gs.ctilde[v.lane];
        if (v.lane == 0) {
            st.ms_lo = ms.lo;
            st.ms_hi = ms.hi;
        }
    }
}

template <int LEVEL, int P>
__global__ void __launch_bounds__(256, 4) k_split_back(int n, int32_t *scratch, SplitState *state, uint8_t *sig,
                                                       int32_t *status, int32_t *iters, int max_iter,
                                                       int *pending) {
    extern __shared__ __align__(16) uint8_t smem[];
    const CtaView v = cta_setup<P>(smem);
    const int task = blockIdx.x * v.groups + v.group;
    if (task >= n) return;
    SplitState &st = state[task];
    if (st.done) return;
    GroupSmem &gs = *v.gs;
    using V = Lv<LEVEL>;
    using S = Scratch<LEVEL>;
    if (v.g == 0) {
        gs.ctilde[v.lane] = st.ctilde[v.lane];
        if (v.lane == 0) {
            gs.flag = 0;
            gs.count = 0;
        }
    }
    group_sync<P>(v.bar);
    int32_t *scr = scratch + (size_t)task * S::SIGN_POLYS * N;
    int32_t *itr = scr + S::PRE_POLYS * N;
    const int rep = st.rep;
    const bool ok = sign_back<LEVEL, P>(V::L * rep, scr, itr, gs, *v.ws, v.zt, v.izt, v.g, v.bar, v.lane);
    uint8_t *tsig = sig + (size_t)task * V::SIG;
    if (ok) {
        sign_pack<LEVEL, P>(tsig, itr, gs, v.g, v.lane);
    } else if (rep + 1 >= max_iter) {
        sign_zero<LEVEL, P>(tsig, v.g, v.lane);
    }
    group_sync<P>(v.bar);
    if (v.g == 0 && v.lane == 0) {
        if (ok || rep + 1 >= max_iter) {
            st.done = 1;
            if (status) status[task] = ok ? DIL_OK : DIL_EITER;
            if (iters) iters[task] = rep + 1;
            atomicSub(pending, 1);
        } else {
            st.rep = rep + 1;
        }
    }
}

#define SPLIT_DISPATCH(KERN, ...)                                                                \
    switch (level * 10 + p) {                                                                    \
        case 21: return launch_plain(KERN<2, 1>, n, warps, p, s, __VA_ARGS__);                   \
        case 22: return launch_plain(KERN<2, 2>, n, warps, p, s, __VA_ARGS__);                   \
        case 31: return launch_plain(KERN<3, 1>, n, warps, p, s, __VA_ARGS__);                   \
        case 32: return launch_plain(KERN<3, 2>, n, warps, p, s, __VA_ARGS__);                   \
        case 51: return launch_plain(KERN<5, 1>, n, warps, p, s, __VA_ARGS__);                   \
        case 52: return launch_plain(KERN<5, 2>, n, warps, p, s, __VA_ARGS__);                   \
    }                                                                                            \
    return cudaErrorInvalidValue;

static cudaError_t split_prepare(int level, int n, const uint8_t *sk, const uint8_t *msg, const uint64_t *off,
                                 int32_t *scratch, SplitState *state, uint8_t *sig, int32_t *status, int32_t *iters,
                                 int *pending, int warps, int p, cudaStream_t s) {
    SPLIT_DISPATCH(k_split_prepare, sk, msg, off, scratch, state, sig, status, iters, pending)
}
static cudaError_t split_front(int level, int n, int32_t *scratch, SplitState *state, int warps, int p,
                               cudaStream_t s) {
    SPLIT_DISPATCH(k_split_front, scratch, state)
}
static cudaError_t split_back(int level, int n, int32_t *scratch, SplitState *state, uint8_t *sig,
                              int32_t *status, int32_t *iters, int max_iter, int *pending, int warps, int p,
                              cudaStream_t s) {
    SPLIT_DISPATCH(k_split_back, scratch, state, sig, status, iters, max_iter, pending)
}

size_t split_state_bytes() { return sizeof(SplitState); }

// Runs the split Sign on one chunk: prepare, then rounds of (front, back)
// until the pending counter (device) reaches zero; `rounds` returns how many.
cudaError_t launch_sign_split(int level, int n, const uint8_t *sk, const uint8_t *msg, const uint64_t *off,
                              uint8_t *sig, int32_t *status, int32_t *iters, int32_t *scratch, void *state_mem,
                              int *pending, int max_iter, int warps, int p, cudaStream_t s, int *rounds) {
    SplitState *state = static_cast<SplitState *>(state_mem);
    *rounds = 0;
    if (n <= 0) return cudaSuccess;
    cudaError_t e = cudaMemcpyAsync(pending, &n, sizeof(int), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = split_prepare(level, n, sk, msg, off, scratch, state, sig, status, iters, pending, warps, p, s);
    int left = n;
    while (e == cudaSuccess && left > 0 && *rounds < max_iter) {
        e = split_front(level, n, scratch, state, warps, p, s);
        if (e == cudaSuccess) e = split_back(level, n, scratch, state, sig, status, iters, max_iter, pending, warps, p, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&left, pending, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        ++*rounds;
    }
    return e;
}

}  // namespace dil

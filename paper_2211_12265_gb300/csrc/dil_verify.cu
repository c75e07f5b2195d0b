// Plain Verify kernel (Alg 3): one task per group of P warps, A^ sampled on
// the fly row by row (section 3.5).
#include "dil_kern.cuh"

namespace dil {

template <int LEVEL, int P>
__global__ void __launch_bounds__(256, 4) k_verify(int n, const uint8_t *__restrict__ pk,
                                                   const uint8_t *__restrict__ msg,
                                                   const uint64_t *__restrict__ off,
                                                   const uint8_t *__restrict__ sig, uint8_t *ok, int32_t *scratch) {
    extern __shared__ __align__(16) uint8_t smem[];
    const CtaView v = cta_setup<P>(smem);
    const int task = blockIdx.x * v.groups + v.group;
    if (task >= n) return;
    using V = Lv<LEVEL>;
    uint64_t m0;
    size_t mlen;
    if (!message_of(off, task, m0, mlen)) {   // decreasing offsets: reject
        if (v.g == 0 && v.lane == 0) ok[task] = 0;
        return;
    }
    int r = verify_task<LEVEL, P>(pk + (size_t)task * V::PK, msg + m0, mlen,
                                  sig + (size_t)task * V::SIG,
                                  scratch + (size_t)task * Scratch<LEVEL>::VERIFY_POLYS * N, *v.gs, *v.ws, v.zt,
                                  v.izt, v.g, v.bar, v.lane);
    if (v.g == 0 && v.lane == 0) ok[task] = (uint8_t)r;
}

cudaError_t launch_verify(int level, int n, const uint8_t *pk, const uint8_t *msg, const uint64_t *off,
                          const uint8_t *sig, uint8_t *ok, int32_t *scratch, int warps, int p, cudaStream_t s) {
    DIL_DISPATCH(k_verify, pk, msg, off, sig, ok, scratch)
}

size_t cta_smem_bytes(int warps, int p) { return cta_bytes(warps, p); }

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

}  // namespace dil

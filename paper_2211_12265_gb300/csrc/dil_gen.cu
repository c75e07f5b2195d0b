// Plain Gen kernel (Alg 1): one task per group of P warps.
#include "dil_kern.cuh"

namespace dil {

template <int LEVEL, int P>
__global__ void __launch_bounds__(256, 4) k_keygen(int n, const uint8_t *__restrict__ seeds, uint8_t *pk,
                                                   uint8_t *sk, int32_t *scratch) {
    extern __shared__ __align__(16) uint8_t smem[];
    const CtaView v = cta_setup<P>(smem);
    const int task = blockIdx.x * v.groups + v.group;
    if (task >= n) return;
    using V = Lv<LEVEL>;
    gen_task<LEVEL, P>(seeds + (size_t)task * 32, pk + (size_t)task * V::PK, sk + (size_t)task * V::SK,
                       scratch + (size_t)task * Scratch<LEVEL>::GEN_POLYS * N, *v.gs, *v.ws, v.zt, v.izt, v.g,
                       v.bar, v.lane);
}

cudaError_t launch_keygen(int level, int n, const uint8_t *seeds, uint8_t *pk, uint8_t *sk, int32_t *scratch,
                          int warps, int p, cudaStream_t s) {
    DIL_DISPATCH(k_keygen, seeds, pk, sk, scratch)
}

}  // namespace dil

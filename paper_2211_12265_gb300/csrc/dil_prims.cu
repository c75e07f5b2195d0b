// Kernels behind the test-only entry points: one primitive of the hot path per
// kernel (SHAKE, NTT/INTT, the four samplers, the coefficient functions), each
// built from the same device functions the fused procedure kernels use.
#include "dil_kern.cuh"

namespace dil {

#define PRIM_PROLOGUE                                                             \
    extern __shared__ __align__(16) uint8_t smem[];                               \
    const CtaView v = cta_setup<1>(smem);                                         \
    const int item = blockIdx.x * v.groups + v.group;                             \
    if (item >= n) return;                                                        \
    const int lane = v.lane;                                                      \
    const int32_t *zt = v.zt, *izt = v.izt;                                       \
    GroupSmem &gs = *v.gs;                                                        \
    WarpSmem &ws = *v.ws;                                                         \
    (void)zt; (void)izt; (void)gs; (void)ws;

constexpr int PRIM_WARPS = 4;

__global__ void k_test_shake(int n, int rate, const uint8_t *in, const uint64_t *off, uint8_t *out, int outlen) {
    PRIM_PROLOGUE
    uint32_t lo = 0, hi = 0;
    absorb_concat(lo, hi, ws.sq, 0, in + off[item], (size_t)(off[item + 1] - off[item]), rate, lane);
    uint8_t *o = out + (size_t)item * outlen;
    for (int p = 0; p < outlen; p += rate) {
        if (p) keccak_f(lo, hi);
        squeeze_words(lo, hi, ws.sq, rate / 8, lane);
        __syncwarp();
        for (int b = lane; b < rate && p + b < outlen; b += 32) o[p + b] = ws.sq[b];
        __syncwarp();
    }
}

// SHAKE256 of byte string `item` carried by a K16Rider through perms[item]
// sixteen-state permutations (the other instances hold zero states), then
// finished on the 25-lane form: the first 32 output bytes to out + 32 item.
__global__ void k_test_k16_rider(int n, const uint8_t *in, const uint64_t *off, const int32_t *perms,
                                 uint8_t *out) {
    PRIM_PROLOGUE
    for (int i = 0; i < 25; ++i) ws.k16[k16_slot(i, lane)] = 0u;
    __syncwarp();
    K16Rider rider(in + off[item], (size_t)(off[item + 1] - off[item]), reinterpret_cast<uint32_t *>(gs.tr));
    const int np = perms[item];
#pragma unroll 1
    for (int p = 0; p < np; ++p) {
        rider.before(ws.k16, lane);
        keccak16_permute(ws.k16);
        rider.after(ws.k16, lane);
    }
    rider.finish(ws.k16, lane);
    out[(size_t)item * 32 + lane] = gs.tr[lane];
}

// SHAKE256 of byte string `item` carried by a K16ChainRider through
// perms[item] sixteen-state permutations; before permutation p the first
// min(len, p * step[item]) bytes count as written, and after every
// permutation instance 15 is overwritten (as the samplers' shared-memory
// union does), so only the saved state may carry the hash.  Then finished on
// the 25-lane form: the first 32 output bytes to out + 32 item.
__global__ void k_test_k16_chain_rider(int n, const uint8_t *in, const uint64_t *off, const int32_t *perms,
                                       const int32_t *step, uint8_t *out) {
    PRIM_PROLOGUE
    for (int i = 0; i < 25; ++i) ws.k16[k16_slot(i, lane)] = 0u;
    __syncwarp();
    const size_t len = (size_t)(off[item + 1] - off[item]);
    K16ChainRider rider(in + off[item], len, reinterpret_cast<uint32_t *>(gs.hb), reinterpret_cast<uint32_t *>(gs.tr));
    const int np = perms[item];
    const size_t st = (size_t)max(step[item], 0);
#pragma unroll 1
    for (int p = 0; p < np; ++p) {
        rider.set_ready(min(len, (size_t)p * st));
        rider.before(ws.k16, lane);
        keccak16_permute(ws.k16);
        rider.after(ws.k16, lane);
        if (lane < 25) {
            ws.k16[k16_slot(lane, 30)] ^= 0x9E3779B9u * (p + 1);
            ws.k16[k16_slot(lane, 31)] ^= 0x7F4A7C15u * (p + 1);
        }
        __syncwarp();
    }
    rider.finish(lane);
    out[(size_t)item * 32 + lane] = gs.tr[lane];
}

__global__ void k_test_ntt(int n, const int32_t *in, int32_t *out, int inverse) {
    PRIM_PROLOGUE
    int32_t r[8];
    const int32_t *src = in + (size_t)item * N;
    int32_t *dst = out + (size_t)item * N;
    if (!inverse) {
#pragma unroll
        for (int m = 0; m < 8; ++m) r[m] = reduce_q(src[lane + 32 * m]);
        ntt_fwd(r, ws.buf, zt, lane);
#pragma unroll
        for (int m = 0; m < 8; ++m) r[m] = to_canonical(reduce_q(r[m]));
        store_l2(dst, r, lane);
    } else {
        // ntt_inv returns INTT(x) * 2^32; feed x * 2^-32 = mont_mul(x, 1)
        load_l2(r, src, lane);
#pragma unroll
        for (int m = 0; m < 8; ++m) r[m] = mont_mul(reduce_q(r[m]), 1);
        ntt_inv(r, ws.buf, izt, lane);
#pragma unroll
        for (int m = 0; m < 8; ++m) r[m] = to_canonical(r[m]);
        store_l0(dst, r, lane);
    }
}

// Keccak-f[1600] of `states` states (25 little-endian 64-bit lanes each) in
// one of the permutation forms; warp `item` permutes states
// [FORM item, FORM item + FORM).
template <int FORM>
__global__ void k_test_keccak_f(int n, int states, const uint64_t *in, uint64_t *out) {
    PRIM_PROLOGUE
    const int s0 = item * FORM;
    if constexpr (FORM == 1 || FORM == 2) {
        uint32_t lo[2] = {0, 0}, hi[2] = {0, 0};
#pragma unroll
        for (int k = 0; k < FORM; ++k) {
            if (lane < 25 && s0 + k < states) {
                const uint64_t w = in[(size_t)(s0 + k) * 25 + lane];
                lo[k] = (uint32_t)w;
                hi[k] = (uint32_t)(w >> 32);
            }
        }
        if constexpr (FORM == 1)
            keccak_f(lo[0], hi[0]);
        else
            keccak_f2(lo[0], hi[0], lo[1], hi[1]);
#pragma unroll
        for (int k = 0; k < FORM; ++k)
            if (lane < 25 && s0 + k < states) out[(size_t)(s0 + k) * 25 + lane] = ((uint64_t)hi[k] << 32) | lo[k];
    } else if constexpr (FORM == 6) {
        for (int w = lane; w < K6_STATES * K6_WORDS; w += 32) {
            const int g = w / K6_WORDS, i = (w % K6_WORDS) >> 1, h = w & 1;
            ws.kst[w] = s0 + g < states ? (uint32_t)(in[(size_t)(s0 + g) * 25 + i] >> (32 * h)) : 0u;
        }
        __syncwarp();
        keccak6_permute(ws.kst, ws.kpi());
        for (int w = lane; w < K6_STATES * 25; w += 32) {
            const int g = w / 25, i = w % 25;
            if (s0 + g < states)
                out[(size_t)(s0 + g) * 25 + i] =
                    ((uint64_t)ws.kst[K6_WORDS * g + 2 * i + 1] << 32) | ws.kst[K6_WORDS * g + 2 * i];
        }
    } else {
        const int st = lane >> 1, h = lane & 1;
        for (int i = 0; i < 25; ++i)
            ws.k16[k16_slot(i, lane)] = s0 + st < states ? (uint32_t)(in[(size_t)(s0 + st) * 25 + i] >> (32 * h)) : 0u;
        __syncwarp();
        keccak16_permute(ws.k16);
        for (int w = lane; w < K16_STATES * 25; w += 32) {
            const int g = w / 25, i = w % 25;
            if (s0 + g < states)
                out[(size_t)(s0 + g) * 25 + i] =
                    ((uint64_t)ws.k16[k16_slot(i, 2 * g + 1)] << 32) | ws.k16[k16_slot(i, 2 * g)];
        }
    }
}

// Covers the single, pair, six- and sixteen-sponge forms: polynomial 0 alone,
// 1-2 as a pair, 3-8 as one six-sponge range, the rest as one range (sixteen
// at a time while at least seven remain, then the tail).
template <int LEVEL>
__global__ void k_test_expand_a(int n, const uint8_t *rho, int32_t *out) {
    PRIM_PROLOGUE
    using V = Lv<LEVEL>;
    stage_bytes(gs.rho, rho + (size_t)item * 32, 32, lane);
    __syncwarp();
    int32_t *o = out + (size_t)item * V::K * V::L * N;
    expand_a_range<LEVEL>(gs.rho, 0, 1, o, ws, lane);
    expand_a_range<LEVEL>(gs.rho, 1, 3, o, ws, lane);
    expand_a_range<LEVEL>(gs.rho, 3, 9, o, ws, lane);
    expand_a_range<LEVEL>(gs.rho, 9, V::K * V::L, o, ws, lane);
}

// ---------------------------------------------------------------- t^0 = NTT(t0)
// The steps of the paper's speedup breakdown (section 5, computation of t^0
// in Sign): unpack t0 from sk and transform it, as (0) an unpack kernel and a
// transform kernel through global memory, (1) one fused kernel with the same
// global-memory round trip, (2) one kernel keeping t0 in registers, with an
// exchange layout that has bank conflicts, (3) registers and the
// conflict-free layout (the form Sign uses).  Every variant writes the k
// polynomials of t^0 per task in index order, reduced to [0, q).

// Forward NTT with the exchanges unpadded (coefficient i at word i): the
// L0 -> L1 reads and the L1 -> L2 writes put 8 lanes on one bank, the
// L1 -> L2 reads 4.  Same arithmetic and output as ntt_fwd.
static __device__ __noinline__ Poly8 ntt_fwd_unpadded_impl(Poly8 p, uint32_t buf, uint32_t zt) {
    const int lane = threadIdx.x & 31;
    int32_t *r = p.v;
    {
        const int32_t z = c_zetas.z[1];
#pragma unroll
        for (int m = 0; m < 4; ++m) ct_bfly(r[m], r[m + 4], z);
    }
    ct_bfly(r[0], r[2], c_zetas.z[2]);
    ct_bfly(r[1], r[3], c_zetas.z[2]);
    ct_bfly(r[4], r[6], c_zetas.z[3]);
    ct_bfly(r[5], r[7], c_zetas.z[3]);
    ct_bfly(r[0], r[1], c_zetas.z[4]);
    ct_bfly(r[2], r[3], c_zetas.z[5]);
    ct_bfly(r[4], r[5], c_zetas.z[6]);
    ct_bfly(r[6], r[7], c_zetas.z[7]);
    // L0 -> L1: coefficient t + 32 m, read back as 32 (t >> 2) + (t & 3) + 4 m
#pragma unroll
    for (int m = 0; m < 8; ++m) sts32(buf + 4 * (lane + 32 * m), r[m]);
    __syncwarp();
    const int b = lane >> 2;
    const uint32_t base1 = buf + 4 * (32 * b + (lane & 3));
#pragma unroll
    for (int m = 0; m < 8; ++m) r[m] = lds32(base1 + 16 * m);
    __syncwarp();
    {
        const int32_t z = ldz32(zt + 4 * (8 + b));
#pragma unroll
        for (int m = 0; m < 4; ++m) ct_bfly(r[m], r[m + 4], z);
    }
    {
        const int2 z = ldz64(zt + 4 * (16 + 2 * b));
        ct_bfly(r[0], r[2], z.x);
        ct_bfly(r[1], r[3], z.x);
        ct_bfly(r[4], r[6], z.y);
        ct_bfly(r[5], r[7], z.y);
    }
    {
        const int4 z = ldz128(zt + 4 * (32 + 4 * b));
        ct_bfly(r[0], r[1], z.x);
        ct_bfly(r[2], r[3], z.y);
        ct_bfly(r[4], r[5], z.z);
        ct_bfly(r[6], r[7], z.w);
    }
    // L1 -> L2: back to coefficient order, read as 8 t + m
#pragma unroll
    for (int m = 0; m < 8; ++m) sts32(base1 + 16 * m, r[m]);
    __syncwarp();
#pragma unroll
    for (int m = 0; m < 8; ++m) r[m] = lds32(buf + 4 * (8 * lane + m));
    __syncwarp();
    {
        const int2 z = ldz64(zt + 4 * (64 + 2 * lane));
        ct_bfly(r[0], r[2], z.x);
        ct_bfly(r[1], r[3], z.x);
        ct_bfly(r[4], r[6], z.y);
        ct_bfly(r[5], r[7], z.y);
    }
    {
        const int4 z = ldz128(zt + 4 * (128 + 4 * lane));
        ct_bfly(r[0], r[1], z.x);
        ct_bfly(r[2], r[3], z.y);
        ct_bfly(r[4], r[5], z.z);
        ct_bfly(r[6], r[7], z.w);
    }
    return p;
}

template <int LEVEL>
__device__ __forceinline__ void t0_unpack(int32_t r[8], const uint8_t *sk, int i, WarpSmem &ws, int lane) {
    using V = Lv<LEVEL>;
    unpack_poly_l0<D>(r, sk + V::SK_T0 + i * V::POLYT0, 1 << (D - 1), ws, lane);
}

__device__ __forceinline__ void t0_store(int32_t *dst, int32_t r[8], int lane) {
#pragma unroll
    for (int m = 0; m < 8; ++m) r[m] = to_canonical(reduce_q(r[m]));
    store_l2(dst, r, lane);
}

// (0a) unpack kernel: t0 of task `item` to tmp (natural order)
template <int LEVEL>
__global__ void k_test_t0_unpack(int n, const uint8_t *sk, int32_t *tmp) {
    PRIM_PROLOGUE
    using V = Lv<LEVEL>;
    int32_t r[8];
#pragma unroll 1
    for (int i = 0; i < V::K; ++i) {
        t0_unpack<LEVEL>(r, sk + (size_t)item * V::SK, i, ws, lane);
        store_l0(tmp + ((size_t)item * V::K + i) * N, r, lane);
    }
}

// (0b) transform kernel: tmp -> t^0
template <int LEVEL>
__global__ void k_test_t0_ntt(int n, const int32_t *tmp, int32_t *out) {
    PRIM_PROLOGUE
    using V = Lv<LEVEL>;
    int32_t r[8];
#pragma unroll 1
    for (int i = 0; i < V::K; ++i) {
        load_l0(r, tmp + ((size_t)item * V::K + i) * N, lane);
        ntt_fwd(r, ws.buf, zt, lane);
        t0_store(out + ((size_t)item * V::K + i) * N, r, lane);
    }
}

// (1) both steps in one kernel, t0 still through global memory
template <int LEVEL>
__global__ void k_test_t0_fused_gmem(int n, const uint8_t *sk, int32_t *tmp, int32_t *out) {
    PRIM_PROLOGUE
    using V = Lv<LEVEL>;
    int32_t r[8];
    int32_t *t = tmp + (size_t)item * V::K * N;
#pragma unroll 1
    for (int i = 0; i < V::K; ++i) {
        t0_unpack<LEVEL>(r, sk + (size_t)item * V::SK, i, ws, lane);
        store_l0(t + i * N, r, lane);
    }
    __syncwarp();
#pragma unroll 1
    for (int i = 0; i < V::K; ++i) {
        load_l0(r, t + i * N, lane);
        ntt_fwd(r, ws.buf, zt, lane);
        t0_store(out + ((size_t)item * V::K + i) * N, r, lane);
    }
}

// (2) / (3) one kernel, t0 in registers; UNPADDED selects the conflicting
// exchange layout
template <int LEVEL, bool UNPADDED>
__global__ void k_test_t0_registers(int n, const uint8_t *sk, int32_t *out) {
    PRIM_PROLOGUE
    using V = Lv<LEVEL>;
    int32_t r[8];
#pragma unroll 1
    for (int i = 0; i < V::K; ++i) {
        t0_unpack<LEVEL>(r, sk + (size_t)item * V::SK, i, ws, lane);
        if constexpr (UNPADDED) {
            Poly8 p;
#pragma unroll
            for (int m = 0; m < 8; ++m) p.v[m] = r[m];
            p = ntt_fwd_unpadded_impl(p, smem_addr(ws.buf), smem_addr(zt));
#pragma unroll
            for (int m = 0; m < 8; ++m) r[m] = p.v[m];
        } else {
            ntt_fwd(r, ws.buf, zt, lane);
        }
        t0_store(out + ((size_t)item * V::K + i) * N, r, lane);
    }
}

template <int LEVEL>
__global__ void k_test_expand_s(int n, const uint8_t *rhop, int32_t *out) {
    PRIM_PROLOGUE
    using V = Lv<LEVEL>;
    stage_bytes(gs.rhop, rhop + (size_t)item * 64, 64, lane);
    __syncwarp();
    int32_t *o = out + (size_t)item * (V::K + V::L) * N;
    if (item % 3 == 2) {   // items 2 mod 3: all l + k sponges in one sixteen-state batch
        expand_s_16<V::ETA>(gs.rhop, V::L + V::K, o, ws.k16, lane);
        return;
    }
    int32_t a[8];
    for (int j = 0; j < V::L + V::K; ++j) {
        if (item % 3 == 1 && j + 1 < V::L + V::K) {   // items 1 mod 3: pairs, then a single tail
            expand_s_pair<V::ETA>(gs.rhop, j, j + 1, ws.buf, ws.buf2, ws.sq, ws.sq2, lane);
            read_buf_l0(a, ws.buf2, lane);
            store_l0(o + (j + 1) * N, a, lane);
        } else {               // items 0 mod 3: one sponge at a time
            expand_s_poly<V::ETA>(gs.rhop, j, ws.buf, ws.sq, lane);
        }
        read_buf_l0(a, ws.buf, lane);
        __syncwarp();
        store_l0(o + j * N, a, lane);
        if (item % 3 == 1 && j + 1 < V::L + V::K) ++j;
    }
}

// Items 0 mod 3: all l polynomials through six-sponge batches (with a pair or
// single tail where l is not a multiple of six); 1 mod 3: single, pair and
// the rest; 2 mod 3: one sixteen-sponge batch of l instances.
template <int LEVEL>
__global__ void k_test_expand_mask(int n, const uint8_t *rhop, const int32_t *kappa, int32_t *out) {
    PRIM_PROLOGUE
    using V = Lv<LEVEL>;
    stage_bytes(gs.rhop, rhop + (size_t)item * 64, 64, lane);
    __syncwarp();
    int32_t *o = out + (size_t)item * V::L * N;
    int32_t a[8], b[8];
    int j = 0;
    if (item % 3 == 2) {
        expand_mask_16<V::ZBITS, V::GAMMA1>(
            gs.rhop, kappa[item], V::L, [&](int s) { return o + s * N; }, ws.k16, ws.k16c, lane);
        return;
    }
    if (item % 3 == 1) {
        expand_mask_poly<V::ZBITS, V::GAMMA1>(gs.rhop, kappa[item], a, ws.sq, lane);
        store_l0(o, a, lane);
        expand_mask_pair<V::ZBITS, V::GAMMA1>(gs.rhop, kappa[item] + 1, kappa[item] + 2, a, b, ws.sq, ws.sq2,
                                              lane);
        store_l0(o + N, a, lane);
        store_l0(o + 2 * N, b, lane);
        j = 3;
    }
    while (V::L - j >= 3 || (j == 0 && V::L > 0)) {
        const int c = min(K6_STATES, V::L - j);
        int32_t *base = o + j * N;
        expand_mask_six<V::ZBITS, V::GAMMA1>(
            gs.rhop, kappa[item] + j, c, [&](int g) { return base + g * N; }, ws.kst, ws.kpi(), ws.win, lane);
        j += c;
    }
    for (; j < V::L; ++j) {
        expand_mask_poly<V::ZBITS, V::GAMMA1>(gs.rhop, kappa[item] + j, a, ws.sq, lane);
        store_l0(o + j * N, a, lane);
    }
}

template <int LEVEL>
__global__ void k_test_sample_in_ball(int n, const uint8_t *ct, int32_t *out) {
    PRIM_PROLOGUE
    using V = Lv<LEVEL>;
    stage_bytes(gs.ctilde, ct + (size_t)item * 32, 32, lane);
    __syncwarp();
    sample_in_ball<V::TAU>(gs.ctilde, ws.buf, ws.sq, lane);
    int32_t a[8];
    read_buf_l0(a, ws.buf, lane);
    store_l0(out + (size_t)item * N, a, lane);
}

// SampleInBall over a given byte stream of `blocks` 136-byte blocks per item
// (the first starting with the 8 sign bytes) instead of SHAKE256(c~), so that
// tests can feed streams that reject many bytes and cross block boundaries.
template <int LEVEL>
__global__ void k_test_sib_stream(int n, const uint8_t *stream, int blocks, int32_t *out) {
    PRIM_PROLOGUE
    using V = Lv<LEVEL>;
    const uint8_t *src = stream + (size_t)item * blocks * 136;
    for (int i = lane; i < 136; i += 32) ws.sq[i] = src[i];
    __syncwarp();
    int next = 1;
    sample_in_ball_blocks<V::TAU>(
        ws.buf, ws.sq,
        [&](uint8_t *dst) {
            const uint8_t *b = src + (size_t)min(next, blocks - 1) * 136;   // past the end: repeat the last
            for (int i = lane; i < 136; i += 32) dst[i] = b[i];
            ++next;
        },
        lane);
    int32_t a[8];
    read_buf_l0(a, ws.buf, lane);
    store_l0(out + (size_t)item * N, a, lane);
}

template <int LEVEL>
__global__ void k_test_rounding(int n, const int32_t *r, const int32_t *z, const uint8_t *h, int32_t *out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t v = r[i], a1, a0;
    int32_t *o = out + (size_t)i * 6;
    power2round(v, a1, a0);
    o[0] = a1;
    o[1] = a0;
    decompose<LEVEL>(v, a1, a0);
    o[2] = a1;
    o[3] = a0;
    o[4] = make_hint<LEVEL>(z[i], v);
    o[5] = use_hint<LEVEL>(h[i], v);
}

template <class Kern, class... Args>
static cudaError_t launch_prim(Kern kern, int n, cudaStream_t s, Args... args) {
    if (n <= 0) return cudaSuccess;
    size_t smem = cta_bytes(PRIM_WARPS, 1);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<(n + PRIM_WARPS - 1) / PRIM_WARPS, PRIM_WARPS * 32, smem, s>>>(n, args...);
    return cudaGetLastError();
}

#define BY_LEVEL(KERN, ...)                                            \
    switch (level) {                                                   \
        case 2: return launch_prim(KERN<2>, n, s, __VA_ARGS__);        \
        case 3: return launch_prim(KERN<3>, n, s, __VA_ARGS__);        \
        case 5: return launch_prim(KERN<5>, n, s, __VA_ARGS__);        \
    }                                                                  \
    return cudaErrorInvalidValue;

cudaError_t launch_test_shake(int kind, int n, const uint8_t *in, const uint64_t *off, uint8_t *out, int outlen,
                              cudaStream_t s) {
    return launch_prim(k_test_shake, n, s, kind == 128 ? 168 : 136, in, off, out, outlen);
}
cudaError_t launch_test_k16_rider(int n, const uint8_t *in, const uint64_t *off, const int32_t *perms, uint8_t *out,
                                  cudaStream_t s) {
    return launch_prim(k_test_k16_rider, n, s, in, off, perms, out);
}
cudaError_t launch_test_k16_chain_rider(int n, const uint8_t *in, const uint64_t *off, const int32_t *perms,
                                        const int32_t *step, uint8_t *out, cudaStream_t s) {
    return launch_prim(k_test_k16_chain_rider, n, s, in, off, perms, step, out);
}
cudaError_t launch_test_ntt(int n, const int32_t *in, int32_t *out, int inverse, cudaStream_t s) {
    return launch_prim(k_test_ntt, n, s, in, out, inverse);
}
cudaError_t launch_test_keccak_f(int form, int states, const uint64_t *in, uint64_t *out, cudaStream_t s) {
    const int items = (states + form - 1) / form;
    switch (form) {
        case 1: return launch_prim(k_test_keccak_f<1>, items, s, states, in, out);
        case 2: return launch_prim(k_test_keccak_f<2>, items, s, states, in, out);
        case 6: return launch_prim(k_test_keccak_f<6>, items, s, states, in, out);
        case 16: return launch_prim(k_test_keccak_f<16>, items, s, states, in, out);
    }
    return cudaErrorInvalidValue;
}
template <int LEVEL>
static cudaError_t launch_t0_variant(int variant, int n, const uint8_t *sk, int32_t *tmp, int32_t *out,
                                     cudaStream_t s) {
    switch (variant) {
        case 0: {
            cudaError_t e = launch_prim(k_test_t0_unpack<LEVEL>, n, s, sk, tmp);
            return e != cudaSuccess ? e : launch_prim(k_test_t0_ntt<LEVEL>, n, s, (const int32_t *)tmp, out);
        }
        case 1: return launch_prim(k_test_t0_fused_gmem<LEVEL>, n, s, sk, tmp, out);
        case 2: return launch_prim(k_test_t0_registers<LEVEL, true>, n, s, sk, out);
        case 3: return launch_prim(k_test_t0_registers<LEVEL, false>, n, s, sk, out);
    }
    return cudaErrorInvalidValue;
}
cudaError_t launch_test_t0_ntt(int level, int variant, int n, const uint8_t *sk, int32_t *tmp, int32_t *out,
                               cudaStream_t s) {
    switch (level) {
        case 2: return launch_t0_variant<2>(variant, n, sk, tmp, out, s);
        case 3: return launch_t0_variant<3>(variant, n, sk, tmp, out, s);
        case 5: return launch_t0_variant<5>(variant, n, sk, tmp, out, s);
    }
    return cudaErrorInvalidValue;
}
cudaError_t launch_test_expand_a(int level, int n, const uint8_t *rho, int32_t *out, cudaStream_t s) {
    BY_LEVEL(k_test_expand_a, rho, out)
}
cudaError_t launch_test_expand_s(int level, int n, const uint8_t *rhop, int32_t *out, cudaStream_t s) {
    BY_LEVEL(k_test_expand_s, rhop, out)
}
cudaError_t launch_test_expand_mask(int level, int n, const uint8_t *rhop, const int32_t *kappa, int32_t *out,
                                    cudaStream_t s) {
    BY_LEVEL(k_test_expand_mask, rhop, kappa, out)
}
cudaError_t launch_test_sample_in_ball(int level, int n, const uint8_t *ct, int32_t *out, cudaStream_t s) {
    BY_LEVEL(k_test_sample_in_ball, ct, out)
}
cudaError_t launch_test_sib_stream(int level, int n, const uint8_t *stream, int blocks, int32_t *out,
                                   cudaStream_t s) {
    BY_LEVEL(k_test_sib_stream, stream, blocks, out)
}
cudaError_t launch_test_rounding(int level, int n, const int32_t *r, const int32_t *z, const uint8_t *h,
                                 int32_t *out, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    int grid = (n + 255) / 256;
    switch (level) {
        case 2: k_test_rounding<2><<<grid, 256, 0, s>>>(n, r, z, h, out); break;
        case 3: k_test_rounding<3><<<grid, 256, 0, s>>>(n, r, z, h, out); break;
        case 5: k_test_rounding<5><<<grid, 256, 0, s>>>(n, r, z, h, out); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace dil

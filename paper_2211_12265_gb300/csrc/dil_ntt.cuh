// Warp-level 256-point negacyclic NTT / INTT mod q (section 2.2; section 3.2 of
// arXiv 2211.12265, single-warp form: each thread holds 8 coefficients in
// registers, three levels run in registers between two shared-memory exchanges,
// and the exchanges are padded so that no two lanes of a warp hit one bank).
//
// Output order (round-3 reading): index j holds f(zeta^(2 brv8(j) + 1)),
// zeta = 1753.  Twiddles are zeta^brv8(k) (forward) and zeta^-brv8(k)
// (inverse) in Montgomery form (times 2^32 mod q).
//
// Register layouts of the 8 values r[0..7] held by lane t:
//   L0: coefficient t + 32 m           (natural order, coalesced loads)
//   L1: coefficient 32 (t>>2) + (t&3) + 4 m
//   L2: coefficient 8 t + m            (two 16-byte vector loads)
// Exchange L0<->L1 uses the padded index i + 4 (i >> 5) (4 words per 32),
// exchange L1<->L2 uses i + (i >> 3) (1 word per 8); both are conflict-free for
// the write and the read side.
#pragma once
#include "dil_arith.cuh"

namespace dil {

struct Zetas {
    int32_t z[256];   // zeta^brv8(k) * 2^32 mod q, centred
    int32_t iz[256];  // zeta^-brv8(k) * 2^32 mod q, centred
};

namespace detail {
constexpr int64_t cpow(int64_t b, int64_t e) {
    int64_t r = 1;
    b %= Q;
    if (b < 0) b += Q;
    while (e) {
        if (e & 1) r = r * b % Q;
        b = b * b % Q;
        e >>= 1;
    }
    return r;
}
constexpr unsigned cbrv8(unsigned j) {
    unsigned r = 0;
    for (int b = 0; b < 8; ++b)
        if (j & (1u << b)) r |= 1u << (7 - b);
    return r;
}
constexpr int64_t MONT = (int64_t(1) << 32) % Q;  // 2^32 mod q
constexpr int32_t centre(int64_t v) {
    v %= Q;
    if (v < 0) v += Q;
    return (int32_t)(v > (Q - 1) / 2 ? v - Q : v);
}
constexpr Zetas make_zetas() {
    Zetas t{};
    for (unsigned k = 0; k < 256; ++k) {
        int64_t e = cbrv8(k);
        t.z[k] = centre(cpow(1753, e) * MONT);
        t.iz[k] = centre(cpow(1753, 512 - e) * MONT);   // zeta^512 = 1
    }
    return t;
}
}  // namespace detail

static __constant__ Zetas c_zetas = detail::make_zetas();

// Final INTT level scale: mont(F, x) = x * 2^32 / 256 and
// mont(G, x) = x * zeta^-brv8(1) * 2^32 / 256 (mod q).
constexpr int32_t NTT_F = detail::centre(detail::MONT * detail::MONT % Q * detail::cpow(256, Q - 2));
constexpr int32_t NTT_G = detail::centre((int64_t)NTT_F * detail::cpow(1753, 512 - detail::cbrv8(1)) % Q);

__device__ __forceinline__ void ct_bfly(int32_t &a, int32_t &b, int32_t z) {
    int32_t t = mont_mul(z, b);
    b = a - t;
    a = a + t;
}

__device__ __forceinline__ void gs_bfly(int32_t &a, int32_t &b, int32_t z) {
    int32_t t = a;
    a = t + b;
    b = mont_mul(z, t - b);
}

// Shared-memory accesses by 32-bit shared-window address (the out-of-line
// transforms receive addresses, not generic pointers).  Exchange-buffer
// accesses are ordered (volatile, memory clobber); twiddle loads read
// constant data and may be scheduled freely.
__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void sts32(uint32_t a, int32_t v) {
    asm volatile("st.shared.b32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}
__device__ __forceinline__ int32_t lds32(uint32_t a) {
    int32_t v;
    asm volatile("ld.shared.b32 %0, [%1];" : "=r"(v) : "r"(a) : "memory");
    return v;
}
__device__ __forceinline__ int32_t ldz32(uint32_t a) {
    int32_t v;
    asm("ld.shared.b32 %0, [%1];" : "=r"(v) : "r"(a));
    return v;
}
__device__ __forceinline__ int2 ldz64(uint32_t a) {
    int2 v;
    asm("ld.shared.v2.b32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "r"(a));
    return v;
}
__device__ __forceinline__ int4 ldz128(uint32_t a) {
    int4 v;
    asm("ld.shared.v4.b32 {%0, %1, %2, %3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(a));
    return v;
}

// Eight coefficients of one lane, passed by value to the out-of-line transforms.
struct Poly8 {
    int32_t v[8];
};

// Forward NTT.  In: L0, |r| < q.  Out: L2, |r| < 9q, unscaled.  buf: the
// warp's exchange buffer (288 words), zt: the forward twiddles (shared).
// Out of line: one copy of the code serves every call site, which keeps the
// fused kernels' instruction footprint small.
static __device__ __noinline__ Poly8 ntt_fwd_impl(Poly8 p, uint32_t buf, uint32_t zt) {
    const int lane = threadIdx.x & 31;
    int32_t *r = p.v;
    // level 1 (len 128): pairs (m, m+4)
    {
        const int32_t z = c_zetas.z[1];
#pragma unroll
        for (int m = 0; m < 4; ++m) ct_bfly(r[m], r[m + 4], z);
    }
    // level 2 (len 64): pairs (m, m+2), twiddle 2 + m/4
    ct_bfly(r[0], r[2], c_zetas.z[2]);
    ct_bfly(r[1], r[3], c_zetas.z[2]);
    ct_bfly(r[4], r[6], c_zetas.z[3]);
    ct_bfly(r[5], r[7], c_zetas.z[3]);
    // level 3 (len 32): pairs (m, m+1), twiddle 4 + m/2
    ct_bfly(r[0], r[1], c_zetas.z[4]);
    ct_bfly(r[2], r[3], c_zetas.z[5]);
    ct_bfly(r[4], r[5], c_zetas.z[6]);
    ct_bfly(r[6], r[7], c_zetas.z[7]);
    // exchange L0 -> L1
#pragma unroll
    for (int m = 0; m < 8; ++m) sts32(buf + 4 * (lane + 36 * m), r[m]);
    __syncwarp();
    const int b = lane >> 2;
    const uint32_t base1 = buf + 4 * (36 * b + (lane & 3));
#pragma unroll
    for (int m = 0; m < 8; ++m) r[m] = lds32(base1 + 16 * m);
    __syncwarp();
    // level 4 (len 16): pairs (m, m+4), twiddle 8 + b
    {
        const int32_t z = ldz32(zt + 4 * (8 + b));
#pragma unroll
        for (int m = 0; m < 4; ++m) ct_bfly(r[m], r[m + 4], z);
    }
    // level 5 (len 8): pairs (m, m+2), twiddles 16 + 2b + {0, 1}
    {
        const int2 z = ldz64(zt + 4 * (16 + 2 * b));
        ct_bfly(r[0], r[2], z.x);
        ct_bfly(r[1], r[3], z.x);
        ct_bfly(r[4], r[6], z.y);
        ct_bfly(r[5], r[7], z.y);
    }
    // level 6 (len 4): pairs (m, m+1), twiddles 32 + 4b + {0..3}
    {
        const int4 z = ldz128(zt + 4 * (32 + 4 * b));
        ct_bfly(r[0], r[1], z.x);
        ct_bfly(r[2], r[3], z.y);
        ct_bfly(r[4], r[5], z.z);
        ct_bfly(r[6], r[7], z.w);
    }
    // exchange L1 -> L2
#pragma unroll
    for (int m = 0; m < 8; ++m) sts32(base1 + 4 * (4 * m + (m >> 1)), r[m]);
    __syncwarp();
#pragma unroll
    for (int m = 0; m < 8; ++m) r[m] = lds32(buf + 4 * (9 * lane + m));
    __syncwarp();
    // level 7 (len 2): pairs (m, m+2), twiddles 64 + 2t + {0, 1} (one 8-byte
    // load per lane: a half-warp reads 128 contiguous bytes, conflict-free)
    {
        const int2 z = ldz64(zt + 4 * (64 + 2 * lane));
        ct_bfly(r[0], r[2], z.x);
        ct_bfly(r[1], r[3], z.x);
        ct_bfly(r[4], r[6], z.y);
        ct_bfly(r[5], r[7], z.y);
    }
    // level 8 (len 1): pairs (m, m+1), twiddles 128 + 4t + {0..3} (16-byte load)
    {
        const int4 z = ldz128(zt + 4 * (128 + 4 * lane));
        ct_bfly(r[0], r[1], z.x);
        ct_bfly(r[2], r[3], z.y);
        ct_bfly(r[4], r[5], z.z);
        ct_bfly(r[6], r[7], z.w);
    }
    return p;
}

// Inverse NTT.  In: L2, |r| < q.  Out: L0, |r| < q, equal to INTT(in) * 2^32,
// so it turns pointwise Montgomery products into plain coefficients.
// izt: the inverse twiddles in shared memory.
static __device__ __noinline__ Poly8 ntt_inv_impl(Poly8 p, uint32_t buf, uint32_t izt) {
    const int lane = threadIdx.x & 31;
    int32_t *r = p.v;
    // len 1: pairs (m, m+1), twiddles 128 + 4t + {0..3}
    {
        const int4 z = ldz128(izt + 4 * (128 + 4 * lane));
        gs_bfly(r[0], r[1], z.x);
        gs_bfly(r[2], r[3], z.y);
        gs_bfly(r[4], r[5], z.z);
        gs_bfly(r[6], r[7], z.w);
    }
    // len 2: pairs (m, m+2), twiddles 64 + 2t + {0, 1}
    {
        const int2 z = ldz64(izt + 4 * (64 + 2 * lane));
        gs_bfly(r[0], r[2], z.x);
        gs_bfly(r[1], r[3], z.x);
        gs_bfly(r[4], r[6], z.y);
        gs_bfly(r[5], r[7], z.y);
    }
    // exchange L2 -> L1
#pragma unroll
    for (int m = 0; m < 8; ++m) sts32(buf + 4 * (9 * lane + m), r[m]);
    __syncwarp();
    const int b = lane >> 2;
    const uint32_t base1 = buf + 4 * (36 * b + (lane & 3));
#pragma unroll
    for (int m = 0; m < 8; ++m) r[m] = lds32(base1 + 4 * (4 * m + (m >> 1)));
    __syncwarp();
    // len 4: pairs (m, m+1), twiddles 32 + 4b + {0..3}
    {
        const int4 z = ldz128(izt + 4 * (32 + 4 * b));
        gs_bfly(r[0], r[1], z.x);
        gs_bfly(r[2], r[3], z.y);
        gs_bfly(r[4], r[5], z.z);
        gs_bfly(r[6], r[7], z.w);
    }
    // len 8: pairs (m, m+2), twiddles 16 + 2b + {0, 1}
    {
        const int2 z = ldz64(izt + 4 * (16 + 2 * b));
        gs_bfly(r[0], r[2], z.x);
        gs_bfly(r[1], r[3], z.x);
        gs_bfly(r[4], r[6], z.y);
        gs_bfly(r[5], r[7], z.y);
    }
    // len 16: pairs (m, m+4), twiddle 8 + b
    {
        const int32_t z = ldz32(izt + 4 * (8 + b));
#pragma unroll
        for (int m = 0; m < 4; ++m) gs_bfly(r[m], r[m + 4], z);
    }
    // exchange L1 -> L0
#pragma unroll
    for (int m = 0; m < 8; ++m) sts32(base1 + 16 * m, r[m]);
    __syncwarp();
#pragma unroll
    for (int m = 0; m < 8; ++m) r[m] = lds32(buf + 4 * (lane + 36 * m));
    __syncwarp();
    // len 32: pairs (m, m+1), twiddle 4 + m/2
    gs_bfly(r[0], r[1], c_zetas.iz[4]);
    gs_bfly(r[2], r[3], c_zetas.iz[5]);
    gs_bfly(r[4], r[5], c_zetas.iz[6]);
    gs_bfly(r[6], r[7], c_zetas.iz[7]);
    // len 64: pairs (m, m+2), twiddle 2 + m/4
    gs_bfly(r[0], r[2], c_zetas.iz[2]);
    gs_bfly(r[1], r[3], c_zetas.iz[2]);
    gs_bfly(r[4], r[6], c_zetas.iz[3]);
    gs_bfly(r[5], r[7], c_zetas.iz[3]);
    // len 128 with the factor 2^32/n folded in (twiddle 1)
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        int32_t a = r[m], c = r[m + 4];
        r[m] = mont_mul(NTT_F, a + c);
        r[m + 4] = mont_mul(NTT_G, a - c);
    }
    return p;
}

__device__ __forceinline__ void ntt_fwd(int32_t r[8], int32_t *buf, const int32_t *zt, int lane) {
    (void)lane;
    Poly8 p;
#pragma unroll
    for (int m = 0; m < 8; ++m) p.v[m] = r[m];
    p = ntt_fwd_impl(p, smem_addr(buf), smem_addr(zt));
#pragma unroll
    for (int m = 0; m < 8; ++m) r[m] = p.v[m];
}

__device__ __forceinline__ void ntt_inv(int32_t r[8], int32_t *buf, const int32_t *izt, int lane) {
    (void)lane;
    Poly8 p;
#pragma unroll
    for (int m = 0; m < 8; ++m) p.v[m] = r[m];
    p = ntt_inv_impl(p, smem_addr(buf), smem_addr(izt));
#pragma unroll
    for (int m = 0; m < 8; ++m) r[m] = p.v[m];
}

// Loads the twiddle tables into shared memory (whole block participates).
__device__ __forceinline__ void load_zetas(int32_t *zt, int32_t *izt) {
    for (int i = threadIdx.x; i < 256; i += blockDim.x) {
        zt[i] = c_zetas.z[i];
        izt[i] = c_zetas.iz[i];
    }
}

// Transposes 8 values from L0 to 8 consecutive coefficients (8 lane + m).
__device__ __forceinline__ void l0_to_seq(int32_t v[8], int32_t *buf, int lane) {
#pragma unroll
    for (int m = 0; m < 8; ++m) buf[lane + 36 * m + (lane >> 3)] = v[m];
    __syncwarp();
#pragma unroll
    for (int m = 0; m < 8; ++m) v[m] = buf[9 * lane + m];
    __syncwarp();
}

}  // namespace dil

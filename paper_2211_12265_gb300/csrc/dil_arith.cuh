// Coefficient arithmetic mod q = 8380417 (section 2.2 "Ring Arithmetic") and the
// bits-extraction / hint functions (section 2.3 "Bits Extraction and Hints").
#pragma once
#include "dil_params.cuh"

namespace dil {

// Signed Montgomery product a*b*2^-32 mod q.  For |a*b| < 2^31 q the result
// lies in (-q, q).  The low words of a*b and u*q agree by the choice of
// u = lo(a*b) * q^-1 mod 2^32, so the difference of the high words is exact.
__device__ __forceinline__ int32_t mont_mul(int32_t a, int32_t b) {
    int32_t lo = a * b;
    int32_t hi = __mulhi(a, b);
    int32_t u = lo * QINV;
    return hi - __mulhi(u, Q);
}

// Representative of a (|a| < 2^31) with |result| <= 6291200 < q:
// a = t 2^23 + e, |e| <= 2^22, and 2^23 - q = 8191, so a - t q = e + 8191 t.
__device__ __forceinline__ int32_t reduce_q(int32_t a) {
    int32_t t = (a + (1 << 22)) >> 23;
    return a - t * Q;
}

// (-q, q) -> [0, q)
__device__ __forceinline__ int32_t to_canonical(int32_t a) { return a + ((a >> 31) & Q); }

// [0, q) -> centred (-(q-1)/2, (q-1)/2]
__device__ __forceinline__ int32_t to_centred(int32_t a) { return a - (((Q - 1) / 2 - a) >> 31 & Q); }

// any |a| < 2q -> centred representative
__device__ __forceinline__ int32_t centre_small(int32_t a) {
    a = to_canonical(a);                 // [0, 2q) for a in (-q, 2q)
    a -= (a >= Q) ? Q : 0;
    return to_centred(a);
}

__device__ __forceinline__ int32_t iabs(int32_t a) { return a < 0 ? -a : a; }

// Power2Round on r in [0, q): r1 = ceil((r - 2^12) / 2^13), r0 = r - r1 2^13 in
// (-2^12, 2^12].
__device__ __forceinline__ void power2round(int32_t r, int32_t &r1, int32_t &r0) {
    r1 = (r + (1 << (D - 1)) - 1) >> D;
    r0 = r - (r1 << D);
}

// Decompose on r in [0, q) with alpha = 2 gamma2: r0 = r mod+- alpha in
// (-gamma2, gamma2], r1 = (r - r0)/alpha; when r - r0 = q - 1 the output is
// (0, r0 - 1).  r1 = ceil((r - gamma2)/alpha) = floor((r + gamma2 - 1)/alpha).
template <int LEVEL>
__device__ __forceinline__ void decompose(int32_t r, int32_t &r1, int32_t &r0) {
    using V = Lv<LEVEL>;
    uint32_t h = (uint32_t)(r + V::GAMMA2 - 1) / (uint32_t)V::ALPHA;
    int32_t l = r - (int32_t)h * V::ALPHA;
    bool wrap = (h == (uint32_t)V::M_HI);
    r1 = wrap ? 0 : (int32_t)h;
    r0 = wrap ? l - 1 : l;
}

template <int LEVEL>
__device__ __forceinline__ int32_t highbits(int32_t r) {
    using V = Lv<LEVEL>;
    uint32_t h = (uint32_t)(r + V::GAMMA2 - 1) / (uint32_t)V::ALPHA;
    return (h == (uint32_t)V::M_HI) ? 0 : (int32_t)h;
}

// MakeHint(z, r) = [HighBits(r) != HighBits(r + z)], both inputs in [0, q).
template <int LEVEL>
__device__ __forceinline__ int make_hint(int32_t z, int32_t r) {
    int32_t s = r + z;
    s -= (s >= Q) ? Q : 0;
    return highbits<LEVEL>(r) != highbits<LEVEL>(s);
}

// UseHint(h, r), r in [0, q): r1 if h = 0, else r1 +- 1 mod+ m by the sign of r0.
template <int LEVEL>
__device__ __forceinline__ int32_t use_hint(int h, int32_t r) {
    using V = Lv<LEVEL>;
    int32_t r1, r0;
    decompose<LEVEL>(r, r1, r0);
    if (!h) return r1;
    if (r0 > 0) return (r1 == V::M_HI - 1) ? 0 : r1 + 1;
    return (r1 == 0) ? V::M_HI - 1 : r1 - 1;
}

}  // namespace dil

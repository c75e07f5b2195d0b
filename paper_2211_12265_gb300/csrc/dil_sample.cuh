// Warp-level samplers (section 2.3 "Sampling"; section 3.4 / Alg 4 of
// arXiv 2211.12265: rejection sampling with a warp vote of the accept bits, an
// inclusive popcount for each lane's write offset and a running count).
// The *_pair variants run two independent sponges through the interleaved
// permutation (keccak_f2), for instruction-level parallelism.
#pragma once
#include "dil_keccak.cuh"
#include "dil_keccak6.cuh"
#include "dil_keccak16.cuh"
#include "dil_ntt.cuh"

namespace dil {

__device__ __forceinline__ uint32_t lanemask_lt(int lane) { return (1u << lane) - 1u; }

// Upper bound on squeezed blocks in any rejection sampler: the samplers need
// 1-6 blocks except with negligible probability; the bound only guarantees
// that no input can make a warp loop forever.
constexpr int MAX_SQUEEZE_BLOCKS = 64;

// Reads a little-endian field of `bits` (<= 25) bits starting at bit `pos`
// from a 4-byte-aligned shared buffer readable one word beyond the field.
__device__ __forceinline__ uint32_t get_field(const uint8_t *buf, int pos, int bits) {
    const uint32_t *w = reinterpret_cast<const uint32_t *>(buf);
    uint32_t v = __funnelshift_r(w[pos >> 5], w[(pos >> 5) + 1], pos & 31);
    return v & ((1u << bits) - 1u);
}

// ---------------------------------------------------------------- ExpandA
// A^_ij from SHAKE128(rho || j || i).  Candidates are 3-byte little-endian
// words with the top bit cleared, kept when < q, in stream order; coefficient
// c is written to buf[c + (c >> 3)] (layout for an L2 read).

// Rejection step over one squeezed 168-byte block (56 candidates).
__device__ __forceinline__ int expand_a_block(const uint8_t *sq, int32_t *buf, int ctr, int lane) {
#pragma unroll
    for (int rnd = 0; rnd < 2; ++rnd) {
        int c = rnd * 32 + lane;
        bool valid = c < 56;
        uint32_t v = valid ? (get_field(sq, 24 * c, 24) & 0x7FFFFFu) : 0u;
        bool acc = valid && v < (uint32_t)Q;
        uint32_t mask = __ballot_sync(FULL, acc);
        int pos = ctr + __popc(mask & lanemask_lt(lane));
        if (acc && pos < N) buf[pos + (pos >> 3)] = (int32_t)v;
        ctr += __popc(mask);
    }
    return ctr;
}

// rho: 32 bytes in shared memory (8-byte aligned); sq: >= 176-byte scratch.
__device__ __forceinline__ void expand_a_poly(const uint8_t *rho, int i, int j, int32_t *buf, uint8_t *sq,
                                              int lane) {
    uint32_t lo, hi;
    absorb_seed(lo, hi, rho, 4, (uint32_t)j | ((uint32_t)i << 8), 2, 168, lane);
    int ctr = 0;
#pragma unroll 1
    for (int blk = 0; blk < MAX_SQUEEZE_BLOCKS; ++blk) {
        squeeze_words(lo, hi, sq, 21, lane);
        __syncwarp();
        ctr = expand_a_block(sq, buf, ctr, lane);
        __syncwarp();
        if (ctr >= N) break;
        keccak_f(lo, hi);
    }
}

// A^_{i0 j0} into buf0 and A^_{i1 j1} into buf1.
__device__ __forceinline__ void expand_a_pair(const uint8_t *rho, int i0, int j0, int i1, int j1, int32_t *buf0,
                                              int32_t *buf1, uint8_t *sq0, uint8_t *sq1, int lane) {
    uint32_t lo0, hi0, lo1, hi1;
    seed_words(lo0, hi0, rho, 4, (uint32_t)j0 | ((uint32_t)i0 << 8), 2, 168, lane);
    seed_words(lo1, hi1, rho, 4, (uint32_t)j1 | ((uint32_t)i1 << 8), 2, 168, lane);
    keccak_f2(lo0, hi0, lo1, hi1);
    int c0 = 0, c1 = 0;
#pragma unroll 1
    for (int blk = 0; blk < MAX_SQUEEZE_BLOCKS; ++blk) {
        squeeze_words(lo0, hi0, sq0, 21, lane);
        squeeze_words(lo1, hi1, sq1, 21, lane);
        __syncwarp();
        if (c0 < N) c0 = expand_a_block(sq0, buf0, c0, lane);
        if (c1 < N) c1 = expand_a_block(sq1, buf1, c1, lane);
        __syncwarp();
        if (c0 >= N && c1 >= N) break;
        keccak_f2(lo0, hi0, lo1, hi1);
    }
}

// Six-instance ExpandA: polynomials p0 .. p0 + count - 1 (count <= 6) of A^
// (p = i l + j), rejection-sampled with the same warp vote straight from the
// states' squeezed blocks into global memory, coefficient c of polynomial p at
// out[(p - p0) 256 + c] (index order).  rho: 32 bytes of shared memory.
template <int L>
__device__ __forceinline__ void expand_a_six(const uint8_t *rho, int p0, int count, int32_t *out, uint32_t *kst,
                                             uint32_t *kpi, int lane) {
    keccak6_seed(
        kst, reinterpret_cast<const uint32_t *>(rho), 8,
        [&](int g) { const int p = p0 + g; return (uint32_t)(p % L) | ((uint32_t)(p / L) << 8) | (0x1Fu << 16); },
        count, 168, lane);
    keccak6_permute(kst, kpi);
    int mine = 0;   // lane g < count: coefficients accepted so far for instance g
#pragma unroll 1
    for (int blk = 0; blk < MAX_SQUEEZE_BLOCKS; ++blk) {
#pragma unroll 1
        for (int g = 0; g < count; ++g) {
            int c = __shfl_sync(FULL, mine, g);
            if (c >= N) continue;
            const uint8_t *sq = reinterpret_cast<const uint8_t *>(kst + K6_WORDS * g);
            int32_t *dst = out + g * N;
#pragma unroll
            for (int rnd = 0; rnd < 2; ++rnd) {
                const int k = rnd * 32 + lane;
                const bool valid = k < 56;
                const uint32_t v = valid ? (get_field(sq, 24 * k, 24) & 0x7FFFFFu) : 0u;
                const bool acc = valid && v < (uint32_t)Q;
                const uint32_t mask = __ballot_sync(FULL, acc);
                const int pos = c + __popc(mask & lanemask_lt(lane));
                if (acc && pos < N) dst[pos] = (int32_t)v;
                c += __popc(mask);
            }
            if (lane == g) mine = c;
        }
        if (!__any_sync(FULL, lane < count && mine < N)) break;
        keccak6_permute(kst, kpi);
    }
}

// Sixteen-instance ExpandA: polynomials p0 .. p0 + count - 1 (count <=
// Rider::KEEP), written like expand_a_six.  The candidates of two instances
// are voted on at once, one per half-warp (4 x 16 candidate slots for a
// block's 56).  `rider` may carry a hash in the last instance (K16Rider).
template <int L, class Rider>
__device__ __forceinline__ void expand_a_16(const uint8_t *rho, int p0, int count, int32_t *out, uint32_t *kst,
                                            int lane, Rider &rider) {
    keccak16_seed(
        kst, reinterpret_cast<const uint32_t *>(rho), 8,
        [&](int s) { const int p = p0 + s; return (uint32_t)(p % L) | ((uint32_t)(p / L) << 8) | (0x1Fu << 16); },
        count, 168, lane, Rider::KEEP);
    rider.before(kst, lane);
    keccak16_permute(kst);
    rider.after(kst, lane);
    const int half = lane >> 4, hl = lane & 15;
    const uint32_t below = (1u << hl) - 1u;
    int mine = 0;   // lane s < count: coefficients accepted so far for instance s
#pragma unroll 1
    for (int blk = 0; blk < MAX_SQUEEZE_BLOCKS; ++blk) {
#pragma unroll 1
        for (int q = 0; 2 * q < count; ++q) {
            const int s = 2 * q + half;
            int c = __shfl_sync(FULL, mine, s);
            const bool live = s < count && c < N;
            if (!__any_sync(FULL, live)) continue;
            int32_t *dst = out + s * N;
#pragma unroll
            for (int rnd = 0; rnd < 4; ++rnd) {
                const int k = rnd * 16 + hl;
                const int pos = 24 * k, w = pos >> 5;
                const uint32_t lo = kst[k16_word(s, w)], hi = kst[k16_word(s, w + 1)];
                const uint32_t v = __funnelshift_r(lo, hi, pos & 31) & 0x7FFFFFu;
                const bool acc = live && k < 56 && v < (uint32_t)Q;
                const uint32_t m = __ballot_sync(FULL, acc) >> (16 * half) & 0xFFFFu;
                const int at = c + __popc(m & below);
                if (acc && at < N) dst[at] = (int32_t)v;
                c += __popc(m);
            }
            const int c_new = __shfl_sync(FULL, c, (lane & 1) << 4);
            if ((lane >> 1) == q) mine = c_new;
        }
        if (!__any_sync(FULL, lane < count && mine < N)) break;
        __syncwarp();
        rider.before(kst, lane);
        keccak16_permute(kst);
        rider.after(kst, lane);
    }
    __syncwarp();
}

template <int L>
__device__ __forceinline__ void expand_a_16(const uint8_t *rho, int p0, int count, int32_t *out, uint32_t *kst,
                                            int lane) {
    K16NoRider none;
    expand_a_16<L>(rho, p0, count, out, kst, lane, none);
}

// Sixteen-instance ExpandMask: y for nonces nonce0 .. nonce0 + count - 1
// (count <= 16), coefficient c of instance s at dst(s)[c] (natural order).
// Fields whose last bit lies in the current block are extracted after each
// permutation; the previous block's last lane (8 bytes, saved in `carry`, 32
// words) supplies the start of a field that straddles two blocks.
template <int ZBITS, int32_t GAMMA1, class Dst>
__device__ __forceinline__ void expand_mask_16(const uint8_t *rhop, int nonce0, int count, Dst dst, uint32_t *kst,
                                               uint32_t *carry, int lane) {
    keccak16_seed(
        kst, reinterpret_cast<const uint32_t *>(rhop), 16,
        [&](int s) { return ((uint32_t)(nonce0 + s) & 0xFFFFu) | (0x1Fu << 16); }, count, 136, lane);
    constexpr int BLOCKS = (N * ZBITS / 8 + 135) / 136;
    const int half = lane >> 4, hl = lane & 15;
    const uint32_t kst_a = smem_addr(kst), carry_a = smem_addr(carry);
#pragma unroll 1
    for (int b = 0; b < BLOCKS; ++b) {
        if (b) {
            carry[lane] = kst[k16_slot(16, lane)];   // lane 16: the block's last 8 bytes
            __syncwarp();
        }
        keccak16_permute(kst);
        const int c_lo = (1088 * b) / ZBITS;
        const int c_hi = min(N, (1088 * (b + 1)) / ZBITS);
#pragma unroll 1
        for (int q = 0; 2 * q < count; ++q) {
            const int s = 2 * q + half;
            if (s >= count) continue;
            int32_t *out = dst(s);
            for (int c = c_lo + hl; c < c_hi; c += 16) {
                // window word u: u < 2 the carry, else block word u - 2
                const int pos = ZBITS * c - 1088 * b + 64, u = pos >> 5;
                const uint32_t a0 = u < 2 ? carry_a + 4 * (2 * s + u) : kst_a + 4 * k16_word(s, u - 2);
                const uint32_t a1 = u + 1 < 2 ? carry_a + 4 * (2 * s + u + 1) : kst_a + 4 * k16_word(s, u - 1);
                const uint32_t f = __funnelshift_r(lds32(a0), lds32(a1), pos & 31) & ((1u << ZBITS) - 1u);
                out[c] = GAMMA1 - (int32_t)f;
            }
        }
        __syncwarp();
    }
}

// Six-instance ExpandMask: y for nonces nonce0 .. nonce0 + count - 1
// (count <= 6), coefficient c of instance g's polynomial at dst(g)[c]
// (natural order).  After each permutation the 136-byte block is copied
// behind the last 8 bytes of the previous one into a per-instance window
// (win: 6 x 38 words), and the fields whose last bit lies in this block are
// extracted.
template <int ZBITS, int32_t GAMMA1, class Dst>
__device__ __forceinline__ void expand_mask_six(const uint8_t *rhop, int nonce0, int count, Dst dst,
                                                uint32_t *kst, uint32_t *kpi, uint32_t *win, int lane) {
    keccak6_seed(
        kst, reinterpret_cast<const uint32_t *>(rhop), 16,
        [&](int g) { return ((uint32_t)(nonce0 + g) & 0xFFFFu) | (0x1Fu << 16); }, count, 136, lane);
    constexpr int BLOCKS = (N * ZBITS / 8 + 135) / 136;
#pragma unroll 1
    for (int b = 0; b < BLOCKS; ++b) {
        keccak6_permute(kst, kpi);
        if (lane < 2 * K6_STATES) {   // carry: the previous block's last 8 bytes
            const int g = lane >> 1, k = lane & 1;
            win[38 * g + k] = win[38 * g + 34 + k];
        }
        __syncwarp();
        for (int w = lane; w < K6_STATES * 34; w += 32) {
            const int g = w / 34, k = w % 34;
            win[38 * g + 2 + k] = kst[K6_WORDS * g + k];
        }
        __syncwarp();
        const int c_lo = (1088 * b) / ZBITS;
        const int c_hi = min(N, (1088 * (b + 1)) / ZBITS);
#pragma unroll 1
        for (int g = 0; g < count; ++g) {
            const uint8_t *wb = reinterpret_cast<const uint8_t *>(win + 38 * g);
            int32_t *out = dst(g);
            for (int c = c_lo + lane; c < c_hi; c += 32)
                out[c] = GAMMA1 - (int32_t)get_field(wb, ZBITS * c - (1088 * b - 64), ZBITS);
        }
        __syncwarp();
    }
}

// ---------------------------------------------------------------- ExpandS
// One polynomial with coefficients in [-eta, eta] from SHAKE256(rho' || nonce);
// each byte gives two 4-bit candidates, low first.  Coefficient c is written
// to buf[c + 4 (c >> 5)] (layout for an L0 read).

template <int ETA>
__device__ __forceinline__ int expand_s_block(const uint8_t *sq, int32_t *buf, int ctr, int lane) {
#pragma unroll
    for (int rnd = 0; rnd < 5; ++rnd) {
        int c = rnd * 32 + lane;
        bool valid = c < 136;
        uint32_t byte = valid ? sq[c] : 0xFFu;
        uint32_t t0 = byte & 15u, t1 = byte >> 4;
        bool a0 = valid && (ETA == 2 ? t0 < 15u : t0 < 9u);
        bool a1 = valid && (ETA == 2 ? t1 < 15u : t1 < 9u);
        uint32_t m0 = __ballot_sync(FULL, a0), m1 = __ballot_sync(FULL, a1);
        uint32_t lt = lanemask_lt(lane);
        int pos0 = ctr + __popc(m0 & lt) + __popc(m1 & lt);
        int pos1 = pos0 + (a0 ? 1 : 0);
        if (a0 && pos0 < N) buf[pos0 + 4 * (pos0 >> 5)] = (ETA == 2) ? 2 - (int32_t)(t0 % 5u) : 4 - (int32_t)t0;
        if (a1 && pos1 < N) buf[pos1 + 4 * (pos1 >> 5)] = (ETA == 2) ? 2 - (int32_t)(t1 % 5u) : 4 - (int32_t)t1;
        ctr += __popc(m0) + __popc(m1);
    }
    return ctr;
}

template <int ETA>
__device__ __forceinline__ void expand_s_poly(const uint8_t *rhop, int nonce, int32_t *buf, uint8_t *sq, int lane) {
    uint32_t lo, hi;
    absorb_seed(lo, hi, rhop, 8, (uint32_t)nonce & 0xFFFFu, 2, 136, lane);
    int ctr = 0;
#pragma unroll 1
    for (int blk = 0; blk < MAX_SQUEEZE_BLOCKS; ++blk) {
        squeeze_words(lo, hi, sq, 17, lane);
        __syncwarp();
        ctr = expand_s_block<ETA>(sq, buf, ctr, lane);
        __syncwarp();
        if (ctr >= N) break;
        keccak_f(lo, hi);
    }
}

template <int ETA>
__device__ __forceinline__ void expand_s_pair(const uint8_t *rhop, int nonce0, int nonce1, int32_t *buf0,
                                              int32_t *buf1, uint8_t *sq0, uint8_t *sq1, int lane) {
    uint32_t lo0, hi0, lo1, hi1;
    seed_words(lo0, hi0, rhop, 8, (uint32_t)nonce0 & 0xFFFFu, 2, 136, lane);
    seed_words(lo1, hi1, rhop, 8, (uint32_t)nonce1 & 0xFFFFu, 2, 136, lane);
    keccak_f2(lo0, hi0, lo1, hi1);
    int c0 = 0, c1 = 0;
#pragma unroll 1
    for (int blk = 0; blk < MAX_SQUEEZE_BLOCKS; ++blk) {
        squeeze_words(lo0, hi0, sq0, 17, lane);
        squeeze_words(lo1, hi1, sq1, 17, lane);
        __syncwarp();
        if (c0 < N) c0 = expand_s_block<ETA>(sq0, buf0, c0, lane);
        if (c1 < N) c1 = expand_s_block<ETA>(sq1, buf1, c1, lane);
        __syncwarp();
        if (c0 >= N && c1 >= N) break;
        keccak_f2(lo0, hi0, lo1, hi1);
    }
}

// Sixteen-instance ExpandS: polynomials with nonces 0 .. count - 1 (count <=
// 16; s1 then s2), coefficient c of polynomial s to out[s N + c] (coefficient
// order, global memory).  The candidates of two instances are voted on at
// once, one per half-warp: 9 rounds of 16 bytes cover a block's 136.
template <int ETA>
__device__ __forceinline__ void expand_s_16(const uint8_t *rhop, int count, int32_t *out, uint32_t *kst,
                                            int lane) {
    keccak16_seed(
        kst, reinterpret_cast<const uint32_t *>(rhop), 16, [](int s) { return (uint32_t)s | (0x1Fu << 16); },
        count, 136, lane);
    keccak16_permute(kst);
    const int half = lane >> 4, hl = lane & 15;
    const uint32_t below = (1u << hl) - 1u;
    int mine = 0;   // lane s < count: coefficients accepted so far for instance s
#pragma unroll 1
    for (int blk = 0; blk < MAX_SQUEEZE_BLOCKS; ++blk) {
#pragma unroll 1
        for (int q = 0; 2 * q < count; ++q) {
            const int s = 2 * q + half;
            int c = __shfl_sync(FULL, mine, s);
            const bool live = s < count && c < N;
            if (!__any_sync(FULL, live)) continue;
            int32_t *dst = out + s * N;
#pragma unroll
            for (int rnd = 0; rnd < 9; ++rnd) {
                const int b = rnd * 16 + hl;
                const bool valid = live && b < 136;
                const uint32_t byte = valid ? (kst[k16_word(s, b >> 2)] >> (8 * (b & 3))) & 0xFFu : 0xFFu;
                const uint32_t t0 = byte & 15u, t1 = byte >> 4;
                const bool a0 = valid && (ETA == 2 ? t0 < 15u : t0 < 9u);
                const bool a1 = valid && (ETA == 2 ? t1 < 15u : t1 < 9u);
                const uint32_t m0 = __ballot_sync(FULL, a0) >> (16 * half) & 0xFFFFu;
                const uint32_t m1 = __ballot_sync(FULL, a1) >> (16 * half) & 0xFFFFu;
                const int pos0 = c + __popc(m0 & below) + __popc(m1 & below);
                const int pos1 = pos0 + (a0 ? 1 : 0);
                if (a0 && pos0 < N) dst[pos0] = (ETA == 2) ? 2 - (int32_t)(t0 % 5u) : 4 - (int32_t)t0;
                if (a1 && pos1 < N) dst[pos1] = (ETA == 2) ? 2 - (int32_t)(t1 % 5u) : 4 - (int32_t)t1;
                c += __popc(m0) + __popc(m1);
            }
            const int c_new = __shfl_sync(FULL, c, (lane & 1) << 4);
            if ((lane >> 1) == q) mine = c_new;
        }
        if (!__any_sync(FULL, lane < count && mine < N)) break;
        __syncwarp();
        keccak16_permute(kst);
    }
    __syncwarp();
}

// ---------------------------------------------------------------- ExpandMask
// y = gamma1 - t for consecutive ZBITS-bit fields t of SHAKE256(rho' || nonce).
// Results are in layout L0.  sq holds 5 x 136 squeezed bytes (+ slack).

template <int ZBITS>
constexpr int mask_blocks() { return (N * ZBITS / 8 + 135) / 136; }

template <int ZBITS, int32_t GAMMA1>
__device__ __forceinline__ void mask_extract(const uint8_t *sq, int32_t r[8], int lane) {
#pragma unroll
    for (int m = 0; m < 8; ++m) r[m] = GAMMA1 - (int32_t)get_field(sq, ZBITS * (lane + 32 * m), ZBITS);
}

template <int ZBITS, int32_t GAMMA1>
__device__ __forceinline__ void expand_mask_poly(const uint8_t *rhop, int nonce, int32_t r[8], uint8_t *sq,
                                                 int lane) {
    uint32_t lo, hi;
    absorb_seed(lo, hi, rhop, 8, (uint32_t)nonce & 0xFFFFu, 2, 136, lane);
#pragma unroll 1
    for (int blk = 0; blk < mask_blocks<ZBITS>(); ++blk) {
        if (blk) keccak_f(lo, hi);
        squeeze_words(lo, hi, sq + 136 * blk, 17, lane);
    }
    __syncwarp();
    mask_extract<ZBITS, GAMMA1>(sq, r, lane);
    __syncwarp();
}

template <int ZBITS, int32_t GAMMA1>
__device__ __forceinline__ void expand_mask_pair(const uint8_t *rhop, int nonce0, int nonce1, int32_t r0[8],
                                                 int32_t r1[8], uint8_t *sq0, uint8_t *sq1, int lane) {
    uint32_t lo0, hi0, lo1, hi1;
    seed_words(lo0, hi0, rhop, 8, (uint32_t)nonce0 & 0xFFFFu, 2, 136, lane);
    seed_words(lo1, hi1, rhop, 8, (uint32_t)nonce1 & 0xFFFFu, 2, 136, lane);
#pragma unroll 1
    for (int blk = 0; blk < mask_blocks<ZBITS>(); ++blk) {
        keccak_f2(lo0, hi0, lo1, hi1);
        squeeze_words(lo0, hi0, sq0 + 136 * blk, 17, lane);
        squeeze_words(lo1, hi1, sq1 + 136 * blk, 17, lane);
    }
    __syncwarp();
    mask_extract<ZBITS, GAMMA1>(sq0, r0, lane);
    mask_extract<ZBITS, GAMMA1>(sq1, r1, lane);
    __syncwarp();
}

// ---------------------------------------------------------------- SampleInBall
// c with TAU coefficients +-1 from SHAKE256(c~): the first 8 bytes give the
// signs, then for step k = 0 .. TAU-1 (i = 256 - TAU + k) a byte b <= i is
// drawn, c_i <- c_b and c_b <- (-1)^(sign bit k).  Coefficient c is written to
// buf[c + 4 (c >> 5)].
//
// The steps are sequential by definition; the warp evaluates them in
// parallel with the same result:
//  1. Which bytes are drawn.  Byte l of a 32-byte chunk is taken iff
//     b_l <= i0 + A_l, A_l the number taken among the bytes before it.  Start
//     from "all taken" and recompute the takes from the prefix counts until
//     nothing changes: the sets only shrink, never below the sequential
//     answer, and each pass settles at least the first wrong byte, so the
//     (unique) fixed point is the sequential result after at most 33 passes.
//  2. Where each position ends.  Step k writes position i_k (the value of
//     position b_k before the step) and then position b_k (its sign).  A
//     step that writes p as b_k comes at or after the step whose i is p, so
//     the final c_p is the sign of the last step with b_k = p, else, for
//     p = i_k, the value step k moved there, else 0.  That moved value is the
//     same rule applied before step k: the sign of the last earlier step with
//     b_j = b_k, else the value moved by the earlier step whose i is b_k, else
//     0 — a chain resolved by pointer jumping.
// next_block(sq) refills sq[0 .. 136) with the next squeezed block.
template <int TAU, class NextBlock>
__device__ __forceinline__ void sample_in_ball_blocks(int32_t *buf, uint8_t *sq, NextBlock next_block, int lane) {
    static_assert(TAU <= 64, "two steps per lane");
    uint8_t *bk = sq + 136;                              // b_k of step k
    int8_t *vk = reinterpret_cast<int8_t *>(sq + 200);   // value moved into i_k by step k
    const uint64_t signs = *reinterpret_cast<const unsigned long long *>(sq);
    const uint32_t below = (1u << lane) - 1u;
    // 1. the drawn bytes
    int taken = 0, pos = 8, blocks = 1;
#pragma unroll 1
    while (taken < TAU) {
        if (pos == 136) {
            if (++blocks > MAX_SQUEEZE_BLOCKS) break;
            __syncwarp();
            next_block(sq);
            __syncwarp();
            pos = 0;
        }
        const int cnt = min(32, 136 - pos);
        const int b = lane < cnt ? (int)sq[pos + lane] : N;
        uint32_t acc = __ballot_sync(FULL, lane < cnt);
#pragma unroll 1
        for (int pass = 0; pass <= 32; ++pass) {
            const int before = taken + __popc(acc & below);
            const uint32_t m = __ballot_sync(FULL, lane < cnt && before < TAU && b <= N - TAU + before);
            if (m == acc) break;
            acc = m;
        }
        if ((acc >> lane) & 1u) bk[taken + __popc(acc & below)] = (uint8_t)b;
        taken += __popc(acc);
        pos += cnt;
    }
    // 2. the last step writing each position as a b_k (buf holds it for now)
#pragma unroll
    for (int m = 0; m < 8; ++m) buf[lane + 36 * m] = -1;
    __syncwarp();
    const int k0 = lane, k1 = lane + 32;
    const int b0 = k0 < taken ? (int)bk[k0] : -1, b1 = k1 < taken ? (int)bk[k1] : -1;
    if (b0 >= 0) atomicMax(&buf[b0 + 4 * (b0 >> 5)], k0);
    if (b1 >= 0) atomicMax(&buf[b1 + 4 * (b1 >> 5)], k1);
    // the last earlier step with the same b
    int lb0 = -1, lb1 = -1;
#pragma unroll 1
    for (int j = 0; j < taken; ++j) {
        const int bj = __shfl_sync(FULL, j < 32 ? b0 : b1, j & 31);
        if (j < k0 && bj == b0) lb0 = j;
        if (j < k1 && bj == b1) lb1 = j;
    }
    // moved values: resolved (r < 0) or equal to step r's
    auto sign_of = [&](int k) { return ((signs >> k) & 1ull) ? -1 : 1; };
    int v0 = 0, v1 = 0, r0 = -1, r1 = -1;
    if (k0 < taken) {
        if (lb0 >= 0) v0 = sign_of(lb0);
        else if (b0 >= N - TAU && b0 - (N - TAU) < k0) r0 = b0 - (N - TAU);
    }
    if (k1 < taken) {
        if (lb1 >= 0) v1 = sign_of(lb1);
        else if (b1 >= N - TAU && b1 - (N - TAU) < k1) r1 = b1 - (N - TAU);
    }
#pragma unroll 1
    for (int pass = 0; pass < TAU; ++pass) {
        if (!__any_sync(FULL, r0 >= 0 || r1 >= 0)) break;
        const int s0 = r0 >= 0 ? r0 : 0, s1 = r1 >= 0 ? r1 : 0;
        const int a0v = __shfl_sync(FULL, v0, s0 & 31), a1v = __shfl_sync(FULL, v1, s0 & 31);
        const int a0r = __shfl_sync(FULL, r0, s0 & 31), a1r = __shfl_sync(FULL, r1, s0 & 31);
        const int c0v = __shfl_sync(FULL, v0, s1 & 31), c1v = __shfl_sync(FULL, v1, s1 & 31);
        const int c0r = __shfl_sync(FULL, r0, s1 & 31), c1r = __shfl_sync(FULL, r1, s1 & 31);
        if (r0 >= 0) {
            v0 = s0 < 32 ? a0v : a1v;
            r0 = s0 < 32 ? a0r : a1r;
        }
        if (r1 >= 0) {
            v1 = s1 < 32 ? c0v : c1v;
            r1 = s1 < 32 ? c0r : c1r;
        }
    }
    if (k0 < taken) vk[k0] = (int8_t)v0;
    if (k1 < taken) vk[k1] = (int8_t)v1;
    __syncwarp();
    // 3. final coefficients (lane t owns positions t + 32 m)
#pragma unroll
    for (int m = 0; m < 8; ++m) {
        const int p = lane + 32 * m, last = buf[lane + 36 * m];
        int c = 0;
        if (last >= 0)
            c = sign_of(last);
        else if (p >= N - TAU && p - (N - TAU) < taken)
            c = vk[p - (N - TAU)];
        buf[lane + 36 * m] = c;
    }
    __syncwarp();
}

template <int TAU>
__device__ __forceinline__ void sample_in_ball(const uint8_t *ctilde, int32_t *buf, uint8_t *sq, int lane) {
    uint32_t lo, hi;
    absorb_seed(lo, hi, ctilde, 4, 0u, 0, 136, lane);
    squeeze_words(lo, hi, sq, 17, lane);
    __syncwarp();
    sample_in_ball_blocks<TAU>(
        buf, sq,
        [&](uint8_t *dst) {
            keccak_f(lo, hi);
            squeeze_words(lo, hi, dst, 17, lane);
        },
        lane);
}

// ---------------------------------------------------------------- packing
// Packs 8 consecutive values (each < 2^BITS) into BITS bytes at out
// (little-endian bit stream).
template <int BITS>
__device__ __forceinline__ void pack8(uint8_t *out, const uint32_t v[8]) {
    uint64_t acc = 0;
    int nb = 0, o = 0;
#pragma unroll
    for (int m = 0; m < 8; ++m) {
        acc |= (uint64_t)v[m] << nb;
        nb += BITS;
#pragma unroll
        for (int s = 0; s < 3; ++s) {
            if (nb >= 8) {
                out[o++] = (uint8_t)acc;
                acc >>= 8;
                nb -= 8;
            }
        }
    }
}

// Copies nbytes from global to shared memory, one byte per lane per step,
// through L2 (coherent with copies into the source made while the kernel runs).
__device__ __forceinline__ void stage_bytes(uint8_t *dst, const uint8_t *__restrict__ src, int nbytes, int lane) {
    for (int i = lane; i < nbytes; i += 32) dst[i] = __ldcg(src + i);
}

}  // namespace dil

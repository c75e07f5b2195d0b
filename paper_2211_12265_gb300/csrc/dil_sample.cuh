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

// Sixteen-instance ExpandA: polynomials p0 .. p0 + count - 1 (count <= 16),
// written like expand_a_six.  The candidates of two instances are voted on at
// once, one per half-warp (4 x 16 candidate slots for a block's 56).
template <int L>
__device__ __forceinline__ void expand_a_16(const uint8_t *rho, int p0, int count, int32_t *out, uint32_t *kst,
                                            int lane) {
    keccak16_seed(
        kst, reinterpret_cast<const uint32_t *>(rho), 8,
        [&](int s) { const int p = p0 + s; return (uint32_t)(p % L) | ((uint32_t)(p / L) << 8) | (0x1Fu << 16); },
        count, 168, lane);
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
        keccak16_permute(kst);
    }
    __syncwarp();
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
// signs, then for i = 256-TAU .. 255 a byte b <= i is drawn, c_i <- c_b and
// c_b <- +-1.  Coefficient c is written to buf[c + 4 (c >> 5)].
template <int TAU>
__device__ __forceinline__ void sample_in_ball(const uint8_t *ctilde, int32_t *buf, uint8_t *sq, int lane) {
    uint32_t lo, hi;
    absorb_seed(lo, hi, ctilde, 4, 0u, 0, 136, lane);
    squeeze_words(lo, hi, sq, 17, lane);
#pragma unroll
    for (int m = 0; m < 8; ++m) buf[lane + 36 * m] = 0;
    __syncwarp();
    uint64_t signs = *reinterpret_cast<const unsigned long long *>(sq);
    int pos = 8, blocks = 1;
#pragma unroll 1
    for (int i = N - TAU; i < N; ++i) {
        int b;
        do {
            if (pos == 136) {
                if (++blocks > MAX_SQUEEZE_BLOCKS) break;
                __syncwarp();
                keccak_f(lo, hi);
                squeeze_words(lo, hi, sq, 17, lane);
                __syncwarp();
                pos = 0;
            }
            b = sq[pos++];
        } while (b > i);
        if (lane == 0) {
            int32_t cb = buf[b + 4 * (b >> 5)];
            buf[i + 4 * (i >> 5)] = cb;
            buf[b + 4 * (b >> 5)] = (signs & 1) ? -1 : 1;
        }
        signs >>= 1;
    }
    __syncwarp();
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

// Copies nbytes from global to shared memory, one byte per lane per step.
__device__ __forceinline__ void stage_bytes(uint8_t *dst, const uint8_t *__restrict__ src, int nbytes, int lane) {
    for (int i = lane; i < nbytes; i += 32) dst[i] = __ldg(src + i);
}

}  // namespace dil

// Warp-cooperative Keccak-f[1600] and the SHAKE128/256 sponge (section 3.3 of
// arXiv 2211.12265: 25 threads of a warp each hold one 64-bit lane of the state
// in registers and exchange lanes with warp shuffles every round; round
// constants live in constant memory; absorb and squeeze move 8-byte words).
//
// Lane t < 25 holds state lane (x, y) = (t mod 5, t div 5) as two 32-bit
// halves.  Lanes 25..31 compute on copies and are never read.  One round costs
// 16 32-bit shuffles: theta's column parity by a rotate-and-reduce over the
// five rows (3 shuffles of 64 bits), its two neighbour columns (2), and pi+chi
// gathering the three rotated lanes each output lane needs (3).
#pragma once
#include <cstdint>

namespace dil {

constexpr unsigned FULL = 0xffffffffu;

// FIPS 202 round constants RC[0..23] (iota).
static __constant__ uint64_t c_keccak_rc[24] = {
    0x0000000000000001ull, 0x0000000000008082ull, 0x800000000000808Aull, 0x8000000080008000ull,
    0x000000000000808Bull, 0x0000000080000001ull, 0x8000000080008081ull, 0x8000000000008009ull,
    0x000000000000008Aull, 0x0000000000000088ull, 0x0000000080008009ull, 0x000000008000000Aull,
    0x000000008000808Bull, 0x800000000000008Bull, 0x8000000000008089ull, 0x8000000000008003ull,
    0x8000000000008002ull, 0x8000000000000080ull, 0x000000000000800Aull, 0x800000008000000Aull,
    0x8000000080008081ull, 0x8000000000008080ull, 0x0000000080000001ull, 0x8000000080008008ull};

// FIPS 202 rho rotation offset of lane (x, y).  Each row's five offsets are
// packed as 6-bit fields of one immediate, so lanes asking for different
// offsets do not serialise on a constant-memory table.
__device__ __forceinline__ int rho_offset(int x, int y) {
    const uint32_t row = y == 0 ? 0x1B73E040u : y == 1 ? 0x14DC6B24u : y == 2 ? 0x2766B283u : y == 3 ? 0x0854FB69u : 0x0EE3D092u;
    return (int)((row >> (6 * x)) & 63u);
}

// Per-thread shuffle sources and rotation for one warp-level Keccak instance.
struct KLane {
    int s5, s10, s20;  // theta: lanes (x, y+1), (x, y+2), (x, y+4)
    int sm, sp;        // theta: lanes (x-1, y), (x+1, y)
    int b0, b1, b2;    // pi+chi: sources of B[x,y], B[x+1,y], B[x+2,y]
    int rot;           // rho amount mod 32
    bool swap;         // rho amount >= 32
    uint32_t iota;     // all ones on the thread holding lane (0,0), else 0
};

__device__ __forceinline__ KLane klane_init(int lane) {
    KLane k;
    int t = lane < 25 ? lane : 0;
    int x = t % 5, y = t / 5;
    k.s5 = (t + 5) % 25;
    k.s10 = (t + 10) % 25;
    k.s20 = (t + 20) % 25;
    k.sm = (x + 4) % 5 + 5 * y;
    k.sp = (x + 1) % 5 + 5 * y;
    // pi: B[X, Y] = A[(X + 3Y) mod 5, X]
    int x1 = (x + 1) % 5, x2 = (x + 2) % 5;
    k.b0 = (x + 3 * y) % 5 + 5 * x;
    k.b1 = (x1 + 3 * y) % 5 + 5 * x1;
    k.b2 = (x2 + 3 * y) % 5 + 5 * x2;
    int r = rho_offset(x, y);
    k.rot = r & 31;
    k.swap = r >= 32;
    k.iota = lane == 0 ? 0xFFFFFFFFu : 0u;
    return k;
}

__device__ __forceinline__ void keccak_round(uint32_t &lo, uint32_t &hi, const KLane &k, uint64_t rc) {
    // theta: column parity C[x] in every lane of column x
    uint32_t clo = lo ^ __shfl_sync(FULL, lo, k.s5);
    uint32_t chi = hi ^ __shfl_sync(FULL, hi, k.s5);
    clo ^= __shfl_sync(FULL, clo, k.s10);
    chi ^= __shfl_sync(FULL, chi, k.s10);
    clo ^= __shfl_sync(FULL, lo, k.s20);
    chi ^= __shfl_sync(FULL, hi, k.s20);
    uint32_t mlo = __shfl_sync(FULL, clo, k.sm);
    uint32_t mhi = __shfl_sync(FULL, chi, k.sm);
    uint32_t plo = __shfl_sync(FULL, clo, k.sp);
    uint32_t phi = __shfl_sync(FULL, chi, k.sp);
    // D[x] = C[x-1] ^ rotl(C[x+1], 1)
    lo ^= mlo ^ ((plo << 1) | (phi >> 31));
    hi ^= mhi ^ ((phi << 1) | (plo >> 31));
    // rho: rotate by rot, then swap halves when the amount is >= 32
    uint32_t nlo = __funnelshift_l(hi, lo, k.rot);
    uint32_t nhi = __funnelshift_l(lo, hi, k.rot);
    lo = k.swap ? nhi : nlo;
    hi = k.swap ? nlo : nhi;
    // pi + chi: A[x,y] = B[x,y] ^ (~B[x+1,y] & B[x+2,y])
    uint32_t a0l = __shfl_sync(FULL, lo, k.b0), a0h = __shfl_sync(FULL, hi, k.b0);
    uint32_t a1l = __shfl_sync(FULL, lo, k.b1), a1h = __shfl_sync(FULL, hi, k.b1);
    uint32_t a2l = __shfl_sync(FULL, lo, k.b2), a2h = __shfl_sync(FULL, hi, k.b2);
    lo = a0l ^ (~a1l & a2l);
    hi = a0h ^ (~a1h & a2h);
    // iota (branch-free, so that two interleaved rounds form one basic block)
    lo ^= (uint32_t)rc & k.iota;
    hi ^= (uint32_t)(rc >> 32) & k.iota;
}

// Out-of-line permutations, called by value so the state stays in registers.
// The lane parameters are recomputed per call (a few dozen instructions per
// 24 rounds) instead of occupying registers at every call site.  The round
// loops stay rolled: the fused kernels are bound by instruction fetch as much
// as by issue, and unrolling them cost more than the saved loop overhead.
static __device__ __noinline__ uint2 keccak_f_impl(uint2 s) {
    const KLane k = klane_init(threadIdx.x & 31);
    uint32_t lo = s.x, hi = s.y;
#pragma unroll 1
    for (int r = 0; r < 24; ++r) keccak_round(lo, hi, k, c_keccak_rc[r]);
    return make_uint2(lo, hi);
}

// Two independent states interleaved round by round: the second instance's
// shuffles fill the latency of the first's.
static __device__ __noinline__ uint4 keccak_f2_impl(uint4 s) {
    const KLane k = klane_init(threadIdx.x & 31);
    uint32_t lo0 = s.x, hi0 = s.y, lo1 = s.z, hi1 = s.w;
#pragma unroll 1
    for (int r = 0; r < 24; ++r) {
        const uint64_t rc = c_keccak_rc[r];
        keccak_round(lo0, hi0, k, rc);
        keccak_round(lo1, hi1, k, rc);
    }
    return make_uint4(lo0, hi0, lo1, hi1);
}

__device__ __forceinline__ void keccak_f(uint32_t &lo, uint32_t &hi) {
    uint2 s = keccak_f_impl(make_uint2(lo, hi));
    lo = s.x;
    hi = s.y;
}

__device__ __forceinline__ void keccak_f2(uint32_t &lo0, uint32_t &hi0, uint32_t &lo1, uint32_t &hi1) {
    uint4 s = keccak_f2_impl(make_uint4(lo0, hi0, lo1, hi1));
    lo0 = s.x;
    hi0 = s.y;
    lo1 = s.z;
    hi1 = s.w;
}

// Writes the first `words` 8-byte words of the rate to dst (8-byte aligned).
__device__ __forceinline__ void squeeze_words(const uint32_t lo, const uint32_t hi, uint8_t *dst, int words, int lane) {
    if (lane < words) *reinterpret_cast<uint2 *>(dst + 8 * lane) = make_uint2(lo, hi);
}

// Pads the final block: SHAKE domain bits 1111 then pad10*1.  `rem` is the
// number of message bytes in the final block (0 <= rem < rate).
__device__ __forceinline__ void pad_word(uint64_t &w, int rem, int rate, int lane) {
    int b0 = 8 * lane;
    if (rem >= b0 && rem < b0 + 8) w ^= (uint64_t)0x1F << (8 * (rem - b0));
    if (lane == rate / 8 - 1) w ^= (uint64_t)0x80 << 56;
}

// Absorbs len bytes from an 8-byte-aligned shared-memory buffer, pads and
// permutes; afterwards the state holds the first squeeze block.  The buffer
// must be readable up to the next multiple of 8 beyond len.
__device__ __forceinline__ void absorb_smem(uint32_t &lo, uint32_t &hi, const uint8_t *buf, int len, int rate,
                                            int lane) {
    const int words = rate / 8;
    int off = 0;
    for (; len - off >= rate; off += rate) {
        if (lane < words) {
            uint2 w = *reinterpret_cast<const uint2 *>(buf + off + 8 * lane);
            lo ^= w.x;
            hi ^= w.y;
        }
        keccak_f(lo, hi);
    }
    int rem = len - off;
    if (lane < words) {
        uint64_t w = 0;
        int b0 = 8 * lane;
        if (b0 < rem) {
            uint2 v = *reinterpret_cast<const uint2 *>(buf + off + b0);
            w = ((uint64_t)v.y << 32) | v.x;
            int have = rem - b0;
            if (have < 8) w &= ((uint64_t)1 << (8 * have)) - 1;
        }
        pad_word(w, rem, rate, lane);
        lo ^= (uint32_t)w;
        hi ^= (uint32_t)(w >> 32);
    }
    keccak_f(lo, hi);
}

// Aligned 8-byte word of global memory, loaded through L2: coherent with
// stores and copies made while the kernel runs (a serving kernel reuses its
// request buffers), unlike the L1 and read-only paths.
__device__ __forceinline__ uint64_t ld_word_cg(const uint8_t *p) {
    return __ldcg(reinterpret_cast<const unsigned long long *>(p));
}

// Absorbs the concatenation A || B where A (lenA bytes, a multiple of 8) is in
// 8-byte-aligned shared memory and B (lenB bytes, any alignment) is in global
// memory; pads and permutes.  B is read in aligned 8-byte words through L2,
// one per lane and block (the section 3.3 wide, aligned input loads): lane i
// takes word i of the block and its neighbour's by a shuffle and realigns
// the pair with a funnel shift; the next block's words are loaded before the
// current block is permuted.  An aligned word that holds a byte of B lies in
// the same page as that byte, so no load can fault; bytes outside B are
// masked off.
__device__ __forceinline__ void absorb_concat(uint32_t &lo, uint32_t &hi, const uint8_t *A, int lenA,
                                              const uint8_t *B, size_t lenB, int rate, int lane) {
    const int words = rate / 8;
    const size_t total = (size_t)lenA + lenB;
    const int shift = 8 * (int)((uintptr_t)B & 7);             // bit offset of B in its aligned word
    const uint8_t *base = B - (shift >> 3);
    // aligned words holding bytes of B (none when B is empty: B may point past its buffer)
    const long long nwords = lenB ? (long long)((lenB + (shift >> 3) + 7) >> 3) : 0;
    // lane k's aligned word of B for a block starting at concatenation byte
    // `off`: index (off - lenA) / 8 + k; words outside B read as 0
    auto word_at = [&](size_t off) -> uint64_t {
        const long long j = ((long long)off - lenA) / 8 + lane;
        return (j >= 0 && j < nwords) ? ld_word_cg(base + 8 * j) : 0ull;
    };
    size_t off = 0;
    uint64_t cur = word_at(0);
    for (;;) {
        const size_t rem = total - off;
        const bool last = rem < (size_t)rate;
        const uint64_t nxt = __shfl_down_sync(FULL, cur, 1);
        const uint64_t ahead = last ? 0ull : word_at(off + rate);   // in flight during the permutation
        if (lane < words) {
            const size_t p = off + 8 * lane;
            uint64_t w;
            if (p < (size_t)lenA) {
                const uint2 v = *reinterpret_cast<const uint2 *>(A + p);
                w = ((uint64_t)v.y << 32) | v.x;
            } else {
                w = shift ? (cur >> shift) | (nxt << (64 - shift)) : cur;
            }
            const long long have = (long long)total - (long long)p;   // bytes of the word inside A || B
            if (have <= 0)
                w = 0;
            else if (have < 8)
                w &= (1ull << (8 * have)) - 1;
            if (last) pad_word(w, (int)rem, rate, lane);
            lo ^= (uint32_t)w;
            hi ^= (uint32_t)(w >> 32);
        }
        keccak_f(lo, hi);
        if (last) break;
        off += rate;
        cur = ahead;
    }
}

// State words of a short padded seed that fits one block: lanes < nwords take
// 8-byte words of `seed` (8-byte aligned shared memory), lane nwords takes
// `tailbytes` extra bytes in tailw.  Used for the fixed-size seeds
// rho || nonce, rho' || nonce and c~; absorb_seed also applies the permutation.
__device__ __forceinline__ void seed_words(uint32_t &lo, uint32_t &hi, const uint8_t *seed, int nwords,
                                           uint32_t tailw, int tailbytes, int rate, int lane) {
    uint64_t w = 0;
    if (lane < nwords) {
        uint2 v = *reinterpret_cast<const uint2 *>(seed + 8 * lane);
        w = ((uint64_t)v.y << 32) | v.x;
    } else if (lane == nwords) {
        w = tailw;
    }
    if (lane < rate / 8) pad_word(w, 8 * nwords + tailbytes, rate, lane);
    lo = (uint32_t)w;
    hi = (uint32_t)(w >> 32);
}

__device__ __forceinline__ void absorb_seed(uint32_t &lo, uint32_t &hi, const uint8_t *seed, int nwords,
                                            uint32_t tailw, int tailbytes, int rate, int lane) {
    seed_words(lo, hi, seed, nwords, tailw, tailbytes, rate, lane);
    keccak_f(lo, hi);
}

}  // namespace dil

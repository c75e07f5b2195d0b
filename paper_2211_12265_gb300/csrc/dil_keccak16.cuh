// Sixteen Keccak-f[1600] instances per warp, two threads per instance (bulk
// sponges of the samplers when a warp has seven or more sponges to run).
//
// Lane 2s + p holds half p of every lane of instance s: the low 32-bit word
// of each 64-bit state lane (p = 0) or the high word (p = 1), i.e. 25
// registers.  Everything in a round but the 64-bit rotations is
// word-local: theta's column parities, chi along the rows and pi (a renaming
// of registers) need no exchange at all.  A 64-bit rotation by r needs both
// words of the lane: each thread fetches its partner's word with one
// shuffle and keeps its own half of the rotated lane with one funnel shift,
// the same expression on both threads (mine m, partner v: r < 32 gives
// fshl(v, m, r), r >= 32 gives fshl(m, v, r - 32)).  Per round that is 24
// shuffles for rho and 5 for theta's rotation by one, about 125 instructions
// per thread for 16 instances (about 8 warp instructions per instance-round,
// against about 15 for the six-state row form and 66 for the 25-lane form),
// and no shared-memory traffic inside the permutation.
//
// Between permutations the states live in shared memory (`kst`, 850 words):
// word i (lane i = x + 5y of the state) of thread `lane` at 34 i + lane, and
// byte-stream word w (4 bytes) of instance s at 34 (w >> 1) + 2 s + (w & 1).
// The two padding words per row put word w of an instance in bank
// (w + 2 s) mod 32, so the samplers' reads of one instance's consecutive
// stream words (16 lanes, a dozen words) do not conflict, while each thread's
// own 25 words stay one per row at constant offsets.
#pragma once
#include "dil_keccak.cuh"
#include "dil_ntt.cuh"

namespace dil {

constexpr int K16_STATES = 16;
constexpr int K16_ROW = 34;                // words per state-word row (32 threads + 2 of padding)
constexpr int K16_WORDS = 25 * K16_ROW;    // shared words of the sixteen states

// Shared-memory word of state word i of thread `lane`.
__host__ __device__ __forceinline__ int k16_slot(int i, int lane) { return K16_ROW * i + lane; }
// Shared-memory word of byte-stream word w of instance s.
__host__ __device__ __forceinline__ int k16_word(int s, int w) { return K16_ROW * (w >> 1) + 2 * s + (w & 1); }

namespace detail {
// FIPS 202 rho offset of lane (x, y).
__host__ __device__ constexpr int k16_rho(int x, int y) {
    return (y == 0)   ? (x == 0 ? 0 : x == 1 ? 1 : x == 2 ? 62 : x == 3 ? 28 : 27)
           : (y == 1) ? (x == 0 ? 36 : x == 1 ? 44 : x == 2 ? 6 : x == 3 ? 55 : 20)
           : (y == 2) ? (x == 0 ? 3 : x == 1 ? 10 : x == 2 ? 43 : x == 3 ? 25 : 39)
           : (y == 3) ? (x == 0 ? 41 : x == 1 ? 45 : x == 2 ? 15 : x == 3 ? 21 : 8)
                      : (x == 0 ? 18 : x == 1 ? 2 : x == 2 ? 61 : x == 3 ? 56 : 14);
}
}  // namespace detail

// This thread's half of rotl64(lane, R) given its word m of the lane.
template <int R>
__device__ __forceinline__ uint32_t k16_rot(uint32_t m) {
    if constexpr (R == 0) {
        return m;
    } else {
        const uint32_t v = __shfl_xor_sync(FULL, m, 1);
        if constexpr (R < 32)
            return __funnelshift_l(v, m, R);
        else
            return __funnelshift_l(m, v, R - 32);
    }
}

// rho + pi for source lane i = x + 5y: B[y + 5 ((2x + 3y) mod 5)] = rotl(A[i]).
template <int I>
__device__ __forceinline__ void k16_rho_pi(uint32_t (&b)[25], const uint32_t (&a)[25]) {
    constexpr int x = I % 5, y = I / 5;
    b[y + 5 * ((2 * x + 3 * y) % 5)] = k16_rot<detail::k16_rho(x, y)>(a[I]);
    if constexpr (I < 24) k16_rho_pi<I + 1>(b, a);
}

// Permutes the sixteen states at shared address kst (K16_WORDS words).  Called
// by all 32 lanes of the warp.  Out of line: one copy serves every sampler.
static __device__ __noinline__ void keccak16_permute_impl(uint32_t kst) {
    const int lane = threadIdx.x & 31;
    const uint32_t base = kst + 4 * lane;
    const bool high = lane & 1;
    uint32_t a[25];
#pragma unroll
    for (int i = 0; i < 25; ++i) asm volatile("ld.shared.u32 %0, [%1];" : "=r"(a[i]) : "r"(base + 4 * K16_ROW * i));
#pragma unroll 1
    for (int round = 0; round < 24; ++round) {
        // theta
        uint32_t c[5], d[5];
#pragma unroll
        for (int x = 0; x < 5; ++x) c[x] = a[x] ^ a[x + 5] ^ a[x + 10] ^ a[x + 15] ^ a[x + 20];
#pragma unroll
        for (int x = 0; x < 5; ++x) d[x] = k16_rot<1>(c[x]);   // this half of rotl(C[x], 1)
#pragma unroll
        for (int i = 0; i < 25; ++i) a[i] ^= c[(i + 4) % 5] ^ d[(i + 1) % 5];
        // rho + pi
        uint32_t b[25];
        k16_rho_pi<0>(b, a);
        // chi
#pragma unroll
        for (int y = 0; y < 5; ++y)
#pragma unroll
            for (int x = 0; x < 5; ++x)
                a[x + 5 * y] = b[x + 5 * y] ^ (~b[(x + 1) % 5 + 5 * y] & b[(x + 2) % 5 + 5 * y]);
        // iota
        const uint64_t rc = c_keccak_rc[round];
        a[0] ^= high ? (uint32_t)(rc >> 32) : (uint32_t)rc;
    }
#pragma unroll
    for (int i = 0; i < 25; ++i)
        asm volatile("st.shared.u32 [%0], %1;" ::"r"(base + 4 * K16_ROW * i), "r"(a[i]) : "memory");
    __syncwarp();
}

__device__ __forceinline__ void keccak16_permute(uint32_t *kst) { keccak16_permute_impl(smem_addr(kst)); }

// Initialises the sixteen states with padded one-block seeds: byte-stream
// words [0, seed_words) from `seed` (shared memory), then the word
// tail_of(s) (the instance's nonce bytes followed by the SHAKE
// domain/padding byte 0x1F), and the final padding bit at the last byte of
// the rate.  Instances >= count get the same seed with tail 0 (their output is
// never read); instances >= keep are left as they are.
template <class Tail>
__device__ __forceinline__ void keccak16_seed(uint32_t *kst, const uint32_t *seed, int seed_words, Tail tail_of,
                                              int count, int rate, int lane, int keep = K16_STATES) {
    const int s = lane >> 1, p = lane & 1;
    const uint32_t tail = s < count ? tail_of(s) : 0u;
    if (s < keep) {
#pragma unroll 1
        for (int i = 0; i < 25; ++i) {
            const int w = 2 * i + p;
            uint32_t v = w < seed_words ? seed[w] : w == seed_words ? tail : 0u;
            if (w == rate / 4 - 1) v ^= 0x80000000u;
            kst[k16_slot(i, lane)] = v;
        }
    }
    __syncwarp();
}

// Lane `lane` (< 17)'s 8 bytes of 136-byte block blk of a `len`-byte SHAKE256
// input at src (global memory, any alignment), padded in the final block
// (total = len / 136 + 1 blocks).  Plain loads: bytes the same warp wrote
// earlier in the kernel are seen.
__device__ __forceinline__ uint64_t rider_word(const uint8_t *src, size_t len, int total, int blk, int lane) {
    const size_t off = (size_t)blk * 136 + 8 * lane;
    const uint8_t *p = src + off;
    uint64_t w = 0;
    if (off + 8 <= len && (reinterpret_cast<uintptr_t>(p) & 7) == 0) {
        const uint2 v = *reinterpret_cast<const uint2 *>(p);
        w = ((uint64_t)v.y << 32) | v.x;
    } else {
#pragma unroll
        for (int k = 0; k < 8; ++k)
            if (off + k < len) w |= (uint64_t)p[k] << (8 * k);
    }
    if (blk == total - 1) pad_word(w, (int)(len - (size_t)blk * 136), 136, lane);
    return w;
}

// A SHAKE256 hash of `len` bytes of global memory (any alignment) that
// rides in the last instance (15) of the sixteen-state batches of a sampler:
// before each of the batch's permutations one 136-byte rate block of the
// input (the last one padded) is absorbed into instance 15, so the hash
// needs no permutation of its own.  Once the permutation after the final
// block has run, the first 32 output bytes go to `out` (8-byte aligned
// shared memory).  A hash longer than the batches' permutations is finished
// on the 25-lane form (finish).  The samplers that carry it use instances
// 0..14 only.  Block counts are 32-bit: an input of 2^31 blocks (292 GB)
// would not fit in device memory.
struct K16Rider {
    static constexpr int SLOT = K16_STATES - 1;
    static constexpr int KEEP = SLOT;   // instances a carrying sampler may seed
    static constexpr int RATE = 136;
    const uint8_t *src;
    size_t len;
    uint32_t out;   // shared-memory address
    int next;       // next block to absorb; total + 1 once the output is taken
    int total;      // blocks of the padded input

    __device__ K16Rider(const uint8_t *src_, size_t len_, uint32_t *out_)
        : src(src_), len(len_), out(smem_addr(out_)), next(0), total((int)(len_ / RATE) + 1) {}

    __device__ __forceinline__ uint64_t word(int blk, int lane) const { return rider_word(src, len, total, blk, lane); }

    // Absorbs the next block into instance SLOT (called by all 32 lanes right
    // before a permutation).
    __device__ __forceinline__ void before(uint32_t *kst, int lane) {
        if (next >= total) return;
        const int blk = next++;
        if (lane < 25) {
            const uint64_t w = lane < RATE / 8 ? word(blk, lane) : 0;
            uint32_t *st = kst + k16_slot(lane, 2 * SLOT);
            if (blk == 0) {
                st[0] = (uint32_t)w;
                st[1] = (uint32_t)(w >> 32);
            } else {
                st[0] ^= (uint32_t)w;
                st[1] ^= (uint32_t)(w >> 32);
            }
        }
        __syncwarp();
    }

    // Takes the output once the final block has been permuted (called by all
    // 32 lanes right after a permutation).
    __device__ __forceinline__ void after(const uint32_t *kst, int lane) {
        if (next != total) return;
        if (lane < 8)
            asm volatile("st.shared.u32 [%0], %1;" ::"r"(out + 4 * lane), "r"(kst[k16_word(SLOT, lane)]) : "memory");
        next = total + 1;
        __syncwarp();
    }

    // Completes an unfinished hash on the 25-lane form from instance SLOT's
    // state (all 32 lanes; kst must still hold the batches' states).  Every
    // before() is followed by a permutation and after(), so here either the
    // output is taken (next > total) or the state is that after the
    // permutation of block next - 1 (next < total).
    __device__ __forceinline__ void finish(const uint32_t *kst, int lane) {
        if (next > total) return;
        uint32_t lo = 0, hi = 0;
        if (next > 0 && lane < 25) {
            lo = kst[k16_slot(lane, 2 * SLOT)];
            hi = kst[k16_slot(lane, 2 * SLOT + 1)];
        }
#pragma unroll 1
        for (; next < total; ++next) {
            const uint64_t w = lane < RATE / 8 ? word(next, lane) : 0;
            lo ^= (uint32_t)w;
            hi ^= (uint32_t)(w >> 32);
            keccak_f(lo, hi);
        }
        if (lane < 4)
            asm volatile("st.shared.v2.u32 [%0], {%1, %2};" ::"r"(out + 8 * lane), "r"(lo), "r"(hi) : "memory");
        next = total + 1;
        __syncwarp();
    }
};

// A SHAKE256 hash that rides like K16Rider over an input that is still being
// written (KeyGen's H(pk) while the rows of t are packed): a permutation
// advances it only when the next block's bytes exist (set_ready), and between
// such permutations its state lives in shared memory (`save`, 25 x 8 bytes,
// 8-byte aligned), so instance 15 may be overwritten in between (the other
// instances' permutations, buffers in the same shared-memory union).  When
// the final block has been permuted the first 32 output bytes go to `out`;
// finish() completes the hash on the 25-lane form and must only be called
// once all `len` bytes are written.
struct K16ChainRider {
    static constexpr int SLOT = K16_STATES - 1;
    static constexpr int KEEP = SLOT;
    static constexpr int RATE = 136;
    const uint8_t *src;
    size_t len;
    uint32_t save, out;   // shared-memory addresses
    int next;             // next block to absorb; total + 1 once the output is taken
    int total;            // blocks of the padded input
    int avail;            // blocks whose bytes exist
    bool absorbed;        // the current permutation advances the hash

    __device__ K16ChainRider(const uint8_t *src_, size_t len_, uint32_t *save_, uint32_t *out_)
        : src(src_), len(len_), save(smem_addr(save_)), out(smem_addr(out_)), next(0),
          total((int)(len_ / RATE) + 1), avail(0), absorbed(false) {}

    // The first `bytes` bytes of the input are written (and visible to the warp).
    __device__ __forceinline__ void set_ready(size_t bytes) {
        avail = bytes >= len ? total : (int)(bytes / RATE);
    }

    __device__ __forceinline__ void before(uint32_t *kst, int lane) {
        absorbed = next < avail;
        if (!absorbed) return;
        if (lane < 25) {
            uint32_t lo = 0, hi = 0;
            if (next > 0) asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(lo), "=r"(hi) : "r"(save + 8 * lane));
            const uint64_t w = lane < RATE / 8 ? rider_word(src, len, total, next, lane) : 0;
            uint32_t *st = kst + k16_slot(lane, 2 * SLOT);
            st[0] = lo ^ (uint32_t)w;
            st[1] = hi ^ (uint32_t)(w >> 32);
        }
        ++next;
        __syncwarp();
    }

    __device__ __forceinline__ void after(const uint32_t *kst, int lane) {
        if (!absorbed) return;
        absorbed = false;
        if (lane < 25) {
            const uint32_t lo = kst[k16_slot(lane, 2 * SLOT)], hi = kst[k16_slot(lane, 2 * SLOT + 1)];
            if (next < total)
                asm volatile("st.shared.v2.u32 [%0], {%1, %2};" ::"r"(save + 8 * lane), "r"(lo), "r"(hi) : "memory");
            else if (lane < 4)
                asm volatile("st.shared.v2.u32 [%0], {%1, %2};" ::"r"(out + 8 * lane), "r"(lo), "r"(hi) : "memory");
        }
        if (next == total) next = total + 1;
        __syncwarp();
    }

    __device__ __forceinline__ void finish(int lane) {
        if (next > total) return;
        uint32_t lo = 0, hi = 0;
        if (next > 0 && lane < 25)
            asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(lo), "=r"(hi) : "r"(save + 8 * lane));
#pragma unroll 1
        for (; next < total; ++next) {
            const uint64_t w = lane < RATE / 8 ? rider_word(src, len, total, next, lane) : 0;
            lo ^= (uint32_t)w;
            hi ^= (uint32_t)(w >> 32);
            keccak_f(lo, hi);
        }
        if (lane < 4)
            asm volatile("st.shared.v2.u32 [%0], {%1, %2};" ::"r"(out + 8 * lane), "r"(lo), "r"(hi) : "memory");
        next = total + 1;
        __syncwarp();
    }
};

// The no-op rider of the samplers that carry none.
struct K16NoRider {
    static constexpr int KEEP = K16_STATES;
    __device__ __forceinline__ void before(uint32_t *, int) {}
    __device__ __forceinline__ void after(const uint32_t *, int) {}
};

}  // namespace dil

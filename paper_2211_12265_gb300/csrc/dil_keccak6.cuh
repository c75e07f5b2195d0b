// Six Keccak-f[1600] instances per warp in a row layout (bulk sponges of the
// samplers).  Still warp-cooperative with the state in registers: instance g
// uses lanes 5g..5g+4 (g < 6; lanes 30, 31 idle), and lane 5g + y holds row y
// of the state, i.e. lanes (x, y) for x = 0..4, as ten 32-bit words.
//
// A row's five lanes are held skewed: register slot j of the lane for row y
// holds column x = (j + y) mod 5.  With that skew, theta's column parities
// take a reduce-scatter (slot 5 - k of row y + k is column y, so 4 shuffles
// per word leave column y's parity on row y) and an all-gather (4 more), 16
// shuffles per round for six instances; D and chi only use neighbouring
// slots, rho is a per-slot rotation, and pi (which moves lane (x, y) to
// (y, 2x + 3y), across rows) goes through a per-warp shared buffer: every lane
// stores its five rotated lanes at their destinations (a rotation by >= 32 is
// folded into the store by swapping the two words) and reads back its new
// row.  The buffer keeps low and high words in separate planes, slot j of the
// lane for row Y of instance g at word 30 j + 5 g + Y of its plane, the high
// plane 160 words (a multiple of the 32 banks) after the low one, so the row
// reads are at fixed offsets and both they and the scattered stores (whichever
// plane each lane's word goes to) hit 30 distinct banks.  Per instance-round that is 2.7 shuffles, 3.3 shared-memory
// accesses and about 9 other instructions, against 16 shuffles and about 20
// others for the 25-lane form.
//
// Between permutations the six states live in shared memory (`kst`, 6 x 50
// words, lane (x, y) of instance g at words 50g + 2(x + 5y), low word first),
// so a state's first bytes are directly its squeezed output block.
#pragma once
#include "dil_keccak.cuh"
#include "dil_ntt.cuh"

namespace dil {

constexpr int K6_WORDS = 50;            // one state: 25 lanes x 2 words
constexpr int K6_STATES = 6;
constexpr int K6_PI_WORDS = 320;        // exchange buffer: two planes of 5 x 30 words, + read slack

// Per-lane constants of the six-state permutation, one word per slot j and a
// word of shuffle sources, built at compile time:
//   slot word: bits 0-10 byte offset in the exchange buffer of the slot's low
//   word after rho (its high word in bits 11-21; the planes are swapped when
//   the rotation is >= 32), bits 22-26 the rotation mod 32, bits 27-29 the
//   column x held by the slot;
//   source word: the lanes of rows y + 1 .. y + 4 of the instance, 5 bits each.
// Read with coalesced cached loads (lanes ask for different words, which a
// constant-memory table would serialise).
struct K6Lanes {
    uint32_t w[6][32];
};

namespace detail {
constexpr int rho_c(int x, int y) {
    constexpr int R[5][5] = {{0, 1, 62, 28, 27}, {36, 44, 6, 55, 20}, {3, 10, 43, 25, 39}, {41, 45, 15, 21, 8},
                             {18, 2, 61, 56, 14}};
    return R[y][x];
}
constexpr K6Lanes make_k6_lanes() {
    K6Lanes t{};
    for (int lane = 0; lane < 32; ++lane) {
        const int g = lane < 30 ? lane / 5 : 5, y = lane < 30 ? lane % 5 : 4;
        for (int j = 0; j < 5; ++j) {
            const int x = (j + y) % 5, r = rho_c(x, y);
            const int Y = (2 * x + 3 * y) % 5, jd = (y - Y + 5) % 5;
            const uint32_t d = 4u * (30 * jd + 5 * g + Y);
            const uint32_t lo = r >= 32 ? d + 640 : d, hi = r >= 32 ? d : d + 640;
            t.w[j][lane] = lo | (hi << 11) | ((uint32_t)(r & 31) << 22) | ((uint32_t)x << 27);
        }
        uint32_t src = 0;
        for (int k = 1; k < 5; ++k) src |= (uint32_t)(5 * g + (y + k) % 5) << (5 * (k - 1));
        t.w[5][lane] = src;
    }
    return t;
}
}  // namespace detail

static __device__ const K6Lanes c_k6_lanes = detail::make_k6_lanes();

// Permutes the six states at shared address kst (300 words) using the
// exchange buffer at shared address kpi (K6_PI_WORDS words).  Called by all 32
// lanes of the warp.
static __device__ __noinline__ void keccak6_permute_impl(uint32_t kst, uint32_t kpi) {
    const int lane = threadIdx.x & 31;
    const bool on = lane < 30;
    const int g = on ? lane / 5 : 5;
    const int y = on ? lane - 5 * g : 4;
    // slot j of this lane holds state lane (x, y) with x = (j + y) mod 5
    const uint32_t sw = __ldg(&c_k6_lanes.w[5][lane]);
    int src[4];   // lanes of rows y + 1 .. y + 4 of the same instance
#pragma unroll
    for (int k = 0; k < 4; ++k) src[k] = (sw >> (5 * k)) & 31;
    const uint32_t row = kst + 4 * (K6_WORDS * g + 10 * y);
    uint32_t a[10], dlo[5], dhi[5], rot[5];
#pragma unroll
    for (int j = 0; j < 5; ++j) {
        const uint32_t w = __ldg(&c_k6_lanes.w[j][lane]);
        dlo[j] = kpi + (w & 0x7FFu);
        dhi[j] = kpi + ((w >> 11) & 0x7FFu);
        rot[j] = (w >> 22) & 31u;
        asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];"
                     : "=r"(a[2 * j]), "=r"(a[2 * j + 1])
                     : "r"(row + 8 * (w >> 27)));
    }
    const uint32_t rd = kpi + 4 * lane;
    const uint32_t iota_mask = (on && y == 0) ? 0xFFFFFFFFu : 0u;   // lane (0, 0) sits in slot 0 of row 0
#pragma unroll 1
    for (int round = 0; round < 24; ++round) {
        // theta, reduce-scatter: lane y collects column y (slot 5 - k of row y + k)
        uint32_t cl = a[0], ch = a[1];
#pragma unroll
        for (int k = 1; k < 5; ++k) {
            cl ^= __shfl_sync(FULL, a[2 * (5 - k)], src[k - 1]);
            ch ^= __shfl_sync(FULL, a[2 * (5 - k) + 1], src[k - 1]);
        }
        // all-gather: slot j takes the parity of column y + j from row y + j
        uint32_t c[10];
        c[0] = cl;
        c[1] = ch;
#pragma unroll
        for (int j = 1; j < 5; ++j) {
            c[2 * j] = __shfl_sync(FULL, cl, src[j - 1]);
            c[2 * j + 1] = __shfl_sync(FULL, ch, src[j - 1]);
        }
        // A[x] ^= C[x-1] ^ rotl(C[x+1], 1): neighbouring columns are neighbouring slots
#pragma unroll
        for (int j = 0; j < 5; ++j) {
            const int jm = 2 * ((j + 4) % 5), jp = 2 * ((j + 1) % 5);
            a[2 * j] ^= c[jm] ^ __funnelshift_l(c[jp + 1], c[jp], 1);
            a[2 * j + 1] ^= c[jm + 1] ^ __funnelshift_l(c[jp], c[jp + 1], 1);
        }
        // rho + pi: rotate slot j by rot[j] and store it at its destination
#pragma unroll
        for (int j = 0; j < 5; ++j) {
            const uint32_t nlo = __funnelshift_l(a[2 * j + 1], a[2 * j], rot[j]);
            const uint32_t nhi = __funnelshift_l(a[2 * j], a[2 * j + 1], rot[j]);
            if (on) {
                asm volatile("st.shared.u32 [%0], %1;" ::"r"(dlo[j]), "r"(nlo) : "memory");
                asm volatile("st.shared.u32 [%0], %1;" ::"r"(dhi[j]), "r"(nhi) : "memory");
            }
        }
        __syncwarp();
        uint32_t b[10];
#pragma unroll
        for (int j = 0; j < 5; ++j) {
            asm volatile("ld.shared.u32 %0, [%1];" : "=r"(b[2 * j]) : "r"(rd + 120 * j) : "memory");
            asm volatile("ld.shared.u32 %0, [%1];" : "=r"(b[2 * j + 1]) : "r"(rd + 640 + 120 * j) : "memory");
        }
        __syncwarp();
        // chi along the row: slots j + 1, j + 2 hold columns x + 1, x + 2
#pragma unroll
        for (int j = 0; j < 5; ++j) {
            const int j1 = 2 * ((j + 1) % 5), j2 = 2 * ((j + 2) % 5);
            a[2 * j] = b[2 * j] ^ (~b[j1] & b[j2]);
            a[2 * j + 1] = b[2 * j + 1] ^ (~b[j1 + 1] & b[j2 + 1]);
        }
        // iota on lane (0, 0): slot 0 of row 0
        const uint64_t rc = c_keccak_rc[round];
        a[0] ^= (uint32_t)rc & iota_mask;
        a[1] ^= (uint32_t)(rc >> 32) & iota_mask;
    }
    if (on) {
#pragma unroll
        for (int j = 0; j < 5; ++j)
            asm volatile("st.shared.v2.u32 [%0], {%1, %2};" ::"r"(row + 8 * (__ldg(&c_k6_lanes.w[j][lane]) >> 27)),
                         "r"(a[2 * j]), "r"(a[2 * j + 1])
                         : "memory");
    }
    __syncwarp();
}

__device__ __forceinline__ void keccak6_permute(uint32_t *kst, uint32_t *kpi) {
    keccak6_permute_impl(smem_addr(kst), smem_addr(kpi));
}

// Initialises `count` (<= 6) states in kst with padded one-block seeds: words
// [0, seed_words) from `seed` (shared memory, 4-byte aligned), then the word
// tail_of(g) (the instance's nonce bytes followed by the SHAKE domain/padding
// byte 0x1F), and the final padding bit at the last byte of the rate.
// States >= count are zeroed.
template <class Tail>
__device__ __forceinline__ void keccak6_seed(uint32_t *kst, const uint32_t *seed, int seed_words, Tail tail_of,
                                             int count, int rate, int lane) {
    for (int w = lane; w < K6_STATES * K6_WORDS; w += 32) {
        const int g = w / K6_WORDS, o = w % K6_WORDS;
        uint32_t v = 0;
        if (g < count) {
            if (o < seed_words) v = seed[o];
            else if (o == seed_words) v = tail_of(g);
            if (o == rate / 4 - 1) v ^= 0x80000000u;
        }
        kst[w] = v;
    }
    __syncwarp();
}

}  // namespace dil

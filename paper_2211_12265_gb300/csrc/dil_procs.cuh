// Fused procedure bodies: Alg 1 (Gen), Alg 2 (Sign) and Alg 3 (Verify) of
// arXiv 2211.12265, run by a group of P warps per task (P = 1 is the paper's
// single-warp form; P = 2 or 4 spreads a task's polynomials over several warps
// like its four-warp form, section 3.1, cutting per-task latency).
//
// Work inside a task is cut into polynomials (or pairs of polynomials whose
// sponges run interleaved); warp g of the group takes every P-th unit.  The
// group synchronises with a named barrier between phases.  Hashes over the
// whole task (mu, rho', c~, tr) run on one warp.  Per-warp shared memory holds
// NTT exchange buffers and squeezed blocks; per-group shared memory holds the
// task's seeds, the packed w1 hash input, c~ and the hint masks.  Per-task
// vectors that do not fit on chip (A^, s^1, s^2, t^0, y, y^, w, z) live in a
// global scratch area: NTT-domain polynomials in index order (lane t reads
// 8t..8t+7 with two 16-byte loads), plain ones in coefficient order (lane t
// reads t + 32m, coalesced).
#pragma once
#include "dil_sample.cuh"

namespace dil {

// Per-warp shared memory.  The sixteen-state sponges, the six-state ones
// (states, field windows) and the one- and two-state ones (sampled
// polynomials, squeezed blocks) are never live at the same time and share one
// area; buf doubles as the six-state permutation's pi exchange.
struct __align__(16) WarpSmem {
    union {
        struct {
            int32_t buf[K6_PI_WORDS];      // NTT exchanges / sampled polynomial (padded) / keccak6 pi exchange
            union {
                struct {
                    int32_t buf2[288];     // second sampled polynomial of a pair
                    uint8_t sq[688];       // squeezed SHAKE blocks (5 x 136 + slack)
                    uint8_t sq2[688];      // squeezed blocks of the second sponge of a pair
                };
                struct {
                    uint32_t kst[K6_STATES * K6_WORDS];   // six Keccak states
                    uint32_t win[K6_STATES * 38];         // ExpandMask field windows
                };
            };
        };
        struct {
            uint32_t k16[K16_WORDS];   // sixteen Keccak states
            uint32_t k16c[32];         // ExpandMask carry: each state's previous last lane
        };
    };
    __device__ uint32_t *kpi() { return reinterpret_cast<uint32_t *>(buf); }
};

// Per-task (per-group) shared memory.  Every region is 8-byte aligned.
struct __align__(16) GroupSmem {
    uint8_t hb[1128];    // K (32) | mu (64) | packed w1 (k * POLYW1) | slack
    uint8_t rhop[64];
    uint8_t rho[32];
    uint8_t ctilde[32];
    uint8_t tr[32];
    uint32_t hmask[64];  // hint bits: 8 words per polynomial
    int flag;            // reject flag of the current attempt
    int count;           // hint count of the current attempt
    int claim;           // broadcast slots of the persistent scheduler
    int claim2;
};

constexpr int HB_K = 0, HB_MU = 32, HB_W1 = 96;
constexpr int CTA_TABLE_BYTES = 2 * 256 * 4;

// Synchronises the P warps of one task group (barrier id `bar`).
template <int P>
__device__ __forceinline__ void group_sync(int bar) {
    if constexpr (P == 1) {
        __syncwarp();
    } else {
        asm volatile("bar.sync %0, %1;" ::"r"(bar), "r"(32 * P) : "memory");
    }
}

// Units of work: polynomials [0, M) cut into pairs when every warp of the
// group gets at least one pair, else into single polynomials.
template <int M, int P>
struct Units {
    static constexpr int SIZE = (M >= 2 * P) ? 2 : 1;
};

__device__ __forceinline__ void load_l2(int32_t v[8], const int32_t *p, int lane) {
    const int4 *q = reinterpret_cast<const int4 *>(p + 8 * lane);
    int4 a = q[0], b = q[1];
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
}

// As load_l2, through L2 only (data written by warps on other SMs).
__device__ __forceinline__ void load_l2_cg(int32_t v[8], const int32_t *p, int lane) {
    const int4 *q = reinterpret_cast<const int4 *>(p + 8 * lane);
    int4 a = __ldcg(q), b = __ldcg(q + 1);
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
}

__device__ __forceinline__ void store_l2(int32_t *p, const int32_t v[8], int lane) {
    int4 *q = reinterpret_cast<int4 *>(p + 8 * lane);
    q[0] = make_int4(v[0], v[1], v[2], v[3]);
    q[1] = make_int4(v[4], v[5], v[6], v[7]);
}

__device__ __forceinline__ void load_l0(int32_t v[8], const int32_t *p, int lane) {
#pragma unroll
    for (int m = 0; m < 8; ++m) v[m] = p[lane + 32 * m];
}

__device__ __forceinline__ void store_l0(int32_t *p, const int32_t v[8], int lane) {
#pragma unroll
    for (int m = 0; m < 8; ++m) p[lane + 32 * m] = v[m];
}

// Reads the shared buffer written by a sampler in L0 / L2 layout.
__device__ __forceinline__ void read_buf_l0(int32_t v[8], const int32_t *buf, int lane) {
#pragma unroll
    for (int m = 0; m < 8; ++m) v[m] = buf[lane + 36 * m];
}
__device__ __forceinline__ void read_buf_l2(int32_t v[8], const int32_t *buf, int lane) {
#pragma unroll
    for (int m = 0; m < 8; ++m) v[m] = buf[9 * lane + m];
}

// Unpacks one polynomial stored as `off - field` (BITS-bit fields) from a
// packed byte string in global memory, into layout L0.  Uses ws.sq as staging.
template <int BITS>
__device__ __forceinline__ void unpack_poly_l0(int32_t v[8], const uint8_t *__restrict__ src, int32_t off,
                                               WarpSmem &ws, int lane) {
    stage_bytes(ws.sq, src, N * BITS / 8, lane);
    __syncwarp();
#pragma unroll
    for (int m = 0; m < 8; ++m) v[m] = off - (int32_t)get_field(ws.sq, BITS * (lane + 32 * m), BITS);
    __syncwarp();
}

// Writes 8 consecutive coefficients (lane t: 8t..8t+7) as `off + sign v` in BITS bits.
template <int BITS>
__device__ __forceinline__ void pack_seq(uint8_t *dst_poly, const int32_t v[8], int32_t off, int sign, int lane) {
    uint32_t u[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) u[m] = (uint32_t)(off + sign * v[m]);
    pack8<BITS>(dst_poly + BITS * lane, u);
}

// Task t's message from the n + 1 byte offsets: start m0 and length.  False
// when the offsets decrease (invalid input): the caller rejects the task
// instead of reading out of bounds.
__device__ __forceinline__ bool message_of(const uint64_t *off, int t, uint64_t &m0, size_t &len) {
    m0 = off[t];
    const uint64_t m1 = off[t + 1];
    len = (size_t)(m1 - m0);
    return m1 >= m0;
}

// Per-task scratch layout (in polynomials of 256 int32).  Sign's area is a
// precomputation part (A^, s^1, s^2, t^0: read-only once prepared, shareable
// between workers) followed by a per-repetition part (y, y^, w, z: private to
// the worker running a repetition).
template <int LEVEL> struct Scratch {
    using V = Lv<LEVEL>;
    static constexpr int AH = 0;
    static constexpr int S1H = AH + V::K * V::L;
    static constexpr int S2H = S1H + V::L;
    static constexpr int T0H = S2H + V::K;
    static constexpr int PRE_POLYS = T0H + V::K;
    // offsets inside the per-repetition part; y is a ring of YRING
    // polynomials indexed by nonce (a one-warp worker samples masks
    // MASK_BATCH nonces at a time and keeps the ones later repetitions need)
    static constexpr int MASK_BATCH = K16_STATES;
    static constexpr int Y = 0;
    static constexpr int YRING = V::L + MASK_BATCH - 1;
    static constexpr int YH = Y + YRING;
    static constexpr int W = YH + V::L;
    static constexpr int Z = W + V::K;
    static constexpr int ITR_POLYS = Z + V::L;
    static constexpr int SIGN_POLYS = PRE_POLYS + ITR_POLYS;
    static constexpr int GEN_S = V::L + V::K * V::L;         // s1 || s2, coefficient order (one-warp groups)
    static constexpr int GEN_POLYS = GEN_S + V::L + V::K;     // s^1 | A^ | s1 || s2
    static constexpr int VERIFY_POLYS = V::L + V::K * V::L;   // z^, A^
    static constexpr int KEYED_VERIFY_POLYS = V::L;           // z^ (A^ is resident)
    // resident key: the Sign precomputation followed by NTT(t1 2^d)
    static constexpr int T1H = PRE_POLYS;
    static constexpr int KEY_POLYS = T1H + V::K;
};

// Warp g's share [share_lo(g), share_lo(g + 1)) of M polynomials cut into P
// contiguous ranges (so that each warp can batch its sponges).
template <int M, int P>
__device__ __forceinline__ int share_lo(int g) { return g * M / P; }

// A^_p (p = i l + j) for p in [lo, hi) into out + p N in index order: up to
// sixteen sponges at a time while at least seven remain, six at a time while
// at least three remain, then a pair or a single.  With a K16Rider the
// sixteen-state batches take fifteen polynomials and carry the rider's hash
// in the sixteenth instance; the hash is finished before the smaller forms
// reuse the batches' shared memory.
template <int LEVEL, class Rider>
__device__ void expand_a_range(const uint8_t *rho, int lo, int hi, int32_t *out, WarpSmem &ws, int lane,
                               Rider &rider) {
    constexpr int L = Lv<LEVEL>::L;
    int p = lo;
    while (hi - p >= 7) {
        const int c = min(Rider::KEEP, hi - p);
        expand_a_16<L>(rho, p, c, out + p * N, ws.k16, lane, rider);
        p += c;
    }
    if constexpr (Rider::KEEP < K16_STATES) rider.finish(ws.k16, lane);
    while (hi - p >= 3) {
        const int c = min(K6_STATES, hi - p);
        expand_a_six<L>(rho, p, c, out + p * N, ws.kst, ws.kpi(), lane);
        p += c;
    }
    int32_t a[8];
    if (hi - p == 2) {
        expand_a_pair(rho, p / L, p % L, (p + 1) / L, (p + 1) % L, ws.buf, ws.buf2, ws.sq, ws.sq2, lane);
        read_buf_l2(a, ws.buf2, lane);
        store_l2(out + (p + 1) * N, a, lane);
    } else if (hi - p == 1) {
        expand_a_poly(rho, p / L, p % L, ws.buf, ws.sq, lane);
    }
    if (hi - p >= 1) {
        read_buf_l2(a, ws.buf, lane);
        store_l2(out + p * N, a, lane);
    }
    __syncwarp();
}

template <int LEVEL>
__device__ __forceinline__ void expand_a_range(const uint8_t *rho, int lo, int hi, int32_t *out, WarpSmem &ws,
                                               int lane) {
    K16NoRider none;
    expand_a_range<LEVEL>(rho, lo, hi, out, ws, lane, none);
}

// Slot of nonce u's mask polynomial y (coefficient order) in the ring.
template <int LEVEL>
__device__ __forceinline__ int32_t *y_slot(int32_t *ring, int u) {
    return ring + (u % Scratch<LEVEL>::YRING) * N;
}

// y_j = ExpandMask(rho', kappa + j) into its ring slot and y^_j = NTT(y_j) in
// index order to yh + j N, for j in [lo, hi) (one warp's share of a
// repetition when a task group has several warps).
template <int LEVEL>
__device__ void expand_mask_range(const uint8_t *rhop, int kappa, int lo, int hi, int32_t *ring, int32_t *yh,
                                  WarpSmem &ws, const int32_t *zt, int lane) {
    using V = Lv<LEVEL>;
    int32_t r[8], a[8];
    int j = lo;
    while (hi - j >= 7) {
        const int c = min(K16_STATES, hi - j), u0 = kappa + j;
        expand_mask_16<V::ZBITS, V::GAMMA1>(
            rhop, u0, c, [&](int s) { return y_slot<LEVEL>(ring, u0 + s); }, ws.k16, ws.k16c, lane);
        __syncwarp();
#pragma unroll 1
        for (int u = j; u < j + c; ++u) {
            load_l0(r, y_slot<LEVEL>(ring, kappa + u), lane);
            ntt_fwd(r, ws.buf, zt, lane);
            store_l2(yh + u * N, r, lane);
        }
        j += c;
    }
    while (hi - j >= 3) {
        const int c = min(K6_STATES, hi - j), u0 = kappa + j;
        expand_mask_six<V::ZBITS, V::GAMMA1>(
            rhop, u0, c, [&](int g) { return y_slot<LEVEL>(ring, u0 + g); }, ws.kst, ws.kpi(), ws.win, lane);
        __syncwarp();
#pragma unroll 1
        for (int u = j; u < j + c; ++u) {
            load_l0(r, y_slot<LEVEL>(ring, kappa + u), lane);
            ntt_fwd(r, ws.buf, zt, lane);
            store_l2(yh + u * N, r, lane);
        }
        j += c;
    }
    if (hi - j == 2) {
        expand_mask_pair<V::ZBITS, V::GAMMA1>(rhop, kappa + j, kappa + j + 1, r, a, ws.sq, ws.sq2, lane);
        store_l0(y_slot<LEVEL>(ring, kappa + j + 1), a, lane);
        ntt_fwd(a, ws.buf, zt, lane);
        store_l2(yh + (j + 1) * N, a, lane);
    } else if (hi - j == 1) {
        expand_mask_poly<V::ZBITS, V::GAMMA1>(rhop, kappa + j, r, ws.sq, lane);
    }
    if (hi - j >= 1) {
        store_l0(y_slot<LEVEL>(ring, kappa + j), r, lane);
        ntt_fwd(r, ws.buf, zt, lane);
        store_l2(yh + j * N, r, lane);
    }
}

// A worker's stream of masks: the ring holds y for nonces [lo, hi).
struct MaskStream {
    int lo, hi;
};

// One-warp form: y for nonces [kappa, kappa + l) from the stream, which
// samples MASK_BATCH (sixteen) consecutive nonces at a time, so the leftovers
// of one repetition serve the next ones (a repetition that does not continue
// the stream restarts it at kappa); y^ into yh.
template <int LEVEL>
__device__ void mask_stream(const uint8_t *rhop, int kappa, MaskStream &ms, int32_t *ring, int32_t *yh,
                            WarpSmem &ws, const int32_t *zt, int lane) {
    using V = Lv<LEVEL>;
    if (kappa < ms.lo || kappa > ms.hi) ms.hi = kappa;
    ms.lo = kappa;
    while (ms.hi < kappa + V::L) {   // live nonces stay within [kappa, kappa + YRING)
        const int u0 = ms.hi;
        expand_mask_16<V::ZBITS, V::GAMMA1>(
            rhop, u0, K16_STATES, [&](int s) { return y_slot<LEVEL>(ring, u0 + s); }, ws.k16, ws.k16c, lane);
        ms.hi += Scratch<LEVEL>::MASK_BATCH;
    }
    __syncwarp();
    int32_t r[8];
#pragma unroll 1
    for (int j = 0; j < V::L; ++j) {
        load_l0(r, y_slot<LEVEL>(ring, kappa + j), lane);
        ntt_fwd(r, ws.buf, zt, lane);
        store_l2(yh + j * N, r, lane);
    }
}

// acc = sum_j A^_ij o v^_j (pointwise Montgomery products) for one row i of A^
// (ahat: the row's l polynomials, index order; read through L2 since another
// warp or kernel may have written them); v^_j (index order) at `vhat`.
__device__ __forceinline__ void accumulate_row(int32_t acc[8], const int32_t *ahat, int l, const int32_t *vhat,
                                               int lane) {
    int32_t a[8], v[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) acc[m] = 0;
#pragma unroll 1
    for (int j = 0; j < l; ++j) {
        load_l2_cg(a, ahat + j * N, lane);
        load_l2(v, vhat + j * N, lane);
#pragma unroll
        for (int m = 0; m < 8; ++m) acc[m] += mont_mul(a[m], v[m]);
    }
}

// c^ = NTT(SampleInBall(c~)) in layout L2 (every warp of a group computes it).
template <int LEVEL>
__device__ __forceinline__ void challenge_hat(int32_t ch[8], const uint8_t *ctilde, WarpSmem &ws,
                                              const int32_t *zt, int lane) {
    sample_in_ball<Lv<LEVEL>::TAU>(ctilde, ws.buf, ws.sq, lane);
    read_buf_l0(ch, ws.buf, lane);
    __syncwarp();
    ntt_fwd(ch, ws.buf, zt, lane);
}

// -------------------------------------------------------------------------
// Alg 1: Gen.  seed: 32 bytes.  pk, sk: outputs.  scratch: GEN_POLYS polys.
// -------------------------------------------------------------------------
template <int LEVEL, int P>
__device__ void gen_task(const uint8_t *__restrict__ seed, uint8_t *pk, uint8_t *sk, int32_t *scratch,
                         GroupSmem &gs, WarpSmem &ws, const int32_t *zt, const int32_t *izt, int g, int bar,
                         int lane) {
    using V = Lv<LEVEL>;
    int32_t r[8], a[8], acc[8];
    // (rho, rho', K) = H(zeta)  (Alg 1)
    if (g == 0) {
        stage_bytes(gs.hb, seed, 32, lane);
        __syncwarp();
        uint32_t lo = 0, hi = 0;
        absorb_smem(lo, hi, gs.hb, 32, 136, lane);
        squeeze_words(lo, hi, gs.hb, 16, lane);
        __syncwarp();
        uint8_t rb = gs.hb[lane], kb = gs.hb[96 + lane];
        gs.rho[lane] = rb;
        pk[lane] = rb;
        sk[lane] = rb;
        sk[32 + lane] = kb;
        gs.rhop[lane] = gs.hb[32 + lane];
        gs.rhop[32 + lane] = gs.hb[64 + lane];
    }
    group_sync<P>(bar);
    using S = Scratch<LEVEL>;
    int32_t *sraw = scratch + S::GEN_S * N;
    if constexpr (P == 1) {
        // s1 || s2 = ExpandS(rho'): all l + k sponges in one sixteen-state batch,
        // then s1: pack into sk, NTT
        expand_s_16<V::ETA>(gs.rhop, V::L + V::K, sraw, ws.k16, lane);
#pragma unroll 1
        for (int j = 0; j < V::L; ++j) {
            load_l2(a, sraw + j * N, lane);
            pack_seq<V::ETABITS>(sk + V::SK_S1 + j * V::POLYETA, a, V::ETA, -1, lane);
            load_l0(r, sraw + j * N, lane);
            ntt_fwd(r, ws.buf, zt, lane);
            store_l2(scratch + j * N, r, lane);
        }
    }
    // s1: sample, pack into sk, NTT (task groups of several warps)
    constexpr int U1 = Units<V::L, P>::SIZE;
#pragma unroll 1
    for (int j = U1 * g; j < V::L && P > 1; j += U1 * P) {
        const bool two = U1 == 2 && j + 1 < V::L;
        if (two)
            expand_s_pair<V::ETA>(gs.rhop, j, j + 1, ws.buf, ws.buf2, ws.sq, ws.sq2, lane);
        else
            expand_s_poly<V::ETA>(gs.rhop, j, ws.buf2, ws.sq, lane);
        for (int h = two ? 0 : 1; h < 2; ++h) {
            const int32_t *src = h ? ws.buf2 : ws.buf;
            const int jj = two ? j + h : j;
#pragma unroll
            for (int m = 0; m < 8; ++m) a[m] = src[8 * lane + m + 4 * (lane >> 2)];
            pack_seq<V::ETABITS>(sk + V::SK_S1 + jj * V::POLYETA, a, V::ETA, -1, lane);
            read_buf_l0(r, src, lane);
            __syncwarp();
            ntt_fwd(r, ws.buf, zt, lane);
            store_l2(scratch + jj * N, r, lane);
        }
    }
    // t = INTT(A^ o s^1) + s2; (t1, t0) = Power2Round(t), row i into pk and sk
    auto row = [&](int i) {
        accumulate_row(acc, scratch + (V::L + i * V::L) * N, V::L, scratch, lane);
#pragma unroll
        for (int m = 0; m < 8; ++m) acc[m] = reduce_q(acc[m]);
        ntt_inv(acc, ws.buf, izt, lane);
        if constexpr (P == 1) {
            load_l2(a, sraw + (V::L + i) * N, lane);
            load_l0(r, sraw + (V::L + i) * N, lane);
        } else {
            expand_s_poly<V::ETA>(gs.rhop, V::L + i, ws.buf, ws.sq, lane);
#pragma unroll
            for (int m = 0; m < 8; ++m) a[m] = ws.buf[8 * lane + m + 4 * (lane >> 2)];
            read_buf_l0(r, ws.buf, lane);
            __syncwarp();
        }
        pack_seq<V::ETABITS>(sk + V::SK_S2 + i * V::POLYETA, a, V::ETA, -1, lane);
        int32_t t1[8], t0[8];
#pragma unroll
        for (int m = 0; m < 8; ++m) {
            int32_t t = to_canonical(acc[m]) + r[m];      // (-eta, q + eta)
            t += (t < 0) ? Q : 0;
            t -= (t >= Q) ? Q : 0;
            power2round(t, t1[m], t0[m]);
        }
        l0_to_seq(t1, ws.buf, lane);
        pack_seq<10>(pk + 32 + i * V::POLYT1, t1, 0, 1, lane);
        l0_to_seq(t0, ws.buf, lane);
        pack_seq<D>(sk + V::SK_T0 + i * V::POLYT0, t0, 1 << (D - 1), -1, lane);
    };
    constexpr int KL = V::K * V::L;
    if constexpr (P == 1 && KL > K16_STATES) {
        // A^ in sixteen-state batches of whole rows (R l <= 15 polynomials), the
        // batch's rows of t computed before the next batch, and tr = H(rho || t1)
        // riding in the batches' spare instance as far as pk is written.
        constexpr int R = (K16_STATES - 1) / V::L;
        K16ChainRider rider(pk, V::PK, reinterpret_cast<uint32_t *>(gs.hb), reinterpret_cast<uint32_t *>(gs.tr));
        rider.set_ready(32);
#pragma unroll 1
        for (int i0 = 0; i0 < V::K; i0 += R) {
            const int rows = min(R, V::K - i0);
            expand_a_16<V::L>(gs.rho, i0 * V::L, rows * V::L, scratch + (V::L + i0 * V::L) * N, ws.k16, lane,
                              rider);
#pragma unroll 1
            for (int i = i0; i < i0 + rows; ++i) row(i);
            __syncwarp();
            rider.set_ready(32 + (size_t)(i0 + rows) * V::POLYT1);
        }
        rider.finish(lane);
        sk[64 + lane] = gs.tr[lane];
    } else {
        // A^ = ExpandA(rho) into scratch after s^1, then the rows of t
        expand_a_range<LEVEL>(gs.rho, share_lo<KL, P>(g), share_lo<KL, P>(g + 1), scratch + V::L * N, ws, lane);
        group_sync<P>(bar);
#pragma unroll 1
        for (int i = g; i < V::K; i += P) row(i);
        __threadfence_block();
        group_sync<P>(bar);
        // tr = H(rho || t1)
        if (g == 0) {
            uint32_t lo = 0, hi = 0;
            absorb_concat(lo, hi, gs.hb, 0, pk, V::PK, 136, lane);
            if (lane < 4) {
#pragma unroll
                for (int q = 0; q < 8; ++q) sk[64 + 8 * lane + q] = (uint8_t)((q < 4 ? lo : hi) >> (8 * (q & 3)));
            }
        }
    }
}

// -------------------------------------------------------------------------
// Alg 2: Sign
// -------------------------------------------------------------------------

// Copies polynomials [lo, hi) of src (a caller's A^, 256 words each) to dst
// with 16-byte loads and stores.
__device__ __forceinline__ void copy_polys(const int32_t *__restrict__ src, int lo, int hi, int32_t *dst, int lane) {
    const int4 *q = reinterpret_cast<const int4 *>(src + lo * N);
    int4 *d = reinterpret_cast<int4 *>(dst + lo * N);
#pragma unroll 2
    for (int i = lane; i < (hi - lo) * (N / 4); i += 32) d[i] = __ldg(q + i);
}

// Precomputation shared by every repetition: mu, rho', A^, s^1, s^2, t^0.
// AHAT: A^ is the caller's (ahat_in: k l polynomials, ExpandA(rho) of the
// task's key) and is copied instead of sampled.
template <int LEVEL, int P, bool AHAT = false>
__device__ void sign_prepare(const uint8_t *__restrict__ sk, const uint8_t *__restrict__ msg, size_t mlen,
                             int32_t *scratch, GroupSmem &gs, WarpSmem &ws, const int32_t *zt, int g, int bar,
                             int lane, const int32_t *__restrict__ ahat_in = nullptr) {
    using V = Lv<LEVEL>;
    using S = Scratch<LEVEL>;
    int32_t r[8];
    if (g == 0) {
        gs.rho[lane] = __ldg(sk + lane);
        gs.hb[HB_K + lane] = __ldg(sk + 32 + lane);
        gs.tr[lane] = __ldg(sk + 64 + lane);
    }
    group_sync<P>(bar);
    if (g == 0) {
        // mu = H(tr || M)  (Alg 2)
        uint32_t lo = 0, hi = 0;
        absorb_concat(lo, hi, gs.tr, 32, msg, mlen, 136, lane);
        squeeze_words(lo, hi, gs.hb + HB_MU, 8, lane);
        __syncwarp();
        // rho' = H(K || mu)
        lo = 0;
        hi = 0;
        absorb_smem(lo, hi, gs.hb + HB_K, 96, 136, lane);
        squeeze_words(lo, hi, gs.rhop, 8, lane);
        __syncwarp();
    }
    // A^ = ExpandA(rho)
    constexpr int KL = V::K * V::L;
    if constexpr (AHAT)
        copy_polys(ahat_in, share_lo<KL, P>(g), share_lo<KL, P>(g + 1), scratch + S::AH * N, lane);
    else
        expand_a_range<LEVEL>(gs.rho, share_lo<KL, P>(g), share_lo<KL, P>(g + 1), scratch + S::AH * N, ws, lane);
    // s^1, s^2, t^0: polynomials u = 0 .. l + 2k - 1 across the group
#pragma unroll 1
    for (int u = g; u < V::L + 2 * V::K; u += P) {
        if (u < V::L) {
            unpack_poly_l0<V::ETABITS>(r, sk + V::SK_S1 + u * V::POLYETA, V::ETA, ws, lane);
        } else if (u < V::L + V::K) {
            unpack_poly_l0<V::ETABITS>(r, sk + V::SK_S2 + (u - V::L) * V::POLYETA, V::ETA, ws, lane);
        } else {
            unpack_poly_l0<D>(r, sk + V::SK_T0 + (u - V::L - V::K) * V::POLYT0, 1 << (D - 1), ws, lane);
        }
        ntt_fwd(r, ws.buf, zt, lane);
        store_l2(scratch + (S::S1H + u) * N, r, lane);   // S1H, S2H, T0H are contiguous
    }
    group_sync<P>(bar);
}

// Per-message precomputation of a Sign with a resident key (A^, s^1, s^2, t^0
// already prepared): mu = H(tr || M) and rho' = H(K || mu) on warp 0.
// mu_in (nullable, global memory, 8-byte aligned): mu computed beforehand.
template <int LEVEL, int P>
__device__ void sign_prepare_keyed(const uint8_t *__restrict__ sk, const uint8_t *__restrict__ msg, size_t mlen,
                                   GroupSmem &gs, int g, int bar, int lane, const uint8_t *mu_in = nullptr) {
    if (g == 0) {
        gs.hb[HB_K + lane] = __ldg(sk + 32 + lane);
        gs.tr[lane] = __ldg(sk + 64 + lane);
        __syncwarp();
        uint32_t lo = 0, hi = 0;
        if (mu_in) {
            if (lane < 8)
                *reinterpret_cast<uint2 *>(gs.hb + HB_MU + 8 * lane) = __ldcg(reinterpret_cast<const uint2 *>(mu_in) + lane);
        } else {
            absorb_concat(lo, hi, gs.tr, 32, msg, mlen, 136, lane);
            squeeze_words(lo, hi, gs.hb + HB_MU, 8, lane);
        }
        __syncwarp();
        lo = 0;
        hi = 0;
        absorb_smem(lo, hi, gs.hb + HB_K, 96, 136, lane);
        squeeze_words(lo, hi, gs.rhop, 8, lane);
    }
    group_sync<P>(bar);
}

// Prepares one resident key: A^ = ExpandA(rho), s^1, s^2, t^0 (from sk, when
// given) and NTT(t1 2^d) into `key` (KEY_POLYS polynomials), tr = H(pk).
template <int LEVEL, int P>
__device__ void key_prepare(const uint8_t *__restrict__ pk, const uint8_t *__restrict__ sk, int32_t *key,
                            uint8_t *tr_out, GroupSmem &gs, WarpSmem &ws, const int32_t *zt, int g, int bar,
                            int lane) {
    using V = Lv<LEVEL>;
    using S = Scratch<LEVEL>;
    int32_t r[8];
    if (g == 0) gs.rho[lane] = __ldg(pk + lane);
    group_sync<P>(bar);
    constexpr int KL = V::K * V::L;
    expand_a_range<LEVEL>(gs.rho, share_lo<KL, P>(g), share_lo<KL, P>(g + 1), key + S::AH * N, ws, lane);
    // s^1, s^2, t^0 (when the secret key is resident) and NTT(t1 2^d)
    const int first = sk ? 0 : V::L + 2 * V::K;
#pragma unroll 1
    for (int u = first + g; u < V::L + 3 * V::K; u += P) {
        if (u < V::L) {
            unpack_poly_l0<V::ETABITS>(r, sk + V::SK_S1 + u * V::POLYETA, V::ETA, ws, lane);
        } else if (u < V::L + V::K) {
            unpack_poly_l0<V::ETABITS>(r, sk + V::SK_S2 + (u - V::L) * V::POLYETA, V::ETA, ws, lane);
        } else if (u < V::L + 2 * V::K) {
            unpack_poly_l0<D>(r, sk + V::SK_T0 + (u - V::L - V::K) * V::POLYT0, 1 << (D - 1), ws, lane);
        } else {
            unpack_poly_l0<10>(r, pk + 32 + (u - V::L - 2 * V::K) * V::POLYT1, 0, ws, lane);
#pragma unroll
            for (int m = 0; m < 8; ++m) r[m] = (-r[m]) << D;   // t1 2^d
        }
        ntt_fwd(r, ws.buf, zt, lane);
        store_l2(key + (S::S1H + u) * N, r, lane);   // S1H, S2H, T0H, T1H are contiguous
    }
    if (g == P - 1) {
        uint32_t lo = 0, hi = 0;
        absorb_concat(lo, hi, gs.tr, 0, pk, V::PK, 136, lane);
        squeeze_words(lo, hi, gs.tr, 4, lane);
        __syncwarp();
        tr_out[lane] = gs.tr[lane];
    }
    group_sync<P>(bar);
}

// First half of one repetition of the rejection loop of Alg 2 with nonce
// base kappa: y, y^ = NTT(y), w = INTT(A^ o y^) (kept in scratch W), w1 and
// c~ = H(mu || w1) into gs.ctilde; leaves gs.flag = 0 and gs.count = 0.
// pre: the task's precomputation part (possibly prepared by another warp
// group, so it is read through L2); itr: this worker's per-repetition part.
// stop_below / rep: a speculative repetition rep of the persistent form
// stops before hashing c~ once *stop_below (the smallest accepting repetition
// found so far) is below rep; it then returns false.
template <int LEVEL, int P>
__device__ bool sign_front(int kappa, const int32_t *pre, int32_t *itr, MaskStream &ms, GroupSmem &gs,
                           WarpSmem &ws, const int32_t *zt, const int32_t *izt, int g, int bar, int lane,
                           const int *stop_below = nullptr, int rep = 0) {
    using V = Lv<LEVEL>;
    using S = Scratch<LEVEL>;
    volatile int *vflag = &gs.flag;
    int32_t r[8], a[8], acc[8];
    // y = ExpandMask(rho', kappa); y^ = NTT(y)
    if constexpr (P == 1)
        mask_stream<LEVEL>(gs.rhop, kappa, ms, itr + S::Y * N, itr + S::YH * N, ws, zt, lane);
    else
        expand_mask_range<LEVEL>(gs.rhop, kappa, share_lo<V::L, P>(g), share_lo<V::L, P>(g + 1), itr + S::Y * N,
                                 itr + S::YH * N, ws, zt, lane);
    group_sync<P>(bar);
    // w = INTT(A^ o y^); w1 = HighBits(w)
#pragma unroll 1
    for (int i = g; i < V::K; i += P) {
#pragma unroll
        for (int m = 0; m < 8; ++m) acc[m] = 0;
#pragma unroll 1
        for (int j = 0; j < V::L; ++j) {
            load_l2_cg(a, pre + (S::AH + i * V::L + j) * N, lane);
            load_l2(r, itr + (S::YH + j) * N, lane);
#pragma unroll
            for (int m = 0; m < 8; ++m) acc[m] += mont_mul(a[m], r[m]);
        }
#pragma unroll
        for (int m = 0; m < 8; ++m) acc[m] = reduce_q(acc[m]);
        ntt_inv(acc, ws.buf, izt, lane);
#pragma unroll
        for (int m = 0; m < 8; ++m) {
            acc[m] = to_canonical(acc[m]);
            r[m] = highbits<LEVEL>(acc[m]);
        }
        store_l0(itr + (S::W + i) * N, acc, lane);
        l0_to_seq(r, ws.buf, lane);
        pack_seq<V::W1BITS>(gs.hb + HB_W1 + i * V::POLYW1, r, 0, 1, lane);
    }
    group_sync<P>(bar);
    // c~ = H(mu || w1)
    if (g == 0) {
        int stop = 0;
        if (stop_below) stop = __shfl_sync(FULL, lane == 0 ? (int)(__ldcg(stop_below) < rep) : 0, 0);
        if (!stop) {
            uint32_t lo = 0, hi = 0;
            absorb_smem(lo, hi, gs.hb + HB_MU, 64 + V::K * V::POLYW1, 136, lane);
            squeeze_words(lo, hi, gs.ctilde, 4, lane);
        }
        if (lane == 0) {
            gs.flag = stop;
            gs.count = 0;
        }
    }
    group_sync<P>(bar);
    return !*vflag;
}

// Second half of the repetition, with early evaluation: each polynomial is
// checked as soon as it is produced.  Needs gs.ctilde, gs.flag = gs.count = 0
// and the first half's scratch (y ring, W).  Returns true (on every warp of
// the group) when (z, h) is accepted; then gs.ctilde, scratch Z and gs.hmask
// hold the signature parts.
template <int LEVEL, int P>
__device__ bool sign_back(int kappa, const int32_t *pre, int32_t *itr, GroupSmem &gs, WarpSmem &ws,
                          const int32_t *zt, const int32_t *izt, int g, int bar, int lane) {
    using V = Lv<LEVEL>;
    using S = Scratch<LEVEL>;
    volatile int *vflag = &gs.flag;
    int32_t r[8], a[8], ch[8];
    // c^ = NTT(SampleInBall(c~))
    challenge_hat<LEVEL>(ch, gs.ctilde, ws, zt, lane);
    // z = y + INTT(c^ o s^1); reject if ||z|| >= gamma1 - beta
#pragma unroll 1
    for (int j = g; j < V::L && !*vflag; j += P) {
        load_l2_cg(a, pre + (S::S1H + j) * N, lane);
#pragma unroll
        for (int m = 0; m < 8; ++m) r[m] = mont_mul(ch[m], a[m]);
        ntt_inv(r, ws.buf, izt, lane);
        load_l0(a, y_slot<LEVEL>(itr + S::Y * N, kappa + j), lane);
        bool bad = false;
#pragma unroll
        for (int m = 0; m < 8; ++m) {
            r[m] = centre_small(to_canonical(r[m]) + a[m]);
            bad |= iabs(r[m]) >= V::GAMMA1 - V::BETA;
        }
        if (__any_sync(FULL, bad)) {
            if (lane == 0) *vflag = 1;
            break;
        }
        store_l0(itr + (S::Z + j) * N, r, lane);
    }
    // v_s = INTT(c^ o s^2); r0 = LowBits(w - v_s)
#pragma unroll 1
    for (int i = g; i < V::K && !*vflag; i += P) {
        load_l2_cg(a, pre + (S::S2H + i) * N, lane);
#pragma unroll
        for (int m = 0; m < 8; ++m) r[m] = mont_mul(ch[m], a[m]);
        ntt_inv(r, ws.buf, izt, lane);
        load_l0(a, itr + (S::W + i) * N, lane);
        bool bad = false;
#pragma unroll
        for (int m = 0; m < 8; ++m) {
            int32_t d = a[m] - r[m];                 // (-q, 2q)
            d += (d < 0) ? Q : 0;
            d -= (d >= Q) ? Q : 0;
            int32_t h1, l0;
            decompose<LEVEL>(d, h1, l0);
            bad |= iabs(l0) >= V::GAMMA2 - V::BETA;
            a[m] = d;
        }
        if (__any_sync(FULL, bad)) {
            if (lane == 0) *vflag = 1;
            break;
        }
        store_l0(itr + (S::W + i) * N, a, lane);  // keep w - c s2 for the hint
    }
    group_sync<P>(bar);
    if (*vflag) return false;
    // v_t = INTT(c^ o t^0); h = MakeHint(-v_t, w - v_s + v_t)
#pragma unroll 1
    for (int i = g; i < V::K && !*vflag; i += P) {
        load_l2_cg(a, pre + (S::T0H + i) * N, lane);
#pragma unroll
        for (int m = 0; m < 8; ++m) r[m] = mont_mul(ch[m], a[m]);
        ntt_inv(r, ws.buf, izt, lane);
        load_l0(a, itr + (S::W + i) * N, lane);
        bool bad = false;
        uint32_t hbits = 0;
#pragma unroll
        for (int m = 0; m < 8; ++m) {
            int32_t vt = to_canonical(r[m]);
            bad |= iabs(to_centred(vt)) >= V::GAMMA2;
            int32_t rr = a[m] + vt;
            rr -= (rr >= Q) ? Q : 0;
            int32_t z = vt ? Q - vt : 0;
            hbits |= (uint32_t)make_hint<LEVEL>(z, rr) << m;
        }
        if (__any_sync(FULL, bad)) {
            if (lane == 0) *vflag = 1;
            break;
        }
        int count = 0;
#pragma unroll
        for (int m = 0; m < 8; ++m) {
            uint32_t w = __ballot_sync(FULL, (hbits >> m) & 1u);
            if (lane == 0) gs.hmask[i * 8 + m] = w;
            count += __popc(w);
        }
        if (lane == 0) atomicAdd(&gs.count, count);
    }
    group_sync<P>(bar);
    return !*vflag && gs.count <= V::OMEGA;
}

// One repetition: the two halves in one kernel.  Returns true when
// (z, h) is accepted.
template <int LEVEL, int P>
__device__ bool sign_attempt(int kappa, const int32_t *pre, int32_t *itr, MaskStream &ms, GroupSmem &gs,
                             WarpSmem &ws, const int32_t *zt, const int32_t *izt, int g, int bar, int lane,
                             const int *stop_below = nullptr, int rep = 0) {
    return sign_front<LEVEL, P>(kappa, pre, itr, ms, gs, ws, zt, izt, g, bar, lane, stop_below, rep) &&
           sign_back<LEVEL, P>(kappa, pre, itr, gs, ws, zt, izt, g, bar, lane);
}

// Writes sig = c~ || z (gamma1 - z in ZBITS bits) || h (indices, then counts).
template <int LEVEL, int P>
__device__ void sign_pack(uint8_t *sig, const int32_t *itr, const GroupSmem &gs, int g, int lane) {
    using V = Lv<LEVEL>;
    using S = Scratch<LEVEL>;
#pragma unroll 1
    for (int j = g; j < V::L; j += P) {
        int32_t v[8];
        load_l2(v, itr + (S::Z + j) * N, lane);   // 8 consecutive coefficients
        pack_seq<V::ZBITS>(sig + V::SIG_Z + j * V::POLYZ, v, V::GAMMA1, -1, lane);
    }
    if (g != P - 1) return;
    sig[lane] = gs.ctilde[lane];
    uint8_t *h = sig + V::SIG_H;
    int base = 0;
#pragma unroll 1
    for (int i = 0; i < V::K; ++i) {
#pragma unroll
        for (int m = 0; m < 8; ++m) {
            uint32_t w = gs.hmask[i * 8 + m];
            if ((w >> lane) & 1u) h[base + __popc(w & lanemask_lt(lane))] = (uint8_t)(lane + 32 * m);
            base += __popc(w);
        }
        if (lane == 0) h[V::OMEGA + i] = (uint8_t)base;
    }
    for (int p = base + lane; p < V::OMEGA; p += 32) h[p] = 0;
}

template <int LEVEL, int P>
__device__ void sign_zero(uint8_t *sig, int g, int lane) {
    for (int p = 32 * g + lane; p < Lv<LEVEL>::SIG; p += 32 * P) sig[p] = 0;
}

// -------------------------------------------------------------------------
// Alg 3: Verify.  Returns 1 (accept) or 0 on every warp of the group.
// scratch: VERIFY_POLYS polys.
// -------------------------------------------------------------------------
// KEYED: the public key is resident; `key` holds its A^ and NTT(t1 2^d)
// (KEY_POLYS layout) and `tr` its H(pk), so neither is recomputed.
// AHAT: `key` is the caller's A^ of this key (k l polynomials, ExpandA(rho));
// t1 and H(pk) come from pk as in the plain form.
// mu_in (nullable, KEYED only, global memory, 8-byte aligned): mu computed
// beforehand.
template <int LEVEL, int P, bool KEYED = false, bool AHAT = false>
__device__ int verify_task(const uint8_t *__restrict__ pk, const uint8_t *__restrict__ msg, size_t mlen,
                           const uint8_t *__restrict__ sig, int32_t *scratch, GroupSmem &gs, WarpSmem &ws,
                           const int32_t *zt, const int32_t *izt, int g, int bar, int lane,
                           const int32_t *key = nullptr, const uint8_t *tr = nullptr,
                           const uint8_t *mu_in = nullptr) {
    using V = Lv<LEVEL>;
    volatile int *vflag = &gs.flag;
    int32_t r[8], acc[8], ch[8];
    if (g == 0) {
        gs.ctilde[lane] = __ldcg(sig + lane);
        gs.rho[lane] = __ldg(pk + lane);
        // strict hint decoding into bit masks
        stage_bytes(ws.sq, sig + V::SIG_H, V::OMEGA + V::K, lane);
        gs.hmask[lane] = 0;
        gs.hmask[32 + lane] = 0;
        __syncwarp();
        bool bad = false;
        int prev = 0;
#pragma unroll 1
        for (int i = 0; i < V::K; ++i) {
            int end = ws.sq[V::OMEGA + i];
            if (end < prev || end > V::OMEGA) {
                bad = true;
                break;
            }
            for (int j = prev + lane; j < end; j += 32) {
                int idx = ws.sq[j];
                if (j > prev && idx <= ws.sq[j - 1]) bad = true;
                atomicOr(&gs.hmask[i * 8 + (idx >> 5)], 1u << (idx & 31));
            }
            prev = end;
        }
        if (!bad)
            for (int j = prev + lane; j < V::OMEGA; j += 32)
                if (ws.sq[j]) bad = true;
        bad = __any_sync(FULL, bad);
        if (lane == 0) gs.flag = bad ? 1 : 0;
    }
    group_sync<P>(bar);
    if (*vflag) return 0;
    // z: unpack, ||z|| < gamma1 - beta, z^ = NTT(z)  (Alg 3)
#pragma unroll 1
    for (int j = g; j < V::L && !*vflag; j += P) {
        unpack_poly_l0<V::ZBITS>(r, sig + V::SIG_Z + j * V::POLYZ, V::GAMMA1, ws, lane);
        bool b = false;
#pragma unroll
        for (int m = 0; m < 8; ++m) b |= iabs(r[m]) >= V::GAMMA1 - V::BETA;
        if (__any_sync(FULL, b)) {
            if (lane == 0) *vflag = 1;
            break;
        }
        ntt_fwd(r, ws.buf, zt, lane);
        store_l2(scratch + j * N, r, lane);
    }
    // A^ = ExpandA(rho) into scratch after z^ (unless resident).  A single
    // warp with more than one sixteen-state batch of A^ carries H(pk) in the
    // batches' spare instance.
    constexpr int KL = V::K * V::L;
    constexpr bool RIDE = P == 1 && !KEYED && !AHAT && KL > K16_STATES;
    if constexpr (RIDE) {
        K16Rider rider(pk, V::PK, reinterpret_cast<uint32_t *>(gs.tr));
        expand_a_range<LEVEL>(gs.rho, 0, KL, scratch + V::L * N, ws, lane, rider);
    } else if (!KEYED && !AHAT) {
        expand_a_range<LEVEL>(gs.rho, share_lo<KL, P>(g), share_lo<KL, P>(g + 1), scratch + V::L * N, ws, lane);
    }
    // mu = H(H(rho || t1) || M), on the last warp
    if (g == P - 1) {
        uint32_t lo = 0, hi = 0;
        if (KEYED) {
            gs.tr[lane] = __ldcg(tr + lane);
        } else if (!RIDE) {
            absorb_concat(lo, hi, gs.tr, 0, pk, V::PK, 136, lane);
            squeeze_words(lo, hi, gs.tr, 4, lane);
        }
        __syncwarp();
        lo = 0;
        hi = 0;
        if (KEYED && mu_in) {
            if (lane < 8)
                *reinterpret_cast<uint2 *>(gs.hb + HB_MU + 8 * lane) = __ldcg(reinterpret_cast<const uint2 *>(mu_in) + lane);
        } else {
            absorb_concat(lo, hi, gs.tr, 32, msg, mlen, 136, lane);
            squeeze_words(lo, hi, gs.hb + HB_MU, 8, lane);
        }
    }
    group_sync<P>(bar);
    if (*vflag) return 0;
    // c^ = NTT(SampleInBall(c~))
    challenge_hat<LEVEL>(ch, gs.ctilde, ws, zt, lane);
    // v = INTT(A^ o z^ - c^ o NTT(t1 2^d)); w1' = UseHint(h, v)
    using S = Scratch<LEVEL>;
    const int32_t *ahat = KEYED ? key + S::AH * N : AHAT ? key : scratch + V::L * N;
#pragma unroll 1
    for (int i = g; i < V::K; i += P) {
        accumulate_row(acc, ahat + i * V::L * N, V::L, scratch, lane);
        if (KEYED) {
            load_l2_cg(r, key + (S::T1H + i) * N, lane);
        } else {
            unpack_poly_l0<10>(r, pk + 32 + i * V::POLYT1, 0, ws, lane);
#pragma unroll
            for (int m = 0; m < 8; ++m) r[m] = (-r[m]) << D;   // t1 2^d, t1 stored as 0 - field
            ntt_fwd(r, ws.buf, zt, lane);
        }
#pragma unroll
        for (int m = 0; m < 8; ++m) acc[m] = reduce_q(acc[m] - mont_mul(ch[m], r[m]));
        ntt_inv(acc, ws.buf, izt, lane);
#pragma unroll
        for (int m = 0; m < 8; ++m) {
            int hbit = (gs.hmask[i * 8 + m] >> lane) & 1u;
            r[m] = use_hint<LEVEL>(hbit, to_canonical(acc[m]));
        }
        l0_to_seq(r, ws.buf, lane);
        pack_seq<V::W1BITS>(gs.hb + HB_W1 + i * V::POLYW1, r, 0, 1, lane);
    }
    group_sync<P>(bar);
    // c~ == H(mu || w1')
    if (g == 0) {
        uint32_t lo = 0, hi = 0;
        absorb_smem(lo, hi, gs.hb + HB_MU, 64 + V::K * V::POLYW1, 136, lane);
        bool eq = true;
        if (lane < 4) {
            uint2 w = *reinterpret_cast<const uint2 *>(gs.ctilde + 8 * lane);
            eq = (w.x == lo) && (w.y == hi);
        }
        eq = __all_sync(FULL, eq);
        if (lane == 0) gs.flag = eq ? 0 : 1;
    }
    group_sync<P>(bar);
    return *vflag ? 0 : 1;
}

}  // namespace dil

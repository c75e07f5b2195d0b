// Fused warp-per-task procedure bodies: Alg 1 (Gen), Alg 2 (Sign) and Alg 3
// (Verify) of arXiv 2211.12265.  One warp owns one task end to end (the
// paper's single-warp form, section 4.2), keeping polynomials in registers and
// a small per-warp shared-memory area, and spilling the per-task vectors that
// do not fit (A^, s^1, s^2, t^0, y, y^, w, z) to a global scratch area.
//
// Global scratch polynomials hold 256 int32 each.  NTT-domain polynomials are
// stored in index order (lane t reads 8t..8t+7 with two 16-byte loads); plain
// polynomials in coefficient order (lane t reads t + 32m, coalesced).
#pragma once
#include "dil_sample.cuh"

namespace dil {

// Per-warp shared memory.  Every region is 8-byte aligned.
struct __align__(16) WarpSmem {
    int32_t buf[288];       // NTT exchanges / sampled polynomials (padded)
    uint8_t sq[688];        // squeezed SHAKE blocks (5 x 136 + slack)
    uint8_t hb[1128];       // K (32) | mu (64) | packed w1 (k * POLYW1) | slack
    uint8_t rhop[64];       // rho'
    uint8_t rho[32];
    uint8_t ctilde[32];
    uint8_t tr[32];
    uint32_t hmask[64];     // hint bits: 8 words per polynomial
};

constexpr int HB_K = 0, HB_MU = 32, HB_W1 = 96;
constexpr int CTA_TABLE_BYTES = 2 * 256 * 4;

__device__ __forceinline__ void load_l2(int32_t v[8], const int32_t *__restrict__ p, int lane) {
    const int4 *q = reinterpret_cast<const int4 *>(p + 8 * lane);
    int4 a = q[0], b = q[1];
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
}

__device__ __forceinline__ void store_l2(int32_t *p, const int32_t v[8], int lane) {
    int4 *q = reinterpret_cast<int4 *>(p + 8 * lane);
    q[0] = make_int4(v[0], v[1], v[2], v[3]);
    q[1] = make_int4(v[4], v[5], v[6], v[7]);
}

__device__ __forceinline__ void load_l0(int32_t v[8], const int32_t *__restrict__ p, int lane) {
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

// Writes 8 consecutive coefficients (lane t: 8t..8t+7) as `off - v` in BITS bits.
template <int BITS>
__device__ __forceinline__ void pack_seq(uint8_t *dst_poly, const int32_t v[8], int32_t off, int sign, int lane) {
    uint32_t u[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) u[m] = (uint32_t)(off + sign * v[m]);
    pack8<BITS>(dst_poly + BITS * lane, u);
}

// Per-task scratch layout (in polynomials of 256 int32).
template <int LEVEL> struct Scratch {
    using V = Lv<LEVEL>;
    static constexpr int AH = 0;
    static constexpr int S1H = AH + V::K * V::L;
    static constexpr int S2H = S1H + V::L;
    static constexpr int T0H = S2H + V::K;
    static constexpr int Y = T0H + V::K;
    static constexpr int YH = Y + V::L;
    static constexpr int W = YH + V::L;
    static constexpr int Z = W + V::K;
    static constexpr int SIGN_POLYS = Z + V::L;
    static constexpr int GEN_POLYS = V::L;     // s^1
    static constexpr int VERIFY_POLYS = V::L;  // z^
};

// -------------------------------------------------------------------------
// Alg 1: Gen.  seed: 32 bytes.  pk, sk: outputs.  scratch: GEN_POLYS polys.
// -------------------------------------------------------------------------
template <int LEVEL>
__device__ void gen_task(const uint8_t *__restrict__ seed, uint8_t *pk, uint8_t *sk,
                         int32_t *__restrict__ scratch, WarpSmem &ws, const int32_t *zt, const int32_t *izt,
                         const KLane &k, int lane) {
    using V = Lv<LEVEL>;
    using S = Scratch<LEVEL>;
    int32_t r[8], a[8], acc[8];
    // (rho, rho', K) = H(zeta)  (Alg 1 l.2)
    stage_bytes(ws.hb, seed, 32, lane);
    __syncwarp();
    uint32_t lo = 0, hi = 0;
    absorb_smem(lo, hi, k, ws.hb, 32, 136, lane);
    squeeze_words(lo, hi, ws.hb, 16, lane);
    __syncwarp();
    if (lane < 32) {
        uint8_t rb = ws.hb[lane], kb = ws.hb[96 + lane];
        ws.rho[lane] = rb;
        pk[lane] = rb;
        sk[lane] = rb;
        sk[32 + lane] = kb;
        ws.rhop[lane] = ws.hb[32 + lane];
        ws.rhop[32 + lane] = ws.hb[64 + lane];
    }
    __syncwarp();
    // s1: sample, pack into sk, NTT  (l.4)
    for (int j = 0; j < V::L; ++j) {
        expand_s_poly<V::ETA>(ws.rhop, j, ws.buf, ws.sq, k, lane);
#pragma unroll
        for (int m = 0; m < 8; ++m) a[m] = ws.buf[8 * lane + m + 4 * (lane >> 2)];
        pack_seq<V::ETABITS>(sk + V::SK_S1 + j * V::POLYETA, a, V::ETA, -1, lane);
        read_buf_l0(r, ws.buf, lane);
        __syncwarp();
        ntt_fwd(r, ws.buf, zt, lane);
        store_l2(scratch + j * N, r, lane);
    }
    // t = INTT(A^ o s^1) + s2; (t1, t0) = Power2Round(t)  (l.3, l.5, l.6)
    for (int i = 0; i < V::K; ++i) {
#pragma unroll
        for (int m = 0; m < 8; ++m) acc[m] = 0;
        for (int j = 0; j < V::L; ++j) {
            expand_a_poly(ws.rho, i, j, ws.buf, ws.sq, k, lane);
            read_buf_l2(a, ws.buf, lane);
            __syncwarp();
            load_l2(r, scratch + j * N, lane);
#pragma unroll
            for (int m = 0; m < 8; ++m) acc[m] += mont_mul(a[m], r[m]);
        }
#pragma unroll
        for (int m = 0; m < 8; ++m) acc[m] = reduce_q(acc[m]);
        ntt_inv(acc, ws.buf, izt, lane);
        expand_s_poly<V::ETA>(ws.rhop, V::L + i, ws.buf, ws.sq, k, lane);
#pragma unroll
        for (int m = 0; m < 8; ++m) a[m] = ws.buf[8 * lane + m + 4 * (lane >> 2)];
        pack_seq<V::ETABITS>(sk + V::SK_S2 + i * V::POLYETA, a, V::ETA, -1, lane);
        read_buf_l0(r, ws.buf, lane);
        __syncwarp();
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
    }
    __syncwarp();
    __threadfence_block();
    // tr = H(rho || t1)  (l.7)
    lo = 0;
    hi = 0;
    absorb_concat(lo, hi, k, ws.hb, 0, pk, V::PK, 136, lane);
    if (lane < 4) {
#pragma unroll
        for (int q = 0; q < 8; ++q) sk[64 + 8 * lane + q] = (uint8_t)((q < 4 ? lo : hi) >> (8 * (q & 3)));
    }
}

// -------------------------------------------------------------------------
// Alg 2: Sign.  Returns 0 on success, -5 when max_iter repetitions rejected.
// scratch: SIGN_POLYS polys.  *iters receives the number of repetitions.
// -------------------------------------------------------------------------

// Precomputation shared by every repetition: mu, rho', A^, s^1, s^2, t^0.
template <int LEVEL>
__device__ void sign_prepare(const uint8_t *__restrict__ sk, const uint8_t *__restrict__ msg, size_t mlen,
                             int32_t *__restrict__ scratch, WarpSmem &ws, const int32_t *zt, const KLane &k,
                             int lane) {
    using V = Lv<LEVEL>;
    using S = Scratch<LEVEL>;
    int32_t r[8];
    if (lane < 32) {
        ws.rho[lane] = __ldg(sk + lane);
        ws.hb[HB_K + lane] = __ldg(sk + 32 + lane);
        ws.tr[lane] = __ldg(sk + 64 + lane);
    }
    __syncwarp();
    // mu = H(tr || M)  (Alg 2 l.1)
    uint32_t lo = 0, hi = 0;
    absorb_concat(lo, hi, k, ws.tr, 32, msg, mlen, 136, lane);
    squeeze_words(lo, hi, ws.hb + HB_MU, 8, lane);
    __syncwarp();
    // rho' = H(K || mu)  (l.2)
    lo = 0;
    hi = 0;
    absorb_smem(lo, hi, k, ws.hb + HB_K, 96, 136, lane);
    squeeze_words(lo, hi, ws.rhop, 8, lane);
    __syncwarp();
    // A^ = ExpandA(rho)  (l.3)
    for (int i = 0; i < V::K; ++i)
        for (int j = 0; j < V::L; ++j) {
            expand_a_poly(ws.rho, i, j, ws.buf, ws.sq, k, lane);
            int32_t a[8];
            read_buf_l2(a, ws.buf, lane);
            __syncwarp();
            store_l2(scratch + (S::AH + i * V::L + j) * N, a, lane);
        }
    // s^1, s^2, t^0  (l.4)
    for (int j = 0; j < V::L; ++j) {
        unpack_poly_l0<V::ETABITS>(r, sk + V::SK_S1 + j * V::POLYETA, V::ETA, ws, lane);
        ntt_fwd(r, ws.buf, zt, lane);
        store_l2(scratch + (S::S1H + j) * N, r, lane);
    }
    for (int i = 0; i < V::K; ++i) {
        unpack_poly_l0<V::ETABITS>(r, sk + V::SK_S2 + i * V::POLYETA, V::ETA, ws, lane);
        ntt_fwd(r, ws.buf, zt, lane);
        store_l2(scratch + (S::S2H + i) * N, r, lane);
    }
    for (int i = 0; i < V::K; ++i) {
        unpack_poly_l0<D>(r, sk + V::SK_T0 + i * V::POLYT0, 1 << (D - 1), ws, lane);
        ntt_fwd(r, ws.buf, zt, lane);
        store_l2(scratch + (S::T0H + i) * N, r, lane);
    }
}

// One repetition of the rejection loop with nonce base kappa (l.6-18), with
// early evaluation: each polynomial is checked as soon as it is produced.
// Returns true when (z, h) is accepted; then ws.ctilde, scratch Z and ws.hmask
// hold the signature parts.
template <int LEVEL>
__device__ bool sign_attempt(int kappa, int32_t *__restrict__ scratch, WarpSmem &ws, const int32_t *zt,
                             const int32_t *izt, const KLane &k, int lane) {
    using V = Lv<LEVEL>;
    using S = Scratch<LEVEL>;
    int32_t r[8], a[8], acc[8], ch[8];
    // y = ExpandMask(rho', kappa); y^ = NTT(y)  (l.6)
    for (int j = 0; j < V::L; ++j) {
        expand_mask_poly<V::ZBITS, V::GAMMA1>(ws.rhop, kappa + j, r, ws.sq, k, lane);
        store_l0(scratch + (S::Y + j) * N, r, lane);
        ntt_fwd(r, ws.buf, zt, lane);
        store_l2(scratch + (S::YH + j) * N, r, lane);
    }
    // w = INTT(A^ o y^); w1 = HighBits(w)  (l.7-8)
    for (int i = 0; i < V::K; ++i) {
#pragma unroll
        for (int m = 0; m < 8; ++m) acc[m] = 0;
        for (int j = 0; j < V::L; ++j) {
            load_l2(a, scratch + (S::AH + i * V::L + j) * N, lane);
            load_l2(r, scratch + (S::YH + j) * N, lane);
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
        store_l0(scratch + (S::W + i) * N, acc, lane);
        l0_to_seq(r, ws.buf, lane);
        pack_seq<V::W1BITS>(ws.hb + HB_W1 + i * V::POLYW1, r, 0, 1, lane);
    }
    __syncwarp();
    // c~ = H(mu || w1)  (l.9)
    {
        uint32_t lo = 0, hi = 0;
        absorb_smem(lo, hi, k, ws.hb + HB_MU, 64 + V::K * V::POLYW1, 136, lane);
        squeeze_words(lo, hi, ws.ctilde, 4, lane);
        __syncwarp();
    }
    // c = SampleInBall(c~); c^ = NTT(c)  (l.10)
    sample_in_ball<V::TAU>(ws.ctilde, ws.buf, ws.sq, k, lane);
    read_buf_l0(ch, ws.buf, lane);
    __syncwarp();
    ntt_fwd(ch, ws.buf, zt, lane);
    // z = y + INTT(c^ o s^1); reject if ||z|| >= gamma1 - beta  (l.11, l.14)
    for (int j = 0; j < V::L; ++j) {
        load_l2(a, scratch + (S::S1H + j) * N, lane);
#pragma unroll
        for (int m = 0; m < 8; ++m) r[m] = mont_mul(ch[m], a[m]);
        ntt_inv(r, ws.buf, izt, lane);
        load_l0(a, scratch + (S::Y + j) * N, lane);
        bool bad = false;
#pragma unroll
        for (int m = 0; m < 8; ++m) {
            r[m] = centre_small(to_canonical(r[m]) + a[m]);
            bad |= iabs(r[m]) >= V::GAMMA1 - V::BETA;
        }
        if (__any_sync(FULL, bad)) return false;
        store_l0(scratch + (S::Z + j) * N, r, lane);
    }
    // v_s = INTT(c^ o s^2); r0 = LowBits(w - v_s)  (l.12-14)
    for (int i = 0; i < V::K; ++i) {
        load_l2(a, scratch + (S::S2H + i) * N, lane);
#pragma unroll
        for (int m = 0; m < 8; ++m) r[m] = mont_mul(ch[m], a[m]);
        ntt_inv(r, ws.buf, izt, lane);
        load_l0(a, scratch + (S::W + i) * N, lane);
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
        if (__any_sync(FULL, bad)) return false;
        store_l0(scratch + (S::W + i) * N, a, lane);  // keep w - c s2 for the hint
    }
    // v_t = INTT(c^ o t^0); h = MakeHint(-v_t, w - v_s + v_t)  (l.17-19)
    int count = 0;
    for (int i = 0; i < V::K; ++i) {
        load_l2(a, scratch + (S::T0H + i) * N, lane);
#pragma unroll
        for (int m = 0; m < 8; ++m) r[m] = mont_mul(ch[m], a[m]);
        ntt_inv(r, ws.buf, izt, lane);
        load_l0(a, scratch + (S::W + i) * N, lane);
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
        if (__any_sync(FULL, bad)) return false;
#pragma unroll
        for (int m = 0; m < 8; ++m) {
            uint32_t w = __ballot_sync(FULL, (hbits >> m) & 1u);
            if (lane == 0) ws.hmask[i * 8 + m] = w;
            count += __popc(w);
        }
        if (count > V::OMEGA) return false;
    }
    __syncwarp();
    return true;
}

// Writes sig = c~ || z (gamma1 - z in ZBITS bits) || h (indices, then counts).
template <int LEVEL>
__device__ void sign_pack(uint8_t *__restrict__ sig, const int32_t *__restrict__ scratch, const WarpSmem &ws,
                          int lane) {
    using V = Lv<LEVEL>;
    using S = Scratch<LEVEL>;
    sig[lane] = ws.ctilde[lane];
    for (int j = 0; j < V::L; ++j) {
        int32_t v[8];
        load_l2(v, scratch + (S::Z + j) * N, lane);   // 8 consecutive coefficients
        pack_seq<V::ZBITS>(sig + V::SIG_Z + j * V::POLYZ, v, V::GAMMA1, -1, lane);
    }
    uint8_t *h = sig + V::SIG_H;
    int base = 0;
    for (int i = 0; i < V::K; ++i) {
#pragma unroll
        for (int m = 0; m < 8; ++m) {
            uint32_t w = ws.hmask[i * 8 + m];
            if ((w >> lane) & 1u) h[base + __popc(w & lanemask_lt(lane))] = (uint8_t)(lane + 32 * m);
            base += __popc(w);
        }
        if (lane == 0) h[V::OMEGA + i] = (uint8_t)base;
    }
    for (int p = base + lane; p < V::OMEGA; p += 32) h[p] = 0;
}

template <int LEVEL>
__device__ void sign_zero(uint8_t *__restrict__ sig, int lane) {
    for (int p = lane; p < Lv<LEVEL>::SIG; p += 32) sig[p] = 0;
}

// -------------------------------------------------------------------------
// Alg 3: Verify.  Returns 1 (accept) or 0.  scratch: VERIFY_POLYS polys.
// -------------------------------------------------------------------------
template <int LEVEL>
__device__ int verify_task(const uint8_t *__restrict__ pk, const uint8_t *__restrict__ msg, size_t mlen,
                           const uint8_t *__restrict__ sig, int32_t *__restrict__ scratch, WarpSmem &ws,
                           const int32_t *zt, const int32_t *izt, const KLane &k, int lane) {
    using V = Lv<LEVEL>;
    int32_t r[8], a[8], acc[8], ch[8];
    // c~ and rho
    ws.ctilde[lane] = __ldg(sig + lane);
    ws.rho[lane] = __ldg(pk + lane);
    // strict hint decoding into bit masks
    stage_bytes(ws.sq, sig + V::SIG_H, V::OMEGA + V::K, lane);
    ws.hmask[lane] = 0;
    ws.hmask[32 + lane] = 0;
    __syncwarp();
    bool bad = false;
    {
        int prev = 0;
        for (int i = 0; i < V::K; ++i) {
            int end = ws.sq[V::OMEGA + i];
            if (end < prev || end > V::OMEGA) {
                bad = true;
                break;
            }
            for (int j = prev + lane; j < end; j += 32) {
                int idx = ws.sq[j];
                if (j > prev && idx <= ws.sq[j - 1]) bad = true;
                atomicOr(&ws.hmask[i * 8 + (idx >> 5)], 1u << (idx & 31));
            }
            prev = end;
        }
        if (!bad)
            for (int j = prev + lane; j < V::OMEGA; j += 32)
                if (ws.sq[j]) bad = true;
    }
    bad = __any_sync(FULL, bad);
    __syncwarp();
    if (bad) return 0;
    // z: unpack, ||z|| < gamma1 - beta, z^ = NTT(z)  (Alg 3 l.6 first term, l.4)
    for (int j = 0; j < V::L; ++j) {
        unpack_poly_l0<V::ZBITS>(r, sig + V::SIG_Z + j * V::POLYZ, V::GAMMA1, ws, lane);
        bool b = false;
#pragma unroll
        for (int m = 0; m < 8; ++m) b |= iabs(r[m]) >= V::GAMMA1 - V::BETA;
        if (__any_sync(FULL, b)) return 0;
        ntt_fwd(r, ws.buf, zt, lane);
        store_l2(scratch + j * N, r, lane);
    }
    // mu = H(H(rho || t1) || M)  (l.2)
    uint32_t lo = 0, hi = 0;
    absorb_concat(lo, hi, k, ws.tr, 0, pk, V::PK, 136, lane);
    squeeze_words(lo, hi, ws.tr, 4, lane);
    __syncwarp();
    lo = 0;
    hi = 0;
    absorb_concat(lo, hi, k, ws.tr, 32, msg, mlen, 136, lane);
    squeeze_words(lo, hi, ws.hb + HB_MU, 8, lane);
    __syncwarp();
    // c^ = NTT(SampleInBall(c~))  (l.3)
    sample_in_ball<V::TAU>(ws.ctilde, ws.buf, ws.sq, k, lane);
    read_buf_l0(ch, ws.buf, lane);
    __syncwarp();
    ntt_fwd(ch, ws.buf, zt, lane);
    // v = INTT(A^ o z^ - c^ o NTT(t1 2^d)); w1' = UseHint(h, v)  (l.4-5)
    for (int i = 0; i < V::K; ++i) {
#pragma unroll
        for (int m = 0; m < 8; ++m) acc[m] = 0;
        for (int j = 0; j < V::L; ++j) {
            expand_a_poly(ws.rho, i, j, ws.buf, ws.sq, k, lane);
            read_buf_l2(a, ws.buf, lane);
            __syncwarp();
            load_l2(r, scratch + j * N, lane);
#pragma unroll
            for (int m = 0; m < 8; ++m) acc[m] += mont_mul(a[m], r[m]);
        }
        unpack_poly_l0<10>(r, pk + 32 + i * V::POLYT1, 0, ws, lane);
#pragma unroll
        for (int m = 0; m < 8; ++m) r[m] = (-r[m]) << D;   // t1 2^d, t1 stored as 0 - field
        ntt_fwd(r, ws.buf, zt, lane);
#pragma unroll
        for (int m = 0; m < 8; ++m) acc[m] = reduce_q(acc[m] - mont_mul(ch[m], r[m]));
        ntt_inv(acc, ws.buf, izt, lane);
#pragma unroll
        for (int m = 0; m < 8; ++m) {
            int hbit = (ws.hmask[i * 8 + m] >> lane) & 1u;
            r[m] = use_hint<LEVEL>(hbit, to_canonical(acc[m]));
        }
        l0_to_seq(r, ws.buf, lane);
        pack_seq<V::W1BITS>(ws.hb + HB_W1 + i * V::POLYW1, r, 0, 1, lane);
    }
    __syncwarp();
    // c~ == H(mu || w1')  (l.6)
    lo = 0;
    hi = 0;
    absorb_smem(lo, hi, k, ws.hb + HB_MU, 64 + V::K * V::POLYW1, 136, lane);
    bool eq = true;
    if (lane < 4) {
        uint2 w = *reinterpret_cast<const uint2 *>(ws.ctilde + 8 * lane);
        eq = (w.x == lo) && (w.y == hi);
    }
    return __all_sync(FULL, eq) ? 1 : 0;
}

}  // namespace dil

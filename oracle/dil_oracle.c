/*
 * dil_oracle.c -- plain CPU oracle for batched CRYSTALS-Dilithium (round 3).
 *
 * TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's
 * CPU-baseline leg are the only users.  Nothing on the product path links,
 * loads or calls this file.  It shares no code with the CUDA path.
 *
 * What it computes: Alg 1 (Gen), Alg 2 (deterministic Sign) and Alg 3 (Verify)
 * of arXiv 2211.12265 literally, with the parameters of Table 1.  Arithmetic
 * is exact: int64 products reduced with `%`.  Where the paper is silent the
 * Dilithium round-3 (v3.1) specification is read as follows ([spec]):
 *   - NTT root zeta = 1753, output j = f(zeta^(2*brv8(j)+1)) (bit-reversed).
 *   - ExpandA: SHAKE128(rho || j || i), 3-byte little-endian candidates with the
 *     top bit cleared, accepted iff < q, in stream order.
 *   - ExpandS: SHAKE256(rho' || nonce16), nibbles low first, eta=2: t<15 ->
 *     2-(t mod 5); eta=4: t<9 -> 4-t.  s1 nonces 0..l-1, s2 nonces l..l+k-1.
 *   - ExpandMask: SHAKE256(rho' || (kappa+i) as 16 bits), 18/20-bit fields t,
 *     coefficient gamma1 - t.
 *   - SampleInBall: SHAKE256(c~); 8 sign bytes, then position bytes b <= i.
 *   - Encodings: little-endian bit streams (t1 10 bits; t0 as 2^12 - t0 in 13;
 *     s as eta - s in 3 or 4; z as gamma1 - z in 18 or 20; w1 in 6 or 4);
 *     hints as omega index bytes then k cumulative counts, decoded strictly.
 *   - The 16-bit nonce caps the Sign loop (status ORC_EITER).
 * Parity of the byte encodings with the official scheme is unpinned (no test
 * vectors are available); every other function is pinned by the CPU tests.
 */
#include "dil_oracle.h"

#include <pthread.h>
#include <stdlib.h>
#include <string.h>

#define N 256
#define Q 8380417
#define D 13
#define ZETA 1753

typedef struct {
    int k, l, eta, tau, beta, omega;
    int32_t gamma1, gamma2;
    int z_bits, w1_bits, eta_bits;
    size_t pk_bytes, sk_bytes, sig_bytes;
} params;

/* Table 1 (Parameter specifications of Dilithium for three NIST levels). */
static int get_params(int level, params *p)
{
    memset(p, 0, sizeof(*p));
    if (level == 2) {
        p->k = 4; p->l = 4; p->eta = 2; p->tau = 39; p->beta = 78; p->omega = 80;
        p->gamma1 = 1 << 17; p->gamma2 = 95232;
    } else if (level == 3) {
        p->k = 6; p->l = 5; p->eta = 4; p->tau = 49; p->beta = 196; p->omega = 55;
        p->gamma1 = 1 << 19; p->gamma2 = 261888;
    } else if (level == 5) {
        p->k = 8; p->l = 7; p->eta = 2; p->tau = 60; p->beta = 120; p->omega = 75;
        p->gamma1 = 1 << 19; p->gamma2 = 261888;
    } else {
        return ORC_EINVAL;
    }
    p->z_bits = (p->gamma1 == (1 << 17)) ? 18 : 20;
    p->w1_bits = (p->gamma2 == (Q - 1) / 88) ? 6 : 4;
    p->eta_bits = (p->eta == 2) ? 3 : 4;
    p->pk_bytes = 32 + (size_t)p->k * (N * 10 / 8);
    p->sk_bytes = 96 + (size_t)(p->k + p->l) * (N * p->eta_bits / 8) + (size_t)p->k * (N * D / 8);
    p->sig_bytes = 32 + (size_t)p->l * (N * p->z_bits / 8) + p->omega + p->k;
    return ORC_OK;
}

int orc_sizes(int level, size_t *pk, size_t *sk, size_t *sig)
{
    params p;
    if (get_params(level, &p)) return ORC_EINVAL;
    if (pk) *pk = p.pk_bytes;
    if (sk) *sk = p.sk_bytes;
    if (sig) *sig = p.sig_bytes;
    return ORC_OK;
}

int orc_params(int level, int64_t out[10])
{
    params p;
    if (get_params(level, &p)) return ORC_EINVAL;
    out[0] = p.k; out[1] = p.l; out[2] = p.eta; out[3] = p.tau; out[4] = p.beta;
    out[5] = p.omega; out[6] = p.gamma1; out[7] = p.gamma2; out[8] = D; out[9] = Q;
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Work counters                                                            */
/* ------------------------------------------------------------------------ */
static uint64_t g_cnt[6];
static __thread uint64_t t_cnt[6];

static void flush_counters(void)
{
    for (int i = 0; i < 6; i++) {
        __atomic_fetch_add(&g_cnt[i], t_cnt[i], __ATOMIC_RELAXED);
        t_cnt[i] = 0;
    }
}

void orc_counters_reset(void)
{
    for (int i = 0; i < 6; i++) __atomic_store_n(&g_cnt[i], 0, __ATOMIC_RELAXED);
    for (int i = 0; i < 6; i++) t_cnt[i] = 0;
}

void orc_counters_get(uint64_t out[6])
{
    flush_counters();
    for (int i = 0; i < 6; i++) out[i] = __atomic_load_n(&g_cnt[i], __ATOMIC_RELAXED);
}

/* ------------------------------------------------------------------------ */
/* Keccak-f[1600] and the sponge (FIPS 202; section 2.3 "Sampling")         */
/* ------------------------------------------------------------------------ */
static uint64_t rotl64(uint64_t x, unsigned r)
{
    r &= 63;
    return r ? (x << r) | (x >> (64 - r)) : x;
}

/* FIPS 202 Algorithm 5: the round-constant bit rc(t) from the LFSR
 * x^8 + x^6 + x^5 + x^4 + 1.  Bit i of R holds R[i]. */
static int rc_bit(int t)
{
    int tm = t % 255;
    if (tm == 0) return 1;
    unsigned R = 1;
    for (int i = 1; i <= tm; i++) {
        unsigned R9 = R << 1;
        unsigned b8 = (R9 >> 8) & 1u;
        R9 ^= b8 | (b8 << 4) | (b8 << 5) | (b8 << 6);
        R = R9 & 0xFFu;
    }
    return (int)(R & 1u);
}

static uint64_t g_rc[24];
static int g_rho[25];
static pthread_once_t g_keccak_once = PTHREAD_ONCE_INIT;

static void keccak_tables(void)
{
    /* iota: RC[2^j - 1] = rc(j + 7 ir)  (FIPS 202 Algorithm 6) */
    for (int ir = 0; ir < 24; ir++) {
        uint64_t rc = 0;
        for (int j = 0; j <= 6; j++)
            if (rc_bit(j + 7 * ir)) rc |= (uint64_t)1 << ((1 << j) - 1);
        g_rc[ir] = rc;
    }
    /* rho offsets (FIPS 202 Algorithm 2): (x,y) starts at (1,0); the offset
     * for step t is (t+1)(t+2)/2, then (x,y) <- (y, 2x+3y). */
    memset(g_rho, 0, sizeof(g_rho));
    int x = 1, y = 0;
    for (int t = 0; t < 24; t++) {
        g_rho[x + 5 * y] = ((t + 1) * (t + 2) / 2) % 64;
        int nx = y, ny = (2 * x + 3 * y) % 5;
        x = nx; y = ny;
    }
}

/* Lane (x, y) is st[x + 5y]. */
void orc_keccak_f1600(uint64_t st[25])
{
    pthread_once(&g_keccak_once, keccak_tables);
    for (int ir = 0; ir < 24; ir++) {
        uint64_t C[5], Dx[5], B[25];
        /* theta */
        for (int x = 0; x < 5; x++)
            C[x] = st[x] ^ st[x + 5] ^ st[x + 10] ^ st[x + 15] ^ st[x + 20];
        for (int x = 0; x < 5; x++)
            Dx[x] = C[(x + 4) % 5] ^ rotl64(C[(x + 1) % 5], 1);
        for (int x = 0; x < 5; x++)
            for (int y = 0; y < 5; y++) st[x + 5 * y] ^= Dx[x];
        /* rho */
        for (int i = 0; i < 25; i++) st[i] = rotl64(st[i], (unsigned)g_rho[i]);
        /* pi: A'[x,y] = A[(x + 3y) mod 5, x] */
        for (int x = 0; x < 5; x++)
            for (int y = 0; y < 5; y++) B[x + 5 * y] = st[((x + 3 * y) % 5) + 5 * x];
        /* chi */
        for (int x = 0; x < 5; x++)
            for (int y = 0; y < 5; y++)
                st[x + 5 * y] = B[x + 5 * y] ^ (~B[((x + 1) % 5) + 5 * y] & B[((x + 2) % 5) + 5 * y]);
        /* iota */
        st[0] ^= g_rc[ir];
    }
    t_cnt[0]++;
}

typedef struct {
    uint64_t st[25];
    unsigned rate;   /* bytes */
    unsigned pos;    /* absorb: bytes absorbed into the current block; squeeze: bytes consumed */
    int squeezing;
} sponge;

static void st_xor_byte(uint64_t st[25], unsigned i, uint8_t b)
{
    st[i / 8] ^= (uint64_t)b << (8 * (i % 8));
}

static uint8_t st_get_byte(const uint64_t st[25], unsigned i)
{
    return (uint8_t)(st[i / 8] >> (8 * (i % 8)));
}

static void sp_init(sponge *s, unsigned rate)
{
    memset(s, 0, sizeof(*s));
    s->rate = rate;
}

static void sp_absorb(sponge *s, const uint8_t *in, size_t len)
{
    for (size_t i = 0; i < len; i++) {
        st_xor_byte(s->st, s->pos, in[i]);
        if (++s->pos == s->rate) {
            orc_keccak_f1600(s->st);
            s->pos = 0;
        }
    }
}

/* SHAKE domain bits 1111 followed by pad10*1. */
static void sp_finalize(sponge *s)
{
    st_xor_byte(s->st, s->pos, 0x1F);
    st_xor_byte(s->st, s->rate - 1, 0x80);
    orc_keccak_f1600(s->st);
    s->pos = 0;
    s->squeezing = 1;
}

static void sp_squeeze(sponge *s, uint8_t *out, size_t len)
{
    for (size_t i = 0; i < len; i++) {
        if (s->pos == s->rate) {
            orc_keccak_f1600(s->st);
            s->pos = 0;
        }
        out[i] = st_get_byte(s->st, s->pos++);
    }
}

static uint8_t sp_next_byte(sponge *s)
{
    uint8_t b;
    sp_squeeze(s, &b, 1);
    return b;
}

static void shake(unsigned rate, const uint8_t *in, size_t inlen, uint8_t *out, size_t outlen)
{
    sponge s;
    sp_init(&s, rate);
    sp_absorb(&s, in, inlen);
    sp_finalize(&s);
    sp_squeeze(&s, out, outlen);
}

void orc_shake128(const uint8_t *in, size_t inlen, uint8_t *out, size_t outlen)
{
    shake(168, in, inlen, out, outlen);
}

void orc_shake256(const uint8_t *in, size_t inlen, uint8_t *out, size_t outlen)
{
    shake(136, in, inlen, out, outlen);
}

/* H = SHAKE256 over a concatenation of two byte strings. */
static void H2(const uint8_t *a, size_t alen, const uint8_t *b, size_t blen, uint8_t *out, size_t outlen)
{
    sponge s;
    sp_init(&s, 136);
    sp_absorb(&s, a, alen);
    sp_absorb(&s, b, blen);
    sp_finalize(&s);
    sp_squeeze(&s, out, outlen);
}

/* ------------------------------------------------------------------------ */
/* Ring arithmetic and the NTT (section 2.2)                                */
/* ------------------------------------------------------------------------ */
static int32_t modq(int64_t a)
{
    int64_t r = a % Q;
    if (r < 0) r += Q;
    return (int32_t)r;
}

/* centred representative in (-(q-1)/2, (q-1)/2] (notation, section 2.1) */
static int32_t centred(int64_t a)
{
    int32_t r = modq(a);
    if (r > (Q - 1) / 2) r -= Q;
    return r;
}

static int64_t powmod(int64_t b, int64_t e)
{
    int64_t r = 1;
    b = modq(b);
    if (e < 0) {
        /* q is prime: b^-1 = b^(q-2) */
        b = powmod(b, Q - 2);
        e = -e;
    }
    while (e) {
        if (e & 1) r = (r * b) % Q;
        b = (b * b) % Q;
        e >>= 1;
    }
    return r;
}

static unsigned brv8(unsigned j)
{
    unsigned r = 0;
    for (int b = 0; b < 8; b++)
        if (j & (1u << b)) r |= 1u << (7 - b);
    return r;
}

static int g_use_def = 0;
void orc_use_def_ntt(int on) { g_use_def = on; }

/* f^_j = sum_i f_i * zeta^((2 brv8(j) + 1) i) */
void orc_ntt_def(const int32_t in[256], int32_t out[256])
{
    int32_t tmp[N];
    for (unsigned j = 0; j < N; j++) {
        int64_t w = powmod(ZETA, 2 * (int64_t)brv8(j) + 1);
        int64_t p = 1, acc = 0;
        for (unsigned i = 0; i < N; i++) {
            acc = (acc + (int64_t)modq(in[i]) * p) % Q;
            p = (p * w) % Q;
        }
        tmp[j] = (int32_t)acc;
    }
    memcpy(out, tmp, sizeof(tmp));
    t_cnt[1] += 1024;
}

/* f_i = n^-1 * sum_j f^_j * zeta^(-(2 brv8(j) + 1) i) */
void orc_intt_def(const int32_t in[256], int32_t out[256])
{
    int32_t tmp[N];
    int64_t ninv = powmod(N, -1);
    for (unsigned i = 0; i < N; i++) {
        int64_t acc = 0;
        for (unsigned j = 0; j < N; j++) {
            int64_t e = -(int64_t)(2 * brv8(j) + 1) * (int64_t)i;
            acc = (acc + (int64_t)modq(in[j]) * powmod(ZETA, e % 512)) % Q;
        }
        tmp[i] = (int32_t)((acc * ninv) % Q);
    }
    memcpy(out, tmp, sizeof(tmp));
    t_cnt[1] += 1024;
}

/* Radix-2 Cooley-Tukey form: level with half-length len splits each block of
 * 2*len coefficients with the twiddle zeta^brv8(128/len + block). */
void orc_ntt_fast(const int32_t in[256], int32_t out[256])
{
    int64_t a[N];
    for (int i = 0; i < N; i++) a[i] = modq(in[i]);
    for (int len = 128; len >= 1; len >>= 1) {
        for (int start = 0, b = 0; start < N; start += 2 * len, b++) {
            int64_t z = powmod(ZETA, brv8((unsigned)(128 / len + b)));
            for (int j = start; j < start + len; j++) {
                int64_t t = (z * a[j + len]) % Q;
                a[j + len] = modq(a[j] - t);
                a[j] = modq(a[j] + t);
            }
        }
    }
    for (int i = 0; i < N; i++) out[i] = (int32_t)a[i];
    t_cnt[1] += 1024;
}

/* Exact inverse of orc_ntt_fast: stages in reverse order, each butterfly
 * (u, v) -> (u + v, (u - v) * zeta^-brv8(...)), then the factor 1/n. */
void orc_intt_fast(const int32_t in[256], int32_t out[256])
{
    int64_t a[N];
    for (int i = 0; i < N; i++) a[i] = modq(in[i]);
    for (int len = 1; len <= 128; len <<= 1) {
        for (int start = 0, b = 0; start < N; start += 2 * len, b++) {
            int64_t zi = powmod(ZETA, -(int64_t)brv8((unsigned)(128 / len + b)));
            for (int j = start; j < start + len; j++) {
                int64_t u = a[j], v = a[j + len];
                a[j] = modq(u + v);
                a[j + len] = modq((u - v) * zi);
            }
        }
    }
    int64_t ninv = powmod(N, -1);
    for (int i = 0; i < N; i++) out[i] = (int32_t)((a[i] * ninv) % Q);
    t_cnt[1] += 1024;
}

static void ntt(const int32_t *in, int32_t *out)
{
    if (g_use_def) orc_ntt_def(in, out); else orc_ntt_fast(in, out);
}

static void intt(const int32_t *in, int32_t *out)
{
    if (g_use_def) orc_intt_def(in, out); else orc_intt_fast(in, out);
}

void orc_poly_mul(const int32_t a[256], const int32_t b[256], int32_t c[256])
{
    int32_t ah[N], bh[N], ch[N];
    ntt(a, ah);
    ntt(b, bh);
    for (int i = 0; i < N; i++) ch[i] = modq((int64_t)ah[i] * bh[i]);
    t_cnt[2] += N;
    intt(ch, c);
}

/* acc += a o b (pointwise, mod q) */
static void pointwise_acc(int32_t *acc, const int32_t *a, const int32_t *b)
{
    for (int i = 0; i < N; i++) acc[i] = modq((int64_t)acc[i] + (int64_t)a[i] * b[i]);
    t_cnt[2] += N;
}

/* ------------------------------------------------------------------------ */
/* Samplers (section 2.3; used by Alg 1 and Alg 2)                          */
/* ------------------------------------------------------------------------ */
/* ExpandA: A^_ij from SHAKE128(rho || j || i); rejection sampling keeps
 * 23-bit candidates below q ("Sampling", section 2.3; Alg 4 compares with q). */
static void expand_a(const params *p, const uint8_t rho[32], int32_t *A)
{
    for (int i = 0; i < p->k; i++) {
        for (int j = 0; j < p->l; j++) {
            uint8_t seed[34];
            memcpy(seed, rho, 32);
            seed[32] = (uint8_t)j;
            seed[33] = (uint8_t)i;
            sponge s;
            sp_init(&s, 168);
            sp_absorb(&s, seed, 34);
            sp_finalize(&s);
            int32_t *a = A + ((size_t)i * p->l + j) * N;
            int ctr = 0;
            while (ctr < N) {
                uint8_t b[3];
                sp_squeeze(&s, b, 3);
                uint32_t t = (uint32_t)b[0] | ((uint32_t)b[1] << 8) | ((uint32_t)(b[2] & 0x7F) << 16);
                if (t < Q) a[ctr++] = (int32_t)t;
            }
            t_cnt[3] += N;
        }
    }
}

int orc_expand_a(int level, const uint8_t rho[32], int32_t *ahat)
{
    params p;
    if (get_params(level, &p)) return ORC_EINVAL;
    expand_a(&p, rho, ahat);
    flush_counters();
    return ORC_OK;
}

/* ExpandS: coefficients in [-eta, eta] by rejection on 4-bit candidates. */
static void sample_eta(const params *p, const uint8_t rhop[64], uint16_t nonce, int32_t *a)
{
    uint8_t seed[66];
    memcpy(seed, rhop, 64);
    seed[64] = (uint8_t)(nonce & 0xFF);
    seed[65] = (uint8_t)(nonce >> 8);
    sponge s;
    sp_init(&s, 136);
    sp_absorb(&s, seed, 66);
    sp_finalize(&s);
    int ctr = 0;
    while (ctr < N) {
        uint8_t b = sp_next_byte(&s);
        int cand[2] = {b & 0x0F, b >> 4};
        for (int h = 0; h < 2 && ctr < N; h++) {
            int t = cand[h];
            if (p->eta == 2 && t < 15) a[ctr++] = 2 - (t % 5);
            else if (p->eta == 4 && t < 9) a[ctr++] = 4 - t;
        }
    }
    t_cnt[3] += N;
}

static void expand_s(const params *p, const uint8_t rhop[64], int32_t *s1, int32_t *s2)
{
    for (int i = 0; i < p->l; i++) sample_eta(p, rhop, (uint16_t)i, s1 + (size_t)i * N);
    for (int i = 0; i < p->k; i++) sample_eta(p, rhop, (uint16_t)(p->l + i), s2 + (size_t)i * N);
}

int orc_expand_s(int level, const uint8_t rhop[64], int32_t *s1, int32_t *s2)
{
    params p;
    if (get_params(level, &p)) return ORC_EINVAL;
    expand_s(&p, rhop, s1, s2);
    flush_counters();
    return ORC_OK;
}

/* little-endian bit stream helpers */
void orc_pack_bits(size_t count, const uint32_t *vals, int bits, uint8_t *out)
{
    size_t nbytes = (count * (size_t)bits + 7) / 8;
    memset(out, 0, nbytes);
    for (size_t i = 0; i < count; i++)
        for (int b = 0; b < bits; b++)
            if ((vals[i] >> b) & 1u) {
                size_t pos = i * (size_t)bits + (size_t)b;
                out[pos / 8] |= (uint8_t)(1u << (pos % 8));
            }
}

void orc_unpack_bits(size_t count, const uint8_t *in, int bits, uint32_t *vals)
{
    for (size_t i = 0; i < count; i++) {
        uint32_t v = 0;
        for (int b = 0; b < bits; b++) {
            size_t pos = i * (size_t)bits + (size_t)b;
            if ((in[pos / 8] >> (pos % 8)) & 1u) v |= 1u << b;
        }
        vals[i] = v;
    }
}

/* ExpandMask: y_i from SHAKE256(rho' || (kappa + i)); coefficient gamma1 - t
 * for a z_bits-bit field t, so y lies in [-gamma1 + 1, gamma1] (section 2.3). */
static void expand_mask(const params *p, const uint8_t rhop[64], uint32_t kappa, int32_t *y)
{
    size_t nbytes = (size_t)N * p->z_bits / 8;
    uint8_t buf[N * 20 / 8];
    uint32_t f[N];
    for (int i = 0; i < p->l; i++) {
        uint16_t nonce = (uint16_t)(kappa + (uint32_t)i);
        uint8_t seed[66];
        memcpy(seed, rhop, 64);
        seed[64] = (uint8_t)(nonce & 0xFF);
        seed[65] = (uint8_t)(nonce >> 8);
        orc_shake256(seed, 66, buf, nbytes);
        orc_unpack_bits(N, buf, p->z_bits, f);
        for (int c = 0; c < N; c++) y[(size_t)i * N + c] = p->gamma1 - (int32_t)f[c];
        t_cnt[3] += N;
    }
}

int orc_expand_mask(int level, const uint8_t rhop[64], uint32_t kappa, int32_t *y)
{
    params p;
    if (get_params(level, &p)) return ORC_EINVAL;
    expand_mask(&p, rhop, kappa, y);
    flush_counters();
    return ORC_OK;
}

/* SampleInBall: tau positions chosen by comparing a random byte with the
 * loop index (section 2.3); signs from the first 8 bytes. */
static void sample_in_ball(const params *p, const uint8_t ctilde[32], int32_t c[256])
{
    sponge s;
    sp_init(&s, 136);
    sp_absorb(&s, ctilde, 32);
    sp_finalize(&s);
    uint8_t sb[8];
    sp_squeeze(&s, sb, 8);
    uint64_t signs = 0;
    for (int i = 0; i < 8; i++) signs |= (uint64_t)sb[i] << (8 * i);
    for (int i = 0; i < N; i++) c[i] = 0;
    for (int i = N - p->tau; i < N; i++) {
        int b;
        do {
            b = sp_next_byte(&s);
        } while (b > i);
        c[i] = c[b];
        c[b] = (signs & 1) ? -1 : 1;
        signs >>= 1;
    }
    t_cnt[3] += (uint64_t)p->tau;
}

int orc_sample_in_ball(int level, const uint8_t ctilde[32], int32_t c[256])
{
    params p;
    if (get_params(level, &p)) return ORC_EINVAL;
    sample_in_ball(&p, ctilde, c);
    flush_counters();
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Bits extraction and hints (section 2.3 "Bits Extraction and Hints")      */
/* ------------------------------------------------------------------------ */
/* Power2Round: a0 = a mod+- 2^d (range (-2^(d-1), 2^(d-1)]), a1 = (a - a0)/2^d,
 * applied to the representative of a in [0, q). */
static void power2round(int32_t a, int32_t *a1, int32_t *a0)
{
    int32_t r = modq(a);
    int32_t r0 = r % (1 << D);
    if (r0 > (1 << (D - 1))) r0 -= (1 << D);
    *a0 = r0;
    *a1 = (r - r0) >> D;
}

/* Decompose: r0 = (r mod+ q) mod+- alpha; if r - r0 = q - 1 the output is
 * (0, r0 - 1), otherwise ((r - r0)/alpha, r0).  HighBits = r1, LowBits = r0. */
static void decompose(int32_t alpha, int32_t r, int32_t *r1, int32_t *r0)
{
    int32_t rp = modq(r);
    int32_t a0 = rp % alpha;
    if (a0 > alpha / 2) a0 -= alpha;
    if (rp - a0 == Q - 1) {
        *r1 = 0;
        *r0 = a0 - 1;
    } else {
        *r1 = (rp - a0) / alpha;
        *r0 = a0;
    }
}

static int32_t highbits(int32_t alpha, int32_t r)
{
    int32_t r1, r0;
    decompose(alpha, r, &r1, &r0);
    return r1;
}

static int32_t lowbits(int32_t alpha, int32_t r)
{
    int32_t r1, r0;
    decompose(alpha, r, &r1, &r0);
    return r0;
}

/* MakeHint(z, r): [[HighBits(r) != HighBits(r + z)]]  (the printed "v1" is
 * read as the z1 it defines). */
static int make_hint(int32_t alpha, int32_t z, int32_t r)
{
    return highbits(alpha, r) != highbits(alpha, modq((int64_t)r + z));
}

/* UseHint(h, r): m = (q-1)/alpha; r1 if h = 0, else (r1 + 1) mod+ m when
 * r0 > 0 and (r1 - 1) mod+ m when r0 <= 0. */
static int32_t use_hint(int32_t alpha, int h, int32_t r)
{
    int32_t m = (Q - 1) / alpha;
    int32_t r1, r0;
    decompose(alpha, r, &r1, &r0);
    if (!h) return r1;
    if (r0 > 0) return (r1 + 1) % m;
    return ((r1 - 1) % m + m) % m;
}

void orc_power2round(size_t n, const int32_t *r, int32_t *r1, int32_t *r0)
{
    for (size_t i = 0; i < n; i++) power2round(r[i], &r1[i], &r0[i]);
}

int orc_decompose(int level, size_t n, const int32_t *r, int32_t *r1, int32_t *r0)
{
    params p;
    if (get_params(level, &p)) return ORC_EINVAL;
    for (size_t i = 0; i < n; i++) decompose(2 * p.gamma2, r[i], &r1[i], &r0[i]);
    return ORC_OK;
}

int orc_make_hint(int level, size_t n, const int32_t *z, const int32_t *r, uint8_t *h)
{
    params p;
    if (get_params(level, &p)) return ORC_EINVAL;
    for (size_t i = 0; i < n; i++) h[i] = (uint8_t)make_hint(2 * p.gamma2, z[i], r[i]);
    return ORC_OK;
}

int orc_use_hint(int level, size_t n, const uint8_t *h, const int32_t *r, int32_t *r1)
{
    params p;
    if (get_params(level, &p)) return ORC_EINVAL;
    for (size_t i = 0; i < n; i++) r1[i] = use_hint(2 * p.gamma2, h[i], r[i]);
    return ORC_OK;
}

/* infinity norm of the centred representatives (section 2.1) */
static int32_t norm_inf(const int32_t *a, size_t n)
{
    int32_t m = 0;
    for (size_t i = 0; i < n; i++) {
        int32_t c = centred(a[i]);
        if (c < 0) c = -c;
        if (c > m) m = c;
    }
    return m;
}

/* ------------------------------------------------------------------------ */
/* Encodings                                                                 */
/* ------------------------------------------------------------------------ */
static void pack_poly(const int32_t *a, int32_t offset, int sign, int bits, uint8_t *out)
{
    /* stores offset + sign * a_i as a bits-wide field */
    uint32_t v[N];
    for (int i = 0; i < N; i++) v[i] = (uint32_t)(offset + sign * a[i]);
    orc_pack_bits(N, v, bits, out);
    t_cnt[3] += N;
}

static void unpack_poly(const uint8_t *in, int32_t offset, int sign, int bits, int32_t *a)
{
    /* reads a bits-wide field f and returns sign * (offset - f) ... written as
     * a_i = offset - f for sign = -1 encodings (offset - a stored) */
    uint32_t v[N];
    orc_unpack_bits(N, in, bits, v);
    for (int i = 0; i < N; i++) a[i] = sign > 0 ? (int32_t)v[i] - offset : offset - (int32_t)v[i];
    t_cnt[3] += N;
}

typedef struct {
    uint8_t rho[32], key[32], tr[32];
    int32_t s1[7 * N], s2[8 * N], t0[8 * N];
} sk_fields;

static void unpack_sk(const params *p, const uint8_t *sk, sk_fields *f)
{
    size_t eb = (size_t)N * p->eta_bits / 8;
    memcpy(f->rho, sk, 32);
    memcpy(f->key, sk + 32, 32);
    memcpy(f->tr, sk + 64, 32);
    const uint8_t *q = sk + 96;
    for (int i = 0; i < p->l; i++, q += eb) unpack_poly(q, p->eta, -1, p->eta_bits, f->s1 + (size_t)i * N);
    for (int i = 0; i < p->k; i++, q += eb) unpack_poly(q, p->eta, -1, p->eta_bits, f->s2 + (size_t)i * N);
    for (int i = 0; i < p->k; i++, q += N * D / 8) unpack_poly(q, 1 << (D - 1), -1, D, f->t0 + (size_t)i * N);
}

/* hint encoding: indices of ones, then k cumulative counts */
static void pack_hint(const params *p, const uint8_t *h, uint8_t *out)
{
    memset(out, 0, (size_t)p->omega + p->k);
    int idx = 0;
    for (int i = 0; i < p->k; i++) {
        for (int j = 0; j < N; j++)
            if (h[(size_t)i * N + j]) out[idx++] = (uint8_t)j;
        out[p->omega + i] = (uint8_t)idx;
    }
}

/* strict decoding: returns 0 on malformed input */
static int unpack_hint(const params *p, const uint8_t *in, uint8_t *h)
{
    memset(h, 0, (size_t)p->k * N);
    int prev = 0;
    for (int i = 0; i < p->k; i++) {
        int end = in[p->omega + i];
        if (end < prev || end > p->omega) return 0;
        for (int j = prev; j < end; j++) {
            if (j > prev && in[j] <= in[j - 1]) return 0;
            h[(size_t)i * N + in[j]] = 1;
        }
        prev = end;
    }
    for (int j = prev; j < p->omega; j++)
        if (in[j]) return 0;
    return 1;
}

/* ------------------------------------------------------------------------ */
/* Alg 1: Gen                                                               */
/* ------------------------------------------------------------------------ */
static void keygen(const params *p, const uint8_t seed[32], uint8_t *pk, uint8_t *sk)
{
    uint8_t hb[128];
    orc_shake256(seed, 32, hb, 128);                 /* Alg 1: (rho, rho', K) = H(zeta) */
    const uint8_t *rho = hb, *rhop = hb + 32, *key = hb + 96;
    int32_t *A = malloc(sizeof(int32_t) * (size_t)p->k * p->l * N);
    int32_t s1[7 * N], s2[8 * N], s1h[7 * N], t[8 * N], t1[8 * N], t0[8 * N];
    expand_a(p, rho, A);                             /* A^ = ExpandA(rho) */
    expand_s(p, rhop, s1, s2);                       /* (s1, s2) = ExpandS(rho') */
    for (int j = 0; j < p->l; j++) ntt(s1 + j * N, s1h + j * N);
    for (int i = 0; i < p->k; i++) {                 /* t = INTT(A^ o NTT(s1)) + s2 */
        int32_t acc[N] = {0};
        for (int j = 0; j < p->l; j++) pointwise_acc(acc, A + ((size_t)i * p->l + j) * N, s1h + j * N);
        intt(acc, t + i * N);
        for (int c = 0; c < N; c++) t[i * N + c] = modq((int64_t)t[i * N + c] + s2[i * N + c]);
    }
    for (int c = 0; c < p->k * N; c++) power2round(t[c], &t1[c], &t0[c]);   /* (t1, t0) */
    memcpy(pk, rho, 32);                              /* pk = rho || t1 */
    for (int i = 0; i < p->k; i++) pack_poly(t1 + i * N, 0, 1, 10, pk + 32 + i * (N * 10 / 8));
    uint8_t tr[32];
    orc_shake256(pk, p->pk_bytes, tr, 32);           /* tr = H(pk) */
    size_t eb = (size_t)N * p->eta_bits / 8;
    memcpy(sk, rho, 32);
    memcpy(sk + 32, key, 32);
    memcpy(sk + 64, tr, 32);
    uint8_t *q = sk + 96;
    for (int i = 0; i < p->l; i++, q += eb) pack_poly(s1 + i * N, p->eta, -1, p->eta_bits, q);
    for (int i = 0; i < p->k; i++, q += eb) pack_poly(s2 + i * N, p->eta, -1, p->eta_bits, q);
    for (int i = 0; i < p->k; i++, q += N * D / 8) pack_poly(t0 + i * N, 1 << (D - 1), -1, D, q);
    free(A);
}

int orc_keygen(int level, const uint8_t seed[32], uint8_t *pk, uint8_t *sk)
{
    params p;
    if (get_params(level, &p)) return ORC_EINVAL;
    keygen(&p, seed, pk, sk);
    flush_counters();
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Alg 2: Sign (deterministic)                                              */
/* ------------------------------------------------------------------------ */
static int max_iter_for(const params *p)
{
    /* nonces kappa .. kappa + l - 1 must fit 16 bits, kappa = l * iteration */
    return (65536 - p->l) / p->l + 1;
}

static int sign(const params *p, const uint8_t *sk, const uint8_t *msg, size_t mlen,
                uint8_t *sig, int max_iter, int *iters_out)
{
    sk_fields *f = malloc(sizeof(sk_fields));
    int32_t *A = malloc(sizeof(int32_t) * (size_t)p->k * p->l * N);
    int32_t *buf = malloc(sizeof(int32_t) * N * 8 * 12);
    int32_t *s1h = buf, *s2h = s1h + 8 * N, *t0h = s2h + 8 * N, *y = t0h + 8 * N,
            *yh = y + 8 * N, *w = yh + 8 * N, *w1 = w + 8 * N, *z = w1 + 8 * N,
            *vs = z + 8 * N, *vt = vs + 8 * N, *r0 = vt + 8 * N, *tmp = r0 + 8 * N;
    uint8_t h[8 * N];
    uint8_t mu[64], rhop[64], ctilde[32];
    int cap = max_iter_for(p);
    if (max_iter <= 0 || max_iter > cap) max_iter = cap;

    unpack_sk(p, sk, f);
    H2(f->tr, 32, msg, mlen, mu, 64);                 /* Alg 2: mu = H(tr || M) */
    H2(f->key, 32, mu, 64, rhop, 64);                 /* rho' = H(K || mu) */
    expand_a(p, f->rho, A);                           /* A^ = ExpandA(rho) */
    for (int j = 0; j < p->l; j++) ntt(f->s1 + j * N, s1h + j * N);
    for (int i = 0; i < p->k; i++) ntt(f->s2 + i * N, s2h + i * N);
    for (int i = 0; i < p->k; i++) ntt(f->t0 + i * N, t0h + i * N);

    int status = ORC_EITER, it;
    uint32_t kappa = 0;
    for (it = 0; it < max_iter; it++, kappa += (uint32_t)p->l) {   /* rejection loop, kappa += l */
        t_cnt[4]++;
        expand_mask(p, rhop, kappa, y);               /* y = ExpandMask(rho', kappa) */
        for (int j = 0; j < p->l; j++) ntt(y + j * N, yh + j * N);
        for (int i = 0; i < p->k; i++) {
            int32_t acc[N] = {0};
            for (int j = 0; j < p->l; j++) pointwise_acc(acc, A + ((size_t)i * p->l + j) * N, yh + j * N);
            intt(acc, w + i * N);
        }
        for (int c = 0; c < p->k * N; c++) w1[c] = highbits(2 * p->gamma2, w[c]);   /* w1 = HighBits(w) */
        size_t w1b = (size_t)N * p->w1_bits / 8;
        uint8_t w1p[8 * N * 6 / 8];
        for (int i = 0; i < p->k; i++) pack_poly(w1 + i * N, 0, 1, p->w1_bits, w1p + i * w1b);
        H2(mu, 64, w1p, (size_t)p->k * w1b, ctilde, 32);   /* c~ = H(mu || w1) */
        int32_t c[N], ch[N];
        sample_in_ball(p, ctilde, c);                 /* c = SampleInBall(c~) */
        ntt(c, ch);
        for (int j = 0; j < p->l; j++) {              /* z = y + c s1 */
            for (int e = 0; e < N; e++) tmp[e] = modq((int64_t)ch[e] * s1h[j * N + e]);
            t_cnt[2] += N;
            intt(tmp, z + j * N);
            for (int e = 0; e < N; e++) z[j * N + e] = centred((int64_t)z[j * N + e] + y[j * N + e]);
        }
        for (int i = 0; i < p->k; i++) {              /* v_s = c s2 */
            for (int e = 0; e < N; e++) tmp[e] = modq((int64_t)ch[e] * s2h[i * N + e]);
            t_cnt[2] += N;
            intt(tmp, vs + i * N);
        }
        int r0_fail_lit = 0, r0_fail_alt = 0;         /* r0 = LowBits(w - v_s), as printed */
        for (int c2 = 0; c2 < p->k * N; c2++) {
            r0[c2] = lowbits(2 * p->gamma2, modq((int64_t)w[c2] - vs[c2]));
            int32_t lit = r0[c2] < 0 ? -r0[c2] : r0[c2];
            int32_t alt = lowbits(2 * p->gamma2, w[c2]) - centred(vs[c2]);
            if (alt < 0) alt = -alt;
            if (lit >= p->gamma2 - p->beta) r0_fail_lit = 1;
            if (alt >= p->gamma2 - p->beta) r0_fail_alt = 1;
        }
        if (r0_fail_lit != r0_fail_alt) t_cnt[5]++;
        int reject = norm_inf(z, (size_t)p->l * N) >= p->gamma1 - p->beta || r0_fail_lit;
        if (!reject) {
            for (int i = 0; i < p->k; i++) {          /* v_t = c t0 */
                for (int e = 0; e < N; e++) tmp[e] = modq((int64_t)ch[e] * t0h[i * N + e]);
                t_cnt[2] += N;
                intt(tmp, vt + i * N);
            }
            int count = 0;                            /* h = MakeHint(-v_t, w - v_s + v_t) */
            for (int c2 = 0; c2 < p->k * N; c2++) {
                int32_t rr = modq((int64_t)w[c2] - vs[c2] + vt[c2]);
                h[c2] = (uint8_t)make_hint(2 * p->gamma2, modq(-(int64_t)vt[c2]), rr);
                count += h[c2];
            }
            if (norm_inf(vt, (size_t)p->k * N) >= p->gamma2 || count > p->omega) reject = 1;
        }
        if (!reject) {
            size_t zb = (size_t)N * p->z_bits / 8;
            memcpy(sig, ctilde, 32);
            for (int j = 0; j < p->l; j++) pack_poly(z + j * N, p->gamma1, -1, p->z_bits, sig + 32 + j * zb);
            pack_hint(p, h, sig + 32 + p->l * zb);
            status = ORC_OK;
            it++;
            break;
        }
    }
    if (status != ORC_OK) memset(sig, 0, p->sig_bytes);
    if (iters_out) *iters_out = it;
    free(buf);
    free(A);
    free(f);
    return status;
}

int orc_sign(int level, const uint8_t *sk, const uint8_t *msg, size_t mlen,
             uint8_t *sig, int max_iter, int *iters)
{
    params p;
    if (get_params(level, &p)) return ORC_EINVAL;
    int r = sign(&p, sk, msg, mlen, sig, max_iter, iters);
    flush_counters();
    return r;
}

/* ------------------------------------------------------------------------ */
/* Alg 3: Verify                                                            */
/* ------------------------------------------------------------------------ */
static int verify(const params *p, const uint8_t *pk, const uint8_t *msg, size_t mlen, const uint8_t *sig)
{
    int32_t *A = malloc(sizeof(int32_t) * (size_t)p->k * p->l * N);
    int32_t t1[8 * N], z[7 * N], zh[7 * N], v[8 * N], w1[8 * N];
    uint8_t h[8 * N];
    size_t zb = (size_t)N * p->z_bits / 8;
    int ok = 1;

    for (int i = 0; i < p->k; i++) unpack_poly(pk + 32 + i * (N * 10 / 8), 0, 1, 10, t1 + i * N);
    for (int j = 0; j < p->l; j++) unpack_poly(sig + 32 + j * zb, p->gamma1, -1, p->z_bits, z + j * N);
    if (!unpack_hint(p, sig + 32 + p->l * zb, h)) ok = 0;
    if (ok && norm_inf(z, (size_t)p->l * N) >= p->gamma1 - p->beta) ok = 0;   /* Alg 3: z norm check */
    if (ok) {
        expand_a(p, pk, A);                           /* A^ = ExpandA(rho) */
        uint8_t tr[32], mu[64], c2[32];
        orc_shake256(pk, p->pk_bytes, tr, 32);
        H2(tr, 32, msg, mlen, mu, 64);                /* mu = H(H(pk) || M) */
        int32_t c[N], ch[N];
        sample_in_ball(p, sig, c);                    /* c = SampleInBall(c~) */
        ntt(c, ch);
        for (int j = 0; j < p->l; j++) ntt(z + j * N, zh + j * N);
        for (int i = 0; i < p->k; i++) {              /* v = A z - c t1 2^d */
            int32_t acc[N] = {0}, t1s[N], t1h[N];
            for (int j = 0; j < p->l; j++) pointwise_acc(acc, A + ((size_t)i * p->l + j) * N, zh + j * N);
            for (int e = 0; e < N; e++) t1s[e] = modq((int64_t)t1[i * N + e] << D);
            ntt(t1s, t1h);
            for (int e = 0; e < N; e++) acc[e] = modq((int64_t)acc[e] - (int64_t)ch[e] * t1h[e]);
            t_cnt[2] += N;
            intt(acc, v + i * N);
        }
        int count = 0;
        for (int e = 0; e < p->k * N; e++) {          /* w1' = UseHint(h, v) */
            w1[e] = use_hint(2 * p->gamma2, h[e], v[e]);
            count += h[e];
        }
        size_t w1b = (size_t)N * p->w1_bits / 8;
        uint8_t w1p[8 * N * 6 / 8];
        for (int i = 0; i < p->k; i++) pack_poly(w1 + i * N, 0, 1, p->w1_bits, w1p + i * w1b);
        H2(mu, 64, w1p, (size_t)p->k * w1b, c2, 32);
        if (memcmp(c2, sig, 32) != 0) ok = 0;          /* c~ == H(mu || w1') */
        if (count > p->omega) ok = 0;
    }
    free(A);
    return ok;
}

int orc_verify(int level, const uint8_t *pk, const uint8_t *msg, size_t mlen, const uint8_t *sig)
{
    params p;
    if (get_params(level, &p)) return 0;
    int r = verify(&p, pk, msg, mlen, sig);
    flush_counters();
    return r;
}

/* ------------------------------------------------------------------------ */
/* Batched forms (host threads over independent tasks)                      */
/* ------------------------------------------------------------------------ */
typedef struct {
    int op;
    params p;
    size_t n;
    const uint8_t *in1, *msg;
    const uint64_t *off;
    uint8_t *out1, *out2;
    int32_t *status, *iters;
    int max_iter;
    size_t next;   /* shared task cursor */
} batch_job;

static void *batch_worker(void *arg)
{
    batch_job *j = (batch_job *)arg;
    for (;;) {
        size_t i = __atomic_fetch_add(&j->next, 1, __ATOMIC_RELAXED);
        if (i >= j->n) break;
        if (j->op == 0) {
            keygen(&j->p, j->in1 + 32 * i, j->out1 + j->p.pk_bytes * i, j->out2 + j->p.sk_bytes * i);
        } else if (j->op == 1) {
            int it = 0;
            int st = sign(&j->p, j->in1 + j->p.sk_bytes * i, j->msg + j->off[i], (size_t)(j->off[i + 1] - j->off[i]),
                          j->out1 + j->p.sig_bytes * i, j->max_iter, &it);
            if (j->status) j->status[i] = st;
            if (j->iters) j->iters[i] = it;
        } else {
            j->out1[i] = (uint8_t)verify(&j->p, j->in1 + j->p.pk_bytes * i, j->msg + j->off[i],
                                         (size_t)(j->off[i + 1] - j->off[i]), j->out2 + j->p.sig_bytes * i);
        }
    }
    flush_counters();
    return NULL;
}

static int run_batch(batch_job *j, int nthreads)
{
    if (nthreads < 1) nthreads = 1;
    if ((size_t)nthreads > j->n) nthreads = j->n ? (int)j->n : 1;
    j->next = 0;
    pthread_t th[256];
    if (nthreads > 256) nthreads = 256;
    for (int t = 1; t < nthreads; t++) pthread_create(&th[t], NULL, batch_worker, j);
    batch_worker(j);
    for (int t = 1; t < nthreads; t++) pthread_join(th[t], NULL);
    return ORC_OK;
}

int orc_keygen_batch(int level, size_t n, const uint8_t *seeds, uint8_t *pk, uint8_t *sk, int nthreads)
{
    batch_job j;
    memset(&j, 0, sizeof(j));
    if (get_params(level, &j.p)) return ORC_EINVAL;
    j.op = 0; j.n = n; j.in1 = seeds; j.out1 = pk; j.out2 = sk;
    return run_batch(&j, nthreads);
}

int orc_sign_batch(int level, size_t n, const uint8_t *sk, const uint8_t *msg, const uint64_t *msg_off,
                   uint8_t *sig, int32_t *status, int32_t *iters, int max_iter, int nthreads)
{
    batch_job j;
    memset(&j, 0, sizeof(j));
    if (get_params(level, &j.p)) return ORC_EINVAL;
    j.op = 1; j.n = n; j.in1 = sk; j.msg = msg; j.off = msg_off; j.out1 = sig;
    j.status = status; j.iters = iters; j.max_iter = max_iter;
    return run_batch(&j, nthreads);
}

int orc_verify_batch(int level, size_t n, const uint8_t *pk, const uint8_t *msg, const uint64_t *msg_off,
                     const uint8_t *sig, uint8_t *ok, int nthreads)
{
    batch_job j;
    memset(&j, 0, sizeof(j));
    if (get_params(level, &j.p)) return ORC_EINVAL;
    j.op = 2; j.n = n; j.in1 = pk; j.msg = msg; j.off = msg_off; j.out1 = ok; j.out2 = (uint8_t *)sig;
    return run_batch(&j, nthreads);
}

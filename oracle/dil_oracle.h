/*
 * dil_oracle.h -- plain CPU oracle for batched CRYSTALS-Dilithium (round 3).
 *
 * TEST INFRASTRUCTURE ONLY.  This header and dil_oracle.c define the slow,
 * obviously-correct reference that the CUDA path is checked against.  Only the
 * test suite, the smoke check and the CPU-baseline leg of the benchmark may
 * load it.  It shares no code, header, table or constant with the CUDA path.
 *
 * All arithmetic is exact integer arithmetic (int64 with plain `%`); there is
 * no Montgomery or Barrett form here.  Every function cites the passage of the
 * paper (arXiv 2211.12265) it follows; "[spec]" marks a reading of the
 * Dilithium round-3 (v3.1) specification that the paper relies on but does not
 * print.
 */
#ifndef DIL_ORACLE_H
#define DIL_ORACLE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_OK 0
#define ORC_EINVAL (-1)
#define ORC_EITER (-5)

/* Table 1: sizes in bytes of pk, sk and signature for a level in {2,3,5}. */
int orc_sizes(int level, size_t *pk_bytes, size_t *sk_bytes, size_t *sig_bytes);
/* Table 1 parameters: out[0..9] = k, l, eta, tau, beta, omega, gamma1, gamma2, d, q */
int orc_params(int level, int64_t out[10]);

/* Section 2.3 "Sampling": SHAKE128/256 (FIPS 202 sponge over Keccak-f[1600]). */
void orc_keccak_f1600(uint64_t st[25]);
void orc_shake128(const uint8_t *in, size_t inlen, uint8_t *out, size_t outlen);
void orc_shake256(const uint8_t *in, size_t inlen, uint8_t *out, size_t outlen);

/* Section 2.2: negacyclic NTT / INTT, coefficients canonical in [0, q).
 * _def is the O(n^2) evaluation map, _fast the radix-2 butterfly form. */
void orc_ntt_def(const int32_t in[256], int32_t out[256]);
void orc_intt_def(const int32_t in[256], int32_t out[256]);
void orc_ntt_fast(const int32_t in[256], int32_t out[256]);
void orc_intt_fast(const int32_t in[256], int32_t out[256]);
/* product in R_q computed as INTT(NTT(a) o NTT(b)) (section 2.2) */
void orc_poly_mul(const int32_t a[256], const int32_t b[256], int32_t c[256]);
/* selects which NTT form the procedures use: 0 = fast (default), 1 = definition */
void orc_use_def_ntt(int on);

/* Samplers (section 2.3; Alg 1 and Alg 2). */
int orc_expand_a(int level, const uint8_t rho[32], int32_t *ahat /* k*l*256 */);
int orc_expand_s(int level, const uint8_t rhop[64], int32_t *s1 /* l*256 */, int32_t *s2 /* k*256 */);
int orc_expand_mask(int level, const uint8_t rhop[64], uint32_t kappa, int32_t *y /* l*256 */);
int orc_sample_in_ball(int level, const uint8_t ctilde[32], int32_t c[256]);

/* Bits extraction and hints (section 2.3), applied to n values. */
void orc_power2round(size_t n, const int32_t *r, int32_t *r1, int32_t *r0);
int orc_decompose(int level, size_t n, const int32_t *r, int32_t *r1, int32_t *r0);
int orc_make_hint(int level, size_t n, const int32_t *z, const int32_t *r, uint8_t *h);
int orc_use_hint(int level, size_t n, const uint8_t *h, const int32_t *r, int32_t *r1);

/* Little-endian bit streams: value i occupies bits [i*bits, (i+1)*bits). */
void orc_pack_bits(size_t count, const uint32_t *vals, int bits, uint8_t *out);
void orc_unpack_bits(size_t count, const uint8_t *in, int bits, uint32_t *vals);

/* Procedures: Alg 1 (Gen), Alg 2 (Sign), Alg 3 (Verify). */
int orc_keygen(int level, const uint8_t seed[32], uint8_t *pk, uint8_t *sk);
/* max_iter <= 0 selects the cap implied by the 16-bit nonce. *iters receives
 * the number of loop repetitions.  Returns ORC_EITER (and a zeroed signature)
 * when the cap is reached. */
int orc_sign(int level, const uint8_t *sk, const uint8_t *msg, size_t mlen,
             uint8_t *sig, int max_iter, int *iters);
/* 1 = accept, 0 = reject */
int orc_verify(int level, const uint8_t *pk, const uint8_t *msg, size_t mlen,
               const uint8_t *sig);

/* Batched forms over n tasks using up to nthreads host threads.  msg_off has
 * n+1 entries; task i's message is msg[msg_off[i] .. msg_off[i+1]). */
int orc_keygen_batch(int level, size_t n, const uint8_t *seeds, uint8_t *pk,
                     uint8_t *sk, int nthreads);
int orc_sign_batch(int level, size_t n, const uint8_t *sk, const uint8_t *msg,
                   const uint64_t *msg_off, uint8_t *sig, int32_t *status,
                   int32_t *iters, int max_iter, int nthreads);
int orc_verify_batch(int level, size_t n, const uint8_t *pk, const uint8_t *msg,
                     const uint64_t *msg_off, const uint8_t *sig, uint8_t *ok,
                     int nthreads);

/* Work counters (accumulated over all calls since the last reset):
 * out[0] Keccak-f permutations, out[1] NTT/INTT butterflies,
 * out[2] pointwise products, out[3] sampled or packed coefficients,
 * out[4] Sign loop repetitions, out[5] Sign iterations in which the two
 *        readings of the r0 check (LowBits(w - cs2) versus LowBits(w) - cs2)
 *        took different decisions. */
void orc_counters_reset(void);
void orc_counters_get(uint64_t out[6]);

#ifdef __cplusplus
}
#endif
#endif

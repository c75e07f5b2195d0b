/*
 * KeyGen, Sign and Verify of n tasks through the C ABI alone (dil.h and
 * libdil.so, host-buffer entry points; no CUDA or Python in this program).
 *
 *   c_abi_roundtrip LEVEL N IN OUT
 *
 * IN holds N 32-byte seeds followed by N 32-byte messages.  OUT receives pk,
 * sk, sig (N each), the N int32 statuses, the N accept bytes, and the N
 * accept bytes of the same signatures with one bit of z flipped.  Exit code:
 * 0 on success, 2 for bad arguments or files, 3 when dil_ctx_create fails
 * (no GPU), 4 when a later call fails.
 */
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "dil.h"

static int fail(const char *what, int rc, int code) {
    fprintf(stderr, "%s: %s (%d)\n", what, dil_status_string(rc), rc);
    return code;
}

int main(int argc, char **argv) {
    if (argc != 5) return 2;
    const int level = atoi(argv[1]);
    const size_t n = (size_t)strtoull(argv[2], NULL, 10);
    size_t pkb, skb, sigb;
    if (dil_sizes(level, &pkb, &skb, &sigb) != DIL_OK || n == 0) return 2;
    uint8_t *in = malloc(64 * n), *pk = malloc(pkb * n), *sk = malloc(skb * n), *sig = malloc(sigb * n);
    uint8_t *ok = malloc(n), *ok_bad = malloc(n);
    int32_t *status = malloc(4 * n);
    uint64_t *off = malloc(8 * (n + 1));
    if (!in || !pk || !sk || !sig || !ok || !ok_bad || !status || !off) return 2;
    FILE *f = fopen(argv[3], "rb");
    if (!f || fread(in, 1, 64 * n, f) != 64 * n) return 2;
    fclose(f);
    for (size_t i = 0; i <= n; ++i) off[i] = 32 * i;
    const uint8_t *seeds = in, *msg = in + 32 * n;

    dil_ctx *ctx = NULL;
    int rc = dil_ctx_create(0, 0, &ctx);
    if (rc != DIL_OK) return fail("dil_ctx_create", rc, 3);
    if ((rc = dil_keygen_host(ctx, level, n, seeds, pk, sk, NULL)) != DIL_OK) return fail("dil_keygen_host", rc, 4);
    if ((rc = dil_sign_host(ctx, level, n, sk, msg, off, sig, status, NULL)) != DIL_OK)
        return fail("dil_sign_host", rc, 4);
    if ((rc = dil_verify_host(ctx, level, n, pk, msg, off, sig, ok, NULL)) != DIL_OK)
        return fail("dil_verify_host", rc, 4);
    for (size_t i = 0; i < n; ++i) sig[i * sigb + 40] ^= 0x04;   /* a bit of z */
    if ((rc = dil_verify_host(ctx, level, n, pk, msg, off, sig, ok_bad, NULL)) != DIL_OK)
        return fail("dil_verify_host", rc, 4);
    for (size_t i = 0; i < n; ++i) sig[i * sigb + 40] ^= 0x04;
    dil_ctx_destroy(ctx);

    f = fopen(argv[4], "wb");
    if (!f) return 2;
    fwrite(pk, 1, pkb * n, f);
    fwrite(sk, 1, skb * n, f);
    fwrite(sig, 1, sigb * n, f);
    fwrite(status, 4, n, f);
    fwrite(ok, 1, n, f);
    fwrite(ok_bad, 1, n, f);
    fclose(f);
    return 0;
}

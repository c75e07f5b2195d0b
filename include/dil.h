/*
 * dil.h -- C ABI of the batched CRYSTALS-Dilithium (round 3) engine for one
 * NVIDIA GB300 (sm_103a).
 *
 * Operations follow arXiv 2211.12265 ("High-Throughput GPU Implementation of
 * Dilithium Post-Quantum Digital Signature"):
 *   Gen    -- Alg 1 (section 2.3), keys from a 32-byte seed zeta;
 *   Sign   -- Alg 2, deterministic (rho' = H(K || mu)), rejection loop;
 *   Verify -- Alg 3;
 * over batches of independent tasks (section 3.1 task-level batching), with
 * the parameters of Table 1 for levels 2, 3 and 5.  Byte layouts of keys and
 * signatures are the round-3 little-endian encodings:
 *   pk  = rho (32) || t1 (k x 320)                         1312 / 1952 / 2592 B
 *   sk  = rho || K || tr (3 x 32) || s1 || s2 || t0        2528 / 4000 / 4864 B
 *   sig = c~ (32) || z (l x 576|640) || h (omega + k)      2420 / 3293 / 4595 B
 *
 * Conventions for every entry point unless stated otherwise:
 *   - Data pointers are DEVICE pointers owned by the caller; batched arrays are
 *     task-major and densely packed (task i's pk starts at pk + i * PK).
 *     Messages are one concatenated byte array `msg` with n + 1 byte offsets
 *     `msg_off` (task i's message is msg[msg_off[i] .. msg_off[i+1]) and may be
 *     empty; msg may be NULL when every message is empty).  Offsets must not
 *     decrease: a task whose offsets do (device arrays are not read on the
 *     host) is rejected by the kernels — Sign writes status DIL_EINVAL and a
 *     zeroed signature, Verify ok = 0 — and the host-buffer forms return
 *     DIL_EINVAL.  No alignment is required.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  Calls are
 *     asynchronous on that stream: the return value reports argument and
 *     launch errors only; per-task results are written to device memory.
 *   - The context owns a device workspace (the scratch the kernels need); the
 *     caller owns everything else.  Calls that share one context must not run
 *     concurrently on the GPU (use one context per concurrently used stream).
 *   - Return values are dil_status codes (0 = success).
 */
#ifndef DIL_H
#define DIL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    DIL_OK = 0,
    DIL_EINVAL = -1,   /* bad level, NULL pointer, size out of range */
    DIL_ENOMEM = -2,   /* workspace does not fit the budget or the device */
    DIL_ECUDA = -3,    /* a CUDA runtime call or kernel launch failed */
    DIL_ETIMEOUT = -4, /* a bounded device-side wait ran out (persistent kernels) */
    DIL_EITER = -5,    /* per task: the Sign loop hit its repetition cap */
    DIL_ECANCELED = -6 /* persistent Sign: the host canceled the launch */
} dil_status;

typedef struct dil_ctx dil_ctx;

/* Sizes in bytes of pk, sk and signature for level 2, 3 or 5 (Table 1 widths).
 * Any output pointer may be NULL.  Returns DIL_EINVAL for another level. */
int dil_sizes(int level, size_t *pk_bytes, size_t *sk_bytes, size_t *sig_bytes);

/* Human-readable name of a status code (static string). */
const char *dil_status_string(int status);

/* Creates a context bound to CUDA device `device`.  workspace_budget caps the
 * device scratch the context may allocate (0 = 8 GiB).  Batches that need more
 * scratch than the budget are processed in several launches on the stream. */
int dil_ctx_create(int device, size_t workspace_budget, dil_ctx **out);
/* Frees the workspace after synchronising the device.  NULL is accepted. */
int dil_ctx_destroy(dil_ctx *ctx);

/* Caps the number of Sign loop repetitions (Alg 2) for this context.
 * 0 restores the default cap implied by the 16-bit nonce (kappa + l - 1 <= 65535).
 * Tasks that reach the cap get DIL_EITER and an all-zero signature. */
int dil_set_max_iter(dil_ctx *ctx, int max_iter);

/* Launch shape of the plain (and keyed) kernels for op 0 = keygen, 1 = sign,
 * 2 = verify at `level` (0 = every level): warps per CTA (1..8) and warps per
 * task (1, 2 or 4, dividing warps_per_cta; 32 x warps_per_task threads
 * cooperate on one task, the paper's single-warp (1) and four-warp (4) forms).
 * Defaults: 8 warps per CTA, 2 warps per task.  The CTA shares the NTT
 * twiddle tables in shared memory. */
int dil_set_tuning(dil_ctx *ctx, int op, int level, int warps_per_cta, int warps_per_task);

/* Alg 1 (Gen): n 32-byte seeds -> n public keys and n secret keys. */
int dil_keygen(dil_ctx *ctx, int level, size_t n, const uint8_t *seeds, uint8_t *pk, uint8_t *sk,
               void *stream);

/* Alg 2 (Sign, deterministic): n secret keys and messages -> n signatures.
 * task_status (nullable, n int32): DIL_OK or DIL_EITER per task. */
int dil_sign(dil_ctx *ctx, int level, size_t n, const uint8_t *sk, const uint8_t *msg,
             const uint64_t *msg_off, uint8_t *sig, int32_t *task_status, void *stream);

/* As dil_sign, also writing the number of loop repetitions per task
 * (iterations: nullable, n int32). */
int dil_sign_ex(dil_ctx *ctx, int level, size_t n, const uint8_t *sk, const uint8_t *msg,
                const uint64_t *msg_off, uint8_t *sig, int32_t *task_status, int32_t *iterations,
                void *stream);

/* Alg 3 (Verify): ok[i] = 1 when signature i is valid for message i under
 * public key i, else 0.  A malformed signature is a reject, not an error. */
int dil_verify(dil_ctx *ctx, int level, size_t n, const uint8_t *pk, const uint8_t *msg,
               const uint64_t *msg_off, const uint8_t *sig, uint8_t *ok, void *stream);

/* ----------------------------------------------------------------------------
 * Caller-owned A^.  The matrix A^ = ExpandA(rho) (Alg 4; Alg 1 samples it in
 * the NTT domain, Alg 2 and Alg 3 use it) depends only on a key's rho, so a
 * caller that signs or verifies many batches under the same keys can expand
 * it once and pass it in.  Layout of one key's A^: k x l polynomials of 256
 * uint32 words, polynomial (i, j) at index i l + j, coefficient m at word m
 * (the NTT-domain evaluation order that ExpandA samples), each in [0, q).
 * A batch's A^ array holds task i's matrix at ahat + i k l 256 (device
 * memory, 16-byte aligned, owned by the caller).  See also the key store
 * below, which keeps the other per-key precomputation resident as well.
 * ------------------------------------------------------------------------- */

/* A^ = ExpandA(rho) for n keys: task i's 32-byte rho at rho + i rho_stride
 * (rho_stride >= 32; pass a public-key array with rho_stride = PK bytes, since
 * pk starts with rho) into ahat (n x k l x 256 uint32).  DIL_EINVAL for a bad
 * level, stride, NULL pointer or a misaligned ahat. */
int dil_expand_a(dil_ctx *ctx, int level, size_t n, const uint8_t *rho, size_t rho_stride, uint32_t *ahat,
                 void *stream);

/* dil_sign_ex with task i's A^ read from ahat instead of expanded from the rho
 * in its secret key; ahat NULL is dil_sign_ex.  The library does not check
 * that ahat matches the keys: an A^ of another rho gives signatures that do
 * not verify.  Runs one warp per task (warps per CTA from the Sign tuning). */
int dil_sign_a(dil_ctx *ctx, int level, size_t n, const uint8_t *sk, const uint8_t *msg,
               const uint64_t *msg_off, const uint32_t *ahat, uint8_t *sig, int32_t *task_status,
               int32_t *iterations, void *stream);

/* dil_verify with task i's A^ read from ahat (NULL: dil_verify).  t1 and
 * tr = H(pk) still come from pk, so a wrong A^ rejects. */
int dil_verify_a(dil_ctx *ctx, int level, size_t n, const uint8_t *pk, const uint8_t *msg,
                 const uint64_t *msg_off, const uint8_t *sig, const uint32_t *ahat, uint8_t *ok, void *stream);

/* Sign that allocates no memory (the paper has no counterpart).  For callers
 * that cannot call cudaMalloc while signing: a service whose device memory is
 * already owned by its own allocator, a latency-critical path that cannot
 * afford cudaMalloc/cudaFree (both may synchronise the device), or code that
 * must not fail with out-of-memory mid-request.  Same arguments and results as
 * dil_sign without a context; runs on the current device with the default
 * repetition cap and a fixed launch shape (4 warps per CTA, one warp per
 * task).  Scratch is a 64 MiB array inside the library's device image (held
 * by every GPU that loads the library until exit), so n may not exceed
 * 1110 / 789 / 532 tasks for levels 2 / 3 / 5: larger n returns DIL_EINVAL.
 * Set-up: the first call on a device looks up the array's address
 * (cudaGetSymbolAddress), loads the Sign kernels and runs each once on no
 * tasks, then synchronises `stream`; dil_sign_noalloc(level, 0, NULL, NULL,
 * NULL, NULL, NULL, stream) does only that.  Make that call before any stream
 * capture and before the first request that must not allocate.  The address
 * is cached per device: do not use this entry point on a device after
 * cudaDeviceReset.  All calls share the array: calls that overlap on the GPU
 * race and must be serialised.  Nothing in it needs clearing (each task's
 * scratch is written before it is read). */
int dil_sign_noalloc(int level, size_t n, const uint8_t *sk, const uint8_t *msg, const uint64_t *msg_off,
                     uint8_t *sig, int32_t *task_status, void *stream);

/* ----------------------------------------------------------------------------
 * Persistent Sign (section 4.3 dynamic task scheduling, on the device): one
 * launch runs every task of up to three jobs (levels may differ).  Resident
 * warp groups pull tasks from a device queue; once it is empty they evaluate
 * further nonces of unfinished tasks, and the signature of the smallest
 * accepting nonce is committed, so outputs equal dil_sign's byte for byte.
 * The launch (queue reset + kernel) is captured once into a CUDA graph per
 * distinct argument set and replayed on later identical calls.
 * ------------------------------------------------------------------------- */
typedef struct {
    int level;               /* 2, 3 or 5 */
    size_t n;                /* tasks in this job */
    const uint8_t *sk;       /* n x SK (device) */
    const uint8_t *msg;      /* concatenated messages (device, nullable if all empty) */
    const uint64_t *msg_off; /* n + 1 offsets (device) */
    uint8_t *sig;            /* n x SIG (device) */
    int32_t *task_status;    /* n (device, nullable): DIL_OK, DIL_EITER, DIL_EINVAL
                                (decreasing offsets), DIL_ECANCELED, or DIL_ETIMEOUT
                                when a bounded device wait on this task ran out
                                (then the signature is zeroed and iterations 0) */
    int32_t *iterations;     /* n (device, nullable): loop repetitions */
} dil_sign_job;

/* Enqueues one persistent Sign launch on `stream` for njobs (1..3) jobs.  The
 * context's repetition cap (dil_set_max_iter) applies.  Uses the context's
 * workspace; calls on one context must not overlap on the GPU.  The launch is
 * asynchronous and reads the jobs' device buffers while it runs: they must
 * stay allocated until the stream has passed the launch (the descriptors are
 * copied, the buffers are not).  A CUDA graph of the launch is cached and
 * replayed while the jobs' pointers and sizes are unchanged. */
int dil_sign_persistent(dil_ctx *ctx, int njobs, const dil_sign_job *jobs, void *stream);

/* Persistent launch shape: warps per CTA (1..8), warps per task group (1, 2
 * or 4), CTAs per SM (0 = as many as fit), fresh tasks claimed per queue
 * access (>= 1), helper groups per unfinished task (0 disables speculation).
 * Defaults 8, 2, 0, 1, 4. */
int dil_set_persistent_tuning(dil_ctx *ctx, int warps_per_cta, int warps_per_task, int ctas_per_sm, int chunk,
                              int speculation);

/* Synchronises `stream` and returns DIL_OK, DIL_ETIMEOUT when a bounded
 * device-side wait of the last persistent launch on this context ran out (the
 * tasks it concerned report DIL_ETIMEOUT; every other task's output is
 * normal), or DIL_ECANCELED when that launch was canceled. */
int dil_persistent_status(dil_ctx *ctx, void *stream);

/* Cancels the persistent launch of this context that is running: sets its
 * queue's cancel word through a copy on a stream of its own (the launch keeps
 * the SMs, so no kernel is involved) and returns once the word is written.
 * The launch then claims no more repetitions: tasks that already hold an
 * accepting repetition finish as DIL_OK with their normal signature, every
 * other task ends with status DIL_ECANCELED, 0 iterations and an all-zero
 * signature, and the grid exits.  A launch that has not started yet resets
 * the word when it starts, so the cancel applies to it only if it arrives
 * after that; a cancel after the launch has finished only changes what
 * dil_persistent_status reports for it.  The context stays usable.  Thread
 * safe with respect to the caller's stream (the call does not touch it). */
int dil_persistent_cancel(dil_ctx *ctx);

/* ----------------------------------------------------------------------------
 * Resident keys (for serving many messages per key): a key store keeps, per
 * key, pk, sk (optional), tr = H(pk) and the key's precomputation (A^ =
 * ExpandA(rho), NTT(s1), NTT(s2), NTT(t0), NTT(t1 2^d)) on the device, so a
 * keyed Sign hashes only mu and rho' per message before its loop (Alg 2)
 * and a keyed Verify skips ExpandA and H(pk) (Alg 3).  Outputs
 * equal dil_sign / dil_verify on the same keys and messages.
 * ------------------------------------------------------------------------- */
typedef struct dil_keystore dil_keystore;

/* Copies n_keys public keys (and secret keys, or NULL for a verify-only
 * store; device pointers) into a new store on ctx's device and enqueues their
 * precomputation on `stream`.  The store owns its device memory
 * (n_keys x (pk + sk + 32 + 4 KB (k l + l + 3k)) bytes). */
int dil_keystore_create(dil_ctx *ctx, int level, size_t n_keys, const uint8_t *pk, const uint8_t *sk,
                        dil_keystore **out, void *stream);
/* Frees the store (synchronises its device).  NULL is accepted. */
int dil_keystore_destroy(dil_keystore *ks);
/* Sign of n messages, task i with resident key key_idx[i] (device int32).
 * Needs a store created with secret keys.  A key index outside the store
 * gives task status DIL_EINVAL and a zero signature. */
int dil_sign_keyed(dil_ctx *ctx, const dil_keystore *ks, size_t n, const int32_t *key_idx, const uint8_t *msg,
                   const uint64_t *msg_off, uint8_t *sig, int32_t *task_status, void *stream);
/* Verify of n signatures against resident public keys key_idx[i]; a key index
 * outside the store gives ok = 0. */
int dil_verify_keyed(dil_ctx *ctx, const dil_keystore *ks, size_t n, const int32_t *key_idx, const uint8_t *msg,
                     const uint64_t *msg_off, const uint8_t *sig, uint8_t *ok, void *stream);

/* ----------------------------------------------------------------------------
 * Serving loop (continuous batching).  A server owns resident key stores (one
 * per level) and, from half of its memory budget each:
 *   - a device request ring with a message arena, served by a resident
 *     serving kernel (the default, continuous policy): a host thread copies
 *     arriving requests into the ring and publishes them; the kernel's
 *     one-warp workers take each request as soon as one is free (no batch
 *     boundaries on the device), idle workers help unfinished Signs with
 *     further nonces while few workers are busy (the smallest accepting one
 *     is committed), under load each SM serves one request type, and results
 *     are written to mapped host memory and handed back as they complete.
 *     The kernel exits after a few idle milliseconds and is relaunched when
 *     requests arrive;
 *   - S CUDA streams ("slots") with device and pinned host buffers for the
 *     static policy (dil_server_set_batching), where a batch of requests runs
 *     as keyed-kernel launches per operation and level.
 * Results equal dil_sign / dil_verify's.  Latency is measured from a
 * request's arrival to the moment its result is visible to the host.  All
 * pointers of the server calls are HOST pointers.
 * ------------------------------------------------------------------------- */
typedef struct dil_server dil_server;

typedef struct {
    uint64_t id;
    int32_t op;          /* 0 = sign, 1 = verify */
    int32_t level;
    int32_t status;      /* sign: DIL_OK, DIL_EITER or DIL_EINVAL (unknown key); any op:
                            DIL_ECUDA when the batch's copies or kernels failed,
                            DIL_ECANCELED when dil_server_cancel withdrew it */
    uint8_t ok;          /* verify: 1 = accept */
    uint8_t sig[4595];   /* sign: the signature (first SIG bytes) */
    double latency_s;    /* arrival to result visible on the host */
} dil_result;

/* Creates a server on `device` with `streams` slots (1..16).  memory_budget
 * (0 = 4 GiB, key stores excluded) is split in two: the slots' device buffers
 * must fit one half (max_batch is halved until they do; DIL_ENOMEM if even 1
 * does not fit), the request ring, arena and serving workers are sized to the
 * other (fewer workers when it is small).  Of that half the message arena
 * takes a quarter, at most 1 GiB, and the ring a slot per 2 KiB of arena, at
 * most 131072 slots.  The host side mirrors the ring in pinned memory: the
 * arena's size again, plus 4.7 KB of mapped result space per slot. */
int dil_server_create(int device, size_t memory_budget, int streams, int max_batch, dil_server **out);
/* Stops the dispatcher after in-flight work, frees everything.  NULL accepted. */
int dil_server_destroy(dil_server *srv);
/* The admission limits chosen at creation. */
int dil_server_limits(const dil_server *srv, int *max_batch, size_t *msg_capacity);
/* Batching policy.  By default (max_wait_s = 0) requests go to the device
 * ring and the serving kernel (continuous batching).  With max_wait_s > 0 a
 * slot starts only when at least min_batch requests are pending (capped by
 * the admission limit) or the oldest pending request has waited max_wait_s
 * seconds: static batching, the plain one-launch-per-batch service, kept for
 * comparison (switching to it stops an idle serving kernel first).
 * DIL_EINVAL for min_batch < 1 or a negative wait. */
int dil_server_set_batching(dil_server *srv, int min_batch, double max_wait_s);

/* Launch shape of the keyed kernels of static batches for one operation (0 =
 * Sign, 1 = Verify) and level: warps per CTA (1..8) and warps per task (1, 2,
 * 4, dividing the former).  Defaults: Sign 8 and 4, Verify 4 and 1.  Takes
 * effect for batches started afterwards (the serving kernel always runs one
 * warp per request).  DIL_EINVAL for other values. */
int dil_server_set_tuning(dil_server *srv, int op, int level, int warps_per_cta, int warps_per_task);

/* Installs n resident key pairs of one level (key ids 0..n-1), replacing the
 * level's previous store; only while no request is outstanding.  Synchronous. */
int dil_server_add_keys(dil_server *srv, int level, size_t n, const uint8_t *pk, const uint8_t *sk);
/* Queues one request (op 0 = sign with key `key`, 1 = verify of `sig` under
 * key `key`); the message (and signature) are copied.  *id identifies it. */
int dil_server_submit(dil_server *srv, int op, int level, int32_t key, const uint8_t *msg, size_t mlen,
                      const uint8_t *sig, uint64_t *id);
/* Withdraws submitted request `id` while it is still pending (not yet taken
 * into a batch): it completes at once with status DIL_ECANCELED (ok 0, no
 * signature) and is returned by dil_server_poll like any other.  DIL_EINVAL
 * when the id is unknown or the request was already dispatched (it then
 * completes normally). */
int dil_server_cancel(dil_server *srv, uint64_t id);
/* Returns up to max_n completed submitted requests (waiting up to wait_us for
 * the first one); *n_out receives the count. */
int dil_server_poll(dil_server *srv, dil_result *out, size_t max_n, size_t *n_out, int wait_us);
/* Open-loop load: request i arrives arrival_s[i] seconds after the call
 * starts (non-decreasing) and is submitted then; returns when all n are done.
 * Signatures in/out use a stride of 4595 bytes; msg/msg_off as for dil_sign.
 * latency_s[i] receives request i's latency, *wall_s the elapsed time. */
int dil_server_replay(dil_server *srv, size_t n, const double *arrival_s, const int32_t *op, const int32_t *level,
                      const int32_t *key, const uint8_t *msg, const uint64_t *msg_off, const uint8_t *sig_in,
                      uint8_t *sig_out, int32_t *status, uint8_t *ok, double *latency_s, double *wall_s);
/* Batches dispatched (static batches and ring publications), requests they
 * carried and kernel launches (keyed-kernel launches of static batches,
 * serving-kernel launches) since creation.  Any output pointer may be NULL. */
int dil_server_stats(const dil_server *srv, uint64_t *batches, uint64_t *requests, uint64_t *launches);
/* Test-only: the number of requests the serving kernel served with a mu =
 * H(tr || M) precomputed by its hasher warps (they hash while more than 2048
 * published requests wait for a worker), since the server was created.
 * Synchronous read of a device counter; DIL_EINVAL for NULL arguments. */
int dil_test_server_mu_hashed(const dil_server *srv, uint64_t *count);

/* Host-buffer forms of the three operations (all pointers are HOST pointers;
 * msg_off too; pinned memory lets the copies overlap).  They copy inputs to
 * the device, run, copy the results back and synchronise `stream` before
 * returning.  A batch of 2048 tasks or more is cut into four chunks, each on
 * its own stream (`stream` and three of the context's), so one chunk's copies
 * overlap the others' kernels (section 4.4 multi-stream overlap); the staging
 * buffers grow on demand and are not part of the workspace budget. */
int dil_keygen_host(dil_ctx *ctx, int level, size_t n, const uint8_t *seeds, uint8_t *pk, uint8_t *sk,
                    void *stream);
int dil_sign_host(dil_ctx *ctx, int level, size_t n, const uint8_t *sk, const uint8_t *msg,
                  const uint64_t *msg_off, uint8_t *sig, int32_t *task_status, void *stream);
int dil_verify_host(dil_ctx *ctx, int level, size_t n, const uint8_t *pk, const uint8_t *msg,
                    const uint64_t *msg_off, const uint8_t *sig, uint8_t *ok, void *stream);

/* ----------------------------------------------------------------------------
 * Test-only entry points: single primitives of the hot path, for component
 * parity against the oracle.  Same conventions (device pointers, async).
 * ------------------------------------------------------------------------- */

/* SHAKE128 (rate 168, kind = 128) or SHAKE256 (rate 136, kind = 256) of n byte
 * strings (in, in_off as for messages) -> outlen bytes each (out: n x outlen). */
int dil_test_shake(dil_ctx *ctx, int kind, size_t n, const uint8_t *in, const uint64_t *in_off,
                   uint8_t *out, size_t outlen, void *stream);
/* SHAKE256 (rate 136) of n byte strings (in, in_off as for messages) -> the
 * first 32 output bytes each (out: n x 32), computed the way Verify computes
 * tr = H(pk) for Dilithium3/5: the hash rides in the spare instance of
 * perms[i] sixteen-state permutations (one rate block absorbed before each)
 * and, if unfinished, completes on the 25-lane form.  perms: n int32
 * (device), any value >= 0; the result does not depend on it. */
int dil_test_k16_rider(dil_ctx *ctx, size_t n, const uint8_t *in, const uint64_t *in_off, const int32_t *perms,
                       uint8_t *out, void *stream);
/* As dil_test_k16_rider, for the hash KeyGen computes as tr = H(pk) while
 * the rows of t1 are still being packed (Dilithium3/5): before permutation p
 * only the first min(len, p * step[i]) bytes count as written (the hash
 * advances only on permutations whose next block is complete), and the
 * riding instance is overwritten between permutations, as the samplers'
 * shared memory is.  step: n int32 (device, negative counts as 0).  The
 * result depends on neither perms nor step. */
int dil_test_k16_chain_rider(dil_ctx *ctx, size_t n, const uint8_t *in, const uint64_t *in_off,
                             const int32_t *perms, const int32_t *step, uint8_t *out, void *stream);
/* Keccak-f[1600] (FIPS 202; section 3.3 of arXiv 2211.12265 for the warp
 * form) of n states, each 25 little-endian 64-bit lanes, lane x + 5y at
 * index x + 5y (in, out: n x 25 uint64, device).  form selects the
 * permutation code the kernels use: 1 = one state on 25 lanes, 2 = two
 * interleaved states, 6 = six states in the skewed row layout, 16 = sixteen
 * states on two threads each.  DIL_EINVAL for another form. */
int dil_test_keccak_f(dil_ctx *ctx, int form, size_t n, const uint64_t *in, uint64_t *out, void *stream);
/* t^0 = NTT(t0) of n secret keys (n x SK bytes) -> n x k x 256 int32 in
 * [0, q), index order: the paper's speedup breakdown of this step (section 5,
 * "Speedup Breakdown").  variant 0: an unpack kernel and a transform kernel
 * with t0 in global memory (the context workspace); 1: one fused kernel with
 * the same global round trip; 2: one kernel with t0 in registers and an
 * exchange layout with bank conflicts; 3: registers and the conflict-free
 * layout, the form Sign uses.  All variants give the same output.
 * DIL_EINVAL for another level or variant; DIL_ENOMEM when the workspace
 * (variants 0, 1) exceeds the budget. */
int dil_test_t0_ntt(dil_ctx *ctx, int level, int variant, size_t n, const uint8_t *sk, int32_t *t0hat,
                    void *stream);
/* Forward (inverse = 0) or inverse (inverse = 1) NTT of n polynomials of 256
 * int32 coefficients (any representatives with |a| < q); outputs in [0, q). */
int dil_test_ntt(dil_ctx *ctx, size_t n, const int32_t *in, int32_t *out, int inverse, void *stream);
/* ExpandA of n seeds rho (n x 32 bytes) -> n x k x l x 256 int32 in [0, q). */
int dil_test_expand_a(dil_ctx *ctx, int level, size_t n, const uint8_t *rho, int32_t *ahat, void *stream);
/* ExpandS of n seeds rho' (n x 64 bytes) -> n x (l + k) x 256 int32 (s1 then s2). */
int dil_test_expand_s(dil_ctx *ctx, int level, size_t n, const uint8_t *rhop, int32_t *s, void *stream);
/* ExpandMask of n (rho', kappa) pairs -> n x l x 256 int32. */
int dil_test_expand_mask(dil_ctx *ctx, int level, size_t n, const uint8_t *rhop, const int32_t *kappa,
                         int32_t *y, void *stream);
/* SampleInBall of n seeds c~ (n x 32 bytes) -> n x 256 int32 in {-1, 0, 1}. */
int dil_test_sample_in_ball(dil_ctx *ctx, int level, size_t n, const uint8_t *ctilde, int32_t *c,
                            void *stream);
/* SampleInBall's drawing and swapping over given bytes instead of
 * SHAKE256(c~): per task `blocks` (1..64) blocks of 136 bytes (n x blocks x
 * 136, device), the first starting with the 8 sign bytes; a task that needs
 * more blocks reuses the last one.  Output as dil_test_sample_in_ball. */
int dil_test_sample_in_ball_stream(dil_ctx *ctx, int level, size_t n, const uint8_t *bytes, int blocks, int32_t *cc,
                                   void *stream);
/* Coefficient functions of section 2.3 on n values r in [0, q) (and z, h):
 * out is n x 6 int32: Power2Round (r1, r0), Decompose (r1, r0),
 * MakeHint(z, r), UseHint(h, r). */
int dil_test_rounding(dil_ctx *ctx, int level, size_t n, const int32_t *r, const int32_t *z,
                      const uint8_t *h, int32_t *out, void *stream);

/* Failure-detection hook: the number of polls after which each bounded wait
 * of later persistent launches on this context (the commit lock, an owner
 * waiting for its helpers) gives up, 1..4194304; 0 restores the default
 * (4194304, about half a second).  A low limit makes the real waits run out
 * under ordinary contention, so tests can check the per-task DIL_ETIMEOUT
 * path.  DIL_EINVAL outside that range. */
int dil_test_set_spin_limit(dil_ctx *ctx, int limit);

/* Failure-detection hook: runs the persistent scheduler's bounded device wait
 * (poll until a flag reads 0, at most `limit` polls of ~128 ns) on a flag set
 * to flag_value, synchronously.  *result = DIL_OK when the flag was 0, else
 * DIL_ETIMEOUT; the context stays usable either way. */
int dil_test_bounded_wait(dil_ctx *ctx, int flag_value, int limit, int *result);

/* Sustained issue rate of one integer instruction class on the current GPU,
 * in thread-operations per SM clock (clock64 over independent dependency
 * chains at full occupancy; synchronous, allocates and frees its buffers).
 * op: 0 = LOP3, 1 = funnel shift, 2 = 32-bit multiply (low), 3 = multiply
 * (high, signed), 4 = warp shuffle.  Used for the integer roofline. */
int dil_test_issue_rate(dil_ctx *ctx, int op, double *thread_ops_per_sm_clk);

/* Test only (fusion ablation, section 4.2): Sign split into kernels instead
 * of one fused kernel per task — a precompute kernel, then per repetition
 * round one kernel for the first half (y, w, w1, c~ = H(mu || w1)) and one
 * for the second (c, z, r0, hint, packing), with the per-task state in global
 * memory and the host repeating rounds until no task is pending.  Same
 * arguments and outputs as dil_sign_ex (signatures, status, repetitions
 * equal the fused kernel's); `rounds` (nullable) returns the rounds run.
 * Synchronous.  Uses the Sign launch shape with at most 2 warps per task. */
int dil_test_sign_split(dil_ctx *ctx, int level, size_t n, const uint8_t *sk, const uint8_t *msg,
                        const uint64_t *msg_off, uint8_t *sig, int32_t *task_status, int32_t *iterations,
                        int *rounds, void *stream);

/* Test only: throughput of the Keccak-f[1600] forms the kernels use (section
 * 3.3 of arXiv 2211.12265 describes the first), in SM clocks per state per
 * round, 32 warps per SM, every state independent.  form: 1 = one state on 25
 * lanes, 2 = two interleaved states, 6 = six states in the skewed row layout,
 * 16 = sixteen states on two threads each.
 * Synchronous; allocates and frees a small buffer.  DIL_EINVAL for another
 * form or a NULL output. */
int dil_test_keccak_rate(dil_ctx *ctx, int form, double *sm_clocks_per_state_round);

#ifdef __cplusplus
}
#endif
#endif /* DIL_H */

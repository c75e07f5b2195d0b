// Internal launch interface between the C ABI (dil_abi.cu) and the kernel
// translation units.  Not part of the public ABI.
#pragma once
#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

// A resident key store (see dil_keystore_create): device copies of the keys,
// tr = H(pk) and each key's precomputation (KEY_POLYS polynomials).
struct dil_keystore {
    int device = 0;
    int level = 0;
    size_t n = 0;
    uint8_t *pk = nullptr, *sk = nullptr, *tr = nullptr;
    int32_t *keys = nullptr;
};

namespace dil {

enum Op { OP_KEYGEN = 0, OP_SIGN = 1, OP_VERIFY = 2 };

// Scratch polynomials (256 int32 each) one task of `op` needs in the plain form.
size_t scratch_polys(int op, int level);
// Dynamic shared memory of a CTA with `warps` warps.
size_t cta_smem_bytes(int warps, int warps_per_task);

// warps: warps per CTA; p: warps per task (1, 2 or 4; divides warps)
cudaError_t launch_keygen(int level, int n, const uint8_t *seeds, uint8_t *pk, uint8_t *sk, int32_t *scratch,
                          int warps, int p, cudaStream_t s);
cudaError_t launch_sign(int level, int n, const uint8_t *sk, const uint8_t *msg, const uint64_t *off,
                        uint8_t *sig, int32_t *status, int32_t *iters, int32_t *scratch, int max_iter,
                        int warps, int p, cudaStream_t s);
cudaError_t launch_verify(int level, int n, const uint8_t *pk, const uint8_t *msg, const uint64_t *off,
                          const uint8_t *sig, uint8_t *ok, int32_t *scratch, int warps, int p, cudaStream_t s);
// Loads the one-warp-per-task Sign kernel of `level` and runs it once on no
// tasks (its code and local-memory reservation are in place afterwards).
cudaError_t warm_sign(int level, int warps, int p, cudaStream_t s);

// Resident-A^ forms (one warp per task, `warps` warps per CTA): A^ of n keys
// from rho (task i's 32 bytes at rho + i rho_stride) into ahat (n x k l x 256
// words, 16-byte aligned); Sign and Verify with task i's A^ at
// ahat + i k l 256 instead of ExpandA.
cudaError_t launch_expand_a(int level, int n, const uint8_t *rho, size_t rho_stride, int32_t *ahat, int warps,
                            cudaStream_t s);
cudaError_t launch_sign_a(int level, int n, const uint8_t *sk, const uint8_t *msg, const uint64_t *off,
                          const int32_t *ahat, uint8_t *sig, int32_t *status, int32_t *iters, int32_t *scratch,
                          int max_iter, int warps, cudaStream_t s);
cudaError_t launch_verify_a(int level, int n, const uint8_t *pk, const uint8_t *msg, const uint64_t *off,
                            const uint8_t *sig, const int32_t *ahat, uint8_t *ok, int32_t *scratch, int warps,
                            cudaStream_t s);

// resident keys: per-key polynomials (A^, s^1, s^2, t^0, NTT(t1 2^d)) and
// per-task scratch of a keyed Sign (y, y^, w, z)
size_t key_polys(int level);
size_t keyed_sign_polys(int level);
size_t keyed_verify_polys(int level);
cudaError_t launch_key_prepare(int level, int n, const uint8_t *pk, const uint8_t *sk, int32_t *keys, uint8_t *tr,
                               int warps, int p, cudaStream_t s);
// key indices outside [0, n_keys) are rejected per task (status DIL_EINVAL / ok 0)
cudaError_t launch_sign_keyed(int level, int n, int n_keys, const int32_t *key_idx, const uint8_t *sk,
                              const int32_t *keys, const uint8_t *msg, const uint64_t *off, uint8_t *sig,
                              int32_t *status, int32_t *iters, int32_t *scratch, int max_iter, int warps, int p,
                              cudaStream_t s);
cudaError_t launch_verify_keyed(int level, int n, int n_keys, const int32_t *key_idx, const uint8_t *pk,
                                const int32_t *keys, const uint8_t *tr, const uint8_t *msg, const uint64_t *off,
                                const uint8_t *sig, uint8_t *ok, int32_t *scratch, int warps, int p, cudaStream_t s);

// primitives (test-only entry points)
cudaError_t launch_test_shake(int kind, int n, const uint8_t *in, const uint64_t *off, uint8_t *out,
                              int outlen, cudaStream_t s);
cudaError_t launch_test_ntt(int n, const int32_t *in, int32_t *out, int inverse, cudaStream_t s);
cudaError_t launch_test_keccak_f(int form, int states, const uint64_t *in, uint64_t *out, cudaStream_t s);
cudaError_t launch_test_k16_rider(int n, const uint8_t *in, const uint64_t *off, const int32_t *perms, uint8_t *out,
                                  cudaStream_t s);
cudaError_t launch_test_k16_chain_rider(int n, const uint8_t *in, const uint64_t *off, const int32_t *perms,
                                        const int32_t *step, uint8_t *out, cudaStream_t s);
// variant 0..3 of the t^0 = NTT(t0) breakdown; tmp: n k 256 int32 (variants 0, 1)
cudaError_t launch_test_t0_ntt(int level, int variant, int n, const uint8_t *sk, int32_t *tmp, int32_t *out,
                               cudaStream_t s);
cudaError_t launch_test_expand_a(int level, int n, const uint8_t *rho, int32_t *out, cudaStream_t s);
cudaError_t launch_test_expand_s(int level, int n, const uint8_t *rhop, int32_t *out, cudaStream_t s);
cudaError_t launch_test_expand_mask(int level, int n, const uint8_t *rhop, const int32_t *kappa, int32_t *out,
                                    cudaStream_t s);
cudaError_t launch_test_sample_in_ball(int level, int n, const uint8_t *ct, int32_t *out, cudaStream_t s);
cudaError_t launch_test_sib_stream(int level, int n, const uint8_t *stream, int blocks, int32_t *out,
                                   cudaStream_t s);
cudaError_t launch_test_rounding(int level, int n, const int32_t *r, const int32_t *z, const uint8_t *h,
                                 int32_t *out, cudaStream_t s);

// ---------------------------------------------------------------- persistent Sign
// One batch of Sign tasks of one level inside a persistent launch.
struct PersistJob {
    int level;
    int n;
    int start;   // first global task index of this job
    const uint8_t *sk;
    const uint8_t *msg;
    const uint64_t *off;
    uint8_t *sig;
    int32_t *status;
    int32_t *iters;
};
constexpr int PERSIST_MAX_JOBS = 3;
struct PersistJobs {
    PersistJob job[PERSIST_MAX_JOBS];
    int njobs;
    int total;
    // home job of each SM: SMs [sm_end[j - 1], sm_end[j]) take job j's fresh
    // tasks first (one level's task body per SM while the jobs last), then
    // the other jobs'; the host splits the SMs in proportion to each job's work
    int sm_end[PERSIST_MAX_JOBS];
};
// Per-task scheduling record (device memory, initialised by the task's owner).
struct PersistTask {
    int next_r;       // next repetition index to hand out (nonce kappa = l * r)
    int best_r;       // smallest accepting repetition seen (INT_MAX: none)
    int committed_r;  // repetition whose signature is in the output
    int lock;         // commit lock
    int helpers;      // helper groups reading this task's precomputation
    int fail;         // a bounded wait on this task ran out (zeroed before each launch)
    int pad[2];
};
// Queue header (device memory, zeroed before each launch).
struct PersistQueue {
    int next_task;    // unused since the per-job cursors
    int error;        // DIL_ETIMEOUT when a bounded wait ran out
    int cancel;       // set by the host (dil_persistent_cancel) while the launch runs
    int next_job[PERSIST_MAX_JOBS];   // per job: next fresh task (job-local index)
    int pad[26];
};
struct PersistTuning {
    int warps = 8;        // warps per CTA
    int p = 2;            // warps per task group
    int ctas_per_sm = 0;  // 0 = as many as fit
    int chunk = 1;        // fresh tasks claimed per queue access
    int spec = 4;         // helper groups per unfinished task (0 = no speculation)
};
// Device bytes a persistent launch needs for `total` tasks of the given levels.
size_t persist_workspace_bytes(const PersistJobs &J, const PersistTuning &t, int device);
// Polls of a bounded device wait before it gives up (the default of a launch).
constexpr int PERSIST_SPIN_LIMIT = 1 << 22;
// Enqueues (memsets, kernel, finalize kernel) on s; ws must hold
// persist_workspace_bytes.  spin_limit: polls per bounded wait (1..PERSIST_SPIN_LIMIT).
cudaError_t launch_sign_persist(const PersistJobs &J, void *ws, const PersistTuning &t, int max_iter_override,
                                int spin_limit, int device, cudaStream_t s);
// Reads the device error word of the last launch on ws (synchronous).
int persist_error(void *ws);
cudaError_t persist_cancel(void *ws, cudaStream_t s);
// Runs the scheduler's bounded wait on a flag holding flag_value (synchronous).
cudaError_t test_bounded_wait(int flag_value, int limit, int *result_host);

// ---------------------------------------------------------------- serving kernel
// One request of the continuous-batching server, in the device request ring
// (slot = ticket mod ring size), copied in by the host before it publishes
// the ticket.
struct __align__(16) ServeReq {
    int32_t op;      // 0 = Sign, 1 = Verify
    int32_t level;   // 2, 3 or 5
    int32_t key;     // resident key index of that level
    int32_t pad;
    uint64_t msg;    // byte offset of the message in the arena
    uint64_t mlen;
    uint64_t sig;    // byte offset of the signature to verify in the arena
    uint64_t pad2;   // 48 bytes: every slot 16-byte aligned
};
static_assert(sizeof(ServeReq) == 48, "ServeReq layout");
// Control words of the serving kernel (device memory, one cache line each).
struct ServeCtl {
    int tail;          // tickets published by the host (written by its copies)
    int pad0[31];
    int head;          // next ticket to claim
    int comp;          // completions issued (slots of the completion ring)
    int error;         // DIL_ETIMEOUT when a bounded wait ran out
    int active;        // workers serving a request of their own ticket
    int pad1[28];
    int stop;          // set by the host: workers exit once nothing is pending
    int pad2[31];
    int hhead;         // next ticket for the mu hashers
    int pad3[31];
    int mu_used;       // requests served with a hasher's mu (a test reads it)
    int pad4[31];
};
// Per-request record of a Sign (ring slot): the scheduling state shared by
// the owner and its helpers and the message's mu and rho'.  tref packs the
// ticket (high 32 bits) with the number of workers holding the record (low
// 32 bits): the one that drops it to zero completes the request.
struct __align__(16) ServeTask {
    unsigned long long tref;
    int next_r, best_r, committed_r, lock, fail, pad;
    uint8_t mu[64];
    uint8_t rhop[64];
};
// A level's resident keys as the serving kernel reads them.
struct ServeKeys {
    const uint8_t *sk, *pk, *tr;
    const int32_t *keys;
    int n;
};
constexpr int SERVE_SIG_STRIDE = 4608;   // bytes per result signature (16-byte multiple >= 4595)
// Request types (operation, level): 3 x op + level index (2, 3, 5 -> 0, 1, 2).
constexpr int SERVE_TYPES = 6;
constexpr int SERVE_MAX_SMS = 256;
constexpr uint8_t SERVE_TYPE_ANY = 255;   // an SM without a home type
// Forwarding queue of one request type: tickets claimed by workers of other
// types' SMs, for the workers of SMs whose home type it is.  Entry i of its
// ring holds (sequence << 32) | ticket; sequence p marks it free for the push
// at position p, p + 1 marks it filled by that push.
struct ServeFifo {
    unsigned head;
    unsigned pad0[31];
    unsigned tail;
    unsigned pad1[31];
};
struct ServeArgs {
    ServeCtl *ctl;
    const ServeReq *req;            // ring of R descriptors
    const uint8_t *arena;           // message / signature bytes
    ServeTask *tasks;               // ring of R records
    int *worker_ticket;             // per worker: the Sign ticket it owns (-1: none), for helpers
    int32_t *scratch;               // per worker: worker_polys polynomials
    uint8_t *sig_stage;             // per worker: SERVE_SIG_STRIDE bytes (device)
    int worker_polys;
    int ring;                       // R, a power of two
    ServeKeys keys[3];              // levels 2, 3, 5
    uint8_t *sig_out;               // R x SERVE_SIG_STRIDE (host-mapped)
    int32_t *status;                // R (host-mapped)
    int32_t *iters;                 // R (host-mapped)
    uint8_t *ok;                    // R (host-mapped)
    unsigned long long *comp;       // completion ring, R entries (host-mapped)
    int spec;                       // helpers per unfinished Sign (0: none)
    int help_below;                 // spec helpers while fewer than this many workers serve their own request, none above
    int forward_above;              // tickets are forwarded to their type's SMs from this many on
    ServeFifo *fifo;                // SERVE_TYPES forwarding queues
    unsigned long long *fifo_ring;  // SERVE_TYPES x R entries
    int type_sms[SERVE_TYPES];      // SMs whose home type it is (0: tickets of that type are not forwarded)
    int fifo_limit;                 // forward to a queue only while it holds fewer than this per home SM
    uint8_t sm_type[SERVE_MAX_SMS]; // home type of each SM (SERVE_TYPE_ANY: serves every type directly)
    int spin_limit;                 // polls of the commit lock
    long long idle_ns;              // an idle worker exits after this long
    // mu = H(tr || M) precomputed by hasher warps (optional: a worker whose
    // request has no mu yet hashes the message itself)
    uint8_t *mu_buf;                // R x 64 bytes
    unsigned long long *mu_tag;     // R: ticket + 1 of the mu in mu_buf, bit 32 while it is written
    int hash_sms;                   // SMs 0 .. hash_sms - 1 run only hasher warps
};
// Polynomials of one serving worker's scratch (the largest level's keyed
// Sign or keyed Verify scratch).
size_t serve_worker_polys();
// Resident workers of one serving launch (all SMs), capped by max_workers.
cudaError_t serve_grid(int device, int max_workers, int &grid, int &workers);
// Launches the serving kernel (grid from serve_grid) on s.
cudaError_t launch_serve(const ServeArgs &a, int grid, cudaStream_t s);

// test-only issue-rate probe (thread-ops per SM clock)
cudaError_t measure_issue_rate(int op, double *rate);
size_t split_state_bytes();
cudaError_t launch_sign_split(int level, int n, const uint8_t *sk, const uint8_t *msg, const uint64_t *off,
                              uint8_t *sig, int32_t *status, int32_t *iters, int32_t *scratch, void *state_mem,
                              int *pending, int max_iter, int warps, int p, cudaStream_t s, int *rounds);
cudaError_t measure_keccak_rate(int form, double *clk_per_state_round);

}  // namespace dil

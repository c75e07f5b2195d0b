// Serving kernel: continuous batching on the device.
//
// One-warp workers stay resident and take requests from a device ring as the
// host publishes them (the host copies a request's descriptor and bytes into
// the ring, then its ticket count into ServeCtl::tail).  A free worker takes
// the next ticket number with one atomicAdd on ServeCtl::head, published or
// not, and serves it once the host has published it, so each request starts
// as soon as its ticket is published (idle workers hold the next tickets) or
// a busy worker frees up: there are no batch boundaries on the device.  Keys are resident (key store: A^, s^1,
// s^2, t^0, NTT(t1 2^d), tr), so a Sign hashes only mu and rho' before its
// rejection loop (Alg 2) and a Verify skips ExpandA and H(pk) (Alg 3).
//
// A worker whose ticket is not yet published helps an unfinished Sign
// meanwhile (the dynamic scheduling of section 4.3, on the device), until its
// ticket is published, only while few workers serve requests of their own
// (under load the speculative repetitions would take issue slots from the
// requests on the same SMs): it joins the request's record,
// draws further repetition indices from the shared counter and evaluates
// those nonces; the signature of the smallest accepting nonce is committed
// under the record's lock, so results equal dil_sign's byte for byte.  The
// record counts the workers holding it (owner and helpers, packed with the
// ticket into one 64-bit word); the worker that drops the count to zero
// writes the request's final status and its completion.  Nobody waits for
// anybody: the only wait is the commit lock, bounded by spin_limit polls
// (then the request fails with DIL_ETIMEOUT and the error word is set).
//
// While requests queue, the warps of a few SMs precompute the requests' mu =
// H(tr || M) for sixteen messages at a time (the mu hashers below); a worker
// whose request already has its mu skips that hash.
//
// Results go straight to mapped host memory: the signature and status (or
// the accept byte), a system-scope fence, then the entry (completion number,
// ticket) in the completion ring that the host polls.  Requests are read
// through L2 only (their ring slots are rewritten while the kernel runs).
// Under load, every SM serves one request type (operation and level; the
// host assigns the SMs in proportion to the recent work of each type): the
// task bodies of different types thrash a shared instruction cache (a mix of
// the three Sign levels on one SM measured 1.6x the warp time of one level).
// A worker that claims a ticket of another type forwards it to that type's
// queue and takes the next number; workers serve their own type's queue
// before taking a number.  A ticket is served where it was claimed when its
// type has no home SMs or a long queue, and at light load.
//
// Workers exit when the host sets `stop` (the host stops an idle kernel)
// unless their ticket is published, then they serve it first; a worker whose
// ticket stays unpublished for idle_ns also exits and sets the error word.
// Tickets taken but never published are abandoned at exit: the host sets
// head back to its oldest uncompleted ticket before the next launch.
#include <climits>
#include <cstddef>

#include "../../include/dil.h"
#include "dil_kern.cuh"

namespace dil {

namespace {

constexpr int SERVE_WARPS = 8;                 // warps (workers) per CTA
constexpr unsigned NO_TICKET = 0xFFFFFFFFu;    // worker_ticket of a worker that owns no Sign
constexpr int SCAN_CHUNKS = 4;                 // 32-entry chunks of worker_ticket an idle worker scans per pass

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int ld_acquire(const int *p) { return (int)ld_acquire(reinterpret_cast<const unsigned *>(p)); }
__device__ __forceinline__ unsigned tail_of(const ServeArgs &a) {
    return ld_acquire(reinterpret_cast<const unsigned *>(&a.ctl->tail));
}

// Tags of precomputed mu (see the mu hashers below).
constexpr unsigned long long MU_WRITING = 1ull << 32, MU_VALID = 1ull << 33;
// Warps of the hashing SMs hash while more than HASH_ON published requests
// wait for a worker, and serve requests again below HASH_OFF.
constexpr int HASH_ON = 2048, HASH_OFF = 512;

__device__ __forceinline__ unsigned long long ld_acquire64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ long long global_ns() {
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Appends ticket t to the completion ring (one thread; the request's results
// are visible system-wide before this is called).
__device__ __forceinline__ void complete(const ServeArgs &a, unsigned t) {
    const unsigned c = atomicAdd(reinterpret_cast<unsigned *>(&a.ctl->comp), 1u);
    volatile unsigned long long *e = a.comp + (c & (unsigned)(a.ring - 1));
    *e = ((unsigned long long)c << 32) | t;
}

// Zeroes a result signature (the whole warp).
__device__ __forceinline__ void zero_sig(uint8_t *sig, int lane) {
    uint4 *q = reinterpret_cast<uint4 *>(sig);
    for (int i = lane; i < SERVE_SIG_STRIDE / 16; i += 32) q[i] = make_uint4(0, 0, 0, 0);
}

// Final result of a Sign request, written by the last worker to leave its
// record: status (and repetitions), a zeroed signature unless one was
// committed, then the completion.
template <int LEVEL>
__device__ void finish_sign(const ServeArgs &a, unsigned t, ServeTask &tk, int lane) {
    const int slot = (int)(t & (unsigned)(a.ring - 1));
    const int fail = atomicOr(&tk.fail, 0);
    const int committed = atomicOr(&tk.committed_r, 0);
    const int status = fail ? DIL_ETIMEOUT : committed != INT_MAX ? DIL_OK : DIL_EITER;
    if (status != DIL_OK) zero_sig(a.sig_out + (size_t)slot * SERVE_SIG_STRIDE, lane);
    if (lane == 0) {
        a.status[slot] = status;
        a.iters[slot] = status == DIL_OK ? committed + 1 : status == DIL_EITER ? Lv<LEVEL>::MAX_ITER : 0;
    }
    __threadfence_system();
    __syncwarp();
    if (lane == 0) complete(a, t);
}

// Drops this worker's hold on record tk (ticket t); the last one out finishes
// the request.
template <int LEVEL>
__device__ void leave(const ServeArgs &a, unsigned t, ServeTask &tk, int lane) {
    __threadfence();
    unsigned long long prev = 0;
    if (lane == 0) prev = atomicAdd(&tk.tref, ~0ull);   // minus one
    prev = __shfl_sync(FULL, prev, 0);
    if ((prev & 0xFFFFFFFFull) == 1) finish_sign<LEVEL>(a, t, tk, lane);
}

// Commits the signature of accepting repetition r if it beats the committed one.
// stage: the worker's SERVE_SIG_STRIDE-byte device buffer for the packed signature.
template <int LEVEL>
__device__ void commit(const ServeArgs &a, unsigned t, ServeTask &tk, int r, const int32_t *itr, GroupSmem &gs,
                       uint8_t *stage, int lane) {
    const int slot = (int)(t & (unsigned)(a.ring - 1));
    int st = 0;
    if (lane == 0) {
        atomicMin(&tk.best_r, r);
        int acquired = 0;
        for (int i = 0; i < a.spin_limit; ++i) {
            if (atomicCAS(&tk.lock, 0, 1) == 0) {
                acquired = 1;
                break;
            }
            __nanosleep(64);
        }
        if (!acquired) {
            atomicExch(&tk.fail, 1);
            atomicExch(&a.ctl->error, DIL_ETIMEOUT);
        }
        __threadfence();
        st = !acquired ? 0 : (r < atomicOr(&tk.committed_r, 0) && !atomicOr(&tk.fail, 0)) ? 2 : 1;
    }
    st = __shfl_sync(FULL, st, 0);
    if (st == 2) {   // pack in device memory, then 16-byte stores to the mapped result
        sign_pack<LEVEL, 1>(stage, itr, gs, 0, lane);
        __syncwarp();
        const uint4 *src = reinterpret_cast<const uint4 *>(stage);
        uint4 *dst = reinterpret_cast<uint4 *>(a.sig_out + (size_t)slot * SERVE_SIG_STRIDE);
        for (int i = lane; i < (Lv<LEVEL>::SIG + 15) / 16; i += 32) dst[i] = src[i];
    }
    __threadfence_system();
    __syncwarp();
    if (lane == 0 && st >= 1) {
        if (st == 2) atomicExch(&tk.committed_r, r);
        __threadfence();
        atomicExch(&tk.lock, 0);
    }
    __syncwarp();
}

// Draws repetitions of record tk until one accepts, the counter passes an
// accepted one, the cap is reached or the request failed.  pre: the key's
// precomputation; gs.hb (mu) and gs.rhop hold the message's hashes.  Two
// consecutive repetitions per claim, so one mask-stream batch serves both.
//
// watch: a helper stops drawing repetitions once its own ticket `mine` is
// published (it has a request to serve), but only between claims: a claimed
// repetition below the best accepted one is always evaluated, else a larger
// nonce than the smallest accepting one could be committed.
template <int LEVEL>
__device__ void repetitions(const ServeArgs &a, unsigned t, ServeTask &tk, const int32_t *pre, int32_t *itr,
                            uint8_t *stage, GroupSmem &gs, WarpSmem &ws, const int32_t *zt, const int32_t *izt,
                            int lane, bool watch = false, unsigned mine = 0) {
    constexpr int PER_BATCH = Scratch<LEVEL>::MASK_BATCH / Lv<LEVEL>::L;
    constexpr int CLAIM = PER_BATCH < 2 ? PER_BATCH : 2;
    MaskStream ms{0, 0};
    int next = 0, end = 0;
    for (;;) {
        int r = -1;
        if (lane == 0) {
            bool claim = true;
            if (next >= end) {
                if (watch && (int)(tail_of(a) - mine) > 0) {
                    claim = false;
                } else {
                    next = atomicAdd(&tk.next_r, CLAIM);
                    end = next + CLAIM;
                }
            }
            if (claim) {
                r = next++;
                const int best = atomicOr(&tk.best_r, 0);
                if (__ldcg(&tk.fail) || r >= Lv<LEVEL>::MAX_ITER || r >= best) r = -1;
            }
        }
        r = __shfl_sync(FULL, r, 0);
        if (r < 0) break;
        if (sign_attempt<LEVEL, 1>(Lv<LEVEL>::L * r, pre, itr, ms, gs, ws, zt, izt, 0, 0, lane, &tk.best_r, r)) {
            commit<LEVEL>(a, t, tk, r, itr, gs, stage, lane);
            break;
        }
    }
}

// The request of ticket t as its owner: Verify to completion, or Sign:
// prepare mu and rho', publish the record to helpers, repeat, leave.
template <int LEVEL>
__device__ void own(const ServeArgs &a, unsigned t, const ServeReq &rq, int worker, int32_t *mine, uint8_t *stage,
                    GroupSmem &gs, WarpSmem &ws, const int32_t *zt, const int32_t *izt, int lane) {
    using V = Lv<LEVEL>;
    using S = Scratch<LEVEL>;
    const int slot = (int)(t & (unsigned)(a.ring - 1));
    const ServeKeys &ks = a.keys[LEVEL == 2 ? 0 : LEVEL == 3 ? 1 : 2];
    const bool key_ok = rq.key >= 0 && rq.key < ks.n;
    const uint8_t *msg = a.arena + rq.msg;
    // a hasher's mu, when the slot's tag names this ticket
    int have_mu = 0;
    if (a.hash_sms > 0 && lane == 0) have_mu = ld_acquire64(a.mu_tag + slot) == (MU_VALID | (unsigned long long)(t + 1u));
    const uint8_t *mu_in = __shfl_sync(FULL, have_mu, 0) ? a.mu_buf + (size_t)slot * 64 : nullptr;
    __syncwarp();   // the lanes that read mu_in do so after lane 0's acquire
    if (mu_in && lane == 0) atomicAdd(&a.ctl->mu_used, 1);
    if (rq.op == 1) {   // Verify
        int r = 0;
        if (key_ok)
            r = verify_task<LEVEL, 1, true>(ks.pk + (size_t)rq.key * V::PK, msg, (size_t)rq.mlen, a.arena + rq.sig,
                                            mine, gs, ws, zt, izt, 0, 0, lane,
                                            ks.keys + (size_t)rq.key * S::KEY_POLYS * N, ks.tr + (size_t)rq.key * 32,
                                            mu_in);
        if (lane == 0) a.ok[slot] = (uint8_t)r;
        __threadfence_system();
        __syncwarp();
        if (lane == 0) complete(a, t);
        return;
    }
    if (!key_ok) {   // unknown key: rejected, not read
        zero_sig(a.sig_out + (size_t)slot * SERVE_SIG_STRIDE, lane);
        if (lane == 0) {
            a.status[slot] = DIL_EINVAL;
            a.iters[slot] = 0;
        }
        __threadfence_system();
        __syncwarp();
        if (lane == 0) complete(a, t);
        return;
    }
    ServeTask &tk = a.tasks[slot];
    if (lane == 0) {
        tk.next_r = 0;
        tk.best_r = INT_MAX;
        tk.committed_r = INT_MAX;
        tk.lock = 0;
        tk.fail = 0;
        atomicExch(&tk.tref, ((unsigned long long)t << 32) | 1ull);   // held by the owner
    }
    sign_prepare_keyed<LEVEL, 1>(ks.sk + (size_t)rq.key * V::SK, msg, (size_t)rq.mlen, gs, 0, 0, lane, mu_in);
    tk.mu[lane] = gs.hb[HB_MU + lane];
    tk.mu[32 + lane] = gs.hb[HB_MU + 32 + lane];
    tk.rhop[lane] = gs.rhop[lane];
    tk.rhop[32 + lane] = gs.rhop[32 + lane];
    __threadfence();
    __syncwarp();
    if (lane == 0) atomicExch(&a.worker_ticket[worker], (int)t);
    repetitions<LEVEL>(a, t, tk, ks.keys + (size_t)rq.key * S::KEY_POLYS * N, mine, stage, gs, ws, zt, izt, lane);
    if (lane == 0) atomicExch(&a.worker_ticket[worker], (int)NO_TICKET);
    leave<LEVEL>(a, t, tk, lane);
}

// Helps the Sign of ticket t (record already joined): its hashes from the
// record, its key's precomputation from the store.
template <int LEVEL>
__device__ void help(const ServeArgs &a, unsigned t, const ServeReq &rq, int32_t *mine, uint8_t *stage, GroupSmem &gs,
                     WarpSmem &ws, const int32_t *zt, const int32_t *izt, int lane, unsigned ticket) {
    const int slot = (int)(t & (unsigned)(a.ring - 1));
    ServeTask &tk = a.tasks[slot];
    const ServeKeys &ks = a.keys[LEVEL == 2 ? 0 : LEVEL == 3 ? 1 : 2];
    __threadfence();   // the owner wrote the hashes before it published the ticket
    gs.hb[HB_MU + lane] = __ldcg(tk.mu + lane);
    gs.hb[HB_MU + 32 + lane] = __ldcg(tk.mu + 32 + lane);
    gs.rhop[lane] = __ldcg(tk.rhop + lane);
    gs.rhop[32 + lane] = __ldcg(tk.rhop + 32 + lane);
    __syncwarp();
    repetitions<LEVEL>(a, t, tk, ks.keys + (size_t)rq.key * Scratch<LEVEL>::KEY_POLYS * N, mine, stage, gs, ws, zt,
                       izt, lane, true, ticket);
    leave<LEVEL>(a, t, tk, lane);
}

__device__ __forceinline__ ServeReq load_req(const ServeArgs &a, unsigned t) {
    const ServeReq *p = a.req + (t & (unsigned)(a.ring - 1));
    ServeReq r;
    const int4 w0 = __ldcg(reinterpret_cast<const int4 *>(p));
    const longlong2 w1 = __ldcg(reinterpret_cast<const longlong2 *>(p) + 1);
    const long long w2 = __ldcg(reinterpret_cast<const long long *>(p) + 4);
    r.op = w0.x;
    r.level = w0.y;
    r.key = w0.z;
    r.pad = w0.w;
    r.msg = (uint64_t)w1.x;
    r.mlen = (uint64_t)w1.y;
    r.sig = (uint64_t)w2;
    return r;
}

__device__ __forceinline__ int type_of(const ServeReq &rq) {
    return 3 * rq.op + (rq.level == 2 ? 0 : rq.level == 3 ? 1 : 2);
}

// Forwarding queues (lane 0 only).  A push reserves a position only when its
// entry is free, so a failed push leaves nothing behind (the caller then
// serves the ticket itself); a pop takes the head only when its entry is
// filled.  Both give up after a few contended tries.
__device__ bool fifo_push(const ServeArgs &a, int type, unsigned t) {
    ServeFifo &f = a.fifo[type];
    unsigned long long *ring = a.fifo_ring + (size_t)type * a.ring;
    for (int tries = 0; tries < 16; ++tries) {
        const unsigned pos = ld_acquire(&f.tail);
        unsigned long long *e = ring + (pos & (unsigned)(a.ring - 1));
        if ((unsigned)(atomicAdd(e, 0ull) >> 32) != pos) return false;   // entry still in use: full
        if (atomicCAS(&f.tail, pos, pos + 1) == pos) {
            atomicExch(e, ((unsigned long long)(pos + 1) << 32) | t);
            return true;
        }
    }
    return false;
}

__device__ bool fifo_pop(const ServeArgs &a, int type, unsigned &t) {
    ServeFifo &f = a.fifo[type];
    unsigned long long *ring = a.fifo_ring + (size_t)type * a.ring;
    for (int tries = 0; tries < 16; ++tries) {
        const unsigned pos = ld_acquire(&f.head);
        unsigned long long *e = ring + (pos & (unsigned)(a.ring - 1));
        const unsigned long long v = atomicAdd(e, 0ull);
        if ((unsigned)(v >> 32) != pos + 1) return false;   // empty (or its push is still writing)
        if (atomicCAS(&f.head, pos, pos + 1) == pos) {
            atomicExch(e, (unsigned long long)(pos + (unsigned)a.ring) << 32);   // free for the push R later
            t = (unsigned)v;
            return true;
        }
    }
    return false;
}

// One pass over SCAN_CHUNKS x 32 entries of worker_ticket from *cursor for a
// Sign that accepts another helper; joins it (CAS on its record) and
// returns its ticket, or NO_TICKET.
__device__ unsigned find_and_join(const ServeArgs &a, int nworkers, unsigned spec, unsigned &cursor, int lane) {
    unsigned found = NO_TICKET;
#pragma unroll 1
    for (int c = 0; c < SCAN_CHUNKS && found == NO_TICKET; ++c) {
        const unsigned idx = (cursor + 32u * c + lane) % (unsigned)nworkers;
        const unsigned u = (unsigned)__ldcg(a.worker_ticket + idx);
        bool cand = false;
        if (u != NO_TICKET) {
            const ServeTask &tk = a.tasks[u & (unsigned)(a.ring - 1)];
            const unsigned long long tr = __ldcg(&tk.tref);
            cand = (unsigned)(tr >> 32) == u && (unsigned)tr > 0 && (unsigned)tr <= spec &&
                   __ldcg(&tk.best_r) == INT_MAX;
        }
        const unsigned m = __ballot_sync(FULL, cand);
        if (m) found = __shfl_sync(FULL, u, __ffs(m) - 1);
    }
    cursor += 32u * SCAN_CHUNKS;
    if (found == NO_TICKET) return NO_TICKET;
    int joined = 0;
    if (lane == 0) {
        ServeTask &tk = a.tasks[found & (unsigned)(a.ring - 1)];
        unsigned long long cur = atomicAdd(&tk.tref, 0ull);
        for (int tries = 0; tries < 8; ++tries) {
            if ((unsigned)(cur >> 32) != found || (unsigned)cur == 0 || (unsigned)cur > spec) break;
            const unsigned long long prev = atomicCAS(&tk.tref, cur, cur + 1);
            if (prev == cur) {
                joined = 1;
                break;
            }
            cur = prev;
        }
    }
    joined = __shfl_sync(FULL, joined, 0);
    return joined ? found : NO_TICKET;
}

// ------------------------------------------------------------- mu hashers
// mu = H(tr || M) of published requests, precomputed in the sixteen-state
// form (about a sixth of the 25-lane form's cost per block under load) by the
// warps of the first hash_sms SMs while more than HASH_ON published requests
// wait for a worker (below HASH_OFF they serve requests like any worker; on
// SMs of their own they add no code to the SMs that serve one request type).
// Each of a hasher's sixteen instances absorbs one request's tr || M block by
// block and, once its message is done, writes mu to the request's slot and
// takes the next ticket, so instances never wait for one another's messages.  A worker uses a request's mu only when the slot's tag
// names that request's ticket; otherwise it hashes the message itself, so no
// worker ever waits for a hasher and a hasher may fall behind, skip or
// abandon tickets.  Tag protocol (64-bit word per slot): MU_VALID | (t + 1)
// once ticket t's mu is in the slot; a hasher claims the slot with
// MU_WRITING | (t + 1) by compare-and-swap only from a finished tag of an
// older ticket, so a stale hash never lands over a newer one.  A newer ticket
// of the same slot is published only after ticket t completed, so the mu a
// worker reads cannot change under it.
// Lane `lane` (< 17)'s 8 bytes of 136-byte block blk of tr (32 bytes, 8-byte
// aligned) || msg (mlen bytes, 8-byte aligned in the arena), padded in the
// final block.  The message is read in aligned words through L2 (the host
// writes the arena while the kernel runs); bytes past its end are masked.
__device__ __forceinline__ uint64_t mu_block_word(const uint8_t *tr, const uint8_t *msg, size_t mlen, int blk,
                                                  int total, int lane) {
    const size_t off = (size_t)blk * 136 + 8 * lane;
    uint64_t w = 0;
    if (off < 32) {
        const uint2 v = __ldg(reinterpret_cast<const uint2 *>(tr + off));
        w = ((uint64_t)v.y << 32) | v.x;
    } else if (off - 32 < mlen) {
        w = ld_word_cg(msg + (off - 32));
        const size_t have = mlen - (off - 32);
        if (have < 8) w &= (1ull << (8 * have)) - 1;
    }
    if (blk == total - 1) pad_word(w, (int)(32 + mlen - (size_t)blk * 136), 136, lane);
    return w;
}

// Writes instance s's mu (stream words 0..15) for ticket t if the slot takes it.
__device__ void publish_mu(const ServeArgs &a, unsigned t, const uint32_t *kst, int s, int lane) {
    const unsigned slot = t & (unsigned)(a.ring - 1);
    unsigned long long *tag = a.mu_tag + slot;
    int won = 0;
    if (lane == 0) {
        const unsigned long long cur = atomicAdd(tag, 0ull);
        won = !(cur & MU_WRITING) && (int)((t + 1u) - (unsigned)cur) > 0 &&
              atomicCAS(tag, cur, MU_WRITING | (unsigned long long)(t + 1u)) == cur;
    }
    if (!__shfl_sync(FULL, won, 0)) return;
    if (lane < 16) reinterpret_cast<uint32_t *>(a.mu_buf + (size_t)slot * 64)[lane] = kst[k16_word(s, lane)];
    __threadfence();
    __syncwarp();
    if (lane == 0) atomicExch(tag, MU_VALID | (unsigned long long)(t + 1u));
}

// Published requests not yet taken by a worker (head may run ahead of tail:
// idle workers hold the next numbers).
__device__ __forceinline__ int backlog(const ServeArgs &a) {
    return (int)(tail_of(a) - (unsigned)ld_acquire(&a.ctl->head));
}

// One hasher pass loop of a warp on a hashing SM; lane s < 16 keeps instance
// s's request.  Returns true when the host set stop, false once the backlog
// falls below HASH_OFF (the warp then serves requests like any worker; the
// hashes it leaves unfinished are simply not used).
__device__ bool hash_worker(const ServeArgs &a, uint32_t *kst, int lane) {
    unsigned t = 0;
    int state = 0;   // 0 free, 1 holding an unpublished ticket, 2 absorbing
    const uint8_t *msg = nullptr, *tr = nullptr;
    size_t mlen = 0;
    int total = 0, next = 0;
    for (;;) {
        // lane 0 reads the control words once per pass (the serving workers poll the same line)
        int stop = 0, low = 0;
        unsigned tail = 0, head = 0;
        if (lane == 0) {
            stop = ld_acquire(&a.ctl->stop);
            tail = tail_of(a);
            head = (unsigned)ld_acquire(&a.ctl->head);
            low = (int)(tail - head) < HASH_OFF;
            // tickets the workers have taken are not worth hashing: move the hashers' counter up
            const unsigned hh = *reinterpret_cast<volatile unsigned *>(&a.ctl->hhead);
            if ((int)(head - hh) > 0) atomicCAS(reinterpret_cast<unsigned *>(&a.ctl->hhead), hh, head);
        }
        if (__shfl_sync(FULL, stop, 0)) return true;
        if (__shfl_sync(FULL, low, 0)) return false;
        tail = __shfl_sync(FULL, tail, 0);
        __syncwarp();   // descriptor loads below come after lane 0's acquire of tail
        if (lane < 16) {
            if (state == 0) {
                t = atomicAdd(reinterpret_cast<unsigned *>(&a.ctl->hhead), 1u);
                state = 1;
            }
            if (state == 1 && (int)(tail - t) > 0) {
                const ServeReq rq = load_req(a, t);
                const ServeKeys &ks = a.keys[rq.level == 2 ? 0 : rq.level == 3 ? 1 : 2];
                state = 0;
                if (rq.key >= 0 && rq.key < ks.n) {   // unknown keys are answered without a mu
                    tr = ks.tr + (size_t)rq.key * 32;
                    msg = a.arena + rq.msg;
                    mlen = (size_t)rq.mlen;
                    total = (int)((32 + mlen) / 136) + 1;
                    next = 0;
                    state = 2;
                }
            }
        }
        const unsigned active = __ballot_sync(FULL, lane < 16 && state == 2);
        if (!active) {
            __nanosleep(500);
            continue;
        }
        // absorb each active instance's next block (lanes 0..24 cover its 25 state lanes)
        for (unsigned m = active; m; m &= m - 1) {
            const int s = __ffs(m) - 1;
            const uint8_t *ms = reinterpret_cast<const uint8_t *>(
                __shfl_sync(FULL, reinterpret_cast<unsigned long long>(msg), s));
            const uint8_t *ts = reinterpret_cast<const uint8_t *>(
                __shfl_sync(FULL, reinterpret_cast<unsigned long long>(tr), s));
            const size_t ml = (size_t)__shfl_sync(FULL, (unsigned long long)mlen, s);
            const int tot = __shfl_sync(FULL, total, s), blk = __shfl_sync(FULL, next, s);
            if (lane < 25) {
                const uint64_t w = lane < 17 ? mu_block_word(ts, ms, ml, blk, tot, lane) : 0;
                uint32_t *st = kst + k16_slot(lane, 2 * s);
                if (blk == 0) {
                    st[0] = (uint32_t)w;
                    st[1] = (uint32_t)(w >> 32);
                } else {
                    st[0] ^= (uint32_t)w;
                    st[1] ^= (uint32_t)(w >> 32);
                }
            }
        }
        __syncwarp();
        keccak16_permute(kst);
        if (lane < 16 && state == 2) ++next;
        const unsigned done = __ballot_sync(FULL, lane < 16 && state == 2 && next == total);
        for (unsigned m = done; m; m &= m - 1) {
            const int s = __ffs(m) - 1;
            publish_mu(a, __shfl_sync(FULL, t, s), kst, s, lane);
        }
        if (lane < 16 && state == 2 && next == total) state = 0;
    }
}

__device__ __forceinline__ unsigned sm_id() {
    unsigned id;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(id));
    return id;
}

// Serves ticket t as its owner, counted in ServeCtl::active.
__device__ __forceinline__ void serve(const ServeArgs &a, unsigned t, const ServeReq &rq, int worker, int32_t *mine,
                                      uint8_t *stage, GroupSmem &gs, WarpSmem &ws, const int32_t *zt,
                                      const int32_t *izt, int lane) {
    if (lane == 0) atomicAdd(&a.ctl->active, 1);
    switch (rq.level) {
        case 2: own<2>(a, t, rq, worker, mine, stage, gs, ws, zt, izt, lane); break;
        case 3: own<3>(a, t, rq, worker, mine, stage, gs, ws, zt, izt, lane); break;
        default: own<5>(a, t, rq, worker, mine, stage, gs, ws, zt, izt, lane); break;
    }
    if (lane == 0) atomicSub(&a.ctl->active, 1);
}

__global__ void __launch_bounds__(SERVE_WARPS * 32, 4) k_serve(ServeArgs a) {
    extern __shared__ __align__(16) uint8_t smem[];
    const CtaView v = cta_setup<1>(smem);
    GroupSmem &gs = *v.gs;
    WarpSmem &ws = *v.ws;
    const int lane = v.lane;
    const int worker = blockIdx.x * v.groups + v.group;
    const int nworkers = gridDim.x * v.groups;
    int32_t *mine = a.scratch + (size_t)worker * a.worker_polys * N;
    uint8_t *stage = a.sig_stage + (size_t)worker * SERVE_SIG_STRIDE;
    unsigned cursor = (unsigned)worker * 2654435761u % (unsigned)nworkers;
    const unsigned smid = sm_id();
    const bool hashing_sm = (int)smid < a.hash_sms;   // its warps hash mu while requests queue
    const int home = smid < SERVE_MAX_SMS ? a.sm_type[smid] : SERVE_TYPE_ANY;
    unsigned ticket = 0;
    bool holding = false;
    long long waiting_since = -1;
    for (;;) {
        if (!holding && hashing_sm) {
            int busy = 0;
            if (lane == 0) busy = backlog(a) > HASH_ON;
            if (__shfl_sync(FULL, busy, 0)) {
                if (hash_worker(a, ws.k16, lane)) break;   // stop: nothing of this warp is in flight
                continue;
            }
        }
        if (!holding) {
            if (home != SERVE_TYPE_ANY) {   // tickets of the home type forwarded from other SMs first
                unsigned f = 0;
                int got = 0;
                if (lane == 0) got = fifo_pop(a, home, f);
                got = __shfl_sync(FULL, got, 0);
                f = __shfl_sync(FULL, f, 0);
                if (got) {
                    serve(a, f, load_req(a, f), worker, mine, stage, gs, ws, v.zt, v.izt, lane);
                    continue;
                }
            }
            unsigned t = 0;   // take the next ticket number
            if (lane == 0) t = atomicAdd(reinterpret_cast<unsigned *>(&a.ctl->head), 1u);
            ticket = __shfl_sync(FULL, t, 0);
            holding = true;
            waiting_since = -1;
        }
        int published = 0, stop = 0;
        long long now = 0;
        if (lane == 0) {
            stop = ld_acquire(&a.ctl->stop);   // stop is written after every tail it follows
            published = (int)(tail_of(a) - ticket) > 0;
            now = global_ns();
        }
        published = __shfl_sync(FULL, published, 0);
        if (published) {
            holding = false;
            const ServeReq rq = load_req(a, ticket);
            const int ty = type_of(rq);
            int fwd = 0;   // under load, hand a ticket of another type to that type's SMs
            if (lane == 0 && ty != home && a.type_sms[ty] > 0 && ld_acquire(&a.ctl->active) >= a.forward_above) {
                const ServeFifo &f = a.fifo[ty];
                const unsigned len = ld_acquire(&f.tail) - ld_acquire(&f.head);
                if (len < (unsigned)(a.fifo_limit * a.type_sms[ty])) fwd = fifo_push(a, ty, ticket);
            }
            if (__shfl_sync(FULL, fwd, 0)) continue;
            serve(a, ticket, rq, worker, mine, stage, gs, ws, v.zt, v.izt, lane);
            continue;
        }
        if (__shfl_sync(FULL, stop, 0)) break;   // the ticket is abandoned: the host resets head
        now = __shfl_sync(FULL, now, 0);
        if (waiting_since < 0) waiting_since = now;
        if (now - waiting_since > a.idle_ns) {   // bounded wait: record it and leave
            if (lane == 0) atomicExch(&a.ctl->error, DIL_ETIMEOUT);
            break;
        }
        // while the ticket is unpublished, help an unfinished Sign: up to spec
        // helpers per Sign while fewer than help_below workers serve their own
        // request, none above
        unsigned spec_now = 0;
        if (lane == 0) spec_now = ld_acquire(&a.ctl->active) < a.help_below ? a.spec : 0;
        spec_now = __shfl_sync(FULL, spec_now, 0);
        const unsigned helped = spec_now ? find_and_join(a, nworkers, spec_now, cursor, lane) : NO_TICKET;
        if (helped != NO_TICKET) {
            const ServeReq rq = load_req(a, helped);
            switch (rq.level) {
                case 2: help<2>(a, helped, rq, mine, stage, gs, ws, v.zt, v.izt, lane, ticket); break;
                case 3: help<3>(a, helped, rq, mine, stage, gs, ws, v.zt, v.izt, lane, ticket); break;
                default: help<5>(a, helped, rq, mine, stage, gs, ws, v.zt, v.izt, lane, ticket); break;
            }
            continue;
        }
        __nanosleep(500);
    }
}

}  // namespace

size_t serve_worker_polys() {
    size_t m = 0;
    const size_t v[] = {(size_t)Scratch<2>::ITR_POLYS, (size_t)Scratch<3>::ITR_POLYS, (size_t)Scratch<5>::ITR_POLYS,
                        (size_t)Scratch<2>::KEYED_VERIFY_POLYS, (size_t)Scratch<3>::KEYED_VERIFY_POLYS,
                        (size_t)Scratch<5>::KEYED_VERIFY_POLYS};
    for (size_t x : v) m = x > m ? x : m;
    return m;
}

cudaError_t serve_grid(int device, int max_workers, int &grid, int &workers) {
    int sms = 0, occ = 0;
    cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    if (e != cudaSuccess) return e;
    const size_t smem = cta_bytes(SERVE_WARPS, 1);
    e = cudaFuncSetAttribute(k_serve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_serve, SERVE_WARPS * 32, smem);
    if (e != cudaSuccess) return e;
    if (occ < 1) occ = 1;
    grid = sms * occ;
    if (max_workers > 0 && grid * SERVE_WARPS > max_workers) grid = max_workers / SERVE_WARPS;
    if (grid < 1) grid = 1;
    workers = grid * SERVE_WARPS;
    return cudaSuccess;
}

cudaError_t launch_serve(const ServeArgs &a, int grid, cudaStream_t s) {
    k_serve<<<grid, SERVE_WARPS * 32, cta_bytes(SERVE_WARPS, 1), s>>>(a);
    return cudaGetLastError();
}

}  // namespace dil

// Persistent Sign with a device work queue (section 4.3 of arXiv 2211.12265,
// dynamic task scheduling, redesigned to run entirely on the device).
//
// Workers are groups of P warps that stay resident for the whole launch.  A
// worker takes a fresh task from the queue (atomic cursor), prepares it into
// its own scratch slot (mu, rho', A^, s^1, s^2, t^0), publishes the slot, and
// then draws repetition indices r from the task's counter, running the loop
// body with nonce kappa = l r.  When the queue is empty, idle workers become
// helpers: they join an unfinished task (at most `spec` per task), read its
// published precomputation through L2 and draw further r from the same
// counter, i.e. they evaluate predicted nonces.  Every accepting r lowers the
// task's best_r; the signature in the output is written under a per-task lock
// only by a smaller r than the one already committed, so the result is the
// signature of the smallest accepting nonce: exactly the sequential result.
// All r below the final one are evaluated (they are handed out in order and an
// r is skipped only when it exceeds an accepted one).
//
// Waits (commit lock, an owner waiting for its helpers before reusing its
// slot) poll at most spin_limit times (PERSIST_SPIN_LIMIT unless a test lowers
// it); then the kernel records DIL_ETIMEOUT in the queue's error word, marks
// the task failed and continues.  Workers draw no further repetitions of a
// failed task and write none of its results; a finalize kernel that runs
// after the grid gives every failed task status DIL_ETIMEOUT, 0 repetitions
// and a zeroed signature, so each task of a launch ends with a defined
// output even though late writers (a helper still running when its owner's
// wait gave up) may have touched it.  The holders of these waits never wait
// on anything themselves, so the limit is a safety net only.
#include <climits>
#include <cstddef>

#include "../../include/dil.h"
#include "dil_kern.cuh"

namespace dil {

constexpr int PERSIST_META_POLYS = 1;   // mu (64 B) and rho' (64 B) of a slot's task

__device__ __forceinline__ int ld_l2(const int *p) { return __ldcg(p); }

// Waits until *p reads 0, at most `limit` polls; false when the limit ran out.
__device__ __forceinline__ bool wait_until_zero(int *p, int limit) {
    for (int i = 0; i < limit; ++i) {
        if (atomicAdd(p, 0) == 0) return true;
        __nanosleep(128);
    }
    return false;
}

// Test hook for the bounded wait: one thread waits on `flag` and records the
// outcome (DIL_OK or DIL_ETIMEOUT) in *result.
__global__ void k_test_bounded_wait(int *flag, int limit, int *result) {
    if (threadIdx.x == 0 && blockIdx.x == 0) *result = wait_until_zero(flag, limit) ? DIL_OK : DIL_ETIMEOUT;
}

__device__ __forceinline__ const PersistJob &job_of(const PersistJobs &J, int t, int &local) {
    int j = 0;
    while (j + 1 < J.njobs && t >= J.job[j + 1].start) ++j;
    local = t - J.job[j].start;
    return J.job[j];
}

template <int LEVEL>
__device__ __forceinline__ int iter_cap(int override_cap) {
    return (override_cap > 0 && override_cap < Lv<LEVEL>::MAX_ITER) ? override_cap : Lv<LEVEL>::MAX_ITER;
}

struct PersistCtx {
    PersistQueue *q;
    PersistTask *tasks;
    int *slot_task;
    int32_t *scratch;
    int slot_polys;
    int slots;
    int max_iter_override;
    int spec;
    int spin_limit;
};

// A bounded wait on task tk ran out: record it launch-wide and on the task.
__device__ __forceinline__ void wait_failed(const PersistCtx &pc, PersistTask &tk) {
    atomicExch(&tk.fail, 1);
    atomicExch(&pc.q->error, DIL_ETIMEOUT);
}

// Writes the signature of repetition r for task t if r beats the committed one.
template <int LEVEL, int P>
__device__ void commit(const PersistCtx &pc, PersistTask &tk, int r, const PersistJob &jb, int local,
                       const int32_t *itr, GroupSmem &gs, int g, int bar, int lane) {
    const bool leader = g == 0 && lane == 0;
    if (leader) {
        atomicMin(&tk.best_r, r);
        int acquired = 0;
        for (int i = 0; i < pc.spin_limit; ++i) {
            if (atomicCAS(&tk.lock, 0, 1) == 0) {
                acquired = 1;
                break;
            }
            __nanosleep(64);
        }
        if (!acquired) wait_failed(pc, tk);
        __threadfence();
        // a failed task's output is the finalize kernel's to write
        const int win = acquired && r < atomicOr(&tk.committed_r, 0) && !atomicOr(&tk.fail, 0);
        gs.claim2 = acquired ? (win ? 2 : 1) : 0;
    }
    group_sync<P>(bar);
    const int st = *(volatile int *)&gs.claim2;
    if (st == 2) {
        sign_pack<LEVEL, P>(jb.sig + (size_t)local * Lv<LEVEL>::SIG, itr, gs, g, lane);
        if (leader) {
            if (jb.status) jb.status[local] = 0;
            if (jb.iters) jb.iters[local] = r + 1;
        }
    }
    __threadfence();
    group_sync<P>(bar);
    if (leader && st >= 1) {
        if (st == 2) atomicExch(&tk.committed_r, r);
        __threadfence();
        atomicExch(&tk.lock, 0);
    }
    group_sync<P>(bar);
}

// Draws repetitions of task t until one accepts, the counter passes an
// accepted r, or the cap is reached.  pre: the task's precomputation.  A
// one-warp worker claims two consecutive repetitions at a time, so that the
// second reuses masks its stream sampled for the first (one stream batch
// covers MASK_BATCH / l repetitions; workers that share a task would
// otherwise each start a new batch for every repetition); longer claims
// reuse more masks but serialise more of a task's repetitions on one worker
// and measured slower.  A worker abandons the rest of its claim once a
// smaller repetition has accepted.
template <int LEVEL, int P>
__device__ void run_repetitions(const PersistCtx &pc, PersistTask &tk, const PersistJob &jb, int local,
                                const int32_t *pre, int32_t *itr, GroupSmem &gs, WarpSmem &ws, const int32_t *zt,
                                const int32_t *izt, int g, int bar, int lane) {
    constexpr int PER_BATCH = Scratch<LEVEL>::MASK_BATCH / Lv<LEVEL>::L;
    constexpr int CLAIM = (P == 1) ? (PER_BATCH < 2 ? PER_BATCH : 2) : 1;
    const int cap = iter_cap<LEVEL>(pc.max_iter_override);
    const bool leader = g == 0 && lane == 0;
    MaskStream ms{0, 0};
    int next = 0, end = 0;   // the leader's current claim [next, end)
    for (;;) {
        if (leader) {
            if (next >= end) {
                next = atomicAdd(&tk.next_r, CLAIM);
                end = next + CLAIM;
            }
            const int r = next++;
            const int best = atomicOr(&tk.best_r, 0);
            const int stop = ld_l2(&pc.q->cancel) || ld_l2(&tk.fail);
            gs.claim2 = (!stop && r < cap && r < best) ? r : -1;
        }
        group_sync<P>(bar);
        const int r = *(volatile int *)&gs.claim2;
        group_sync<P>(bar);
        if (r < 0) break;
        if (sign_attempt<LEVEL, P>(Lv<LEVEL>::L * r, pre, itr, ms, gs, ws, zt, izt, g, bar, lane, &tk.best_r, r)) {
            commit<LEVEL, P>(pc, tk, r, jb, local, itr, gs, g, bar, lane);
            break;
        }
    }
}

// A task left unsigned because the host canceled the launch: zeroed
// signature, status DIL_ECANCELED, 0 repetitions.
template <int LEVEL, int P>
__device__ void mark_canceled(const PersistJob &jb, int local, int g, int lane) {
    sign_zero<LEVEL, P>(jb.sig + (size_t)local * Lv<LEVEL>::SIG, g, lane);
    if (g == 0 && lane == 0) {
        if (jb.status) jb.status[local] = DIL_ECANCELED;
        if (jb.iters) jb.iters[local] = 0;
    }
}

// Works on task t, as its owner (own: prepare, publish, repeat, release, and
// report a capped or canceled task) or as a helper of the owner in slot s
// (read the published precomputation and repeat).  One function for both
// roles, so that the kernel holds a single copy of the repetition loop per
// level: instruction fetch is the kernels' first stall, and a second copy for
// helpers measured 7% slower at 10,000 tasks.  `slot` is the caller's own
// slot; s the owner's (equal to slot when own).
template <int LEVEL, int P>
__device__ void work_task(const PersistCtx &pc, bool own, int t, const PersistJob &jb, int local, int slot, int s,
                          int32_t *mine, GroupSmem &gs, WarpSmem &ws, const int32_t *zt, const int32_t *izt, int g,
                          int bar, int lane) {
    using V = Lv<LEVEL>;
    using S = Scratch<LEVEL>;
    const bool leader = g == 0 && lane == 0;
    PersistTask &tk = pc.tasks[t];
    const int32_t *pre = mine;
    if (own) {
        if (leader) {
            tk.next_r = 0;
            tk.best_r = INT_MAX;
            tk.committed_r = INT_MAX;
            tk.lock = 0;
            tk.helpers = 0;
        }
        uint64_t m0;
        size_t mlen;
        if (!message_of(jb.off, local, m0, mlen)) {   // decreasing offsets: reject (never published, so no helpers)
            sign_zero<LEVEL, P>(jb.sig + (size_t)local * V::SIG, g, lane);
            if (leader) {
                if (jb.status) jb.status[local] = DIL_EINVAL;
                if (jb.iters) jb.iters[local] = 0;
            }
            group_sync<P>(bar);
            return;
        }
        sign_prepare<LEVEL, P>(jb.sk + (size_t)local * V::SK, jb.msg + m0, mlen, mine, gs, ws, zt, g, bar, lane);
        uint8_t *meta = reinterpret_cast<uint8_t *>(mine + S::SIGN_POLYS * N);
        if (g == 0) {
            meta[lane] = gs.hb[HB_MU + lane];
            meta[32 + lane] = gs.hb[HB_MU + 32 + lane];
            meta[64 + lane] = gs.rhop[lane];
            meta[96 + lane] = gs.rhop[32 + lane];
        }
        __threadfence();
        group_sync<P>(bar);
        if (leader) atomicExch(&pc.slot_task[slot], t);
    } else {
        pre = pc.scratch + (size_t)s * pc.slot_polys * N;
        const uint8_t *meta = reinterpret_cast<const uint8_t *>(pre + S::SIGN_POLYS * N);
        if (g == 0) {
            gs.hb[HB_MU + lane] = __ldcg(meta + lane);
            gs.hb[HB_MU + 32 + lane] = __ldcg(meta + 32 + lane);
            gs.rhop[lane] = __ldcg(meta + 64 + lane);
            gs.rhop[32 + lane] = __ldcg(meta + 96 + lane);
        }
        group_sync<P>(bar);
    }
    run_repetitions<LEVEL, P>(pc, tk, jb, local, pre, mine + S::PRE_POLYS * N, gs, ws, zt, izt, g, bar, lane);
    if (!own) return;
    if (leader) {
        atomicExch(&pc.slot_task[slot], -1);
        __threadfence();
        if (!wait_until_zero(&tk.helpers, pc.spin_limit)) wait_failed(pc, tk);
        // no accepting repetition: the cap was reached, or the host canceled the launch
        gs.claim2 = (atomicOr(&tk.best_r, 0) != INT_MAX) ? 0 : ld_l2(&pc.q->cancel) ? 2 : 1;
    }
    group_sync<P>(bar);
    const int unsigned_task = *(volatile int *)&gs.claim2;
    group_sync<P>(bar);
    if (unsigned_task == 1) {
        sign_zero<LEVEL, P>(jb.sig + (size_t)local * V::SIG, g, lane);
        if (leader) {
            if (jb.status) jb.status[local] = DIL_EITER;
            if (jb.iters) jb.iters[local] = iter_cap<LEVEL>(pc.max_iter_override);
        }
    } else if (unsigned_task == 2) {
        mark_canceled<LEVEL, P>(jb, local, g, lane);
    }
}

// ONLY = 0 compiles the task bodies of all three levels (launches that mix
// levels); ONLY = 2, 3 or 5 compiles one level's, a smaller kernel with less
// register pressure for the common single-level launch.
template <int P, int ONLY>
__global__ void __launch_bounds__(256, 4) k_sign_persist(PersistJobs J, PersistQueue *q, PersistTask *tasks,
                                                         int *slot_task, int32_t *scratch, int slot_polys,
                                                         int max_iter_override, int chunk, int spec,
                                                         int spin_limit) {
    extern __shared__ __align__(16) uint8_t smem[];
    const CtaView v = cta_setup<P>(smem);
    GroupSmem &gs = *v.gs;
    WarpSmem &ws = *v.ws;
    const int g = v.g, bar = v.bar, lane = v.lane;
    const bool leader = g == 0 && lane == 0;
    PersistCtx pc{q, tasks, slot_task, scratch, slot_polys, (int)gridDim.x * v.groups, max_iter_override, spec,
                  spin_limit};
    const int slot = blockIdx.x * v.groups + v.group;
    int32_t *mine = scratch + (size_t)slot * slot_polys * N;
    // One scheduling loop: fresh tasks from the queue (owned; after a host
    // cancel only marked), then speculative help on unfinished tasks
    // (predicted nonces).  Both roles go through the one work_task call below.
    bool canceled = false, fresh = true;
    int cur = 0, end = 0;
    int start = (int)(((unsigned)slot * 2654435761u) % (unsigned)pc.slots);
    // the job whose fresh tasks this SM takes first (leader only); advances
    // once that job's tasks are all claimed
    int home = 0;
    if (leader) {
        unsigned smid;
        asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
        while (home + 1 < J.njobs && (int)smid >= J.sm_end[home]) ++home;
    }
    for (int round = 0; round < 4096;) {
        int t, s;
        bool own;
        if (fresh) {
            if (cur >= end) {
                if (leader) {   // up to `chunk` fresh tasks of the home job, else of the next job with any left
                    int got = -1;
                    for (int k = 0; k < J.njobs && got < 0; ++k) {
                        const int c = atomicAdd(&q->next_job[home], chunk);
                        if (c < J.job[home].n)
                            got = J.job[home].start + c;
                        else
                            home = (home + 1) % J.njobs;
                    }
                    gs.claim = got;
                    gs.claim2 = ld_l2(&q->cancel);
                }
                group_sync<P>(bar);
                const int c0 = *(volatile int *)&gs.claim;
                canceled = *(volatile int *)&gs.claim2 != 0;
                group_sync<P>(bar);
                if (c0 < 0) {
                    fresh = false;
                    if (spec <= 0 || canceled || ld_l2(&q->cancel)) break;
                    continue;
                }
                int local;
                const PersistJob &jc = job_of(J, c0, local);
                cur = c0;
                end = jc.start + min(local + chunk, jc.n);
            }
            t = cur++;
            s = slot;
            own = true;
            if (canceled) {
                int local;
                const PersistJob &jb = job_of(J, t, local);
                switch (jb.level) {
                    case 2: if constexpr (ONLY == 0 || ONLY == 2) mark_canceled<2, P>(jb, local, g, lane); break;
                    case 3: if constexpr (ONLY == 0 || ONLY == 3) mark_canceled<3, P>(jb, local, g, lane); break;
                    default: if constexpr (ONLY == 0 || ONLY == 5) mark_canceled<5, P>(jb, local, g, lane); break;
                }
                continue;
            }
        } else {
            ++round;
            if (g == 0) {
                int found_s = -1, found_t = -1;
                // after a host cancel there is nothing left to help
                const int stop = __shfl_sync(FULL, lane == 0 ? ld_l2(&q->cancel) : 0, 0);
                for (int base = 0; base < pc.slots && found_s < 0 && !stop; base += 32) {
                    const int idx = base + lane;
                    const int cs = (start + idx) % pc.slots;
                    int ct = idx < pc.slots ? ld_l2(slot_task + cs) : -1;
                    bool cand = false;
                    if (ct >= 0) cand = ld_l2(&tasks[ct].best_r) == INT_MAX && ld_l2(&tasks[ct].helpers) < spec;
                    const unsigned m = __ballot_sync(FULL, cand);
                    if (m) {
                        const int src = __ffs(m) - 1;
                        found_s = __shfl_sync(FULL, cs, src);
                        found_t = __shfl_sync(FULL, ct, src);
                    }
                }
                int joined = 0;
                if (found_s >= 0 && lane == 0) {
                    atomicAdd(&tasks[found_t].helpers, 1);
                    __threadfence();
                    if (atomicOr(&slot_task[found_s], 0) == found_t && atomicOr(&tasks[found_t].best_r, 0) == INT_MAX)
                        joined = 1;
                    else
                        atomicSub(&tasks[found_t].helpers, 1);
                }
                joined = __shfl_sync(FULL, joined, 0);
                if (lane == 0) {
                    gs.claim = found_s < 0 ? -2 : (joined ? found_s : -1);
                    gs.claim2 = found_t;
                }
            }
            group_sync<P>(bar);
            s = *(volatile int *)&gs.claim;
            t = *(volatile int *)&gs.claim2;
            group_sync<P>(bar);
            if (s == -2) break;
            if (s == -1) continue;
            own = false;
        }
        int local;
        const PersistJob &jb = job_of(J, t, local);
        switch (jb.level) {
            case 2:
                if constexpr (ONLY == 0 || ONLY == 2)
                    work_task<2, P>(pc, own, t, jb, local, slot, s, mine, gs, ws, v.zt, v.izt, g, bar, lane);
                break;
            case 3:
                if constexpr (ONLY == 0 || ONLY == 3)
                    work_task<3, P>(pc, own, t, jb, local, slot, s, mine, gs, ws, v.zt, v.izt, g, bar, lane);
                break;
            default:
                if constexpr (ONLY == 0 || ONLY == 5)
                    work_task<5, P>(pc, own, t, jb, local, slot, s, mine, gs, ws, v.zt, v.izt, g, bar, lane);
                break;
        }
        if (!own) {
            __threadfence();
            group_sync<P>(bar);
            if (leader) atomicSub(&tasks[t].helpers, 1);
            start = (start + 1) % pc.slots;
        }
    }
}

// Runs after the persistent grid: every task whose bounded wait ran out ends
// with status DIL_ETIMEOUT, 0 repetitions and a zeroed signature (nothing of
// the launch writes to it any more).  One thread per task.
__global__ void k_persist_finalize(PersistJobs J, const PersistTask *tasks) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < J.total; t += gridDim.x * blockDim.x) {
        if (!tasks[t].fail) continue;
        int local;
        const PersistJob &jb = job_of(J, t, local);
        const int sigb = jb.level == 2 ? Lv<2>::SIG : jb.level == 3 ? Lv<3>::SIG : Lv<5>::SIG;
        uint8_t *sig = jb.sig + (size_t)local * sigb;
        for (int b = 0; b < sigb; ++b) sig[b] = 0;
        if (jb.status) jb.status[local] = DIL_ETIMEOUT;
        if (jb.iters) jb.iters[local] = 0;
    }
}

// ---------------------------------------------------------------- host side
namespace {

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

int slot_polys_for(const PersistJobs &J) {
    int m = 0;
    for (int j = 0; j < J.njobs; ++j) {
        int p = (int)scratch_polys(OP_SIGN, J.job[j].level);
        m = p > m ? p : m;
    }
    return m + PERSIST_META_POLYS;
}

using PersistKernel = void (*)(PersistJobs, PersistQueue *, PersistTask *, int *, int32_t *, int, int, int, int,
                               int);

// The kernel for a launch: one-warp groups whose jobs share one level get
// that level's kernel, everything else the all-level one.
PersistKernel kernel_for(const PersistJobs &J, int p) {
    int only = J.job[0].level;
    for (int j = 1; j < J.njobs; ++j)
        if (J.job[j].level != only) only = 0;
    if (p == 1) {
        switch (only) {
            case 2: return k_sign_persist<1, 2>;
            case 3: return k_sign_persist<1, 3>;
            case 5: return k_sign_persist<1, 5>;
        }
    }
    switch (p) {
        case 1: return k_sign_persist<1, 0>;
        case 2: return k_sign_persist<2, 0>;
        case 4: return k_sign_persist<4, 0>;
    }
    return nullptr;
}

cudaError_t grid_of(const PersistJobs &J, const PersistTuning &t, int device, int &grid) {
    const PersistKernel kern = kernel_for(J, t.p);
    if (!kern) return cudaErrorInvalidValue;
    int sms = 0, occ = 0;
    cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    if (e != cudaSuccess) return e;
    const size_t smem = cta_bytes(t.warps, t.p);
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, t.warps * 32, smem);
    if (e != cudaSuccess) return e;
    if (occ < 1) occ = 1;
    int per_sm = (t.ctas_per_sm > 0 && t.ctas_per_sm < occ) ? t.ctas_per_sm : occ;
    grid = sms * per_sm;
    return cudaSuccess;
}

struct Layout {
    size_t q, tasks, slots, scratch, total;
    int nslots, slot_polys, grid;
};

cudaError_t layout_of(const PersistJobs &J, const PersistTuning &t, int device, Layout &L) {
    cudaError_t e = grid_of(J, t, device, L.grid);
    if (e != cudaSuccess) return e;
    L.nslots = L.grid * (t.warps / t.p);
    L.slot_polys = slot_polys_for(J);
    L.q = 0;
    L.tasks = al256(sizeof(PersistQueue));
    L.slots = L.tasks + al256((size_t)J.total * sizeof(PersistTask));
    L.scratch = L.slots + al256((size_t)L.nslots * sizeof(int));
    L.total = L.scratch + (size_t)L.nslots * L.slot_polys * N * sizeof(int32_t);
    return cudaSuccess;
}

}  // namespace

size_t persist_workspace_bytes(const PersistJobs &J, const PersistTuning &t, int device) {
    Layout L;
    if (layout_of(J, t, device, L) != cudaSuccess) return 0;
    return L.total;
}

cudaError_t launch_sign_persist(const PersistJobs &J, void *ws, const PersistTuning &t, int max_iter_override,
                                int spin_limit, int device, cudaStream_t s) {
    if (J.total <= 0) return cudaSuccess;
    Layout L;
    cudaError_t e = layout_of(J, t, device, L);
    if (e != cudaSuccess) return e;
    uint8_t *base = static_cast<uint8_t *>(ws);
    e = cudaMemsetAsync(base + L.q, 0, sizeof(PersistQueue), s);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(base + L.slots, 0xFF, (size_t)L.nslots * sizeof(int), s);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(base + L.tasks, 0, (size_t)J.total * sizeof(PersistTask), s);   // clears every fail flag
    if (e != cudaSuccess) return e;
    auto *q = reinterpret_cast<PersistQueue *>(base + L.q);
    auto *tasks = reinterpret_cast<PersistTask *>(base + L.tasks);
    auto *slot_task = reinterpret_cast<int *>(base + L.slots);
    auto *scratch = reinterpret_cast<int32_t *>(base + L.scratch);
    const size_t smem = cta_bytes(t.warps, t.p);
    const int chunk = t.chunk > 0 ? t.chunk : 1;
    const PersistKernel kern = kernel_for(J, t.p);
    const int limit = (spin_limit > 0 && spin_limit < PERSIST_SPIN_LIMIT) ? spin_limit : PERSIST_SPIN_LIMIT;
    kern<<<L.grid, t.warps * 32, smem, s>>>(J, q, tasks, slot_task, scratch, L.slot_polys, max_iter_override, chunk,
                                            t.spec, limit);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int fin_blocks = (J.total + 255) / 256 < 4 * L.grid ? (J.total + 255) / 256 : 4 * L.grid;
    k_persist_finalize<<<fin_blocks, 256, 0, s>>>(J, tasks);
    return cudaGetLastError();
}

cudaError_t test_bounded_wait(int flag_value, int limit, int *result_host) {
    int *d = nullptr;
    cudaError_t e = cudaMalloc(&d, 2 * sizeof(int));
    if (e != cudaSuccess) return e;
    int h[2] = {flag_value, -99};
    e = cudaMemcpy(d, h, sizeof(h), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        k_test_bounded_wait<<<1, 32>>>(d, limit, d + 1);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(h, d, sizeof(h), cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e == cudaSuccess) *result_host = h[1];
    return e;
}

int persist_error(void *ws) {
    PersistQueue h;
    if (cudaMemcpy(&h, ws, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess) return DIL_ECUDA;
    return h.error ? DIL_ETIMEOUT : h.cancel ? DIL_ECANCELED : DIL_OK;
}

// Sets the queue's cancel word of a running launch through a copy engine on
// stream s (a kernel could not start while the persistent grid holds the SMs).
cudaError_t persist_cancel(void *ws, cudaStream_t s) {
    static const int one = 1;
    cudaError_t e = cudaMemcpyAsync(static_cast<char *>(ws) + offsetof(PersistQueue, cancel), &one, sizeof(int),
                                    cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return e;
}

}  // namespace dil

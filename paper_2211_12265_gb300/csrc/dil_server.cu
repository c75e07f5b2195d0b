// Serving loop: continuous batching of mixed Sign / Verify requests of any
// level and message length over resident keys.
//
// Each of the S stream slots has its own dispatcher thread.  Whenever its slot
// is free and requests are pending it takes them in arrival order, as many as
// the slot's admission limits allow (max_batch requests, msg_capacity message
// bytes; the slot's device buffers are sized once from the memory budget) and,
// under a backlog, about a 1/S share of it, so that the slots split a burst
// instead of one slot taking it all.  It groups them by (operation, level),
// copies their inputs through pinned buffers, launches
// the keyed kernels and copies the results back.  The groups of one batch run
// concurrently on the slot's group streams (forked from and joined into the
// slot's copy stream with events), so a batch takes as long as its slowest
// group rather than the sum.  New requests therefore join as soon as any slot
// frees up, and batches on different slots run concurrently on the device.
// A request's latency runs from its arrival to the moment its result is
// visible to the host.
//
// For comparison the dispatcher can also batch statically: a slot then starts
// only when min_batch requests are pending or the oldest has waited
// max_wait (the plain one-launch-per-batch service).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/dil.h"
#include "dil_launch.h"

namespace {

using Clock = std::chrono::steady_clock;
double now_s() { return std::chrono::duration<double>(Clock::now().time_since_epoch()).count(); }

constexpr int MAX_SIG = 4595;
constexpr size_t POLY = 256 * sizeof(int32_t);
// Scratch polynomials of the largest keyed task (Sign or Verify, any level).
size_t max_task_polys() {
    size_t m = 0;
    for (int level : {2, 3, 5}) m = std::max({m, dil::keyed_sign_polys(level), dil::keyed_verify_polys(level)});
    return m;
}

int level_slot(int level) { return level == 2 ? 0 : level == 3 ? 1 : level == 5 ? 2 : -1; }
size_t sig_bytes(int level) { return level == 2 ? 2420 : level == 3 ? 3293 : 4595; }

struct Req {
    uint64_t id = 0;
    int op = 0, level = 2;
    int32_t key = 0;
    const uint8_t *msg = nullptr;
    size_t mlen = 0;
    const uint8_t *sig_in = nullptr;
    double t_arrive = 0;
    // result destinations
    uint8_t *sig_out = nullptr;
    int32_t *status = nullptr;
    uint8_t *ok = nullptr;
    double *latency = nullptr;
    // owned storage (submit / poll mode)
    std::vector<uint8_t> own_msg, own_sig_in;
    dil_result res;
    bool owned = false;
};

struct Group {
    int op, level, first, count;
    size_t off_first;   // index of the group's first offset in the offset array
    size_t sig_first;   // byte offset of the group's signatures
};

constexpr int MAX_GROUPS = 6;   // (operation, level) pairs

struct Slot {
    cudaStream_t stream = nullptr;          // copies in and out
    cudaStream_t gstream[MAX_GROUPS] = {};  // one per group of a batch
    cudaEvent_t done = nullptr, ev_in = nullptr, ev_grp[MAX_GROUPS] = {};
    bool busy = false;
    bool failed = false;   // a copy, launch or the batch's kernels failed: its requests report DIL_ECUDA
    uint8_t *d_msg = nullptr, *d_sig_in = nullptr, *d_sig_out = nullptr, *d_ok = nullptr;
    uint64_t *d_off = nullptr;
    int32_t *d_key = nullptr, *d_status = nullptr, *d_scratch = nullptr;
    uint8_t *h_msg = nullptr, *h_sig_in = nullptr, *h_sig_out = nullptr, *h_ok = nullptr;
    uint64_t *h_off = nullptr;
    int32_t *h_key = nullptr, *h_status = nullptr;
    std::vector<Req *> reqs;
    std::vector<Group> groups;
    size_t sig_used = 0;
};

}  // namespace

struct dil_server {
    int device = 0;
    int max_batch = 0;
    size_t msg_cap = 0;
    dil_ctx *ctx = nullptr;
    dil_keystore *ks[3] = {nullptr, nullptr, nullptr};
    int nkeys[3] = {0, 0, 0};
    std::vector<Slot> slots;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Req *> pending;
    std::deque<Req *> completed;
    size_t outstanding = 0;   // submitted and not yet completed
    std::vector<std::thread> workers;   // one dispatcher per slot
    bool stop = false;
    uint64_t next_id = 1;
    std::atomic<uint64_t> batches{0}, batched_reqs{0}, launches{0};
    int min_batch = 1;        // static batching: start a slot only with this many pending
    double max_wait_s = 0;    // ... or once the oldest pending request waited this long
    // launch shape per (operation, level): Sign 8 warps per CTA, 4 per task
    // (short per-task latency); Verify 4 warps per CTA, one per task
    int warps[2][3] = {{8, 8, 8}, {4, 4, 4}};
    int wpt[2][3] = {{4, 4, 4}, {1, 1, 1}};
};

namespace {

void free_slot(Slot &s) {
    cudaFree(s.d_msg); cudaFree(s.d_sig_in); cudaFree(s.d_sig_out); cudaFree(s.d_ok);
    cudaFree(s.d_off); cudaFree(s.d_key); cudaFree(s.d_status); cudaFree(s.d_scratch);
    cudaFreeHost(s.h_msg); cudaFreeHost(s.h_sig_in); cudaFreeHost(s.h_sig_out); cudaFreeHost(s.h_ok);
    cudaFreeHost(s.h_off); cudaFreeHost(s.h_key); cudaFreeHost(s.h_status);
    if (s.done) cudaEventDestroy(s.done);
    if (s.ev_in) cudaEventDestroy(s.ev_in);
    for (int g = 0; g < MAX_GROUPS; ++g) {
        if (s.ev_grp[g]) cudaEventDestroy(s.ev_grp[g]);
        if (s.gstream[g]) cudaStreamDestroy(s.gstream[g]);
    }
    if (s.stream) cudaStreamDestroy(s.stream);
    s = Slot();
}

bool alloc_slot(Slot &s, int max_batch, size_t msg_cap) {
    const size_t n = (size_t)max_batch, offs = n + 6;
    bool ok = cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming) == cudaSuccess &&
              cudaEventCreateWithFlags(&s.ev_in, cudaEventDisableTiming) == cudaSuccess &&
              cudaMalloc(&s.d_msg, msg_cap + 16) == cudaSuccess &&
              cudaMalloc(&s.d_sig_in, n * MAX_SIG) == cudaSuccess &&
              cudaMalloc(&s.d_sig_out, n * MAX_SIG) == cudaSuccess && cudaMalloc(&s.d_ok, n) == cudaSuccess &&
              cudaMalloc(&s.d_off, offs * 8) == cudaSuccess && cudaMalloc(&s.d_key, n * 4) == cudaSuccess &&
              cudaMalloc(&s.d_status, n * 4) == cudaSuccess &&
              cudaMalloc(&s.d_scratch, n * max_task_polys() * POLY) == cudaSuccess &&
              cudaMallocHost(&s.h_msg, msg_cap + 16) == cudaSuccess &&
              cudaMallocHost(&s.h_sig_in, n * MAX_SIG) == cudaSuccess &&
              cudaMallocHost(&s.h_sig_out, n * MAX_SIG) == cudaSuccess && cudaMallocHost(&s.h_ok, n) == cudaSuccess &&
              cudaMallocHost(&s.h_off, offs * 8) == cudaSuccess && cudaMallocHost(&s.h_key, n * 4) == cudaSuccess &&
              cudaMallocHost(&s.h_status, n * 4) == cudaSuccess;
    for (int g = 0; ok && g < MAX_GROUPS; ++g)
        ok = cudaStreamCreateWithFlags(&s.gstream[g], cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&s.ev_grp[g], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) cudaGetLastError();
    return ok;
}

size_t slot_device_bytes(int max_batch, size_t msg_cap) {
    const size_t n = (size_t)max_batch;
    return msg_cap + 16 + 2 * n * MAX_SIG + n + (n + 6) * 8 + 8 * n + n * max_task_polys() * POLY;
}

void finish_request(dil_server *sv, Req *r, double t) {
    if (r->latency) *r->latency = t - r->t_arrive;
    r->res.latency_s = t - r->t_arrive;
}

// Starts the next batch on a free slot; returns false when nothing was pending.
bool dispatch(dil_server *sv, Slot &s) {
    s.reqs.clear();
    s.groups.clear();
    int warps[2][3], wpt[2][3];
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        if (sv->pending.empty()) return false;
        if ((int)sv->pending.size() < std::min(sv->min_batch, sv->max_batch) &&
            now_s() - sv->pending.front()->t_arrive < sv->max_wait_s && !sv->stop)
            return false;   // static batching: wait for a fuller batch
        memcpy(warps, sv->warps, sizeof(warps));
        memcpy(wpt, sv->wpt, sizeof(wpt));
        // continuous batching takes about a 1/S share of a backlog (at least 64)
        size_t cap = (size_t)sv->max_batch;
        if (sv->max_wait_s <= 0) {
            const size_t share = (sv->pending.size() + sv->slots.size() - 1) / sv->slots.size();
            cap = std::min(cap, std::max<size_t>(64, share));
        }
        size_t bytes = 0;
        while (!sv->pending.empty() && s.reqs.size() < cap) {
            Req *r = sv->pending.front();
            if (bytes + r->mlen > sv->msg_cap && !s.reqs.empty()) break;   // waits for the next batch
            sv->pending.pop_front();
            bytes += r->mlen;
            s.reqs.push_back(r);
        }
        if (!sv->pending.empty()) sv->cv_work.notify_one();   // another slot may take the rest
    }
    if (s.reqs.empty()) return false;
    nvtxRangePushA("dil_server_batch");   // host side of one batch: staging and launches
    // group by (op, level), stable within a group
    std::stable_sort(s.reqs.begin(), s.reqs.end(), [](const Req *a, const Req *b) {
        return a->op != b->op ? a->op < b->op : a->level < b->level;
    });
    size_t mbytes = 0, noff = 0, sig_off = 0;
    for (int i = 0; i < (int)s.reqs.size();) {
        Group g{s.reqs[i]->op, s.reqs[i]->level, i, 0, noff, sig_off};
        int j = i;
        while (j < (int)s.reqs.size() && s.reqs[j]->op == g.op && s.reqs[j]->level == g.level) {
            Req *r = s.reqs[j];
            const size_t sb = sig_bytes(r->level);
            s.h_key[j] = r->key;
            s.h_off[noff++] = mbytes;
            if (r->mlen) memcpy(s.h_msg + mbytes, r->msg, std::min(r->mlen, sv->msg_cap - mbytes));
            mbytes += std::min(r->mlen, sv->msg_cap - mbytes);
            if (g.op == 1) memcpy(s.h_sig_in + sig_off, r->sig_in, sb);
            sig_off += sb;
            ++j;
        }
        s.h_off[noff++] = mbytes;
        g.count = j - i;
        s.groups.push_back(g);
        i = j;
    }
    s.sig_used = sig_off;
    const size_t n = s.reqs.size();
    cudaStream_t st = s.stream;
    cudaError_t err = cudaSuccess;
    auto check = [&err](cudaError_t e) {
        if (e != cudaSuccess && err == cudaSuccess) err = e;
    };
    check(cudaMemcpyAsync(s.d_key, s.h_key, n * 4, cudaMemcpyHostToDevice, st));
    check(cudaMemcpyAsync(s.d_off, s.h_off, noff * 8, cudaMemcpyHostToDevice, st));
    if (mbytes) check(cudaMemcpyAsync(s.d_msg, s.h_msg, mbytes, cudaMemcpyHostToDevice, st));
    bool any_verify = false;
    for (auto &g : s.groups) any_verify |= g.op == 1;
    if (any_verify) check(cudaMemcpyAsync(s.d_sig_in, s.h_sig_in, sig_off, cudaMemcpyHostToDevice, st));
    check(cudaEventRecord(s.ev_in, st));
    for (size_t gi = 0; gi < s.groups.size(); ++gi) {
        const Group &g = s.groups[gi];
        const int li = level_slot(g.level);
        dil_keystore *ks = sv->ks[li];
        int32_t *scratch = s.d_scratch + (size_t)g.first * max_task_polys() * 256;
        cudaStream_t gs = s.gstream[gi];
        check(cudaStreamWaitEvent(gs, s.ev_in, 0));
        if (g.op == 0) {
            const int l = g.level == 2 ? 4 : g.level == 3 ? 5 : 7;
            check(dil::launch_sign_keyed(g.level, g.count, sv->nkeys[li], s.d_key + g.first, ks->sk, ks->keys, s.d_msg,
                                   s.d_off + g.off_first, s.d_sig_out + g.sig_first, s.d_status + g.first, nullptr,
                                   scratch, (65536 - l) / l + 1, warps[0][li], wpt[0][li], gs));
        } else {
            check(dil::launch_verify_keyed(g.level, g.count, sv->nkeys[li], s.d_key + g.first, ks->pk, ks->keys, ks->tr,
                                     s.d_msg, s.d_off + g.off_first, s.d_sig_in + g.sig_first, s.d_ok + g.first,
                                     scratch, warps[1][li], wpt[1][li], gs));
        }
        check(cudaEventRecord(s.ev_grp[gi], gs));
        check(cudaStreamWaitEvent(st, s.ev_grp[gi], 0));
    }
    check(cudaMemcpyAsync(s.h_sig_out, s.d_sig_out, sig_off, cudaMemcpyDeviceToHost, st));
    check(cudaMemcpyAsync(s.h_status, s.d_status, n * 4, cudaMemcpyDeviceToHost, st));
    check(cudaMemcpyAsync(s.h_ok, s.d_ok, n, cudaMemcpyDeviceToHost, st));
    check(cudaEventRecord(s.done, st));
    s.failed = err != cudaSuccess;
    s.busy = true;
    nvtxRangePop();
    sv->batches++;
    sv->launches += s.groups.size();
    sv->batched_reqs += n;
    return true;
}

void complete(dil_server *sv, Slot &s) {
    const double t = now_s();
    for (auto &g : s.groups) {
        size_t so = g.sig_first;
        for (int i = g.first; i < g.first + g.count; ++i) {
            Req *r = s.reqs[i];
            const size_t sb = sig_bytes(r->level);
            r->res.status = 0;
            r->res.ok = 0;
            if (s.failed) {
                r->res.status = DIL_ECUDA;
                if (g.op == 0 && r->status) *r->status = DIL_ECUDA;
                if (g.op == 1 && r->ok) *r->ok = 0;
            } else if (g.op == 0) {
                r->res.status = s.h_status[i];
                if (r->status) *r->status = s.h_status[i];
                if (r->sig_out) memcpy(r->sig_out, s.h_sig_out + so, sb);
                if (r->owned) memcpy(r->res.sig, s.h_sig_out + so, sb);
            } else {
                r->res.ok = s.h_ok[i];
                if (r->ok) *r->ok = s.h_ok[i];
            }
            so += sb;
            finish_request(sv, r, t);
        }
    }
    s.busy = false;
    std::lock_guard<std::mutex> lk(sv->mu);
    for (Req *r : s.reqs) {
        if (r->owned)
            sv->completed.push_back(r);
        else
            delete r;
        sv->outstanding--;
    }
    s.reqs.clear();
    sv->cv_done.notify_all();
}

// Dispatcher of one slot: takes a batch, stages and launches it, waits for
// its completion event and hands the results back; slots run in parallel, so
// one slot's host-side copies do not hold up another's next batch.
void slot_loop(dil_server *sv, Slot *s) {
    cudaSetDevice(sv->device);
    for (;;) {
        if (dispatch(sv, *s)) {
            cudaError_t q;
            while ((q = cudaEventQuery(s->done)) == cudaErrorNotReady)
                std::this_thread::sleep_for(std::chrono::microseconds(5));
            if (q != cudaSuccess) s->failed = true;
            complete(sv, *s);
            continue;
        }
        std::unique_lock<std::mutex> lk(sv->mu);
        if (sv->stop && sv->pending.empty()) return;
        if (sv->pending.empty()) {
            sv->cv_work.wait_for(lk, std::chrono::milliseconds(5), [&] { return sv->stop || !sv->pending.empty(); });
        } else {   // a static batch filling up
            lk.unlock();
            std::this_thread::sleep_for(std::chrono::microseconds(20));
        }
    }
}

void enqueue(dil_server *sv, std::vector<Req *> &batch) {
    std::lock_guard<std::mutex> lk(sv->mu);
    for (Req *r : batch) sv->pending.push_back(r);
    sv->outstanding += batch.size();
    batch.clear();
    sv->cv_work.notify_one();
}

}  // namespace

extern "C" {

int dil_server_create(int device, size_t memory_budget, int streams, int max_batch, dil_server **out) {
    if (!out || streams < 1 || streams > 16 || max_batch < 1) return DIL_EINVAL;
    *out = nullptr;
    dil_server *sv = new dil_server;
    sv->device = device;
    int rc = dil_ctx_create(device, 0, &sv->ctx);
    if (rc) {
        delete sv;
        return rc;
    }
    cudaSetDevice(device);
    const size_t budget = memory_budget ? memory_budget : ((size_t)4 << 30);
    // admission limits from the budget: shrink the batch until S slots fit
    size_t msg_cap = (size_t)max_batch * 4096;
    while (max_batch > 1 && (size_t)streams * slot_device_bytes(max_batch, msg_cap) > budget) {
        max_batch /= 2;
        msg_cap = (size_t)max_batch * 4096;
    }
    if ((size_t)streams * slot_device_bytes(max_batch, msg_cap) > budget) {
        dil_ctx_destroy(sv->ctx);
        delete sv;
        return DIL_ENOMEM;
    }
    if (msg_cap < 16384) msg_cap = 16384;   // any single message fits a batch of its own
    sv->max_batch = max_batch;
    sv->msg_cap = msg_cap;
    sv->slots.resize(streams);
    for (auto &s : sv->slots) {
        if (!alloc_slot(s, max_batch, msg_cap)) {
            for (auto &t : sv->slots) free_slot(t);
            dil_ctx_destroy(sv->ctx);
            delete sv;
            return DIL_ENOMEM;
        }
    }
    for (auto &s : sv->slots) sv->workers.emplace_back(slot_loop, sv, &s);
    *out = sv;
    return DIL_OK;
}

int dil_server_destroy(dil_server *sv) {
    if (!sv) return DIL_OK;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
        sv->cv_work.notify_all();
    }
    for (auto &w : sv->workers)
        if (w.joinable()) w.join();
    cudaSetDevice(sv->device);
    cudaDeviceSynchronize();
    for (auto &s : sv->slots) free_slot(s);
    for (auto &r : sv->completed) delete r;
    for (int i = 0; i < 3; ++i) dil_keystore_destroy(sv->ks[i]);
    dil_ctx_destroy(sv->ctx);
    delete sv;
    return DIL_OK;
}

int dil_server_limits(const dil_server *sv, int *max_batch, size_t *msg_capacity) {
    if (!sv) return DIL_EINVAL;
    if (max_batch) *max_batch = sv->max_batch;
    if (msg_capacity) *msg_capacity = sv->msg_cap;
    return DIL_OK;
}

int dil_server_set_batching(dil_server *sv, int min_batch, double max_wait_s) {
    if (!sv || min_batch < 1 || !(max_wait_s >= 0)) return DIL_EINVAL;
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->min_batch = min_batch;
    sv->max_wait_s = max_wait_s;
    return DIL_OK;
}

int dil_server_set_tuning(dil_server *sv, int op, int level, int warps_per_cta, int warps_per_task) {
    const int li = level_slot(level);
    if (!sv || (op != 0 && op != 1) || li < 0 || warps_per_cta < 1 || warps_per_cta > 8) return DIL_EINVAL;
    if (warps_per_task != 1 && warps_per_task != 2 && warps_per_task != 4) return DIL_EINVAL;
    if (warps_per_cta % warps_per_task) return DIL_EINVAL;
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->warps[op][li] = warps_per_cta;
    sv->wpt[op][li] = warps_per_task;
    return DIL_OK;
}

int dil_server_add_keys(dil_server *sv, int level, size_t n, const uint8_t *pk, const uint8_t *sk) {
    const int li = level_slot(level);
    if (!sv || li < 0 || n == 0 || n > (size_t)INT32_MAX || !pk || !sk) return DIL_EINVAL;
    std::lock_guard<std::mutex> lk(sv->mu);
    if (sv->outstanding) return DIL_EINVAL;   // keys change only while idle
    size_t pkb, skb, sigb;
    dil_sizes(level, &pkb, &skb, &sigb);
    cudaSetDevice(sv->device);
    uint8_t *dpk = nullptr, *dsk = nullptr;
    if (cudaMalloc(&dpk, pkb * n) != cudaSuccess || cudaMalloc(&dsk, skb * n) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(dpk);
        return DIL_ENOMEM;
    }
    int rc = DIL_OK;
    if (cudaMemcpy(dpk, pk, pkb * n, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(dsk, sk, skb * n, cudaMemcpyHostToDevice) != cudaSuccess)
        rc = DIL_ECUDA;
    dil_keystore *ks = nullptr;
    if (!rc) rc = dil_keystore_create(sv->ctx, level, n, dpk, dsk, &ks, nullptr);
    if (!rc && cudaDeviceSynchronize() != cudaSuccess) rc = DIL_ECUDA;
    cudaFree(dpk);
    cudaFree(dsk);
    if (rc) {
        dil_keystore_destroy(ks);
        return rc;
    }
    dil_keystore_destroy(sv->ks[li]);
    sv->ks[li] = ks;
    sv->nkeys[li] = (int)n;
    return DIL_OK;
}

int dil_server_submit(dil_server *sv, int op, int level, int32_t key, const uint8_t *msg, size_t mlen,
                      const uint8_t *sig, uint64_t *id) {
    const int li = level_slot(level);
    if (!sv || li < 0 || (op != 0 && op != 1) || !sv->ks[li] || (mlen && !msg) || (op == 1 && !sig)) return DIL_EINVAL;
    if (mlen > sv->msg_cap) return DIL_EINVAL;
    Req *r = new Req;
    r->owned = true;
    r->op = op;
    r->level = level;
    r->key = key;
    r->own_msg.assign(msg, msg + mlen);
    r->msg = r->own_msg.data();
    r->mlen = mlen;
    if (op == 1) {
        r->own_sig_in.assign(sig, sig + sig_bytes(level));
        r->sig_in = r->own_sig_in.data();
    }
    memset(&r->res, 0, sizeof(r->res));
    r->t_arrive = now_s();
    std::vector<Req *> b{r};
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        r->id = sv->next_id++;
        r->res.id = r->id;
        r->res.op = op;
        r->res.level = level;
    }
    if (id) *id = r->id;
    enqueue(sv, b);
    return DIL_OK;
}

int dil_server_cancel(dil_server *sv, uint64_t id) {
    if (!sv) return DIL_EINVAL;
    std::lock_guard<std::mutex> lk(sv->mu);
    for (auto it = sv->pending.begin(); it != sv->pending.end(); ++it) {
        Req *r = *it;
        if (r->id != id || !r->owned) continue;
        sv->pending.erase(it);
        r->res.status = DIL_ECANCELED;
        r->res.ok = 0;
        r->res.latency_s = now_s() - r->t_arrive;
        sv->completed.push_back(r);
        sv->outstanding--;
        sv->cv_done.notify_all();
        return DIL_OK;
    }
    return DIL_EINVAL;   // unknown, already dispatched or completed
}

int dil_server_poll(dil_server *sv, dil_result *out, size_t max_n, size_t *n_out, int wait_us) {
    if (!sv || !out || !n_out) return DIL_EINVAL;
    std::unique_lock<std::mutex> lk(sv->mu);
    if (sv->completed.empty() && wait_us > 0)
        sv->cv_done.wait_for(lk, std::chrono::microseconds(wait_us), [&] { return !sv->completed.empty(); });
    size_t k = 0;
    while (k < max_n && !sv->completed.empty()) {
        Req *r = sv->completed.front();
        sv->completed.pop_front();
        out[k++] = r->res;
        delete r;
    }
    *n_out = k;
    return DIL_OK;
}

int dil_server_replay(dil_server *sv, size_t n, const double *arrival_s, const int32_t *op, const int32_t *level,
                      const int32_t *key, const uint8_t *msg, const uint64_t *msg_off, const uint8_t *sig_in,
                      uint8_t *sig_out, int32_t *status, uint8_t *ok, double *latency_s, double *wall_s) {
    if (!sv || !arrival_s || !op || !level || !key || !msg_off || !latency_s) return DIL_EINVAL;
    for (size_t i = 0; i < n; ++i) {
        const int li = level_slot(level[i]);
        if (li < 0 || !sv->ks[li] || (op[i] != 0 && op[i] != 1)) return DIL_EINVAL;
        if (op[i] == 1 && !sig_in) return DIL_EINVAL;
        if (op[i] == 0 && (!sig_out || !status)) return DIL_EINVAL;
        if (op[i] == 1 && !ok) return DIL_EINVAL;
        if (msg_off[i + 1] - msg_off[i] > sv->msg_cap) return DIL_EINVAL;
    }
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        if (sv->outstanding) return DIL_EINVAL;
    }
    const double t0 = now_s();
    std::vector<Req *> batch;
    size_t i = 0;
    while (i < n) {
        const double t = now_s() - t0;
        while (i < n && arrival_s[i] <= t) {
            Req *r = new Req;
            r->op = op[i];
            r->level = level[i];
            r->key = key[i];
            r->msg = msg + msg_off[i];
            r->mlen = (size_t)(msg_off[i + 1] - msg_off[i]);
            r->sig_in = sig_in ? sig_in + i * MAX_SIG : nullptr;
            r->sig_out = sig_out ? sig_out + i * MAX_SIG : nullptr;
            r->status = status ? status + i : nullptr;
            r->ok = ok ? ok + i : nullptr;
            r->latency = latency_s + i;
            r->t_arrive = t0 + arrival_s[i];
            batch.push_back(r);
            ++i;
        }
        if (!batch.empty()) enqueue(sv, batch);
        if (i < n) {
            const double wait = arrival_s[i] - (now_s() - t0);
            if (wait > 200e-6) std::this_thread::sleep_for(std::chrono::microseconds((int64_t)((wait - 100e-6) * 1e6)));
        }
    }
    std::unique_lock<std::mutex> lk(sv->mu);
    sv->cv_done.wait(lk, [&] { return sv->outstanding == 0; });
    if (wall_s) *wall_s = now_s() - t0;
    return DIL_OK;
}

int dil_server_stats(const dil_server *sv, uint64_t *batches, uint64_t *requests, uint64_t *launches) {
    if (!sv) return DIL_EINVAL;
    if (batches) *batches = sv->batches;
    if (requests) *requests = sv->batched_reqs;
    if (launches) *launches = sv->launches;
    return DIL_OK;
}

}  // extern "C"

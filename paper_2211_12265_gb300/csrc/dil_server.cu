// Serving loop: continuous batching of mixed Sign / Verify requests of any
// level and message length over resident keys.
//
// Continuous batching (the default policy) runs on the device: a ring thread
// takes pending requests in arrival order as long as the request ring and the
// message arena (both sized from the memory budget) have room, copies their
// descriptors and bytes into the device ring through pinned staging buffers
// and then publishes their ticket count, all on one copy stream; the serving
// kernel (dil_serve.cu: resident one-warp workers, Sign helpers, results in
// mapped host memory) picks them up while it runs, and the same thread polls
// the completion ring and hands the results back.  It launches the kernel
// when requests are outstanding and no launch is running (the kernel exits
// by itself after a few idle milliseconds).  A request's latency runs from
// its arrival to the moment its result is visible to the host.
//
// Static batching, kept as the baseline (the plain one-launch-per-batch
// service), uses stream slots.  Each of the S slots has its own dispatcher
// thread.  Whenever its slot
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
// A slot starts only when min_batch requests are pending or the oldest has
// waited max_wait.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <functional>
#include <memory>
#include <mutex>
#include <thread>
#include <utility>
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
    // the outcome (every request)
    int32_t st = 0;
    uint8_t okv = 0;
    double lat = 0;
    // owned storage and the result handed to dil_server_poll (submit / poll mode)
    std::vector<uint8_t> own_msg, own_sig_in;
    std::unique_ptr<dil_result> res;
    bool owned = false;
    bool pooled = false;   // part of a replay's request array: not deleted on completion
};

// A few host threads that share the per-request copies of the ring thread
// (staging request bytes, copying results out): run(n, fn) calls fn(i) for
// every i in [0, n), the calling thread taking a share, and returns when all
// calls have returned.
class CopyPool {
public:
    explicit CopyPool(int helpers) {
        for (int h = 0; h < helpers; ++h) threads_.emplace_back([this, h] { loop(h); });
    }
    ~CopyPool() {
        {
            std::lock_guard<std::mutex> lk(mu_);
            quit_ = true;
        }
        cv_.notify_all();
        for (auto &t : threads_) t.join();
    }
    template <class F>
    void run(size_t n, F &&fn) {
        const size_t parts = threads_.size() + 1;
        if (n < 64 || threads_.empty()) {
            for (size_t i = 0; i < n; ++i) fn(i);
            return;
        }
        std::function<void(size_t)> f = fn;
        {
            std::lock_guard<std::mutex> lk(mu_);
            job_ = &f;
            n_ = n;
            parts_ = parts;
            pending_ = threads_.size();
            ++gen_;
        }
        cv_.notify_all();
        for (size_t i = part_lo(0); i < part_lo(1); ++i) f(i);
        std::unique_lock<std::mutex> lk(mu_);
        done_cv_.wait(lk, [&] { return pending_ == 0; });
        job_ = nullptr;
    }

private:
    size_t part_lo(size_t p) const { return n_ * p / parts_; }
    void loop(int h) {
        uint64_t seen = 0;
        for (;;) {
            std::function<void(size_t)> *job;
            size_t lo, hi;
            {
                std::unique_lock<std::mutex> lk(mu_);
                cv_.wait(lk, [&] { return quit_ || gen_ != seen; });
                if (quit_) return;
                seen = gen_;
                job = job_;
                lo = part_lo(h + 1);
                hi = part_lo(h + 2);
            }
            for (size_t i = lo; i < hi; ++i) (*job)(i);
            std::lock_guard<std::mutex> lk(mu_);
            if (--pending_ == 0) done_cv_.notify_one();
        }
    }
    std::vector<std::thread> threads_;
    std::mutex mu_;
    std::condition_variable cv_, done_cv_;
    std::function<void(size_t)> *job_ = nullptr;
    size_t n_ = 0, parts_ = 1, pending_ = 0;
    uint64_t gen_ = 0;
    bool quit_ = false;
};
constexpr int RING_COPY_HELPERS = 6;   // per pool (two pools: staging and results)

// Device request ring of the continuous policy (see the file comment).
// Tickets count published requests (unsigned, wrapping); ticket t uses ring
// slot t mod R.  Arena positions are monotone byte counts, the physical
// offset is the position mod the arena size; a request's bytes never wrap.
struct Ring {
    int R = 0;                      // ring slots (power of two)
    size_t arena = 0;               // arena bytes
    int grid = 0, workers = 0;
    dil::ServeCtl *d_ctl = nullptr;
    dil::ServeReq *d_req = nullptr;
    uint8_t *d_arena = nullptr;
    dil::ServeTask *d_tasks = nullptr;
    int *d_worker_ticket = nullptr;
    int32_t *d_scratch = nullptr;
    uint8_t *d_sig_stage = nullptr;     // per worker: a signature packed before it goes to mapped memory
    dil::ServeFifo *d_fifo = nullptr;   // forwarding queues by request type
    unsigned long long *d_fifo_ring = nullptr;
    uint8_t *d_mu = nullptr;                 // R x 64: mu precomputed by the hasher warps
    unsigned long long *d_mu_tag = nullptr;  // R: which ticket's mu a slot holds
    unsigned long long *h_fifo_init = nullptr;   // pinned: the queues' entries as every launch starts them
    int sms = 0;
    double type_work[dil::SERVE_TYPES] = {};    // recent warp time per request type (publisher), for the SM shares
    dil::ServeReq *h_req = nullptr;     // pinned staging of the descriptors
    uint8_t *h_arena = nullptr;         // pinned staging of the arena
    unsigned *h_words = nullptr;        // pinned sources of the tail / stop copies
    uint8_t *m_sig = nullptr;           // mapped results
    int32_t *m_status = nullptr, *m_iters = nullptr;
    uint8_t *m_ok = nullptr;
    unsigned long long *m_comp = nullptr;
    cudaStream_t kstream = nullptr, cstream = nullptr;
    cudaEvent_t kdone = nullptr, ev_pub = nullptr, ev_words[2] = {nullptr, nullptr};
    bool launched = false;
    bool stop_set = false;                  // the device stop word holds 1
    std::atomic<bool> broken{false};        // a launch or copy failed: requests complete with DIL_ECUDA
    // The publisher thread takes tickets and arena room; the completer thread
    // frees them in ticket order.
    std::atomic<unsigned> next_ticket{0};   // published (publisher)
    std::atomic<unsigned> oldest{0};        // oldest ticket whose slot is not yet free (completer)
    std::atomic<unsigned> consumed{0};      // completions consumed (completer)
    unsigned comp_seen = 0;                 // completer's copy of `consumed`
    uint64_t apos = 0;                      // arena: next free position (publisher)
    std::atomic<uint64_t> atail{0};         // arena: oldest position in use (completer)
    uint64_t words_used = 0;                // h_words entries issued (under kmu)
    std::unique_ptr<std::atomic<Req *>[]> slot_req;
    std::unique_ptr<std::atomic<uint64_t>[]> slot_aend;
    std::vector<uint8_t> slot_done;         // completer only
    std::atomic<uint64_t> batches{0}, launches{0};
    std::recursive_mutex kmu;               // launches, halts and the word copies (publisher and API calls)
    std::unique_ptr<CopyPool> pool_in, pool_out;   // staging (publisher), results (completer)
    std::thread completer;
    std::atomic<bool> quit{false};
    unsigned in_flight() const { return next_ticket.load() - oldest.load(std::memory_order_acquire); }
};
constexpr unsigned RING_WORDS = 4096;   // h_words entries (two halves, reused after an event)
// Largest publication: the first requests of a burst reach the device while
// the host stages the rest.
constexpr size_t RING_CHUNK = 1024, RING_CHUNK_BYTES = (size_t)4 << 20;
constexpr size_t RING_ARENA_MAX = (size_t)1 << 30;   // message arena, bytes
constexpr size_t RING_SLOTS_MAX = (size_t)1 << 17;   // R: request slots, mapped result slots
constexpr double RING_IDLE_STOP_S = 0.002;   // the host stops a kernel idle this long
constexpr int RING_FIFO_PER_SM = 16;          // forwarding stops while a queue holds this many per home SM
// Sign helpers: SERVE_SPEC per unfinished Sign while fewer than
// SERVE_HELP_BELOW_PCT percent of the workers serve a request of their own,
// none above.  Helping shortens a Sign, but a helper finishes its claimed
// repetitions before it starts its own request, and under load its
// repetitions take issue slots from the requests on its SM.  On the serving
// mix: p99 1.8 ms at half load against 5.7 ms with helpers up to 80% busy,
// and 4.3 M ops/s saturated against 4.07 M without helpers.
// SMs whose warps hash mu = H(tr || M) while requests queue (the serving
// kernel's mu hashers): on the serving mix, 4.33-4.38 M ops/s saturated
// without them, 4.55-4.65 M with 6-12 such SMs, p99 unchanged at quarter and
// half load and 3-6% lower at 75% load.
constexpr int RING_HASH_SMS = 12;
constexpr int SERVE_SPEC = 4;
constexpr int SERVE_HELP_BELOW_PCT = 10;
// Warp time of one request by type in microseconds (GB300, 32 of 32 warps per
// SM busy: Sign 2 / 3 / 5, Verify 2 / 3 / 5), plus the hash of its message.
constexpr double RING_TYPE_US[dil::SERVE_TYPES] = {720, 1030, 1110, 80, 94, 122};
constexpr double RING_MSG_US_PER_BYTE = 0.05;

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
    Ring ring;                          // continuous policy: device ring and serving kernel
    std::thread ring_thread;
    std::condition_variable cv_ring;
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
    r->lat = t - r->t_arrive;
}

// Starts the next batch on a free slot; returns false when nothing was pending.
bool dispatch(dil_server *sv, Slot &s) {
    s.reqs.clear();
    s.groups.clear();
    int warps[2][3], wpt[2][3];
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        if (sv->pending.empty() || sv->max_wait_s <= 0) return false;   // continuous: the ring serves
        if ((int)sv->pending.size() < std::min(sv->min_batch, sv->max_batch) &&
            now_s() - sv->pending.front()->t_arrive < sv->max_wait_s && !sv->stop)
            return false;   // static batching: wait for a fuller batch
        memcpy(warps, sv->warps, sizeof(warps));
        memcpy(wpt, sv->wpt, sizeof(wpt));
        const size_t cap = (size_t)sv->max_batch;
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
            r->st = 0;
            r->okv = 0;
            if (s.failed) {
                r->st = DIL_ECUDA;
                if (g.op == 0 && r->status) *r->status = DIL_ECUDA;
                if (g.op == 1 && r->ok) *r->ok = 0;
            } else if (g.op == 0) {
                r->st = s.h_status[i];
                if (r->status) *r->status = s.h_status[i];
                if (r->sig_out) memcpy(r->sig_out, s.h_sig_out + so, sb);
                if (r->owned) memcpy(r->res->sig, s.h_sig_out + so, sb);
            } else {
                r->okv = s.h_ok[i];
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
        else if (!r->pooled)
            delete r;
        sv->outstanding--;
    }
    s.reqs.clear();
    sv->cv_done.notify_all();
}

// ---------------------------------------------------------------- device ring (continuous policy)

size_t pow2_floor(size_t x) {
    size_t p = 1;
    while (p * 2 <= x) p *= 2;
    return p;
}

void ring_free(Ring &g) {
    if (g.kstream) cudaStreamSynchronize(g.kstream);
    if (g.cstream) cudaStreamSynchronize(g.cstream);
    cudaFree(g.d_ctl); cudaFree(g.d_req); cudaFree(g.d_arena); cudaFree(g.d_tasks);
    cudaFree(g.d_worker_ticket); cudaFree(g.d_scratch); cudaFree(g.d_sig_stage);
    cudaFree(g.d_fifo); cudaFree(g.d_fifo_ring); cudaFreeHost(g.h_fifo_init);
    cudaFree(g.d_mu); cudaFree(g.d_mu_tag);
    cudaFreeHost(g.h_req); cudaFreeHost(g.h_arena); cudaFreeHost(g.h_words);
    cudaFreeHost(g.m_sig); cudaFreeHost(g.m_status); cudaFreeHost(g.m_iters); cudaFreeHost(g.m_ok);
    cudaFreeHost(g.m_comp);
    for (cudaEvent_t e : {g.kdone, g.ev_pub, g.ev_words[0], g.ev_words[1]})
        if (e) cudaEventDestroy(e);
    if (g.kstream) cudaStreamDestroy(g.kstream);
    if (g.cstream) cudaStreamDestroy(g.cstream);
    g.d_ctl = nullptr;
    g.R = 0;
    g.pool_in.reset();
    g.pool_out.reset();
}

// Sizes the ring from its share of the memory budget: the arena takes a
// quarter (at most RING_ARENA_MAX, at least two of the largest requests), the
// descriptors and records an eighth at most, the workers' scratch the rest.
//
// Tickets are published in order and a slot (and its arena bytes) frees only
// when every older request has completed, so one long Sign holds back
// publishing once R tickets or `arena` bytes lie beyond it.  A Sign with 30
// repetitions runs about 20 ms under full load, some 80,000 requests at the
// saturated rate: the ring gets a slot per 2 KB of arena (the serving mix's
// requests take 2.6 KB of message and, for Verify, a signature), up to
// RING_SLOTS_MAX.
bool ring_alloc(Ring &g, int device, size_t budget, size_t msg_cap) {
    const size_t big = msg_cap + MAX_SIG + 64;
    size_t arena = std::min<size_t>(budget / 4, RING_ARENA_MAX);
    arena = std::max(arena, 2 * big);
    arena = (arena + 4095) & ~(size_t)4095;
    size_t R = std::min<size_t>(budget / 8 / (sizeof(dil::ServeReq) + sizeof(dil::ServeTask)), arena / 2048);
    R = std::min<size_t>(pow2_floor(std::max<size_t>(R, 64)), RING_SLOTS_MAX);
    const size_t per_worker = dil::serve_worker_polys() * POLY;
    const size_t used = arena + R * (sizeof(dil::ServeReq) + sizeof(dil::ServeTask));
    const size_t left = budget > used ? budget - used : 0;
    int max_workers = (int)std::min<size_t>(left / per_worker, 1 << 20);
    if (max_workers < 8) max_workers = 8;
    if (dil::serve_grid(device, max_workers, g.grid, g.workers) != cudaSuccess) return false;
    g.R = (int)R;
    g.arena = arena;
    bool ok = cudaStreamCreateWithFlags(&g.kstream, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamCreateWithFlags(&g.cstream, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&g.kdone, cudaEventDisableTiming) == cudaSuccess &&
              cudaEventCreateWithFlags(&g.ev_pub, cudaEventDisableTiming) == cudaSuccess &&
              cudaEventCreateWithFlags(&g.ev_words[0], cudaEventDisableTiming) == cudaSuccess &&
              cudaEventCreateWithFlags(&g.ev_words[1], cudaEventDisableTiming) == cudaSuccess &&
              cudaMalloc(&g.d_ctl, sizeof(dil::ServeCtl)) == cudaSuccess &&
              cudaMalloc(&g.d_req, R * sizeof(dil::ServeReq)) == cudaSuccess &&
              cudaMalloc(&g.d_arena, arena) == cudaSuccess &&
              cudaMalloc(&g.d_tasks, R * sizeof(dil::ServeTask)) == cudaSuccess &&
              cudaMalloc(&g.d_worker_ticket, (size_t)g.workers * sizeof(int)) == cudaSuccess &&
              cudaMalloc(&g.d_scratch, (size_t)g.workers * per_worker) == cudaSuccess &&
              cudaMalloc(&g.d_sig_stage, (size_t)g.workers * dil::SERVE_SIG_STRIDE) == cudaSuccess &&
              cudaMalloc(&g.d_fifo, dil::SERVE_TYPES * sizeof(dil::ServeFifo)) == cudaSuccess &&
              cudaMalloc(&g.d_fifo_ring, dil::SERVE_TYPES * R * sizeof(unsigned long long)) == cudaSuccess &&
              cudaMalloc(&g.d_mu, R * 64) == cudaSuccess &&
              cudaMalloc(&g.d_mu_tag, R * sizeof(unsigned long long)) == cudaSuccess &&
              cudaMallocHost(&g.h_fifo_init, dil::SERVE_TYPES * R * sizeof(unsigned long long)) == cudaSuccess &&
              cudaMallocHost(&g.h_req, R * sizeof(dil::ServeReq)) == cudaSuccess &&
              cudaMallocHost(&g.h_arena, arena) == cudaSuccess &&
              cudaMallocHost(&g.h_words, RING_WORDS * sizeof(unsigned)) == cudaSuccess &&
              cudaHostAlloc(&g.m_sig, R * dil::SERVE_SIG_STRIDE, cudaHostAllocMapped) == cudaSuccess &&
              cudaHostAlloc(&g.m_status, R * sizeof(int32_t), cudaHostAllocMapped) == cudaSuccess &&
              cudaHostAlloc(&g.m_iters, R * sizeof(int32_t), cudaHostAllocMapped) == cudaSuccess &&
              cudaHostAlloc(&g.m_ok, R, cudaHostAllocMapped) == cudaSuccess &&
              cudaHostAlloc(&g.m_comp, R * sizeof(unsigned long long), cudaHostAllocMapped) == cudaSuccess;
    if (ok) {
        ok = cudaMemset(g.d_ctl, 0, sizeof(dil::ServeCtl)) == cudaSuccess &&
             cudaMemset(g.d_worker_ticket, 0xFF, (size_t)g.workers * sizeof(int)) == cudaSuccess &&
             cudaMemset(g.d_tasks, 0, R * sizeof(dil::ServeTask)) == cudaSuccess &&
             cudaMemset(g.d_mu_tag, 0, R * sizeof(unsigned long long)) == cudaSuccess;
        // completion entry i first expects completion number i: start every
        // entry at a number it cannot hold then
        for (size_t i = 0; ok && i < R; ++i) g.m_comp[i] = (unsigned long long)(unsigned)(i - R) << 32;
        // forwarding entry i is free for the push at position i
        for (size_t ty = 0; ok && ty < (size_t)dil::SERVE_TYPES; ++ty)
            for (size_t i = 0; i < R; ++i) g.h_fifo_init[ty * R + i] = (unsigned long long)i << 32;
        ok = ok && cudaDeviceGetAttribute(&g.sms, cudaDevAttrMultiProcessorCount, device) == cudaSuccess;
    }
    if (!ok) {
        cudaGetLastError();
        ring_free(g);
        return false;
    }
    g.slot_req.reset(new std::atomic<Req *>[R]);
    g.slot_aend.reset(new std::atomic<uint64_t>[R]);
    for (size_t i = 0; i < R; ++i) {
        g.slot_req[i].store(nullptr);
        g.slot_aend[i].store(0);
    }
    g.slot_done.assign(R, 0);
    g.pool_in.reset(new CopyPool(RING_COPY_HELPERS));
    g.pool_out.reset(new CopyPool(RING_COPY_HELPERS));
    return true;
}

// Copies a 32-bit word from the pinned word ring to device address dst on
// the copy stream (the sources are reused in halves, each after the copies
// that read it have run).
bool ring_copy_word(Ring &g, unsigned *dst, unsigned value) {
    std::lock_guard<std::recursive_mutex> lk(g.kmu);
    const uint64_t i = g.words_used++;
    const unsigned half = (unsigned)(i / (RING_WORDS / 2)) & 1u;
    if (i % (RING_WORDS / 2) == 0 && i >= RING_WORDS) cudaEventSynchronize(g.ev_words[half]);
    unsigned *src = g.h_words + (i % RING_WORDS);
    *src = value;
    bool ok = cudaMemcpyAsync(dst, src, sizeof(unsigned), cudaMemcpyHostToDevice, g.cstream) == cudaSuccess;
    if (i % (RING_WORDS / 2) == RING_WORDS / 2 - 1) ok = ok && cudaEventRecord(g.ev_words[half], g.cstream) == cudaSuccess;
    return ok;
}

bool kernel_running(Ring &g) { return g.launched && cudaEventQuery(g.kdone) == cudaErrorNotReady; }

size_t ring_poll(dil_server *sv, bool fail_all = false);

// Home request type of each SM, in proportion to the recent warp time of each
// type (largest remainders; a type with work gets at least one SM); no
// recent work: every SM serves every type.  The history halves per launch.
void assign_home_types(Ring &g, dil::ServeArgs &a) {
    for (int s = 0; s < dil::SERVE_MAX_SMS; ++s) a.sm_type[s] = dil::SERVE_TYPE_ANY;
    for (int ty = 0; ty < dil::SERVE_TYPES; ++ty) a.type_sms[ty] = 0;
    double total = 0;
    for (double w : g.type_work) total += w;
    const int first = a.hash_sms;   // SMs before it only hash
    const int sms = std::min(g.sms, dil::SERVE_MAX_SMS) - first;
    int active_types = 0;
    for (double w : g.type_work) active_types += w > 0;
    if (total <= 0 || sms < active_types) return;
    int given = 0;
    double rem[dil::SERVE_TYPES];
    for (int ty = 0; ty < dil::SERVE_TYPES; ++ty) {
        const double share = g.type_work[ty] / total * sms;
        a.type_sms[ty] = g.type_work[ty] > 0 ? std::max(1, (int)share) : 0;
        rem[ty] = share - a.type_sms[ty];
        given += a.type_sms[ty];
    }
    while (given < sms) {   // largest remainders
        int best = -1;
        for (int ty = 0; ty < dil::SERVE_TYPES; ++ty)
            if (g.type_work[ty] > 0 && (best < 0 || rem[ty] > rem[best])) best = ty;
        a.type_sms[best]++;
        rem[best] -= 1;
        ++given;
    }
    while (given > sms) {   // the at-least-one rule overshot: take from the largest
        int big = 0;
        for (int ty = 1; ty < dil::SERVE_TYPES; ++ty)
            if (a.type_sms[ty] > a.type_sms[big]) big = ty;
        a.type_sms[big]--;
        --given;
    }
    int s = first;
    for (int ty = 0; ty < dil::SERVE_TYPES; ++ty)
        for (int k = 0; k < a.type_sms[ty]; ++k) a.sm_type[s++] = (uint8_t)ty;
    for (double &w : g.type_work) w *= 0.5;
}

// Launches the serving kernel on the resident keys (after the copies issued
// so far).  The previous launch has exited: every ticket it served is
// complete and the ones its workers took unpublished were abandoned, so the
// ticket counter restarts at the oldest uncompleted ticket.
bool ring_launch(dil_server *sv) {
    Ring &g = sv->ring;
    std::lock_guard<std::recursive_mutex> lk(g.kmu);
    if (g.launched) {   // the previous launch has finished: wait until its completions are consumed
        unsigned issued = 0;
        if (cudaMemcpy(&issued, &g.d_ctl->comp, sizeof(unsigned), cudaMemcpyDeviceToHost) != cudaSuccess) return false;
        for (long spin = 0; g.consumed.load(std::memory_order_acquire) != issued; ++spin) {
            if (spin > (1l << 26)) return false;   // the completer stopped consuming
            std::this_thread::yield();
        }
    }
    if (!ring_copy_word(g, reinterpret_cast<unsigned *>(&g.d_ctl->head), g.oldest.load(std::memory_order_acquire)) ||
        !ring_copy_word(g, reinterpret_cast<unsigned *>(&g.d_ctl->hhead), g.oldest.load(std::memory_order_acquire)))
        return false;
    if (g.stop_set) {
        if (!ring_copy_word(g, reinterpret_cast<unsigned *>(&g.d_ctl->stop), 0)) return false;
        g.stop_set = false;
    }
    dil::ServeArgs a{};
    a.ctl = g.d_ctl;
    a.req = g.d_req;
    a.arena = g.d_arena;
    a.tasks = g.d_tasks;
    a.worker_ticket = g.d_worker_ticket;
    a.scratch = g.d_scratch;
    a.sig_stage = g.d_sig_stage;
    a.worker_polys = (int)dil::serve_worker_polys();
    a.ring = g.R;
    for (int li = 0; li < 3; ++li) {
        const dil_keystore *ks = sv->ks[li];
        a.keys[li] = ks ? dil::ServeKeys{ks->sk, ks->pk, ks->tr, ks->keys, sv->nkeys[li]}
                        : dil::ServeKeys{nullptr, nullptr, nullptr, nullptr, 0};
    }
    bool ok = cudaHostGetDevicePointer((void **)&a.sig_out, g.m_sig, 0) == cudaSuccess &&
              cudaHostGetDevicePointer((void **)&a.status, g.m_status, 0) == cudaSuccess &&
              cudaHostGetDevicePointer((void **)&a.iters, g.m_iters, 0) == cudaSuccess &&
              cudaHostGetDevicePointer((void **)&a.ok, g.m_ok, 0) == cudaSuccess &&
              cudaHostGetDevicePointer((void **)&a.comp, g.m_comp, 0) == cudaSuccess;
    a.spec = SERVE_SPEC;
    a.help_below = g.workers * SERVE_HELP_BELOW_PCT / 100;
    a.forward_above = g.workers / 2;
    // forwarding queues start empty (a ticket left in one by the previous
    // launch is uncompleted and is claimed again through head)
    ok = ok && cudaMemsetAsync(g.d_fifo, 0, dil::SERVE_TYPES * sizeof(dil::ServeFifo), g.cstream) == cudaSuccess &&
         cudaMemcpyAsync(g.d_fifo_ring, g.h_fifo_init, dil::SERVE_TYPES * (size_t)g.R * sizeof(unsigned long long),
                         cudaMemcpyHostToDevice, g.cstream) == cudaSuccess;
    a.fifo = g.d_fifo;
    a.fifo_ring = g.d_fifo_ring;
    a.fifo_limit = RING_FIFO_PER_SM;
    // hashing SMs only when at least one CTA per SM lands elsewhere (an SM
    // holds at most 8 CTAs of 8 warps): their warps hash only while requests
    // queue, and the requests must still be served by other SMs' workers
    a.hash_sms = std::min(RING_HASH_SMS, g.sms / 4);
    if (g.grid < a.hash_sms * 8 + g.sms) a.hash_sms = 0;
    assign_home_types(g, a);
    a.spin_limit = dil::PERSIST_SPIN_LIMIT;
    a.idle_ns = 10000000000ll;   // a ticket unpublished for 10 s (the host stops an idle kernel long before)
    a.mu_buf = g.d_mu;
    a.mu_tag = g.d_mu_tag;
    ok = ok && cudaEventRecord(g.ev_pub, g.cstream) == cudaSuccess &&
         cudaStreamWaitEvent(g.kstream, g.ev_pub, 0) == cudaSuccess &&
         dil::launch_serve(a, g.grid, g.kstream) == cudaSuccess &&
         cudaEventRecord(g.kdone, g.kstream) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        return false;
    }
    g.launched = true;
    g.launches++;
    return true;
}

// Asks a running kernel to exit once nothing is pending and waits for it.
void ring_halt(Ring &g) {
    std::lock_guard<std::recursive_mutex> lk(g.kmu);
    if (!g.d_ctl || !g.launched) return;
    if (!g.stop_set) {
        ring_copy_word(g, reinterpret_cast<unsigned *>(&g.d_ctl->stop), 1);
        g.stop_set = true;
    }
    cudaStreamSynchronize(g.cstream);
    cudaEventSynchronize(g.kdone);
    cudaGetLastError();
}

// Result of ticket t's request (from mapped memory) into its destinations.
void ring_result(Ring &g, Req *r, int slot, bool failed) {
    const size_t sb = sig_bytes(r->level);
    r->st = 0;
    r->okv = 0;
    if (failed) {
        r->st = DIL_ECUDA;
        if (r->op == 0 && r->status) *r->status = DIL_ECUDA;
        if (r->op == 1 && r->ok) *r->ok = 0;
    } else if (r->op == 0) {
        const uint8_t *sig = g.m_sig + (size_t)slot * dil::SERVE_SIG_STRIDE;
        r->st = g.m_status[slot];
        if (r->status) *r->status = g.m_status[slot];
        if (r->sig_out) memcpy(r->sig_out, sig, sb);
        if (r->owned) memcpy(r->res->sig, sig, sb);
    } else {
        r->okv = g.m_ok[slot];
        if (r->ok) *r->ok = g.m_ok[slot];
    }
}

// Consumes every completion available; frees slots and arena in ticket order.
// With `fail_all` (the kernel or a copy failed) every outstanding request
// completes with DIL_ECUDA.  Returns the number consumed.
size_t ring_poll(dil_server *sv, bool fail_all) {
    Ring &g = sv->ring;
    const unsigned mask = (unsigned)g.R - 1;
    std::vector<Req *> done;
    std::vector<int> slots;
    const double t = now_s();
    for (;;) {
        const unsigned long long e = __atomic_load_n(g.m_comp + (g.comp_seen & mask), __ATOMIC_ACQUIRE);
        if ((unsigned)(e >> 32) != g.comp_seen) break;
        const int slot = (int)((unsigned)e & mask);
        if (Req *r = g.slot_req[slot].exchange(nullptr, std::memory_order_acquire)) {
            done.push_back(r);
            slots.push_back(slot);
        }
        g.slot_done[slot] = 1;
        g.comp_seen++;
    }
    g.pool_out->run(done.size(), [&](size_t i) {   // results out of mapped memory, several threads
        ring_result(g, done[i], slots[i], false);
        finish_request(sv, done[i], t);
    });
    const unsigned published = g.next_ticket.load(std::memory_order_acquire);
    unsigned old = g.oldest.load(std::memory_order_relaxed);
    if (fail_all) {
        for (unsigned u = old; u != published; ++u) {
            const int slot = (int)(u & mask);
            if (g.slot_done[slot]) continue;
            if (Req *r = g.slot_req[slot].exchange(nullptr, std::memory_order_acquire)) {
                ring_result(g, r, slot, true);
                finish_request(sv, r, t);
                done.push_back(r);
            }
            g.slot_done[slot] = 1;
        }
    }
    while (old != published && g.slot_done[old & mask]) {
        g.slot_done[old & mask] = 0;
        g.atail.store(g.slot_aend[old & mask].load(std::memory_order_relaxed), std::memory_order_release);
        ++old;
    }
    g.oldest.store(old, std::memory_order_release);
    g.consumed.store(g.comp_seen, std::memory_order_release);
    if (!done.empty()) {
        std::lock_guard<std::mutex> lk(sv->mu);
        for (Req *r : done) {
            if (r->owned)
                sv->completed.push_back(r);
            else if (!r->pooled)
                delete r;
        }
        sv->outstanding -= done.size();
        sv->cv_done.notify_all();
    }
    return done.size();
}

// Arena bytes of a request: its message, then (Verify) the signature at a
// 16-byte boundary.
size_t req_bytes(const Req *r) {
    const size_t m = (r->mlen + 15) & ~(size_t)15;
    return m + (r->op == 1 ? ((sig_bytes(r->level) + 15) & ~(size_t)15) : 0);
}

// Reserves arena room for `need` bytes; false when it does not fit yet.
bool arena_reserve(Ring &g, size_t need, uint64_t &start) {
    uint64_t pos = g.apos;
    const uint64_t phys = pos % g.arena;
    if (phys + need > g.arena) pos += g.arena - phys;   // a request's bytes never wrap
    if (pos + need - g.atail.load(std::memory_order_acquire) > g.arena) return false;
    start = pos;
    g.apos = pos + need;
    return true;
}

// Publishes pending requests while the ring and the arena have room.
bool ring_publish(dil_server *sv) {
    Ring &g = sv->ring;
    std::vector<Req *> batch;
    std::vector<uint64_t> starts;
    const uint64_t apos0 = g.apos;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        if (sv->max_wait_s > 0) return false;   // static batching: the slots serve
        size_t bytes = 0;
        while (!sv->pending.empty() && g.in_flight() + batch.size() < (unsigned)g.R && batch.size() < RING_CHUNK &&
               bytes < RING_CHUNK_BYTES) {
            Req *r = sv->pending.front();
            uint64_t start;
            if (!arena_reserve(g, req_bytes(r), start)) break;
            bytes += req_bytes(r);
            sv->pending.pop_front();
            batch.push_back(r);
            starts.push_back(start);
        }
    }
    if (batch.empty()) return false;
    const unsigned t0 = g.next_ticket.load(std::memory_order_relaxed), mask = (unsigned)g.R - 1;
    if (g.broken) {   // a launch or copy failed earlier: the completer fails them
        for (size_t i = 0; i < batch.size(); ++i) {
            const int slot = (int)((t0 + i) & mask);
            g.slot_aend[slot].store(starts[i] + req_bytes(batch[i]), std::memory_order_relaxed);
            g.slot_req[slot].store(batch[i], std::memory_order_release);
        }
        g.next_ticket.store(t0 + (unsigned)batch.size(), std::memory_order_release);
        return true;
    }
    g.pool_in->run(batch.size(), [&](size_t i) {   // descriptors and bytes into the staging buffers, several threads
        Req *r = batch[i];
        const int slot = (int)((t0 + i) & mask);
        const uint64_t phys = starts[i] % g.arena;
        dil::ServeReq &d = g.h_req[slot];
        d.op = r->op;
        d.level = r->level;
        d.key = r->key;
        d.pad = 0;
        d.msg = phys;
        d.mlen = r->mlen;
        d.sig = phys + ((r->mlen + 15) & ~(size_t)15);
        d.pad2 = 0;
        if (r->mlen) memcpy(g.h_arena + d.msg, r->msg, r->mlen);
        if (r->op == 1) memcpy(g.h_arena + d.sig, r->sig_in, sig_bytes(r->level));
    });
    for (size_t i = 0; i < batch.size(); ++i) {
        const int slot = (int)((t0 + i) & mask);
        g.slot_aend[slot].store(starts[i] + req_bytes(batch[i]), std::memory_order_relaxed);
        g.slot_req[slot].store(batch[i], std::memory_order_release);
        const Req *r = batch[i];
        const int ty = 3 * r->op + level_slot(r->level);
        g.type_work[ty] += RING_TYPE_US[ty] + RING_MSG_US_PER_BYTE * (double)r->mlen;
    }
    bool ok = true;
    auto h2d = [&](void *dst, const void *src, size_t n) {
        if (n && ok) ok = cudaMemcpyAsync(dst, src, n, cudaMemcpyHostToDevice, g.cstream) == cudaSuccess;
    };
    // descriptors: slots [t0, t0 + k) mod R in at most two pieces
    const size_t k = batch.size(), s0 = t0 & mask, first = std::min(k, (size_t)g.R - s0);
    h2d(g.d_req + s0, g.h_req + s0, first * sizeof(dil::ServeReq));
    h2d(g.d_req, g.h_req, (k - first) * sizeof(dil::ServeReq));
    // arena: positions [starts[0], apos) in at most two pieces (skipped bytes copy along)
    const uint64_t span = g.apos - apos0;
    const uint64_t p0 = apos0 % g.arena, a_first = std::min<uint64_t>(span, g.arena - p0);
    h2d(g.d_arena + p0, g.h_arena + p0, a_first);
    h2d(g.d_arena, g.h_arena, span - a_first);
    g.next_ticket.store(t0 + (unsigned)k, std::memory_order_release);
    ok = ok && ring_copy_word(g, reinterpret_cast<unsigned *>(&g.d_ctl->tail), t0 + (unsigned)k);
    if (!ok || (!kernel_running(g) && !ring_launch(sv))) {
        cudaGetLastError();
        g.broken = true;
    }
    g.batches++;
    sv->batched_reqs += k;
    return true;
}

// The completer thread: consumes completions while the server lives; fails
// the outstanding requests once a failure is recorded and no launch runs.
void completer_loop(dil_server *sv) {
    cudaSetDevice(sv->device);
    Ring &g = sv->ring;
    for (;;) {
        const size_t n = ring_poll(sv, g.broken.load() && !kernel_running(g));
        if (n) continue;
        if (g.quit.load() && g.in_flight() == 0) break;
        if (g.in_flight())
            std::this_thread::yield();
        else
            std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
}

// The publisher thread: publishes pending requests, keeps the kernel running
// while requests are outstanding and stops it after a short idle time.
void ring_loop(dil_server *sv) {
    cudaSetDevice(sv->device);
    Ring &g = sv->ring;
    double idle_since = -1;
    for (;;) {
        const bool progress = ring_publish(sv);
        const bool running = kernel_running(g);
        if (g.broken.load()) {
            if (running) ring_halt(g);   // the completer fails what is left once the kernel is gone
        } else if (g.in_flight() && !running && g.launched) {   // outstanding requests, launch finished
            const cudaError_t q = cudaEventQuery(g.kdone);
            if ((q != cudaSuccess && q != cudaErrorNotReady) || !ring_launch(sv)) {
                cudaGetLastError();
                g.broken = true;
            }
        }
        if (g.in_flight() || progress) {
            idle_since = -1;
        } else if (running) {   // nothing outstanding: stop the kernel after a short while
            const double t = now_s();
            if (idle_since < 0) idle_since = t;
            if (t - idle_since > RING_IDLE_STOP_S) {
                ring_halt(g);
                idle_since = -1;
            }
        }
        std::unique_lock<std::mutex> lk(sv->mu);
        if (sv->stop && sv->pending.empty() && g.in_flight() == 0) break;
        if (progress) continue;
        if (!sv->pending.empty() && sv->max_wait_s <= 0 && !g.broken.load()) {
            lk.unlock();   // waiting for ring or arena room
            std::this_thread::yield();
        } else if (g.in_flight() || kernel_running(g)) {
            lk.unlock();
            std::this_thread::yield();
        } else {
            sv->cv_ring.wait_for(lk, std::chrono::milliseconds(2),
                                 [&] { return sv->stop || (!sv->pending.empty() && sv->max_wait_s <= 0); });
        }
    }
    ring_halt(g);
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
        if (sv->pending.empty() || sv->max_wait_s <= 0) {
            sv->cv_work.wait_for(lk, std::chrono::milliseconds(5),
                                 [&] { return sv->stop || (!sv->pending.empty() && sv->max_wait_s > 0); });
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
    if (sv->max_wait_s > 0)
        sv->cv_work.notify_one();
    else
        sv->cv_ring.notify_one();
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
    const size_t total = memory_budget ? memory_budget : ((size_t)4 << 30);
    // half of the budget for the device ring of continuous batching, half for
    // the static-batching slots: shrink the batch until S slots fit
    const size_t budget = total / 2;
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
    if (!ring_alloc(sv->ring, device, total - budget, msg_cap)) {
        for (auto &t : sv->slots) free_slot(t);
        dil_ctx_destroy(sv->ctx);
        delete sv;
        return DIL_ENOMEM;
    }
    for (auto &s : sv->slots) sv->workers.emplace_back(slot_loop, sv, &s);
    sv->ring.completer = std::thread(completer_loop, sv);
    sv->ring_thread = std::thread(ring_loop, sv);
    *out = sv;
    return DIL_OK;
}

int dil_server_destroy(dil_server *sv) {
    if (!sv) return DIL_OK;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
        sv->cv_work.notify_all();
        sv->cv_ring.notify_all();
    }
    for (auto &w : sv->workers)
        if (w.joinable()) w.join();
    if (sv->ring_thread.joinable()) sv->ring_thread.join();
    sv->ring.quit = true;
    if (sv->ring.completer.joinable()) sv->ring.completer.join();
    cudaSetDevice(sv->device);
    cudaDeviceSynchronize();
    ring_free(sv->ring);
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
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->min_batch = min_batch;
        sv->max_wait_s = max_wait_s;
        sv->cv_ring.notify_all();
        sv->cv_work.notify_all();
    }
    if (max_wait_s > 0) {   // static batches need the SMs the serving kernel holds while it idles
        cudaSetDevice(sv->device);
        ring_halt(sv->ring);
    }
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
    ring_halt(sv->ring);   // a running serving kernel holds the old stores' addresses
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
    r->res.reset(new dil_result());
    r->t_arrive = now_s();
    std::vector<Req *> b{r};
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        r->id = sv->next_id++;
        r->res->id = r->id;
        r->res->op = op;
        r->res->level = level;
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
        r->st = DIL_ECANCELED;
        r->okv = 0;
        r->lat = now_s() - r->t_arrive;
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
        r->res->status = r->st;
        r->res->ok = r->okv;
        r->res->latency_s = r->lat;
        out[k++] = *r->res;
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
    std::vector<Req> reqs(n);   // completed requests are not freed one by one
    const double t0 = now_s();
    std::vector<Req *> batch;
    size_t i = 0;
    while (i < n) {
        const double t = now_s() - t0;
        while (i < n && arrival_s[i] <= t) {
            Req *r = &reqs[i];
            r->pooled = true;
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
            if (batch.size() == 256) enqueue(sv, batch);   // a burst reaches the ring while the rest is built
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
    if (batches) *batches = sv->batches + sv->ring.batches;
    if (requests) *requests = sv->batched_reqs;
    if (launches) *launches = sv->launches + sv->ring.launches;
    return DIL_OK;
}

int dil_test_server_mu_hashed(const dil_server *sv, uint64_t *count) {
    if (!sv || !count) return DIL_EINVAL;
    *count = 0;
    if (!sv->ring.d_ctl) return DIL_OK;
    int v = 0;
    cudaSetDevice(sv->device);
    if (cudaMemcpy(&v, &sv->ring.d_ctl->mu_used, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
        cudaGetLastError();
        return DIL_ECUDA;
    }
    *count = (uint64_t)(unsigned)v;
    return DIL_OK;
}

}  // extern "C"

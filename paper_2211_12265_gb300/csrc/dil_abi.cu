// C ABI of the batched Dilithium engine (declarations and contracts in
// include/dil.h).  Host-side argument checking, the device workspace owned by a
// context, batch chunking to the workspace budget, and the host-buffer forms.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>

#include <nvtx3/nvToolsExt.h>

#include "../../include/dil.h"
#include "dil_launch.h"

struct dil_ctx {
    int device = 0;
    size_t budget = 0;
    void *ws = nullptr;       // device scratch
    size_t ws_bytes = 0;
    int max_iter = 0;         // 0 = nonce cap
    // plain-kernel launch shape per operation (keygen / sign / verify) and level (2 / 3 / 5)
    int warps[3][3] = {{8, 8, 8}, {8, 8, 8}, {8, 8, 8}};   // warps per CTA
    int wpt[3][3] = {{2, 2, 2}, {2, 2, 2}, {2, 2, 2}};     // warps per task
    // host-form staging (device memory)
    void *stage = nullptr;
    size_t stage_bytes = 0;
    // persistent Sign: workspace, tuning and the cached captured launch
    void *pws = nullptr;
    size_t pws_bytes = 0;
    dil::PersistTuning ptune;
    cudaStream_t cap_stream = nullptr;
    cudaStream_t cancel_stream = nullptr;   // carries the cancel word's copy
    cudaGraphExec_t gexec = nullptr;
    dil::PersistJobs gjobs{};
    dil::PersistTuning gtune;
    int gmax_iter = -1;
    int spin_limit = 0;       // polls per bounded device wait (0 = PERSIST_SPIN_LIMIT); tests lower it
    int gspin_limit = -1;
    void *gws = nullptr;
    // host-form pipeline: extra streams and the fork / join events
    cudaStream_t aux[3] = {nullptr, nullptr, nullptr};
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    std::mutex mu;
};

namespace {

constexpr size_t POLY_BYTES = 256 * sizeof(int32_t);

// NVTX range over one API call (a no-op unless a profiler is attached), so
// traces show which entry point issued which launches.
struct TraceRange {
    explicit TraceRange(const char *name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange &) = delete;
    TraceRange &operator=(const TraceRange &) = delete;
};

bool level_ok(int level) { return level == 2 || level == 3 || level == 5; }
int lidx(int level) { return level == 2 ? 0 : level == 3 ? 1 : 2; }

int cuda_fail(cudaError_t e) { return e == cudaErrorMemoryAllocation ? DIL_ENOMEM : DIL_ECUDA; }

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

// Ensures at least `bytes` of workspace; returns DIL_OK or an error.
int ensure_ws(dil_ctx *c, size_t bytes) {
    if (bytes <= c->ws_bytes) return DIL_OK;
    if (bytes > c->budget) return DIL_ENOMEM;
    if (c->ws) {
        cudaDeviceSynchronize();
        cudaFree(c->ws);
        c->ws = nullptr;
        c->ws_bytes = 0;
    }
    cudaError_t e = cudaMalloc(&c->ws, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        c->ws = nullptr;
        return DIL_ENOMEM;
    }
    c->ws_bytes = bytes;
    return DIL_OK;
}

// Largest number of tasks per launch whose scratch fits the budget.
size_t chunk_tasks(dil_ctx *c, int op, int level, size_t n) {
    size_t per = dil::scratch_polys(op, level) * POLY_BYTES;
    if (per == 0) return n;
    size_t fit = c->budget / per;
    size_t lim = std::min<size_t>(n, std::min<size_t>(fit, (size_t)1 << 30));
    return lim;
}

void sizes_of(int level, size_t &pk, size_t &sk, size_t &sig) { dil_sizes(level, &pk, &sk, &sig); }

}  // namespace

extern "C" {

int dil_sizes(int level, size_t *pk_bytes, size_t *sk_bytes, size_t *sig_bytes) {
    size_t pk, sk, sig;
    switch (level) {
        case 2: pk = 1312; sk = 2528; sig = 2420; break;
        case 3: pk = 1952; sk = 4000; sig = 3293; break;
        case 5: pk = 2592; sk = 4864; sig = 4595; break;
        default: return DIL_EINVAL;
    }
    if (pk_bytes) *pk_bytes = pk;
    if (sk_bytes) *sk_bytes = sk;
    if (sig_bytes) *sig_bytes = sig;
    return DIL_OK;
}

const char *dil_status_string(int status) {
    switch (status) {
        case DIL_OK: return "ok";
        case DIL_EINVAL: return "invalid argument";
        case DIL_ENOMEM: return "out of workspace or device memory";
        case DIL_ECUDA: return "CUDA error";
        case DIL_ETIMEOUT: return "device wait timed out";
        case DIL_EITER: return "sign repetition cap reached";
        case DIL_ECANCELED: return "canceled";
    }
    return "unknown status";
}

int dil_ctx_create(int device, size_t workspace_budget, dil_ctx **out) {
    if (!out) return DIL_EINVAL;
    *out = nullptr;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess) {
        cudaGetLastError();
        return DIL_ECUDA;
    }
    if (device < 0 || device >= count) return DIL_EINVAL;
    dil_ctx *c = new dil_ctx;
    c->device = device;
    c->budget = workspace_budget ? workspace_budget : ((size_t)8 << 30);
    *out = c;
    return DIL_OK;
}

int dil_ctx_destroy(dil_ctx *c) {
    if (!c) return DIL_OK;
    {
        DeviceGuard g(c->device);
        cudaDeviceSynchronize();
        if (c->ws) cudaFree(c->ws);
        if (c->stage) cudaFree(c->stage);
        if (c->pws) cudaFree(c->pws);
        if (c->gexec) cudaGraphExecDestroy(c->gexec);
        if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
        if (c->cancel_stream) cudaStreamDestroy(c->cancel_stream);
        for (cudaStream_t a : c->aux)
            if (a) cudaStreamDestroy(a);
        if (c->ev_fork) cudaEventDestroy(c->ev_fork);
        if (c->ev_join) cudaEventDestroy(c->ev_join);
    }
    delete c;
    return DIL_OK;
}

int dil_set_tuning(dil_ctx *c, int op, int level, int warps_per_cta, int warps_per_task) {
    if (!c || op < 0 || op > 2 || warps_per_cta < 1 || warps_per_cta > 8) return DIL_EINVAL;
    if (level != 0 && !level_ok(level)) return DIL_EINVAL;
    if (warps_per_task != 1 && warps_per_task != 2 && warps_per_task != 4) return DIL_EINVAL;
    if (warps_per_cta % warps_per_task) return DIL_EINVAL;
    std::lock_guard<std::mutex> lk(c->mu);
    for (int li = 0; li < 3; ++li) {
        if (level && lidx(level) != li) continue;
        c->warps[op][li] = warps_per_cta;
        c->wpt[op][li] = warps_per_task;
    }
    return DIL_OK;
}

int dil_set_max_iter(dil_ctx *c, int max_iter) {
    if (!c || max_iter < 0) return DIL_EINVAL;
    c->max_iter = max_iter;
    return DIL_OK;
}

int dil_keygen(dil_ctx *c, int level, size_t n, const uint8_t *seeds, uint8_t *pk, uint8_t *sk, void *stream) {
    TraceRange trace("dil_keygen");
    if (!c || !level_ok(level)) return DIL_EINVAL;
    if (n == 0) return DIL_OK;
    if (!seeds || !pk || !sk || n > (size_t)INT32_MAX) return DIL_EINVAL;
    std::lock_guard<std::mutex> lk(c->mu);
    DeviceGuard g(c->device);
    size_t pkb, skb, sigb;
    sizes_of(level, pkb, skb, sigb);
    size_t chunk = chunk_tasks(c, dil::OP_KEYGEN, level, n);
    if (chunk == 0) return DIL_ENOMEM;
    int rc = ensure_ws(c, chunk * dil::scratch_polys(dil::OP_KEYGEN, level) * POLY_BYTES);
    if (rc) return rc;
    for (size_t s0 = 0; s0 < n; s0 += chunk) {
        int m = (int)std::min(chunk, n - s0);
        cudaError_t e = dil::launch_keygen(level, m, seeds + 32 * s0, pk + pkb * s0, sk + skb * s0,
                                           (int32_t *)c->ws, c->warps[0][lidx(level)], c->wpt[0][lidx(level)], (cudaStream_t)stream);
        if (e != cudaSuccess) return cuda_fail(e);
    }
    return DIL_OK;
}

int dil_sign_ex(dil_ctx *c, int level, size_t n, const uint8_t *sk, const uint8_t *msg, const uint64_t *msg_off,
                uint8_t *sig, int32_t *task_status, int32_t *iterations, void *stream) {
    TraceRange trace("dil_sign_ex");
    if (!c || !level_ok(level)) return DIL_EINVAL;
    if (n == 0) return DIL_OK;
    if (!sk || !msg_off || !sig || n > (size_t)INT32_MAX) return DIL_EINVAL;
    std::lock_guard<std::mutex> lk(c->mu);
    DeviceGuard g(c->device);
    size_t pkb, skb, sigb;
    sizes_of(level, pkb, skb, sigb);
    int l = level == 2 ? 4 : level == 3 ? 5 : 7;
    int cap = (65536 - l) / l + 1;
    int max_iter = (c->max_iter > 0 && c->max_iter < cap) ? c->max_iter : cap;
    size_t chunk = chunk_tasks(c, dil::OP_SIGN, level, n);
    if (chunk == 0) return DIL_ENOMEM;
    int rc = ensure_ws(c, chunk * dil::scratch_polys(dil::OP_SIGN, level) * POLY_BYTES);
    if (rc) return rc;
    for (size_t s0 = 0; s0 < n; s0 += chunk) {
        int m = (int)std::min(chunk, n - s0);
        cudaError_t e = dil::launch_sign(level, m, sk + skb * s0, msg, msg_off + s0, sig + sigb * s0,
                                         task_status ? task_status + s0 : nullptr,
                                         iterations ? iterations + s0 : nullptr, (int32_t *)c->ws, max_iter,
                                         c->warps[1][lidx(level)], c->wpt[1][lidx(level)], (cudaStream_t)stream);
        if (e != cudaSuccess) return cuda_fail(e);
    }
    return DIL_OK;
}

int dil_sign(dil_ctx *c, int level, size_t n, const uint8_t *sk, const uint8_t *msg, const uint64_t *msg_off,
             uint8_t *sig, int32_t *task_status, void *stream) {
    return dil_sign_ex(c, level, n, sk, msg, msg_off, sig, task_status, nullptr, stream);
}

int dil_verify(dil_ctx *c, int level, size_t n, const uint8_t *pk, const uint8_t *msg, const uint64_t *msg_off,
               const uint8_t *sig, uint8_t *ok, void *stream) {
    TraceRange trace("dil_verify");
    if (!c || !level_ok(level)) return DIL_EINVAL;
    if (n == 0) return DIL_OK;
    if (!pk || !msg_off || !sig || !ok || n > (size_t)INT32_MAX) return DIL_EINVAL;
    std::lock_guard<std::mutex> lk(c->mu);
    DeviceGuard g(c->device);
    size_t pkb, skb, sigb;
    sizes_of(level, pkb, skb, sigb);
    size_t chunk = chunk_tasks(c, dil::OP_VERIFY, level, n);
    if (chunk == 0) return DIL_ENOMEM;
    int rc = ensure_ws(c, chunk * dil::scratch_polys(dil::OP_VERIFY, level) * POLY_BYTES);
    if (rc) return rc;
    for (size_t s0 = 0; s0 < n; s0 += chunk) {
        int m = (int)std::min(chunk, n - s0);
        cudaError_t e = dil::launch_verify(level, m, pk + pkb * s0, msg, msg_off + s0, sig + sigb * s0, ok + s0,
                                           (int32_t *)c->ws, c->warps[2][lidx(level)], c->wpt[2][lidx(level)],
                                           (cudaStream_t)stream);
        if (e != cudaSuccess) return cuda_fail(e);
    }
    return DIL_OK;
}

// ---------------------------------------------------------------- caller-owned A^
namespace {
bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }
size_t ahat_words(int level) {
    const int k = level == 2 ? 4 : level == 3 ? 6 : 8, l = level == 2 ? 4 : level == 3 ? 5 : 7;
    return (size_t)k * l * 256;
}
}  // namespace

int dil_expand_a(dil_ctx *c, int level, size_t n, const uint8_t *rho, size_t rho_stride, uint32_t *ahat,
                 void *stream) {
    TraceRange trace("dil_expand_a");
    if (!c || !level_ok(level) || rho_stride < 32) return DIL_EINVAL;
    if (n == 0) return DIL_OK;
    if (!rho || !ahat || !aligned16(ahat) || n > (size_t)INT32_MAX) return DIL_EINVAL;
    std::lock_guard<std::mutex> lk(c->mu);
    DeviceGuard g(c->device);
    // one warp per key, in the CTA size of Verify's tuning (the other kernel
    // whose first step is ExpandA); the output needs no workspace
    cudaError_t e = dil::launch_expand_a(level, (int)n, rho, rho_stride, reinterpret_cast<int32_t *>(ahat),
                                         c->warps[2][lidx(level)], (cudaStream_t)stream);
    return e != cudaSuccess ? cuda_fail(e) : DIL_OK;
}

int dil_sign_a(dil_ctx *c, int level, size_t n, const uint8_t *sk, const uint8_t *msg, const uint64_t *msg_off,
               const uint32_t *ahat, uint8_t *sig, int32_t *task_status, int32_t *iterations, void *stream) {
    if (!ahat) return dil_sign_ex(c, level, n, sk, msg, msg_off, sig, task_status, iterations, stream);
    TraceRange trace("dil_sign_a");
    if (!c || !level_ok(level)) return DIL_EINVAL;
    if (n == 0) return DIL_OK;
    if (!sk || !msg_off || !sig || !aligned16(ahat) || n > (size_t)INT32_MAX) return DIL_EINVAL;
    std::lock_guard<std::mutex> lk(c->mu);
    DeviceGuard g(c->device);
    size_t pkb, skb, sigb;
    sizes_of(level, pkb, skb, sigb);
    const int l = level == 2 ? 4 : level == 3 ? 5 : 7;
    const int cap = (65536 - l) / l + 1;
    const int max_iter = (c->max_iter > 0 && c->max_iter < cap) ? c->max_iter : cap;
    const size_t chunk = chunk_tasks(c, dil::OP_SIGN, level, n);
    if (chunk == 0) return DIL_ENOMEM;
    int rc = ensure_ws(c, chunk * dil::scratch_polys(dil::OP_SIGN, level) * POLY_BYTES);
    if (rc) return rc;
    const int32_t *a = reinterpret_cast<const int32_t *>(ahat);
    for (size_t s0 = 0; s0 < n; s0 += chunk) {
        const int m = (int)std::min(chunk, n - s0);
        cudaError_t e = dil::launch_sign_a(level, m, sk + skb * s0, msg, msg_off + s0, a + ahat_words(level) * s0,
                                           sig + sigb * s0, task_status ? task_status + s0 : nullptr,
                                           iterations ? iterations + s0 : nullptr, (int32_t *)c->ws, max_iter,
                                           c->warps[1][lidx(level)], (cudaStream_t)stream);
        if (e != cudaSuccess) return cuda_fail(e);
    }
    return DIL_OK;
}

int dil_verify_a(dil_ctx *c, int level, size_t n, const uint8_t *pk, const uint8_t *msg, const uint64_t *msg_off,
                 const uint8_t *sig, const uint32_t *ahat, uint8_t *ok, void *stream) {
    if (!ahat) return dil_verify(c, level, n, pk, msg, msg_off, sig, ok, stream);
    TraceRange trace("dil_verify_a");
    if (!c || !level_ok(level)) return DIL_EINVAL;
    if (n == 0) return DIL_OK;
    if (!pk || !msg_off || !sig || !ok || !aligned16(ahat) || n > (size_t)INT32_MAX) return DIL_EINVAL;
    std::lock_guard<std::mutex> lk(c->mu);
    DeviceGuard g(c->device);
    size_t pkb, skb, sigb;
    sizes_of(level, pkb, skb, sigb);
    const size_t chunk = chunk_tasks(c, dil::OP_VERIFY, level, n);
    if (chunk == 0) return DIL_ENOMEM;
    int rc = ensure_ws(c, chunk * dil::scratch_polys(dil::OP_VERIFY, level) * POLY_BYTES);
    if (rc) return rc;
    const int32_t *a = reinterpret_cast<const int32_t *>(ahat);
    for (size_t s0 = 0; s0 < n; s0 += chunk) {
        const int m = (int)std::min(chunk, n - s0);
        cudaError_t e = dil::launch_verify_a(level, m, pk + pkb * s0, msg, msg_off + s0, sig + sigb * s0,
                                             a + ahat_words(level) * s0, ok + s0, (int32_t *)c->ws,
                                             c->warps[2][lidx(level)], (cudaStream_t)stream);
        if (e != cudaSuccess) return cuda_fail(e);
    }
    return DIL_OK;
}

// ---------------------------------------------------------------- persistent
int dil_set_persistent_tuning(dil_ctx *c, int warps_per_cta, int warps_per_task, int ctas_per_sm, int chunk,
                              int speculation) {
    if (!c || warps_per_cta < 1 || warps_per_cta > 8 || ctas_per_sm < 0 || chunk < 1 || speculation < 0)
        return DIL_EINVAL;
    if (warps_per_task != 1 && warps_per_task != 2 && warps_per_task != 4) return DIL_EINVAL;
    if (warps_per_cta % warps_per_task) return DIL_EINVAL;
    std::lock_guard<std::mutex> lk(c->mu);
    c->ptune.warps = warps_per_cta;
    c->ptune.p = warps_per_task;
    c->ptune.ctas_per_sm = ctas_per_sm;
    c->ptune.chunk = chunk;
    c->ptune.spec = speculation;
    return DIL_OK;
}

namespace {
bool same_jobs(const dil::PersistJobs &a, const dil::PersistJobs &b) { return memcmp(&a, &b, sizeof(a)) == 0; }
bool same_tune(const dil::PersistTuning &a, const dil::PersistTuning &b) {
    return a.warps == b.warps && a.p == b.p && a.ctas_per_sm == b.ctas_per_sm && a.chunk == b.chunk &&
           a.spec == b.spec;
}
}  // namespace

int dil_sign_persistent(dil_ctx *c, int njobs, const dil_sign_job *jobs, void *stream) {
    TraceRange trace("dil_sign_persistent");
    if (!c || njobs < 1 || njobs > dil::PERSIST_MAX_JOBS || !jobs) return DIL_EINVAL;
    dil::PersistJobs J;
    memset(&J, 0, sizeof(J));
    size_t total = 0;
    for (int j = 0; j < njobs; ++j) {
        const dil_sign_job &x = jobs[j];
        if (!level_ok(x.level)) return DIL_EINVAL;
        if (x.n && (!x.sk || !x.msg_off || !x.sig)) return DIL_EINVAL;
        J.job[j].level = x.level;
        J.job[j].n = (int)x.n;
        J.job[j].start = (int)total;
        J.job[j].sk = x.sk;
        J.job[j].msg = x.msg;
        J.job[j].off = x.msg_off;
        J.job[j].sig = x.sig;
        J.job[j].status = x.task_status;
        J.job[j].iters = x.iterations;
        total += x.n;
        if (total > (size_t)INT32_MAX / 2) return DIL_EINVAL;
    }
    J.njobs = njobs;
    J.total = (int)total;
    if (total == 0) return DIL_OK;
    std::lock_guard<std::mutex> lk(c->mu);
    DeviceGuard g(c->device);
    {   // SMs per job in proportion to its work (a task's relative cost by level:
        // persistent Sign rates 3.65 / 2.42 / 1.98 M/s at 10,000 tasks)
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess) return DIL_ECUDA;
        double w[dil::PERSIST_MAX_JOBS], sum = 0;
        for (int j = 0; j < njobs; ++j) {
            const int lv = J.job[j].level;
            w[j] = (double)J.job[j].n * (lv == 2 ? 1.0 : lv == 3 ? 1.51 : 1.84);
            sum += w[j];
        }
        double acc = 0;
        for (int j = 0; j < njobs; ++j) {
            acc += w[j];
            J.sm_end[j] = j + 1 == njobs ? (1 << 30) : (int)(sms * acc / sum + 0.5);
        }
    }
    const size_t need = dil::persist_workspace_bytes(J, c->ptune, c->device);
    if (need == 0) return DIL_ECUDA;
    if (need > c->budget) return DIL_ENOMEM;
    if (need > c->pws_bytes) {
        if (c->pws) {
            cudaDeviceSynchronize();
            cudaFree(c->pws);
            c->pws = nullptr;
            c->pws_bytes = 0;
        }
        if (cudaMalloc(&c->pws, need) != cudaSuccess) {
            cudaGetLastError();
            return DIL_ENOMEM;
        }
        c->pws_bytes = need;
    }
    const int max_iter = c->max_iter;
    if (!c->gexec || !same_jobs(J, c->gjobs) || !same_tune(c->ptune, c->gtune) || max_iter != c->gmax_iter ||
        c->spin_limit != c->gspin_limit || c->gws != c->pws) {
        if (c->gexec) {
            cudaGraphExecDestroy(c->gexec);
            c->gexec = nullptr;
        }
        if (!c->cap_stream && cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
            return DIL_ECUDA;
        // warm the attribute / occupancy queries outside the capture
        if (dil::persist_workspace_bytes(J, c->ptune, c->device) == 0) return DIL_ECUDA;
        cudaGraph_t graph = nullptr;
        if (cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeRelaxed) != cudaSuccess) return DIL_ECUDA;
        cudaError_t e = dil::launch_sign_persist(J, c->pws, c->ptune, max_iter, c->spin_limit, c->device,
                                                 c->cap_stream);
        cudaError_t e2 = cudaStreamEndCapture(c->cap_stream, &graph);
        if (e != cudaSuccess || e2 != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            cudaGetLastError();
            return DIL_ECUDA;
        }
        e = cudaGraphInstantiate(&c->gexec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            c->gexec = nullptr;
            return DIL_ECUDA;
        }
        c->gjobs = J;
        c->gtune = c->ptune;
        c->gmax_iter = max_iter;
        c->gspin_limit = c->spin_limit;
        c->gws = c->pws;
    }
    return cudaGraphLaunch(c->gexec, (cudaStream_t)stream) == cudaSuccess ? DIL_OK : DIL_ECUDA;
}

int dil_persistent_status(dil_ctx *c, void *stream) {
    if (!c) return DIL_EINVAL;
    DeviceGuard g(c->device);
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return DIL_ECUDA;
    std::lock_guard<std::mutex> lk(c->mu);
    if (!c->pws) return DIL_OK;
    return dil::persist_error(c->pws);
}

int dil_persistent_cancel(dil_ctx *c) {
    TraceRange trace("dil_persistent_cancel");
    if (!c) return DIL_EINVAL;
    DeviceGuard g(c->device);
    std::lock_guard<std::mutex> lk(c->mu);
    if (!c->pws) return DIL_OK;
    if (!c->cancel_stream && cudaStreamCreateWithFlags(&c->cancel_stream, cudaStreamNonBlocking) != cudaSuccess)
        return DIL_ECUDA;
    return dil::persist_cancel(c->pws, c->cancel_stream) == cudaSuccess ? DIL_OK : DIL_ECUDA;
}

// ---------------------------------------------------------------- key stores
}  // extern "C"

extern "C" {

int dil_keystore_create(dil_ctx *c, int level, size_t n_keys, const uint8_t *pk, const uint8_t *sk,
                        dil_keystore **out, void *stream) {
    TraceRange trace("dil_keystore_create");
    if (!c || !out || !level_ok(level) || n_keys == 0 || !pk || n_keys > (size_t)INT32_MAX) return DIL_EINVAL;
    *out = nullptr;
    size_t pkb, skb, sigb;
    sizes_of(level, pkb, skb, sigb);
    DeviceGuard g(c->device);
    dil_keystore *ks = new dil_keystore;
    ks->device = c->device;
    ks->level = level;
    ks->n = n_keys;
    const size_t kbytes = n_keys * dil::key_polys(level) * POLY_BYTES;
    bool okm = cudaMalloc(&ks->pk, pkb * n_keys) == cudaSuccess && cudaMalloc(&ks->tr, 32 * n_keys) == cudaSuccess &&
               cudaMalloc(&ks->keys, kbytes) == cudaSuccess;
    if (okm && sk) okm = cudaMalloc(&ks->sk, skb * n_keys) == cudaSuccess;
    if (!okm) {
        cudaGetLastError();
        dil_keystore_destroy(ks);
        return DIL_ENOMEM;
    }
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(ks->pk, pk, pkb * n_keys, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess && sk) e = cudaMemcpyAsync(ks->sk, sk, skb * n_keys, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess)
        e = dil::launch_key_prepare(level, (int)n_keys, ks->pk, ks->sk, ks->keys, ks->tr, 8, 2, s);
    if (e != cudaSuccess) {
        dil_keystore_destroy(ks);
        return cuda_fail(e);
    }
    *out = ks;
    return DIL_OK;
}

int dil_keystore_destroy(dil_keystore *ks) {
    if (!ks) return DIL_OK;
    {
        DeviceGuard g(ks->device);
        cudaDeviceSynchronize();
        if (ks->pk) cudaFree(ks->pk);
        if (ks->sk) cudaFree(ks->sk);
        if (ks->tr) cudaFree(ks->tr);
        if (ks->keys) cudaFree(ks->keys);
    }
    delete ks;
    return DIL_OK;
}

int dil_sign_keyed(dil_ctx *c, const dil_keystore *ks, size_t n, const int32_t *key_idx, const uint8_t *msg,
                   const uint64_t *msg_off, uint8_t *sig, int32_t *task_status, void *stream) {
    TraceRange trace("dil_sign_keyed");
    if (!c || !ks || !ks->sk || ks->device != c->device) return DIL_EINVAL;
    if (n == 0) return DIL_OK;
    if (!key_idx || !msg_off || !sig || n > (size_t)INT32_MAX) return DIL_EINVAL;
    std::lock_guard<std::mutex> lk(c->mu);
    DeviceGuard g(c->device);
    size_t pkb, skb, sigb;
    sizes_of(ks->level, pkb, skb, sigb);
    const int l = ks->level == 2 ? 4 : ks->level == 3 ? 5 : 7;
    const int cap = (65536 - l) / l + 1;
    const int max_iter = (c->max_iter > 0 && c->max_iter < cap) ? c->max_iter : cap;
    const size_t per = dil::keyed_sign_polys(ks->level) * POLY_BYTES;
    size_t chunk = std::min<size_t>(n, c->budget / per);
    if (chunk == 0) return DIL_ENOMEM;
    int rc = ensure_ws(c, chunk * per);
    if (rc) return rc;
    for (size_t s0 = 0; s0 < n; s0 += chunk) {
        int m = (int)std::min(chunk, n - s0);
        cudaError_t e = dil::launch_sign_keyed(ks->level, m, (int)ks->n, key_idx + s0, ks->sk, ks->keys, msg,
                                               msg_off + s0, sig + sigb * s0,
                                               task_status ? task_status + s0 : nullptr, nullptr, (int32_t *)c->ws,
                                               max_iter, c->warps[1][lidx(ks->level)], c->wpt[1][lidx(ks->level)],
                                               (cudaStream_t)stream);
        if (e != cudaSuccess) return cuda_fail(e);
    }
    return DIL_OK;
}

int dil_verify_keyed(dil_ctx *c, const dil_keystore *ks, size_t n, const int32_t *key_idx, const uint8_t *msg,
                     const uint64_t *msg_off, const uint8_t *sig, uint8_t *ok, void *stream) {
    TraceRange trace("dil_verify_keyed");
    if (!c || !ks || ks->device != c->device) return DIL_EINVAL;
    if (n == 0) return DIL_OK;
    if (!key_idx || !msg_off || !sig || !ok || n > (size_t)INT32_MAX) return DIL_EINVAL;
    std::lock_guard<std::mutex> lk(c->mu);
    DeviceGuard g(c->device);
    size_t pkb, skb, sigb;
    sizes_of(ks->level, pkb, skb, sigb);
    const size_t per = dil::keyed_verify_polys(ks->level) * POLY_BYTES;
    size_t chunk = std::min<size_t>(n, c->budget / per);
    if (chunk == 0) return DIL_ENOMEM;
    int rc = ensure_ws(c, chunk * per);
    if (rc) return rc;
    for (size_t s0 = 0; s0 < n; s0 += chunk) {
        int m = (int)std::min(chunk, n - s0);
        cudaError_t e = dil::launch_verify_keyed(ks->level, m, (int)ks->n, key_idx + s0, ks->pk, ks->keys, ks->tr,
                                                 msg, msg_off + s0, sig + sigb * s0, ok + s0, (int32_t *)c->ws,
                                                 c->warps[2][lidx(ks->level)], c->wpt[2][lidx(ks->level)],
                                                 (cudaStream_t)stream);
        if (e != cudaSuccess) return cuda_fail(e);
    }
    return DIL_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- host forms
namespace {

// Device staging for the host forms: grows on demand (not part of the budget).
int ensure_stage(dil_ctx *c, size_t bytes) {
    if (bytes <= c->stage_bytes) return DIL_OK;
    if (c->stage) {
        cudaDeviceSynchronize();
        cudaFree(c->stage);
        c->stage = nullptr;
        c->stage_bytes = 0;
    }
    if (cudaMalloc(&c->stage, bytes) != cudaSuccess) {
        cudaGetLastError();
        return DIL_ENOMEM;
    }
    c->stage_bytes = bytes;
    return DIL_OK;
}

size_t al(size_t x) { return (x + 255) & ~(size_t)255; }

// Host-buffer forms as a pipeline (the paper's section 4.4 multi-stream
// overlap): a large batch is cut into PIPE_STREAMS chunks, each on its own
// stream (the caller's and the context's extra ones) with its own part of the
// workspace.  A chunk copies its inputs in, runs its kernel and copies its
// outputs back; the chunks' kernels run concurrently (together they fill the
// GPU like one launch, and their tails overlap), while the copies of one
// chunk overlap the kernels of the others.  When the budget cannot hold the
// whole batch's scratch, chunks shrink and cycle over the streams.
constexpr size_t PIPE_MIN_TASKS = 2048;   // smaller batches run as one chunk
constexpr size_t PIPE_STREAMS = 4;

int ensure_aux(dil_ctx *c) {
    if (c->aux[0]) return DIL_OK;
    for (cudaStream_t &a : c->aux)
        if (cudaStreamCreateWithFlags(&a, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            return DIL_ECUDA;
        }
    if (cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        return DIL_ECUDA;
    }
    return DIL_OK;
}

// Runs chunk(c0, c1, stream, scratch) over the batch and waits for the
// caller's stream.  `per_task` is the kernel scratch of one task.
template <class Chunk>
int run_pipeline(dil_ctx *c, size_t n, size_t per_task, cudaStream_t s0, Chunk chunk) {
    const size_t ns = n >= PIPE_MIN_TASKS ? PIPE_STREAMS : 1;
    size_t per = (n + ns - 1) / ns;
    const size_t fit = per_task ? c->budget / (ns * per_task) : per;
    if (fit == 0) return DIL_ENOMEM;
    per = std::min(per, fit);
    const size_t k = (n + per - 1) / per;
    int rc = ensure_ws(c, ns * per * per_task);
    if (!rc && ns > 1) rc = ensure_aux(c);
    if (rc) return rc;
    cudaStream_t st[PIPE_STREAMS] = {s0, c->aux[0], c->aux[1], c->aux[2]};
    if (ns > 1) {
        if (cudaEventRecord(c->ev_fork, s0) != cudaSuccess) return DIL_ECUDA;
        for (size_t j = 1; j < ns; ++j)
            if (cudaStreamWaitEvent(st[j], c->ev_fork, 0) != cudaSuccess) return DIL_ECUDA;
    }
    for (size_t i = 0; i < k && !rc; ++i) {
        const size_t c0 = i * per, c1 = std::min(n, c0 + per);
        int32_t *scratch = (int32_t *)c->ws + (i % ns) * per * (per_task / sizeof(int32_t));
        rc = chunk(c0, c1, st[i % ns], scratch);
    }
    for (size_t j = 1; j < ns; ++j)
        if ((cudaEventRecord(c->ev_join, st[j]) != cudaSuccess ||
             cudaStreamWaitEvent(s0, c->ev_join, 0) != cudaSuccess) && !rc)
            rc = DIL_ECUDA;
    const cudaError_t e = cudaStreamSynchronize(s0);
    if (rc) return rc;
    return e == cudaSuccess ? DIL_OK : DIL_ECUDA;
}

// Host offsets of the host forms: non-decreasing (a task's message is
// msg[off[i] .. off[i + 1])).
bool offsets_ok(const uint64_t *off, size_t n) {
    for (size_t i = 0; i < n; ++i)
        if (off[i + 1] < off[i]) return false;
    return true;
}

bool h2d(void *dst, const void *src, size_t bytes, cudaStream_t s) {
    return bytes == 0 || cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s) == cudaSuccess;
}
bool d2h(void *dst, const void *src, size_t bytes, cudaStream_t s) {
    return bytes == 0 || cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, s) == cudaSuccess;
}

}  // namespace

extern "C" {

int dil_keygen_host(dil_ctx *c, int level, size_t n, const uint8_t *seeds, uint8_t *pk, uint8_t *sk,
                    void *stream) {
    TraceRange trace("dil_keygen_host");
    if (!c || !level_ok(level)) return DIL_EINVAL;
    if (n == 0) return DIL_OK;
    if (!seeds || !pk || !sk || n > (size_t)INT32_MAX) return DIL_EINVAL;
    size_t pkb, skb, sigb;
    sizes_of(level, pkb, skb, sigb);
    std::lock_guard<std::mutex> lk(c->mu);
    DeviceGuard g(c->device);
    int rc = ensure_stage(c, al(32 * n) + al(pkb * n) + al(skb * n));
    if (rc) return rc;
    uint8_t *d_seed = (uint8_t *)c->stage, *d_pk = d_seed + al(32 * n), *d_sk = d_pk + al(pkb * n);
    const int w = c->warps[0][lidx(level)], p = c->wpt[0][lidx(level)];
    return run_pipeline(c, n, dil::scratch_polys(dil::OP_KEYGEN, level) * POLY_BYTES, (cudaStream_t)stream,
                        [&](size_t c0, size_t c1, cudaStream_t s, int32_t *scratch) -> int {
                            const size_t m = c1 - c0;
                            if (!h2d(d_seed + 32 * c0, seeds + 32 * c0, 32 * m, s)) return DIL_ECUDA;
                            cudaError_t e = dil::launch_keygen(level, (int)m, d_seed + 32 * c0, d_pk + pkb * c0,
                                                               d_sk + skb * c0, scratch, w, p, s);
                            if (e != cudaSuccess) return cuda_fail(e);
                            if (!d2h(pk + pkb * c0, d_pk + pkb * c0, pkb * m, s) ||
                                !d2h(sk + skb * c0, d_sk + skb * c0, skb * m, s))
                                return DIL_ECUDA;
                            return DIL_OK;
                        });
}

int dil_sign_host(dil_ctx *c, int level, size_t n, const uint8_t *sk, const uint8_t *msg, const uint64_t *msg_off,
                  uint8_t *sig, int32_t *task_status, void *stream) {
    TraceRange trace("dil_sign_host");
    if (!c || !level_ok(level)) return DIL_EINVAL;
    if (n == 0) return DIL_OK;
    if (!sk || !msg_off || !sig || n > (size_t)INT32_MAX) return DIL_EINVAL;
    size_t pkb, skb, sigb;
    sizes_of(level, pkb, skb, sigb);
    const size_t mlen = (size_t)msg_off[n];
    if ((mlen && !msg) || !offsets_ok(msg_off, n)) return DIL_EINVAL;
    std::lock_guard<std::mutex> lk(c->mu);
    DeviceGuard g(c->device);
    int rc = ensure_stage(c, al(skb * n) + al(mlen + 1) + al(8 * (n + 1)) + al(sigb * n) + al(4 * n));
    if (rc) return rc;
    uint8_t *d_sk = (uint8_t *)c->stage, *d_msg = d_sk + al(skb * n);
    uint64_t *d_off = (uint64_t *)(d_msg + al(mlen + 1));
    uint8_t *d_sig = (uint8_t *)d_off + al(8 * (n + 1));
    int32_t *d_st = (int32_t *)(d_sig + al(sigb * n));
    const int l = level == 2 ? 4 : level == 3 ? 5 : 7, cap = (65536 - l) / l + 1;
    const int max_iter = (c->max_iter > 0 && c->max_iter < cap) ? c->max_iter : cap;
    const int w = c->warps[1][lidx(level)], p = c->wpt[1][lidx(level)];
    return run_pipeline(c, n, dil::scratch_polys(dil::OP_SIGN, level) * POLY_BYTES, (cudaStream_t)stream,
                        [&](size_t c0, size_t c1, cudaStream_t s, int32_t *scratch) -> int {
                            const size_t m = c1 - c0;
                            if (!h2d(d_sk + skb * c0, sk + skb * c0, skb * m, s) ||
                                !h2d(d_msg + msg_off[c0], msg ? msg + msg_off[c0] : nullptr,
                                     (size_t)(msg_off[c1] - msg_off[c0]), s) ||
                                !h2d(d_off + c0, msg_off + c0, 8 * (m + 1), s))
                                return DIL_ECUDA;
                            cudaError_t e = dil::launch_sign(level, (int)m, d_sk + skb * c0, d_msg, d_off + c0,
                                                             d_sig + sigb * c0, d_st + c0, nullptr, scratch,
                                                             max_iter, w, p, s);
                            if (e != cudaSuccess) return cuda_fail(e);
                            if (!d2h(sig + sigb * c0, d_sig + sigb * c0, sigb * m, s) ||
                                (task_status && !d2h(task_status + c0, d_st + c0, 4 * m, s)))
                                return DIL_ECUDA;
                            return DIL_OK;
                        });
}

int dil_verify_host(dil_ctx *c, int level, size_t n, const uint8_t *pk, const uint8_t *msg,
                    const uint64_t *msg_off, const uint8_t *sig, uint8_t *ok, void *stream) {
    TraceRange trace("dil_verify_host");
    if (!c || !level_ok(level)) return DIL_EINVAL;
    if (n == 0) return DIL_OK;
    if (!pk || !msg_off || !sig || !ok || n > (size_t)INT32_MAX) return DIL_EINVAL;
    size_t pkb, skb, sigb;
    sizes_of(level, pkb, skb, sigb);
    const size_t mlen = (size_t)msg_off[n];
    if ((mlen && !msg) || !offsets_ok(msg_off, n)) return DIL_EINVAL;
    std::lock_guard<std::mutex> lk(c->mu);
    DeviceGuard g(c->device);
    int rc = ensure_stage(c, al(pkb * n) + al(mlen + 1) + al(8 * (n + 1)) + al(sigb * n) + al(n));
    if (rc) return rc;
    uint8_t *d_pk = (uint8_t *)c->stage, *d_msg = d_pk + al(pkb * n);
    uint64_t *d_off = (uint64_t *)(d_msg + al(mlen + 1));
    uint8_t *d_sig = (uint8_t *)d_off + al(8 * (n + 1));
    uint8_t *d_ok = d_sig + al(sigb * n);
    const int w = c->warps[2][lidx(level)], p = c->wpt[2][lidx(level)];
    return run_pipeline(c, n, dil::scratch_polys(dil::OP_VERIFY, level) * POLY_BYTES, (cudaStream_t)stream,
                        [&](size_t c0, size_t c1, cudaStream_t s, int32_t *scratch) -> int {
                            const size_t m = c1 - c0;
                            if (!h2d(d_pk + pkb * c0, pk + pkb * c0, pkb * m, s) ||
                                !h2d(d_msg + msg_off[c0], msg ? msg + msg_off[c0] : nullptr,
                                     (size_t)(msg_off[c1] - msg_off[c0]), s) ||
                                !h2d(d_off + c0, msg_off + c0, 8 * (m + 1), s) ||
                                !h2d(d_sig + sigb * c0, sig + sigb * c0, sigb * m, s))
                                return DIL_ECUDA;
                            cudaError_t e = dil::launch_verify(level, (int)m, d_pk + pkb * c0, d_msg, d_off + c0,
                                                               d_sig + sigb * c0, d_ok + c0, scratch, w, p, s);
                            if (e != cudaSuccess) return cuda_fail(e);
                            if (!d2h(ok + c0, d_ok + c0, m, s)) return DIL_ECUDA;
                            return DIL_OK;
                        });
}

// ---------------------------------------------------------------- test-only
#define TEST_PROLOGUE(ctx)                  \
    if (!(ctx)) return DIL_EINVAL;          \
    std::lock_guard<std::mutex> lk((ctx)->mu); \
    DeviceGuard g((ctx)->device);

static int status_of(cudaError_t e) { return e == cudaSuccess ? DIL_OK : cuda_fail(e); }

int dil_test_shake(dil_ctx *c, int kind, size_t n, const uint8_t *in, const uint64_t *in_off, uint8_t *out,
                   size_t outlen, void *stream) {
    TEST_PROLOGUE(c)
    if ((kind != 128 && kind != 256) || n > (size_t)INT32_MAX || outlen > (1u << 20)) return DIL_EINVAL;
    if (n == 0) return DIL_OK;
    if (!in_off || !out) return DIL_EINVAL;
    return status_of(dil::launch_test_shake(kind, (int)n, in, in_off, out, (int)outlen, (cudaStream_t)stream));
}

int dil_test_k16_rider(dil_ctx *c, size_t n, const uint8_t *in, const uint64_t *in_off, const int32_t *perms,
                       uint8_t *out, void *stream) {
    TEST_PROLOGUE(c)
    if (n > (size_t)INT32_MAX) return DIL_EINVAL;
    if (n == 0) return DIL_OK;
    if (!in_off || !perms || !out) return DIL_EINVAL;
    return status_of(dil::launch_test_k16_rider((int)n, in, in_off, perms, out, (cudaStream_t)stream));
}

int dil_test_k16_chain_rider(dil_ctx *c, size_t n, const uint8_t *in, const uint64_t *in_off, const int32_t *perms,
                             const int32_t *step, uint8_t *out, void *stream) {
    TEST_PROLOGUE(c)
    if (n > (size_t)INT32_MAX) return DIL_EINVAL;
    if (n == 0) return DIL_OK;
    if (!in_off || !perms || !step || !out) return DIL_EINVAL;
    return status_of(dil::launch_test_k16_chain_rider((int)n, in, in_off, perms, step, out, (cudaStream_t)stream));
}

int dil_test_keccak_f(dil_ctx *c, int form, size_t n, const uint64_t *in, uint64_t *out, void *stream) {
    TEST_PROLOGUE(c)
    if ((form != 1 && form != 2 && form != 6 && form != 16) || n > (size_t)INT32_MAX) return DIL_EINVAL;
    if (n == 0) return DIL_OK;
    if (!in || !out) return DIL_EINVAL;
    return status_of(dil::launch_test_keccak_f(form, (int)n, in, out, (cudaStream_t)stream));
}

int dil_test_t0_ntt(dil_ctx *c, int level, int variant, size_t n, const uint8_t *sk, int32_t *t0hat, void *stream) {
    TEST_PROLOGUE(c)
    if (!level_ok(level) || variant < 0 || variant > 3 || n > (size_t)INT32_MAX) return DIL_EINVAL;
    if (n == 0) return DIL_OK;
    if (!sk || !t0hat) return DIL_EINVAL;
    int32_t *tmp = nullptr;
    if (variant <= 1) {
        const size_t k = level == 2 ? 4 : level == 3 ? 6 : 8;
        const int rc = ensure_ws(c, n * k * POLY_BYTES);
        if (rc) return rc;
        tmp = static_cast<int32_t *>(c->ws);
    }
    return status_of(dil::launch_test_t0_ntt(level, variant, (int)n, sk, tmp, t0hat, (cudaStream_t)stream));
}

int dil_test_ntt(dil_ctx *c, size_t n, const int32_t *in, int32_t *out, int inverse, void *stream) {
    TEST_PROLOGUE(c)
    if (n > (size_t)INT32_MAX || (n && (!in || !out))) return DIL_EINVAL;
    return status_of(dil::launch_test_ntt((int)n, in, out, inverse ? 1 : 0, (cudaStream_t)stream));
}

int dil_test_expand_a(dil_ctx *c, int level, size_t n, const uint8_t *rho, int32_t *ahat, void *stream) {
    TEST_PROLOGUE(c)
    if (!level_ok(level) || n > (size_t)INT32_MAX || (n && (!rho || !ahat))) return DIL_EINVAL;
    return status_of(dil::launch_test_expand_a(level, (int)n, rho, ahat, (cudaStream_t)stream));
}

int dil_test_expand_s(dil_ctx *c, int level, size_t n, const uint8_t *rhop, int32_t *s, void *stream) {
    TEST_PROLOGUE(c)
    if (!level_ok(level) || n > (size_t)INT32_MAX || (n && (!rhop || !s))) return DIL_EINVAL;
    return status_of(dil::launch_test_expand_s(level, (int)n, rhop, s, (cudaStream_t)stream));
}

int dil_test_expand_mask(dil_ctx *c, int level, size_t n, const uint8_t *rhop, const int32_t *kappa, int32_t *y,
                         void *stream) {
    TEST_PROLOGUE(c)
    if (!level_ok(level) || n > (size_t)INT32_MAX || (n && (!rhop || !kappa || !y))) return DIL_EINVAL;
    return status_of(dil::launch_test_expand_mask(level, (int)n, rhop, kappa, y, (cudaStream_t)stream));
}

int dil_test_sample_in_ball_stream(dil_ctx *c, int level, size_t n, const uint8_t *bytes, int blocks, int32_t *cc,
                                   void *stream) {
    TEST_PROLOGUE(c)
    if (!level_ok(level) || n > (size_t)INT32_MAX || blocks < 1 || blocks > 64 || (n && (!bytes || !cc)))
        return DIL_EINVAL;
    return status_of(dil::launch_test_sib_stream(level, (int)n, bytes, blocks, cc, (cudaStream_t)stream));
}

int dil_test_sample_in_ball(dil_ctx *c, int level, size_t n, const uint8_t *ctilde, int32_t *cc, void *stream) {
    TEST_PROLOGUE(c)
    if (!level_ok(level) || n > (size_t)INT32_MAX || (n && (!ctilde || !cc))) return DIL_EINVAL;
    return status_of(dil::launch_test_sample_in_ball(level, (int)n, ctilde, cc, (cudaStream_t)stream));
}

int dil_test_rounding(dil_ctx *c, int level, size_t n, const int32_t *r, const int32_t *z, const uint8_t *h,
                      int32_t *out, void *stream) {
    TEST_PROLOGUE(c)
    if (!level_ok(level) || n > (size_t)INT32_MAX || (n && (!r || !z || !h || !out))) return DIL_EINVAL;
    return status_of(dil::launch_test_rounding(level, (int)n, r, z, h, out, (cudaStream_t)stream));
}

int dil_test_bounded_wait(dil_ctx *c, int flag_value, int limit, int *result) {
    TEST_PROLOGUE(c)
    if (!result || limit < 1 || limit > (1 << 24)) return DIL_EINVAL;
    return status_of(dil::test_bounded_wait(flag_value, limit, result));
}

int dil_test_set_spin_limit(dil_ctx *c, int limit) {
    TEST_PROLOGUE(c)
    if (limit < 0 || limit > dil::PERSIST_SPIN_LIMIT) return DIL_EINVAL;
    c->spin_limit = limit;
    return DIL_OK;
}

int dil_test_issue_rate(dil_ctx *c, int op, double *thread_ops_per_sm_clk) {
    TEST_PROLOGUE(c)
    if (op < 0 || op > 4 || !thread_ops_per_sm_clk) return DIL_EINVAL;
    return status_of(dil::measure_issue_rate(op, thread_ops_per_sm_clk));
}

int dil_test_sign_split(dil_ctx *c, int level, size_t n, const uint8_t *sk, const uint8_t *msg,
                        const uint64_t *msg_off, uint8_t *sig, int32_t *task_status, int32_t *iterations,
                        int *rounds, void *stream) {
    TEST_PROLOGUE(c)
    if (!level_ok(level)) return DIL_EINVAL;
    if (rounds) *rounds = 0;
    if (n == 0) return DIL_OK;
    if (!sk || !msg_off || !sig || n > (size_t)INT32_MAX) return DIL_EINVAL;
    size_t pkb, skb, sigb;
    sizes_of(level, pkb, skb, sigb);
    const int l = level == 2 ? 4 : level == 3 ? 5 : 7, cap = (65536 - l) / l + 1;
    const int max_iter = (c->max_iter > 0 && c->max_iter < cap) ? c->max_iter : cap;
    const int p = std::min(c->wpt[1][lidx(level)], 2), w = std::max(c->warps[1][lidx(level)] / p * p, p);
    const size_t per = dil::scratch_polys(dil::OP_SIGN, level) * POLY_BYTES + dil::split_state_bytes();
    const size_t chunk = std::min<size_t>(n, (c->budget - 256) / per);
    if (chunk == 0) return DIL_ENOMEM;
    int rc = ensure_ws(c, chunk * per + 256);
    if (rc) return rc;
    int32_t *scratch = (int32_t *)c->ws;
    void *state = (uint8_t *)c->ws + chunk * dil::scratch_polys(dil::OP_SIGN, level) * POLY_BYTES;
    int *pending = (int *)((uint8_t *)state + chunk * dil::split_state_bytes());
    for (size_t s0 = 0; s0 < n; s0 += chunk) {
        const int m = (int)std::min(chunk, n - s0);
        int r = 0;
        cudaError_t e = dil::launch_sign_split(level, m, sk + skb * s0, msg, msg_off + s0, sig + sigb * s0,
                                               task_status ? task_status + s0 : nullptr,
                                               iterations ? iterations + s0 : nullptr, scratch, state, pending,
                                               max_iter, w, p, (cudaStream_t)stream, &r);
        if (e != cudaSuccess) return cuda_fail(e);
        if (rounds) *rounds = std::max(*rounds, r);
    }
    return DIL_OK;
}

int dil_test_keccak_rate(dil_ctx *c, int form, double *sm_clocks_per_state_round) {
    TEST_PROLOGUE(c)
    if ((form != 1 && form != 2 && form != 6 && form != 16) || !sm_clocks_per_state_round) return DIL_EINVAL;
    return status_of(dil::measure_keccak_rate(form, sm_clocks_per_state_round));
}

}  // extern "C"

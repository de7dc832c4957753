// Host side of the C ABI: argument checks, error reporting, per-stream workspaces and
// the single-set entry points (Section 4 of the paper; see include/cc.h).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "cc_internal.cuh"

namespace cc {

size_t single_ws_bytes(int64_t n, bool sum, bool allow_tc);
cc_status single_enqueue(const cc_points *p, int64_t n, uint32_t r2, unsigned long long *d_count,
                         float *d_sum, void *ws, cudaStream_t stream, bool allow_tc);
cc_status validate_enqueue(const cc_points *p, int64_t n, void *ws, cudaStream_t stream);
size_t straight_ws_bytes(int64_t n);
void tc_set_enabled(bool on);
size_t linear_ws_bytes(int64_t n);
cc_status linear_enqueue(const cc_points *p, int64_t n, int contacts, unsigned long long *d_count, void *ws,
                         cudaStream_t s);
cc_status straight_enqueue(const cc_points *p, int64_t n, uint32_t r2, unsigned long long *d_count, void *ws,
                           cudaStream_t stream);

static thread_local std::string t_last_error;
static std::atomic<uint64_t> g_wait_ns{2000000000ull};
static std::atomic<int> g_stall{0};

void set_error(const std::string &msg) { t_last_error = msg; }

cc_status fail(cc_status s, const std::string &msg) {
    set_error(msg);
    return s;
}

cc_status cuda_fail(cudaError_t e, const char *what) {
    set_error(std::string(what) + ": " + cudaGetErrorString(e));
    return CC_ERR_CUDA;
}

uint64_t wait_limit_ns() { return g_wait_ns.load(); }

// ---- benchmark timing hook ---------------------------------------------------------------
static std::atomic<bool> g_prof{false};
static std::mutex g_prof_mu;
static std::vector<std::pair<cudaEvent_t, cudaEvent_t>> g_prof_pending;
static std::vector<cudaEvent_t> g_prof_pool;

bool profiling() { return g_prof.load(); }

static cudaEvent_t prof_event() {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (!g_prof_pool.empty()) {
        cudaEvent_t e = g_prof_pool.back();
        g_prof_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

cudaError_t profile_begin(cudaStream_t s, cudaEvent_t *e0, cudaEvent_t *e1) {
    *e0 = prof_event();
    *e1 = prof_event();
    if (!*e0 || !*e1) return cudaErrorMemoryAllocation;
    return cudaEventRecord(*e0, s);
}

void profile_end(cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1) {
    cudaEventRecord(e1, s);
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_prof_pending.emplace_back(e0, e1);
}
int debug_stall() { return g_stall.load(); }

int sm_count() {
    static int count = 0;
    if (count == 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess) return 1;
        int c = 0;
        if (cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || c <= 0)
            return 1;
        count = c;
    }
    return count;
}

// ---------------------------------------------------------------------------------------
// per-stream workspaces
// ---------------------------------------------------------------------------------------
struct Workspace {
    void *ptr = nullptr;
    size_t bytes = 0;
};

static std::mutex g_ws_mu;
static std::map<cudaStream_t, Workspace> g_ws;

// Returns a workspace of at least `bytes` for `stream`, growing it stream-ordered.
static cc_status workspace_for(cudaStream_t stream, size_t bytes, void **out) {
    std::lock_guard<std::mutex> lk(g_ws_mu);
    Workspace &w = g_ws[stream];
    if (w.bytes < bytes) {
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        CC_CUDA(cudaStreamIsCapturing(stream, &cap));
        if (cap != cudaStreamCaptureStatusNone)
            return fail(CC_ERR_NOMEM, "workspace too small during stream capture; call cc_reserve first");
        size_t want = bytes + bytes / 4;
        void *p = nullptr;
        if (w.ptr) CC_CUDA(cudaFreeAsync(w.ptr, stream));
        w.ptr = nullptr;
        w.bytes = 0;
        cudaError_t e = cudaMallocAsync(&p, want, stream);
        if (e != cudaSuccess) return fail(CC_ERR_NOMEM, std::string("cudaMallocAsync: ") + cudaGetErrorString(e));
        // the status word must start cleared
        CC_CUDA(cudaMemsetAsync(p, 0, sizeof(WsHeader), stream));
        w.ptr = p;
        w.bytes = want;
    }
    *out = w.ptr;
    return CC_OK;
}

static bool aligned(const void *p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

static cc_status check_points(const cc_points *p, int64_t n) {
    if (!p) return fail(CC_ERR_INVALID_ARG, "points is NULL");
    if (n < 0) return fail(CC_ERR_INVALID_ARG, "n < 0");
    if (n >= (int64_t(1) << 31) - (int64_t(1) << 22))
        return fail(CC_ERR_INVALID_ARG, "n too large (must be below 2^31 - 2^22)");
    if (p->dtype != CC_I32 && p->dtype != CC_F32) return fail(CC_ERR_INVALID_ARG, "unknown dtype");
    if (n == 0) return CC_OK;
    if (!p->x || !p->y || !p->z) return fail(CC_ERR_INVALID_ARG, "coordinate pointer is NULL");
    if (p->dtype == CC_F32 && !p->r) return fail(CC_ERR_INVALID_ARG, "radius pointer is NULL");
    if (!aligned(p->x, 4) || !aligned(p->y, 4) || !aligned(p->z, 4) ||
        (p->dtype == CC_F32 && !aligned(p->r, 4)))
        return fail(CC_ERR_INVALID_ARG, "coordinate arrays must be 4-byte aligned");
    return CC_OK;
}

}  // namespace cc

using namespace cc;

extern "C" {

const char *cc_status_string(cc_status s) {
    switch (s) {
        case CC_OK: return "CC_OK";
        case CC_ERR_INVALID_ARG: return "CC_ERR_INVALID_ARG";
        case CC_ERR_RANGE: return "CC_ERR_RANGE";
        case CC_ERR_NOMEM: return "CC_ERR_NOMEM";
        case CC_ERR_CUDA: return "CC_ERR_CUDA";
        case CC_ERR_TIMEOUT: return "CC_ERR_TIMEOUT";
        case CC_ERR_BUSY: return "CC_ERR_BUSY";
        case CC_ERR_NOT_FOUND: return "CC_ERR_NOT_FOUND";
    }
    return "CC_ERR_UNKNOWN";
}

const char *cc_last_error(void) { return t_last_error.c_str(); }

const char *cc_version(void) { return "cc 0.1 sm_103a"; }

void cc_set_wait_limit_ns(uint64_t ns) { g_wait_ns.store(ns ? ns : 1); }

void cc_debug_stall_copies(int stall) { g_stall.store(stall ? 1 : 0); }

void cc_profile_enable(int on) { g_prof.store(on != 0); }

cc_status cc_profile_read(double *total_ms, int64_t *launches) {
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev;
    {
        std::lock_guard<std::mutex> lk(g_prof_mu);
        ev.swap(g_prof_pending);
    }
    double tot = 0.0;
    cudaError_t err = cudaSuccess;
    for (auto &p : ev) {
        float ms = 0.f;
        cudaError_t e = cudaEventSynchronize(p.second);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, p.first, p.second);
        if (e != cudaSuccess && err == cudaSuccess) err = e;
        tot += ms;
    }
    {
        std::lock_guard<std::mutex> lk(g_prof_mu);
        for (auto &p : ev) {
            g_prof_pool.push_back(p.first);
            g_prof_pool.push_back(p.second);
        }
    }
    if (total_ms) *total_ms = tot;
    if (launches) *launches = static_cast<int64_t>(ev.size());
    if (err != cudaSuccess) return cuda_fail(err, "cc_profile_read");
    return CC_OK;
}

cc_status cc_reserve(int64_t max_n, void *stream) {
    if (max_n < 0) return fail(CC_ERR_INVALID_ARG, "max_n < 0");
    size_t b = std::max(single_ws_bytes(max_n, true, true), single_ws_bytes(max_n, false, true));
    void *ws = nullptr;
    return workspace_for(static_cast<cudaStream_t>(stream), b, &ws);
}

cc_status cc_release(void *stream) {
    std::lock_guard<std::mutex> lk(g_ws_mu);
    auto it = g_ws.find(static_cast<cudaStream_t>(stream));
    if (it == g_ws.end()) return CC_OK;
    if (it->second.ptr) CC_CUDA(cudaFreeAsync(it->second.ptr, static_cast<cudaStream_t>(stream)));
    g_ws.erase(it);
    return CC_OK;
}

cc_status cc_count_pairs(const cc_points *p, int64_t n, uint32_t r2, unsigned long long *d_count,
                         void *stream) {
    cc_status st = check_points(p, n);
    if (st != CC_OK) return st;
    if (!d_count) return fail(CC_ERR_INVALID_ARG, "d_count is NULL");
    if (!aligned(d_count, 8)) return fail(CC_ERR_INVALID_ARG, "d_count must be 8-byte aligned");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    void *ws = nullptr;
    st = workspace_for(s, single_ws_bytes(n, false, true), &ws);
    if (st != CC_OK) return st;
    return single_enqueue(p, n, r2, d_count, nullptr, ws, s, true);
}

cc_status cc_interaction_sum(const cc_points *p, int64_t n, uint32_t r2, float *d_sum,
                             unsigned long long *d_count, void *stream) {
    cc_status st = check_points(p, n);
    if (st != CC_OK) return st;
    if (!d_sum) return fail(CC_ERR_INVALID_ARG, "d_sum is NULL");
    if (!aligned(d_sum, 4) || (d_count && !aligned(d_count, 8)))
        return fail(CC_ERR_INVALID_ARG, "misaligned output pointer");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    void *ws = nullptr;
    st = workspace_for(s, single_ws_bytes(n, true, true), &ws);
    if (st != CC_OK) return st;
    return single_enqueue(p, n, r2, d_count, d_sum, ws, s, true);
}

cc_status cc_count_pairs_straightforward(const cc_points *p, int64_t n, uint32_t r2,
                                        unsigned long long *d_count, void *stream) {
    cc_status st = check_points(p, n);
    if (st != CC_OK) return st;
    if (!d_count || !aligned(d_count, 8)) return fail(CC_ERR_INVALID_ARG, "d_count is NULL or misaligned");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    void *ws = nullptr;
    st = workspace_for(s, std::max(straight_ws_bytes(n), sizeof(WsHeader)), &ws);
    if (st != CC_OK) return st;
    return straight_enqueue(p, n, r2, d_count, ws, s);
}

static cc_status linear_call(const cc_points *p, int64_t n, int contacts, unsigned long long *d_count,
                             void *stream) {
    cc_status st = check_points(p, n);
    if (st != CC_OK) return st;
    if (p->dtype != CC_I32) return fail(CC_ERR_INVALID_ARG, "the linear-time counts need integer points");
    if (!d_count || !aligned(d_count, 8)) return fail(CC_ERR_INVALID_ARG, "d_count is NULL or misaligned");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    void *ws = nullptr;
    st = workspace_for(s, linear_ws_bytes(n), &ws);
    if (st != CC_OK) return st;
    return linear_enqueue(p, n, contacts, d_count, ws, s);
}

cc_status cc_count_same_site(const cc_points *p, int64_t n, unsigned long long *d_count, void *stream) {
    return linear_call(p, n, 0, d_count, stream);
}

cc_status cc_count_contacts(const cc_points *p, int64_t n, unsigned long long *d_count, void *stream) {
    return linear_call(p, n, 1, d_count, stream);
}

cc_status cc_stream_status(void *stream) {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    void *ws = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_ws_mu);
        auto it = g_ws.find(s);
        if (it == g_ws.end() || !it->second.ptr) {
            CC_CUDA(cudaStreamSynchronize(s));
            return CC_OK;
        }
        ws = it->second.ptr;
    }
    uint32_t status = 0;
    WsHeader *h = reinterpret_cast<WsHeader *>(ws);
    CC_CUDA(cudaMemcpyAsync(&status, &h->status, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    CC_CUDA(cudaMemsetAsync(&h->status, 0, sizeof(uint32_t), s));
    CC_CUDA(cudaStreamSynchronize(s));
    if (status & ST_TIMEOUT) return fail(CC_ERR_TIMEOUT, "a bounded device-side wait ran out");
    if (status & ST_RANGE) return fail(CC_ERR_RANGE, "integer coordinate span above 32767 on some axis");
    return CC_OK;
}

cc_status cc_set_tensor_cores(int32_t enable) {
    tc_set_enabled(enable != 0);
    return CC_OK;
}

cc_status cc_stream_mode(void *stream, int32_t *mode) {
    if (!mode) return fail(CC_ERR_INVALID_ARG, "mode is NULL");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    void *ws = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_ws_mu);
        auto it = g_ws.find(s);
        if (it == g_ws.end() || !it->second.ptr) return fail(CC_ERR_NOT_FOUND, "no call has run on this stream");
        ws = it->second.ptr;
    }
    int32_t m = -1;
    CC_CUDA(cudaMemcpyAsync(&m, &reinterpret_cast<WsHeader *>(ws)->mode, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    CC_CUDA(cudaStreamSynchronize(s));
    *mode = m;
    return CC_OK;
}

cc_status cc_validate_points(const cc_points *p, int64_t n, void *stream) {
    cc_status st = check_points(p, n);
    if (st != CC_OK) return st;
    if (p->dtype == CC_F32 || n < 2) return CC_OK;
    // Runs only the per-axis min/max reduction and reads the device status.
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    st = cc_stream_status(stream);   // clear earlier status
    if (st != CC_OK && st != CC_ERR_RANGE && st != CC_ERR_TIMEOUT) return st;
    void *ws = nullptr;
    st = workspace_for(s, sizeof(WsHeader), &ws);
    if (st != CC_OK) return st;
    st = validate_enqueue(p, n, ws, s);
    if (st != CC_OK) return st;
    return cc_stream_status(stream);
}

}  // extern "C"

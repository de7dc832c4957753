// Serving loop: device-resident sets, count/sum queries admitted by a memory budget and
// a slot limit, continuous batching over two streams.
//
// Requests go into a host queue (thread-safe submit). One scheduler thread owns two
// "lanes"; each lane has its own stream, batching plan (captured graph, work queue) and
// pinned result buffers. Whenever a lane is idle and requests are waiting, the scheduler
// admits as many as the free slots and the memory budget allow, launches them as one
// batch on that lane and goes back to polling; the other lane's batch keeps running
// meanwhile, so requests arriving while the GPU is busy are batched and launched as
// soon as a lane frees up. Results carry host steady-clock timestamps of arrival and of
// completion.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "cc_internal.cuh"

namespace cc {

struct SetDescHost {   // layout identical to the device SetDesc of the batching layer
    const void *x, *y, *z;
    const float *r;
    int64_t n;
    int32_t dtype;
    uint32_t r2;
};

cc_status plan_launch_sets(cc_plan *P, int32_t n_sets, int32_t want_sum, unsigned long long *d_counts,
                           float *d_sums, cudaStream_t s);
size_t single_ws_bytes(int64_t n, bool sum, bool allow_tc);
bool tc_enabled();
// Sets at least this large have their count and sum queries served by the single-set
// path (a tensor-core kernel when the set admits it) instead of the batch.
constexpr int64_t kServerTcMinN = 16384;
// Batches of at most this many requests, all on sets below the single-set path's small-set
// limit, skip the batching graph: each request is one launch of the small-set kernel,
// which for so few requests is sooner done than the graph's six kernels.
constexpr size_t kDirectMaxRequests = 4;
int64_t tc_min_n();
void *plan_sets_buffer_v(cc_plan *P);
size_t plan_set_desc_bytes();

static double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

}  // namespace cc

using namespace cc;

namespace {

struct Req {
    uint64_t req_id;
    int32_t set_id;
    int32_t op;
    uint32_t r2;
    double t_arrive;
    size_t scratch;
};

struct SetRec {
    void *buf = nullptr;    // one allocation: x | y | z | (r)
    int64_t n = 0;
    int32_t dtype = 0;
    size_t bytes = 0;
    int32_t refs = 0;
    bool alive = false;
    bool single = false;    // queries go to the single-set (tensor-core) path
};

struct Lane {
    cudaStream_t stream = nullptr;
    cc_plan *plan = nullptr;
    SetDescHost *h_sets = nullptr;           // pinned
    unsigned long long *d_counts = nullptr;
    float *d_sums = nullptr;
    unsigned long long *h_counts = nullptr;  // pinned
    float *h_sums = nullptr;                 // pinned
    cudaEvent_t done = nullptr;
    std::vector<Req> batch;
    std::vector<int32_t> singles;            // batch entries served by the single-set path
    cc_status fail_status = CC_OK;           // the batch could not be enqueued
    bool busy = false;
    size_t scratch = 0;
};

constexpr int kLanes = 2;
// Points per batch (sizes each lane's work queue: about 200 MB per lane at 2^24); sets
// larger than this always take the single-set route.
constexpr int64_t kPlanMaxPoints = int64_t(1) << 24;

}  // namespace

struct cc_server {
    size_t budget = 0;
    int32_t max_slots = 0;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Req> pending;
    std::atomic<int64_t> npending{0};   // pending.size(), readable without the lock
    std::vector<SetRec> sets;
    size_t resident_bytes = 0;
    size_t inflight_bytes = 0;
    size_t single_ws_reserved = 0;   // budget held for the lanes' single-set workspaces
    int64_t inflight = 0;
    int64_t submitted = 0;
    int64_t finished = 0;
    std::deque<cc_result> done;
    Lane lanes[kLanes];
    std::thread sched;
    bool stop = false;
    int device = 0;
    // stats
    int64_t batches = 0, admitted = 0, peak_inflight = 0, single_launches = 0;
    int64_t peak_bytes = 0;
    std::string sched_error;
};

static size_t req_scratch(int64_t n) {
    // work items and per-item partials of the batching layer (about n/16 + 2 items of
    // 20 bytes) plus the outputs; rounded up generously
    return 256 + static_cast<size_t>(n) * 2;
}

// NVTX ranges mark batch formation/launch and harvesting on the scheduler thread (visible
// in Nsight Systems timelines; no cost when no tool is attached).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};

// Moves a finished batch's results to the done queue. A count of CC_COUNT_INVALID marks a
// device-detected error: on the batched path a set beyond the integer range; on the
// single-set route whichever condition the lane stream's status word recorded (a bounded
// wait that ran out, or the range), read here, off the lock, only when such a count
// appears.
static void harvest(cc_server *S, Lane &L) {
    NvtxRange range("cc_server harvest");
    const double t = now_s();
    cc_status single_err = CC_OK;
    for (int32_t k : L.singles) {
        if (L.h_counts[k] == CC_COUNT_INVALID) {
            single_err = cc_stream_status(L.stream);
            if (single_err == CC_OK) single_err = CC_ERR_RANGE;
            break;
        }
    }
    std::vector<char> is_single(L.batch.size(), 0);
    for (int32_t k : L.singles) is_single[k] = 1;
    std::lock_guard<std::mutex> lk(S->mu);
    for (size_t k = 0; k < L.batch.size(); ++k) {
        const Req &q = L.batch[k];
        cc_result r{};
        r.req_id = q.req_id;
        r.set_id = q.set_id;
        r.op = q.op;
        const unsigned long long c = L.h_counts[k];
        r.status = L.fail_status != CC_OK ? L.fail_status
                   : c != CC_COUNT_INVALID ? CC_OK
                   : (is_single[k] ? single_err : CC_ERR_RANGE);
        r.count = c;
        r.sum = q.op == CC_OP_SUM ? L.h_sums[k] : 0.0f;
        r.t_arrive_s = q.t_arrive;
        r.t_done_s = t;
        S->done.push_back(r);
        S->sets[q.set_id].refs -= 1;
    }
    S->inflight -= static_cast<int64_t>(L.batch.size());
    S->inflight_bytes -= L.scratch;
    S->finished += static_cast<int64_t>(L.batch.size());
    L.batch.clear();
    L.singles.clear();
    L.fail_status = CC_OK;
    L.scratch = 0;
    L.busy = false;
    S->cv.notify_all();
}

// Forms one batch on lane L under S->mu (admission, descriptors), then enqueues its copies,
// graph launch and single-set calls with the lock released, so that client submit() and
// poll() never wait for CUDA calls. Only the scheduler thread touches L, and an admitted
// request holds a reference on its set, so the set's buffers stay valid meanwhile.
static bool launch(cc_server *S, Lane &L) {
    NvtxRange range("cc_server form+launch batch");
    std::vector<Req> batch;
    std::vector<cc_points> single_pts;   // points of the single-set entries (same order as L.singles)
    std::vector<int64_t> single_n;
    size_t scratch = 0;
    int64_t points = 0;
    bool any_sum = false;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        while (!S->pending.empty()) {
            const Req &q = S->pending.front();
            if (S->inflight + static_cast<int64_t>(batch.size()) >= S->max_slots) break;
            const size_t need = S->resident_bytes + S->inflight_bytes + scratch + q.scratch;
            if (need > S->budget && !(batch.empty() && S->inflight == 0)) break;
            const int64_t n = S->sets[q.set_id].n;
            if (!batch.empty() && points + n > kPlanMaxPoints) break;
            batch.push_back(q);
            scratch += q.scratch;
            points += n;
            S->pending.pop_front();
            S->npending.fetch_sub(1);
        }
        if (batch.empty()) return false;
        // a few requests on small sets: one small-set kernel launch each, no graph
        bool direct = batch.size() <= kDirectMaxRequests;
        for (size_t k = 0; direct && k < batch.size(); ++k) direct = S->sets[batch[k].set_id].n < tc_min_n();
        S->inflight += static_cast<int64_t>(batch.size());
        S->inflight_bytes += scratch;
        S->admitted += static_cast<int64_t>(batch.size());
        S->batches += 1;
        S->peak_inflight = std::max(S->peak_inflight, S->inflight);
        S->peak_bytes = std::max<int64_t>(S->peak_bytes, static_cast<int64_t>(S->resident_bytes + S->inflight_bytes));
        L.singles.clear();
        for (size_t k = 0; k < batch.size(); ++k) {
            const SetRec &sr = S->sets[batch[k].set_id];
            SetDescHost d;
            const size_t col = static_cast<size_t>(sr.n) * 4;
            d.x = sr.buf;
            d.y = static_cast<char *>(sr.buf) + col;
            d.z = static_cast<char *>(sr.buf) + 2 * col;
            d.r = sr.dtype == CC_F32 ? reinterpret_cast<const float *>(static_cast<char *>(sr.buf) + 3 * col) : nullptr;
            d.n = sr.n;
            d.dtype = sr.dtype;
            d.r2 = batch[k].r2;
            if (sr.single || direct) {
                cc_points pts;
                pts.dtype = sr.dtype;
                pts.x = d.x;
                pts.y = d.y;
                pts.z = d.z;
                pts.r = d.r;
                single_pts.push_back(pts);
                single_n.push_back(sr.n);
                d.n = 0;   // the batch writes 0; the single-set call below writes the result
                L.singles.push_back(static_cast<int32_t>(k));
            }
            L.h_sets[k] = d;
            any_sum = any_sum || batch[k].op == CC_OP_SUM;
        }
        S->single_launches += static_cast<int64_t>(L.singles.size());
    }
    L.batch = std::move(batch);
    L.scratch = scratch;
    L.busy = true;
    const int32_t nb = static_cast<int32_t>(L.batch.size());
    cudaError_t e = cudaSuccess;
    cc_status st = CC_OK;
    if (L.singles.size() < L.batch.size()) {   // some entries run in the batching graph
        e = cudaMemcpyAsync(plan_sets_buffer_v(L.plan), L.h_sets, sizeof(SetDescHost) * nb, cudaMemcpyHostToDevice,
                            L.stream);
        st = e == cudaSuccess ? plan_launch_sets(L.plan, nb, any_sum ? 1 : 0, L.d_counts, L.d_sums, L.stream)
                              : CC_ERR_CUDA;
    }
    // queries on large sets: one single-set call each, stream-ordered after the batch
    // (this thread is the lane stream's only user, so its workspace is too)
    for (size_t j = 0; st == CC_OK && j < L.singles.size(); ++j) {
        const int32_t k = L.singles[j];
        st = L.batch[k].op == CC_OP_SUM
                 ? cc_interaction_sum(&single_pts[j], single_n[j], L.batch[k].r2, L.d_sums + k, L.d_counts + k, L.stream)
                 : cc_count_pairs(&single_pts[j], single_n[j], L.batch[k].r2, L.d_counts + k, L.stream);
    }
    if (st == CC_OK) e = cudaMemcpyAsync(L.h_counts, L.d_counts, sizeof(unsigned long long) * nb,
                                         cudaMemcpyDeviceToHost, L.stream);
    if (st == CC_OK && e == cudaSuccess && any_sum)
        e = cudaMemcpyAsync(L.h_sums, L.d_sums, sizeof(float) * nb, cudaMemcpyDeviceToHost, L.stream);
    if (st == CC_OK && e == cudaSuccess) e = cudaEventRecord(L.done, L.stream);
    if (st != CC_OK || e != cudaSuccess) {
        const std::string msg = std::string("batch launch failed: ") + cudaGetErrorString(e) + " " + cc_last_error();
        cudaStreamSynchronize(L.stream);
        for (size_t k = 0; k < L.batch.size(); ++k) L.h_counts[k] = CC_COUNT_INVALID;
        L.fail_status = st != CC_OK ? st : CC_ERR_CUDA;   // every entry of this batch reports it
        cudaEventRecord(L.done, L.stream);
        std::lock_guard<std::mutex> lk(S->mu);
        S->sched_error = msg;
    }
    return true;
}

// The scheduler thread. While a lane's batch runs it polls the lanes' completion events
// (and, with a lane idle, the request queue) without sleeping for up to 200 us, so that a
// finished batch is harvested and a new request launched within a few microseconds; it
// sleeps on the condition variable only after that, or when nothing is in flight.
static void scheduler(cc_server *S) {
    cudaSetDevice(S->device);
    for (;;) {
        bool progressed = false;
        for (Lane &L : S->lanes) {
            if (L.busy && cudaEventQuery(L.done) == cudaSuccess) {
                harvest(S, L);
                progressed = true;
            }
        }
        bool tried = false;   // a launch was attempted and admitted nothing
        for (Lane &L : S->lanes) {
            if (!L.busy) {
                if (launch(S, L)) progressed = true;
                else tried = true;
            }
        }
        if (progressed) continue;
        if (S->lanes[0].busy || S->lanes[1].busy) {
            // with a lane idle, a new request is worth a launch attempt, unless the one just
            // made admitted nothing (slots or budget exhausted): then only a finishing batch
            // changes anything, and polling the queue would contend for the lock
            const int64_t seen = S->npending.load();
            const bool idle_lane = !S->lanes[0].busy || !S->lanes[1].busy;
            const auto t0 = std::chrono::steady_clock::now();
            for (;;) {
                bool done = false;
                for (Lane &L : S->lanes) done = done || (L.busy && cudaEventQuery(L.done) == cudaSuccess);
                const int64_t np = S->npending.load();
                if (done || (idle_lane && np > 0 && (!tried || np > seen))) break;
                if (std::chrono::steady_clock::now() - t0 > std::chrono::microseconds(200)) {
                    std::unique_lock<std::mutex> lk(S->mu);
                    S->cv.wait_for(lk, std::chrono::microseconds(20));
                    break;
                }
                std::this_thread::yield();
            }
            continue;
        }
        std::unique_lock<std::mutex> lk(S->mu);
        if (S->stop && S->pending.empty() && S->inflight == 0) return;
        if (S->pending.empty() && !S->stop) S->cv.wait_for(lk, std::chrono::milliseconds(2));
    }
}

extern "C" {

cc_status cc_server_create(cc_server **srv, size_t mem_budget_bytes, int32_t max_slots) {
    return cc_server_create_tuned(srv, mem_budget_bytes, max_slots, nullptr);
}

cc_status cc_server_create_tuned(cc_server **srv, size_t mem_budget_bytes, int32_t max_slots,
                                 const char *tune_table_json) {
    if (!srv) return fail(CC_ERR_INVALID_ARG, "srv is NULL");
    *srv = nullptr;
    if (max_slots <= 0 || max_slots > 65536) return fail(CC_ERR_INVALID_ARG, "max_slots must be in 1..65536");
    if (mem_budget_bytes == 0) return fail(CC_ERR_INVALID_ARG, "zero memory budget");
    cc_server *S = new cc_server();
    S->budget = mem_budget_bytes;
    S->max_slots = max_slots;
    cudaGetDevice(&S->device);
    for (Lane &L : S->lanes) {
        cudaError_t e = cudaStreamCreateWithFlags(&L.stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&L.done, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void **>(&L.h_sets), sizeof(SetDescHost) * max_slots);
        if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void **>(&L.h_counts), 8 * max_slots);
        if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void **>(&L.h_sums), 4 * max_slots);
        if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void **>(&L.d_counts), 8 * max_slots);
        if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void **>(&L.d_sums), 4 * max_slots);
        if (e != cudaSuccess) {
            cc_server_destroy(S);
            return fail(CC_ERR_NOMEM, std::string("server allocation: ") + cudaGetErrorString(e));
        }
        cc_status st = cc_plan_create(&L.plan, tune_table_json, max_slots, kPlanMaxPoints);
        if (st != CC_OK) {
            cc_server_destroy(S);
            return st;
        }
    }
    S->sched = std::thread(scheduler, S);
    *srv = S;
    return CC_OK;
}

cc_status cc_server_register_set(cc_server *S, const cc_points *p, int64_t n, int32_t *set_id) {
    if (!S || !p || !set_id) return fail(CC_ERR_INVALID_ARG, "NULL argument");
    if (n < 0 || n >= (int64_t(1) << 31)) return fail(CC_ERR_INVALID_ARG, "n out of range");
    if (p->dtype != CC_I32 && p->dtype != CC_F32) return fail(CC_ERR_INVALID_ARG, "unknown dtype");
    if (n > 0 && (!p->x || !p->y || !p->z || (p->dtype == CC_F32 && !p->r)))
        return fail(CC_ERR_INVALID_ARG, "NULL coordinate pointer");
    const int cols = p->dtype == CC_F32 ? 4 : 3;
    const size_t col = static_cast<size_t>(n) * 4;
    const size_t bytes = std::max<size_t>(col * cols, 16);
    bool single = false;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->resident_bytes + S->inflight_bytes + bytes > S->budget)
            return fail(CC_ERR_NOMEM, "memory budget exceeded by this set");
        S->resident_bytes += bytes;
        if (n >= kServerTcMinN && (tc_enabled() || n > kPlanMaxPoints)) {
            // both lanes may hold a workspace of this size (allocated by the scheduler on
            // first use); without room in the budget the set stays on the batched path,
            // unless it is too large for a batch
            const size_t need = 2 * std::max(single_ws_bytes(n, false, true), single_ws_bytes(n, true, true));
            const size_t extra = need > S->single_ws_reserved ? need - S->single_ws_reserved : 0;
            if (S->resident_bytes + S->inflight_bytes + extra <= S->budget) {
                S->resident_bytes += extra;
                S->single_ws_reserved += extra;
                single = true;
            } else if (n > kPlanMaxPoints) {
                S->resident_bytes -= bytes;
                return fail(CC_ERR_NOMEM, "memory budget too small for the workspace of a set this large");
            }
        }
    }
    void *buf = nullptr;
    cudaError_t e = cudaMalloc(&buf, bytes);
    if (e != cudaSuccess) {
        std::lock_guard<std::mutex> lk(S->mu);
        S->resident_bytes -= bytes;
        return fail(CC_ERR_NOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    const void *src[4] = {p->x, p->y, p->z, p->r};
    for (int c = 0; c < cols && n > 0; ++c) {
        e = cudaMemcpy(static_cast<char *>(buf) + c * col, src[c], col, cudaMemcpyDefault);
        if (e != cudaSuccess) {
            cudaFree(buf);
            std::lock_guard<std::mutex> lk(S->mu);
            S->resident_bytes -= bytes;
            return cuda_fail(e, "cudaMemcpy (register set)");
        }
    }
    std::lock_guard<std::mutex> lk(S->mu);
    SetRec r;
    r.buf = buf;
    r.n = n;
    r.dtype = p->dtype;
    r.bytes = bytes;
    r.alive = true;
    r.single = single;
    S->sets.push_back(r);
    *set_id = static_cast<int32_t>(S->sets.size() - 1);
    S->peak_bytes = std::max<int64_t>(S->peak_bytes, static_cast<int64_t>(S->resident_bytes + S->inflight_bytes));
    return CC_OK;
}

cc_status cc_server_unregister_set(cc_server *S, int32_t set_id) {
    if (!S) return fail(CC_ERR_INVALID_ARG, "NULL server");
    void *buf = nullptr;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (set_id < 0 || set_id >= static_cast<int32_t>(S->sets.size()) || !S->sets[set_id].alive)
            return fail(CC_ERR_NOT_FOUND, "unknown set id");
        SetRec &r = S->sets[set_id];
        if (r.refs > 0) return fail(CC_ERR_BUSY, "set is used by admitted or queued requests");
        buf = r.buf;
        S->resident_bytes -= r.bytes;
        r.alive = false;
        r.buf = nullptr;
    }
    cudaError_t e = cudaFree(buf);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFree (unregister set)");
    return CC_OK;
}

cc_status cc_server_submit(cc_server *S, int32_t set_id, int32_t op, uint32_t r2, uint64_t req_id) {
    if (!S) return fail(CC_ERR_INVALID_ARG, "NULL server");
    if (op != CC_OP_COUNT && op != CC_OP_SUM) return fail(CC_ERR_INVALID_ARG, "unknown op");
    const double t = now_s();
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stop) return fail(CC_ERR_BUSY, "server is stopping");
    if (set_id < 0 || set_id >= static_cast<int32_t>(S->sets.size()) || !S->sets[set_id].alive)
        return fail(CC_ERR_NOT_FOUND, "unknown set id");
    SetRec &r = S->sets[set_id];
    r.refs += 1;
    S->pending.push_back(Req{req_id, set_id, op, r2, t, req_scratch(r.n)});
    S->npending.fetch_add(1);
    S->submitted += 1;
    S->cv.notify_all();
    return CC_OK;
}

cc_status cc_server_poll(cc_server *S, cc_result *out, int32_t max, int32_t *n_out) {
    if (!S || !n_out || (max > 0 && !out)) return fail(CC_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(S->mu);
    int32_t k = 0;
    while (k < max && !S->done.empty()) {
        out[k++] = S->done.front();
        S->done.pop_front();
    }
    *n_out = k;
    if (!S->sched_error.empty()) return fail(CC_ERR_CUDA, S->sched_error);
    return CC_OK;
}

cc_status cc_server_drain(cc_server *S, double timeout_s) {
    if (!S) return fail(CC_ERR_INVALID_ARG, "NULL server");
    std::unique_lock<std::mutex> lk(S->mu);
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::duration<double>(timeout_s);
    while (S->finished < S->submitted) {
        if (S->cv.wait_until(lk, deadline) == std::cv_status::timeout && S->finished < S->submitted)
            return fail(CC_ERR_TIMEOUT, "drain timed out");
    }
    return CC_OK;
}

cc_status cc_server_stats(cc_server *S, int64_t *batches, int64_t *admitted, int64_t *peak_inflight,
                          int64_t *peak_bytes) {
    if (!S) return fail(CC_ERR_INVALID_ARG, "NULL server");
    std::lock_guard<std::mutex> lk(S->mu);
    if (batches) *batches = S->batches;
    if (admitted) *admitted = S->admitted;
    if (peak_inflight) *peak_inflight = S->peak_inflight;
    if (peak_bytes) *peak_bytes = S->peak_bytes;
    return CC_OK;
}

void cc_server_destroy(cc_server *S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
        S->cv.notify_all();
    }
    if (S->sched.joinable()) S->sched.join();
    for (Lane &L : S->lanes) {
        if (L.stream) cudaStreamSynchronize(L.stream);
        if (L.plan) cc_plan_destroy(L.plan);
        if (L.done) cudaEventDestroy(L.done);
        if (L.h_sets) cudaFreeHost(L.h_sets);
        if (L.h_counts) cudaFreeHost(L.h_counts);
        if (L.h_sums) cudaFreeHost(L.h_sums);
        if (L.d_counts) cudaFree(L.d_counts);
        if (L.d_sums) cudaFree(L.d_sums);
        if (L.stream) cudaStreamDestroy(L.stream);
    }
    for (SetRec &r : S->sets)
        if (r.alive && r.buf) cudaFree(r.buf);
    delete S;
}

}  // extern "C"

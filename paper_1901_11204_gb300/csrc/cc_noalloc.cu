// cc_count_pairs_noalloc: the single-set count for callers that must not allocate.
//
// Some callers cannot call cudaMalloc (or any allocating routine) at the point where
// they need a count: code that records work into a CUDA graph, engines whose memory is
// owned by one allocator that forbids side allocations, processes that run with a fixed
// device-memory budget and must not fail half-way on an allocation, or latency-critical
// loops that keep allocation out of their steady state. This entry point serves them: it
// runs the same kernels as cc_count_pairs, but its scratch memory is one file-scope
// device array of fixed size, so a call allocates nothing.
//
// The array (kNoAllocScratchBytes) is part of the library image: every GPU that loads
// the library holds it until the process exits. Its device address is looked up once
// per device with cudaGetSymbolAddress; in host code the array's name is only a host-side
// stand-in and is never handed to a kernel.
#include <cuda_runtime.h>

#include <mutex>
#include <string>
#include <unordered_map>

#include "cc_internal.cuh"

namespace cc {

size_t single_ws_bytes(int64_t n, bool sum, bool allow_tc);
cc_status single_enqueue(const cc_points *p, int64_t n, uint32_t r2, unsigned long long *d_count,
                         float *d_sum, void *ws, cudaStream_t stream, bool allow_tc);

// 8 MiB of scratch: enough for sets of about 349 thousand objects (the extended record
// array of 32 bytes per pair of objects, per-CTA slots and the header).
constexpr size_t kNoAllocScratchBytes = size_t(8) << 20;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

namespace {
std::mutex g_noalloc_mu;
std::unordered_map<int, void *> g_noalloc_addr;   // device ordinal -> device address
}  // namespace

// Device address of the scratch array on the current device (set up on first use).
static cc_status noalloc_scratch(void **out) {
    int dev = 0;
    CC_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    auto it = g_noalloc_addr.find(dev);
    if (it != g_noalloc_addr.end()) {
        *out = it->second;
        return CC_OK;
    }
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) return cuda_fail(e, "cudaGetSymbolAddress(noalloc scratch)");
    g_noalloc_addr.emplace(dev, p);
    *out = p;
    return CC_OK;
}

// Largest set size whose workspace fits in the scratch array (computed once; function-
// local static initialisation is thread-safe).
static int64_t noalloc_max_n() {
    static const int64_t cached = []() {
        int64_t lo = 1, hi = int64_t(1) << 26;
        while (lo < hi) {
            const int64_t mid = lo + (hi - lo + 1) / 2;
            const size_t b = single_ws_bytes(mid, false, false);
            if (b != 0 && b <= kNoAllocScratchBytes) lo = mid;
            else hi = mid - 1;
        }
        return lo;
    }();
    return cached;
}

}  // namespace cc

using namespace cc;

extern "C" {

cc_status cc_count_pairs_noalloc(const cc_points *p, int64_t n, uint32_t r2, unsigned long long *d_count,
                                 void *stream) {
    if (!p) return fail(CC_ERR_INVALID_ARG, "points is NULL");
    if (!d_count || (reinterpret_cast<uintptr_t>(d_count) & 7))
        return fail(CC_ERR_INVALID_ARG, "d_count is NULL or not 8-byte aligned");
    if (n < 0) return fail(CC_ERR_INVALID_ARG, "n < 0");
    if (p->dtype != CC_I32 && p->dtype != CC_F32) return fail(CC_ERR_INVALID_ARG, "unknown dtype");
    if (n > 0 && (!p->x || !p->y || !p->z || (p->dtype == CC_F32 && !p->r)))
        return fail(CC_ERR_INVALID_ARG, "coordinate pointer is NULL");
    const int64_t max_n = noalloc_max_n();
    if (n > max_n)
        return fail(CC_ERR_INVALID_ARG, "n = " + std::to_string(n) + " exceeds the no-allocation limit of " +
                                            std::to_string(max_n) + " objects (" +
                                            std::to_string(kNoAllocScratchBytes >> 20) + " MiB static scratch)");
    void *ws = nullptr;
    cc_status st = noalloc_scratch(&ws);
    if (st != CC_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // The header's status word keeps the previous call's bits: start each call from zero.
    // A condition the device detects for this call (integer span beyond the range, a
    // bounded wait that ran out) makes the call's last kernel write CC_COUNT_INVALID.
    CC_CUDA(cudaMemsetAsync(&reinterpret_cast<WsHeader *>(ws)->status, 0, sizeof(uint32_t), s));
    // the tensor-core operands would need about three times the scratch: the static
    // array serves the FP32-pipe kernels only
    return single_enqueue(p, n, r2, d_count, nullptr, ws, s, false);
}

}  // extern "C"

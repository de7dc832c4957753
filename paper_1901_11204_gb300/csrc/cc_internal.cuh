// Internal declarations shared by the library's translation units (not installed).
//
// Device helpers: Blackwell bulk-copy (TMA engine, non-tensor form) with mbarrier
// completion, bounded mbarrier waits, and packed FP32x2 arithmetic (sm_100+ PTX
// add/sub/mul/fma .f32x2), all written as inline PTX.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/cc.h"

namespace cc {

// ---------------------------------------------------------------------------------------
// error plumbing (host)
// ---------------------------------------------------------------------------------------
void set_error(const std::string &msg);
cc_status fail(cc_status s, const std::string &msg);
cc_status cuda_fail(cudaError_t e, const char *what);

#define CC_CUDA(call)                                              \
    do {                                                           \
        cudaError_t e__ = (call);                                  \
        if (e__ != cudaSuccess) return ::cc::cuda_fail(e__, #call); \
    } while (0)

uint64_t wait_limit_ns();
// Benchmark timing hook: true while cc_profile_enable(1); record_profiled_launch() is
// called with the events bracketing one launch.
bool profiling();
cudaError_t profile_begin(cudaStream_t s, cudaEvent_t *e0, cudaEvent_t *e1);
void profile_end(cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1);
int debug_stall();
int sm_count();

// ---------------------------------------------------------------------------------------
// device status bits (accumulated with atomicOr in the workspace header)
// ---------------------------------------------------------------------------------------
enum : uint32_t { ST_RANGE = 1u, ST_TIMEOUT = 2u };

// Single-set execution modes chosen on the device by the preparation kernel.
enum : int32_t {
    MODE_I32_FAST = 0,   // centred int coordinates as exact FP32, expanded-square form
    MODE_I32_WIDE = 1,   // int32 difference form (spans up to 32767)
    MODE_RANGE_ERR = 2,  // span above 32767: nothing is counted
    MODE_F32 = 3,        // FP32 spheres
    MODE_I32_TC = 4,     // fast exact form as a TF32 tensor-core contraction
    MODE_F32_TC = 5      // FP32 spheres: exact integer screen on the tensor cores, then the
                         // FP32 predicate for the screened pairs
};

// Cells of the occupancy histogram (16 per axis over the bounding box) from which the
// integer tensor-core path estimates its expected hits per pair.
constexpr int TC_HIST_CELLS = 16 * 16 * 16;
constexpr int TC_HIST_STRIDE = 8;   // one object in 8 enters the histogram
// Expected hits per pair below which the integer tensor-core count walks hit blocks
// instead of counting every block in registers (the measured crossover lies between
// 1e-7 and 3e-5 hits per pair on uniform sets).
constexpr double TC_SPARSE_HITS = 2e-6;

// Workspace header: lives at the start of each stream's scratch buffer.
struct WsHeader {
    uint32_t umin[3];     // order-preserving encodings of the per-axis minimum
    uint32_t umax[3];     // ... and maximum
    int32_t mode;         // MODE_*
    int32_t cx, cy, cz;   // integer centre subtracted before the FP32 conversion
    uint32_t r2e;         // r2 clamped to the largest possible squared distance
    int32_t ai_off;       // r2e + 1 (used as n_i - ai_off), exact in FP32
    uint32_t ticket0;     // last-block ticket of the min/max reduction
    uint32_t ticket1;     // last-block ticket of the sum reduction
    uint32_t status;      // ST_* bits since the last cc_stream_status()
    float qmin[3];        // FP32 spheres, tensor-core screen: per-axis minimum coordinate
    uint32_t qbad;        // ... non-zero when a coordinate or radius is not finite
    uint32_t qrmax;       // ... largest |radius| (bits of a non-negative float)
    double qscale;        // ... quantisation scale, 2046 / the largest per-axis span
    int32_t tc_form;      // integer tensor-core count: 0 = count blocks in registers,
                          // 1 = walk the (rare) blocks with a hit (sparse hits expected)
    uint32_t cstatus;     // ST_* bits of the current call only (cleared by each call's
                          // reset); a non-zero value invalidates the call's outputs
    uint32_t sticket;     // small-set kernel: last-CTA ticket (0 between calls)
    uint32_t pad[7];
};
static_assert(sizeof(WsHeader) == 128, "header size");
static_assert(int{MODE_I32_FAST} == int{CC_MODE_FP32_EXACT} && int{MODE_I32_WIDE} == int{CC_MODE_INT_WIDE} &&
                  int{MODE_RANGE_ERR} == int{CC_MODE_RANGE_ERROR} && int{MODE_F32} == int{CC_MODE_FP32_SPHERES} &&
                  int{MODE_I32_TC} == int{CC_MODE_TENSOR} && int{MODE_F32_TC} == int{CC_MODE_TENSOR_SPHERES},
              "device modes are the public CC_MODE_* values");

// Largest half-span m = ceil(span/2) for which the FP32 expanded-square form is exact:
// every partial |n_j - 2 p_i.p_j| <= 9 m^2 and |n_i - r2e - 1| <= 12 m^2 + 1 stay
// below 2^24.
constexpr int32_t FAST_MAX_HALF_SPAN = 1182;
// Tensor-core form: exact when the absolute values of the eight TF32 terms of
// d^2 - r2e - 1 sum to less than 2^24 (every partial sum is then an exact FP32 integer):
//   6 m^2 (three -2 p_i p_j products) + 3 m^2 (|p_j|^2 as two digits)
//   + |n_i - r2e - 1| (<= max(r2e + 1, 3 m^2)) + 2^22 + 2^11 (slack of the balanced digits).
__host__ __device__ inline bool tc_exact(int64_t m, int64_t r2e) {
    const int64_t m2 = m * m;
    const int64_t c = (r2e + 1) > 3 * m2 ? (r2e + 1) : 3 * m2;
    return 9 * m2 + c + (int64_t{1} << 22) + 2048 < (int64_t{1} << 24);
}
// Integer precondition: per-axis span such that the squared distance fits in u32.
constexpr int32_t WIDE_MAX_SPAN = 32767;

// Tile configuration of the single-set kernel.
struct SingleCfg {
    int nt;      // consumer threads per CTA (multiple of 32)
    int r;       // objects per consumer thread
    int js;      // objects per staged j-stage (even)
    int ns;      // pipeline depth (stages in shared memory)
};

// ---------------------------------------------------------------------------------------
// device helpers
// ---------------------------------------------------------------------------------------
#ifdef __CUDACC__

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile(
        "mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
        "r"(bytes)
        : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// One try_wait with a suspend-time hint: the warp sleeps until the phase completes or the
// hint (ns) elapses, instead of spinning on the barrier word.
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity, uint32_t hint_ns) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(hint_ns)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Waits for phase `parity` of *bar to complete, at most limit_ns nanoseconds (measured
// with the global timer), or until *abort becomes non-zero. Returns false when the
// bound ran out or the wait was aborted.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, uint64_t limit_ns,
                                                  const volatile int *abort = nullptr) {
    if (mbar_try_wait(bar, parity, 20000u)) return true;
    const uint64_t t0 = globaltimer_ns();
    for (;;) {
        if (mbar_try_wait(bar, parity, 200000u)) return true;
        if (abort && *abort) return false;
        if (globaltimer_ns() - t0 > limit_ns) return false;
    }
}

// Waits for phase `parity` like mbar_wait_bounded, with try_wait's own (system-defined)
// suspend time instead of a hint: the warp leaves the issue slots to the other warps of
// its SMSP and resumes when the phase completes.
__device__ __forceinline__ bool mbar_try_wait_nohint(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool mbar_sleep_bounded(uint64_t *bar, uint32_t parity, uint64_t limit_ns,
                                                   const volatile int *abort = nullptr) {
    if (mbar_try_wait_nohint(bar, parity)) return true;
    const uint64_t t0 = globaltimer_ns();
    for (;;) {
        if (mbar_try_wait_nohint(bar, parity)) return true;
        if (abort && *abort) return false;
        if (globaltimer_ns() - t0 > limit_ns) return false;
    }
}

// Non-blocking test of phase `parity` (never suspends the thread).
__device__ __forceinline__ bool mbar_test_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Like mbar_wait_bounded, but polls without suspending: for waits on the critical path
// of a short pipeline, where the wake-up latency of a suspended wait would dominate.
// The global timer and the abort flag are read every 256 polls.
__device__ __forceinline__ bool mbar_spin_bounded(uint64_t *bar, uint32_t parity, uint64_t limit_ns,
                                                  const volatile int *abort = nullptr) {
    if (mbar_test_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer_ns();
    for (;;) {
#pragma unroll 1
        for (int k = 0; k < 256; ++k)
            if (mbar_test_wait(bar, parity)) return true;
        if (abort && *abort) return false;
        if (globaltimer_ns() - t0 > limit_ns) return false;
    }
}

// Orders this thread's earlier generic-proxy shared-memory accesses before later
// async-proxy (bulk copy) accesses.
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// 1-D bulk copy global -> shared, completion signalled on *bar (complete_tx bytes).
// dst, src 16-byte aligned and bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes,
                                         uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Packed FP32x2 arithmetic (two lanes in one 64-bit register; low word = lane 0).
// Round to nearest even, no flush to zero, no contraction beyond the explicit fma.
typedef unsigned long long f2;

__device__ __forceinline__ f2 f2_fma(f2 a, f2 b, f2 c) {
    f2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ f2 f2_add(f2 a, f2 b) {
    f2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 f2_sub(f2 a, f2 b) {
    f2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 f2_mul(f2 a, f2 b) {
    f2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 f2_dup(float v) {
    uint32_t u = __float_as_uint(v);
    return (static_cast<f2>(u) << 32) | u;
}
__device__ __forceinline__ float f2_lo(f2 v) { return __uint_as_float(static_cast<uint32_t>(v)); }
__device__ __forceinline__ float f2_hi(f2 v) {
    return __uint_as_float(static_cast<uint32_t>(v >> 32));
}

// Order-preserving unsigned encoding of int32 (for atomicMin/atomicMax on u32).
__device__ __forceinline__ uint32_t ord_enc(int32_t v) { return static_cast<uint32_t>(v) ^ 0x80000000u; }
__device__ __forceinline__ int32_t ord_dec(uint32_t u) { return static_cast<int32_t>(u ^ 0x80000000u); }
// Order-preserving encoding of a finite float (larger float, larger code) and its inverse.
__device__ __forceinline__ uint32_t ord_enc_f(float f) {
    const uint32_t b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float ord_dec_f(uint32_t u) {
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7FFFFFFFu) : ~u);
}

// Records a device-detected condition (ST_* bits) for the current call and for
// cc_stream_status(): the call's outputs are invalidated by its finalisation.
__device__ __forceinline__ void flag_status(WsHeader *h, uint32_t bits) {
    atomicOr(&h->status, bits);
    atomicOr(&h->cstatus, bits);
}

#endif  // __CUDACC__

}  // namespace cc

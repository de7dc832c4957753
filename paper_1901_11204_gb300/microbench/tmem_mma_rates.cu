// Rates that bound the tensor-core pair kernel, measured with one CTA on every SM:
//  (1) TMEM -> register reads in the kernel's load shape: W warps (W/4 per TMEM lane
//      quarter) each loop over tcgen05.ld.red.sync.aligned.32x32b.x{32,64,128}.min (the
//      accumulator values and their minimum), tcgen05.wait::ld and a warp vote on the
//      minimum; bytes read per SM clock (clock64 over 4000 loads, all warps, mean over SMs);
//  (2) tcgen05.mma kind::tf32 M=128 N=256 K=8 (the kernel's shape) issued back to back by
//      one thread into alternating accumulators, one commit at the end: SM clocks per MMA;
//  (3) the accumulator hand-over loop alone, for several accumulator splits and one or two
//      issuing threads (k_handover);
//  (4) the cost of a shared-memory read that the next MMA issue waits for (k_dep).
// Output: one JSON line. Build and run: python -m paper_1901_11204_gb300.microbench
#include <cuda_runtime.h>
#include <cstdio>
#include <cstdint>
#include "../csrc/cc_internal.cuh"
#include "../csrc/cc_tcgen05.cuh"
using namespace cc;

template <int C, int WARPS>
__global__ void __launch_bounds__(WARPS * 32, 1) k_read(int iters, unsigned long long *cycles, float *sink) {
    __shared__ uint32_t tslot;
    const int warp = threadIdx.x >> 5;
    if (warp == 0) { tmem_alloc(&tslot, 512); tmem_relinquish(); }
    tc_fence_before(); __syncthreads(); tc_fence_after();
    const uint32_t tb = tslot;
    const int quarter = warp & 3;
    const uint32_t lane_addr = (uint32_t)(quarter * 32) << 16;
    const int nw = blockDim.x >> 5;
    const int per_q = nw / 4;                 // warps per lane quarter
    const int slice = (warp >> 2);            // which column slice this warp reads
    float acc = 0.f;
    __syncthreads();
    const unsigned long long t0 = clock64();
    for (int it = 0; it < iters; ++it) {
        uint32_t v[C];
        const uint32_t col = (uint32_t)((slice * C + it * C * per_q) & 511);
        const float mn = tmem_ld_min<C>(tb + lane_addr + col, v);
        acc += __any_sync(0xFFFFFFFFu, mn < -1e30f) ? 1.f : 0.f;
        acc += __uint_as_float(v[0]) * 0.f;
    }
    const unsigned long long t1 = clock64();
    __syncthreads();
    if ((threadIdx.x & 31) == 0) atomicMax(&cycles[blockIdx.x], t1 - t0);
    if (acc == 12345.f) sink[0] = acc;
    tc_fence_before(); __syncthreads();
    if (warp == 0) { tc_fence_after(); tmem_dealloc(tb, 512); }
}

template <int N, bool EACH>
__global__ void k_mma(int iters, unsigned long long *cycles) {
    extern __shared__ __align__(1024) uint8_t sm[];
    __shared__ uint32_t tslot;
    __shared__ __align__(8) uint64_t done, each;
    const int warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) { mbar_init(&done, 1); mbar_init(&each, 1); fence_mbar_init(); }
    for (int i = threadIdx.x; i < 16384; i += blockDim.x) reinterpret_cast<uint32_t *>(sm)[i] = 0u;
    if (warp == 0) { tmem_alloc(&tslot, 512); tmem_relinquish(); }
    fence_proxy_async_smem();
    tc_fence_before(); __syncthreads(); tc_fence_after();
    const uint32_t tb = tslot;
    if (threadIdx.x == 32) {
        const uint64_t ad = smem_desc_k_noswizzle(smem_u32(sm), 128, 256);
        const uint64_t bd = smem_desc_k_noswizzle(smem_u32(sm + 4096), 128, 256);
        const uint32_t idesc = idesc_tf32_f32(128, N);
        const unsigned long long t0 = clock64();
        for (int it = 0; it < iters; ++it) {
            tc_mma_tf32(tb + (uint32_t)((it & 1) * 256), ad, bd, idesc, 0u);
            // a barrier nobody waits on: each commit completes one of its phases
            if constexpr (EACH) tc_commit(&each);
        }
        tc_commit(&done);
        (void)mbar_wait_bounded(&done, 0u, 2000000000ull);
        const unsigned long long t1 = clock64();
        cycles[blockIdx.x] = t1 - t0;
    }
    tc_fence_before(); __syncthreads();
    if (warp == 0) { tc_fence_after(); tmem_dealloc(tb, 512); }
}

// (3) The accumulator hand-over loop of the pair kernel with nothing else in it: NMT
//     threads (lane 0 of warp 0, and of warps EPW+1.. for NMT > 1) issue one M=128 N=NCOL
//     K=8 MMA per unit, thread k the units u = k mod NMT, into NB rotating accumulators, and
//     commit each to t_full[b]; EPW epilogue warps (warps 1..EPW, EPW/4 per lane quarter,
//     each owning a column part) wait for t_full[b], load their part with
//     tcgen05.ld.red...min (LOAD), vote, and release the accumulator by one arrival each on
//     rel[b], which the issuing thread waits for before the next MMA into b. SPIN selects
//     polling instead of sleeping waits for the epilogue. Clocks per unit at thread 0 over
//     units WARM..U-1. Every wait is bounded (one second), and a timeout stops all sides.
template <int NB, int NCOL, int EPW, bool SPIN, bool LOAD, int NMT>
__global__ void __launch_bounds__((NMT + EPW) * 32, 1) k_handover(int units, int warm, unsigned long long *cycles,
                                                                   int *err, float *sink) {
    static_assert(NB * NCOL <= 512 && EPW % 4 == 0 && NB % NMT == 0, "shape");
    constexpr int CW = NCOL / (EPW / 4);        // columns per epilogue warp
    constexpr int CH = CW > 128 ? 128 : CW;     // columns per load
    static_assert(CW % CH == 0 && CH >= 32, "load shape");
    constexpr uint64_t kLimit = 1000000000ull;
    extern __shared__ __align__(1024) uint8_t sm[];
    __shared__ uint32_t tslot;
    __shared__ __align__(8) uint64_t t_full[NB], rel[NB], done;
    __shared__ volatile int abort_flag;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int b = 0; b < NB; ++b) { mbar_init(&t_full[b], 1); mbar_init(&rel[b], EPW); }
        mbar_init(&done, NMT);
        abort_flag = 0;
        fence_mbar_init();
    }
    for (int i = threadIdx.x; i < 16384; i += blockDim.x) reinterpret_cast<uint32_t *>(sm)[i] = 0u;
    if (warp == 0) { tmem_alloc(&tslot, 512); tmem_relinquish(); }
    fence_proxy_async_smem();
    tc_fence_before(); __syncthreads(); tc_fence_after();
    const uint32_t tb = tslot;
    if (warp == 0 || warp > EPW) {
        if (lane == 0) {
            const int k = warp == 0 ? 0 : warp - EPW;   // issuing thread index
            const uint64_t ad = smem_desc_k_noswizzle(smem_u32(sm), 128, 256);
            const uint64_t bd = smem_desc_k_noswizzle(smem_u32(sm + 4096), 128, 256);
            const uint32_t idesc = idesc_tf32_f32(128, NCOL);
            unsigned long long t0 = 0;
            int u = k, ufirst = -1, ulast = -1;
            for (; u < units; u += NMT) {
                const int b = u % NB;
                if (u >= NB && !mbar_spin_bounded(&rel[b], static_cast<uint32_t>(((u / NB) - 1) & 1), kLimit, &abort_flag)) {
                    *err = 1;
                    abort_flag = 1;
                    break;
                }
                tc_fence_after();
                if (ufirst < 0 && u >= warm) { ufirst = u; t0 = clock64(); }
                tc_mma_tf32(tb + static_cast<uint32_t>(b * NCOL), ad, bd, idesc, 0u);
                tc_commit(&t_full[b]);
                ulast = u;
            }
            const unsigned long long t1 = clock64();
            tc_commit(&done);
            if (!mbar_wait_bounded(&done, 0u, kLimit)) *err = 1;
            // clocks per unit, scaled by 1000
            if (k == 0 && u >= units && ulast > ufirst && ufirst >= 0)
                cycles[blockIdx.x] = (t1 - t0) * 1000ull / static_cast<unsigned long long>(ulast - ufirst);
        }
    } else {
        const int e = warp - 1;
        const int part = e >> 2;
        const uint32_t lane_addr = static_cast<uint32_t>((warp & 3) * 32) << 16;
        float acc = 0.f;
        for (int u = 0; u < units; ++u) {
            const int b = u % NB;
            const uint32_t ph = static_cast<uint32_t>((u / NB) & 1);
            bool w;
            if constexpr (SPIN) w = mbar_spin_bounded(&t_full[b], ph, kLimit, &abort_flag);
            else w = mbar_sleep_bounded(&t_full[b], ph, kLimit, &abort_flag);
            if (!__all_sync(0xFFFFFFFFu, w)) {
                if (lane == 0) { *err = 1; abort_flag = 1; }
                break;
            }
            tc_fence_after();
#pragma unroll
            for (int c = 0; c < (LOAD ? CW : 0); c += CH) {
                uint32_t v[CH];
                const float mn = tmem_ld_min<CH>(tb + lane_addr + static_cast<uint32_t>(b * NCOL + part * CW + c), v);
                acc += __any_sync(0xFFFFFFFFu, mn < 0.0f) ? 1.f : 0.f;
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&rel[b]);
        }
        if (acc == 12345.f) sink[0] = acc;
    }
    tc_fence_before(); __syncthreads();
    if (warp == 0) { tc_fence_after(); tmem_dealloc(tb, 512); }
}

// (4) What a shared-memory read costs the issuing thread when the next MMA waits for its
//     value: one thread loops {read; branch on it; MMA N=64; commit to one of 8 rotating
//     barriers}, the read being none (MODE 0), mbarrier.test_wait on a completed phase (1),
//     or ld.volatile.shared of a flag (2). SM clocks per iteration.
template <int MODE>
__global__ void k_dep(int iters, unsigned long long *cycles, int *err) {
    extern __shared__ __align__(1024) uint8_t sm[];
    __shared__ uint32_t tslot, flag;
    __shared__ __align__(8) uint64_t tf[8], full, done;
    const int warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        for (int i = 0; i < 8; ++i) mbar_init(&tf[i], 1);
        mbar_init(&full, 1);
        mbar_init(&done, 1);
        fence_mbar_init();
        mbar_arrive(&full);   // phase 0 of `full` completes
        flag = 1u;
    }
    for (int i = threadIdx.x; i < 16384; i += blockDim.x) reinterpret_cast<uint32_t *>(sm)[i] = 0u;
    if (warp == 0) { tmem_alloc(&tslot, 512); tmem_relinquish(); }
    fence_proxy_async_smem();
    tc_fence_before(); __syncthreads(); tc_fence_after();
    const uint32_t tb = tslot;
    if (threadIdx.x == 0) {
        const uint64_t ad = smem_desc_k_noswizzle(smem_u32(sm), 128, 256);
        const uint64_t bd = smem_desc_k_noswizzle(smem_u32(sm + 4096), 128, 256);
        const uint32_t idesc = idesc_tf32_f32(128, 64);
        const volatile uint32_t *vflag = &flag;
        const unsigned long long t0 = clock64();
        for (int it = 0; it < iters; ++it) {
            bool ok = true;
            if constexpr (MODE == 1) ok = mbar_test_wait(&full, 0u);
            if constexpr (MODE == 2) ok = *vflag == 1u;
            if (!ok) { *err = 1; break; }
            tc_fence_after();
            tc_mma_tf32(tb + static_cast<uint32_t>((it & 7) * 64), ad, bd, idesc, 0u);
            tc_commit(&tf[it & 7]);
        }
        const unsigned long long t1 = clock64();
        tc_commit(&done);
        if (!mbar_wait_bounded(&done, 0u, 1000000000ull)) *err = 1;
        cycles[blockIdx.x] = t1 - t0;
    }
    tc_fence_before(); __syncthreads();
    if (warp == 0) { tc_fence_after(); tmem_dealloc(tb, 512); }
}

template <int N, bool EACH>
static void run_mma(int sms, unsigned long long *d_cyc, int iters, const char *name) {
    cudaFuncSetAttribute(k_mma<N, EACH>, cudaFuncAttributeMaxDynamicSharedMemorySize, 65536);
    cudaMemset(d_cyc, 0, sizeof(unsigned long long) * sms);
    k_mma<N, EACH><<<sms, 64, 65536>>>(iters, d_cyc);
    cudaError_t e = cudaDeviceSynchronize();
    unsigned long long h[1024];
    cudaMemcpy(h, d_cyc, sizeof(unsigned long long) * sms, cudaMemcpyDeviceToHost);
    double mean = 0; for (int i = 0; i < sms; ++i) mean += (double)h[i]; mean /= sms;
    printf(", \"%s\": {\"n\": %d, \"commit_each\": %s, \"ok\": %s, \"cycles_per_mma\": %.1f}", name, N,
           EACH ? "true" : "false", e == cudaSuccess ? "true" : "false", mean / iters);
}

template <int NB, int NCOL, int EPW, bool SPIN, bool LOAD, int NMT>
static void run_handover(int sms, unsigned long long *d_cyc, int *d_err, float *d_sink, bool last) {
    const int units = 6000, warm = 1000;
    auto kern = k_handover<NB, NCOL, EPW, SPIN, LOAD, NMT>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 65536);
    cudaMemset(d_cyc, 0, sizeof(unsigned long long) * sms);
    cudaMemset(d_err, 0, sizeof(int));
    kern<<<sms, (NMT + EPW) * 32, 65536>>>(units, warm, d_cyc, d_err, d_sink);
    cudaError_t e = cudaDeviceSynchronize();
    unsigned long long h[1024];
    int herr = 0;
    cudaMemcpy(h, d_cyc, sizeof(unsigned long long) * sms, cudaMemcpyDeviceToHost);
    cudaMemcpy(&herr, d_err, sizeof(int), cudaMemcpyDeviceToHost);
    double mean = 0; for (int i = 0; i < sms; ++i) mean += (double)h[i]; mean /= sms * 1000.0;
    printf("{\"nb\": %d, \"ncol\": %d, \"epilogue_warps\": %d, \"mma_threads\": %d, \"wait\": \"%s\", "
           "\"load\": %s, \"ok\": %s, \"cycles_per_unit\": %.1f, \"pair_tests_per_clk_sm\": %.1f}%s",
           NB, NCOL, EPW, NMT, SPIN ? "spin" : "sleep", LOAD ? "true" : "false",
           (e == cudaSuccess && herr == 0) ? "true" : "false", mean, 128.0 * NCOL / mean, last ? "" : ", ");
}

template <int MODE>
static void run_dep(int sms, unsigned long long *d_cyc, int *d_err, const char *name, bool last) {
    const int iters = 2000;
    cudaFuncSetAttribute(k_dep<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, 65536);
    cudaMemset(d_cyc, 0, sizeof(unsigned long long) * sms);
    cudaMemset(d_err, 0, sizeof(int));
    k_dep<MODE><<<sms, 64, 65536>>>(iters, d_cyc, d_err);
    cudaError_t e = cudaDeviceSynchronize();
    unsigned long long h[1024];
    int herr = 0;
    cudaMemcpy(h, d_cyc, sizeof(unsigned long long) * sms, cudaMemcpyDeviceToHost);
    cudaMemcpy(&herr, d_err, sizeof(int), cudaMemcpyDeviceToHost);
    double mean = 0; for (int i = 0; i < sms; ++i) mean += (double)h[i]; mean /= sms;
    printf("\"%s\": {\"ok\": %s, \"cycles_per_iteration\": %.1f}%s", name,
           (e == cudaSuccess && herr == 0) ? "true" : "false", mean / iters, last ? "" : ", ");
}

template <int C, int WARPS>
static double run_read(int sms, unsigned long long *d_cyc, float *d_sink) {
    const int warps = WARPS;
    const int iters = 4000;
    cudaMemset(d_cyc, 0, sizeof(unsigned long long) * sms);
    k_read<C, WARPS><<<sms, WARPS * 32>>>(iters, d_cyc, d_sink);
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) { printf("error %s\n", cudaGetErrorString(e)); return -1; }
    unsigned long long h[1024];
    cudaMemcpy(h, d_cyc, sizeof(unsigned long long) * sms, cudaMemcpyDeviceToHost);
    double mean = 0; for (int i = 0; i < sms; ++i) mean += (double)h[i]; mean /= sms;
    const double bytes = (double)iters * warps * 32 * C * 4;
    return bytes / mean;   // bytes per clock per SM
}

int main() {
    int sms = 0; cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
    unsigned long long *d_cyc; float *d_sink;
    cudaMalloc(&d_cyc, sizeof(unsigned long long) * 1024); cudaMalloc(&d_sink, 4);
    printf("{\"sms\": %d, \"read\": [", sms);
    bool first = true;
#define ROW(W, R128) { double a = -1; if constexpr (R128) a = run_read<128, (R128 ? W : 4)>(sms, d_cyc, d_sink); double b = run_read<64, W>(sms, d_cyc, d_sink); \
        double c = run_read<32, W>(sms, d_cyc, d_sink); \
        printf("%s{\"warps\": %d, \"x128_B_per_clk\": %.1f, \"x64_B_per_clk\": %.1f, \"x32_B_per_clk\": %.1f}", first ? "" : ", ", W, a, b, c); first = false; }
    ROW(4, 1) ROW(8, 1) ROW(12, 1) ROW(16, 0)
    printf("], ");
    cudaFuncSetAttribute(k_mma<256, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 65536);
    for (int iters : {64, 2000}) {
        cudaMemset(d_cyc, 0, sizeof(unsigned long long) * sms);
        k_mma<256, false><<<sms, 64, 65536>>>(iters, d_cyc);
        cudaError_t e = cudaDeviceSynchronize();
        if (e != cudaSuccess) { printf("error %s\n", cudaGetErrorString(e)); return 1; }
        unsigned long long h[1024];
        cudaMemcpy(h, d_cyc, sizeof(unsigned long long) * sms, cudaMemcpyDeviceToHost);
        double mean = 0; for (int i = 0; i < sms; ++i) mean += (double)h[i]; mean /= sms;
        printf("\"mma_%d\": {\"cycles_per_mma\": %.1f}%s", iters, mean / iters, iters == 64 ? ", " : "");
    }
    run_mma<256, true>(sms, d_cyc, 2000, "mma_commit_each_n256");
    run_mma<64, true>(sms, d_cyc, 2000, "mma_commit_each_n64");
    int *d_err; cudaMalloc(&d_err, sizeof(int));
    printf(", \"read_before_mma\": {");
    run_dep<0>(sms, d_cyc, d_err, "none", false);
    run_dep<1>(sms, d_cyc, d_err, "mbarrier_test_wait", false);
    run_dep<2>(sms, d_cyc, d_err, "ld_volatile_shared", true);
    printf("}, \"handover\": [");
    run_handover<1, 256, 8, false, true, 1>(sms, d_cyc, d_err, d_sink, false);
    run_handover<2, 256, 8, false, true, 1>(sms, d_cyc, d_err, d_sink, false);
    run_handover<2, 256, 8, true, true, 1>(sms, d_cyc, d_err, d_sink, false);
    run_handover<2, 256, 8, false, false, 1>(sms, d_cyc, d_err, d_sink, false);
    run_handover<4, 128, 8, false, true, 1>(sms, d_cyc, d_err, d_sink, false);
    run_handover<8, 64, 8, false, true, 1>(sms, d_cyc, d_err, d_sink, false);
    run_handover<8, 64, 8, false, false, 1>(sms, d_cyc, d_err, d_sink, false);
    run_handover<2, 256, 8, false, true, 2>(sms, d_cyc, d_err, d_sink, false);
    run_handover<4, 128, 8, false, true, 2>(sms, d_cyc, d_err, d_sink, true);
    printf("]}\n");
    return 0;
}

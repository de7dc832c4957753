// Rates that bound the tensor-core pair kernel, measured with one CTA on every SM:
//  (1) TMEM -> register reads in the kernel's load shape: W warps (W/4 per TMEM lane
//      quarter) each loop over tcgen05.ld.red.sync.aligned.32x32b.x{32,64,128}.min (the
//      accumulator values and their minimum), tcgen05.wait::ld and a warp vote on the
//      minimum; bytes read per SM clock (clock64 over 4000 loads, all warps, mean over SMs);
//  (2) tcgen05.mma kind::tf32 M=128 N=256 K=8 (the kernel's shape) issued back to back by
//      one thread into alternating accumulators, one commit at the end: SM clocks per MMA.
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

__global__ void k_mma(int iters, unsigned long long *cycles) {
    extern __shared__ __align__(1024) uint8_t sm[];
    __shared__ uint32_t tslot;
    __shared__ __align__(8) uint64_t done;
    const int warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) { mbar_init(&done, 1); fence_mbar_init(); }
    for (int i = threadIdx.x; i < 16384; i += blockDim.x) reinterpret_cast<uint32_t *>(sm)[i] = 0u;
    if (warp == 0) { tmem_alloc(&tslot, 512); tmem_relinquish(); }
    fence_proxy_async_smem();
    tc_fence_before(); __syncthreads(); tc_fence_after();
    const uint32_t tb = tslot;
    if (threadIdx.x == 32) {
        const uint64_t ad = smem_desc_k_noswizzle(smem_u32(sm), 128, 256);
        const uint64_t bd = smem_desc_k_noswizzle(smem_u32(sm + 4096), 128, 256);
        const uint32_t idesc = idesc_tf32_f32(128, 256);
        const unsigned long long t0 = clock64();
        for (int it = 0; it < iters; ++it) tc_mma_tf32(tb + (uint32_t)((it & 1) * 256), ad, bd, idesc, 0u);
        tc_commit(&done);
        (void)mbar_wait_bounded(&done, 0u, 2000000000ull);
        const unsigned long long t1 = clock64();
        cycles[blockIdx.x] = t1 - t0;
    }
    tc_fence_before(); __syncthreads();
    if (warp == 0) { tc_fence_after(); tmem_dealloc(tb, 512); }
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
    cudaFuncSetAttribute(k_mma, cudaFuncAttributeMaxDynamicSharedMemorySize, 65536);
    for (int iters : {64, 2000}) {
        cudaMemset(d_cyc, 0, sizeof(unsigned long long) * sms);
        k_mma<<<sms, 64, 65536>>>(iters, d_cyc);
        cudaError_t e = cudaDeviceSynchronize();
        if (e != cudaSuccess) { printf("error %s\n", cudaGetErrorString(e)); return 1; }
        unsigned long long h[1024];
        cudaMemcpy(h, d_cyc, sizeof(unsigned long long) * sms, cudaMemcpyDeviceToHost);
        double mean = 0; for (int i = 0; i < sms; ++i) mean += (double)h[i]; mean /= sms;
        printf("\"mma_%d\": {\"cycles_per_mma\": %.1f}%s", iters, mean / iters, iters == 64 ? ", " : "");
    }
    printf("}\n");
    return 0;
}

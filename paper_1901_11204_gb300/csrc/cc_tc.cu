// Tensor-core pair kernel for integer points (fast exact mode): the balanced cyclic
// schedule of Section 4 with the per-pair collision predicate evaluated as a dense
// contraction on the 5th-generation tensor cores (tcgen05, kind::tf32, FP32 accumulation
// in Tensor Memory).
//
// With centred integer coordinates p' (|p'| <= m per axis) and n = |p'|^2,
//     d^2 - r2e - 1 = -2 p'_i . p'_j + n_j + (n_i - r2e - 1) = sum_k a_ik * b_jk
// over K = 8 slots:
//     a_i = [-2x'_i, -2y'_i, -2z'_i, 1, 1, cA*2^22, cB*2^11, cC]
//     b_j = [ x'_j,   y'_j,   z'_j, nH*2^11, nL, 1, 1, 1]
// where n_j = nH*2^11 + nL (0 <= nL < 2^11) and c_i = n_i - r2e - 1 = cA*2^22 + cB*2^11 + cC
// with balanced digits cB, cC in [-1024, 1023]. Every operand is an integer of at most
// 11 significant bits times a power of two, so it is exact in TF32, every product is
// exact, and the mode test on the device admits the TF32 path only when the sum of the
// absolute values of all eight terms stays below 2^24. Then every partial sum, in any
// order and with any alignment the tensor core uses, is an integer below 2^24 and exact
// in FP32: the accumulator holds d^2 - r2e - 1 exactly, and the pair collides (d^2 <= r2)
// iff it is negative.
//
// Counting the negatives: with acc in [2^23, 2^24) (unit spacing), fma.rm(v, 2^-25, acc)
// gives acc - 1 if v <= -1 and acc if v >= 0 (|v| < 2^24 keeps |v| 2^-25 below 1/2), so
// one packed FP32x2 instruction counts two pairs exactly.
//
// Per CTA (one per SM, persistent, an equal contiguous share of the (tile, stage) units):
//   warp 0        bulk-copies the i-tile operand (128 rows, 4 KB) when the tile changes
//                 and every j-stage operand (256 rows, 8 KB) into an NS-deep ring,
//   warp 1        allocates 512 TMEM columns; its lane 0 issues one
//                 tcgen05.mma (M=128, N=256, K=8) per unit into one of two TMEM
//                 accumulators and commits to that accumulator's barrier,
//   warps 2..     (EPW warps) read the accumulator rows of their TMEM lane quarter
//                 (tcgen05.ld 32x32b) and count; stages that touch the ends of the
//                 cyclic range take the per-pair validity mask. The first of them also
//                 returns each j-stage slot and i-tile slot to the copy warp once it has
//                 seen the MMAs that read them complete.
// Every wait is bounded by the global timer; on expiry the kernel records ST_TIMEOUT,
// lets the other roles stop, waits (bounded) for its MMAs, frees TMEM and returns.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdlib>

#include "cc_internal.cuh"
#include "cc_tcgen05.cuh"

namespace cc {

constexpr int TC_T = 128;                  // objects per i-tile (MMA M)
constexpr int TC_ROW = 32;                 // bytes per operand row (8 TF32)
constexpr int TC_ATILE = TC_T * TC_ROW;    // 4096

// Byte offset of element k of row r in the no-swizzle K-major core-matrix layout:
// 8-row groups of 256 bytes, each two 128-byte core matrices (k 0-3, k 4-7).
__host__ __device__ constexpr uint32_t tc_off(int64_t r, int k) {
    return static_cast<uint32_t>((r & 7) * 16 + (k >> 2) * 128 + (k & 3) * 4);
}
__host__ __device__ constexpr int64_t tc_group(int64_t r) { return (r >> 3) * 256; }

// Geometry of one call for j-stages of JS objects (the MMA's N).
struct TcGeom {
    int64_t M, K, units, elen;
    size_t a_bytes, b_bytes;
};

TcGeom tc_geometry(int64_t n, int js) {
    TcGeom g;
    const int64_t h = (n - 1) / 2;
    g.M = (n + TC_T - 1) / TC_T;
    g.K = (TC_T + h + 1 + js - 1) / js;
    g.units = g.M * g.K;
    g.elen = (g.M - 1) * TC_T + g.K * js;
    g.a_bytes = static_cast<size_t>(g.M) * TC_ATILE;
    g.b_bytes = static_cast<size_t>(g.elen) * TC_ROW;
    return g;
}

// Operand bytes for any of the compiled stage widths (128 or 256).
size_t tc_region_bytes(int64_t n) {
    size_t b = 0;
    for (int js : {128, 256}) {
        const TcGeom g = tc_geometry(n, js);
        b = std::max(b, g.a_bytes + g.b_bytes);
    }
    return b;
}

// ---------------------------------------------------------------------------------------
// operand fill (runs only when the device chose MODE_I32_TC or MODE_F32_TC)
// ---------------------------------------------------------------------------------------

// Integer coordinate of object p on one axis, before centring: the caller's integer, or
// for FP32 spheres the quantised floor((v - min) * S) in [0, 2046] (computed in FP64).
template <bool F32>
__device__ __forceinline__ int32_t tc_coord(const void *c, int64_t p, int axis, const WsHeader *h) {
    if constexpr (F32) {
        const double v = static_cast<double>(static_cast<const float *>(c)[p]);
        return static_cast<int32_t>(floor((v - static_cast<double>(h->qmin[axis])) * h->qscale));
    } else {
        return static_cast<const int32_t *>(c)[p];
    }
}

template <bool F32>
__global__ void k_fill_tc(const void *__restrict__ x, const void *__restrict__ y, const void *__restrict__ z,
                          int64_t n, int64_t arows, int64_t elen, uint8_t *__restrict__ Aop,
                          uint8_t *__restrict__ Bop, WsHeader *__restrict__ h, uint32_t *__restrict__ hist) {
    if (h->mode != (F32 ? MODE_F32_TC : MODE_I32_TC)) return;   // uniform over the grid
    const int32_t cx = h->cx, cy = h->cy, cz = h->cz;
    // integer points: 16 cells per axis over the bounding box, for the occupancy histogram
    // (in this mode every span is at most 2046, so the cell arithmetic fits 32 bits)
    int32_t box_lo[3] = {0, 0, 0}, box_n[3] = {1, 1, 1};   // minimum and span + 1 per axis
    if (!F32 && hist) {
        for (int a = 0; a < 3; ++a) {
            box_lo[a] = ord_dec(h->umin[a]);
            box_n[a] = ord_dec(h->umax[a]) - box_lo[a] + 1;
        }
    }
    const int32_t off = h->ai_off;   // r2e + 1
    const int64_t rows = arows > elen ? arows : elen;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < rows;
         r += (int64_t)gridDim.x * blockDim.x) {
        uint8_t *ga = Aop + tc_group(r);
        uint8_t *gb = Bop + tc_group(r);
        if (r < arows) {
            float4 lo, hi;
            if (r < n) {
                const int32_t xi = tc_coord<F32>(x, r, 0, h) - cx, yi = tc_coord<F32>(y, r, 1, h) - cy,
                              zi = tc_coord<F32>(z, r, 2, h) - cz;
                if (!F32 && hist && (r & (TC_HIST_STRIDE - 1)) == 0) {   // every 8th object
                    const int32_t qx = (xi + cx - box_lo[0]) * 16 / box_n[0];
                    const int32_t qy = (yi + cy - box_lo[1]) * 16 / box_n[1];
                    const int32_t qz = (zi + cz - box_lo[2]) * 16 / box_n[2];
                    atomicAdd(&hist[(qx * 16 + qy) * 16 + qz], 1u);
                }
                const int32_t c = xi * xi + yi * yi + zi * zi - off;
                const int32_t cC = ((c + 1024) & 2047) - 1024;
                const int32_t c1 = (c - cC) >> 11;   // exact: c - cC is a multiple of 2^11
                const int32_t cB = ((c1 + 1024) & 2047) - 1024;
                const int32_t cA = (c1 - cB) >> 11;
                lo = make_float4(static_cast<float>(-2 * xi), static_cast<float>(-2 * yi),
                                 static_cast<float>(-2 * zi), 1.0f);
                hi = make_float4(1.0f, static_cast<float>(cA) * 4194304.0f, static_cast<float>(cB) * 2048.0f,
                                 static_cast<float>(cC));
            } else {
                // ragged tile end: v = 1 for every j, never a hit
                lo = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                hi = make_float4(0.0f, 0.0f, 0.0f, 1.0f);
            }
            *reinterpret_cast<float4 *>(ga + tc_off(r, 0)) = lo;
            *reinterpret_cast<float4 *>(ga + tc_off(r, 4)) = hi;
        }
        if (r < elen) {
            // extended rows stay below 2n (elen < 2n for the sizes this path serves): a
            // subtraction, not a 64-bit remainder, maps them back
            const int64_t p = r < n ? r : (r < 2 * n ? r - n : r % n);
            const int32_t xj = tc_coord<F32>(x, p, 0, h) - cx, yj = tc_coord<F32>(y, p, 1, h) - cy,
                          zj = tc_coord<F32>(z, p, 2, h) - cz;
            const int32_t nj = xj * xj + yj * yj + zj * zj;
            const float4 lo = make_float4(static_cast<float>(xj), static_cast<float>(yj),
                                          static_cast<float>(zj), static_cast<float>(nj >> 11) * 2048.0f);
            const float4 hi = make_float4(static_cast<float>(nj & 2047), 1.0f, 1.0f, 1.0f);
            *reinterpret_cast<float4 *>(gb + tc_off(r, 0)) = lo;
            *reinterpret_cast<float4 *>(gb + tc_off(r, 4)) = hi;
        }
    }
    if (F32 || !hist) return;
    // The last block refines the count form from the histogram (of a systematic sample of
    // one object in TC_HIST_STRIDE): pairs that share a cell,
    // times the chance that a pair inside one cell is within reach (ball / cell sites),
    // and never below the bounding-box estimate. Clustered sets, whose bounding box hides
    // their density, then take the in-register form. The pair counts are exact integers
    // and the estimate FP32: it only picks the faster of two exact forms, and the FP64
    // pipe of this part is slow enough that the same tail in FP64 took about 13 us.
    __shared__ bool last;
    __shared__ unsigned long long red[32];
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(&h->ticket0, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    unsigned long long same = 0;
    for (int c = threadIdx.x; c < TC_HIST_CELLS; c += blockDim.x) {
        const unsigned long long k = __ldcg(&hist[c]);
        same += k * (k - 1) / 2;   // 0 when k = 0 (the wrapped factor is multiplied by 0)
    }
    for (int o = 16; o > 0; o >>= 1) same += __shfl_down_sync(0xFFFFFFFFu, same, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = same;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long tot = 0;
        for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) tot += red[w];
        const float ns = static_cast<float>((n + TC_HIST_STRIDE - 1) / TC_HIST_STRIDE);   // sampled
        const float pairs = 0.5f * ns * (ns - 1.0f);
        const float rad = sqrtf(static_cast<float>(h->r2e)) + 1.0f;
        const float ball = 4.18879020f * rad * rad * rad;   // (4/3) pi rad^3
        const float sites = static_cast<float>(box_n[0]) * static_cast<float>(box_n[1]) * static_cast<float>(box_n[2]);
        const float cell_sites = sites / static_cast<float>(TC_HIST_CELLS);
        const float est = fmaxf(ball / sites, (static_cast<float>(tot) / pairs) * fminf(1.0f, ball / cell_sites));
        h->tc_form = est < static_cast<float>(TC_SPARSE_HITS) ? 1 : 0;
        h->ticket0 = 0;
    }
}

// ---------------------------------------------------------------------------------------
// the kernel
// ---------------------------------------------------------------------------------------

struct TcArgs {
    const uint8_t *Aop;     // i-tile operands, M tiles of 4 KB
    const uint8_t *Bop;     // extended j operands, elen rows
    int64_t n;
    int64_t units;          // M * K
    int32_t K;              // stages per tile
    int32_t h;              // (n-1)/2
    WsHeader *hdr;
    unsigned long long *d_count;
    float *d_sum;           // interaction sum (sum kernels only)
    double *partial;        // one FP64 slot per CTA (sum kernels only)
    const float *px, *py, *pz, *pr;   // FP32 spheres: the caller's coordinates and radii
    uint64_t wait_ns;
    int32_t stall;          // test hook: the copy warp issues nothing
    int32_t form;           // integer counts: run only when the header's tc_form equals
                            // this (0 or 1); -1 runs whatever the form
};

// Shape of the kernel: j-stages of TC_JS objects (the MMA's N), TC_NB accumulators of
// TC_JS TMEM columns (TC_NB * TC_JS = 512, all of TMEM), TC_EPW epilogue warps (two per
// TMEM lane quarter, TC_CPW columns each), a TC_NS-deep ring of j-stages.
constexpr int TC_JS = 256;
constexpr int TC_NB = 2;
constexpr int TC_EPW = 8;
constexpr int TC_NS = 12;
constexpr int TC_CPW = TC_JS / (TC_EPW / 4);   // accumulator columns per epilogue warp and unit
// warps: copy, MMA, TC_EPW epilogue warps (warps 2 .. 2 + TC_EPW - 1, so that warp & 3 is the
// TMEM lane quarter each may read), and one slot-return warp
constexpr int TC_THREADS = (3 + TC_EPW) * 32;
static_assert(TC_NB * TC_JS == 512, "the accumulators fill the 512 TMEM columns");
static_assert(TC_NS > TC_NB, "a unit's stage slot outlives the release of its accumulator");
// Least number of stages (units) per i-tile: the slot-return warp frees an i-tile slot once
// the ready phase two units after the tile's last unit completed, and that unit's copy must
// come before the tile two later's (true for n >= 257 objects; the path starts far above).
constexpr int TC_MIN_K = 2;

struct TcSmem {
    static constexpr int kStage = TC_JS * TC_ROW;         // bytes of one j-stage
    static constexpr int kA = 0;                          // 2 i-tile slots
    static constexpr int kB = 2 * TC_ATILE;               // TC_NS j-stage slots
    static constexpr int kBars = kB + TC_NS * kStage;
    // a_full[2] a_empty[2] ready[NS] b_empty[NS] t_full[NB] done (t_full2[NB] at kFull2)
    static constexpr int kNBars = 5 + 2 * TC_NS + TC_NB;
    static constexpr int kMisc = kBars + kNBars * 8;      // tmem address, abort flag, copy drain words
    static constexpr int kRed = kMisc + 16;               // per-epilogue-warp counts
    static constexpr int kRedSum = kRed + TC_EPW * 8;     // per-epilogue-warp sums
    static constexpr int kFull2 = kRedSum + TC_EPW * 8;   // t_full2[NB]
    static constexpr int kTotal = kFull2 + TC_NB * 8;
};

__device__ __forceinline__ f2 f2_fma_rm(f2 a, f2 b, f2 c) {
    f2 d;
    asm("fma.rm.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

// acc lanes start at 2^24 - 1 (0x4B7FFFFF); the count is 2^24 - 1 - acc = ~bits & 0x7FFFFF.
constexpr f2 kAccInit = 0x4B7FFFFF4B7FFFFFull;
constexpr f2 kScale = 0x3300000033000000ull;   // 2^-25 in both lanes

__device__ __forceinline__ uint32_t acc_count(f2 a) {
    const uint32_t lo = static_cast<uint32_t>(a), hi = static_cast<uint32_t>(a >> 32);
    return ((~lo) & 0x7FFFFFu) + ((~hi) & 0x7FFFFFu);
}

// One interaction term 1/max(d, 1e-6) from the exact d^2: square root and reciprocal each
// correctly rounded in FP32 (the FP32-pipe kernels' term, before its widening to FP64).
__device__ __forceinline__ float term_f32(float d2) {
    return __frcp_rn(fmaxf(__fsqrt_rn(d2), 1e-6f));
}

// The FP32 sphere predicate, the same operations in the same order and rounding as the
// FP32-pipe kernels (differences, squares and sums each rounded to nearest, never fused):
// collide iff (dx*dx + dy*dy) + dz*dz <= (r_i + r_j)^2; d2 is returned for the term.
__device__ __forceinline__ bool sphere_pair(float xi, float yi, float zi, float ri, float xj, float yj, float zj,
                                            float rj, float &d2) {
    const float dx = __fsub_rn(xi, xj);
    const float dy = __fsub_rn(yi, yj);
    const float dz = __fsub_rn(zi, zj);
    d2 = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
    const float s = __fadd_rn(ri, rj);
    return d2 <= __fmul_rn(s, s);
}

// Kahan's compensated summation: the error stays within (2u + O(k u^2)) times the sum of the
// k (positive) terms, u = 2^-24, so FP32 serves for the whole kernel (k u^2 < 1e-8 for the
// largest per-thread term counts) and the FP64 pipe, slow on this part, is kept off the
// per-hit path.
__device__ __forceinline__ void kahan_add(float &s, float &c, float x) {
    const float y = __fsub_rn(x, c);
    const float t = __fadd_rn(s, y);
    c = __fsub_rn(__fsub_rn(t, s), y);
    s = t;
}

// The epilogue forms. Every form reads the accumulator with tcgen05.ld.red .min, which
// also gives each thread the minimum of its 128 values: a warp whose minima are all
// non-negative (every pair of its block misses, the common case at collision radii)
// only votes.
//   WALK = false (integer count, dense hits): the buffer is handed back right after the
//     load and warps holding a negative value count their 128 values with the rounding-
//     down packed FMA on the accumulators in registers.
//   WALK = true (integer count at sparse hits; interaction sums SUMT; FP32 spheres SPH):
//     warps holding a negative value OR each group of 8 columns, re-read the flagged
//     groups from TMEM (the accumulator is still held) and walk them exactly: count the
//     negatives inside the row's schedule window; for sums add 1/max(d, 1e-6) with
//     d^2 = v + r2e + 1 (exact in FP32) to a Kahan-compensated FP32 sum per thread; for
//     spheres apply the FP32 predicate to the pair's own coordinates. No value stays
//     live past the load, so the loop stays lean.
// The host launches both integer count forms and each runs only when the preparation
// kernel chose it (hdr->tc_form, from the expected hit density; TcArgs::form).
//
// Barriers (mbarrier, shared memory):
//   a_full/a_empty[2]  i-tile slots: copied by warp 0, freed by the slot-return warp
//                      once the tile's last MMA of this CTA completed (seen as below);
//   ready[NS]          unit q may run: the stage copy of q landed (the copy warp's
//                      arrive.expect_tx and the copy's bytes) AND every epilogue warp
//                      released the accumulator unit q will overwrite (the one of unit
//                      q - NB; arrive count 1 + EPW, the first NB units pre-arrived), so
//                      that the MMA thread, the pipeline's critical path, tests one
//                      barrier per unit. That thread's loop bounds the kernel: a barrier
//                      test whose outcome the next MMA issue waits for queues behind the
//                      thread's own MMA and commit (about 200 cycles on GB300, measured),
//                      and the loop alone takes about 458 cycles per unit;
//   b_empty[NS]        stage slot free again: the slot-return warp, once unit q's MMA
//                      completed, which it sees as the completion of the ready phase of
//                      unit q + NB (that phase needs every epilogue warp's release of unit
//                      q's accumulator, read after the MMA completed). The warp watches these
//                      phases in unit order, and the next phase of the barrier it watches
//                      (unit q + NB + NS) needs the copy into the very slot it frees only
//                      later, so it can never fall a phase behind and misread a parity
//                      (watching t_full instead, a lagging warp could). It is a warp of its
//                      own so that the epilogue warps, all of which must release an
//                      accumulator before the next MMA into it, do equal work: an epilogue
//                      warp with this extra duty trailed the others by about 300 cycles per
//                      unit and paced the pipeline. The slots of the share's last NB units
//                      are never needed again and are not returned;
//   t_full[NB]         accumulator written: tcgen05.commit after the unit's MMA;
//   t_full2[NB]        the same, committed a second time in the in-register count form
//                      and the FP32-sphere sum (FULL2), for warps 6-9 (the second
//                      epilogue warp of each SMSP): two warps of an SMSP sleeping on one
//                      barrier woke one after the other, and with a barrier each those
//                      forms run 3.6 % faster (in-register count at dense hits, sphere
//                      sums); the others keep one barrier, where the second commit
//                      lengthens the MMA thread's loop, their critical path (walk count
//                      8 %, integer sum at sparse hits 6 %, sphere count 4.5 % slower);
//   done               every MMA of this CTA completed (before TMEM is freed).
template <bool SUMT, bool SPH, bool WALKC>
__global__ void __launch_bounds__(TC_THREADS, 1) k_pairs_tc(TcArgs A) {
    using L = TcSmem;
    constexpr int JS = TC_JS, NB = TC_NB, EPW = TC_EPW, NS = TC_NS, CPW = TC_CPW;
    constexpr int kStage = L::kStage;
    constexpr bool WALK = SUMT || SPH || WALKC;   // screened values are walked one by one
    // forms whose second epilogue warp of each SMSP waits on its own accumulator barrier
    constexpr bool FULL2 = !WALK || (SUMT && SPH);
    extern __shared__ __align__(1024) uint8_t smem[];
    // uniform: another kernel handles this call
    if (A.hdr->mode != (SPH ? MODE_F32_TC : MODE_I32_TC)) return;
    if (A.form >= 0 && A.hdr->tc_form != A.form) return;   // the other count form runs

    uint8_t *sA = smem + L::kA;
    uint8_t *sB = smem + L::kB;
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + L::kBars);
    uint64_t *a_full = bars, *a_empty = bars + 2;
    uint64_t *ready = bars + 4, *b_empty = bars + 4 + NS;
    uint64_t *t_full = bars + 4 + 2 * NS, *done = t_full + NB;
    // FULL2 forms: the second epilogue warp of each SMSP waits here (after the
    // other buffers, so that the other forms' layout and code stay as they were)
    uint64_t *t_full2 = reinterpret_cast<uint64_t *>(smem + L::kFull2);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + L::kMisc);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(smem + L::kMisc + 4);
    // the copy warp's number of issued stage copies, published when it stops (drain)
    volatile int *copy_issued = reinterpret_cast<volatile int *>(smem + L::kMisc + 8);
    volatile int *copy_stopped = reinterpret_cast<volatile int *>(smem + L::kMisc + 12);
    unsigned long long *red = reinterpret_cast<unsigned long long *>(smem + L::kRed);
    double *red_sum = reinterpret_cast<double *>(smem + L::kRedSum);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int i = 0; i < 2; ++i) {
            mbar_init(&a_full[i], 1);
            mbar_init(&a_empty[i], 1);
        }
        for (int i = 0; i < NB; ++i) {
            mbar_init(&t_full[i], 1);
            if constexpr (FULL2) mbar_init(&t_full2[i], 1);
        }
        for (int i = 0; i < NS; ++i) {
            mbar_init(&ready[i], 1 + EPW);
            mbar_init(&b_empty[i], 1);
        }
        mbar_init(done, 1);
        *abort_flag = 0;
        *copy_issued = 0;
        *copy_stopped = 0;
        fence_mbar_init();
    }
    if (warp == 1) {
        tmem_alloc(tmem_slot, 512);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = *tmem_slot;

    const int64_t G = gridDim.x;
    const int64_t u0 = (A.units * blockIdx.x) / G;
    const int64_t u1 = (A.units * (blockIdx.x + 1)) / G;
    const int64_t K = A.K;
    // Loop state below is kept in 32-bit counters (ring slot and phase, accumulator and
    // phase, stage within the tile): the copy and MMA lanes are single threads sharing
    // their SMSP with two epilogue warps, so their per-unit instruction count is the
    // pipeline's critical path.
    const int32_t nu = static_cast<int32_t>(u1 - u0);   // units of this CTA
    const int32_t K32 = A.K;
    const int64_t t0 = u0 / K;
    const int32_t s0 = static_cast<int32_t>(u0 - t0 * K);
    if (warp == 0) {
        // ------------------------------- copy warp -------------------------------------
        if (lane == 0) {
            int32_t q = 0;
            uint32_t na = 0;
            if (!A.stall) {
                int64_t t = t0;
                int32_t st = s0;
                const uint8_t *bsrc = A.Bop + (t * TC_T + static_cast<int64_t>(st) * JS) * TC_ROW;
                int64_t cur_t = -1;
                int32_t slot = 0;
                uint32_t eph = 1;   // parity of the b_empty phase to wait for (first pass: free)
                for (; q < nu; ++q) {
                    if (t != cur_t) {
                        const uint32_t as = na & 1u;
                        if (!mbar_sleep_bounded(&a_empty[as], ((na >> 1) & 1u) ^ 1u, A.wait_ns, abort_flag)) break;
                        mbar_arrive_expect_tx(&a_full[as], TC_ATILE);
                        bulk_g2s(sA + as * TC_ATILE, A.Aop + t * TC_ATILE, TC_ATILE, &a_full[as]);
                        ++na;
                        cur_t = t;
                    }
                    if (!mbar_sleep_bounded(&b_empty[slot], eph, A.wait_ns, abort_flag)) break;
                    mbar_arrive_expect_tx(&ready[slot], kStage);
                    bulk_g2s(sB + slot * kStage, bsrc, kStage, &ready[slot]);
                    bsrc += JS * TC_ROW;
                    if (++st == K32) {
                        st = 0;
                        ++t;
                        bsrc = A.Bop + t * TC_T * TC_ROW;
                    }
                    if (++slot == NS) {
                        slot = 0;
                        eph ^= 1u;
                    }
                }
            }
            *copy_issued = q;
            __threadfence_block();
            *copy_stopped = 1;
            // Every copy issued above is waited for by the MMA lane before it retires the
            // slot; after an abort the MMA lane may have stopped early, so wait here
            // (bounded) for the last copy of every slot (the epilogue warps make their
            // remaining ready arrivals for these units) and of both i-tile slots.
            if (*abort_flag) {
                const int32_t issued = q;
                for (int32_t qq = issued > NS ? issued - NS : 0; qq < issued; ++qq)
                    (void)mbar_wait_bounded(&ready[qq % NS], static_cast<uint32_t>((qq / NS) & 1), A.wait_ns);
                for (uint32_t k = (na > 2 ? na - 2 : 0); k < na; ++k)
                    (void)mbar_wait_bounded(&a_full[k & 1u], (k >> 1) & 1u, A.wait_ns);
            }
        }
    } else if (warp == 1) {
        // ------------------------------- MMA lane --------------------------------------
        if (lane == 0) {
            constexpr uint32_t idesc = idesc_tf32_f32(TC_T, JS);
            // descriptors of slot 0; a slot's is this plus its byte offset >> 4 (the start
            // address field cannot carry: shared addresses stay below 2^18)
            const uint64_t ad0 = smem_desc_k_noswizzle(smem_u32(sA), 128, 256);
            const uint64_t bd0 = smem_desc_k_noswizzle(smem_u32(sB), 128, 256);
            int32_t st = s0;
            bool new_tile = true;
            uint32_t na = 0;
            int32_t slot = 0, buf = 0;
            uint32_t rph = 0;   // ready phase parity
            bool ok = true;
            // outcome of the next unit's barrier test, taken early (right after the
            // previous commit) so that its latency overlaps the MMA
            bool pre_ready = false;
            for (int32_t q = 0; q < nu; ++q) {
                if (new_tile) {
                    ok = mbar_spin_bounded(&a_full[na & 1u], (na >> 1) & 1u, A.wait_ns, abort_flag);
                    if (!ok) break;
                    ++na;
                }
                const uint32_t as = (na - 1) & 1u;
                ok = pre_ready || mbar_spin_bounded(&ready[slot], rph, A.wait_ns, abort_flag);
                if (!ok) break;
                tc_fence_after();
                tc_mma_tf32(tbase + static_cast<uint32_t>(buf * JS), ad0 + as * (TC_ATILE >> 4),
                            bd0 + static_cast<uint32_t>(slot) * (kStage >> 4), idesc, 0u);
                tc_commit(&t_full[buf]);
                if constexpr (FULL2) tc_commit(&t_full2[buf]);
                new_tile = ++st == K32;
                if (new_tile) st = 0;
                if (++slot == NS) {
                    slot = 0;
                    rph ^= 1u;
                }
                if (++buf == NB) buf = 0;
                pre_ready = mbar_test_wait(&ready[slot], rph);
            }
            if (!ok) {
                flag_status(A.hdr, ST_TIMEOUT);
                *abort_flag = 1;
            }
            // all MMAs issued by this thread complete before TMEM is freed
            tc_commit(done);
            if (!mbar_wait_bounded(done, 0u, A.wait_ns)) flag_status(A.hdr, ST_TIMEOUT);
        }
    } else if (warp == 2 + EPW) {
        // ------------------------------- slot-return warp ------------------------------
        if (lane == 0) {
            int32_t st = s0, buf = 0, rslot = 0;
            uint32_t fph = 0, tord = 0;
            for (int32_t q = 0; q + NB < nu; ++q) {
                const int32_t u = q + NB;
                if (!mbar_sleep_bounded(&ready[u % NS], static_cast<uint32_t>((u / NS) & 1), A.wait_ns, abort_flag)) {
                    if (!*abort_flag) {
                        flag_status(A.hdr, ST_TIMEOUT);
                        *abort_flag = 1;
                    }
                    break;
                }
                // unit q's MMA (and every earlier one) is complete: its j-stage slot, and
                // after a tile's last unit the i-tile slot, can be refilled
                mbar_arrive(&b_empty[rslot]);
                if (st == K32 - 1) mbar_arrive(&a_empty[tord & 1u]);
                if (++buf == NB) {
                    buf = 0;
                    fph ^= 1u;
                }
                if (++rslot == NS) rslot = 0;
                if (++st == K32) {
                    st = 0;
                    ++tord;
                }
            }
        }
    } else {
        // ------------------------------- epilogue warps --------------------------------
        const int ew = warp - 2;
        const int quarter = warp & 3;          // TMEM lanes this warp may access
        const int part = ew >> 2;              // which CPW-column part of the accumulator
        const int row = quarter * 32 + lane;   // object offset inside the i-tile
        const uint32_t lane_addr = static_cast<uint32_t>(quarter * 32) << 16;
        // the accumulators of the first NB units start free
        if (lane == 0)
            for (int i = 0; i < NB; ++i) mbar_arrive(&ready[i]);
        f2 acc[4] = {kAccInit, kAccInit, kAccInit, kAccInit};
        unsigned long long cnt = 0;
        double sum = 0.0;
        float ks = 0.0f, kc = 0.0f;   // Kahan-compensated FP32 sum of the terms
        const float off_f = static_cast<float>(A.hdr->ai_off);   // r2e + 1, exact in FP32
        int64_t t = t0;
        int32_t st = s0;
        int32_t buf = 0;
        uint32_t fph = 0;   // t_full phase parity
        int32_t rslot = 0;  // j-stage ring slot of unit q
        int32_t q = 0;
        for (; q < nu; ++q) {
            const int32_t eo0 = st * JS;
            // warp-uniform outcome: the TMEM loads below are .sync.aligned
            const bool got = __all_sync(0xFFFFFFFFu, mbar_sleep_bounded(FULL2 && ew >= 4 ? &t_full2[buf] : &t_full[buf], fph,
                                                                        A.wait_ns, abort_flag));
            if (!got) {
                if (lane == 0) {
                    flag_status(A.hdr, ST_TIMEOUT);
                    *abort_flag = 1;
                }
                break;
            }
            // the ready barrier of the unit that overwrites this accumulator next
            uint64_t *release = &ready[rslot + NB < NS ? rslot + NB : rslot + NB - NS];
            tc_fence_after();
            uint32_t v[CPW];
            const float vmin = tmem_ld_min<CPW>(tbase + lane_addr + static_cast<uint32_t>(buf * JS + part * CPW), v);
            // does any lane of the warp hold a negative value? (warp-uniform)
            const bool warp_neg = __any_sync(0xFFFFFFFFu, vmin < 0.0f);
            if (!WALK) {
                // the accumulator is in registers: hand the TMEM buffer back before
                // counting, so the next MMA into it overlaps this warp's arithmetic
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(release);
            }
            const bool full = eo0 >= TC_T && eo0 + JS - 1 <= A.h;
            if (WALK) {
                if (warp_neg) {
                    // one bit per group of 8 columns holding a negative value, warp-uniform
                    uint32_t gm = 0;
#pragma unroll
                    for (int g = 0; g < CPW / 8; ++g) {
                        uint32_t o8 = 0;
#pragma unroll
                        for (int j = 0; j < 8; ++j) o8 |= v[8 * g + j];
                        gm |= (o8 >> 31) << g;
                    }
                    gm = __reduce_or_sync(0xFFFFFFFFu, gm);
                    // spheres: this row's object (rows past n are never flagged)
                    const int64_t io = t * TC_T + row;
                    float xi = 0.0f, yi = 0.0f, zi = 0.0f, ri = 0.0f;
                    if (SPH && io < A.n) {
                        xi = A.px[io];
                        yi = A.py[io];
                        zi = A.pz[io];
                        ri = A.pr[io];
                    }
                    // columns c of this row that the schedule assigns: 1 <= d0 + c <= ev
                    int32_t clo = 0, cspan = CPW - 1;
                    if (!full) {
                        const int64_t i = t * TC_T + row;
                        const int64_t ev = i < A.n ? A.h + (((A.n & 1) == 0 && i < A.n / 2) ? 1 : 0) : -1;
                        const int64_t d0 = static_cast<int64_t>(eo0) + part * CPW - row;   // e - i of column 0
                        const int64_t lo = 1 - d0 > 0 ? 1 - d0 : 0;
                        const int64_t hi = ev - d0 < CPW - 1 ? ev - d0 : CPW - 1;
                        if (hi >= lo) {
                            clo = static_cast<int32_t>(lo);
                            cspan = static_cast<int32_t>(hi - lo);
                        } else {   // none: c - clo is negative, above any span as unsigned
                            clo = 1 << 30;
                            cspan = 0;
                        }
                    }
                    do {
                        const int g = __ffs(gm) - 1;
                        gm &= gm - 1;
                        // re-read the group from TMEM (the buffer is still held): no dynamic
                        // register indexing, and v is dead past the screen
                        uint32_t w[8], m8 = 0;
                        tmem_ld8(tbase + lane_addr + static_cast<uint32_t>(buf * JS + part * CPW + 8 * g), w);
#pragma unroll
                        for (int j = 0; j < 8; ++j) m8 |= __uint_as_float(w[j]) < 0.0f ? (1u << j) : 0u;
                        uint32_t ok = 0;   // columns 8g+j inside the row's window
#pragma unroll
                        for (int j = 0; j < 8; ++j)
                            ok |= static_cast<uint32_t>(8 * g + j - clo) <= static_cast<uint32_t>(cspan) ? (1u << j) : 0u;
                        m8 &= ok;
                        if constexpr (!SPH && !SUMT) {   // a count needs only how many
                            cnt += __popc(m8);
                            m8 = 0;
                        }
                        while (m8) {
                            const int j = __ffs(m8) - 1;
                            m8 &= m8 - 1;
                            uint32_t u = w[0];
#pragma unroll
                            for (int k = 1; k < 8; ++k) u = j == k ? w[k] : u;
                            if constexpr (SPH) {
                                // screened pair: the FP32 predicate decides (column -> object)
                                const int64_t e = io + (static_cast<int64_t>(eo0) + part * CPW + 8 * g + j - row);
                                const int64_t jo = e < A.n ? e : e - A.n;
                                float d2;
                                if (sphere_pair(xi, yi, zi, ri, A.px[jo], A.py[jo], A.pz[jo], A.pr[jo], d2)) {
                                    ++cnt;
                                    if (SUMT) kahan_add(ks, kc, term_f32(d2));
                                }
                            } else {
                                ++cnt;
                                if (SUMT) kahan_add(ks, kc, term_f32(__fadd_rn(__uint_as_float(u), off_f)));
                            }
                        }
                    } while (gm);
                }
                // the walk is done with the accumulator: hand the TMEM buffer back
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(release);
            } else if (warp_neg) {
                if (full) {
#pragma unroll
                    for (int j = 0; j < CPW / 2; ++j) {
                        const f2 pv = static_cast<f2>(v[2 * j]) | (static_cast<f2>(v[2 * j + 1]) << 32);
                        acc[j & 3] = f2_fma_rm(pv, kScale, acc[j & 3]);
                    }
                } else {
                    const int64_t i = t * TC_T + row;
                    const int64_t ev = i < A.n ? A.h + (((A.n & 1) == 0 && i < A.n / 2) ? 1 : 0) : -1;
                    const int64_t d0 = static_cast<int64_t>(eo0) + part * CPW - row;   // e - i of column 0
#pragma unroll
                    for (int j = 0; j < CPW; ++j)
                        cnt += (d0 + j >= 1 && d0 + j <= ev && __uint_as_float(v[j]) < 0.0f) ? 1u : 0u;
                }
            }
            if ((q & 1023) == 1023) {
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    cnt += acc_count(acc[a]);
                    acc[a] = kAccInit;
                }
            }
            if (++buf == NB) {
                buf = 0;
                fph ^= 1u;
            }
            if (++rslot == NS) rslot = 0;
            if (++st == K32) {
                st = 0;
                ++t;
            }
        }
        if (q < nu) {
            // Aborted at unit q (not released). The copy warp drains the stage copies it
            // issued by waiting for their ready phases, which also need this warp's
            // releases: make them (units q + NB .. issued - 1) in order, each after the
            // previous phase of its slot completed, so that no arrival lands in the wrong
            // phase. Every wait is bounded.
            const uint64_t t_stop = globaltimer_ns();
            bool have = true;
            while (!*copy_stopped) {
                if (globaltimer_ns() - t_stop > A.wait_ns) {
                    have = false;
                    break;
                }
            }
            __syncwarp();
            if (have && lane == 0) {
                const int32_t issued = *copy_issued;
                for (int32_t u = q + NB; u < issued; ++u) {
                    if (u >= NS &&
                        !mbar_wait_bounded(&ready[u % NS], static_cast<uint32_t>(((u - NS) / NS) & 1), A.wait_ns))
                        break;
                    mbar_arrive(&ready[u % NS]);
                }
            }
            __syncwarp();
        }
#pragma unroll
        for (int a = 0; a < 4; ++a) cnt += acc_count(acc[a]);
        if (SUMT) sum += static_cast<double>(ks) - static_cast<double>(kc);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            cnt += __shfl_down_sync(0xFFFFFFFFu, cnt, o);
            if (SUMT) sum += __shfl_down_sync(0xFFFFFFFFu, sum, o);
        }
        if (lane == 0) {
            red[ew] = cnt;
            if (SUMT) red_sum[ew] = sum;
        }
    }
    __syncwarp();   // lanes 1-31 of the copy and MMA warps wait for their lane 0
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tbase, 512);
    }
    if (threadIdx.x == 0) {
        unsigned long long c = 0;
        for (int i = 0; i < EPW; ++i) c += red[i];
        if (c && A.d_count) atomicAdd(A.d_count, c);
        if (SUMT) {
            // per-CTA FP64 partials, summed in CTA order by the last CTA to finish
            double sm = 0.0;
            for (int i = 0; i < EPW; ++i) sm += red_sum[i];
            A.partial[blockIdx.x] = sm;
            __threadfence();
            const unsigned ticket = atomicAdd(&A.hdr->ticket1, 1u);
            if (ticket == gridDim.x - 1) {
                __threadfence();
                double tot = 0.0;
                for (unsigned b = 0; b < gridDim.x; ++b) tot += *reinterpret_cast<volatile double *>(&A.partial[b]);
                *A.d_sum = static_cast<float>(tot);
                A.hdr->ticket1 = 0;
            }
        }
    }
}

// ---------------------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------------------

// Dynamic shared memory requested per CTA: more than half of the SM's 228 KB, so that
// exactly one CTA (and one 512-column TMEM allocation) is resident per SM.
constexpr int TC_SMEM_REQ = 120 * 1024;

// Tensor-core kernel switch: initialised from CC_TC (0 disables), then cc_set_tensor_cores.
static std::atomic<int> g_tc_enabled{-1};

bool tc_enabled() {
    int v = g_tc_enabled.load(std::memory_order_relaxed);
    if (v < 0) {
        const char *e = getenv("CC_TC");
        v = (e && e[0] == '0') ? 0 : 1;
        int expected = -1;
        g_tc_enabled.compare_exchange_strong(expected, v);
        v = g_tc_enabled.load(std::memory_order_relaxed);
    }
    return v == 1;
}

void tc_set_enabled(bool on) { g_tc_enabled.store(on ? 1 : 0, std::memory_order_relaxed); }

struct TcLaunch {
    const void *fn;
    int js, threads;
};

template <bool SUMT, bool SPH, bool WALKC>
static cc_status tc_launch_of(TcLaunch &L) {
    static_assert(TcSmem::kTotal <= TC_SMEM_REQ, "shared memory layout");
    auto fn = k_pairs_tc<SUMT, SPH, WALKC>;
    // shared-memory attribute, once per instance (thread-safe static initialisation)
    static const cudaError_t attr =
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM_REQ);
    CC_CUDA(attr);
    L.fn = reinterpret_cast<const void *>(fn);
    L.js = TC_JS;
    L.threads = TC_THREADS;
    return CC_OK;
}

// The compiled epilogue forms: the integer count in registers (dense hits) or by the walk
// (sparse hits), the integer interaction sum, and the FP32 sphere count and sum (walks
// behind the integer screen). The alternatives measured slower on GB300 are listed with
// their rates in the design notes.
enum class TcForm { CountRegisters, CountWalk, Sum, SphereCount, SphereSum };

static cc_status tc_form_launch(TcLaunch &L, TcForm f) {
    switch (f) {
        case TcForm::CountRegisters: return tc_launch_of<false, false, false>(L);
        case TcForm::CountWalk: return tc_launch_of<false, false, true>(L);
        case TcForm::Sum: return tc_launch_of<true, false, false>(L);
        case TcForm::SphereCount: return tc_launch_of<false, true, false>(L);
        default: return tc_launch_of<true, true, false>(L);
    }
}

// Enqueues the operand fill; it does nothing unless the preparation kernel chose
// MODE_I32_TC (integer points) or MODE_F32_TC (spheres) for this call. `region` holds
// tc_region_bytes(n).
cc_status tc_enqueue_fill(const cc_points *p, int64_t n, uint8_t *region, WsHeader *hdr, uint32_t *hist,
                          cudaStream_t stream) {
    TcLaunch L;
    cc_status st = tc_form_launch(L, TcForm::CountWalk);   // every form has the same stage width
    if (st != CC_OK) return st;
    const TcGeom g = tc_geometry(n, L.js);
    const int64_t rows = std::max<int64_t>(g.M * TC_T, g.elen);
    const int blocks = static_cast<int>(std::min<int64_t>((rows + 255) / 256, static_cast<int64_t>(sm_count()) * 8));
    if (p->dtype == CC_F32) {
        k_fill_tc<true><<<blocks, 256, 0, stream>>>(p->x, p->y, p->z, n, g.M * TC_T, g.elen, region,
                                                    region + g.a_bytes, hdr, nullptr);
    } else {
        k_fill_tc<false><<<blocks, 256, 0, stream>>>(p->x, p->y, p->z, n, g.M * TC_T, g.elen, region,
                                                     region + g.a_bytes, hdr, hist);
    }
    CC_CUDA(cudaGetLastError());
    return CC_OK;
}

// Enqueues the tensor-core kernel (returns at once unless the mode is MODE_I32_TC, or
// MODE_F32_TC for spheres).
cc_status tc_enqueue_pairs(const cc_points *p, int64_t n, const uint8_t *region, WsHeader *hdr,
                           unsigned long long *d_count, float *d_sum, double *partial, cudaStream_t stream) {
    TcLaunch L;
    const bool sph = p->dtype == CC_F32;
    const bool sum = d_sum != nullptr;
    cc_status st = tc_form_launch(L, sph ? (sum ? TcForm::SphereSum : TcForm::SphereCount)
                                         : (sum ? TcForm::Sum : TcForm::CountRegisters));
    if (st != CC_OK) return st;
    const TcGeom g = tc_geometry(n, L.js);
    if (g.K < TC_MIN_K) return fail(CC_ERR_INVALID_ARG, "set too small for the tensor-core kernel");
    TcArgs A;
    A.Aop = region;
    A.Bop = region + g.a_bytes;
    A.n = n;
    A.units = g.units;
    A.K = static_cast<int32_t>(g.K);
    A.h = static_cast<int32_t>((n - 1) / 2);
    A.hdr = hdr;
    A.d_count = d_count;
    A.d_sum = d_sum;
    A.partial = partial;
    A.px = sph ? static_cast<const float *>(p->x) : nullptr;
    A.py = sph ? static_cast<const float *>(p->y) : nullptr;
    A.pz = sph ? static_cast<const float *>(p->z) : nullptr;
    A.pr = sph ? p->r : nullptr;
    A.wait_ns = wait_limit_ns();
    A.stall = debug_stall();
    A.form = -1;
    const int grid = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(g.units, sm_count())));
    void *args[] = {&A};
    if (!sph && !sum) {
        // integer count: both count forms are launched and the one the preparation
        // kernel chose (hdr->tc_form, from the expected hit density) runs
        TcLaunch W;
        st = tc_form_launch(W, TcForm::CountWalk);
        if (st != CC_OK) return st;
        A.form = 0;
        CC_CUDA(cudaLaunchKernel(L.fn, dim3(grid), dim3(L.threads), args, TC_SMEM_REQ, stream));
        A.form = 1;
        CC_CUDA(cudaLaunchKernel(W.fn, dim3(grid), dim3(W.threads), args, TC_SMEM_REQ, stream));
        return CC_OK;
    }
    CC_CUDA(cudaLaunchKernel(L.fn, dim3(grid), dim3(L.threads), args, TC_SMEM_REQ, stream));
    return CC_OK;
}

}  // namespace cc

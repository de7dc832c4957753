// Single-set kernels: the balanced cyclic pair enumeration of Section 4 (proposed
// algorithm, with the even-N extra step), lifted to tiles for sm_103a.
//
// Layout in HBM (per call, in the stream's workspace):
//   WsHeader | Rec E[nrec] | double partial[grid] | uint32 hist[TC_HIST_CELLS]
// E is the "extended" sequence E[e] = P[e mod n] for e in [0, 2*nrec), stored as
// pair-interleaved 32-byte records {x0,x1,y0,y1,z0,z1,w0,w1} so that (a) every j-range
// of the cyclic schedule is one contiguous, 32-byte aligned span (no modulo in the hot
// loop, bulk-copyable by the TMA engine) and (b) two consecutive objects j, j+1 sit in
// 64-bit register pairs ready for the packed FP32x2 instructions.
//
// Work decomposition (balance is the point of the paper's scheme): the n objects are cut
// into i-tiles of T = NT*R objects; for tile start a, object i in the tile evaluates
// extended indices e = i+1 .. i+h_i (h_i = (n-1)/2, plus one for i < n/2 when n is
// even). The tile's j-range [a, a+K*JS) is cut into K stages of JS objects; every
// (tile, stage) unit holds the same T*JS candidate pairs, and each persistent CTA takes a
// contiguous, equal share of the M*K units. Only stages that touch the first T or the
// last T offsets of the range need the per-pair validity mask.
//
// Per CTA: NT consumer threads (R objects each, held in registers) plus one producer
// warp that streams j-stages into an NS-deep shared-memory ring with cp.async.bulk and
// mbarrier completion. Every wait is bounded (global timer) and reports CC_ERR_TIMEOUT.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <utility>

#include "cc_internal.cuh"
#include "cc_pairs.cuh"

#ifndef CC_OPAQUE_ISTATE
#define CC_OPAQUE_ISTATE 1
#endif

namespace cc {

// tensor-core path (cc_tc.cu)
size_t tc_region_bytes(int64_t n);
bool tc_enabled();
cc_status tc_enqueue_fill(const cc_points *p, int64_t n, uint8_t *region, WsHeader *hdr, uint32_t *hist,
                          cudaStream_t stream);
cc_status tc_enqueue_pairs(const cc_points *p, int64_t n, const uint8_t *region, WsHeader *hdr,
                           unsigned long long *d_count, float *d_sum, double *partial, cudaStream_t stream);
// Smallest set for which counts and sums take a tensor-core form (and below which they
// take the one-launch small-set kernel): 8192 objects (the measured crossover between the
// tensor-core and FP32-pipe forms: at 8192 both take about 33 us per call, at 12288 the
// tensor cores 25-30 % less), or the environment variable CC_TC_MIN_N (read once).
int64_t tc_min_n() {
    // at least 1024: the tensor-core kernel's pipeline needs every i-tile to span at least
    // two of its units (TC_MIN_K; true from n = 257 on)
    static const int64_t v = []() {
        const char *e = getenv("CC_TC_MIN_N");
        const int64_t want = e ? static_cast<int64_t>(atoll(e)) : int64_t{8192};
        return want >= 1024 ? want : int64_t{1024};
    }();
    return v;
}

// ---------------------------------------------------------------------------------------
// preparation kernels
// ---------------------------------------------------------------------------------------

// Resets the per-call words of the header and the outputs.
__global__ void k_reset(WsHeader *h, int32_t mode, unsigned long long *d_count, float *d_sum) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        for (int a = 0; a < 3; ++a) {
            h->umin[a] = 0xFFFFFFFFu;
            h->umax[a] = 0u;
        }
        h->mode = mode;
        h->cx = h->cy = h->cz = 0;
        h->ticket0 = 0;
        h->ticket1 = 0;
        h->qbad = 0u;
        h->qrmax = 0u;
        h->cstatus = 0u;
        if (d_count) *d_count = 0ull;
        if (d_sum) *d_sum = 0.0f;
    }
}

// Last kernel of every single-set call: when the device detected a condition for this
// call (a bounded wait that ran out, an integer span beyond the supported range), the
// partial results the pair kernels may have added are replaced by the invalid markers:
// CC_COUNT_INVALID for the count and a quiet NaN for the sum.
__global__ void k_finalize(const WsHeader *h, unsigned long long *d_count, float *d_sum) {
    if (threadIdx.x == 0 && blockIdx.x == 0 && h->cstatus != 0u) {
        if (d_count) *d_count = CC_COUNT_INVALID;
        if (d_sum) *d_sum = __int_as_float(0x7fc00000);
    }
}

// Per-axis min/max of the integer coordinates; the last block to finish derives the
// execution mode, the integer centre and the clamped r2 (no spin: last-block ticket).
__global__ void k_minmax(const int32_t *__restrict__ x, const int32_t *__restrict__ y,
                         const int32_t *__restrict__ z, int64_t n, uint32_t r2, WsHeader *h,
                         unsigned long long *d_count, int32_t allow_tc, uint32_t *hist) {
    // tensor-core path: clear the occupancy histogram the operand fill builds
    if (hist)
        for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < TC_HIST_CELLS;
             i += (int64_t)gridDim.x * blockDim.x)
            hist[i] = 0u;
    uint32_t mn[3] = {0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu};
    uint32_t mx[3] = {0u, 0u, 0u};
    const int32_t *c[3] = {x, y, z};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            uint32_t u = ord_enc(c[a][i]);
            mn[a] = min(mn[a], u);
            mx[a] = max(mx[a], u);
        }
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        mn[a] = __reduce_min_sync(0xFFFFFFFFu, mn[a]);
        mx[a] = __reduce_max_sync(0xFFFFFFFFu, mx[a]);
    }
    // one set of global atomics per block (per-warp atomics on the same six words serialise)
    __shared__ uint32_t wred[32][6];
    if ((threadIdx.x & 31) == 0)
        for (int a = 0; a < 3; ++a) {
            wred[threadIdx.x >> 5][a] = mn[a];
            wred[threadIdx.x >> 5][3 + a] = mx[a];
        }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < static_cast<int>(blockDim.x >> 5); ++w)
            for (int a = 0; a < 3; ++a) {
                mn[a] = min(mn[a], wred[w][a]);
                mx[a] = max(mx[a], wred[w][3 + a]);
            }
        for (int a = 0; a < 3; ++a) {
            atomicMin(&h->umin[a], mn[a]);
            atomicMax(&h->umax[a], mx[a]);
        }
    }
    __syncthreads();
    __shared__ bool last;
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(&h->ticket0, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last || threadIdx.x != 0) return;
    __threadfence();
    int64_t span[3], lo[3];
    int64_t m = 0, dmax = 0;
    bool range_ok = true;
    for (int a = 0; a < 3; ++a) {
        // L2 reads (the per-block atomics above are all in L2 and fenced by the ticket)
        lo[a] = ord_dec(__ldcg(&h->umin[a]));
        int64_t hi = ord_dec(__ldcg(&h->umax[a]));
        span[a] = hi - lo[a];
        if (span[a] > WIDE_MAX_SPAN) range_ok = false;
        m = max(m, (span[a] + 1) / 2);
        dmax += span[a] * span[a];
    }
    int32_t mode;
    if (!range_ok) {
        mode = MODE_RANGE_ERR;
        flag_status(h, ST_RANGE);
        if (d_count) *d_count = CC_COUNT_INVALID;
    } else if (m <= FAST_MAX_HALF_SPAN) {
        mode = MODE_I32_FAST;
        h->cx = static_cast<int32_t>(lo[0] + span[0] / 2);
        h->cy = static_cast<int32_t>(lo[1] + span[1] / 2);
        h->cz = static_cast<int32_t>(lo[2] + span[2] / 2);
    } else {
        mode = MODE_I32_WIDE;
    }
    int64_t r2e = static_cast<int64_t>(r2) < dmax ? static_cast<int64_t>(r2) : dmax;
    if (mode == MODE_I32_FAST && allow_tc && tc_exact(m, r2e)) mode = MODE_I32_TC;
    // Which tensor-core count form (first estimate; the operand fill refines it from an
    // occupancy histogram): the expected hits per pair of a set spread uniformly over its
    // bounding box, (lattice points within the r2 ball) / (box sites), bounded above by
    // the ball of radius sqrt(r2) + 1. Below TC_SPARSE_HITS the walk form (a lean loop;
    // measured +9 % at 1e-7) runs, above it the in-register count (+19 % at 3e-5).
    // Either form gives the exact count; only the speed depends on the choice, so the
    // estimate is FP32 (a dependent FP64 chain is slow on this part's FP64 pipe).
    {
        const float rad = sqrtf(static_cast<float>(r2e)) + 1.0f;
        const float ball = 4.18879020f * rad * rad * rad;   // (4/3) pi rad^3
        const float sites = static_cast<float>(span[0] + 1) * static_cast<float>(span[1] + 1) *
                            static_cast<float>(span[2] + 1);
        h->tc_form = ball < static_cast<float>(TC_SPARSE_HITS) * sites ? 1 : 0;
    }
    h->r2e = static_cast<uint32_t>(r2e);
    h->ai_off = static_cast<int32_t>(r2e + 1);
    h->mode = mode;
    h->ticket0 = 0;
}

// FP32 spheres, tensor-core screen: per-axis min/max of the coordinates, the largest
// |radius| and whether any value is not finite; the last block decides between the
// screened tensor-core form (MODE_F32_TC) and the FP32-pipe kernel (MODE_F32).
//
// Screen: coordinates are quantised as X = floor((x - min) * S), S = 2046 / the largest
// per-axis span, so |(X_i - X_j) - (x_i - x_j) S| < 1 per axis and the integer distance
// D of a pair is below d S + sqrt(3). A pair the FP32 predicate accepts has
// d <= |r_i + r_j| (1 + 2.5e-7) (five roundings in d^2, three in (r_i + r_j)^2), or d so
// small that d^2 underflows (then D <= sqrt(3)). So every such pair has
// D^2 <= r2q = ceil((2 rmax S (1 + 1e-6) + 1.7331)^2), and the tensor-core kernel counts
// the integer form D^2 <= r2q exactly (the same 8-term contraction as integer points,
// coordinates within [0, 2046]) and applies the FP32 predicate to those pairs only.
// Admitted while r2q <= 2048 (2 rmax at most about 2.2 % of the span), so that screened
// pairs stay rare for spread-out sets.
constexpr int64_t F32_TC_MAX_R2Q = 2048;

__global__ void k_minmax_f32(const float *__restrict__ x, const float *__restrict__ y,
                             const float *__restrict__ z, const float *__restrict__ r, int64_t n, WsHeader *h,
                             int32_t allow_tc) {
    uint32_t mn[3] = {0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu};
    uint32_t mx[3] = {0u, 0u, 0u};
    uint32_t rmax = 0u, bad = 0u;
    const float *c[3] = {x, y, z};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float v = c[a][i];
            bad |= isfinite(v) ? 0u : 1u;
            const uint32_t u = ord_enc_f(v);
            mn[a] = min(mn[a], u);
            mx[a] = max(mx[a], u);
        }
        const float rv = r[i];
        bad |= isfinite(rv) ? 0u : 1u;
        rmax = max(rmax, __float_as_uint(fabsf(rv)));   // non-negative floats order as their bits
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        mn[a] = __reduce_min_sync(0xFFFFFFFFu, mn[a]);
        mx[a] = __reduce_max_sync(0xFFFFFFFFu, mx[a]);
    }
    rmax = __reduce_max_sync(0xFFFFFFFFu, rmax);
    bad = __reduce_or_sync(0xFFFFFFFFu, bad);
    // one set of global atomics per block (per-warp atomics on the same words serialise)
    __shared__ uint32_t wred[32][8];
    if ((threadIdx.x & 31) == 0) {
        for (int a = 0; a < 3; ++a) {
            wred[threadIdx.x >> 5][a] = mn[a];
            wred[threadIdx.x >> 5][3 + a] = mx[a];
        }
        wred[threadIdx.x >> 5][6] = rmax;
        wred[threadIdx.x >> 5][7] = bad;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < static_cast<int>(blockDim.x >> 5); ++w) {
            for (int a = 0; a < 3; ++a) {
                mn[a] = min(mn[a], wred[w][a]);
                mx[a] = max(mx[a], wred[w][3 + a]);
            }
            rmax = max(rmax, wred[w][6]);
            bad |= wred[w][7];
        }
        for (int a = 0; a < 3; ++a) {
            atomicMin(&h->umin[a], mn[a]);
            atomicMax(&h->umax[a], mx[a]);
        }
        atomicMax(&h->qrmax, rmax);
        if (bad) atomicOr(&h->qbad, 1u);
    }
    __syncthreads();
    __shared__ bool last;
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(&h->ticket0, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last || threadIdx.x != 0) return;
    __threadfence();
    int32_t mode = MODE_F32;
    if (allow_tc && atomicAdd(&h->qbad, 0u) == 0u) {
        double span = 0.0;
        float lo[3];
        for (int a = 0; a < 3; ++a) {
            lo[a] = ord_dec_f(atomicAdd(&h->umin[a], 0u));
            const float hi = ord_dec_f(atomicAdd(&h->umax[a], 0u));
            span = fmax(span, static_cast<double>(hi) - static_cast<double>(lo[a]));
        }
        const double S = span > 0.0 ? 2046.0 / span : 1.0;
        const double rm = static_cast<double>(__uint_as_float(atomicAdd(&h->qrmax, 0u)));
        const double reach = 2.0 * rm * S * (1.0 + 1e-6) + 1.7331;
        if (reach < 64.0 && isfinite(S)) {
            const int64_t r2q = static_cast<int64_t>(ceil(reach * reach));
            if (r2q <= F32_TC_MAX_R2Q && tc_exact(1023, r2q)) {
                mode = MODE_F32_TC;
                for (int a = 0; a < 3; ++a) h->qmin[a] = lo[a];
                h->qscale = S;
                h->cx = h->cy = h->cz = 1023;
                h->r2e = static_cast<uint32_t>(r2q);
                h->ai_off = static_cast<int32_t>(r2q + 1);
            }
        }
    }
    h->mode = mode;
    h->ticket0 = 0;
}

// Fills the extended pair-interleaved array from integer SoA input.
__global__ void k_fill_i32(const int32_t *__restrict__ x, const int32_t *__restrict__ y,
                           const int32_t *__restrict__ z, int64_t n, int64_t nrec,
                           Rec *__restrict__ E, const WsHeader *__restrict__ h) {
    const int32_t mode = h->mode;
    if (mode == MODE_RANGE_ERR || mode == MODE_I32_TC) return;
    const int32_t cx = h->cx, cy = h->cy, cz = h->cz;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nrec;
         q += (int64_t)gridDim.x * blockDim.x) {
        Rec rec;
#pragma unroll
        for (int l = 0; l < 2; ++l) {
            int64_t e = 2 * q + l;
            int64_t p = e < n ? e : (e < 2 * n ? e - n : e % n);   // no 64-bit remainder in practice
            if (mode == MODE_I32_FAST) {
                int32_t xi = x[p] - cx, yi = y[p] - cy, zi = z[p] - cz;
                rec.x[l] = static_cast<float>(xi);
                rec.y[l] = static_cast<float>(yi);
                rec.z[l] = static_cast<float>(zi);
                rec.w[l] = static_cast<float>(xi * xi + yi * yi + zi * zi);
            } else {
                rec.x[l] = __int_as_float(x[p]);
                rec.y[l] = __int_as_float(y[p]);
                rec.z[l] = __int_as_float(z[p]);
                rec.w[l] = 0.0f;
            }
        }
        E[q] = rec;
    }
}

// Fills the extended pair-interleaved array from FP32 sphere SoA input.
__global__ void k_fill_f32(const float *__restrict__ x, const float *__restrict__ y,
                           const float *__restrict__ z, const float *__restrict__ r, int64_t n,
                           int64_t nrec, Rec *__restrict__ E, const WsHeader *__restrict__ h) {
    if (h->mode == MODE_F32_TC) return;   // the tensor-core kernel has its own operands
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nrec;
         q += (int64_t)gridDim.x * blockDim.x) {
        Rec rec;
#pragma unroll
        for (int l = 0; l < 2; ++l) {
            int64_t e = 2 * q + l;
            int64_t p = e < n ? e : (e < 2 * n ? e - n : e % n);   // no 64-bit remainder in practice
            rec.x[l] = x[p];
            rec.y[l] = y[p];
            rec.z[l] = z[p];
            rec.w[l] = r[p];
        }
        E[q] = rec;
    }
}

// ---------------------------------------------------------------------------------------
// the pair kernel
// ---------------------------------------------------------------------------------------

struct PairArgs {
    const Rec *E;
    int64_t n;
    int64_t units;      // M * K
    int32_t K;          // stages per tile
    int32_t h;          // (n-1)/2
    WsHeader *hdr;
    double *partial;    // one FP64 slot per CTA (sum only)
    unsigned long long *d_count;
    float *d_sum;
    uint64_t wait_ns;
    int32_t stall;      // test hook: producer issues no copies
    int32_t pad;
};

// Kernel classes: one kernel for integer points (fast exact-FP32 form or the integer
// difference form, chosen on the device) and one for FP32 spheres.
enum : int { CLASS_I32 = 0, CLASS_F32 = 1 };

// Loads the R objects of consumer thread `tid` for the tile starting at `a`.
template <int NT, int R>
__device__ __forceinline__ void load_i(IState<R> &s, const PairArgs &A, int32_t mode, int64_t a,
                                       int tid, int32_t ai_off) {
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int64_t i = a + tid + r * NT;
        const bool valid = i < A.n;
        float x = 0.f, y = 0.f, z = 0.f, w = 0.f;
        if (valid) {
            const Rec &q = A.E[i >> 1];
            const int l = static_cast<int>(i & 1);
            x = q.x[l];
            y = q.y[l];
            z = q.z[l];
            w = q.w[l];
        }
        if (mode == MODE_I32_FAST) {
            s.a[r] = f2_dup(-2.0f * x);
            s.b[r] = f2_dup(-2.0f * y);
            s.c[r] = f2_dup(-2.0f * z);
            s.d[r] = f2_dup(valid ? static_cast<float>(static_cast<int32_t>(w) - ai_off)
                                  : __int_as_float(0x7f800000));   // +inf: never hits
        } else if (mode == MODE_F32) {
            s.a[r] = f2_dup(valid ? x : __int_as_float(0x7fc00000));  // NaN: never hits
            s.b[r] = f2_dup(y);
            s.c[r] = f2_dup(z);
            s.d[r] = f2_dup(w);
        } else {
            s.a[r] = f2_dup(x);
            s.b[r] = f2_dup(y);
            s.c[r] = f2_dup(z);
            s.d[r] = 0;
        }
#if CC_OPAQUE_ISTATE
        // Route the duplicated operands through a shuffle so that the code generator
        // keeps them as genuine register pairs instead of rebuilding the pair before
        // every packed instruction.
        s.a[r] = __shfl_sync(0xFFFFFFFFu, s.a[r], tid & 31);
        s.b[r] = __shfl_sync(0xFFFFFFFFu, s.b[r], tid & 31);
        s.c[r] = __shfl_sync(0xFFFFFFFFu, s.c[r], tid & 31);
        s.d[r] = __shfl_sync(0xFFFFFFFFu, s.d[r], tid & 31);
#endif
    }
}

// ---------------------------------------------------------------------------------------
// warp-independent variant: every warp owns its i-tile (32*R objects) and its own
// NS-deep ring of j-stages, refilled by its own lane 0 with cp.async.bulk. Warps never
// wait for each other, so a slow warp cannot stall the others, and the masked share of
// the work shrinks with the smaller i-tile (2*32*R of every 32*R + h offsets).
// ---------------------------------------------------------------------------------------

template <int NW, int JS, int NS>
struct WarpSmem {
    static constexpr int kSlotBytes = JS * 16;
    static constexpr int kPerWarp = NS * kSlotBytes;
    static constexpr int kStages = NW * kPerWarp;
    static constexpr int kBars = NW * NS * 8;
    static constexpr int kRed = (NW + 1) * 16;
    static constexpr int kTotal = kStages + kBars + kRed + 16;
};

template <int MODE, int R, int JS, int NS, bool SUM>
__device__ __forceinline__ void warp_loop(const PairArgs &A, uint8_t *ring, uint64_t *full,
                                          int64_t u0, int64_t u1, int lane,
                                          unsigned long long &cnt64, double &sum) {
    constexpr int T = 32 * R;
    constexpr uint32_t kBytes = JS * 16;
    const int32_t ai_off = A.hdr->ai_off;
    const uint32_t r2 = A.hdr->r2e;
    const bool stall = A.stall != 0;
    int64_t issued = 0;   // copies issued (meaningful in lane 0)
    if (lane == 0 && !stall) {
        for (int64_t u = u0; u < u1 && u < u0 + NS; ++u) {
            const int slot = static_cast<int>(u - u0);
            const int64_t t = u / A.K;
            const int64_t e0 = t * T + (u - t * A.K) * JS;
            mbar_arrive_expect_tx(&full[slot], kBytes);
            bulk_g2s(ring + slot * kBytes, A.E + (e0 >> 1), kBytes, &full[slot]);
            ++issued;
        }
    }
    __syncwarp();
    IState<R> s;
    int64_t cur_tile = -1;
    int64_t q = 0;
    bool timed_out = false;
    for (int64_t u = u0; u < u1; ++u, ++q) {
        const int64_t t = u / A.K;
        const int32_t k = static_cast<int32_t>(u - t * A.K);
        if (t != cur_tile) {
            load_i<32, R>(s, A, MODE, t * T, lane, ai_off);
            cur_tile = t;
        }
        const int slot = static_cast<int>(q % NS);
        if (!mbar_wait_bounded(&full[slot], static_cast<uint32_t>((q / NS) & 1), A.wait_ns)) {
            if (lane == 0) flag_status(A.hdr, ST_TIMEOUT);
            timed_out = true;
            break;
        }
        const ulonglong2 *st = reinterpret_cast<const ulonglong2 *>(ring + slot * kBytes);
        const int32_t eo0 = k * JS;
        const bool full_stage = (MODE != MODE_I32_WIDE) && (eo0 >= T) && (eo0 + JS - 1 <= A.h);
        const uint32_t c =
            full_stage ? stage_run<MODE, 32, R, JS, false, SUM>(s, st, eo0, lane, t * T, A.n, A.h, r2, sum)
                       : stage_run<MODE, 32, R, JS, true, SUM>(s, st, eo0, lane, t * T, A.n, A.h, r2, sum);
        cnt64 += c;
        __syncwarp();
        if (lane == 0 && !stall && u + NS < u1) {
            // every lane has consumed this slot (its loads fed the arithmetic above)
            fence_proxy_async_smem();
            const int64_t un = u + NS;
            const int64_t tn = un / A.K;
            const int64_t e0 = tn * T + (un - tn * A.K) * JS;
            mbar_arrive_expect_tx(&full[slot], kBytes);
            bulk_g2s(ring + slot * kBytes, A.E + (e0 >> 1), kBytes, &full[slot]);
            ++issued;
        }
    }
    // after a timeout, wait (bounded) for the copies this warp issued but did not consume
    if (timed_out && lane == 0 && !stall) {
        for (int64_t qq = q; qq < u0 + issued - u0 && qq < q + NS; ++qq) {
            const int sl = static_cast<int>(qq % NS);
            (void)mbar_wait_bounded(&full[sl], static_cast<uint32_t>((qq / NS) & 1), A.wait_ns);
        }
    }
}

template <int CLASS, int NW, int R, int JS, int NS, bool SUM, int MINB>
__global__ void __launch_bounds__(NW * 32, MINB) k_pairs_w(PairArgs A) {
    using L = WarpSmem<NW, JS, NS>;
    extern __shared__ __align__(128) uint8_t smem[];
    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const int lane = tid & 31;
    uint8_t *ring = smem + warp * L::kPerWarp;
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + L::kStages) + warp * NS;
    unsigned long long *red_cnt = reinterpret_cast<unsigned long long *>(smem + L::kStages + L::kBars);
    double *red_sum = reinterpret_cast<double *>(red_cnt + (NW + 1));

    const int32_t hmode = A.hdr->mode;
    const int32_t mode = CLASS == CLASS_F32 ? MODE_F32 : hmode;
    // invalid, or one of the tensor-core forms runs this call
    if (mode == MODE_RANGE_ERR || mode == MODE_I32_TC || hmode == MODE_F32_TC) return;

    if (lane == 0) {
        for (int i = 0; i < NS; ++i) mbar_init(&full[i], 1);
        fence_mbar_init();
    }
    __syncwarp();

    const int64_t W = static_cast<int64_t>(gridDim.x) * NW;
    const int64_t w = static_cast<int64_t>(blockIdx.x) * NW + warp;
    const int64_t u0 = (A.units * w) / W;
    const int64_t u1 = (A.units * (w + 1)) / W;

    unsigned long long cnt64 = 0;
    double sum = 0.0;
    if (CLASS == CLASS_F32)
        warp_loop<MODE_F32, R, JS, NS, SUM>(A, ring, full, u0, u1, lane, cnt64, sum);
    else if (mode == MODE_I32_FAST)
        warp_loop<MODE_I32_FAST, R, JS, NS, SUM>(A, ring, full, u0, u1, lane, cnt64, sum);
    else
        warp_loop<MODE_I32_WIDE, R, JS, NS, SUM>(A, ring, full, u0, u1, lane, cnt64, sum);

#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        cnt64 += __shfl_down_sync(0xFFFFFFFFu, cnt64, o);
        if (SUM) sum += __shfl_down_sync(0xFFFFFFFFu, sum, o);
    }
    if (lane == 0) {
        red_cnt[warp] = cnt64;
        if (SUM) red_sum[warp] = sum;
    }
    __syncthreads();
    if (tid == 0) {
        unsigned long long c = 0;
        double sm = 0.0;
        for (int i = 0; i < NW; ++i) {
            c += red_cnt[i];
            if (SUM) sm += red_sum[i];
        }
        if (c && A.d_count) atomicAdd(A.d_count, c);
        if (SUM) {
            A.partial[blockIdx.x] = sm;
            __threadfence();
            const unsigned ticket = atomicAdd(&A.hdr->ticket1, 1u);
            if (ticket == gridDim.x - 1) {
                __threadfence();
                double tot = 0.0;
                for (unsigned b = 0; b < gridDim.x; ++b)
                    tot += *reinterpret_cast<volatile double *>(&A.partial[b]);
                *A.d_sum = static_cast<float>(tot);
                A.hdr->ticket1 = 0;
            }
        }
    }
}

// ---------------------------------------------------------------------------------------
// straightforward schedule (the comparison kernel of Section 5): CTA b takes the group of
// objects [b*G, (b+1)*G) and every warp its tile of 32*R of them against ALL later
// objects, so tiles near the start carry much more work than tiles near the end. Same
// records, same stage loop and same per-warp copy ring as the cyclic kernel; only the
// schedule differs, which isolates the effect the paper measures.
// ---------------------------------------------------------------------------------------

template <int MODE, int R, int JS, int NS>
__device__ __forceinline__ void straight_loop(const PairArgs &A, uint8_t *ring, uint64_t *full, int64_t tile,
                                              int lane, unsigned long long &cnt64) {
    constexpr int T = 32 * R;
    constexpr uint32_t kBytes = JS * 16;
    const int64_t a = tile * T;
    if (a >= A.n) return;
    const int64_t K = (A.n - a + JS - 1) / JS;   // stages from the tile start to the end
    const int32_t ai_off = A.hdr->ai_off;
    const uint32_t r2 = A.hdr->r2e;
    int64_t issued = 0;
    if (lane == 0) {
        for (int64_t k = 0; k < K && k < NS; ++k) {
            mbar_arrive_expect_tx(&full[k], kBytes);
            bulk_g2s(ring + k * kBytes, A.E + ((a + k * JS) >> 1), kBytes, &full[k]);
            ++issued;
        }
    }
    __syncwarp();
    IState<R> s;
    load_i<32, R>(s, A, MODE, a, lane, ai_off);
    double unused = 0.0;
    bool timed_out = false;
    int64_t k = 0;
    for (; k < K; ++k) {
        const int slot = static_cast<int>(k % NS);
        if (!mbar_wait_bounded(&full[slot], static_cast<uint32_t>((k / NS) & 1), A.wait_ns)) {
            if (lane == 0) flag_status(A.hdr, ST_TIMEOUT);
            timed_out = true;
            break;
        }
        const ulonglong2 *st = reinterpret_cast<const ulonglong2 *>(ring + slot * kBytes);
        const int32_t eo0 = static_cast<int32_t>(k * JS);
        const bool full_stage = (MODE != MODE_I32_WIDE) && (eo0 >= T) && (a + eo0 + JS - 1 <= A.n - 1);
        cnt64 += full_stage ? stage_run<MODE, 32, R, JS, false, false>(s, st, eo0, lane, a, A.n, -1, r2, unused)
                            : stage_run<MODE, 32, R, JS, true, false>(s, st, eo0, lane, a, A.n, -1, r2, unused);
        __syncwarp();
        if (lane == 0 && k + NS < K) {
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(&full[slot], kBytes);
            bulk_g2s(ring + slot * kBytes, A.E + ((a + (k + NS) * JS) >> 1), kBytes, &full[slot]);
            ++issued;
        }
    }
    if (timed_out && lane == 0) {
        for (int64_t kk = k; kk < issued && kk < k + NS; ++kk)
            (void)mbar_wait_bounded(&full[kk % NS], static_cast<uint32_t>((kk / NS) & 1), A.wait_ns);
    }
}

template <int CLASS, int NW, int R, int JS, int NS>
__global__ void __launch_bounds__(NW * 32, 1) k_pairs_straight(PairArgs A) {
    using L = WarpSmem<NW, JS, NS>;
    extern __shared__ __align__(128) uint8_t smem[];
    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const int lane = tid & 31;
    uint8_t *ring = smem + warp * L::kPerWarp;
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + L::kStages) + warp * NS;
    unsigned long long *red_cnt = reinterpret_cast<unsigned long long *>(smem + L::kStages + L::kBars);
    const int32_t mode = CLASS == CLASS_F32 ? MODE_F32 : A.hdr->mode;
    if (mode == MODE_RANGE_ERR) return;
    if (lane == 0) {
        for (int i = 0; i < NS; ++i) mbar_init(&full[i], 1);
        fence_mbar_init();
    }
    __syncwarp();
    const int64_t tile = static_cast<int64_t>(blockIdx.x) * NW + warp;
    unsigned long long cnt64 = 0;
    if (CLASS == CLASS_F32) straight_loop<MODE_F32, R, JS, NS>(A, ring, full, tile, lane, cnt64);
    else if (mode == MODE_I32_FAST) straight_loop<MODE_I32_FAST, R, JS, NS>(A, ring, full, tile, lane, cnt64);
    else straight_loop<MODE_I32_WIDE, R, JS, NS>(A, ring, full, tile, lane, cnt64);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cnt64 += __shfl_down_sync(0xFFFFFFFFu, cnt64, o);
    if (lane == 0) red_cnt[warp] = cnt64;
    __syncthreads();
    if (tid == 0) {
        unsigned long long c = 0;
        for (int i = 0; i < NW; ++i) c += red_cnt[i];
        if (c && A.d_count) atomicAdd(A.d_count, c);
    }
}

// ---------------------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------------------

// ---------------------------------------------------------------------------------------
// small sets (n below the tensor-core threshold): one launch, no preparation pass
// ---------------------------------------------------------------------------------------
// Warp tiles of 32*R objects and j-stages of 64 objects staged by each warp from the
// caller's arrays into its own shared-memory slot; a unit is (tile, stage) and every warp
// takes an equal contiguous share of the units (the balance of the proposed algorithm,
// Section 4). Instead of a set-wide min/max pass, each unit centres its objects on the
// midpoint of their own bounding box: the fast form (exact FP32, see FAST_MAX_HALF_SPAN)
// runs when that box's half-span is within the bound, the integer difference form
// otherwise. The set-wide span (range precondition) is reduced from the tile objects
// while the units run; per-CTA partials (count, sum, bounding box, wide flag) go to slots
// that the last CTA to finish (ticket in the header, reset by that CTA) reduces with all
// its threads in a fixed order, then it writes the count (or CC_COUNT_INVALID) and the
// sum. No global atomics are contended but the ticket.

constexpr int SMALL_WARPS = 8;   // warps per CTA
constexpr int SMALL_JS = 64;     // objects per j-stage
// r2 as compared by the fast form: every pair it evaluates has d^2 <= 12 * 1182^2, so
// clamping r2 there keeps n_i - r2e - 1 exact in FP32 without changing any decision.
constexpr uint32_t SMALL_R2E_MAX = 12u * FAST_MAX_HALF_SPAN * FAST_MAX_HALF_SPAN;

struct SmallArgs {
    const void *x, *y, *z;
    const float *r;
    int32_t n, h, K;             // objects, (n-1)/2, stages per tile
    int32_t units;
    uint32_t r2;
    WsHeader *hdr;
    unsigned long long *slot_cnt;   // one per CTA
    double *slot_sum;               // one per CTA (sums only)
    uint32_t *slot_box;             // eight words per CTA: ~min and max codes per axis, wide flag
    unsigned long long *d_count;
    float *d_sum;
};

template <int R>
struct TileRaw {
    int32_t x[R], y[R], z[R];   // raw integer coordinates of the lane's tile objects
};

// Integer units: load the stage, centre it and the tile on the unit's bounding box and
// run the fast form, or the wide form when the box is too wide for it.
template <int R, bool SUM>
__device__ __forceinline__ uint32_t small_unit_i32(const SmallArgs &A, const TileRaw<R> &tr, int32_t tile0,
                                                   int32_t k, Rec *slot, int lane, double &sum, bool &wide) {
    constexpr int T = 32 * R;
    const int32_t eo0 = k * SMALL_JS;
    const int32_t *X = static_cast<const int32_t *>(A.x);
    const int32_t *Y = static_cast<const int32_t *>(A.y);
    const int32_t *Z = static_cast<const int32_t *>(A.z);
    int32_t sx[2], sy[2], sz[2];
    uint32_t mn[3] = {0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu}, mx[3] = {0u, 0u, 0u};
#pragma unroll
    for (int l = 0; l < 2; ++l) {
        const int32_t e = tile0 + eo0 + 2 * lane + l;
        const int32_t p = e < A.n ? e : e % A.n;
        sx[l] = X[p];
        sy[l] = Y[p];
        sz[l] = Z[p];
        mn[0] = min(mn[0], ord_enc(sx[l]));
        mx[0] = max(mx[0], ord_enc(sx[l]));
        mn[1] = min(mn[1], ord_enc(sy[l]));
        mx[1] = max(mx[1], ord_enc(sy[l]));
        mn[2] = min(mn[2], ord_enc(sz[l]));
        mx[2] = max(mx[2], ord_enc(sz[l]));
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        // objects past n repeat the tile's first object (their evaluations are masked)
        mn[0] = min(mn[0], ord_enc(tr.x[r]));
        mx[0] = max(mx[0], ord_enc(tr.x[r]));
        mn[1] = min(mn[1], ord_enc(tr.y[r]));
        mx[1] = max(mx[1], ord_enc(tr.y[r]));
        mn[2] = min(mn[2], ord_enc(tr.z[r]));
        mx[2] = max(mx[2], ord_enc(tr.z[r]));
    }
    int32_t c[3];
    int64_t m = 0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int64_t lo = ord_dec(__reduce_min_sync(0xFFFFFFFFu, mn[a]));
        const int64_t hi = ord_dec(__reduce_max_sync(0xFFFFFFFFu, mx[a]));
        c[a] = static_cast<int32_t>(lo + (hi - lo) / 2);
        m = max(m, (hi - lo + 1) / 2);
    }
    const bool full = eo0 >= T && eo0 + SMALL_JS - 1 <= A.h;
    __syncwarp();   // every lane is done reading the slot's previous stage
    if (m <= FAST_MAX_HALF_SPAN) {
        const uint32_t r2e = A.r2 < SMALL_R2E_MAX ? A.r2 : SMALL_R2E_MAX;
        const int32_t ai_off = static_cast<int32_t>(r2e) + 1;
        Rec rec;
#pragma unroll
        for (int l = 0; l < 2; ++l) {
            const int32_t xi = sx[l] - c[0], yi = sy[l] - c[1], zi = sz[l] - c[2];
            rec.x[l] = static_cast<float>(xi);
            rec.y[l] = static_cast<float>(yi);
            rec.z[l] = static_cast<float>(zi);
            rec.w[l] = static_cast<float>(xi * xi + yi * yi + zi * zi);
        }
        slot[lane] = rec;
        IState<R> s;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const bool valid = tile0 + lane + 32 * r < A.n;
            const int32_t xi = tr.x[r] - c[0], yi = tr.y[r] - c[1], zi = tr.z[r] - c[2];
            s.a[r] = f2_dup(-2.0f * static_cast<float>(xi));
            s.b[r] = f2_dup(-2.0f * static_cast<float>(yi));
            s.c[r] = f2_dup(-2.0f * static_cast<float>(zi));
            s.d[r] = f2_dup(valid ? static_cast<float>(xi * xi + yi * yi + zi * zi - ai_off)
                                  : __int_as_float(0x7f800000));   // +inf: never hits
        }
        __syncwarp();
        const ulonglong2 *st = reinterpret_cast<const ulonglong2 *>(slot);
        return full ? stage_run<MODE_I32_FAST, 32, R, SMALL_JS, false, SUM>(s, st, eo0, lane, tile0, A.n, A.h, r2e,
                                                                            sum)
                    : stage_run<MODE_I32_FAST, 32, R, SMALL_JS, true, SUM>(s, st, eo0, lane, tile0, A.n, A.h, r2e,
                                                                           sum);
    }
    wide = true;
    Rec rec;
#pragma unroll
    for (int l = 0; l < 2; ++l) {
        rec.x[l] = __int_as_float(sx[l]);
        rec.y[l] = __int_as_float(sy[l]);
        rec.z[l] = __int_as_float(sz[l]);
        rec.w[l] = 0.0f;
    }
    slot[lane] = rec;
    IState<R> s;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        s.a[r] = f2_dup(__int_as_float(tr.x[r]));
        s.b[r] = f2_dup(__int_as_float(tr.y[r]));
        s.c[r] = f2_dup(__int_as_float(tr.z[r]));
        s.d[r] = 0;
    }
    __syncwarp();
    const ulonglong2 *st = reinterpret_cast<const ulonglong2 *>(slot);
    return stage_run<MODE_I32_WIDE, 32, R, SMALL_JS, true, SUM>(s, st, eo0, lane, tile0, A.n, A.h, A.r2, sum);
}

template <bool F32, int R, bool SUM>
__global__ void __launch_bounds__(SMALL_WARPS * 32, 2) k_small(SmallArgs A) {
    constexpr int T = 32 * R;
    __shared__ Rec slots[SMALL_WARPS][SMALL_JS / 2];
    __shared__ unsigned long long red_cnt[SMALL_WARPS];
    __shared__ double red_sum[SMALL_WARPS];
    __shared__ uint32_t red_box[SMALL_WARPS][7];
    __shared__ bool last;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    Rec *slot = slots[warp];
    const int64_t W = static_cast<int64_t>(gridDim.x) * SMALL_WARPS;
    const int64_t w = static_cast<int64_t>(blockIdx.x) * SMALL_WARPS + warp;
    const int32_t u0 = static_cast<int32_t>((A.units * w) / W);
    const int32_t u1 = static_cast<int32_t>((A.units * (w + 1)) / W);
    uint32_t cnt = 0;
    unsigned long long cnt64 = 0;
    double sum = 0.0;
    bool wide = false;
    // set-wide bounding box of the tile objects (range precondition), order-preserving codes
    uint32_t bmn[3] = {0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu}, bmx[3] = {0u, 0u, 0u};
    int32_t cur = -1;
    TileRaw<R> tr;
    IState<R> fs;   // spheres: the tile's register state
    const RawSet rs{A.x, A.y, A.z, A.r, A.n, 0, 0, 0, 0};
    for (int32_t u = u0; u < u1; ++u) {
        const int32_t t = u / A.K;
        const int32_t k = u - t * A.K;
        const int32_t tile0 = t * T;
        if (t != cur) {
            cur = t;
            if constexpr (F32) {
                load_i_raw<MODE_F32, R>(fs, rs, tile0, lane);
            } else {
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const int32_t i = tile0 + lane + 32 * r;
                    const int32_t ii = i < A.n ? i : tile0;   // past n: a valid object, masked
                    tr.x[r] = static_cast<const int32_t *>(A.x)[ii];
                    tr.y[r] = static_cast<const int32_t *>(A.y)[ii];
                    tr.z[r] = static_cast<const int32_t *>(A.z)[ii];
                    bmn[0] = min(bmn[0], ord_enc(tr.x[r]));
                    bmx[0] = max(bmx[0], ord_enc(tr.x[r]));
                    bmn[1] = min(bmn[1], ord_enc(tr.y[r]));
                    bmx[1] = max(bmx[1], ord_enc(tr.y[r]));
                    bmn[2] = min(bmn[2], ord_enc(tr.z[r]));
                    bmx[2] = max(bmx[2], ord_enc(tr.z[r]));
                }
            }
        }
        if constexpr (F32) {
            const int32_t eo0 = k * SMALL_JS;
            __syncwarp();
            stage_load_raw<MODE_F32>(slot, rs, tile0 + eo0, lane);
            __syncwarp();
            const ulonglong2 *st = reinterpret_cast<const ulonglong2 *>(slot);
            const bool full = eo0 >= T && eo0 + SMALL_JS - 1 <= A.h;
            cnt += full ? stage_run<MODE_F32, 32, R, SMALL_JS, false, SUM>(fs, st, eo0, lane, tile0, A.n, A.h, 0u,
                                                                           sum)
                        : stage_run<MODE_F32, 32, R, SMALL_JS, true, SUM>(fs, st, eo0, lane, tile0, A.n, A.h, 0u,
                                                                          sum);
        } else {
            cnt += small_unit_i32<R, SUM>(A, tr, tile0, k, slot, lane, sum, wide);
        }
        if (((u - u0) & 1023) == 1023) {   // keep the per-lane counter far from overflow
            cnt64 += cnt;
            cnt = 0;
        }
    }
    cnt64 += cnt;
    // ---- per CTA: counts, sums, box, wide flag -------------------------------------------
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        cnt64 += __shfl_down_sync(0xFFFFFFFFu, cnt64, o);
        if (SUM) sum += __shfl_down_sync(0xFFFFFFFFu, sum, o);
    }
    if (!F32) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            bmn[a] = __reduce_min_sync(0xFFFFFFFFu, bmn[a]);
            bmx[a] = __reduce_max_sync(0xFFFFFFFFu, bmx[a]);
        }
    }
    const uint32_t wide_any = __any_sync(0xFFFFFFFFu, wide) ? 1u : 0u;
    if (lane == 0) {
        red_cnt[warp] = cnt64;
        red_sum[warp] = sum;
        for (int a = 0; a < 3; ++a) {
            red_box[warp][a] = ~bmn[a];   // merged with max, like the maximum
            red_box[warp][3 + a] = bmx[a];
        }
        red_box[warp][6] = wide_any;
    }
    __syncthreads();
    WsHeader *h = A.hdr;
    if (threadIdx.x == 0) {
        unsigned long long c = 0;
        double sm = 0.0;
        uint32_t box[7] = {0u, 0u, 0u, 0u, 0u, 0u, 0u};
        for (int i = 0; i < SMALL_WARPS; ++i) {
            c += red_cnt[i];
            sm += red_sum[i];
            for (int j = 0; j < 7; ++j) box[j] = max(box[j], red_box[i][j]);
        }
        A.slot_cnt[blockIdx.x] = c;
        if (SUM) A.slot_sum[blockIdx.x] = sm;
        if (!F32)
            for (int j = 0; j < 7; ++j) A.slot_box[blockIdx.x * 8 + j] = box[j];
        __threadfence();
        last = atomicAdd(&h->sticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    // The last CTA adds the per-CTA slots with all its threads: thread t takes slots t,
    // t + blockDim, ..., then a fixed tree (warp shuffles, then the warps in order), so
    // the sum's rounding depends only on the grid size.
    unsigned long long tot = 0;
    double stot = 0.0;
    uint32_t bx[7] = {0u, 0u, 0u, 0u, 0u, 0u, 0u};
    for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x) {
        tot += *reinterpret_cast<volatile unsigned long long *>(&A.slot_cnt[b]);
        if (SUM) stot += *reinterpret_cast<volatile double *>(&A.slot_sum[b]);
        if (!F32)
            for (int j = 0; j < 7; ++j)
                bx[j] = max(bx[j], *reinterpret_cast<volatile uint32_t *>(&A.slot_box[b * 8 + j]));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        tot += __shfl_down_sync(0xFFFFFFFFu, tot, o);
        if (SUM) stot += __shfl_down_sync(0xFFFFFFFFu, stot, o);
    }
    if (!F32)
        for (int j = 0; j < 7; ++j) bx[j] = __reduce_max_sync(0xFFFFFFFFu, bx[j]);
    if (lane == 0) {
        red_cnt[warp] = tot;
        red_sum[warp] = stot;
        for (int j = 0; j < 7; ++j) red_box[warp][j] = bx[j];
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    tot = 0;
    stot = 0.0;
    for (int i = 0; i < SMALL_WARPS; ++i) {
        tot += red_cnt[i];
        if (SUM) stot += red_sum[i];
        for (int j = 0; j < 7; ++j) bx[j] = max(bx[j], red_box[i][j]);
    }
    int32_t mode = MODE_F32;
    if (!F32) {
        bool range_ok = true;
        for (int a = 0; a < 3; ++a) {
            const int64_t lo = ord_dec(~bx[a]);
            const int64_t hi = ord_dec(bx[3 + a]);
            if (hi - lo > WIDE_MAX_SPAN) range_ok = false;
        }
        mode = !range_ok ? MODE_RANGE_ERR : (bx[6] ? MODE_I32_WIDE : MODE_I32_FAST);
        if (!range_ok) flag_status(h, ST_RANGE);
    }
    h->mode = mode;
    h->sticket = 0u;
    if (A.d_count) *A.d_count = mode == MODE_RANGE_ERR ? CC_COUNT_INVALID : tot;
    if (SUM) *A.d_sum = mode == MODE_RANGE_ERR ? __int_as_float(0x7fc00000) : static_cast<float>(stot);
}

struct SmallLaunch {
    const void *fn;
    int R;
};

template <bool F32, int R, bool SUM>
static SmallLaunch small_launch_of() {
    return SmallLaunch{reinterpret_cast<const void *>(k_small<F32, R, SUM>), R};
}

// Objects per lane of the small-set kernel: 2 below 3072 objects (more, smaller units for
// the few objects there are), else 4 (measured per call: 9.6 against 11.3 us at 2500
// objects, 16.4 against 11.3 us at 4096).
static SmallLaunch small_pick(int64_t n, bool f32, bool sum) {
    if (n < 3072) {
        if (f32) return sum ? small_launch_of<true, 2, true>() : small_launch_of<true, 2, false>();
        return sum ? small_launch_of<false, 2, true>() : small_launch_of<false, 2, false>();
    }
    if (f32) return sum ? small_launch_of<true, 4, true>() : small_launch_of<true, 4, false>();
    return sum ? small_launch_of<false, 4, true>() : small_launch_of<false, 4, false>();
}

struct SmallGeom {
    int32_t K, units, grid;
};

static SmallGeom small_geometry(int64_t n, int R) {
    SmallGeom g;
    const int64_t T = 32 * R;
    const int64_t h = (n - 1) / 2;
    const int64_t M = (n + T - 1) / T;
    g.K = static_cast<int32_t>((T + h + 1 + SMALL_JS - 1) / SMALL_JS);
    g.units = static_cast<int32_t>(M * g.K);
    g.grid = static_cast<int>(std::max<int64_t>(
        1, std::min<int64_t>((g.units + SMALL_WARPS - 1) / SMALL_WARPS, static_cast<int64_t>(sm_count()) * 2)));
    return g;
}

// ---------------------------------------------------------------------------------------
// host side of the large-set path
// ---------------------------------------------------------------------------------------

struct Launch {
    SingleCfg cfg;       // cfg.nt = 32 (objects' stride inside a warp tile); tile = 32 * cfg.r
    const void *fn;
    int smem;
    int blocks_per_sm;
    int threads;         // threads per CTA
};

template <int CLASS, int NW, int R, int JS, int NS, bool SUM>
static cc_status get_launch_w(Launch &L) {
    using S = WarpSmem<NW, JS, NS>;
    // attribute and occupancy, once per instance (thread-safe static initialisation)
    static const std::pair<cudaError_t, int> once = []() {
        auto f = k_pairs_w<CLASS, NW, R, JS, NS, SUM, 1>;
        cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, S::kTotal);
        int b = 0;
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, f, NW * 32, S::kTotal);
        return std::make_pair(e, std::max(b, 1));
    }();
    CC_CUDA(once.first);
    L.cfg = SingleCfg{32, R, JS, NS};
    L.fn = reinterpret_cast<const void *>(k_pairs_w<CLASS, NW, R, JS, NS, SUM, 1>);
    L.smem = S::kTotal;
    L.blocks_per_sm = once.second;
    L.threads = NW * 32;
    return CC_OK;
}

// FP32-pipe kernel shapes (warps per CTA, objects per lane, stage width, ring depth):
// large sets 12 x 8 objects per lane, 256-object stages, 4-deep rings (the measured
// best on GB300, with the object state kept in genuine register pairs, see load_i);
// mid-size sets (from the small-set limit to 65536) 8 x 4, 128-object stages, 4-deep.
template <int CLASS, bool SUM>
static cc_status pick_class(int64_t n, Launch &L) {
    if (n >= 65536) return get_launch_w<CLASS, 12, 8, 256, 4, SUM>(L);
    return get_launch_w<CLASS, 8, 4, 128, 4, SUM>(L);
}

// Geometry of one call.
struct Geometry {
    int64_t M, K, units, nrec;
    int grid;
};

static Geometry geometry(int64_t n, const Launch &L) {
    Geometry g;
    const int64_t T = static_cast<int64_t>(L.cfg.nt) * L.cfg.r;
    const int64_t h = (n - 1) / 2;
    g.M = (n + T - 1) / T;
    g.K = (T + h + 1 + L.cfg.js - 1) / L.cfg.js;
    g.units = g.M * g.K;
    const int64_t elen = (g.M - 1) * T + g.K * L.cfg.js;
    g.nrec = elen / 2;
    const int64_t slots = static_cast<int64_t>(sm_count()) * L.blocks_per_sm;
    const int64_t per_cta = L.threads / 32;   // units are split per warp
    g.grid = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>((g.units + per_cta - 1) / per_cta, slots)));
    return g;
}

static cc_status pick_launch(int64_t n, bool f32, bool sum, Launch &L) {
    if (f32) return sum ? pick_class<CLASS_F32, true>(n, L) : pick_class<CLASS_F32, false>(n, L);
    return sum ? pick_class<CLASS_I32, true>(n, L) : pick_class<CLASS_I32, false>(n, L);
}

static bool use_tc(int64_t n, bool allow_tc) { return allow_tc && n >= tc_min_n() && tc_enabled(); }

// Sets below this size take the one-launch small-set kernel.
static bool use_small(int64_t n) { return n < tc_min_n(); }

// Record region and per-CTA slots of the large-set path: the larger over both kernel
// classes (and the tensor-core operands when they may run), so that one workspace serves
// counts and sums of either dtype.
struct Regions {
    size_t region, slots;
};

static cc_status large_regions(int64_t n, bool sum, bool tc, Regions &R) {
    R.region = 0;
    R.slots = static_cast<size_t>(sm_count());
    for (bool f32 : {false, true}) {
        Launch L;
        const cc_status st = pick_launch(n, f32, sum, L);
        if (st != CC_OK) return st;
        const Geometry g = geometry(n, L);
        R.region = std::max(R.region, static_cast<size_t>(g.nrec) * sizeof(Rec));
        R.slots = std::max(R.slots, static_cast<size_t>(g.grid));
    }
    if (tc) R.region = std::max(R.region, tc_region_bytes(n));
    R.region = (R.region + 255) & ~static_cast<size_t>(255);
    return CC_OK;
}

// Workspace layout: WsHeader | region | double partial[slots] | uint32 hist[TC_HIST_CELLS],
// where the region holds the extended record array or (tensor-core mode) the two operand
// arrays, and the histogram is the integer tensor-core path's occupancy count. Small
// sets: WsHeader | u64 count slots | FP64 sum slots (one each per CTA).
size_t single_ws_bytes(int64_t n, bool sum, bool allow_tc) {
    if (n < 2) return sizeof(WsHeader);
    if (use_small(n)) {
        const size_t slots = static_cast<size_t>(sm_count()) * 2;
        return sizeof(WsHeader) + slots * (sizeof(unsigned long long) + sizeof(double) + 8 * sizeof(uint32_t)) + 256;
    }
    Regions R;
    if (large_regions(n, sum, use_tc(n, allow_tc), R) != CC_OK) return 0;
    return sizeof(WsHeader) + R.region + R.slots * sizeof(double) + TC_HIST_CELLS * sizeof(uint32_t) + 256;
}

static cc_status small_enqueue(const cc_points *p, int64_t n, uint32_t r2, unsigned long long *d_count,
                               float *d_sum, void *ws, cudaStream_t stream) {
    WsHeader *hdr = reinterpret_cast<WsHeader *>(ws);
    const bool f32 = p->dtype == CC_F32;
    const SmallLaunch L = small_pick(n, f32, d_sum != nullptr);
    const SmallGeom g = small_geometry(n, L.R);
    const size_t slots = static_cast<size_t>(sm_count()) * 2;
    uint8_t *base = reinterpret_cast<uint8_t *>(ws) + sizeof(WsHeader);
    SmallArgs A;
    A.x = p->x;
    A.y = p->y;
    A.z = p->z;
    A.r = f32 ? p->r : nullptr;
    A.n = static_cast<int32_t>(n);
    A.h = static_cast<int32_t>((n - 1) / 2);
    A.K = g.K;
    A.units = g.units;
    A.r2 = r2;
    A.hdr = hdr;
    A.slot_cnt = reinterpret_cast<unsigned long long *>(base);
    A.slot_sum = reinterpret_cast<double *>(base + slots * sizeof(unsigned long long));
    A.slot_box = reinterpret_cast<uint32_t *>(base + slots * (sizeof(unsigned long long) + sizeof(double)));
    A.d_count = d_count;
    A.d_sum = d_sum;
    void *args[] = {&A};
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    const bool prof = profiling();
    if (prof) CC_CUDA(profile_begin(stream, &e0, &e1));
    CC_CUDA(cudaLaunchKernel(L.fn, dim3(g.grid), dim3(SMALL_WARPS * 32), args, 0, stream));
    if (prof) profile_end(stream, e0, e1);
    return CC_OK;
}

// Enqueues the whole single-set path on `stream` using workspace `ws` (>= single_ws_bytes).
cc_status single_enqueue(const cc_points *p, int64_t n, uint32_t r2, unsigned long long *d_count,
                         float *d_sum, void *ws, cudaStream_t stream, bool allow_tc) {
    WsHeader *hdr = reinterpret_cast<WsHeader *>(ws);
    const bool f32 = p->dtype == CC_F32;
    if (n >= 2 && use_small(n)) return small_enqueue(p, n, r2, d_count, d_sum, ws, stream);
    k_reset<<<1, 32, 0, stream>>>(hdr, f32 ? MODE_F32 : MODE_I32_FAST, d_count, d_sum);
    CC_CUDA(cudaGetLastError());
    if (n < 2) return CC_OK;
    const bool sum = d_sum != nullptr;
    Launch L;
    cc_status st = pick_launch(n, f32, sum, L);
    if (st != CC_OK) return st;
    Geometry g = geometry(n, L);
    const bool tc = use_tc(n, allow_tc);
    Regions R;
    st = large_regions(n, sum, tc, R);
    if (st != CC_OK) return st;
    uint8_t *region = reinterpret_cast<uint8_t *>(ws) + sizeof(WsHeader);
    Rec *E = reinterpret_cast<Rec *>(region);
    double *partial = reinterpret_cast<double *>(region + R.region);
    uint32_t *hist = reinterpret_cast<uint32_t *>(partial + R.slots);
    const int prep_threads = 256;
    const int64_t prep_blocks_full = (g.nrec + prep_threads - 1) / prep_threads;
    const int prep_blocks = static_cast<int>(std::min<int64_t>(prep_blocks_full, sm_count() * 8));
    if (!f32) {
        const int mm_blocks = static_cast<int>(std::min<int64_t>((n + 255) / 256, sm_count() * 2));
        k_minmax<<<mm_blocks, 256, 0, stream>>>(static_cast<const int32_t *>(p->x),
                                                 static_cast<const int32_t *>(p->y),
                                                 static_cast<const int32_t *>(p->z), n, r2, hdr,
                                                 d_count, tc ? 1 : 0, tc ? hist : nullptr);
        CC_CUDA(cudaGetLastError());
        k_fill_i32<<<prep_blocks, prep_threads, 0, stream>>>(
            static_cast<const int32_t *>(p->x), static_cast<const int32_t *>(p->y),
            static_cast<const int32_t *>(p->z), n, g.nrec, E, hdr);
        CC_CUDA(cudaGetLastError());
        if (tc) {
            st = tc_enqueue_fill(p, n, region, hdr, f32 ? nullptr : hist, stream);
            if (st != CC_OK) return st;
        }
    } else {
        if (tc) {
            const int mm_blocks = static_cast<int>(std::min<int64_t>((n + 255) / 256, sm_count() * 2));
            k_minmax_f32<<<mm_blocks, 256, 0, stream>>>(static_cast<const float *>(p->x),
                                                         static_cast<const float *>(p->y),
                                                         static_cast<const float *>(p->z), p->r, n, hdr, 1);
            CC_CUDA(cudaGetLastError());
        }
        k_fill_f32<<<prep_blocks, prep_threads, 0, stream>>>(
            static_cast<const float *>(p->x), static_cast<const float *>(p->y),
            static_cast<const float *>(p->z), p->r, n, g.nrec, E, hdr);
        CC_CUDA(cudaGetLastError());
        if (tc) {
            st = tc_enqueue_fill(p, n, region, hdr, f32 ? nullptr : hist, stream);
            if (st != CC_OK) return st;
        }
    }
    CC_CUDA(cudaGetLastError());
    PairArgs A;
    A.E = E;
    A.n = n;
    A.units = g.units;
    A.K = static_cast<int32_t>(g.K);
    A.h = static_cast<int32_t>((n - 1) / 2);
    A.hdr = hdr;
    A.partial = partial;
    A.d_count = d_count;
    A.d_sum = d_sum;
    A.wait_ns = wait_limit_ns();
    A.stall = debug_stall();
    A.pad = 0;
    void *args[] = {&A};
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    const bool prof = profiling();
    if (prof) CC_CUDA(profile_begin(stream, &e0, &e1));
    // In tensor-core mode the device picks between the two kernels: each returns at once
    // unless the preparation kernel chose its mode (integer points: MODE_I32_TC or an
    // FP32-pipe mode; spheres: MODE_F32_TC or MODE_F32).
    if (tc) {
        st = tc_enqueue_pairs(p, n, region, hdr, d_count, d_sum, partial, stream);
        if (st != CC_OK) return st;
    }
    CC_CUDA(cudaLaunchKernel(L.fn, dim3(g.grid), dim3(L.threads), args, L.smem, stream));
    if (prof) profile_end(stream, e0, e1);
    k_finalize<<<1, 32, 0, stream>>>(hdr, d_count, d_sum);
    CC_CUDA(cudaGetLastError());
    return CC_OK;
}

// Straightforward-schedule count (comparison path): same preparation, records padded to
// whole stages, one CTA per group of 1024 objects.
size_t straight_ws_bytes(int64_t n) {
    constexpr int JS = 256;
    // a tile may start mid-stage, so its last stage can end up to JS objects past n
    const int64_t nrec = ((n + JS - 1) / JS + 1) * JS / 2;
    return sizeof(WsHeader) + static_cast<size_t>(nrec) * sizeof(Rec) + 256;
}

cc_status straight_enqueue(const cc_points *p, int64_t n, uint32_t r2, unsigned long long *d_count, void *ws,
                           cudaStream_t stream) {
    constexpr int NW = 8, R = 4, JS = 256, NS = 4;
    WsHeader *hdr = reinterpret_cast<WsHeader *>(ws);
    const bool f32 = p->dtype == CC_F32;
    k_reset<<<1, 32, 0, stream>>>(hdr, f32 ? MODE_F32 : MODE_I32_FAST, d_count, nullptr);
    CC_CUDA(cudaGetLastError());
    if (n < 2) return CC_OK;
    Rec *E = reinterpret_cast<Rec *>(reinterpret_cast<uint8_t *>(ws) + sizeof(WsHeader));
    const int64_t nrec = ((n + JS - 1) / JS + 1) * JS / 2;   // see straight_ws_bytes
    const int blocks = static_cast<int>(std::min<int64_t>((nrec + 255) / 256, sm_count() * 8));
    if (!f32) {
        const int mm_blocks = static_cast<int>(std::min<int64_t>((n + 255) / 256, sm_count() * 2));
        k_minmax<<<mm_blocks, 256, 0, stream>>>(static_cast<const int32_t *>(p->x),
                                                 static_cast<const int32_t *>(p->y),
                                                 static_cast<const int32_t *>(p->z), n, r2, hdr, d_count, 0,
                                                 nullptr);
        k_fill_i32<<<blocks, 256, 0, stream>>>(static_cast<const int32_t *>(p->x),
                                               static_cast<const int32_t *>(p->y),
                                               static_cast<const int32_t *>(p->z), n, nrec, E, hdr);
    } else {
        k_fill_f32<<<blocks, 256, 0, stream>>>(static_cast<const float *>(p->x), static_cast<const float *>(p->y),
                                               static_cast<const float *>(p->z), p->r, n, nrec, E, hdr);
    }
    CC_CUDA(cudaGetLastError());
    using L = WarpSmem<NW, JS, NS>;
    const void *fn = f32 ? reinterpret_cast<const void *>(k_pairs_straight<CLASS_F32, NW, R, JS, NS>)
                         : reinterpret_cast<const void *>(k_pairs_straight<CLASS_I32, NW, R, JS, NS>);
    // shared-memory attribute, once per kernel class (thread-safe static initialisation)
    static const cudaError_t attr_i32 = cudaFuncSetAttribute(
        k_pairs_straight<CLASS_I32, NW, R, JS, NS>, cudaFuncAttributeMaxDynamicSharedMemorySize, L::kTotal);
    static const cudaError_t attr_f32 = cudaFuncSetAttribute(
        k_pairs_straight<CLASS_F32, NW, R, JS, NS>, cudaFuncAttributeMaxDynamicSharedMemorySize, L::kTotal);
    CC_CUDA(f32 ? attr_f32 : attr_i32);
    PairArgs A{};
    A.E = E;
    A.n = n;
    A.units = 0;
    A.K = 0;
    A.h = -1;
    A.hdr = hdr;
    A.d_count = d_count;
    A.wait_ns = wait_limit_ns();
    void *args[] = {&A};
    const int grid = static_cast<int>((n + NW * 32 * R - 1) / (NW * 32 * R));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    const bool prof = profiling();
    if (prof) CC_CUDA(profile_begin(stream, &e0, &e1));
    CC_CUDA(cudaLaunchKernel(fn, dim3(grid), dim3(NW * 32), args, L::kTotal, stream));
    if (prof) profile_end(stream, e0, e1);
    k_finalize<<<1, 32, 0, stream>>>(hdr, d_count, nullptr);
    CC_CUDA(cudaGetLastError());
    return CC_OK;
}

// Range check only: reset + per-axis min/max (sets ST_RANGE in the header status).
cc_status validate_enqueue(const cc_points *p, int64_t n, void *ws, cudaStream_t stream) {
    WsHeader *hdr = reinterpret_cast<WsHeader *>(ws);
    k_reset<<<1, 32, 0, stream>>>(hdr, MODE_I32_FAST, nullptr, nullptr);
    CC_CUDA(cudaGetLastError());
    const int mm_blocks = static_cast<int>(std::min<int64_t>((n + 255) / 256, sm_count() * 2));
    k_minmax<<<mm_blocks, 256, 0, stream>>>(static_cast<const int32_t *>(p->x),
                                             static_cast<const int32_t *>(p->y),
                                             static_cast<const int32_t *>(p->z), n, 0u, hdr, nullptr, 0, nullptr);
    CC_CUDA(cudaGetLastError());
    return CC_OK;
}

}  // namespace cc

// Batched sets: many independent sets (the pruned cells a broad phase emits) in one
// persistent launch with a device-built work queue, replayed as one CUDA graph.
//
// Each set runs the proposed algorithm of Section 4 on its own: object i of a set of n
// evaluates (i+s) mod n for s = 1..(n-1)/2, plus s = n/2 for i < n/2 when n is even.
// A set is cut like the single-set kernel: warp tiles of 32*R objects, each with its
// extended j-range [tile start, +K*64) cut into stages of 64 objects; a work item is
// (set, tile, chunk of SC stages). Because every object does the same number of steps,
// all tiles of a set carry the same work. The warp stages each 64-object j-stage into
// its own shared-memory slot (centred exact-FP32 records for integer sets) and runs the
// same stage loop as the single-set kernel. R and SC come from a per-size-band table
// (the autotuner writes it); tile choice is a pure function of (n, table), so results
// are reproducible.
//
// Graph (all kernels read the call's parameters from a device descriptor, so the
// captured graph is replayed unchanged for every call):
//   k_b_prepare  one warp per set: set descriptor, per-set range check, item count
//   k_b_scan1/2  exclusive prefix sum of the item counts (two levels)
//   k_b_emit     one warp per set: writes its items to the queue
//   k_b_main     persistent warps pull items with an atomic cursor; per-item partials
//   k_b_finish   one warp per set: fixed-order sum of its items' partials
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "cc_internal.cuh"
#include "cc_pairs.cuh"

namespace cc {

constexpr int kMaxBands = 8;
constexpr int kScanBlock = 1024;
constexpr int kJSB = 64;          // objects per staged j-stage
constexpr int kMainWarps = 8;     // warps per CTA of the main kernel
constexpr int kWarpSetMax = 256;  // largest set a band with r = 0 (one warp per set) may take

struct Band {
    int64_t n_max;   // sets with n <= n_max (and above the previous band) use this band
    int32_t r;       // objects per lane (1, 2 or 4): warp tile of 32*r objects
    int32_t sc;      // stages (of 64 objects) per work item; 0 = the whole tile range
};

// Per-set execution data derived on the device by the prepare kernel.
struct SetAux {
    int32_t cx, cy, cz;   // integer centre (fast integer form)
    int32_t mode;         // MODE_I32_FAST / MODE_I32_WIDE / MODE_F32
    uint32_t r2e;         // r2 clamped to the largest possible squared distance
    int32_t ai_off;       // r2e + 1
    int32_t pad[2];
};

struct BandTable {
    int32_t count;
    int32_t pad;
    Band band[kMaxBands];
};

// One set of the batch.
struct SetDesc {
    const void *x, *y, *z;
    const float *r;
    int64_t n;
    int32_t dtype;
    uint32_t r2;
};

// Per-call parameters (device-resident, rewritten before each graph replay).
struct BatchParams {
    cc_points pts;                 // shared coordinate arrays (offsets mode)
    const int64_t *offsets;        // device offsets, or NULL when sets[] is pre-filled
    int32_t n_sets;
    uint32_t r2;
    int32_t want_sum;
    int32_t pad;
    unsigned long long *d_counts;
    float *d_sums;
};

// Device-side state of a plan.
struct BatchState {
    int64_t total_items;
    int64_t cursor;
    uint32_t status;
    uint32_t pad;
};

struct Item {
    int32_t set;
    int32_t local;
};

enum : uint32_t { SET_OK = 0, SET_BAD_RANGE = 1, SET_BAD_OFFSETS = 2, SET_OVERFLOW = 4 };

__device__ __forceinline__ const Band &band_of(const BandTable &bt, int64_t n) {
    for (int b = 0; b < bt.count - 1; ++b)
        if (n <= bt.band[b].n_max) return bt.band[b];
    return bt.band[bt.count - 1];
}

// The helpers below take the integer type I: int64_t on the host (a plan's point budget
// may pass 2^31), int32_t on the device, where every set has fewer than 2^31 objects
// (larger sets are flagged by the prepare kernel) and a 32-bit division by the band's
// runtime widths costs a fraction of a 64-bit one (these run once per set and per item).
template <typename I>
__host__ __device__ __forceinline__ I tile_of(const Band &b) { return 32 * static_cast<I>(b.r); }

// Tiles of a set, ceil(n / T), written so that n close to the largest I cannot overflow.
template <typename I>
__host__ __device__ __forceinline__ I tiles_of(const Band &b, I n) {
    return n > 0 ? (n - 1) / tile_of<I>(b) + 1 : 0;
}

// Stages (of kJSB objects) in one tile's extended j-range: offsets 0 .. T + h.
template <typename I>
__host__ __device__ __forceinline__ I stages_of(const Band &b, I n) {
    const I h = (n - 1) / 2;
    return (tile_of<I>(b) + h + 1 + kJSB - 1) / kJSB;
}

// Most work items one set may produce, beyond one per tile: without a bound the items of a
// set would grow with n^2 (tiles times chunks), and with them the queue a plan reserves.
constexpr int64_t kMaxItemsPerSet = 16384;

// Stages (of kJSB objects) per work item: the band's sc (0 = the whole tile range),
// widened where needed so that a set has at most max(tiles, kMaxItemsPerSet) items.
template <typename I>
__host__ __device__ __forceinline__ I chunk_stages(const Band &b, I n) {
    const I K = stages_of<I>(b, n);
    const I M = tiles_of<I>(b, n);
    I per = b.sc > 0 ? static_cast<I>(b.sc) : K;
    const I cap = static_cast<I>(kMaxItemsPerSet);
    const I maxch = cap / M > 1 ? cap / M : 1;
    if ((K + per - 1) / per > maxch) per = (K + maxch - 1) / maxch;
    return per;
}

template <typename I>
__host__ __device__ __forceinline__ I chunks_of(const Band &b, I n) {
    const I K = stages_of<I>(b, n);
    const I per = chunk_stages<I>(b, n);
    return (K + per - 1) / per;
}

// Work items of a set: tiles times chunks, at most max(tiles, kMaxItemsPerSet) (so it
// fits I whenever n does).
template <typename I>
__host__ __device__ __forceinline__ I items_of(const Band &b, I n) {
    if (n < 2) return 0;
    if (b.r == 0) return 1;   // one warp per set (sets of at most kWarpSetMax objects)
    return tiles_of<I>(b, n) * chunks_of<I>(b, n);
}

// ---------------------------------------------------------------------------------------

template <int MODE, bool SUM>
__device__ void run_tiny(const SetDesc &d, const SetAux &x, unsigned long long &cnt_out, double &sum_out);

// Sets of at most 32 objects on a one-warp-per-set band are counted by the prepare kernel
// itself, by the warp that has just reduced them (their objects are in its lanes' cache
// lines): they get no work item, and their count and sum go to dcnt / dsum.
__global__ void k_b_prepare(const BatchParams *__restrict__ P, SetDesc *sets, SetAux *aux,
                            const BandTable *bt, int32_t *cnt, uint32_t *flags, BatchState *st,
                            unsigned long long *dcnt, double *dsum) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int32_t S = P->n_sets;
    if (warp == 0 && lane == 0) {
        st->cursor = 0;
        st->status = 0;
    }
    // the offsets of this warp's next set are loaded while the current one is reduced
    int64_t na = 0, nb = 0;
    if (P->offsets && warp < S) {
        na = P->offsets[warp];
        nb = P->offsets[warp + 1];
    }
    for (int64_t k = warp; k < S; k += nwarps) {
        SetDesc d;
        uint32_t flag = SET_OK;
        if (P->offsets) {
            const int64_t a = na, b = nb;
            if (k + nwarps < S) {
                na = P->offsets[k + nwarps];
                nb = P->offsets[k + nwarps + 1];
            }
            const size_t es = 4;
            d.x = static_cast<const char *>(P->pts.x) + a * es;
            d.y = static_cast<const char *>(P->pts.y) + a * es;
            d.z = static_cast<const char *>(P->pts.z) + a * es;
            d.r = P->pts.dtype == CC_F32 ? P->pts.r + a : nullptr;
            d.n = b - a;
            d.dtype = P->pts.dtype;
            d.r2 = P->r2;
            if (a < 0 || b < a || b - a >= (int64_t(1) << 31)) {
                flag = SET_BAD_OFFSETS;
                d.n = 0;
            }
            if (lane == 0) sets[k] = d;
        } else {
            d = sets[k];
            if (d.n < 0 || d.n >= (int64_t(1) << 31)) {   // the per-set arithmetic is 32-bit
                flag = SET_BAD_OFFSETS;
                d.n = 0;
            }
        }
        SetAux x{};
        x.mode = MODE_F32;
        // integer sets: per-axis range (precondition span <= 32767), centre, mode
        if (flag == SET_OK && d.dtype == CC_I32 && d.n >= 2) {
            uint32_t mn[3] = {0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu}, mx[3] = {0, 0, 0};
            const int32_t *c[3] = {static_cast<const int32_t *>(d.x), static_cast<const int32_t *>(d.y),
                                   static_cast<const int32_t *>(d.z)};
            // four elements per lane per step, all loads issued before the reductions (a
            // set of up to 128 objects costs one memory latency)
            int64_t i = lane;
            for (; i + 96 < d.n; i += 128) {
                uint32_t u[3][4];
#pragma unroll
                for (int a = 0; a < 3; ++a)
#pragma unroll
                    for (int e = 0; e < 4; ++e) u[a][e] = ord_enc(c[a][i + 32 * e]);
#pragma unroll
                for (int a = 0; a < 3; ++a)
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        mn[a] = min(mn[a], u[a][e]);
                        mx[a] = max(mx[a], u[a][e]);
                    }
            }
            {
                uint32_t u[3][4];
                bool ok[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) ok[e] = i + 32 * e < d.n;
#pragma unroll
                for (int a = 0; a < 3; ++a)
#pragma unroll
                    for (int e = 0; e < 4; ++e) u[a][e] = ok[e] ? ord_enc(c[a][i + 32 * e]) : 0u;
#pragma unroll
                for (int a = 0; a < 3; ++a)
#pragma unroll
                    for (int e = 0; e < 4; ++e)
                        if (ok[e]) {
                            mn[a] = min(mn[a], u[a][e]);
                            mx[a] = max(mx[a], u[a][e]);
                        }
            }
            int64_t m = 0, dmax = 0, lo[3], span[3];
            for (int a = 0; a < 3; ++a) {
                mn[a] = __reduce_min_sync(0xFFFFFFFFu, mn[a]);
                mx[a] = __reduce_max_sync(0xFFFFFFFFu, mx[a]);
                lo[a] = ord_dec(mn[a]);
                span[a] = static_cast<int64_t>(ord_dec(mx[a])) - lo[a];
                if (span[a] > WIDE_MAX_SPAN) flag = SET_BAD_RANGE;
                m = max(m, (span[a] + 1) / 2);
                dmax += span[a] * span[a];
            }
            const int64_t r2e = static_cast<int64_t>(d.r2) < dmax ? static_cast<int64_t>(d.r2) : dmax;
            x.r2e = static_cast<uint32_t>(r2e);
            x.ai_off = static_cast<int32_t>(r2e + 1);
            if (m <= FAST_MAX_HALF_SPAN) {
                x.mode = MODE_I32_FAST;
                x.cx = static_cast<int32_t>(lo[0] + span[0] / 2);
                x.cy = static_cast<int32_t>(lo[1] + span[1] / 2);
                x.cz = static_cast<int32_t>(lo[2] + span[2] / 2);
            } else {
                x.mode = MODE_I32_WIDE;
            }
        } else if (d.dtype == CC_I32) {
            x.mode = MODE_I32_WIDE;
        }
        const Band &bb = band_of(*bt, d.n);
        const bool direct = flag == SET_OK && bb.r == 0 && d.n >= 2 && d.n <= 32;   // warp-uniform
        unsigned long long dc = 0;
        double ds = 0.0;
        if (direct) {
            const bool sum = P->want_sum != 0;
            if (x.mode == MODE_I32_FAST) {
                if (sum) run_tiny<MODE_I32_FAST, true>(d, x, dc, ds);
                else run_tiny<MODE_I32_FAST, false>(d, x, dc, ds);
            } else if (x.mode == MODE_F32) {
                if (sum) run_tiny<MODE_F32, true>(d, x, dc, ds);
                else run_tiny<MODE_F32, false>(d, x, dc, ds);
            } else {
                if (sum) run_tiny<MODE_I32_WIDE, true>(d, x, dc, ds);
                else run_tiny<MODE_I32_WIDE, false>(d, x, dc, ds);
            }
        }
        if (lane == 0) {
            aux[k] = x;
            dcnt[k] = dc;
            dsum[k] = ds;
            const int64_t it =
                flag == SET_OK && !direct ? items_of<int32_t>(bb, static_cast<int32_t>(d.n)) : 0;
            cnt[k] = static_cast<int32_t>(it < 0x7FFFFFFF ? it : 0x7FFFFFFF);
            flags[k] = flag;
        }
    }
}

// Block-level exclusive scan of cnt (kScanBlock per block); block totals to bsum.
__global__ void k_b_scan1(const BatchParams *__restrict__ P, const int32_t *cnt, int64_t *start,
                          int64_t *bsum) {
    __shared__ int64_t warp_tot[kScanBlock / 32];
    const int32_t S = P->n_sets;
    const int64_t k = blockIdx.x * (int64_t)kScanBlock + threadIdx.x;
    if (blockIdx.x * (int64_t)kScanBlock >= S) {
        if (threadIdx.x == 0) bsum[blockIdx.x] = 0;
        return;
    }
    int64_t v = k < S ? cnt[k] : 0;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int64_t incl = v;
    for (int o = 1; o < 32; o <<= 1) {
        int64_t t = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) warp_tot[w] = incl;
    __syncthreads();
    if (w == 0) {
        int64_t t = lane < kScanBlock / 32 ? warp_tot[lane] : 0;
        int64_t ti = t;
        for (int o = 1; o < 32; o <<= 1) {
            int64_t u = __shfl_up_sync(0xFFFFFFFFu, ti, o);
            if (lane >= o) ti += u;
        }
        if (lane < kScanBlock / 32) warp_tot[lane] = ti - t;   // exclusive warp offsets
        if (lane == kScanBlock / 32 - 1) bsum[blockIdx.x] = ti;
    }
    __syncthreads();
    if (k < S) start[k] = incl - v + warp_tot[w];
}

// Exclusive scan of the block totals (one block); writes the grand total.
__global__ void k_b_scan2(int64_t *bsum, int32_t nblocks, BatchState *st, int64_t capacity) {
    __shared__ int64_t buf[kScanBlock];
    const int t = threadIdx.x;
    buf[t] = t < nblocks ? bsum[t] : 0;
    __syncthreads();
    for (int o = 1; o < kScanBlock; o <<= 1) {
        int64_t u = t >= o ? buf[t - o] : 0;
        __syncthreads();
        buf[t] += u;
        __syncthreads();
    }
    if (t < nblocks) bsum[t] = buf[t] - (t < nblocks ? bsum[t] : 0);
    if (t == kScanBlock - 1) {
        st->total_items = buf[t];
        if (buf[t] > capacity) {
            st->status |= SET_OVERFLOW;
            st->total_items = 0;
        }
    }
}

__global__ void k_b_emit(const BatchParams *__restrict__ P, const int32_t *cnt, const int64_t *start,
                         const int64_t *bsum, Item *items, const BatchState *st) {
    if (st->status & SET_OVERFLOW) return;
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t k = warp; k < P->n_sets; k += nwarps) {
        const int64_t s0 = start[k] + bsum[k / kScanBlock];
        const int32_t c = cnt[k];
        for (int32_t t = lane; t < c; t += 32) items[s0 + t] = Item{static_cast<int32_t>(k), t};
    }
}

// ---- the per-item pair loop -------------------------------------------------------------

template <int MODE, int R, bool SUM>
__device__ void run_item(const SetDesc &d, const SetAux &x, const Band &b, int32_t local, Rec *slot,
                         unsigned long long &cnt_out, double &sum_out) {
    const int lane = threadIdx.x & 31;
    constexpr int T = 32 * R;
    const int32_t n = static_cast<int32_t>(d.n);
    const int32_t h = (n - 1) / 2;
    const int32_t M = (n - 1) / T + 1;   // n >= 2 here; T is a constant
    const int32_t K = stages_of<int32_t>(b, n);
    const int32_t tile = local % M;
    const int32_t chunk = local / M;
    const int32_t per = chunk_stages<int32_t>(b, n);
    const int32_t k0 = chunk * per;
    const int32_t k1 = min(k0 + per, K);
    const int32_t tile0 = tile * T;
    const RawSet rs{d.x, d.y, d.z, d.r, n, x.cx, x.cy, x.cz, x.ai_off};
    IState<R> s;
    load_i_raw<MODE, R>(s, rs, tile0, lane);
    const uint32_t r2 = MODE == MODE_F32 ? 0u : x.r2e;
    const ulonglong2 *st = reinterpret_cast<const ulonglong2 *>(slot);
    unsigned long long cnt = 0;
    double sum = 0.0;
    for (int32_t k = k0; k < k1; ++k) {
        const int32_t eo0 = k * kJSB;
        __syncwarp();
        stage_load_raw<MODE>(slot, rs, tile0 + eo0, lane);
        __syncwarp();
        const bool full_stage = (MODE != MODE_I32_WIDE) && (eo0 >= T) && (eo0 + kJSB - 1 <= h);
        cnt += full_stage ? stage_run<MODE, 32, R, kJSB, false, SUM>(s, st, eo0, lane, tile0, n, h, r2, sum)
                          : stage_run<MODE, 32, R, kJSB, true, SUM>(s, st, eo0, lane, tile0, n, h, r2, sum);
    }
    for (int o = 16; o > 0; o >>= 1) {
        cnt += __shfl_down_sync(0xFFFFFFFFu, cnt, o);
        if (SUM) sum += __shfl_down_sync(0xFFFFFFFFu, sum, o);
    }
    cnt_out = cnt;
    sum_out = sum;
}

template <int R, bool SUM>
__device__ __forceinline__ void run_item_mode(const SetDesc &d, const SetAux &x, const Band &b, int32_t local,
                                              Rec *slot, unsigned long long &c, double &s) {
    if (x.mode == MODE_I32_FAST) run_item<MODE_I32_FAST, R, SUM>(d, x, b, local, slot, c, s);
    else if (x.mode == MODE_F32) run_item<MODE_F32, R, SUM>(d, x, b, local, slot, c, s);
    else run_item<MODE_I32_WIDE, R, SUM>(d, x, b, local, slot, c, s);
}

// ---- one warp per set (band r = 0): sets of at most kWarpSetMax objects -----------------

// One object in the convention of the warp-per-set paths: centred coordinates and |p'|^2
// (integers below 2^24, exact in FP32) for the fast integer form, the caller's values and
// radius for FP32 spheres, the int32 bits for the wide integer form.
template <int MODE>
__device__ __forceinline__ float4 set_obj(const SetDesc &d, const SetAux &x, int32_t i) {
    if (MODE == MODE_I32_FAST) {
        const int32_t a = static_cast<const int32_t *>(d.x)[i] - x.cx;
        const int32_t b = static_cast<const int32_t *>(d.y)[i] - x.cy;
        const int32_t c = static_cast<const int32_t *>(d.z)[i] - x.cz;
        return make_float4(static_cast<float>(a), static_cast<float>(b), static_cast<float>(c),
                           static_cast<float>(a * a + b * b + c * c));
    } else if (MODE == MODE_F32) {
        return make_float4(static_cast<const float *>(d.x)[i], static_cast<const float *>(d.y)[i],
                           static_cast<const float *>(d.z)[i], d.r[i]);
    } else {
        return make_float4(__int_as_float(static_cast<const int32_t *>(d.x)[i]),
                           __int_as_float(static_cast<const int32_t *>(d.y)[i]),
                           __int_as_float(static_cast<const int32_t *>(d.z)[i]), 0.0f);
    }
}

// An object tested against partners: its value and, for the fast form, the coefficients of
// d^2 - r2 - 1 = n_j - 2 p'_i.p'_j + (n_i - r2 - 1).
struct OwnObj {
    float4 p;
    float ax, ay, az, di;
};

template <int MODE>
__device__ __forceinline__ OwnObj own_obj(float4 p, const SetAux &x) {
    OwnObj o;
    o.p = p;
    o.ax = -2.0f * p.x;
    o.ay = -2.0f * p.y;
    o.az = -2.0f * p.z;
    o.di = MODE == MODE_I32_FAST ? static_cast<float>(static_cast<int32_t>(p.w) - x.ai_off) : 0.0f;
    return o;
}

// One pair test of an own object against partner q (the predicate of the mode, exact for
// integers, in the specified FP32 rounding for spheres); with SUM the interaction term of
// a hit is added to sum.
template <int MODE, bool SUM>
__device__ __forceinline__ uint32_t pair_test(const OwnObj &o, float4 q, const SetAux &x, double &sum) {
    uint32_t hit;
    uint32_t d2i = 0;
    if (MODE == MODE_I32_FAST) {
        const float v = __fadd_rn(__fmaf_rn(o.az, q.z, __fmaf_rn(o.ay, q.y, __fmaf_rn(o.ax, q.x, q.w))), o.di);
        hit = __float_as_uint(v) >> 31;
        if (SUM) {
            const int32_t ex = static_cast<int32_t>(o.p.x) - static_cast<int32_t>(q.x);
            const int32_t ey = static_cast<int32_t>(o.p.y) - static_cast<int32_t>(q.y);
            const int32_t ez = static_cast<int32_t>(o.p.z) - static_cast<int32_t>(q.z);
            d2i = static_cast<uint32_t>(ex * ex + ey * ey + ez * ez);
        }
    } else if (MODE == MODE_F32) {
        hit = sphere_hit(o.p.x, o.p.y, o.p.z, o.p.w, q.x, q.y, q.z, q.w);
    } else {
        d2i = wide_d2(o.p.x, o.p.y, o.p.z, q.x, q.y, q.z);
        hit = d2i <= x.r2e ? 1u : 0u;
    }
    if (SUM && hit) {
        if (MODE == MODE_F32) {
            const float dx = __fsub_rn(o.p.x, q.x), dy = __fsub_rn(o.p.y, q.y), dz = __fsub_rn(o.p.z, q.z);
            sum += term_from_d2f(__fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz)));
        } else {
            sum += term_from_d2f(static_cast<float>(d2i));
        }
    }
    return hit;
}

// Sets of at most 32 objects: lane l holds object l and, at step s, gets its partner
// (l + s) mod n from another lane by shuffles: the proposed algorithm with one object per
// lane, exactly evals(i) tests per object and no staging or masks.
template <int MODE, bool SUM>
__device__ void run_tiny(const SetDesc &d, const SetAux &x, unsigned long long &cnt_out, double &sum_out) {
    const int lane = threadIdx.x & 31;
    const int32_t n = static_cast<int32_t>(d.n);
    const int32_t h = (n - 1) / 2;
    const bool even = (n & 1) == 0;
    const bool valid = lane < n;
    const OwnObj o = own_obj<MODE>(set_obj<MODE>(d, x, valid ? lane : 0), x);
    const int32_t steps = h + (even ? 1 : 0);
    uint32_t cnt = 0;
    double sum = 0.0;
    int32_t src = lane + 1 < n ? lane + 1 : lane + 1 - n;
    for (int32_t s = 1; s <= steps; ++s) {
        float4 q;
        q.x = __shfl_sync(0xFFFFFFFFu, o.p.x, src);
        q.y = __shfl_sync(0xFFFFFFFFu, o.p.y, src);
        q.z = __shfl_sync(0xFFFFFFFFu, o.p.z, src);
        q.w = __shfl_sync(0xFFFFFFFFu, o.p.w, src);
        // the even-N extra step (s = n/2) belongs to the objects i < n/2
        if (valid && (s <= h || lane < n / 2)) cnt += pair_test<MODE, SUM>(o, q, x, sum);
        src = src + 1 < n ? src + 1 : 0;
    }
    unsigned long long c64 = cnt;
    for (int o2 = 16; o2 > 0; o2 >>= 1) {
        c64 += __shfl_down_sync(0xFFFFFFFFu, c64, o2);
        if (SUM) sum += __shfl_down_sync(0xFFFFFFFFu, sum, o2);
    }
    cnt_out = c64;
    sum_out = sum;
}

// Sets of 33 .. kWarpSetMax objects: the whole set in the warp's shared-memory buffer, lane
// l owning objects l, l + 32, ..; at step s every owned object i tests (i + s) mod n read
// from the buffer (consecutive lanes read consecutive objects). The proposed algorithm's
// order with exactly evals(i) tests per object: no tiles, so no masked candidate pairs.
template <int MODE, bool SUM>
__device__ void run_warpset(const SetDesc &d, const SetAux &x, float4 *buf, unsigned long long &cnt_out,
                            double &sum_out) {
    const int lane = threadIdx.x & 31;
    const int32_t n = static_cast<int32_t>(d.n);
    const int32_t h = (n - 1) / 2;
    const int32_t half = (n & 1) == 0 ? n / 2 : 0;   // objects below it take the extra step
    __syncwarp();   // the previous item's reads of the buffer are done
    for (int32_t i = lane; i < n; i += 32) buf[i] = set_obj<MODE>(d, x, i);
    __syncwarp();
    const int mo = (n + 31) >> 5;   // warp-uniform
    uint32_t cnt = 0;
    double sum = 0.0;
    const int32_t steps = h + (half > 0 ? 1 : 0);
    // one owned object at a time (few registers): its evals(i) partners in step order
    for (int m = 0; m < mo; ++m) {
        const int32_t i = lane + 32 * m;
        const OwnObj o = own_obj<MODE>(buf[i < n ? i : 0], x);
        const int32_t ev = i < n ? (i < half ? steps : h) : 0;
        int32_t j = i + 1 < n ? i + 1 : i + 1 - n;
        for (int32_t s = 1; s <= steps; ++s) {
            if (s <= ev) cnt += pair_test<MODE, SUM>(o, buf[j], x, sum);
            j = j + 1 < n ? j + 1 : 0;
        }
    }
    unsigned long long c64 = cnt;
    for (int o2 = 16; o2 > 0; o2 >>= 1) {
        c64 += __shfl_down_sync(0xFFFFFFFFu, c64, o2);
        if (SUM) sum += __shfl_down_sync(0xFFFFFFFFu, sum, o2);
    }
    cnt_out = c64;
    sum_out = sum;
}

template <bool SUM>
__device__ __forceinline__ void run_item_r(const SetDesc &d, const SetAux &x, const Band &b, int32_t local,
                                           Rec *slot, unsigned long long &c, double &s) {
    switch (b.r) {
        case 0:
            if (d.n <= 32) {
                if (x.mode == MODE_I32_FAST) run_tiny<MODE_I32_FAST, SUM>(d, x, c, s);
                else if (x.mode == MODE_F32) run_tiny<MODE_F32, SUM>(d, x, c, s);
                else run_tiny<MODE_I32_WIDE, SUM>(d, x, c, s);
            } else {   // the warp's buffer holds kWarpSetMax objects (the band table checks n_max)
                float4 *buf = reinterpret_cast<float4 *>(slot);
                if (x.mode == MODE_I32_FAST) run_warpset<MODE_I32_FAST, SUM>(d, x, buf, c, s);
                else if (x.mode == MODE_F32) run_warpset<MODE_F32, SUM>(d, x, buf, c, s);
                else run_warpset<MODE_I32_WIDE, SUM>(d, x, buf, c, s);
            }
            break;
        case 1: run_item_mode<1, SUM>(d, x, b, local, slot, c, s); break;
        case 2: run_item_mode<2, SUM>(d, x, b, local, slot, c, s); break;
        default: run_item_mode<4, SUM>(d, x, b, local, slot, c, s); break;
    }
}

// MINB: resident CTAs per SM the register allocation must allow (the items are small, so
// more warps in flight hide more of their load latency).
template <int MINB>
__global__ void __launch_bounds__(kMainWarps * 32, MINB) k_b_main(const BatchParams *__restrict__ P,
                                                           const SetDesc *sets, const SetAux *aux,
                                                           const BandTable *bt, const Item *items,
                                                           BatchState *st, unsigned long long *pcnt,
                                                           double *psum) {
    // per warp: a j-stage of records (tiled items) or a whole set (one warp per set)
    static_assert(kWarpSetMax * sizeof(float4) >= (kJSB / 2) * sizeof(Rec), "warp buffer");
    __shared__ float4 wbuf[kMainWarps][kWarpSetMax];
    const int lane = threadIdx.x & 31;
    Rec *slot = reinterpret_cast<Rec *>(wbuf[threadIdx.x >> 5]);
    const int64_t total = st->total_items;
    const bool want_sum = P->want_sum != 0;
    unsigned long long *cursor = reinterpret_cast<unsigned long long *>(&st->cursor);
    // the next item's index is taken before the current item is worked on, so the
    // atomic's round trip overlaps the work
    int64_t next = 0;
    if (lane == 0) next = static_cast<int64_t>(atomicAdd(cursor, 1ull));
    for (;;) {
        const int64_t it = __shfl_sync(0xFFFFFFFFu, next, 0);
        if (it >= total) break;
        if (lane == 0) next = static_cast<int64_t>(atomicAdd(cursor, 1ull));
        const Item item = items[it];
        const SetDesc d = sets[item.set];
        const SetAux x = aux[item.set];
        const Band b = band_of(*bt, d.n);
        unsigned long long c = 0;
        double s = 0.0;
        if (want_sum) run_item_r<true>(d, x, b, item.local, slot, c, s);
        else run_item_r<false>(d, x, b, item.local, slot, c, s);
        if (lane == 0) {
            pcnt[it] = c;
            if (want_sum) psum[it] = s;
        }
    }
}

__global__ void k_b_finish(const BatchParams *__restrict__ P, const int32_t *cnt, const int64_t *start,
                           const int64_t *bsum, const uint32_t *flags, const BatchState *st,
                           const unsigned long long *pcnt, const double *psum,
                           const unsigned long long *dcnt, const double *dsum) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const bool overflow = (st->status & SET_OVERFLOW) != 0;
    const bool want_sum = P->want_sum != 0;
    for (int64_t k = warp; k < P->n_sets; k += nwarps) {
        const int64_t s0 = start[k] + bsum[k / kScanBlock];
        const int32_t c = cnt[k];
        unsigned long long tc = 0;
        double ts = 0.0;
        if (!overflow) {
            for (int32_t t = lane; t < c; t += 32) {
                tc += pcnt[s0 + t];
                if (want_sum) ts += psum[s0 + t];
            }
            for (int o = 16; o > 0; o >>= 1) {
                tc += __shfl_down_sync(0xFFFFFFFFu, tc, o);
                if (want_sum) ts += __shfl_down_sync(0xFFFFFFFFu, ts, o);
            }
        }
        if (lane == 0) {
            tc += dcnt[k];   // sets counted by the prepare kernel (0 for the others)
            if (want_sum) ts += dsum[k];
            const bool bad = overflow || flags[k] != SET_OK;
            P->d_counts[k] = bad ? CC_COUNT_INVALID : tc;
            if (want_sum && P->d_sums) P->d_sums[k] = bad ? __int_as_float(0x7fc00000) : static_cast<float>(ts);
        }
    }
}

// ---------------------------------------------------------------------------------------
// host side: plan, band table, graph
// ---------------------------------------------------------------------------------------

static BandTable default_bands() {
    BandTable t{};
    t.count = 5;
    t.band[0] = Band{32, 0, 0};
    t.band[1] = Band{kWarpSetMax, 0, 0};
    t.band[2] = Band{512, 2, 8};
    t.band[3] = Band{8192, 4, 8};
    t.band[4] = Band{INT64_MAX, 4, 64};
    return t;
}

// Minimal parser for {"bands": [{"n_max": N, "r": R, "sc": S}, ...]} (n_max -1 = no limit;
// r objects per lane in {1, 2, 4}, or 0 for one warp per set, sets of at most kWarpSetMax
// objects (not the last band); sc stages of 64 objects per work item, 0 = all).
static bool parse_bands(const char *json, BandTable &out, std::string &err) {
    BandTable t{};
    const char *p = strstr(json, "\"bands\"");
    if (!p) { err = "missing \"bands\""; return false; }
    p = strchr(p, '[');
    if (!p) { err = "missing band list"; return false; }
    ++p;
    while (true) {
        const char *ob = strchr(p, '{');
        const char *end = strchr(p, ']');
        if (!ob || (end && end < ob)) break;
        const char *cb = strchr(ob, '}');
        if (!cb) { err = "unterminated band"; return false; }
        std::string obj(ob, cb - ob);
        auto field = [&](const char *name, long long &v) {
            size_t q = obj.find(std::string("\"") + name + "\"");
            if (q == std::string::npos) return false;
            q = obj.find(':', q);
            if (q == std::string::npos) return false;
            v = strtoll(obj.c_str() + q + 1, nullptr, 10);
            return true;
        };
        long long nmax = 0, r = 0, sc = 0;
        if (!field("n_max", nmax) || !field("r", r) || !field("sc", sc)) { err = "band needs n_max, r, sc"; return false; }
        if (t.count >= kMaxBands) { err = "too many bands"; return false; }
        if (!(r == 0 || r == 1 || r == 2 || r == 4) || sc < 0) {
            err = "r must be 0, 1, 2 or 4 and sc >= 0";
            return false;
        }
        if (r == 0 && (nmax < 0 || nmax > kWarpSetMax)) {
            err = "r = 0 (one warp per set) needs 0 <= n_max <= " + std::to_string(kWarpSetMax);
            return false;
        }
        t.band[t.count++] = Band{nmax < 0 ? INT64_MAX : nmax, static_cast<int32_t>(r), static_cast<int32_t>(sc)};
        p = cb + 1;
    }
    if (t.count == 0) { err = "no bands"; return false; }
    if (t.band[t.count - 1].r == 0) { err = "the last band (all larger sets) cannot have r = 0"; return false; }
    t.band[t.count - 1].n_max = INT64_MAX;
    out = t;
    return true;
}

// Largest items-per-object ratio a table can produce for sets of up to max_n objects.
static double items_per_object(const BandTable &t, int64_t max_n) {
    double worst = 0.0;
    int64_t lo = 2;
    for (int b = 0; b < t.count && lo <= max_n; ++b) {
        const int64_t hi = std::min(t.band[b].n_max, max_n);
        // sample the band densely near its ends and geometrically inside
        for (int64_t n = lo; n <= hi; n = (n < lo + 4096 ? n + 1 : n + n / 64 + 1))
            worst = std::max(worst, static_cast<double>(items_of<int64_t>(t.band[b], n)) / n);
        worst = std::max(worst, static_cast<double>(items_of<int64_t>(t.band[b], hi)) / hi);
        lo = hi + 1;
    }
    return worst;
}

}  // namespace cc

using namespace cc;

struct cc_plan {
    BandTable bands;
    int32_t max_sets = 0;
    int64_t max_points = 0;
    int64_t item_cap = 0;
    int32_t scan_blocks = 0;
    // device buffers
    BatchParams *d_params = nullptr;
    BandTable *d_bands = nullptr;
    SetDesc *d_sets = nullptr;
    SetAux *d_aux = nullptr;
    int32_t *d_cnt = nullptr;
    uint32_t *d_flags = nullptr;
    unsigned long long *d_dcnt = nullptr;   // per set: count made by the prepare kernel
    double *d_dsum = nullptr;
    int64_t *d_start = nullptr;
    int64_t *d_bsum = nullptr;
    Item *d_items = nullptr;
    unsigned long long *d_pcnt = nullptr;
    double *d_psum = nullptr;
    BatchState *d_state = nullptr;
    // graph
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t exec = nullptr;
    int main_grid = 0;
    const void *main_fn = nullptr;   // k_b_main instance (resident CTAs per SM)
    std::mutex mu;
};

// k_b_main instance: registers capped for 3 resident CTAs per SM. Measured on config 4
// (100k small sets) with 1, 2, 3 and 4 CTAs per SM: 0.57, 0.40, 0.38 and 0.38 ms (4 spills
// heavily in the wide bands).
static const void *main_kernel() { return reinterpret_cast<const void *>(k_b_main<3>); }

static cc_status plan_enqueue(cc_plan *P, cudaStream_t s) {
    const int sms = sm_count();
    k_b_prepare<<<sms * 8, 256, 0, s>>>(P->d_params, P->d_sets, P->d_aux, P->d_bands, P->d_cnt, P->d_flags,
                                        P->d_state, P->d_dcnt, P->d_dsum);
    k_b_scan1<<<P->scan_blocks, kScanBlock, 0, s>>>(P->d_params, P->d_cnt, P->d_start, P->d_bsum);
    k_b_scan2<<<1, kScanBlock, 0, s>>>(P->d_bsum, P->scan_blocks, P->d_state, P->item_cap);
    k_b_emit<<<sms * 8, 256, 0, s>>>(P->d_params, P->d_cnt, P->d_start, P->d_bsum, P->d_items, P->d_state);
    {
        void *args[] = {&P->d_params, &P->d_sets, &P->d_aux, &P->d_bands, &P->d_items,
                        &P->d_state, &P->d_pcnt, &P->d_psum};
        CC_CUDA(cudaLaunchKernel(P->main_fn, dim3(P->main_grid), dim3(kMainWarps * 32), args, 0, s));
    }
    k_b_finish<<<sms * 8, 256, 0, s>>>(P->d_params, P->d_cnt, P->d_start, P->d_bsum, P->d_flags, P->d_state,
                                       P->d_pcnt, P->d_psum, P->d_dcnt, P->d_dsum);
    CC_CUDA(cudaGetLastError());
    return CC_OK;
}

static cc_status plan_capture(cc_plan *P) {
    if (P->exec) return CC_OK;
    cudaGraph_t g = nullptr;
    CC_CUDA(cudaStreamBeginCapture(P->cap_stream, cudaStreamCaptureModeThreadLocal));
    cc_status st = plan_enqueue(P, P->cap_stream);
    cudaError_t e = cudaStreamEndCapture(P->cap_stream, &g);
    if (st != CC_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&P->exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
    return CC_OK;
}

namespace cc {

// Used by the server: launches the plan's graph for sets already described in d_sets.
cc_status plan_launch_sets(cc_plan *P, int32_t n_sets, int32_t want_sum, unsigned long long *d_counts,
                           float *d_sums, cudaStream_t s) {
    BatchParams bp{};
    bp.offsets = nullptr;
    bp.n_sets = n_sets;
    bp.want_sum = want_sum;
    bp.d_counts = d_counts;
    bp.d_sums = d_sums;
    std::lock_guard<std::mutex> lk(P->mu);
    cc_status st = plan_capture(P);
    if (st != CC_OK) return st;
    CC_CUDA(cudaMemcpyAsync(P->d_params, &bp, sizeof(bp), cudaMemcpyHostToDevice, s));
    CC_CUDA(cudaGraphLaunch(P->exec, s));
    return CC_OK;
}

void *plan_sets_buffer_v(cc_plan *P) { return P->d_sets; }
size_t plan_set_desc_bytes() { return sizeof(SetDesc); }

}  // namespace cc

extern "C" {

cc_status cc_plan_create(cc_plan **plan, const char *tune_table_json, int32_t max_sets, int64_t max_points) {
    if (!plan) return fail(CC_ERR_INVALID_ARG, "plan is NULL");
    *plan = nullptr;
    if (max_sets <= 0 || max_sets > kScanBlock * kScanBlock)
        return fail(CC_ERR_INVALID_ARG, "max_sets must be in 1..1048576");
    if (max_points < 0) return fail(CC_ERR_INVALID_ARG, "max_points < 0");
    cc_plan *P = new cc_plan();
    P->bands = default_bands();
    if (tune_table_json) {
        std::string err;
        if (!parse_bands(tune_table_json, P->bands, err)) {
            delete P;
            return fail(CC_ERR_INVALID_ARG, "tune table: " + err);
        }
    }
    P->max_sets = max_sets;
    P->max_points = max_points;
    const double ipo = items_per_object(P->bands, std::max<int64_t>(max_points, 2));
    P->item_cap = static_cast<int64_t>(2 * static_cast<int64_t>(max_sets) + std::ceil(ipo * max_points) + 1024);
    P->scan_blocks = (max_sets + kScanBlock - 1) / kScanBlock;
    auto alloc = [&](void **p, size_t b) { return cudaMalloc(p, std::max<size_t>(b, 16)); };
    cudaError_t e = cudaSuccess;
    e = e ? e : alloc(reinterpret_cast<void **>(&P->d_params), sizeof(BatchParams));
    e = e ? e : alloc(reinterpret_cast<void **>(&P->d_bands), sizeof(BandTable));
    e = e ? e : alloc(reinterpret_cast<void **>(&P->d_sets), sizeof(SetDesc) * max_sets);
    e = e ? e : alloc(reinterpret_cast<void **>(&P->d_aux), sizeof(SetAux) * max_sets);
    e = e ? e : alloc(reinterpret_cast<void **>(&P->d_cnt), sizeof(int32_t) * max_sets);
    e = e ? e : alloc(reinterpret_cast<void **>(&P->d_flags), sizeof(uint32_t) * max_sets);
    e = e ? e : alloc(reinterpret_cast<void **>(&P->d_dcnt), sizeof(unsigned long long) * max_sets);
    e = e ? e : alloc(reinterpret_cast<void **>(&P->d_dsum), sizeof(double) * max_sets);
    e = e ? e : alloc(reinterpret_cast<void **>(&P->d_start), sizeof(int64_t) * max_sets);
    e = e ? e : alloc(reinterpret_cast<void **>(&P->d_bsum), sizeof(int64_t) * P->scan_blocks);
    e = e ? e : alloc(reinterpret_cast<void **>(&P->d_items), sizeof(Item) * P->item_cap);
    e = e ? e : alloc(reinterpret_cast<void **>(&P->d_pcnt), sizeof(unsigned long long) * P->item_cap);
    e = e ? e : alloc(reinterpret_cast<void **>(&P->d_psum), sizeof(double) * P->item_cap);
    e = e ? e : alloc(reinterpret_cast<void **>(&P->d_state), sizeof(BatchState));
    e = e ? e : cudaMemcpy(P->d_bands, &P->bands, sizeof(BandTable), cudaMemcpyHostToDevice);
    e = e ? e : cudaMemset(P->d_state, 0, sizeof(BatchState));
    e = e ? e : cudaStreamCreateWithFlags(&P->cap_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        cc_plan_destroy(P);
        return fail(CC_ERR_NOMEM, std::string("plan allocation: ") + cudaGetErrorString(e));
    }
    int bps = 0;
    P->main_fn = main_kernel();
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, P->main_fn, kMainWarps * 32, 0);
    P->main_grid = sm_count() * std::max(bps, 1);
    *plan = P;
    return CC_OK;
}

void cc_plan_destroy(cc_plan *P) {
    if (!P) return;
    if (P->exec) cudaGraphExecDestroy(P->exec);
    if (P->cap_stream) cudaStreamDestroy(P->cap_stream);
    void *bufs[] = {P->d_params, P->d_bands, P->d_sets, P->d_aux, P->d_cnt, P->d_flags, P->d_dcnt,
                    P->d_dsum, P->d_start, P->d_bsum, P->d_items, P->d_pcnt, P->d_psum, P->d_state};
    for (void *b : bufs)
        if (b) cudaFree(b);
    delete P;
}

cc_status cc_count_pairs_batched(cc_plan *P, const cc_points *p, const int64_t *d_offsets, int32_t n_sets,
                                 uint32_t r2, unsigned long long *d_counts, float *d_sums, void *stream) {
    if (!P || !p || !d_offsets || !d_counts) return fail(CC_ERR_INVALID_ARG, "NULL argument");
    if (n_sets < 0 || n_sets > P->max_sets) return fail(CC_ERR_INVALID_ARG, "n_sets outside 0..max_sets");
    if (p->dtype != CC_I32 && p->dtype != CC_F32) return fail(CC_ERR_INVALID_ARG, "unknown dtype");
    if (p->dtype == CC_F32 && !p->r) return fail(CC_ERR_INVALID_ARG, "radius pointer is NULL");
    if ((reinterpret_cast<uintptr_t>(d_offsets) & 7) || (reinterpret_cast<uintptr_t>(d_counts) & 7))
        return fail(CC_ERR_INVALID_ARG, "offsets and counts must be 8-byte aligned");
    if (n_sets == 0) return CC_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    BatchParams bp{};
    bp.pts = *p;
    bp.offsets = d_offsets;
    bp.n_sets = n_sets;
    bp.r2 = r2;
    bp.want_sum = d_sums != nullptr;
    bp.d_counts = d_counts;
    bp.d_sums = d_sums;
    std::lock_guard<std::mutex> lk(P->mu);
    cc_status st = plan_capture(P);
    if (st != CC_OK) return st;
    // pageable source: the copy is staged before cudaMemcpyAsync returns
    CC_CUDA(cudaMemcpyAsync(P->d_params, &bp, sizeof(bp), cudaMemcpyHostToDevice, s));
    CC_CUDA(cudaGraphLaunch(P->exec, s));
    return CC_OK;
}

cc_status cc_plan_last_items(cc_plan *P, int64_t *items) {
    if (!P || !items) return fail(CC_ERR_INVALID_ARG, "NULL argument");
    BatchState st{};
    CC_CUDA(cudaDeviceSynchronize());
    CC_CUDA(cudaMemcpy(&st, P->d_state, sizeof(st), cudaMemcpyDeviceToHost));
    *items = st.total_items;
    if (st.status & SET_OVERFLOW) return fail(CC_ERR_NOMEM, "work-queue capacity exceeded");
    return CC_OK;
}

}  // extern "C"

// Device-side pieces of the pair test shared by the single-set and the batched kernels:
// the staged record layout, the per-object register state and one stage of the cyclic
// schedule (Section 4, proposed algorithm) for one warp's objects.
#pragma once

#include "cc_internal.cuh"

// FP32 sphere predicate on packed FP32x2 registers (two pairs per instruction); 0 selects
// the scalar form.
#ifndef CC_F32_PACKED
#define CC_F32_PACKED 1
#endif

namespace cc {

struct __align__(16) Rec {
    float x[2], y[2], z[2], w[2];
};
static_assert(sizeof(Rec) == 32, "record size");

// Register state of one consumer thread's R objects: packed, duplicated operands.
//   fast int : a = -2x, b = -2y, c = -2z, d = n_i - r2e - 1   (v = n_j - 2 p_i.p_j + d)
//   f32      : a = x, b = y, c = z, d = r
//   wide int : a, b, c = raw int32 bits of x, y, z
template <int R>
struct IState {
    f2 a[R], b[R], c[R], d[R];
};

__device__ __forceinline__ uint32_t sign_lo(f2 v) { return static_cast<uint32_t>(v) >> 31; }
__device__ __forceinline__ uint32_t sign_hi(f2 v) { return static_cast<uint32_t>(v >> 32) >> 31; }

// Evaluations of object i (0 for i >= n): (n-1)/2, plus one for i < n/2 when n is even.
// h < 0 selects the straightforward schedule used for comparison (Section 5): object i
// evaluates every later object, n - 1 - i of them.
__device__ __forceinline__ uint32_t evals_of(int64_t i, int64_t n, int32_t h) {
    if (i >= n) return 0u;
    if (h < 0) return static_cast<uint32_t>(n - 1 - i);
    return static_cast<uint32_t>(h) + (((n & 1) == 0 && i < n / 2) ? 1u : 0u);
}

// ---- per-pair predicates ----------------------------------------------------------------

// Fast integer form for the pairs (i, j0), (i, j1): the sign bits of v mark the hits.
__device__ __forceinline__ f2 fast_v(f2 a, f2 b, f2 c, f2 d, ulonglong2 p0, ulonglong2 p1) {
    f2 t = f2_fma(a, p0.x, p1.y);
    t = f2_fma(b, p0.y, t);
    t = f2_fma(c, p1.x, t);
    return f2_add(t, d);
}

// FP32 sphere predicate for two pairs, in the specified order and rounding, written with
// scalar __fadd_rn/__fsub_rn/__fmul_rn intrinsics: these are never contracted into a fused
// multiply-add (packed multiply/add pairs were observed to be contracted by the code
// generator, which would change the rounding), and reading the halves of the staged
// register pairs directly avoids any packing/unpacking moves.
__device__ __forceinline__ uint32_t sphere_hit(float xi, float yi, float zi, float ri, float xj, float yj,
                                               float zj, float rj) {
    const float dx = __fsub_rn(xi, xj);
    const float dy = __fsub_rn(yi, yj);
    const float dz = __fsub_rn(zi, zj);
    const float d2 = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
    const float s = __fadd_rn(ri, rj);
    return d2 <= __fmul_rn(s, s) ? 1u : 0u;
}

// The same predicate for two pairs at once on packed FP32x2 registers. The squares are
// fma.rn(d, d, +0): exactly RN(d*d) (the product is never negative, and +0 + RN(p) =
// RN(p)), but, unlike a multiply, an FMA is never contracted into the following add, so
// every operation keeps the specified rounding. (An FMA with a +0 addend cannot be
// rewritten as a multiply either: for d = -0 the sum is +0.)
__device__ __forceinline__ f2 f2_sq_rn(f2 v) {
    f2 d;
    asm("fma.rn.f32x2 %0, %1, %1, %2;" : "=l"(d) : "l"(v), "l"(0ull));
    return d;
}

__device__ __forceinline__ void sphere_hit2(f2 xi, f2 yi, f2 zi, f2 ri, f2 xj, f2 yj, f2 zj, f2 rj, uint32_t &h0,
                                            uint32_t &h1) {
    const f2 d2 = f2_add(f2_add(f2_sq_rn(f2_sub(xi, xj)), f2_sq_rn(f2_sub(yi, yj))), f2_sq_rn(f2_sub(zi, zj)));
    const f2 s = f2_add(ri, rj);
    const f2 s2 = f2_mul(s, s);
    h0 = f2_lo(d2) <= f2_lo(s2) ? 1u : 0u;
    h1 = f2_hi(d2) <= f2_hi(s2) ? 1u : 0u;
}

__device__ __forceinline__ uint32_t wide_d2(float xi, float yi, float zi, float xj, float yj, float zj) {
    int32_t dx = __float_as_int(xi) - __float_as_int(xj);
    int32_t dy = __float_as_int(yi) - __float_as_int(yj);
    int32_t dz = __float_as_int(zi) - __float_as_int(zj);
    return static_cast<uint32_t>(dx * dx) + static_cast<uint32_t>(dy * dy) + static_cast<uint32_t>(dz * dz);
}

__device__ __forceinline__ double term_from_d2f(float d2) {
    float d = __fsqrt_rn(d2);
    return static_cast<double>(__fdiv_rn(1.0f, fmaxf(d, 1e-6f)));
}

// Interaction terms of object slot r of this thread against the two objects of one
// staged record (extended offsets eo, eo+1 from the tile start). Only called for record
// groups that produced a hit (rare), so it is kept out of line.
template <int MODE, int NT>
__device__ __noinline__ double pair_terms(f2 a, f2 b, f2 c, f2 d, ulonglong2 p0, ulonglong2 p1,
                                          int32_t eo, int32_t ioff, uint32_t evals, uint32_t r2) {
    double sum = 0.0;
    for (int l = 0; l < 2; ++l) {
        const uint32_t so = static_cast<uint32_t>(eo + l - ioff - 1);
        if (!(so < evals)) continue;
        const float xj = l ? f2_hi(p0.x) : f2_lo(p0.x);
        const float yj = l ? f2_hi(p0.y) : f2_lo(p0.y);
        const float zj = l ? f2_hi(p1.x) : f2_lo(p1.x);
        const float wj = l ? f2_hi(p1.y) : f2_lo(p1.y);
        if (MODE == MODE_F32) {
            const float dx = __fsub_rn(f2_lo(a), xj);
            const float dy = __fsub_rn(f2_lo(b), yj);
            const float dz = __fsub_rn(f2_lo(c), zj);
            const float d2 = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
            const float sr = __fadd_rn(f2_lo(d), wj);
            if (d2 <= __fmul_rn(sr, sr)) sum += term_from_d2f(d2);
        } else if (MODE == MODE_I32_FAST) {
            // exact integer d2 from the centred coordinates (a = -2x etc.)
            const int32_t dx = static_cast<int32_t>(-0.5f * f2_lo(a)) - static_cast<int32_t>(xj);
            const int32_t dy = static_cast<int32_t>(-0.5f * f2_lo(b)) - static_cast<int32_t>(yj);
            const int32_t dz = static_cast<int32_t>(-0.5f * f2_lo(c)) - static_cast<int32_t>(zj);
            const uint32_t d2 = static_cast<uint32_t>(dx * dx + dy * dy + dz * dz);
            if (d2 <= r2) sum += term_from_d2f(static_cast<float>(d2));
        } else {
            const uint32_t d2 = wide_d2(f2_lo(a), f2_lo(b), f2_lo(c), xj, yj, zj);
            if (d2 <= r2) sum += term_from_d2f(static_cast<float>(d2));
        }
    }
    return sum;
}

// ---- staging straight from the caller's SoA arrays (batched kernel) ----------------------

// A set as the caller holds it, with the integer centre and offset of the fast form.
struct RawSet {
    const void *x, *y, *z;
    const float *r;
    int32_t n;
    int32_t cx, cy, cz;   // integer centre subtracted before the FP32 conversion
    int32_t ai_off;       // r2e + 1 (fast integer form)
};

// Loads the R objects of this lane for the warp tile starting at tile0 (objects
// tile0 + lane + 32 r) in the register form of MODE. Objects past n get a state that
// never hits (fast form, spheres) or no evaluations (wide form: evals_of is 0).
template <int MODE, int R>
__device__ __forceinline__ void load_i_raw(IState<R> &s, const RawSet &d, int32_t tile0, int lane) {
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int32_t i = tile0 + lane + 32 * r;
        const bool valid = i < d.n;
        const int32_t ii = valid ? i : 0;
        if (MODE == MODE_I32_FAST) {
            const int32_t xi = static_cast<const int32_t *>(d.x)[ii] - d.cx;
            const int32_t yi = static_cast<const int32_t *>(d.y)[ii] - d.cy;
            const int32_t zi = static_cast<const int32_t *>(d.z)[ii] - d.cz;
            s.a[r] = f2_dup(-2.0f * static_cast<float>(xi));
            s.b[r] = f2_dup(-2.0f * static_cast<float>(yi));
            s.c[r] = f2_dup(-2.0f * static_cast<float>(zi));
            s.d[r] = f2_dup(valid ? static_cast<float>(xi * xi + yi * yi + zi * zi - d.ai_off)
                                  : __int_as_float(0x7f800000));   // +inf: never hits
        } else if (MODE == MODE_F32) {
            const float xi = static_cast<const float *>(d.x)[ii];
            s.a[r] = f2_dup(valid ? xi : __int_as_float(0x7fc00000));   // NaN: never hits
            s.b[r] = f2_dup(static_cast<const float *>(d.y)[ii]);
            s.c[r] = f2_dup(static_cast<const float *>(d.z)[ii]);
            s.d[r] = f2_dup(d.r[ii]);
        } else {
            s.a[r] = f2_dup(__int_as_float(static_cast<const int32_t *>(d.x)[ii]));
            s.b[r] = f2_dup(__int_as_float(static_cast<const int32_t *>(d.y)[ii]));
            s.c[r] = f2_dup(__int_as_float(static_cast<const int32_t *>(d.z)[ii]));
            s.d[r] = 0;
        }
    }
}

// Stages the extended objects [e0, e0 + 64) of the set (indices mod n) into a warp's
// slot as 32 pair-interleaved records: lane l writes record l (objects e0+2l, e0+2l+1).
template <int MODE>
__device__ __forceinline__ void stage_load_raw(Rec *slot, const RawSet &d, int32_t e0, int lane) {
    Rec rec;
#pragma unroll
    for (int l = 0; l < 2; ++l) {
        const int32_t e = e0 + 2 * lane + l;
        const int32_t p = e < d.n ? e : e % d.n;
        if (MODE == MODE_I32_FAST) {
            const int32_t xi = static_cast<const int32_t *>(d.x)[p] - d.cx;
            const int32_t yi = static_cast<const int32_t *>(d.y)[p] - d.cy;
            const int32_t zi = static_cast<const int32_t *>(d.z)[p] - d.cz;
            rec.x[l] = static_cast<float>(xi);
            rec.y[l] = static_cast<float>(yi);
            rec.z[l] = static_cast<float>(zi);
            rec.w[l] = static_cast<float>(xi * xi + yi * yi + zi * zi);
        } else if (MODE == MODE_F32) {
            rec.x[l] = static_cast<const float *>(d.x)[p];
            rec.y[l] = static_cast<const float *>(d.y)[p];
            rec.z[l] = static_cast<const float *>(d.z)[p];
            rec.w[l] = d.r[p];
        } else {
            rec.x[l] = __int_as_float(static_cast<const int32_t *>(d.x)[p]);
            rec.y[l] = __int_as_float(static_cast<const int32_t *>(d.y)[p]);
            rec.z[l] = __int_as_float(static_cast<const int32_t *>(d.z)[p]);
            rec.w[l] = 0.0f;
        }
    }
    slot[lane] = rec;
}

// One stage for one consumer thread: JS staged objects against the thread's R objects.
// MASKED applies the cyclic schedule's validity per pair: s = e - i must be in 1..evals(i).
// With SUM, record pairs that produced a hit are re-walked for their interaction terms.
// Each object slot r has its own counter so that the accumulations do not form one long
// dependency chain.
template <int MODE, int NT, int R, int JS, bool MASKED, bool SUM>
__device__ __forceinline__ uint32_t stage_run(const IState<R> &s, const ulonglong2 *__restrict__ st,
                                              int32_t eo0, int tid, int64_t tile0, int64_t n,
                                              int32_t h, uint32_t r2, double &sum) {
    uint32_t cr[R];
    uint32_t base[R], ev[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        cr[r] = 0;
        if (MASKED || SUM) {
            const int32_t ioff = tid + r * NT;
            ev[r] = evals_of(tile0 + ioff, n, h);
            base[r] = static_cast<uint32_t>(eo0 - ioff - 1);   // s - 1 of the stage's first object
        }
    }
    if (MODE == MODE_I32_FAST && !MASKED && !SUM) {
        // Unmasked fast form, i-outer over blocks of QB staged record pairs: each
        // object's coefficients are the operand repeated by consecutive instructions.
        constexpr int QB = 4;
#pragma unroll 1
        for (int q0 = 0; q0 < JS / 2; q0 += QB) {
            f2 X[QB], Y[QB], Z[QB], B[QB];
#pragma unroll
            for (int q = 0; q < QB; ++q) {
                const ulonglong2 p0 = st[2 * (q0 + q)];
                const ulonglong2 p1 = st[2 * (q0 + q) + 1];
                X[q] = p0.x;
                Y[q] = p0.y;
                Z[q] = p1.x;
                B[q] = p1.y;
            }
#pragma unroll
            for (int r = 0; r < R; ++r) {
                f2 t[QB];
#pragma unroll
                for (int q = 0; q < QB; ++q) t[q] = f2_fma(s.a[r], X[q], B[q]);
#pragma unroll
                for (int q = 0; q < QB; ++q) t[q] = f2_fma(s.b[r], Y[q], t[q]);
#pragma unroll
                for (int q = 0; q < QB; ++q) t[q] = f2_fma(s.c[r], Z[q], t[q]);
#pragma unroll
                for (int q = 0; q < QB; ++q) t[q] = f2_add(t[q], s.d[r]);
#pragma unroll
                for (int q = 0; q < QB; ++q) {
                    cr[r] += sign_lo(t[q]);
                    cr[r] += sign_hi(t[q]);
                }
            }
        }
    } else if (MODE == MODE_F32 && CC_F32_PACKED && !MASKED && !SUM) {
        // Unmasked FP32 spheres, object-outer over blocks of QB staged record pairs (the
        // object's coordinates are the operand repeated by consecutive instructions).
        constexpr int QB = 4;
#pragma unroll 1
        for (int q0 = 0; q0 < JS / 2; q0 += QB) {
            f2 X[QB], Y[QB], Z[QB], W[QB];
#pragma unroll
            for (int q = 0; q < QB; ++q) {
                const ulonglong2 p0 = st[2 * (q0 + q)];
                const ulonglong2 p1 = st[2 * (q0 + q) + 1];
                X[q] = p0.x;
                Y[q] = p0.y;
                Z[q] = p1.x;
                W[q] = p1.y;
            }
#pragma unroll
            for (int r = 0; r < R; ++r) {
#pragma unroll
                for (int q = 0; q < QB; ++q) {
                    uint32_t h0, h1;
                    sphere_hit2(s.a[r], s.b[r], s.c[r], s.d[r], X[q], Y[q], Z[q], W[q], h0, h1);
                    cr[r] += h0 + h1;   // one three-input integer add for both pairs
                }
            }
        }
    } else {
    // Groups of up to 64 record pairs; with SUM, the groups that produced a hit are
    // marked in a 64-bit mask and their interaction terms are added after the group, so
    // the rarely taken term code stays out of the inner loop.
#pragma unroll 1
    for (int g0 = 0; g0 < JS / 2; g0 += 64) {
    uint64_t hitmask = 0;
    const int gend = (g0 + 64 < JS / 2) ? g0 + 64 : JS / 2;
#pragma unroll(MASKED ? 1 : 2)
    for (int q = g0; q < gend; ++q) {
        const ulonglong2 p0 = st[2 * q];
        const ulonglong2 p1 = st[2 * q + 1];
        uint32_t any = 0;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            uint32_t h0, h1;
            if (MODE == MODE_I32_FAST) {
                const f2 v = fast_v(s.a[r], s.b[r], s.c[r], s.d[r], p0, p1);
                h0 = sign_lo(v);
                h1 = sign_hi(v);
            } else if (MODE == MODE_F32) {
#if CC_F32_PACKED
                sphere_hit2(s.a[r], s.b[r], s.c[r], s.d[r], p0.x, p0.y, p1.x, p1.y, h0, h1);
#else
                const float xi = f2_lo(s.a[r]), yi = f2_lo(s.b[r]), zi = f2_lo(s.c[r]), ri = f2_lo(s.d[r]);
                h0 = sphere_hit(xi, yi, zi, ri, f2_lo(p0.x), f2_lo(p0.y), f2_lo(p1.x), f2_lo(p1.y));
                h1 = sphere_hit(xi, yi, zi, ri, f2_hi(p0.x), f2_hi(p0.y), f2_hi(p1.x), f2_hi(p1.y));
#endif
            } else {
                h0 = wide_d2(f2_lo(s.a[r]), f2_lo(s.b[r]), f2_lo(s.c[r]), f2_lo(p0.x), f2_lo(p0.y),
                             f2_lo(p1.x)) <= r2 ? 1u : 0u;
                h1 = wide_d2(f2_lo(s.a[r]), f2_lo(s.b[r]), f2_lo(s.c[r]), f2_hi(p0.x), f2_hi(p0.y),
                             f2_hi(p1.x)) <= r2 ? 1u : 0u;
            }
            if (MASKED) {
                const uint32_t s0 = base[r] + 2u * static_cast<uint32_t>(q);
                h0 &= (s0 < ev[r]) ? 1u : 0u;
                h1 &= (s0 + 1u < ev[r]) ? 1u : 0u;
            }
            cr[r] += h0;
            cr[r] += h1;
            if (SUM) any |= h0 | h1;
        }
        if (SUM) hitmask |= static_cast<uint64_t>(any) << (q - g0);
    }
    if (SUM) {
        while (hitmask) {
            const int b = __ffsll(static_cast<long long>(hitmask)) - 1;
            hitmask &= hitmask - 1;
            const int q = g0 + b;
            const ulonglong2 p0 = st[2 * q];
            const ulonglong2 p1 = st[2 * q + 1];
#pragma unroll 1
            for (int r = 0; r < R; ++r)
                sum += pair_terms<MODE, NT>(s.a[r], s.b[r], s.c[r], s.d[r], p0, p1, eo0 + 2 * q,
                                            tid + r * NT, ev[r], r2);
        }
    }
    }
    }
    uint32_t cnt = 0;
#pragma unroll
    for (int r = 0; r < R; ++r) cnt += cr[r];
    return cnt;
}

}  // namespace cc

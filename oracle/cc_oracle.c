/*
 * CPU oracle for exact pair-collision counting and the pairwise interaction sum.
 *
 * TEST INFRASTRUCTURE ONLY. This file is the slow, plain, obviously correct reference
 * that the CUDA path is checked against. Only the tests, the smoke check of the entry
 * script and the CPU-baseline leg of bench.py may load it. The product library never
 * links, loads or calls it, and it shares no source, header, table or helper with the
 * CUDA path.
 *
 * Paper: Saldanha and de Souza, "High Performance Algorithms for Counting Collisions
 * and Pairwise Interactions" (ICCS 2019, arXiv 1901.11204).
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -fPIC -shared (no -ffast-math). FP
 * contraction must stay off so that the FP32 sphere predicate below rounds after every
 * operation, in the order written (a pin in the tests fails if a build contracts).
 *
 * What each function follows:
 *   oracle_count_i32 / oracle_sum_i32 / oracle_count_f32 -- the standard algorithm for symmetric
 *       pairwise interactions (Section 4, "Standard algorithm for calculating SPI"):
 *       for every i, accumulate interact(obj[i], obj[j]) over every later j.
 *       The loop over i may be split across OpenMP threads; counts are integers, so
 *       the result does not depend on the split.
 *   oracle_cyclic_schedule / oracle_count_i32_cyclic -- the proposed balanced
 *       algorithm (Section 4, "Proposed algorithm for calculating SPI"): every i
 *       evaluates (i+s) mod N for s = 1..(N-1)/2, and for even N the first half of the
 *       objects (i < N/2) evaluate one more step, s = N/2 (Section 4, even-N paragraph).
 *   oracle_count_colls -- Algorithm 1 (Section 3, countColls): a space array of
 *       per-site bead counts; each bead adds the count already at its site.
 *   oracle_count_contacts -- Algorithm 2 (Section 3, countContacts): place every bead,
 *       then sum the counts at the six face neighbours of every bead and halve.
 *
 * Readings of points the paper leaves open:
 *   - interact() for counting is the collision indicator. Integer points collide when
 *     their squared distance is <= r2 (r2 = 0 is the paper's same-site collision of
 *     Section 3). FP32 spheres collide when (dx*dx + dy*dy) + dz*dz <= (ri+rj)*(ri+rj),
 *     every operation rounded to nearest in FP32 in exactly that order.
 *   - The interaction sum adds 1/max(d, 1e-6) over the colliding pairs, with d the
 *     Euclidean distance computed in FP64 from the FP32 coordinates (spheres) or the
 *     FP64 square root of the exact integer squared distance (integer points).
 *   - Counts are unsigned 64-bit (the paper's int counters would overflow).
 *   - Integer squared distances are formed in int64, so no input range limit applies.
 *   - NaN coordinates or radii make the FP32 comparison false.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* Number of OpenMP threads the oracle may use (0 = library default). */
static int g_threads = 0;

void oracle_set_threads(int t) { g_threads = t; }

int oracle_get_threads(void) {
#ifdef _OPENMP
    return g_threads > 0 ? g_threads : omp_get_max_threads();
#else
    return 1;
#endif
}

/* ---- interact() instances -------------------------------------------------------- */

/* Integer collision: squared Euclidean distance (exact, int64) against r2. */
static int collide_i32(int32_t xi, int32_t yi, int32_t zi,
                       int32_t xj, int32_t yj, int32_t zj, uint32_t r2) {
    int64_t dx = (int64_t)xi - (int64_t)xj;
    int64_t dy = (int64_t)yi - (int64_t)yj;
    int64_t dz = (int64_t)zi - (int64_t)zj;
    int64_t d2 = dx * dx + dy * dy + dz * dz;
    return d2 <= (int64_t)r2;
}

/* FP32 sphere collision, every step rounded in FP32, in the stated order. The function
 * is written for a pair (a, b); the same rounding results for (b, a) because a-b and
 * b-a differ only in sign and + and * commute. */
static int collide_f32(float xa, float ya, float za, float ra,
                       float xb, float yb, float zb, float rb) {
    float dx = xa - xb;
    float dy = ya - yb;
    float dz = za - zb;
    float d2 = (dx * dx + dy * dy) + dz * dz;  /* five roundings, this order */
    float s = ra + rb;
    float s2 = s * s;
    return d2 <= s2;
}

/* Interaction term for a colliding sphere pair: 1 / max(d, 1e-6), d in FP64. */
static double term_f64(float xa, float ya, float za, float xb, float yb, float zb) {
    double dx = (double)xa - (double)xb;
    double dy = (double)ya - (double)yb;
    double dz = (double)za - (double)zb;
    double d = sqrt(dx * dx + dy * dy + dz * dz);
    return 1.0 / (d > 1e-6 ? d : 1e-6);
}

/* ---- standard algorithm (Section 4): for i, for j > i ----------------------------- */

uint64_t oracle_count_i32(const int32_t *x, const int32_t *y, const int32_t *z,
                          int64_t n, uint32_t r2) {
    uint64_t count = 0;
    int nt = oracle_get_threads();
    (void)nt;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : count) num_threads(nt)
    for (int64_t i = 0; i < n; ++i) {
        uint64_t c = 0;
        for (int64_t j = i + 1; j < n; ++j)
            c += (uint64_t)collide_i32(x[i], y[i], z[i], x[j], y[j], z[j], r2);
        count += c;
    }
    return count;
}

/* Integer points: returns the count; *sum_out receives the FP64 interaction sum, each
 * colliding pair adding 1 / max(d, 1e-6) with d = sqrt of the exact integer d2. */
uint64_t oracle_sum_i32(const int32_t *x, const int32_t *y, const int32_t *z,
                        int64_t n, uint32_t r2, double *sum_out) {
    uint64_t count = 0;
    double sum = 0.0;
    int nt = oracle_get_threads();
    (void)nt;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : count, sum) num_threads(nt)
    for (int64_t i = 0; i < n; ++i) {
        uint64_t c = 0;
        double s = 0.0;
        for (int64_t j = i + 1; j < n; ++j) {
            int64_t dx = (int64_t)x[i] - (int64_t)x[j];
            int64_t dy = (int64_t)y[i] - (int64_t)y[j];
            int64_t dz = (int64_t)z[i] - (int64_t)z[j];
            int64_t d2 = dx * dx + dy * dy + dz * dz;
            if (d2 <= (int64_t)r2) {
                double d = sqrt((double)d2);
                c += 1;
                s += 1.0 / (d > 1e-6 ? d : 1e-6);
            }
        }
        count += c;
        sum += s;
    }
    if (sum_out) *sum_out = sum;
    return count;
}

/* FP32 spheres: returns the count; *sum_out receives the FP64 interaction sum. */
uint64_t oracle_count_f32(const float *x, const float *y, const float *z, const float *r,
                          int64_t n, double *sum_out) {
    uint64_t count = 0;
    double sum = 0.0;
    int nt = oracle_get_threads();
    (void)nt;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : count, sum) num_threads(nt)
    for (int64_t i = 0; i < n; ++i) {
        uint64_t c = 0;
        double s = 0.0;
        for (int64_t j = i + 1; j < n; ++j) {
            if (collide_f32(x[i], y[i], z[i], r[i], x[j], y[j], z[j], r[j])) {
                c += 1;
                s += term_f64(x[i], y[i], z[i], x[j], y[j], z[j]);
            }
        }
        count += c;
        sum += s;
    }
    if (sum_out) *sum_out = sum;
    return count;
}

/* Batched forms: the same loop applied to every set [off[k], off[k+1]). */
void oracle_count_i32_sets(const int32_t *x, const int32_t *y, const int32_t *z,
                           const int64_t *off, int64_t nsets, uint32_t r2,
                           uint64_t *counts) {
    int nt = oracle_get_threads();
    (void)nt;
#pragma omp parallel for schedule(dynamic, 64) num_threads(nt)
    for (int64_t k = 0; k < nsets; ++k) {
        int64_t a = off[k], b = off[k + 1];
        uint64_t c = 0;
        for (int64_t i = a; i < b; ++i)
            for (int64_t j = i + 1; j < b; ++j)
                c += (uint64_t)collide_i32(x[i], y[i], z[i], x[j], y[j], z[j], r2);
        counts[k] = c;
    }
}

void oracle_count_f32_sets(const float *x, const float *y, const float *z, const float *r,
                           const int64_t *off, int64_t nsets, uint64_t *counts,
                           double *sums) {
    int nt = oracle_get_threads();
    (void)nt;
#pragma omp parallel for schedule(dynamic, 64) num_threads(nt)
    for (int64_t k = 0; k < nsets; ++k) {
        int64_t a = off[k], b = off[k + 1];
        uint64_t c = 0;
        double s = 0.0;
        for (int64_t i = a; i < b; ++i)
            for (int64_t j = i + 1; j < b; ++j)
                if (collide_f32(x[i], y[i], z[i], r[i], x[j], y[j], z[j], r[j])) {
                    c += 1;
                    s += term_f64(x[i], y[i], z[i], x[j], y[j], z[j]);
                }
        counts[k] = c;
        if (sums) sums[k] = s;
    }
}

/* Single FP32 predicate evaluation (used by the symmetry and near-tie pins). */
int oracle_collide_f32(float xa, float ya, float za, float ra,
                       float xb, float yb, float zb, float rb) {
    return collide_f32(xa, ya, za, ra, xb, yb, zb, rb);
}

/* ---- proposed algorithm (Section 4) ----------------------------------------------- */

/* Writes the pairs (i, j) in the order the proposed algorithm evaluates them: for each
 * i, steps s = 1..(N-1)/2 evaluate j = (i+s) mod N; for even N, objects i < N/2 then
 * evaluate one extra step s = N/2. Returns the number of pairs (written only while
 * fewer than cap). Passing cap = 0 only counts. */
int64_t oracle_cyclic_schedule(int64_t n, int64_t *pi, int64_t *pj, int64_t cap) {
    int64_t k = 0;
    if (n < 2) return 0;
    int64_t steps = (n - 1) / 2;
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t s = 1; s <= steps; ++s) {
            if (k < cap) { pi[k] = i; pj[k] = (i + s) % n; }
            ++k;
        }
        if (n % 2 == 0 && i < n / 2) {
            if (k < cap) { pi[k] = i; pj[k] = i + n / 2; }
            ++k;
        }
    }
    return k;
}

/* Number of evaluations object i performs under the proposed algorithm. */
int64_t oracle_cyclic_work(int64_t n, int64_t i) {
    if (n < 2 || i < 0 || i >= n) return 0;
    return (n - 1) / 2 + ((n % 2 == 0 && i < n / 2) ? 1 : 0);
}

/* Integer count taken in the proposed algorithm's order. */
uint64_t oracle_count_i32_cyclic(const int32_t *x, const int32_t *y, const int32_t *z,
                                 int64_t n, uint32_t r2) {
    uint64_t count = 0;
    if (n < 2) return 0;
    int64_t steps = (n - 1) / 2;
    int nt = oracle_get_threads();
    (void)nt;
#pragma omp parallel for schedule(static) reduction(+ : count) num_threads(nt)
    for (int64_t i = 0; i < n; ++i) {
        uint64_t c = 0;
        for (int64_t s = 1; s <= steps; ++s) {
            int64_t j = (i + s) % n;
            c += (uint64_t)collide_i32(x[i], y[i], z[i], x[j], y[j], z[j], r2);
        }
        if (n % 2 == 0 && i < n / 2) {
            int64_t j = i + n / 2;
            c += (uint64_t)collide_i32(x[i], y[i], z[i], x[j], y[j], z[j], r2);
        }
        count += c;
    }
    return count;
}

/* ---- Algorithms 1 and 2 (Section 3) ------------------------------------------------ */

/* The space array covers the beads' bounding box grown by one site on every side, so
 * that the six neighbours of every bead are inside it (the paper translates the space
 * so that indices are non-negative; Section 3). Returns NULL when the box is too big. */
static uint32_t *space_alloc(const int32_t *x, const int32_t *y, const int32_t *z,
                             int64_t n, int64_t lo[3], int64_t dim[3]) {
    int64_t mn[3] = {INT64_MAX, INT64_MAX, INT64_MAX};
    int64_t mx[3] = {INT64_MIN, INT64_MIN, INT64_MIN};
    const int32_t *c[3] = {x, y, z};
    for (int64_t i = 0; i < n; ++i)
        for (int a = 0; a < 3; ++a) {
            if (c[a][i] < mn[a]) mn[a] = c[a][i];
            if (c[a][i] > mx[a]) mx[a] = c[a][i];
        }
    int64_t cells = 1;
    for (int a = 0; a < 3; ++a) {
        lo[a] = mn[a] - 1;
        dim[a] = mx[a] - mn[a] + 3;
        if (dim[a] > (1 << 12)) return NULL;
        cells *= dim[a];
    }
    if (cells > ((int64_t)1 << 31)) return NULL;
    return (uint32_t *)calloc((size_t)cells, sizeof(uint32_t));
}

#define SITE(xx, yy, zz) \
    ((((int64_t)(xx) - lo[0]) * dim[1] + ((int64_t)(yy) - lo[1])) * dim[2] + ((int64_t)(zz) - lo[2]))

/* Algorithm 1: same-site collisions. Returns UINT64_MAX if the space does not fit. */
uint64_t oracle_count_colls(const int32_t *x, const int32_t *y, const int32_t *z, int64_t n) {
    if (n <= 0) return 0;
    int64_t lo[3], dim[3];
    uint32_t *space = space_alloc(x, y, z, n, lo, dim);
    if (!space) return UINT64_MAX;
    uint64_t collisions = 0;
    for (int64_t b = 0; b < n; ++b) {
        int64_t s = SITE(x[b], y[b], z[b]);
        collisions += space[s];   /* beads already at this site */
        space[s] += 1;
    }
    free(space);
    return collisions;
}

/* Algorithm 2: contacts (pairs of beads on face-adjacent sites). UINT64_MAX if the
 * space does not fit. */
uint64_t oracle_count_contacts(const int32_t *x, const int32_t *y, const int32_t *z, int64_t n) {
    if (n <= 0) return 0;
    int64_t lo[3], dim[3];
    uint32_t *space = space_alloc(x, y, z, n, lo, dim);
    if (!space) return UINT64_MAX;
    for (int64_t b = 0; b < n; ++b) space[SITE(x[b], y[b], z[b])] += 1;
    uint64_t contacts = 0;
    for (int64_t b = 0; b < n; ++b) {
        contacts += space[SITE(x[b] + 1, y[b], z[b])];
        contacts += space[SITE(x[b] - 1, y[b], z[b])];
        contacts += space[SITE(x[b], y[b] + 1, z[b])];
        contacts += space[SITE(x[b], y[b] - 1, z[b])];
        contacts += space[SITE(x[b], y[b], z[b] + 1)];
        contacts += space[SITE(x[b], y[b], z[b] - 1)];
    }
    free(space);
    return contacts / 2;
}

// Linear-time counting for integer beads (Section 3 of the paper).
//
// Algorithm 1 (countColls): keep, for every lattice site, the number of beads placed
// there so far; placing a bead adds the count already at its site to the collision
// total, then increments it. The total is sum_k k(k-1)/2 over the sites whatever the
// order of placement, so on the GPU each bead is placed by one thread with an atomic
// increment whose returned old value is exactly the paper's beadCnt.
//
// Algorithm 2 (countContacts): place every bead, then add the counts at the six face
// neighbours of every bead and halve.
//
// The paper indexes a dense array by the coordinates, translated to be non-negative,
// and initialises only the sites that beads touch. Here:
//   dense   when the bounding box grown by one site has at most max(2^24, 16 N) cells:
//           the array covers the box, and a first pass zeroes exactly the sites the
//           counting pass reads or writes (own site; for contacts also the six
//           neighbours), as the paper does;
//   hashed  otherwise: an open-addressing table (linear probing, 2^ceil(log2(2N))
//           slots of {key, count}) stands in for the array; the key packs the site's
//           offsets from the box origin in 21 bits per axis, so spans up to 2^21 - 3
//           per axis are supported (beyond that the call reports CC_ERR_RANGE).
#include <cuda_runtime.h>

#include <algorithm>

#include "cc_internal.cuh"

namespace cc {

constexpr int64_t kHashMaxDim = (int64_t(1) << 21) - 1;

struct LinHeader {
    uint32_t umin[3];
    uint32_t umax[3];
    int32_t dense;          // 1: dense box, 0: hash table, -1: span too large
    uint32_t ticket;
    int64_t lo[3];          // box origin (min - 1)
    int64_t dim[3];         // box extent (span + 3)
    uint64_t cap_mask;      // hash slots - 1
    int64_t dense_cells;    // dense limit for this call
    uint32_t *status;       // the stream workspace's status word
    uint32_t pad[6];
};

struct Slot {
    unsigned long long key;   // 0 = empty
    uint32_t count;
    uint32_t pad;
};
static_assert(sizeof(Slot) == 16, "slot size");

__global__ void k_lin_reset(LinHeader *h, uint32_t *status, unsigned long long *d_count, uint64_t slots,
                            int64_t dense_cells) {
    if (threadIdx.x == 0) {
        h->status = status;
        for (int a = 0; a < 3; ++a) {
            h->umin[a] = 0xFFFFFFFFu;
            h->umax[a] = 0u;
        }
        h->ticket = 0;
        h->cap_mask = slots - 1;
        h->dense_cells = dense_cells;
        *d_count = 0ull;
    }
}

// Bounding box of the beads; the last block picks dense or hashed storage.
__global__ void k_lin_box(const int32_t *__restrict__ x, const int32_t *__restrict__ y,
                          const int32_t *__restrict__ z, int64_t n, LinHeader *h, unsigned long long *d_count) {
    uint32_t mn[3] = {0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu}, mx[3] = {0, 0, 0};
    const int32_t *c[3] = {x, y, z};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        for (int a = 0; a < 3; ++a) {
            const uint32_t u = ord_enc(c[a][i]);
            mn[a] = min(mn[a], u);
            mx[a] = max(mx[a], u);
        }
    __shared__ uint32_t smn[3], smx[3];
    if (threadIdx.x < 3) {
        smn[threadIdx.x] = 0xFFFFFFFFu;
        smx[threadIdx.x] = 0u;
    }
    __syncthreads();
    for (int a = 0; a < 3; ++a) {
        mn[a] = __reduce_min_sync(0xFFFFFFFFu, mn[a]);
        mx[a] = __reduce_max_sync(0xFFFFFFFFu, mx[a]);
        if ((threadIdx.x & 31) == 0) {
            atomicMin(&smn[a], mn[a]);
            atomicMax(&smx[a], mx[a]);
        }
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        atomicMin(&h->umin[threadIdx.x], smn[threadIdx.x]);
        atomicMax(&h->umax[threadIdx.x], smx[threadIdx.x]);
    }
    __syncthreads();
    __shared__ bool last;
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(&h->ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last || threadIdx.x != 0) return;
    __threadfence();
    int64_t cells = 1;
    bool fits_dense = true, fits_hash = true;
    for (int a = 0; a < 3; ++a) {
        const int64_t lo = ord_dec(atomicAdd(&h->umin[a], 0u));
        const int64_t hi = ord_dec(atomicAdd(&h->umax[a], 0u));
        h->lo[a] = lo - 1;
        h->dim[a] = hi - lo + 3;
        if (h->dim[a] > kHashMaxDim) fits_hash = false;
        if (fits_dense && h->dim[a] <= h->dense_cells / cells) cells *= h->dim[a];
        else fits_dense = false;
    }
    h->dense = fits_dense ? 1 : (fits_hash ? 0 : -1);
    if (h->dense < 0) {
        atomicOr(h->status, ST_RANGE);
        *d_count = CC_COUNT_INVALID;
    }
    h->ticket = 0;
}

__device__ __forceinline__ int64_t dense_site(const LinHeader &h, int64_t x, int64_t y, int64_t z) {
    return ((x - h.lo[0]) * h.dim[1] + (y - h.lo[1])) * h.dim[2] + (z - h.lo[2]);
}

// Unique non-zero key of a site inside the box (offsets < 2^21 per axis).
__device__ __forceinline__ unsigned long long site_key(const LinHeader &h, int64_t x, int64_t y, int64_t z) {
    return (static_cast<unsigned long long>(x - h.lo[0]) << 42) |
           (static_cast<unsigned long long>(y - h.lo[1]) << 21) |
           static_cast<unsigned long long>(z - h.lo[2]) | (1ull << 63);
}

__device__ __forceinline__ uint64_t mix64(uint64_t k) {
    k ^= k >> 33;
    k *= 0xff51afd7ed558ccdull;
    k ^= k >> 33;
    k *= 0xc4ceb9fe1a85ec53ull;
    k ^= k >> 33;
    return k;
}

// The slot of a key, inserting it when `insert` (nullptr if absent, or if the table is
// full, which cannot happen with 2N slots for N beads).
__device__ __forceinline__ Slot *hash_slot(Slot *tab, uint64_t mask, unsigned long long key, bool insert) {
    uint64_t i = mix64(key) & mask;
    for (uint64_t probe = 0; probe <= mask; ++probe, i = (i + 1) & mask) {
        unsigned long long k = *reinterpret_cast<volatile unsigned long long *>(&tab[i].key);
        if (k == key) return &tab[i];
        if (k == 0ull) {
            if (!insert) return nullptr;
            k = atomicCAS(&tab[i].key, 0ull, key);
            if (k == 0ull || k == key) return &tab[i];
        }
    }
    return nullptr;
}

// Pass 0: zero the sites the next passes touch (dense) or empty the table (hashed).
__global__ void k_lin_init(const int32_t *__restrict__ x, const int32_t *__restrict__ y,
                           const int32_t *__restrict__ z, int64_t n, const LinHeader *h, uint32_t *space,
                           Slot *tab, int neighbours) {
    const LinHeader H = *h;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    if (H.dense == 1) {
        const int64_t sx = H.dim[1] * H.dim[2], sy = H.dim[2];
        for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < n; b += stride) {
            const int64_t s = dense_site(H, x[b], y[b], z[b]);
            space[s] = 0;
            if (neighbours) {
                space[s + sx] = 0;
                space[s - sx] = 0;
                space[s + sy] = 0;
                space[s - sy] = 0;
                space[s + 1] = 0;
                space[s - 1] = 0;
            }
        }
    } else if (H.dense == 0) {
        for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i <= H.cap_mask; i += stride) {
            tab[i].key = 0ull;
            tab[i].count = 0u;
        }
    }
}

// Pass 1 (Algorithm 1, and the placing loop of Algorithm 2): the old count at a bead's
// site is the number of collisions that bead adds.
__global__ void k_lin_place(const int32_t *__restrict__ x, const int32_t *__restrict__ y,
                            const int32_t *__restrict__ z, int64_t n, const LinHeader *h, uint32_t *space,
                            Slot *tab, unsigned long long *d_collisions) {
    const LinHeader H = *h;
    if (H.dense < 0) return;
    unsigned long long c = 0;
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < n; b += (int64_t)gridDim.x * blockDim.x) {
        if (H.dense == 1) {
            c += atomicAdd(&space[dense_site(H, x[b], y[b], z[b])], 1u);
        } else {
            Slot *s = hash_slot(tab, H.cap_mask, site_key(H, x[b], y[b], z[b]), true);
            if (s) c += atomicAdd(&s->count, 1u);
        }
    }
    for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xFFFFFFFFu, c, o);
    if ((threadIdx.x & 31) == 0 && c && d_collisions) atomicAdd(d_collisions, c);
}

// Pass 2 of Algorithm 2: add the counts at the six face neighbours of every bead.
__global__ void k_lin_contacts(const int32_t *__restrict__ x, const int32_t *__restrict__ y,
                               const int32_t *__restrict__ z, int64_t n, const LinHeader *h,
                               const uint32_t *space, Slot *tab, unsigned long long *d_twice) {
    const LinHeader H = *h;
    if (H.dense < 0) return;
    unsigned long long c = 0;
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < n; b += (int64_t)gridDim.x * blockDim.x) {
        const int64_t bx = x[b], by = y[b], bz = z[b];
        const int64_t nb[6][3] = {{bx + 1, by, bz}, {bx - 1, by, bz}, {bx, by + 1, bz},
                                  {bx, by - 1, bz}, {bx, by, bz + 1}, {bx, by, bz - 1}};
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            if (H.dense == 1) {
                c += space[dense_site(H, nb[k][0], nb[k][1], nb[k][2])];
            } else {
                Slot *s = hash_slot(tab, H.cap_mask, site_key(H, nb[k][0], nb[k][1], nb[k][2]), false);
                if (s) c += s->count;
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xFFFFFFFFu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(d_twice, c);
}

__global__ void k_lin_halve(const LinHeader *h, unsigned long long *d_count) {
    if (threadIdx.x == 0 && h->dense >= 0) *d_count /= 2ull;
}

static uint64_t hash_slots(int64_t n) {
    uint64_t c = 1;
    while (c < static_cast<uint64_t>(2 * std::max<int64_t>(n, 1))) c <<= 1;
    return c;
}

static int64_t dense_limit(int64_t n) { return std::max<int64_t>(int64_t(1) << 24, 16 * n); }

// Workspace: the stream's WsHeader (status word) | LinHeader | dense array or hash table.
static size_t header_bytes() { return 256 + ((sizeof(LinHeader) + 255) / 256) * 256; }

size_t linear_ws_bytes(int64_t n) {
    const size_t dense = static_cast<size_t>(dense_limit(n)) * sizeof(uint32_t);
    const size_t hashed = hash_slots(n) * sizeof(Slot);
    return header_bytes() + std::max(dense, hashed);
}

// contacts = 0: Algorithm 1 into d_count; 1: Algorithm 2 into d_count.
cc_status linear_enqueue(const cc_points *p, int64_t n, int contacts, unsigned long long *d_count, void *ws,
                         cudaStream_t s) {
    WsHeader *wh = reinterpret_cast<WsHeader *>(ws);
    LinHeader *h = reinterpret_cast<LinHeader *>(reinterpret_cast<uint8_t *>(ws) + 256);
    uint8_t *body = reinterpret_cast<uint8_t *>(ws) + header_bytes();
    uint32_t *space = reinterpret_cast<uint32_t *>(body);
    Slot *tab = reinterpret_cast<Slot *>(body);
    k_lin_reset<<<1, 32, 0, s>>>(h, &wh->status, d_count, hash_slots(n), dense_limit(n));
    CC_CUDA(cudaGetLastError());
    if (n == 0) return CC_OK;
    const int32_t *x = static_cast<const int32_t *>(p->x);
    const int32_t *y = static_cast<const int32_t *>(p->y);
    const int32_t *z = static_cast<const int32_t *>(p->z);
    const int blocks = static_cast<int>(std::min<int64_t>((n + 255) / 256, sm_count() * 8));
    k_lin_box<<<std::min(blocks, sm_count() * 4), 256, 0, s>>>(x, y, z, n, h, d_count);
    const uint64_t init_n = std::max<uint64_t>(hash_slots(n), static_cast<uint64_t>(n));
    const int init_blocks =
        static_cast<int>(std::min<uint64_t>((init_n + 255) / 256, static_cast<uint64_t>(sm_count()) * 8));
    k_lin_init<<<init_blocks, 256, 0, s>>>(x, y, z, n, h, space, tab, contacts);
    k_lin_place<<<blocks, 256, 0, s>>>(x, y, z, n, h, space, tab, contacts ? nullptr : d_count);
    if (contacts) {
        k_lin_contacts<<<blocks, 256, 0, s>>>(x, y, z, n, h, space, tab, d_count);
        k_lin_halve<<<1, 32, 0, s>>>(h, d_count);
    }
    CC_CUDA(cudaGetLastError());
    return CC_OK;
}

}  // namespace cc

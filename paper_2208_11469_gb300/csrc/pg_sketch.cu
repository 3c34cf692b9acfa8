// Sketch construction kernels (Sec. II-D): Bloom filters, k-Hash and 1-Hash
// MinHash of every neighbourhood N_v.
//
// Work mapping. One warp builds one vertex's sketch when d_v is at most a
// per-kind threshold. Heavier rows ("hubs": R-MAT graphs have rows of
// hundreds of thousands of entries) are appended to a hub list by that warp
// and finished by a second kernel, so that no single warp serialises a hub:
//   Bloom, k-Hash: hub rows are cut into fixed-size chunks; any block takes
//     any chunk and merges its partial sketch into the row with global
//     atomicOr (Bloom) / atomicMin (k-Hash). The row is initialised by the
//     first kernel (all zero / all 0xFFFFFFFF), which runs before in stream
//     order.
//   1-Hash: one block per hub; each warp keeps the bottom-k of its slice and
//     the block merges the warps' lists.
// The hub list lives in the caller's build workspace:
//   [0] uint64 packed counter (hubs << 32 | chunks), [1] uint64 ticket,
//   then hub records {int32 vertex, int32 first_chunk} in append order, so
//   first_chunk is increasing along the list.
#include "pg_internal.cuh"

namespace pg {

namespace {

constexpr uint32_t kEmpty = 0xFFFFFFFFu;
constexpr int kBuildThreads = 256;
constexpr int kBloomUnroll = 4;  // 32-id chunks of a row loaded together

struct HubList {
    unsigned long long *packed;  // hubs << 32 | chunks
    unsigned long long *ticket;
    int2 *rec;                   // {vertex, first_chunk}
};

__device__ __forceinline__ HubList hub_list(int32_t *base) {
    HubList h;
    h.packed = reinterpret_cast<unsigned long long *>(base);
    h.ticket = reinterpret_cast<unsigned long long *>(base) + 1;
    h.rec = reinterpret_cast<int2 *>(base + 4);
    return h;
}

__device__ __forceinline__ void hub_append(HubList h, int32_t v, int32_t nchunks) {
    unsigned long long old = atomicAdd(h.packed, (1ull << 32) | (unsigned long long)nchunks);
    h.rec[old >> 32] = make_int2(v, (int32_t)(old & 0xffffffffull));
}

// Find the hub record owning chunk ticket t (records sorted by first_chunk).
__device__ __forceinline__ int hub_find(const int2 *rec, int count, int64_t t) {
    int lo = 0, hi = count - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (rec[mid].y <= t)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// Batched graphs (pg_batch_*): vertex v of this launch is global vertex
// bm.v_base + v; its graph g = gid[.] sets its hash count b_of[g] and the id
// offset voff[g] that turns global neighbour ids back into the graph's own ids
// (so a graph's sketch is the same alone and in a batch).
__device__ __forceinline__ void vertex_params(const BatchMap &bm, int64_t v, uint32_t &b, int32_t &id0) {
    if (bm.gid) {
        const int32_t g = __ldg(bm.gid + bm.v_base + v);
        b = bm.b_of[g];
        id0 = __ldg(bm.voff + g);
    }
}

// ---------------------------------------------------------------- Bloom --
// A warp takes 32 consecutive vertices at a time (their 33 row offsets in one
// coalesced load).
//   Short rows (at most kLaneRow ids, LANE only): each lane builds its own
//     vertex's filter in a lane-private shared-memory column (word w of lane r
//     at [w * 32 + r], so every access of lane r is in bank r and needs no
//     atomic), walking its row with eight id loads in flight, and stores the
//     row as 16-byte vectors.
//   Longer rows: the warp builds one row at a time in a warp-shared filter
//     with shared atomicOr (32 ids per step, four steps of loads in flight),
//     fetching the next such row's first ids while hashing the current one.
//   Hub rows (above hub_threshold): stored empty here and filled by
//     k_bloom_hub.
// B: the hash count b fixed at compile time (1 or 2; the seeds' pre-images
// then live in registers), or 0 to take it per vertex (vertex_params).
constexpr int32_t kLaneRow = 32;

template <int kMaxWords32, bool LANE, int B>
__global__ void __launch_bounds__(kBuildThreads) k_bloom_warp(
    const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col, int32_t n, uint32_t l,
    uint32_t b, uint32_t seed, uint8_t *__restrict__ data, int64_t stride, int32_t hub_threshold,
    int32_t chunk, int32_t *hub_base, BatchMap bm) {
    __shared__ uint32_t filt[kBuildThreads / 32][kMaxWords32];
    __shared__ uint32_t pre_s[16];
    extern __shared__ uint32_t lane_filters[];  // LANE: [warps][words32][32]
    const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
    uint32_t *f = filt[warp];
    const int words32 = (int)(stride >> 2);  // whole row including zero padding
    uint32_t *lf = lane_filters + (size_t)warp * words32 * 32 + lane;
    if (threadIdx.x < 16) pre_s[threadIdx.x] = fmix_pre(hash_seed(seed, threadIdx.x));
    for (int t = lane; t < words32; t += 32) f[t] = 0u;
    // with a compile-time hash count B, the seeds' pre-images live in registers
    uint32_t pre_b[B > 0 ? B : 1];
#pragma unroll
    for (int i = 0; i < (B > 0 ? B : 1); ++i) pre_b[i] = fmix_pre(hash_seed(seed, (uint32_t)i));
    __syncthreads();
    HubList hubs = hub_list(hub_base);
    const int64_t warps_total = (int64_t)gridDim.x * (kBuildThreads / 32);
    for (int64_t v0 = ((int64_t)blockIdx.x * (kBuildThreads / 32) + warp) * 32; v0 < n; v0 += warps_total * 32) {
        const int cnt = (int)min((int64_t)32, (int64_t)n - v0);
        // offsets, hash count and id offset of the 32 vertices, one per lane
        const int32_t my_a = (int)lane < cnt ? __ldg(row_ptr + v0 + lane) : 0;
        const int32_t my_e = (int)lane < cnt ? __ldg(row_ptr + v0 + lane + 1) : 0;
        uint32_t my_b = b;
        int32_t my_id0 = 0;
        if ((int)lane < cnt) vertex_params(bm, v0 + lane, my_b, my_id0);
        const bool mine = LANE && (int)lane < cnt && my_e - my_a <= kLaneRow;
        if (mine) {
            for (int w = 0; w < words32; ++w) lf[w * 32] = 0u;
            // eight ids in flight per step
            for (int32_t j = my_a; j < my_e; j += 8) {
                int32_t xs[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) xs[q] = j + q < my_e ? __ldg(col + j + q) : 0;
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    if (j + q >= my_e) break;
                    const uint32_t px = fmix_pre((uint32_t)(xs[q] - my_id0));
                    if (B > 0) {
#pragma unroll
                        for (int i = 0; i < B; ++i) {
                            const uint32_t p = bit_pos(hash_pre(px, pre_b[i]), l);
                            lf[(p >> 5) * 32] |= 1u << (p & 31u);
                        }
                    } else {
                        for (uint32_t i = 0; i < my_b; ++i) {
                            const uint32_t p = bit_pos(hash_pre(px, pre_s[i]), l);
                            lf[(p >> 5) * 32] |= 1u << (p & 31u);
                        }
                    }
                }
            }
            uint4 *row4 = reinterpret_cast<uint4 *>(data + (v0 + lane) * stride);
            for (int q = 0; q < words32 / 4; ++q)
                row4[q] = make_uint4(lf[(4 * q) * 32], lf[(4 * q + 1) * 32], lf[(4 * q + 2) * 32], lf[(4 * q + 3) * 32]);
        }
        // the other vertices of the batch, one warp-wide row at a time
        unsigned rest = __ballot_sync(0xffffffffu, (int)lane < cnt && !mine);
        if (!rest) continue;
        int t = __ffs(rest) - 1;
        int32_t a = __shfl_sync(0xffffffffu, my_a, t), e = __shfl_sync(0xffffffffu, my_e, t);
        int32_t x = (a + (int32_t)lane < e && e - a <= hub_threshold) ? __ldg(col + a + lane) : 0;
        while (true) {
            rest &= rest - 1;
            const int tn = rest ? __ffs(rest) - 1 : 0;
            const int32_t an = __shfl_sync(0xffffffffu, my_a, tn), en = __shfl_sync(0xffffffffu, my_e, tn);
            const uint32_t bv = __shfl_sync(0xffffffffu, my_b, t);
            const int32_t id0 = __shfl_sync(0xffffffffu, my_id0, t);
            // the next row's first ids, in flight while this one is hashed
            const int32_t xn =
                (rest && an + (int32_t)lane < en && en - an <= hub_threshold) ? __ldg(col + an + lane) : 0;
            const int32_t deg = e - a;
            if (deg > hub_threshold) {
                if (lane == 0) hub_append(hubs, (int32_t)(v0 + t), (deg + chunk - 1) / chunk);
            } else if (deg > 0) {
                if ((int32_t)lane < deg) {
                    const uint32_t px = fmix_pre((uint32_t)(x - id0));
                    if (B > 0) {
#pragma unroll
                        for (int i = 0; i < B; ++i) {
                            const uint32_t p = bit_pos(hash_pre(px, pre_b[i]), l);
                            atomicOr(&f[p >> 5], 1u << (p & 31u));
                        }
                    } else {
#pragma unroll 4
                        for (uint32_t i = 0; i < bv; ++i) {
                            const uint32_t p = bit_pos(hash_pre(px, pre_s[i]), l);
                            atomicOr(&f[p >> 5], 1u << (p & 31u));
                        }
                    }
                }
                // longer rows: four 32-id loads in flight before hashing them
                for (int32_t j0 = a + 32; j0 < e; j0 += 32 * kBloomUnroll) {
                    int32_t xs[kBloomUnroll];
#pragma unroll
                    for (int q = 0; q < kBloomUnroll; ++q) {
                        const int32_t j = j0 + 32 * q + (int32_t)lane;
                        xs[q] = j < e ? __ldg(col + j) : 0;
                    }
#pragma unroll
                    for (int q = 0; q < kBloomUnroll; ++q) {
                        if (j0 + 32 * q + (int32_t)lane >= e) continue;
                        const uint32_t px = fmix_pre((uint32_t)(xs[q] - id0));
                        if (B > 0) {
#pragma unroll
                            for (int i = 0; i < B; ++i) {
                                const uint32_t p = bit_pos(hash_pre(px, pre_b[i]), l);
                                atomicOr(&f[p >> 5], 1u << (p & 31u));
                            }
                        } else {
#pragma unroll 4
                            for (uint32_t i = 0; i < bv; ++i) {
                                const uint32_t p = bit_pos(hash_pre(px, pre_s[i]), l);
                                atomicOr(&f[p >> 5], 1u << (p & 31u));
                            }
                        }
                    }
                }
            }
            __syncwarp();
            uint32_t *row = reinterpret_cast<uint32_t *>(data + (v0 + t) * stride);
            for (int w = lane; w < words32; w += 32) {
                row[w] = f[w];  // a hub row is stored empty here and filled by k_bloom_hub
                f[w] = 0u;
            }
            __syncwarp();
            if (!rest) break;
            t = tn;
            a = an;
            e = en;
            x = xn;
        }
    }
}

// Hub chunks: the block ORs its chunk's bits into a shared filter, then
// merges it into the row with 64-bit global atomicOr. Each block takes a
// contiguous range of chunk tickets (the chunks cost the same, so the ranges
// are balanced) and finds the owning hub record once, then steps through the
// records as the tickets pass their first chunks. Each thread keeps
// kHubUnroll loads of ids in flight before hashing them.
constexpr int kHubUnroll = 8;

template <int kMaxWords32>
__global__ void __launch_bounds__(kBuildThreads) k_bloom_hub(
    const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col, uint32_t l, uint32_t b,
    uint32_t seed, uint8_t *__restrict__ data, int64_t stride, int32_t chunk, int32_t *hub_base,
    BatchMap bm) {
    __shared__ uint32_t f[kMaxWords32];
    __shared__ uint32_t pre_s[16];
    if (threadIdx.x < 16) pre_s[threadIdx.x] = fmix_pre(hash_seed(seed, threadIdx.x));
    HubList hubs = hub_list(hub_base);
    const unsigned long long packed = *reinterpret_cast<volatile unsigned long long *>(hubs.packed);
    const int count = (int)(packed >> 32);
    const int64_t total = (int64_t)(packed & 0xffffffffull);
    const int words32 = (int)(stride >> 2);
    const int64_t t0 = total * blockIdx.x / gridDim.x, t1 = total * (blockIdx.x + 1) / gridDim.x;
    if (t0 >= t1) return;  // the whole block
    int h = hub_find(hubs.rec, count, t0);
    int2 rec = hubs.rec[h];
    int64_t next = h + 1 < count ? (int64_t)hubs.rec[h + 1].y : INT64_MAX;
    int32_t a = row_ptr[rec.x], e = row_ptr[rec.x + 1];
    uint32_t bv = b;
    int32_t id0 = 0;
    vertex_params(bm, rec.x, bv, id0);
    for (int64_t t = t0; t < t1; ++t) {
        while (t >= next) {
            ++h;
            rec = hubs.rec[h];
            next = h + 1 < count ? (int64_t)hubs.rec[h + 1].y : INT64_MAX;
            a = row_ptr[rec.x];
            e = row_ptr[rec.x + 1];
            bv = b;
            id0 = 0;
            vertex_params(bm, rec.x, bv, id0);
        }
        for (int q = threadIdx.x; q < words32; q += blockDim.x) f[q] = 0u;
        __syncthreads();
        const int32_t c0 = a + (int32_t)(t - rec.y) * chunk;
        const int32_t c1 = min(e, c0 + chunk);
        for (int32_t j0 = c0 + (int32_t)threadIdx.x; j0 < c1; j0 += kHubUnroll * (int32_t)blockDim.x) {
            int32_t xs[kHubUnroll];
#pragma unroll
            for (int q = 0; q < kHubUnroll; ++q) {
                const int32_t j = j0 + q * (int32_t)blockDim.x;
                xs[q] = j < c1 ? __ldg(col + j) : 0;
            }
#pragma unroll
            for (int q = 0; q < kHubUnroll; ++q) {
                if (j0 + q * (int32_t)blockDim.x >= c1) continue;
                const uint32_t px = fmix_pre((uint32_t)(xs[q] - id0));
                for (uint32_t i = 0; i < bv; ++i) {
                    const uint32_t p = bit_pos(hash_pre(px, pre_s[i]), l);
                    atomicOr(&f[p >> 5], 1u << (p & 31u));
                }
            }
        }
        __syncthreads();
        unsigned long long *row = reinterpret_cast<unsigned long long *>(data + (int64_t)rec.x * stride);
        for (int q = threadIdx.x; q < words32 / 2; q += blockDim.x) {
            unsigned long long w = (unsigned long long)f[2 * q] | ((unsigned long long)f[2 * q + 1] << 32);
            if (w) atomicOr(row + q, w);
        }
        __syncthreads();
    }
}

// --------------------------------------------------------------- k-Hash --
// Lane r owns hash indices i = r + t*(32/P) (t < KPL); with P > 1 the warp
// splits into P partitions that walk disjoint element subsets and are
// min-combined at the end. Elements are loaded 32 at a time (coalesced, the
// next 32 in flight while the current ones are hashed) and broadcast by
// shuffles.
template <int KPL, int P>
__device__ __forceinline__ void khash_slice(const int32_t *__restrict__ col, int32_t a, int32_t e,
                                            const uint32_t (&pre_s)[KPL], uint32_t (&mn)[KPL]) {
    constexpr int kLanesPerPart = 32 / P;
    const unsigned lane = lane_id();
    const unsigned part = lane / kLanesPerPart;
    int32_t nx = (a + (int32_t)lane < e) ? __ldg(col + a + lane) : 0;
    for (int32_t base = a; base < e; base += 32) {
        const int32_t cnt = min(32, e - base);
        const uint32_t px_mine = (lane < (unsigned)cnt) ? fmix_pre((uint32_t)nx) : 0u;
        // the next 32 ids in flight while these are hashed
        nx = (base + 32 + (int32_t)lane < e) ? __ldg(col + base + 32 + lane) : 0;
        if (P == 1 && cnt == 32) {
            // a full chunk, two entries per step: one three-input min takes both hashes, and no
            // per-entry bound check
#pragma unroll 4
            for (int s = 0; s < 32; s += 2) {
                const uint32_t p1 = __shfl_sync(0xffffffffu, px_mine, s);
                const uint32_t p2 = __shfl_sync(0xffffffffu, px_mine, s + 1);
#pragma unroll
                for (int t = 0; t < KPL; ++t)
                    mn[t] = __vimin3_u32(mn[t], hash_pre(p1, pre_s[t]), hash_pre(p2, pre_s[t]));
            }
            continue;
        }
        for (int s = 0; s < cnt; s += P) {
            const int src = s + (int)part;
            const uint32_t px = __shfl_sync(0xffffffffu, px_mine, src & 31);
            if (src < cnt) {
#pragma unroll
                for (int t = 0; t < KPL; ++t) mn[t] = min(mn[t], hash_pre(px, pre_s[t]));
            }
        }
    }
}

template <int KPL, int P>
__global__ void __launch_bounds__(kBuildThreads) k_khash_warp(
    const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col, int32_t n, uint32_t k,
    uint32_t seed, uint8_t *__restrict__ data, int64_t stride, int32_t hub_threshold,
    int32_t chunk, int32_t *hub_base) {
    constexpr int kLanesPerPart = 32 / P;
    const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
    const unsigned slot = lane % kLanesPerPart;
    uint32_t pre_s[KPL];
#pragma unroll
    for (int t = 0; t < KPL; ++t) {
        const uint32_t i = slot + t * kLanesPerPart;
        pre_s[t] = fmix_pre(hash_seed(seed, i < k ? i : 0u));
    }
    HubList hubs = hub_list(hub_base);
    const int64_t warps_total = (int64_t)gridDim.x * (kBuildThreads / 32);
    for (int64_t v = blockIdx.x * (int64_t)(kBuildThreads / 32) + warp; v < n; v += warps_total) {
        const int32_t a = row_ptr[v], e = row_ptr[v + 1];
        uint32_t mn[KPL];
#pragma unroll
        for (int t = 0; t < KPL; ++t) mn[t] = kEmpty;
        if (e - a > hub_threshold) {
            if (lane == 0) hub_append(hubs, (int32_t)v, (e - a + chunk - 1) / chunk);
        } else {
            khash_slice<KPL, P>(col, a, e, pre_s, mn);
        }
#pragma unroll
        for (int o = kLanesPerPart; o < 32; o <<= 1)
#pragma unroll
            for (int t = 0; t < KPL; ++t) mn[t] = min(mn[t], __shfl_xor_sync(0xffffffffu, mn[t], o));
        uint32_t *row = reinterpret_cast<uint32_t *>(data + v * stride);
        if (lane < (unsigned)kLanesPerPart) {
#pragma unroll
            for (int t = 0; t < KPL; ++t) {
                const uint32_t i = slot + t * kLanesPerPart;
                if (i < k) row[i] = mn[t];
            }
        }
    }
}

// Hub chunks of 2048 ids: the block's warps take equal slices, min-combine
// them in shared memory and merge into the row with global atomicMin. As in
// k_bloom_hub, each block takes a contiguous range of chunk tickets and
// locates the owning hub record once.
template <int KPL, int P>
__global__ void __launch_bounds__(kBuildThreads) k_khash_hub(
    const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col, uint32_t k, uint32_t seed,
    uint8_t *__restrict__ data, int64_t stride, int32_t chunk, int32_t *hub_base) {
    constexpr int kLanesPerPart = 32 / P;
    __shared__ uint32_t smin[256];
    const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
    const unsigned slot = lane % kLanesPerPart;
    uint32_t pre_s[KPL];
#pragma unroll
    for (int t = 0; t < KPL; ++t) {
        const uint32_t i = slot + t * kLanesPerPart;
        pre_s[t] = fmix_pre(hash_seed(seed, i < k ? i : 0u));
    }
    HubList hubs = hub_list(hub_base);
    const unsigned long long packed = *reinterpret_cast<volatile unsigned long long *>(hubs.packed);
    const int count = (int)(packed >> 32);
    const int64_t total = (int64_t)(packed & 0xffffffffull);
    constexpr int kWarps = kBuildThreads / 32;
    const int64_t t0 = total * blockIdx.x / gridDim.x, t1 = total * (blockIdx.x + 1) / gridDim.x;
    if (t0 >= t1) return;  // the whole block
    int h = hub_find(hubs.rec, count, t0);
    int2 rec = hubs.rec[h];
    int64_t next = h + 1 < count ? (int64_t)hubs.rec[h + 1].y : INT64_MAX;
    int32_t a = row_ptr[rec.x], e = row_ptr[rec.x + 1];
    for (int64_t t = t0; t < t1; ++t) {
        while (t >= next) {
            ++h;
            rec = hubs.rec[h];
            next = h + 1 < count ? (int64_t)hubs.rec[h + 1].y : INT64_MAX;
            a = row_ptr[rec.x];
            e = row_ptr[rec.x + 1];
        }
        for (int q = threadIdx.x; q < (int)k; q += blockDim.x) smin[q] = kEmpty;
        __syncthreads();
        const int32_t c0 = a + (int32_t)(t - rec.y) * chunk;
        const int32_t c1 = min(e, c0 + chunk);
        // warp w takes the w-th of kWarps equal slices of the chunk
        const int32_t len = c1 - c0;
        const int32_t per = (len + kWarps - 1) / kWarps;
        const int32_t w0 = min(c1, c0 + (int32_t)warp * per), w1 = min(c1, w0 + per);
        uint32_t mn[KPL];
#pragma unroll
        for (int q = 0; q < KPL; ++q) mn[q] = kEmpty;
        khash_slice<KPL, P>(col, w0, w1, pre_s, mn);
#pragma unroll
        for (int o = kLanesPerPart; o < 32; o <<= 1)
#pragma unroll
            for (int q = 0; q < KPL; ++q) mn[q] = min(mn[q], __shfl_xor_sync(0xffffffffu, mn[q], o));
        if (lane < (unsigned)kLanesPerPart) {
#pragma unroll
            for (int q = 0; q < KPL; ++q) {
                const uint32_t i = slot + q * kLanesPerPart;
                if (i < k) atomicMin(&smin[i], mn[q]);
            }
        }
        __syncthreads();
        uint32_t *row = reinterpret_cast<uint32_t *>(data + (int64_t)rec.x * stride);
        for (int q = threadIdx.x; q < (int)k; q += blockDim.x)
            if (smin[q] != kEmpty) atomicMin(row + q, smin[q]);
        __syncthreads();
    }
}

// --------------------------------------------------------------- 1-Hash --
// A warp keeps the current bottom-k as one value per lane, sorted ascending
// (lane r holds the r-th smallest). A chunk of 32 new hashes is sorted with a
// bitonic network across lanes, merged against the reversed current list by
// lane-wise min (the result is bitonic) and re-sorted by a bitonic merge.
// Hash values are distinct within a row (h_0 is a bijection), so value
// order is a total order and no ties arise.
__device__ __forceinline__ uint32_t bitonic_sort32(uint32_t x) {
    const unsigned lane = lane_id();
#pragma unroll
    for (int size = 2; size <= 32; size <<= 1) {
#pragma unroll
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            const uint32_t y = __shfl_xor_sync(0xffffffffu, x, stride);
            const bool up = ((lane & size) == 0);
            const bool lower = ((lane & stride) == 0);
            x = (lower == up) ? min(x, y) : max(x, y);
        }
    }
    return x;
}

__device__ __forceinline__ uint32_t bitonic_merge32(uint32_t x) {
    const unsigned lane = lane_id();
#pragma unroll
    for (int stride = 16; stride > 0; stride >>= 1) {
        const uint32_t y = __shfl_xor_sync(0xffffffffu, x, stride);
        x = ((lane & stride) == 0) ? min(x, y) : max(x, y);
    }
    return x;
}

// Merge a sorted 32-list `cand` into the sorted 32-list `best`, keeping the
// 32 smallest, sorted.
__device__ __forceinline__ uint32_t merge_keep_smallest(uint32_t best, uint32_t cand) {
    const uint32_t rev = __shfl_sync(0xffffffffu, cand, 31 - (int)lane_id());
    return bitonic_merge32(min(best, rev));
}

// Bottom-32 of h_0 over col[a, e): returns lane r's r-th smallest value.
// `filled` counts how many real values the list holds (min(32, seen)).
__device__ __forceinline__ uint32_t bottom32(const int32_t *__restrict__ col, int32_t a, int32_t e,
                                             uint32_t pre_s, uint32_t best, int &filled) {
    const unsigned lane = lane_id();
    for (int32_t base = a; base < e; base += 32) {
        const int32_t cnt = min(32, e - base);
        const bool valid = lane < (unsigned)cnt;
        const uint32_t h = valid ? hash_pre(fmix_pre((uint32_t)__ldg(col + base + lane)), pre_s) : kEmpty;
        const uint32_t thr = __shfl_sync(0xffffffffu, best, 31);
        const bool cand = valid && (filled < 32 || h < thr);
        if (__ballot_sync(0xffffffffu, cand) == 0u) continue;
        const uint32_t sorted = bitonic_sort32(cand ? h : kEmpty);
        best = merge_keep_smallest(best, sorted);
        filled = min(32, filled + cnt);
    }
    return best;
}

__global__ void __launch_bounds__(kBuildThreads) k_1hash_warp(
    const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col, int32_t n, uint32_t k,
    uint32_t seed, uint8_t *__restrict__ data, int64_t stride, int32_t hub_threshold,
    int32_t *hub_base) {
    const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
    const uint32_t pre_s = fmix_pre(hash_seed(seed, 0));
    HubList hubs = hub_list(hub_base);
    const int64_t warps_total = (int64_t)gridDim.x * (kBuildThreads / 32);
    for (int64_t v = blockIdx.x * (int64_t)(kBuildThreads / 32) + warp; v < n; v += warps_total) {
        const int32_t a = row_ptr[v], e = row_ptr[v + 1];
        if (e - a > hub_threshold) {
            if (lane == 0) hub_append(hubs, (int32_t)v, 1);
            continue;
        }
        int filled = 0;
        const uint32_t best = bottom32(col, a, e, pre_s, kEmpty, filled);
        uint32_t *row = reinterpret_cast<uint32_t *>(data + v * stride);
        if (lane < k) row[lane] = best;
    }
}

__global__ void __launch_bounds__(1024) k_1hash_hub(const int32_t *__restrict__ row_ptr,
                                                    const int32_t *__restrict__ col, uint32_t k,
                                                    uint32_t seed, uint8_t *__restrict__ data,
                                                    int64_t stride, int32_t *hub_base) {
    __shared__ uint32_t lists[32][32];
    const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
    const unsigned nwarps = blockDim.x >> 5;
    const uint32_t pre_s = fmix_pre(hash_seed(seed, 0));
    HubList hubs = hub_list(hub_base);
    const unsigned long long packed = *reinterpret_cast<volatile unsigned long long *>(hubs.packed);
    const int count = (int)(packed >> 32);
    for (int h = blockIdx.x; h < count; h += gridDim.x) {
        const int32_t v = hubs.rec[h].x;
        const int32_t a = row_ptr[v], e = row_ptr[v + 1];
        const int32_t len = e - a;
        const int32_t per = (len + (int)nwarps - 1) / (int)nwarps;
        const int32_t w0 = min(e, a + (int32_t)warp * per), w1 = min(e, w0 + per);
        int filled = 0;
        lists[warp][lane] = bottom32(col, w0, w1, pre_s, kEmpty, filled);
        __syncthreads();
        if (warp == 0) {
            uint32_t best = lists[0][lane];
            for (unsigned w = 1; w < nwarps; ++w) best = merge_keep_smallest(best, lists[w][lane]);
            uint32_t *row = reinterpret_cast<uint32_t *>(data + (int64_t)v * stride);
            if (lane < k) row[lane] = best;
        }
        __syncthreads();
    }
}

int build_grid(int32_t n) {
    int64_t want = ((int64_t)n + (kBuildThreads / 32) - 1) / (kBuildThreads / 32);
    int64_t cap = (int64_t)device_info().sm_count * 8;
    if (want > cap) want = cap;
    return want < 1 ? 1 : (int)want;
}

}  // namespace

constexpr int32_t kBloomHub = 8192, kBloomChunk = 8192;
constexpr int32_t kKhashHub = 2048, kKhashChunk = 2048;
constexpr int32_t k1hashHub = 4096;

// Hub-list scratch: two counters + one record per possible hub (a hub has
// more entries than the smallest threshold).
size_t build_workspace_bytes(int64_t nnz) {
    int32_t t = kBloomHub;
    if (kKhashHub < t) t = kKhashHub;
    if (k1hashHub < t) t = k1hashHub;
    const int64_t max_hubs = nnz / ((int64_t)t + 1) + 1;
    return round_up(16 + 8 * (size_t)max_hubs, 256);
}

cudaError_t launch_build_bloom(const int32_t *row_ptr, const int32_t *col, int32_t n, uint32_t l,
                               uint32_t b, uint32_t seed, uint8_t *data, int64_t stride,
                               int32_t *hub_base, cudaStream_t s, const BatchMap *bmap) {
    if (n == 0) return cudaSuccess;
    const BatchMap bm = bmap ? *bmap : BatchMap{};
    launch_fill_u64(reinterpret_cast<uint64_t *>(hub_base), 2, 0, s);
    const int grid = build_grid(n);
    const int hub_grid = device_info().sm_count * 8;
    if (stride <= 128) {
        // lane-private filters for short rows: words x 32 lanes x warps
        const size_t lane_smem = (size_t)(stride / 4) * 32 * (kBuildThreads / 32) * 4;
        // the hash count fixed at compile time for b = 1 and b = 2 (a batched launch covers whole
        // graphs of one bucket, which all have the bucket's b)
        if (b == 2)
            k_bloom_warp<32, true, 2><<<grid, kBuildThreads, lane_smem, s>>>(
                row_ptr, col, n, l, b, seed, data, stride, kBloomHub, kBloomChunk, hub_base, bm);
        else if (b == 1)
            k_bloom_warp<32, true, 1><<<grid, kBuildThreads, lane_smem, s>>>(
                row_ptr, col, n, l, b, seed, data, stride, kBloomHub, kBloomChunk, hub_base, bm);
        else
            k_bloom_warp<32, true, 0><<<grid, kBuildThreads, lane_smem, s>>>(
                row_ptr, col, n, l, b, seed, data, stride, kBloomHub, kBloomChunk, hub_base, bm);
        k_bloom_hub<32><<<hub_grid, kBuildThreads, 0, s>>>(row_ptr, col, l, b, seed, data, stride,
                                                           kBloomChunk, hub_base, bm);
        note_launch(2);
    } else {
        k_bloom_warp<256, false, 0><<<grid, kBuildThreads, 0, s>>>(row_ptr, col, n, l, b, seed, data, stride,
                                                                kBloomHub, kBloomChunk, hub_base, bm);
        k_bloom_hub<256><<<hub_grid, kBuildThreads, 0, s>>>(row_ptr, col, l, b, seed, data, stride,
                                                            kBloomChunk, hub_base, bm);
        note_launch(2);
    }
    return cudaGetLastError();
}

template <int KPL, int P>
static void khash_pair(const int32_t *row_ptr, const int32_t *col, int32_t n, uint32_t k,
                       uint32_t seed, uint8_t *data, int64_t stride, int32_t *hub_base,
                       cudaStream_t s) {
    k_khash_warp<KPL, P><<<build_grid(n), kBuildThreads, 0, s>>>(row_ptr, col, n, k, seed, data,
                                                                 stride, kKhashHub, kKhashChunk,
                                                                 hub_base);
    k_khash_hub<KPL, P><<<device_info().sm_count * 5, kBuildThreads, 0, s>>>(
        row_ptr, col, k, seed, data, stride, kKhashChunk, hub_base);
    note_launch(2);
}

cudaError_t launch_build_khash(const int32_t *row_ptr, const int32_t *col, int32_t n, uint32_t k,
                               uint32_t seed, uint8_t *data, int64_t stride, int32_t *hub_base,
                               cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    launch_fill_u64(reinterpret_cast<uint64_t *>(hub_base), 2, 0, s);
    if (k <= 16 && (16 % k) == 0) {
        switch (k) {
            case 1: khash_pair<1, 32>(row_ptr, col, n, k, seed, data, stride, hub_base, s); break;
            case 2: khash_pair<1, 16>(row_ptr, col, n, k, seed, data, stride, hub_base, s); break;
            case 4: khash_pair<1, 8>(row_ptr, col, n, k, seed, data, stride, hub_base, s); break;
            case 8: khash_pair<1, 4>(row_ptr, col, n, k, seed, data, stride, hub_base, s); break;
            default: khash_pair<1, 2>(row_ptr, col, n, k, seed, data, stride, hub_base, s); break;
        }
    } else if (k <= 32) {
        khash_pair<1, 1>(row_ptr, col, n, k, seed, data, stride, hub_base, s);
    } else if (k <= 64) {
        khash_pair<2, 1>(row_ptr, col, n, k, seed, data, stride, hub_base, s);
    } else if (k <= 128) {
        khash_pair<4, 1>(row_ptr, col, n, k, seed, data, stride, hub_base, s);
    } else {
        khash_pair<8, 1>(row_ptr, col, n, k, seed, data, stride, hub_base, s);
    }
    return cudaGetLastError();
}

cudaError_t launch_build_1hash(const int32_t *row_ptr, const int32_t *col, int32_t n, uint32_t k,
                               uint32_t seed, uint8_t *data, int64_t stride, int32_t *hub_base,
                               cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    launch_fill_u64(reinterpret_cast<uint64_t *>(hub_base), 2, 0, s);
    k_1hash_warp<<<build_grid(n), kBuildThreads, 0, s>>>(row_ptr, col, n, k, seed, data, stride,
                                                         k1hashHub, hub_base);
    k_1hash_hub<<<device_info().sm_count * 2, 1024, 0, s>>>(row_ptr, col, k, seed, data, stride,
                                                            hub_base);
    note_launch(2);
    return cudaGetLastError();
}

}  // namespace pg

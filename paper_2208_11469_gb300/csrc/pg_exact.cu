// Exact |N_u ∩ N_v| on the GPU — the plain comparison for the sketched path.
//
// Triangle count and per-vertex triangles follow the node-iterator of
// Sec. III, Listing 1, over the degree-oriented neighbourhoods
// N+_v = {u in N_v : (d_u, u) > (d_v, v)} (K9): every triangle is counted
// exactly once, at its lowest-ranked edge, and the longest oriented list is
// O(sqrt(m)). Orientation runs flat over the CSR entries:
//   keep[j] = rank(col[j]) > rank(row(j)), exclusive scan of keep, scatter.
// Counting runs per vertex u with N+_u staged in shared memory (sorted by
// id): the lists N+_v of all v in N+_u are walked, 32 entries per warp
// step, and each entry w is looked up in N+_u held in a shared-memory hash
// table; w found = triangle (u, v, w). Vertices with at most kWarpList
// oriented neighbours take one warp each (the lists N+_v walked as one flat
// sequence); longer lists take a whole block with a larger table (lists
// beyond the block's shared memory are searched in global memory).
// Pair queries and per-edge exact counts intersect the full rows: a group of
// kL lanes binary-searches each element of the shorter list in the longer.
#include "pg_internal.cuh"

namespace pg {

namespace {

constexpr int kThreads = 256;
constexpr int kL = 8;  // lanes per edge

__device__ __forceinline__ bool rank_less(int32_t du, int32_t u, int32_t dv, int32_t v) {
    return du < dv || (du == dv && u < v);
}

// Each thread walks a contiguous slice of CSR entries; keep[j] is 1 when the
// entry points to a higher-ranked neighbour. keep has nnz + 1 entries.
__global__ void __launch_bounds__(kThreads) k_orient_flags(const int32_t *__restrict__ row_ptr,
                                                           const int32_t *__restrict__ col,
                                                           int32_t n, int64_t nnz,
                                                           int32_t *__restrict__ keep) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t T = (int64_t)gridDim.x * blockDim.x;
    const int64_t j0 = t * nnz / T, j1 = (t + 1) * nnz / T;
    if (t == 0) keep[nnz] = 0;
    if (j0 >= j1) return;
    int32_t lo = 0, hi = n - 1;  // largest u with row_ptr[u] <= j0
    while (lo < hi) {
        const int32_t mid = (lo + hi + 1) >> 1;
        if (row_ptr[mid] <= j0)
            lo = mid;
        else
            hi = mid - 1;
    }
    int32_t u = lo;
    int32_t end = row_ptr[u + 1];
    int32_t du = end - row_ptr[u];
    for (int64_t j = j0; j < j1; ++j) {
        while (j >= end) {
            ++u;
            const int32_t s = end;
            end = row_ptr[u + 1];
            du = end - s;
        }
        const int32_t v = __ldg(col + j);
        const int32_t dv = __ldg(row_ptr + v + 1) - __ldg(row_ptr + v);
        keep[j] = rank_less(du, u, dv, v) ? 1 : 0;
    }
}

__global__ void k_orient_scatter(const int32_t *__restrict__ row_ptr,
                                 const int32_t *__restrict__ col, int32_t n, int64_t nnz,
                                 const int32_t *__restrict__ pos, int32_t *__restrict__ plus_off,
                                 int32_t *__restrict__ plus_col) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < nnz; j += stride)
        if (pos[j + 1] != pos[j]) plus_col[pos[j]] = col[j];
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u <= n; u += stride)
        plus_off[u] = pos[row_ptr[u]];
}

// |A ∩ B| restricted to this lane's share of the shorter list; calls f(w)
// for every common element this lane finds.
template <class F>
__device__ __forceinline__ uint32_t lane_intersect(const int32_t *A, int32_t la, const int32_t *B,
                                                   int32_t lb, unsigned g, F f) {
    if (la > lb) {
        const int32_t *T = A;
        A = B;
        B = T;
        const int32_t t = la;
        la = lb;
        lb = t;
    }
    uint32_t c = 0;
    for (int32_t i = (int32_t)g; i < la; i += kL) {
        const int32_t x = __ldg(A + i);
        int32_t lo = 0, hi = lb;
        while (lo < hi) {
            const int32_t mid = (lo + hi) >> 1;
            if (__ldg(B + mid) < x)
                lo = mid + 1;
            else
                hi = mid;
        }
        if (lo < lb && __ldg(B + lo) == x) {
            ++c;
            f(x);
        }
    }
    return c;
}

constexpr int kWarpList = 256;   // oriented list length handled by one warp
constexpr int kBlockThreads = 512;
constexpr int kBlockListBytes = 32 * 1024;  // shared-memory hash table of the block kernel (4 blocks per SM)

constexpr int kHashSlots = 2 * kWarpList;  // open-addressing table of N+_u, at most half full

__device__ __forceinline__ uint32_t slot_of(int32_t x) { return ((uint32_t)x * 0x9E3779B1u) >> 23; }  // 9 bits

// One warp per vertex u with 2 <= |N+_u| <= kWarpList. N+_u goes into a
// shared-memory hash table (linear probing, -1 = empty); the lists N+_v of
// its vertices v are walked as one flat sequence of pre[a] entries, lane p
// taking entries p, p + 32, ...: entry p belongs to the last i with
// pre[i] <= p (found by moving forward from the previous entry's i, as p
// only grows), and its w is a triangle (u, v, w) iff w is in the table.
template <bool WANT_S>
__global__ void __launch_bounds__(kThreads) k_exact_warp(const int32_t *__restrict__ plus_off,
                                                         const int32_t *__restrict__ plus_col, int32_t n, double *S,
                                                         unsigned long long *tc_total) {
    __shared__ int32_t s_hash[kThreads / 32][kHashSlots];
    __shared__ int32_t s_list[kThreads / 32][kWarpList];
    __shared__ int32_t s_pre[kThreads / 32][kWarpList + 1];
    __shared__ int32_t s_beg[kThreads / 32][kWarpList];
    const unsigned lane = lane_id(), wib = threadIdx.x >> 5;
    int32_t *hash = s_hash[wib], *list = s_list[wib], *pre = s_pre[wib], *beg = s_beg[wib];
    const int64_t warp = ((int64_t)blockIdx.x * kThreads + threadIdx.x) >> 5;
    const int64_t warps = (int64_t)gridDim.x * (kThreads >> 5);
    unsigned long long my = 0;
    for (int i = lane; i < kHashSlots; i += 32) hash[i] = -1;
    for (int64_t u = warp; u < n; u += warps) {
        const int32_t a0 = __ldg(plus_off + u), a = __ldg(plus_off + u + 1) - a0;
        if (a < 2 || a > kWarpList) continue;
        __syncwarp();
        // stage N+_u (list and hash table), the list starts and lengths of its vertices, and the prefix
        int32_t carry = 0;
        for (int32_t i0 = 0; i0 < a; i0 += 32) {
            const int32_t i = i0 + (int32_t)lane;
            int32_t len = 0;
            if (i < a) {
                const int32_t v = __ldg(plus_col + a0 + i);
                list[i] = v;
                uint32_t h = slot_of(v);
                while (atomicCAS(hash + h, -1, v) != -1) h = (h + 1) & (kHashSlots - 1);
                const int32_t b0 = __ldg(plus_off + v);
                beg[i] = b0;
                len = __ldg(plus_off + v + 1) - b0;
            }
            int32_t incl = len;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int32_t t = __shfl_up_sync(0xffffffffu, incl, o);
                if ((int)lane >= o) incl += t;
            }
            if (i < a) pre[i] = carry + incl - len;
            carry += __shfl_sync(0xffffffffu, incl, 31);
        }
        if (lane == 0) pre[a] = carry;
        __syncwarp();
        uint32_t c = 0;
        int32_t lo = 0;  // the last i with pre[i] <= p; p only grows, so lo moves forward
        for (int32_t p = (int32_t)lane; p < carry; p += 32) {
            while (lo + 1 < a && pre[lo + 1] <= p) ++lo;
            const int32_t w = __ldg(plus_col + beg[lo] + (p - pre[lo]));
            uint32_t h = slot_of(w);
            int32_t x;
            while ((x = hash[h]) != -1 && x != w) h = (h + 1) & (kHashSlots - 1);
            if (x == w) {
                ++c;
                if (WANT_S) {
                    atomicAdd(S + w, 2.0);
                    atomicAdd(S + list[lo], 2.0);
                }
            }
        }
        const uint32_t tot = __reduce_add_sync(0xffffffffu, c);
        my += tot;
        if (WANT_S && lane == 0 && tot) atomicAdd(S + u, 2.0 * tot);
        __syncwarp();
        for (int32_t i = (int32_t)lane; i < a; i += 32) {  // clear the table entries this vertex used
            uint32_t h = slot_of(list[i]);
            while (hash[h] != list[i]) h = (h + 1) & (kHashSlots - 1);
            hash[h] = -1;
        }
    }
    if (lane == 0 && my) atomicAdd(tc_total, my);
}

// The vertices with more than kWarpList oriented neighbours, listed for
// k_exact_block (ids[0 .. *count)).
__global__ void k_exact_long_list(const int32_t *__restrict__ plus_off, int32_t n, int32_t *count,
                                  int32_t *ids) {
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x)
        if (plus_off[u + 1] - plus_off[u] > kWarpList) ids[atomicAdd(count, 1)] = (int32_t)u;
}

// One block per listed vertex u: N+_u in a shared-memory hash table of the
// next power of two at or above 2 |N+_u| slots (up to kBlockSlots; longer
// lists are binary-searched in global memory, where they are sorted); warp j
// walks the lists N+_v of v = N+_u[j], N+_u[j + warps], ..., 32 entries per
// step, looking each entry up.
constexpr int kBlockSlots = kBlockListBytes / 4;  // power of two

template <bool WANT_S>
__global__ void __launch_bounds__(kBlockThreads) k_exact_block(const int32_t *__restrict__ plus_off,
                                                               const int32_t *__restrict__ plus_col,
                                                               const int32_t *count, const int32_t *ids, double *S,
                                                               unsigned long long *tc_total) {
    extern __shared__ __align__(16) int32_t s_hash[];
    __shared__ uint32_t s_tot;
    const unsigned lane = lane_id(), wib = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int32_t cnt = *count;
    unsigned long long my = 0;
    for (int32_t t = blockIdx.x; t < cnt; t += gridDim.x) {
        const int32_t u = ids[t];
        const int32_t a0 = plus_off[u], a = plus_off[u + 1] - a0;
        int32_t bits = 1;
        while (bits < 30 && (1 << bits) < 2 * a) ++bits;
        const bool hashed = (1 << bits) <= kBlockSlots;
        const uint32_t mask = (1u << bits) - 1u;
        if (threadIdx.x == 0) s_tot = 0;
        if (hashed) {
            for (int32_t i = threadIdx.x; i <= (int32_t)mask; i += blockDim.x) s_hash[i] = -1;
            __syncthreads();
            for (int32_t i = threadIdx.x; i < a; i += blockDim.x) {
                const int32_t x = __ldg(plus_col + a0 + i);
                uint32_t h = ((uint32_t)x * 0x9E3779B1u) >> (32 - bits);
                while (atomicCAS(s_hash + h, -1, x) != -1) h = (h + 1) & mask;
            }
        }
        __syncthreads();
        uint32_t c = 0;
        for (int32_t i = (int32_t)wib; i < a; i += (int32_t)nw) {
            const int32_t v = __ldg(plus_col + a0 + i);
            const int32_t b0 = __ldg(plus_off + v), b = __ldg(plus_off + v + 1) - b0;
            for (int32_t j = (int32_t)lane; j < b; j += 32) {
                const int32_t w = __ldg(plus_col + b0 + j);
                bool hit;
                if (hashed) {
                    uint32_t h = ((uint32_t)w * 0x9E3779B1u) >> (32 - bits);
                    int32_t x;
                    while ((x = s_hash[h]) != -1 && x != w) h = (h + 1) & mask;
                    hit = x == w;
                } else {
                    int32_t x = 0, y = a;
                    while (x < y) {
                        const int32_t mid = (x + y) >> 1;
                        if (__ldg(plus_col + a0 + mid) < w)
                            x = mid + 1;
                        else
                            y = mid;
                    }
                    hit = x < a && __ldg(plus_col + a0 + x) == w;
                }
                if (hit) {
                    ++c;
                    if (WANT_S) {
                        atomicAdd(S + w, 2.0);
                        atomicAdd(S + v, 2.0);
                    }
                }
            }
        }
        const uint32_t wsum = __reduce_add_sync(0xffffffffu, c);
        if (lane == 0 && wsum) atomicAdd(&s_tot, wsum);
        __syncthreads();
        if (threadIdx.x == 0) {
            my += s_tot;
            if (WANT_S && s_tot) atomicAdd(S + u, 2.0 * s_tot);
        }
        __syncthreads();  // the table and s_tot are rewritten for the next vertex
    }
    if (threadIdx.x == 0 && my) atomicAdd(tc_total, my);
}

__global__ void k_exact_result(const unsigned long long *tc_total, const int32_t *upper_off,
                               int32_t n, pg_tc_result *out) {
    const unsigned long long t = *tc_total;
    out->edges = (uint64_t)upper_off[n];
    out->count_sum = 3ull * t;
    out->exact_tc = t;
    out->reserved = 0;
    out->est_tc = (double)t;
    out->est_tc_alt = 0.0;
}

// Exact |N_u ∩ N_v| per upper edge (lists eu/ev) or pair over the full rows.
template <bool PAIRS>
__global__ void __launch_bounds__(kThreads) k_exact_pairs(const int32_t *__restrict__ row_ptr,
                                                          const int32_t *__restrict__ col,
                                                          int32_t n, EdgeIndex ix,
                                                          const int32_t *__restrict__ pairs,
                                                          int64_t P, bool list_order, int32_t *count, float *cn,
                                                          float *jac, float *ovl, float *tot) {
    const unsigned lane = lane_id();
    const unsigned g = lane % kL;
    const int64_t group = ((int64_t)blockIdx.x * kThreads + threadIdx.x) / kL;
    const int64_t groups = (int64_t)gridDim.x * kThreads / kL;
    int64_t total = PAIRS ? P : (int64_t)ix.upper_off[n];
    if (!PAIRS && total > ix.cap) total = ix.cap;
    const int64_t e0 = group * total / groups, e1 = (group + 1) * total / groups;
    const int32_t my_n = (int32_t)(e1 - e0);
    const int32_t warp_n = (int32_t)__reduce_max_sync(0xffffffffu, (unsigned)(my_n > 0 ? my_n : 0));
    for (int32_t i = 0; i < warp_n; ++i) {
        const int64_t e = e0 + i;
        uint32_t c = 0;
        int32_t du = 0, dv = 0, xu = 0;
        if (e < e1) {
            int32_t x, y;
            bool ok = true;
            if (PAIRS) {
                const int2 pr = __ldg(reinterpret_cast<const int2 *>(pairs) + e);
                // an id outside [0, n) makes an invalid pair: treated as two empty sets
                ok = pr.x >= 0 && pr.x < n && pr.y >= 0 && pr.y < n;
                x = pr.x;
                y = pr.y;
            } else {
                x = __ldg(ix.eu + e);
                y = __ldg(ix.ev + e);
            }
            xu = x;
            if (ok) {
                const int32_t a = __ldg(row_ptr + x);
                du = __ldg(row_ptr + x + 1) - a;
                const int32_t b = __ldg(row_ptr + y);
                dv = __ldg(row_ptr + y + 1) - b;
                c = lane_intersect(col + a, du, col + b, dv, g, [](int32_t) {});
            }
        }
#pragma unroll
        for (int o = kL / 2; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
        if (e < e1 && g == 0) {
            // outputs: pairs and list-order requests at e, upper edges at their upper-edge index
            const int64_t o = (PAIRS || list_order || ix.groups == 1)
                                  ? e
                                  : upper_pos(row_ptr, n, ix.upper_off, ix.goff, ix.seg_end,
                                              list_group(ix.goff, n, ix.groups, e), xu, e);
            if (count) count[o] = (int32_t)c;
            if (cn) cn[o] = (float)c;
            const float I = (float)c, den = (float)du + (float)dv - I, mn = fminf((float)du, (float)dv);
            if (jac) jac[o] = den > 0.0f ? I / den : 0.0f;
            if (ovl) ovl[o] = mn > 0.0f ? I / mn : 0.0f;
            if (tot) tot[o] = den;
        }
    }
}

int persistent_grid() { return device_info().sm_count * (2048 / kThreads); }

}  // namespace

size_t exact_workspace_bytes(int32_t n, int64_t nnz) {
    // pos/keep [nnz+1] | plus_off [n+1] | plus_col [nnz/2] | scan scratch | counter
    return round_up(4 * (size_t)(nnz + 1), 256) + round_up(4 * (size_t)(n + 1), 256) +
           round_up(4 * (size_t)(nnz / 2 + 1), 256) + scan_scratch_bytes(nnz + 1) + 256;
}

cudaError_t launch_exact_tc(const int32_t *row_ptr, const int32_t *col, int32_t n, int64_t nnz,
                            const int32_t *upper_off, void *ws, double *S, pg_tc_result *tc,
                            cudaStream_t s) {
    uint8_t *w = static_cast<uint8_t *>(ws);
    int32_t *pos = reinterpret_cast<int32_t *>(w);
    w += round_up(4 * (size_t)(nnz + 1), 256);
    int32_t *plus_off = reinterpret_cast<int32_t *>(w);
    w += round_up(4 * (size_t)(n + 1), 256);
    int32_t *plus_col = reinterpret_cast<int32_t *>(w);
    w += round_up(4 * (size_t)(nnz / 2 + 1), 256);
    int32_t *scratch = reinterpret_cast<int32_t *>(w);
    w += scan_scratch_bytes(nnz + 1);
    unsigned long long *counter = reinterpret_cast<unsigned long long *>(w);
    launch_fill_u64(reinterpret_cast<uint64_t *>(counter), 1, 0, s);
    if (n > 0) {
        k_orient_flags<<<persistent_grid(), kThreads, 0, s>>>(row_ptr, col, n, nnz, pos);
        cudaError_t e = launch_exclusive_scan(pos, nnz + 1, scratch, s);
        if (e != cudaSuccess) return e;
        k_orient_scatter<<<persistent_grid(), kThreads, 0, s>>>(row_ptr, col, n, nnz, pos, plus_off,
                                                                plus_col);
        // pos is free after the scatter: pos[0] counts the long lists and pos[1..] lists them (a long
        // list holds more than 256 of the nnz / 2 oriented edges, so at most nnz / 514 vertices have one)
        int32_t *long_count = pos;
        int32_t *long_ids = pos + 1;
        launch_fill_u64(reinterpret_cast<uint64_t *>(long_count), 1, 0, s);
        cudaError_t ea = cudaFuncSetAttribute(S ? k_exact_block<true> : k_exact_block<false>,
                                              cudaFuncAttributeMaxDynamicSharedMemorySize, kBlockListBytes);
        if (ea != cudaSuccess) return ea;
        k_exact_long_list<<<persistent_grid(), kThreads, 0, s>>>(plus_off, n, long_count, long_ids);
        if (S) {
            k_exact_warp<true><<<persistent_grid(), kThreads, 0, s>>>(plus_off, plus_col, n, S, counter);
            k_exact_block<true><<<4 * device_info().sm_count, kBlockThreads, kBlockListBytes, s>>>(
                plus_off, plus_col, long_count, long_ids, S, counter);
        } else {
            k_exact_warp<false><<<persistent_grid(), kThreads, 0, s>>>(plus_off, plus_col, n, S, counter);
            k_exact_block<false><<<4 * device_info().sm_count, kBlockThreads, kBlockListBytes, s>>>(
                plus_off, plus_col, long_count, long_ids, S, counter);
        }
        note_launch(5);
    }
    if (tc) {
        k_exact_result<<<1, 1, 0, s>>>(counter, upper_off, n, tc);
        note_launch();
    }
    return cudaGetLastError();
}

cudaError_t launch_orient(const int32_t *row_ptr, const int32_t *col, int32_t n, int64_t nnz, void *ws,
                          int32_t **plus_off_out, int32_t **plus_col_out, cudaStream_t s) {
    uint8_t *w = static_cast<uint8_t *>(ws);
    int32_t *pos = reinterpret_cast<int32_t *>(w);
    w += round_up(4 * (size_t)(nnz + 1), 256);
    int32_t *plus_off = reinterpret_cast<int32_t *>(w);
    w += round_up(4 * (size_t)(n + 1), 256);
    int32_t *plus_col = reinterpret_cast<int32_t *>(w);
    w += round_up(4 * (size_t)(nnz / 2 + 1), 256);
    int32_t *scratch = reinterpret_cast<int32_t *>(w);
    *plus_off_out = plus_off;
    *plus_col_out = plus_col;
    if (n == 0) {
        launch_fill_u64(reinterpret_cast<uint64_t *>(plus_off), 1, 0, s);
        return cudaGetLastError();
    }
    k_orient_flags<<<persistent_grid(), kThreads, 0, s>>>(row_ptr, col, n, nnz, pos);
    cudaError_t e = launch_exclusive_scan(pos, nnz + 1, scratch, s);
    if (e != cudaSuccess) return e;
    k_orient_scatter<<<persistent_grid(), kThreads, 0, s>>>(row_ptr, col, n, nnz, pos, plus_off, plus_col);
    note_launch(2);
    return cudaGetLastError();
}

cudaError_t launch_exact_pairs(const int32_t *row_ptr, const int32_t *col, int32_t n,
                               const EdgeIndex &ix, const int32_t *pairs, int64_t P,
                               const EdgeOutputs &out, cudaStream_t s) {
    if (pairs) {
        if (P > 0)
        {
            k_exact_pairs<true><<<persistent_grid(), kThreads, 0, s>>>(row_ptr, col, n, ix, pairs, P, false,
                                                                       out.count, out.cn, out.jac, out.ovl,
                                                                       out.tot);
            note_launch();
        }
    } else if (n > 0) {
        k_exact_pairs<false><<<persistent_grid(), kThreads, 0, s>>>(row_ptr, col, n, ix, nullptr, 0,
                                                                    out.list_order, out.count, out.cn, out.jac,
                                                                    out.ovl, out.tot);
        note_launch();
    }
    return cudaGetLastError();
}

}  // namespace pg

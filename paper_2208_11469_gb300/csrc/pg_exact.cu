// Exact |N_u ∩ N_v| on the GPU — the plain comparison for the sketched path.
//
// Triangle count and per-vertex triangles follow the node-iterator of
// Sec. III, Listing 1, over the degree-oriented neighbourhoods
// N+_v = {u in N_v : (d_u, u) > (d_v, v)} (K9): every triangle is counted
// exactly once, at its lowest-ranked edge, and the longest oriented list is
// O(sqrt(m)). Orientation runs flat over the CSR entries:
//   keep[j] = rank(col[j]) > rank(row(j)), exclusive scan of keep, scatter.
// Counting runs flat over the oriented edges: a group of kL lanes intersects
// N+_u and N+_v by binary-searching each element of the shorter list in the
// longer one (both sorted by id).
// Pair queries and per-edge exact counts intersect the full rows the same way.
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

// Oriented node iteration: TC and S_v = 2 * (triangles at v).
__global__ void __launch_bounds__(kThreads) k_exact_oriented(const int32_t *__restrict__ plus_off,
                                                             const int32_t *__restrict__ plus_col,
                                                             int32_t n, double *S,
                                                             unsigned long long *tc_total) {
    __shared__ unsigned long long s_tc;
    if (threadIdx.x == 0) s_tc = 0ull;
    __syncthreads();
    const unsigned lane = lane_id();
    const unsigned g = lane % kL;
    const int64_t group = ((int64_t)blockIdx.x * kThreads + threadIdx.x) / kL;
    const int64_t groups = (int64_t)gridDim.x * kThreads / kL;
    const int64_t m = plus_off[n];
    const int64_t e0 = group * m / groups, e1 = (group + 1) * m / groups;
    unsigned long long my_tc = 0;
    int32_t u = 0, next = 0;
    if (e0 < e1) {
        int32_t lo = 0, hi = n - 1;
        while (lo < hi) {
            const int32_t mid = (lo + hi + 1) >> 1;
            if (plus_off[mid] <= e0)
                lo = mid;
            else
                hi = mid - 1;
        }
        u = lo;
        next = plus_off[u + 1];
    }
    double acc = 0.0;
    int32_t acc_v = -1;
    const int32_t my_n = (int32_t)(e1 - e0);
    const int32_t warp_n = (int32_t)__reduce_max_sync(0xffffffffu, (unsigned)(my_n > 0 ? my_n : 0));
    for (int32_t i = 0; i < warp_n; ++i) {
        const int64_t e = e0 + i;
        uint32_t c = 0;
        int32_t v = -1;
        if (e < e1) {
            while (e >= next) {
                ++u;
                next = plus_off[u + 1];
            }
            v = __ldg(plus_col + e);
            const int32_t au = plus_off[u], av = __ldg(plus_off + v);
            c = lane_intersect(plus_col + au, next - au, plus_col + av, __ldg(plus_off + v + 1) - av,
                               g, [&](int32_t w) {
                                   if (S) atomicAdd(S + w, 2.0);
                               });
        }
#pragma unroll
        for (int o = kL / 2; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
        if (e < e1 && g == 0) {
            my_tc += c;
            if (S && c) {
                if (u != acc_v) {
                    if (acc_v >= 0) atomicAdd(S + acc_v, acc);
                    acc_v = u;
                    acc = 0.0;
                }
                acc += 2.0 * c;
                atomicAdd(S + v, 2.0 * c);
            }
        }
    }
    if (S && g == 0 && acc_v >= 0 && acc != 0.0) atomicAdd(S + acc_v, acc);
    if (my_tc) atomicAdd(&s_tc, my_tc);
    __syncthreads();
    if (threadIdx.x == 0 && s_tc) atomicAdd(tc_total, s_tc);
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
                                                          int64_t P, int32_t *count, float *cn,
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
        int32_t du = 0, dv = 0;
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
            if (count) count[e] = (int32_t)c;
            if (cn) cn[e] = (float)c;
            const float I = (float)c, den = (float)du + (float)dv - I, mn = fminf((float)du, (float)dv);
            if (jac) jac[e] = den > 0.0f ? I / den : 0.0f;
            if (ovl) ovl[e] = mn > 0.0f ? I / mn : 0.0f;
            if (tot) tot[e] = den;
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
        k_exact_oriented<<<persistent_grid(), kThreads, 0, s>>>(plus_off, plus_col, n, S, counter);
        note_launch(3);
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
            k_exact_pairs<true><<<persistent_grid(), kThreads, 0, s>>>(row_ptr, col, n, ix, pairs, P,
                                                                       out.count, out.cn, out.jac, out.ovl,
                                                                       out.tot);
            note_launch();
        }
    } else if (n > 0) {
        k_exact_pairs<false><<<persistent_grid(), kThreads, 0, s>>>(row_ptr, col, n, ix, nullptr, 0,
                                                                    out.count, out.cn, out.jac, out.ovl,
                                                                    out.tot);
        note_launch();
    }
    return cudaGetLastError();
}

}  // namespace pg

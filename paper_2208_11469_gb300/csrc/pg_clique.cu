// 4-clique counting (Sec. III-A, Listing "Reformulated 4-Clique Counting").
//
// Vertices are ranked by (degree, id); N+_v holds the neighbours ranked above
// v. For every oriented edge u -> v, C3 = N+_u ∩ N+_v lists the 3-cliques
// (u, v, w) once each, and the 4-cliques are sum over w in C3 of
// |N+_w ∩ C3|. ProbGraph estimates that innermost intersection from Bloom
// filters of the oriented neighbourhoods: |N+_w ∩ C3| = |N+_u ∩ N+_v ∩ N+_w|
// is read off popcount(BF+_u AND BF+_v AND BF+_w) with the AND (or L)
// estimator, C3 itself being enumerated exactly.
//
// Kernel: flat over the oriented edges, a group of kG lanes per edge
// intersects N+_u and N+_v by binary-searching each element of the shorter
// list in the longer one (both in increasing id order); the lane that finds
// w handles that 3-clique: with a sketch it adds the triple-AND popcount to a
// shared histogram (exact integers, reduced once per block), exactly it
// counts the members of N+_w that lie in both N+_u and N+_v.
#include "pg_internal.cuh"

namespace pg {
namespace {

constexpr int kThreads = 256;
constexpr int kG = 8;  // lanes per oriented edge

__device__ __forceinline__ bool in_sorted(const int32_t *__restrict__ B, int32_t lb, int32_t x) {
    int32_t lo = 0, hi = lb;
    while (lo < hi) {
        const int32_t mid = (lo + hi) >> 1;
        if (__ldg(B + mid) < x)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo < lb && __ldg(B + lo) == x;
}

// NV = 16-byte vectors per filter row (a power of two >= l / 128); words at or
// beyond l / 32 are row padding and masked.
template <int NV>
__device__ __forceinline__ uint32_t triple_and_ones(const uint8_t *ru, const uint8_t *rv, const uint8_t *rw,
                                                    uint32_t l, int32_t nvec) {
    const uint32_t wl = l / 32u;
    uint32_t c = 0;
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        if (q < nvec) {
            const uint4 a = __ldg(reinterpret_cast<const uint4 *>(ru) + q);
            const uint4 b = __ldg(reinterpret_cast<const uint4 *>(rv) + q);
            const uint4 d = __ldg(reinterpret_cast<const uint4 *>(rw) + q);
            const uint32_t w0 = 4u * (uint32_t)q;
            c += __popc(a.x & b.x & d.x) + __popc(a.y & b.y & d.y) +
                 (w0 + 2 < wl ? __popc(a.z & b.z & d.z) + __popc(a.w & b.w & d.w) : 0u);
        }
    }
    return c;
}

template <bool EXACT, int NV>
__global__ void __launch_bounds__(kThreads) k_clique4(const int32_t *__restrict__ plus_off,
                                                      const int32_t *__restrict__ plus_col, int32_t n,
                                                      const uint8_t *__restrict__ data, int64_t stride, uint32_t l,
                                                      int32_t nvec, unsigned long long *hist,
                                                      unsigned long long *totals) {
    extern __shared__ uint32_t h32[];  // sketch: l + 1 bins
    __shared__ unsigned long long s_tri, s_ck;
    if (!EXACT)
        for (uint32_t i = threadIdx.x; i <= l; i += blockDim.x) h32[i] = 0u;
    if (threadIdx.x == 0) s_tri = s_ck = 0ull;
    __syncthreads();
    const unsigned lane = lane_id();
    const unsigned g = lane % kG;
    const int64_t group = ((int64_t)blockIdx.x * kThreads + threadIdx.x) / kG;
    const int64_t groups = (int64_t)gridDim.x * kThreads / kG;
    const int64_t m = plus_off[n];
    const int64_t e0 = group * m / groups, e1 = (group + 1) * m / groups;
    unsigned long long my_tri = 0, my_ck = 0;
    int32_t u = 0, next = 0;
    if (e0 < e1) {  // largest u with plus_off[u] <= e0
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
    for (int64_t e = e0; e < e1; ++e) {
        while (e >= next) {
            ++u;
            next = plus_off[u + 1];
        }
        const int32_t v = __ldg(plus_col + e);
        const int32_t au = plus_off[u], lu = next - au;
        const int32_t av = __ldg(plus_off + v), lv = __ldg(plus_off + v + 1) - av;
        const int32_t *Nu = plus_col + au, *Nv = plus_col + av;
        // this lane's share of the shorter list, searched in the longer one
        const int32_t *A = lu <= lv ? Nu : Nv, *Bl = lu <= lv ? Nv : Nu;
        const int32_t la = lu <= lv ? lu : lv, lb = lu <= lv ? lv : lu;
        for (int32_t i = (int32_t)g; i < la; i += kG) {
            const int32_t w = __ldg(A + i);
            if (!in_sorted(Bl, lb, w)) continue;
            ++my_tri;
            if (EXACT) {
                const int32_t aw = __ldg(plus_off + w), lw = __ldg(plus_off + w + 1) - aw;
                for (int32_t t = 0; t < lw; ++t) {
                    const int32_t x = __ldg(plus_col + aw + t);
                    my_ck += (in_sorted(Nu, lu, x) && in_sorted(Nv, lv, x)) ? 1u : 0u;
                }
            } else {
                const uint32_t c = triple_and_ones<NV>(data + (int64_t)u * stride, data + (int64_t)v * stride,
                                                       data + (int64_t)w * stride, l, nvec);
                atomicAdd(h32 + c, 1u);
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        my_tri += __shfl_xor_sync(0xffffffffu, my_tri, o);
        my_ck += __shfl_xor_sync(0xffffffffu, my_ck, o);
    }
    if (lane == 0) {
        if (my_tri) atomicAdd(&s_tri, my_tri);
        if (my_ck) atomicAdd(&s_ck, my_ck);
    }
    __syncthreads();
    if (!EXACT)
        for (uint32_t i = threadIdx.x; i <= l; i += blockDim.x)
            if (h32[i]) atomicAdd(hist + i, (unsigned long long)h32[i]);
    if (threadIdx.x == 0) {
        if (s_tri) atomicAdd(totals, s_tri);
        if (s_ck) atomicAdd(totals + 1, s_ck);
    }
}

// Totals from the histogram in a fixed order (one block): the estimate with
// the chosen estimator, the alternative one, and the popcount sum.
__global__ void __launch_bounds__(256) k_clique4_result(const unsigned long long *hist,
                                                        const unsigned long long *totals, int32_t est, uint32_t l,
                                                        uint32_t b, pg_clique4_result *out) {
    __shared__ double s_a[256], s_b[256];
    __shared__ unsigned long long s_c[256];
    double fa = 0.0, fb = 0.0;
    unsigned long long cs = 0;
    if (hist) {
        for (uint32_t j = threadIdx.x; j <= l; j += blockDim.x) {
            const unsigned long long h = hist[j];
            const double B1 = (j == l) ? (double)j - 1.0 : (double)j;
            const double f_and = -((double)l / (double)b) * log(1.0 - B1 / (double)l);
            const double f_l = (double)j / (double)b;
            fa += (double)h * (est == PG_EST_BF_L ? f_l : f_and);
            fb += (double)h * (est == PG_EST_BF_L ? f_and : f_l);
            cs += h * j;
        }
    }
    s_a[threadIdx.x] = fa;
    s_b[threadIdx.x] = fb;
    s_c[threadIdx.x] = cs;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            s_a[threadIdx.x] += s_a[threadIdx.x + o];
            s_b[threadIdx.x] += s_b[threadIdx.x + o];
            s_c[threadIdx.x] += s_c[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out->triangles = totals[0];
        out->exact = hist ? 0ull : totals[1];
        out->count_sum = s_c[0];
        out->reserved = 0;
        out->est = hist ? s_a[0] : (double)totals[1];
        out->est_alt = hist ? s_b[0] : 0.0;
    }
}

struct C4Layout {
    size_t orient, sketch, build, hist, totals, total;
};
C4Layout c4_layout(const pg_csr *g, int32_t est, uint32_t bits) {
    C4Layout L{};
    size_t o = 0;
    auto take = [&](size_t b) {
        const size_t at = o;
        o += round_up(b ? b : 1, 256);
        return at;
    };
    L.orient = take(exact_workspace_bytes(g->n, g->nnz));
    if (est != PG_EST_EXACT) {
        L.sketch = take((size_t)g->n * (size_t)pg_sketch_stride(PG_SK_BLOOM, bits, 0) + 16);
        L.build = take(build_workspace_bytes(g->nnz / 2 + 1));
        L.hist = take(8 * ((size_t)bits + 1));
    }
    L.totals = take(16);
    L.total = o;
    return L;
}

int c4_grid() { return device_info().sm_count * (2048 / kThreads); }

template <bool EXACT, int NV>
cudaError_t run_c4(const int32_t *po, const int32_t *pc, int32_t n, const uint8_t *data, int64_t stride, uint32_t l,
                   unsigned long long *hist, unsigned long long *totals, cudaStream_t s) {
    const size_t smem = EXACT ? 0 : 4 * ((size_t)l + 1);
    k_clique4<EXACT, NV><<<c4_grid(), kThreads, smem, s>>>(po, pc, n, data, stride, l, (int32_t)((l + 127) / 128),
                                                           hist, totals);
    note_launch();
    return cudaGetLastError();
}

}  // namespace
}  // namespace pg

using namespace pg;

extern "C" {

size_t pg_clique4_workspace_bytes(const pg_csr *g, int32_t estimator, uint32_t bits) {
    if (!g || g->n < 0 || g->nnz < 0) return 0;
    return c4_layout(g, estimator, bits).total;
}

pg_status pg_clique4_count(const pg_csr *g, int32_t estimator, uint32_t bits, uint32_t b, uint32_t seed,
                           void *workspace, size_t workspace_bytes, pg_clique4_result *out, pg_stream_t stream) {
    PG_TRACE("pg_clique4_count");
    pg_status st = check_graph(g);
    if (st) return st;
    PG_REQUIRE(estimator == PG_EST_EXACT || estimator == PG_EST_BF_AND || estimator == PG_EST_BF_L,
               PG_ERR_UNSUPPORTED, "pg_clique4_count: estimator %d (EXACT, BF_AND or BF_L)", estimator);
    if (estimator != PG_EST_EXACT)
        PG_REQUIRE(bits >= 64 && bits <= 1024 && bits % 64 == 0 && b >= 1 && b <= 16, PG_ERR_UNSUPPORTED,
                   "pg_clique4_count: bits %u (multiple of 64 in [64, 1024]), b %u (1..16)", bits, b);
    PG_REQUIRE(out != nullptr && (reinterpret_cast<uintptr_t>(out) & 7u) == 0, PG_ERR_INVALID_ARG,
               "pg_clique4_count: out must be an 8-byte aligned device pg_clique4_result");
    const C4Layout L = c4_layout(g, estimator, bits);
    PG_REQUIRE(workspace && aligned16(workspace) && workspace_bytes >= L.total, PG_ERR_NO_MEMORY,
               "pg_clique4_count: workspace has %zu bytes, needs %zu", workspace_bytes, L.total);
    uint8_t *w = static_cast<uint8_t *>(workspace);
    cudaStream_t s = stream;
    int32_t *po = nullptr, *pc = nullptr;
    PG_TRY_CUDA(launch_orient(g->row_ptr, g->col, g->n, g->nnz, w + L.orient, &po, &pc, s), "pg_clique4_count");
    unsigned long long *totals = reinterpret_cast<unsigned long long *>(w + L.totals);
    launch_fill_u64(reinterpret_cast<uint64_t *>(totals), 2, 0, s);
    unsigned long long *hist = nullptr;
    uint8_t *data = nullptr;
    int64_t stride = 0;
    if (estimator != PG_EST_EXACT) {
        hist = reinterpret_cast<unsigned long long *>(w + L.hist);
        launch_fill_u64(reinterpret_cast<uint64_t *>(hist), (size_t)bits + 1, 0, s);
        data = w + L.sketch;
        stride = pg_sketch_stride(PG_SK_BLOOM, bits, 0);
        // filters of the oriented neighbourhoods N+_v
        PG_TRY_CUDA(launch_build_bloom(po, pc, g->n, bits, b, seed, data, stride,
                                       reinterpret_cast<int32_t *>(w + L.build), s),
                    "pg_clique4_count: Bloom build");
    }
    cudaError_t e = cudaSuccess;
    if (g->n > 0) {
        if (estimator == PG_EST_EXACT) {
            e = run_c4<true, 1>(po, pc, g->n, nullptr, 0, 0, nullptr, totals, s);
        } else {
            const int nv = (int)((bits + 127) / 128);
            e = nv <= 1   ? run_c4<false, 1>(po, pc, g->n, data, stride, bits, hist, totals, s)
                : nv <= 2 ? run_c4<false, 2>(po, pc, g->n, data, stride, bits, hist, totals, s)
                : nv <= 4 ? run_c4<false, 4>(po, pc, g->n, data, stride, bits, hist, totals, s)
                          : run_c4<false, 8>(po, pc, g->n, data, stride, bits, hist, totals, s);
        }
    }
    PG_TRY_CUDA(e, "pg_clique4_count");
    k_clique4_result<<<1, 256, 0, s>>>(hist, totals, estimator, bits, b, out);
    note_launch();
    PG_TRY_CUDA(cudaGetLastError(), "pg_clique4_count: result");
    return PG_OK;
}

}  // extern "C"

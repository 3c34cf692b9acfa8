// Jarvis-Patrick clustering (Sec. III, Listing "Jarvis-Patrick
// clustering"): an edge (u, v) stays in the clustering C when its
// common-neighbour count |N_u ∩ N_v| (exact or estimated) exceeds tau; the
// clusters are the connected components of (V, C).
//
// One call = the per-edge count pass of the chosen estimator (the same
// kernels as pg_edge_counts) -> k_jp_union: the keep test of every upper
// edge and a lock-free union-find over the kept ones -> k_jp_labels: every
// vertex's root and the cluster count.
//
// Union-find: parent[v] <= v always holds, because a union only ever makes
// the larger of two roots point at the smaller one (atomicCAS on the larger
// root), and path halving only replaces a parent by one of its ancestors.
// Parent values therefore only decrease, every find ends after at most n
// steps, a failed hook is retried only because another thread hooked that
// root first, and each component's final root is its smallest vertex id
// whatever the order of the unions: the labels are deterministic.
//
// The keep test per estimator (the oracle takes the same decisions in the
// same double arithmetic): exact count > tau; Bloom AND: count >= the
// smallest count whose AND estimate exceeds tau (computed on the host, the
// estimate being non-decreasing in the count); Bloom L: count / b > tau;
// k-Hash and 1-Hash: J / (1 + J) * (d_u + d_v) > tau with J = c / K.
#include <cmath>

#include "pg_internal.cuh"

namespace pg {
namespace {

constexpr int kJpThreads = 256;

__device__ __forceinline__ int32_t jp_find(int32_t *parent, int32_t x) {
    int32_t cur = __ldcg(parent + x);
    if (cur != x) {
        int32_t prev = x, next;
        while (cur > (next = __ldcg(parent + cur))) {
            __stcg(parent + prev, next);  // path halving: an ancestor, so still <= prev
            prev = cur;
            cur = next;
        }
    }
    return cur;
}

__device__ __forceinline__ void jp_unite(int32_t *parent, int32_t u, int32_t v) {
    int32_t a = jp_find(parent, u), b = jp_find(parent, v);
    while (a != b) {
        const int32_t big = a > b ? a : b, small = a > b ? b : a;
        const int32_t old = atomicCAS(parent + big, big, small);
        if (old == big) return;
        // `big` was hooked by another union meanwhile: continue from its new root
        a = jp_find(parent, old);
        b = jp_find(parent, small);
    }
}

struct JpTest {
    int32_t est;
    double tau;
    int32_t bstar;  // Bloom AND: keep iff count >= bstar
    double b;       // Bloom L divisor
    double k;       // k-Hash / literal 1-Hash K
};

__device__ __forceinline__ bool jp_keep(const JpTest &t, int32_t c, int32_t aux, int32_t du, int32_t dv) {
    switch (t.est) {
        case PG_EST_EXACT: return (double)c > t.tau;
        case PG_EST_BF_AND: return c >= t.bstar;
        case PG_EST_BF_L: return (double)c / t.b > t.tau;
        default: {
            double K;
            double cc;
            if (t.est == PG_EST_KH) {
                K = t.k;
                cc = (double)c;
            } else if (t.est == PG_EST_1H) {
                K = (double)(aux & 0xFFFF);
                cc = (double)c;
            } else {  // PG_EST_1H_LITERAL
                K = t.k;
                cc = (double)((uint32_t)aux >> 16);
            }
            const double J = K > 0.0 ? cc / K : 0.0;
            const double s = (double)du + (double)dv;
            return J / (1.0 + J) * s > t.tau;
        }
    }
}

__global__ void __launch_bounds__(kJpThreads) k_jp_init(int32_t *parent, int32_t n, unsigned long long *counters) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        parent[v] = (int32_t)v;
    if (blockIdx.x == 0 && threadIdx.x < 2) counters[threadIdx.x] = 0ull;
}

// count / aux are in the edge list's order (entry e is (eu[e], ev[e])).
__global__ void __launch_bounds__(kJpThreads) k_jp_union(EdgeIndex ix, int32_t n,
                                                         const int32_t *__restrict__ count,
                                                         const int32_t *__restrict__ aux, JpTest t, int32_t *parent,
                                                         unsigned long long *kept) {
    int64_t m = ix.upper_off[n];
    if (m > ix.cap) m = ix.cap;
    uint32_t mine = 0;
    const bool need_deg = t.est != PG_EST_EXACT && t.est != PG_EST_BF_AND && t.est != PG_EST_BF_L;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t c = __ldg(count + e);
        const int32_t a = aux ? __ldg(aux + e) : 0;
        const int32_t u = __ldg(ix.eu + e), v = __ldg(ix.ev + e);
        const int32_t ds = need_deg ? __ldg(ix.eds + e) : 0;  // the MinHash tests use d_u + d_v only
        if (jp_keep(t, c, a, ds, 0)) {
            jp_unite(parent, u, v);
            ++mine;
        }
    }
    for (int o = 16; o > 0; o >>= 1) mine += __shfl_xor_sync(0xffffffffu, mine, o);
    if ((threadIdx.x & 31) == 0 && mine) atomicAdd(kept, (unsigned long long)mine);
}

// Root of x without path halving: the walk only reads.
__device__ __forceinline__ int32_t jp_root(const int32_t *parent, int32_t x) {
    int32_t next;
    while ((next = __ldcg(parent + x)) < x) x = next;
    return x;
}

// After the unions: every vertex's label is its root (the smallest id of its
// cluster), and the roots are counted. The walks only read and the only
// stores are final roots, so a walk that meets an already relabelled vertex
// still ends at the same root. (Path halving here could overwrite a stored
// root with an older, non-root ancestor read before that store.)
__global__ void __launch_bounds__(kJpThreads) k_jp_labels(int32_t *parent, int32_t n, unsigned long long *roots) {
    uint32_t mine = 0;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const int32_t r = jp_root(parent, (int32_t)v);
        __stcg(parent + v, r);
        mine += r == (int32_t)v;
    }
    for (int o = 16; o > 0; o >>= 1) mine += __shfl_xor_sync(0xffffffffu, mine, o);
    if ((threadIdx.x & 31) == 0 && mine) atomicAdd(roots, (unsigned long long)mine);
}

__global__ void k_jp_result(const unsigned long long *counters, const EdgeIndex ix, int32_t n, pg_jp_result *out) {
    int64_t m = ix.upper_off[n];
    if (m > ix.cap) m = ix.cap;
    out->clusters = (int64_t)counters[1];
    out->kept = (int64_t)counters[0];
    out->edges = m;
    out->reserved = 0;
}

int grid_for(int64_t items) {
    int64_t g = (items + kJpThreads - 1) / kJpThreads;
    const int64_t cap = 8LL * device_info().sm_count;
    if (g > cap) g = cap;
    return (int)(g < 1 ? 1 : g);
}

// Smallest count j in [0, l] whose AND estimate exceeds tau (l + 1 if none),
// in the oracle's double arithmetic: -(l / b) * log(1 - j~ / l), j~ = j - [j = l].
int32_t and_threshold(uint32_t l, uint32_t b, double tau) {
    for (uint32_t j = 0; j <= l; ++j) {
        const double o = (j == l) ? (double)j - 1.0 : (double)j;
        const double e = -((double)l / (double)b) * std::log(1.0 - o / (double)l);
        if (e > tau) return (int32_t)j;
    }
    return (int32_t)l + 1;
}

struct JpLayout {
    size_t table, count, aux, parent, counters, total;
};
JpLayout jp_layout(const pg_csr *g, const pg_sketch *sk, int32_t est) {
    JpLayout L{};
    size_t o = 0;
    auto take = [&](size_t b) {
        const size_t at = o;
        o += round_up(b ? b : 1, 256);
        return at;
    };
    const int64_t cap = g->nnz / 2 + 1;
    L.table = take(est == PG_EST_EXACT || !sk ? 0 : intersect_table_bytes(sk->kind, sk->bits, sk->k));
    L.count = take(4 * (size_t)cap);
    L.aux = take(est == PG_EST_1H || est == PG_EST_1H_LITERAL ? 4 * (size_t)cap : 0);
    L.parent = take(4 * ((size_t)g->n + 1));
    L.counters = take(16);
    L.total = o;
    return L;
}

}  // namespace
}  // namespace pg

using namespace pg;

extern "C" {

size_t pg_jarvis_patrick_workspace_bytes(const pg_csr *g, const pg_sketch *sk, int32_t estimator) {
    if (!g || g->n < 0 || g->nnz < 0) return 0;
    return jp_layout(g, sk, estimator).total;
}

pg_status pg_jarvis_patrick(const pg_csr *g, const void *index, const pg_sketch *sk, int32_t estimator, double tau,
                            void *workspace, size_t workspace_bytes, int32_t *labels, pg_jp_result *out,
                            pg_stream_t stream) {
    PG_TRACE("pg_jarvis_patrick");
    pg_status st = check_graph(g);
    if (st) return st;
    PG_REQUIRE(estimator >= PG_EST_EXACT && estimator <= PG_EST_1H_LITERAL, PG_ERR_INVALID_ARG,
               "pg_jarvis_patrick: unknown estimator %d", estimator);
    if (estimator != PG_EST_EXACT) {
        PG_REQUIRE(sk != nullptr, PG_ERR_INVALID_ARG, "pg_jarvis_patrick: estimator %d needs a sketch", estimator);
        st = check_estimator(sk, estimator);
        if (st) return st;
        st = check_sketch(g, sk);
        if (st) return st;
    }
    PG_REQUIRE(!std::isnan(tau), PG_ERR_INVALID_ARG, "pg_jarvis_patrick: tau is NaN");
    PG_REQUIRE(index != nullptr && aligned16(index), PG_ERR_INVALID_ARG,
               "pg_jarvis_patrick: edge index must be a 16-byte aligned device buffer");
    PG_REQUIRE(out != nullptr && (reinterpret_cast<uintptr_t>(out) & 7u) == 0, PG_ERR_INVALID_ARG,
               "pg_jarvis_patrick: out must be an 8-byte aligned device pg_jp_result");
    PG_REQUIRE(labels == nullptr || (reinterpret_cast<uintptr_t>(labels) & 3u) == 0, PG_ERR_INVALID_ARG,
               "pg_jarvis_patrick: misaligned labels");
    const JpLayout L = jp_layout(g, sk, estimator);
    PG_REQUIRE(workspace && aligned16(workspace) && workspace_bytes >= L.total, PG_ERR_NO_MEMORY,
               "pg_jarvis_patrick: workspace has %zu bytes, needs %zu", workspace_bytes, L.total);
    uint8_t *w = static_cast<uint8_t *>(workspace);
    int32_t *count = reinterpret_cast<int32_t *>(w + L.count);
    int32_t *aux = (estimator == PG_EST_1H || estimator == PG_EST_1H_LITERAL)
                       ? reinterpret_cast<int32_t *>(w + L.aux)
                       : nullptr;
    int32_t *parent = labels ? labels : reinterpret_cast<int32_t *>(w + L.parent);
    unsigned long long *counters = reinterpret_cast<unsigned long long *>(w + L.counters);
    const EdgeIndex ix = edge_index_view(index, g->n, g->nnz);
    cudaStream_t s = stream;

    k_jp_init<<<grid_for(g->n), kJpThreads, 0, s>>>(parent, g->n, counters);
    note_launch();
    PG_TRY_CUDA(cudaGetLastError(), "pg_jarvis_patrick: init");
    EdgeOutputs eo{};
    eo.count = count;
    eo.aux = aux;
    eo.list_order = true;  // k_jp_union walks the list itself
    if (estimator == PG_EST_EXACT) {
        PG_TRY_CUDA(launch_exact_pairs(g->row_ptr, g->col, g->n, ix, nullptr, 0, eo, s), "pg_jarvis_patrick: counts");
    } else {
        PG_TRY_CUDA(launch_intersect_ws(g->row_ptr, g->col, g->n, ix, nullptr, 0, *sk, estimator, eo,
                                        reinterpret_cast<double *>(w + L.table), s),
                    "pg_jarvis_patrick: counts");
    }
    JpTest t{};
    t.est = estimator;
    t.tau = tau;
    t.bstar = estimator == PG_EST_BF_AND ? and_threshold(sk->bits, sk->b, tau) : 0;
    t.b = sk ? (double)sk->b : 1.0;
    t.k = sk ? (double)sk->k : 0.0;
    if (g->n > 0) {
        k_jp_union<<<grid_for(g->nnz / 2 + 1), kJpThreads, 0, s>>>(ix, g->n, count, aux, t, parent, counters);
        k_jp_labels<<<grid_for(g->n), kJpThreads, 0, s>>>(parent, g->n, counters + 1);
        note_launch(2);
    }
    k_jp_result<<<1, 1, 0, s>>>(counters, ix, g->n, out);
    note_launch();
    PG_TRY_CUDA(cudaGetLastError(), "pg_jarvis_patrick");
    return PG_OK;
}

}  // extern "C"

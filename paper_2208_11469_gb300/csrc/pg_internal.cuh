// Internal declarations shared by the CUDA translation units of libpg.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include "../../include/pg.h"

namespace pg {

// ------------------------------------------------------------ error helpers
pg_status set_error(pg_status st, const char *fmt, ...);
pg_status cuda_status(cudaError_t e, const char *what);
#define PG_TRY_CUDA(expr, what)                                                   \
    do {                                                                          \
        cudaError_t _e = (expr);                                                  \
        if (_e != cudaSuccess) return ::pg::cuda_status(_e, what);                \
    } while (0)
#define PG_CHECK_LAUNCH(what) PG_TRY_CUDA(cudaGetLastError(), what)
#define PG_REQUIRE(cond, st, ...)                                                 \
    do {                                                                          \
        if (!(cond)) return ::pg::set_error(st, __VA_ARGS__);                     \
    } while (0)

// NVTX range around an entry point (visible in Nsight tools; no cost when no
// tool is attached).
struct TraceRange {
    explicit TraceRange(const char *name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange &) = delete;
    TraceRange &operator=(const TraceRange &) = delete;
};
#define PG_TRACE(name) ::pg::TraceRange pg_trace_range_(name)

// Argument checks shared by the entry points (pg_api.cu).
pg_status check_graph(const pg_csr *g);
pg_status check_sketch(const pg_csr *g, const pg_sketch *sk);
pg_status check_estimator(const pg_sketch *sk, int32_t est);

struct DeviceInfo {
    int sm_count;
    int max_threads_per_sm;
};
const DeviceInfo &device_info();

// Process-wide count of kernels this library has enqueued (pg_kernel_launches).
void note_launch(int count = 1);

inline bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }
inline size_t round_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// ------------------------------------------------------- device primitives
// MurmurHash3's 32-bit finaliser (two multiply / xor-shift rounds).
__device__ __forceinline__ uint32_t fmix32(uint32_t h) {
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
}
// Seed of hash function i.
__device__ __forceinline__ uint32_t hash_seed(uint32_t seed, uint32_t i) {
    return fmix32(seed + i * 0x9E3779B9u);
}
// The first xor-shift round of fmix32 is linear over XOR, so
// fmix32(x ^ s) = tail(pre(x) ^ pre(s)) with pre(y) = y ^ (y >> 16).
// Hoisting pre(x) out of a loop over hash functions saves two operations
// per hash without changing any value.
__device__ __forceinline__ uint32_t fmix_pre(uint32_t y) { return y ^ (y >> 16); }
__device__ __forceinline__ uint32_t fmix_tail(uint32_t h) {
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
}
// h_i(x) given pre(s_i).
__device__ __forceinline__ uint32_t hash_pre(uint32_t pre_x, uint32_t pre_s) {
    return fmix_tail(pre_x ^ pre_s);
}
// Position of hash h in an l-bit filter: floor(h * l / 2^32).
__device__ __forceinline__ uint32_t bit_pos(uint32_t h, uint32_t l) { return __umulhi(h, l); }

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

// Per-vertex sums avoid double-precision arithmetic on the hot path (double
// throughput is a small fraction of the integer and float pipes on this GPU):
// an estimate is carried as the exact integer V = round(value * 2^kFixBits)
// (the uint64 column of the estimator tables), summed with integer adds, and
// turned into a double by integer bit manipulation.
constexpr int kFixBits = 42;
// x * 2^-frac as a double, truncated to 53 significant bits (within 2^-52
// relative); no floating-point instruction.
__device__ __forceinline__ double fixed_to_f64(unsigned long long x, int frac) {
    if (x == 0ull) return 0.0;
    const int e = 63 - __clzll((long long)x);  // position of the leading one
    const unsigned long long mant = e >= 52 ? (x >> (e - 52)) : (x << (52 - e));
    const unsigned long long bits = ((unsigned long long)(e - frac + 1023) << 52) | (mant & 0xFFFFFFFFFFFFFull);
    return __longlong_as_double((long long)bits);
}

// ------------------------------------------------------------ launchers
// Defined in pg_index.cu
void launch_fill_u64(uint64_t *p, size_t count, uint64_t value, cudaStream_t s);
void launch_fill_f64(double *p, size_t count, double value, cudaStream_t s);
// View of an upper-edge index buffer (pg_build_edge_index).
// The upper edges as the passes stream them: grouped by the block of v
// (2^shift vertex ids per block), each group in upper-edge order.
struct EdgeIndex {
    const int32_t *upper_off;  // [n+1]
    const int32_t *eu;         // [cap] u of list entry i
    const int32_t *ev;         // [cap] v of list entry i
    const int32_t *eds;        // [cap] degree sum d_u + d_v of list entry i
    const int32_t *goff;       // [groups][n+1]: group j's entries of row u are [goff_j[u], goff_j[u+1])
    const int32_t *seg_end;    // [groups][n]: CSR position one past row u's entries in group j
    int64_t cap;               // list capacity; edges read = min(upper_off[n], cap)
    int32_t shift;             // vertex group = id >> shift
    int32_t groups;            // at most kMaxGroups
};
constexpr int32_t kMaxGroups = 8;
// Upper-edge index (per-edge output position) of list entry e = (u, v) of group j.
__device__ __forceinline__ int64_t upper_pos(const int32_t *row_ptr, int32_t n, const int32_t *upper_off,
                                             const int32_t *goff, const int32_t *seg_end, int32_t j, int32_t u,
                                             int64_t e) {
    const int64_t gs = (int64_t)n + 1;
    const int64_t pos = (int64_t)__ldg(seg_end + (int64_t)j * n + u) - ((int64_t)__ldg(goff + (int64_t)j * gs + u + 1) - e);
    return (int64_t)__ldg(upper_off + u + 1) - ((int64_t)__ldg(row_ptr + u + 1) - pos);
}
// Group of list entry e (the last j with goff_j[0] <= e).
__device__ __forceinline__ int32_t list_group(const int32_t *goff, int32_t n, int32_t groups, int64_t e) {
    int32_t j = 0;
    for (int32_t t = 1; t < groups; ++t)
        if ((int64_t)__ldg(goff + (int64_t)t * ((int64_t)n + 1)) <= e) j = t;
    return j;
}
int32_t group_shift(int32_t n);
size_t upper_index_bytes(int32_t n, int64_t nnz);
EdgeIndex edge_index_view(const void *index, int32_t n, int64_t nnz);
size_t scan_scratch_bytes(int64_t count);
// In-place exclusive prefix sum of count int32 values (scratch: scan_scratch_bytes).
cudaError_t launch_exclusive_scan(int32_t *data, int64_t count, int32_t *scratch, cudaStream_t s);
cudaError_t launch_upper_index(const int32_t *row_ptr, const int32_t *col, int32_t n, int64_t nnz,
                               void *index, cudaStream_t s);
cudaError_t launch_validate(const int32_t *row_ptr, const int32_t *col, int32_t n, int64_t nnz,
                            int check_symmetry, int64_t *result, cudaStream_t s);

// Per-vertex parameters of batched graphs (pg_batch.cu): global vertex of local
// vertex v = v_base + v, its graph gid[.], the graph's first global id voff[g]
// and hash count b_of[g]. gid == nullptr: a single graph. A batched build
// launch covers whole graphs of one bucket, so b_of[g] equals the launch's b
// for every graph in it (launch_build_bloom relies on this).
struct BatchMap {
    const int32_t *gid;
    const int32_t *voff;
    const uint8_t *b_of;
    int64_t v_base;
};

// Defined in pg_sketch.cu. hub_base: build workspace (build_workspace_bytes).
size_t build_workspace_bytes(int64_t nnz);
cudaError_t launch_build_bloom(const int32_t *row_ptr, const int32_t *col, int32_t n,
                               uint32_t l, uint32_t b, uint32_t seed, uint8_t *data,
                               int64_t stride, int32_t *hub_base, cudaStream_t s,
                               const BatchMap *bmap = nullptr);
cudaError_t launch_build_khash(const int32_t *row_ptr, const int32_t *col, int32_t n, uint32_t k,
                               uint32_t seed, uint8_t *data, int64_t stride, int32_t *hub_base,
                               cudaStream_t s);
cudaError_t launch_build_1hash(const int32_t *row_ptr, const int32_t *col, int32_t n, uint32_t k,
                               uint32_t seed, uint8_t *data, int64_t stride, int32_t *hub_base,
                               cudaStream_t s);

// Defined in pg_intersect.cu
struct EdgeOutputs {
    double *S;          // [n] sum over incident edges of the estimate (zeroed by caller) or null
    float *cn;          // per edge/pair
    float *jac;         // per edge/pair
    float *ovl;         // per edge/pair: overlap similarity
    float *tot;         // per edge/pair: total-neighbour similarity
    int32_t *count;     // per edge/pair
    int32_t *aux;       // per edge/pair (1-Hash)
    uint64_t *hist;     // [bins] (zeroed by caller) or null
    bool list_order;    // per-edge outputs in the edge list's own order (internal), not upper-edge order
    int32_t u_begin = 0;  // edge source: only the edges (u, v) with u_begin <= u < u_end
    int32_t u_end = -1;   // -1: every vertex
};
// Histogram bins of a pass: Bloom l + 1 (plus one for the OR estimator's
// degree sum), k-Hash 2 (k + 1), 1-Hash 2 (k + 1)^2 + 2 (k + 1) (plus two for the KMV sum).
int64_t hist_bins(int32_t kind, uint32_t l, uint32_t k, int32_t estimator);
size_t intersect_table_bytes(int32_t kind, uint32_t l, uint32_t k);
// Enqueue the estimator-table kernel (into table_ws) and the intersection
// kernel over every upper edge (pairs == nullptr) or over P pairs.
cudaError_t launch_intersect_ws(const int32_t *row_ptr, const int32_t *col, int32_t n,
                                const EdgeIndex &ix, const int32_t *pairs, int64_t P,
                                const pg_sketch &sk, int32_t estimator, const EdgeOutputs &out,
                                double *table_ws, cudaStream_t s);
cudaError_t launch_tc_finalize(const uint64_t *hist, const pg_sketch &sk, int32_t estimator,
                               pg_tc_result *out, cudaStream_t s);
// The estimator table of (kind, estimator, l, b, k) into table_ws
// (intersect_table_bytes): double [len] | uint64 fixed point [len] | float [len],
// indexed by the integer count (k-Hash: c / (k + c), scaled by d_u + d_v by the user).
cudaError_t launch_estimator_table(double *table_ws, int32_t kind, int32_t estimator, uint32_t l, uint32_t b,
                                   uint32_t k, cudaStream_t s);
cudaError_t launch_batch_finalize(const uint64_t *hist, const int64_t *hoff, const uint32_t *bits_of,
                                  const uint8_t *b_of, int32_t graphs, int32_t estimator, pg_tc_result *out,
                                  cudaStream_t s);
cudaError_t launch_lcc_finalize(const int32_t *row_ptr, int32_t n, double *S, float *lcc,
                                double *tri, cudaStream_t s);

// Defined in pg_exact.cu
size_t exact_workspace_bytes(int32_t n, int64_t nnz);
// Exact triangle count and per-vertex S_v = 2 * (triangles at v) by
// degree-ordered node iteration. S: DEVICE double [n] zeroed by the caller,
// or null. tc: DEVICE pg_tc_result or null.
cudaError_t launch_exact_tc(const int32_t *row_ptr, const int32_t *col, int32_t n, int64_t nnz,
                            const int32_t *upper_off, void *ws, double *S, pg_tc_result *tc,
                            cudaStream_t s);
// Degree orientation N+_v = {u in N_v : (d_u, u) > (d_v, v)} as a CSR, built
// in an exact_workspace_bytes(n, nnz) workspace; the lists keep increasing
// id order. *plus_off / *plus_col point into ws.
cudaError_t launch_orient(const int32_t *row_ptr, const int32_t *col, int32_t n, int64_t nnz, void *ws,
                          int32_t **plus_off, int32_t **plus_col, cudaStream_t s);
// Exact |N_u ∩ N_v| per upper edge (pairs == nullptr) or per pair, into
// out.count / out.cn / out.jac.
cudaError_t launch_exact_pairs(const int32_t *row_ptr, const int32_t *col, int32_t n,
                               const EdgeIndex &ix, const int32_t *pairs, int64_t P,
                               const EdgeOutputs &out, cudaStream_t s);

}  // namespace pg

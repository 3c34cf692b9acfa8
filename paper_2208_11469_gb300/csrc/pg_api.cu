// The C ABI of include/pg.h: argument checks, workspace carving, launches.
#include <algorithm>
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include "pg_internal.cuh"

namespace pg {

static thread_local char g_err[512] = "";
static std::atomic<uint64_t> g_launches{0};

void note_launch(int count) { g_launches.fetch_add((uint64_t)count, std::memory_order_relaxed); }

pg_status set_error(pg_status st, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return st;
}

pg_status cuda_status(cudaError_t e, const char *what) {
    snprintf(g_err, sizeof(g_err), "%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
    return PG_ERR_CUDA;
}

const DeviceInfo &device_info() {
    static std::mutex mu;
    static DeviceInfo cache[64];
    static bool have[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    std::lock_guard<std::mutex> lock(mu);
    if (!have[dev]) {
        int sms = 0, thr = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaDeviceGetAttribute(&thr, cudaDevAttrMaxThreadsPerMultiProcessor, dev);
        cache[dev].sm_count = sms > 0 ? sms : 1;
        cache[dev].max_threads_per_sm = thr > 0 ? thr : 2048;
        have[dev] = true;
    }
    return cache[dev];
}

pg_status check_graph(const pg_csr *g) {
    PG_REQUIRE(g != nullptr, PG_ERR_INVALID_ARG, "graph is NULL");
    PG_REQUIRE(g->n >= 0, PG_ERR_INVALID_ARG, "n = %d is negative", g->n);
    PG_REQUIRE(g->nnz >= 0, PG_ERR_INVALID_ARG, "nnz = %lld is negative", (long long)g->nnz);
    PG_REQUIRE(g->nnz < (int64_t(1) << 31), PG_ERR_TOO_LARGE, "nnz = %lld does not fit int32 CSR",
               (long long)g->nnz);
    PG_REQUIRE(g->row_ptr != nullptr, PG_ERR_INVALID_ARG, "row_ptr is NULL");
    PG_REQUIRE(g->nnz == 0 || g->col != nullptr, PG_ERR_INVALID_ARG, "col is NULL");
    PG_REQUIRE((reinterpret_cast<uintptr_t>(g->row_ptr) & 3u) == 0 &&
                   (reinterpret_cast<uintptr_t>(g->col) & 3u) == 0,
               PG_ERR_INVALID_ARG, "row_ptr/col must be 4-byte aligned");
    return PG_OK;
}

int64_t payload_bytes(const pg_sketch *sk) {
    return sk->kind == PG_SK_BLOOM ? (int64_t)sk->bits / 8 : 4 * (int64_t)sk->k;
}

pg_status check_sketch(const pg_csr *g, const pg_sketch *sk) {
    PG_REQUIRE(sk != nullptr, PG_ERR_INVALID_ARG, "sketch is NULL");
    PG_REQUIRE(sk->kind == PG_SK_BLOOM || sk->kind == PG_SK_KHASH || sk->kind == PG_SK_1HASH,
               PG_ERR_INVALID_ARG, "unknown sketch kind %d", sk->kind);
    PG_REQUIRE(sk->n == g->n, PG_ERR_INVALID_ARG, "sketch has %d rows, graph %d vertices", sk->n, g->n);
    if (sk->kind == PG_SK_BLOOM) {
        PG_REQUIRE(sk->bits >= 64 && sk->bits % 64 == 0, PG_ERR_INVALID_ARG,
                   "Bloom bits = %u must be a positive multiple of 64", sk->bits);
        PG_REQUIRE(sk->bits <= 1024, PG_ERR_UNSUPPORTED, "Bloom bits = %u > 1024", sk->bits);
        PG_REQUIRE(sk->b >= 1 && sk->b <= 16, PG_ERR_INVALID_ARG, "Bloom b = %u not in [1, 16]", sk->b);
    } else if (sk->kind == PG_SK_KHASH) {
        PG_REQUIRE(sk->k >= 1, PG_ERR_INVALID_ARG, "k must be >= 1");
        PG_REQUIRE(sk->k <= 256, PG_ERR_UNSUPPORTED, "k-Hash k = %u > 256", sk->k);
    } else {
        PG_REQUIRE(sk->k >= 1, PG_ERR_INVALID_ARG, "k must be >= 1");
        PG_REQUIRE(sk->k <= 32, PG_ERR_UNSUPPORTED, "1-Hash k = %u > 32", sk->k);
    }
    PG_REQUIRE(sk->stride_bytes % 16 == 0 && sk->stride_bytes >= payload_bytes(sk),
               PG_ERR_INVALID_ARG, "stride %lld must be a multiple of 16 and >= %lld",
               (long long)sk->stride_bytes, (long long)payload_bytes(sk));
    PG_REQUIRE(sk->stride_bytes <= 1024, PG_ERR_UNSUPPORTED, "stride %lld > 1024",
               (long long)sk->stride_bytes);
    PG_REQUIRE(g->n == 0 || sk->data != nullptr, PG_ERR_INVALID_ARG, "sketch data is NULL");
    PG_REQUIRE(aligned16(sk->data), PG_ERR_INVALID_ARG, "sketch data must be 16-byte aligned");
    return PG_OK;
}

pg_status check_estimator(const pg_sketch *sk, int32_t est) {
    switch (est) {
        case PG_EST_EXACT: return PG_OK;
        case PG_EST_BF_AND:
        case PG_EST_BF_L:
        case PG_EST_BF_OR:
        case PG_EST_BF_SS:
            PG_REQUIRE(sk && sk->kind == PG_SK_BLOOM, PG_ERR_INVALID_ARG,
                       "estimator %d needs a Bloom sketch", est);
            return PG_OK;
        case PG_EST_KH:
            PG_REQUIRE(sk && sk->kind == PG_SK_KHASH, PG_ERR_INVALID_ARG,
                       "estimator %d needs a k-Hash sketch", est);
            return PG_OK;
        case PG_EST_1H:
        case PG_EST_1H_LITERAL:
        case PG_EST_1H_KMV:
            PG_REQUIRE(sk && sk->kind == PG_SK_1HASH, PG_ERR_INVALID_ARG,
                       "estimator %d needs a 1-Hash sketch", est);
            return PG_OK;
        default: return set_error(PG_ERR_INVALID_ARG, "unknown estimator %d", est);
    }
}

namespace {

// Workspace layout of the analysis calls:
//   [estimator table][histogram][S: n doubles][exact path scratch]
struct Workspace {
    double *table;
    uint64_t *hist;
    double *S;
    void *exact;
    size_t total;
};

Workspace carve(const pg_csr *g, const pg_sketch *sk, int32_t est, void *base) {
    Workspace w{};
    uint8_t *p = static_cast<uint8_t *>(base);
    size_t off = 0;
    if (est != PG_EST_EXACT && sk) {
        w.table = reinterpret_cast<double *>(p + off);
        off += intersect_table_bytes(sk->kind, sk->bits, sk->k);
        w.hist = reinterpret_cast<uint64_t *>(p + off);
        off += round_up(8 * (size_t)hist_bins(sk->kind, sk->bits, sk->k, est), 256);
    }
    w.S = reinterpret_cast<double *>(p + off);
    off += round_up(8 * (size_t)g->n + 8, 256);
    if (est == PG_EST_EXACT) {
        w.exact = p + off;
        off += exact_workspace_bytes(g->n, g->nnz);
    }
    w.total = off;
    return w;
}

pg_status common_checks(const pg_csr *g, const void *index, bool need_index, const pg_sketch *sk,
                        int32_t est, void *ws, size_t ws_bytes, Workspace *w) {
    pg_status st = check_graph(g);
    if (st) return st;
    st = check_estimator(sk, est);
    if (st) return st;
    if (est != PG_EST_EXACT) {
        st = check_sketch(g, sk);
        if (st) return st;
    }
    PG_REQUIRE(!need_index || index != nullptr, PG_ERR_INVALID_ARG, "edge index is NULL");
    PG_REQUIRE(index == nullptr || aligned16(index), PG_ERR_INVALID_ARG,
               "edge index must be 16-byte aligned");
    *w = carve(g, est == PG_EST_EXACT ? nullptr : sk, est, ws);
    PG_REQUIRE(ws != nullptr || w->total == 0, PG_ERR_INVALID_ARG, "workspace is NULL");
    PG_REQUIRE(aligned16(ws), PG_ERR_INVALID_ARG, "workspace must be 16-byte aligned");
    PG_REQUIRE(ws_bytes >= w->total, PG_ERR_NO_MEMORY, "workspace has %zu bytes, needs %zu",
               ws_bytes, w->total);
    return PG_OK;
}

}  // namespace
}  // namespace pg

using namespace pg;

extern "C" {

const char *pg_status_string(pg_status s) {
    switch (s) {
        case PG_OK: return "PG_OK";
        case PG_ERR_INVALID_ARG: return "PG_ERR_INVALID_ARG";
        case PG_ERR_INVALID_GRAPH: return "PG_ERR_INVALID_GRAPH";
        case PG_ERR_TOO_LARGE: return "PG_ERR_TOO_LARGE";
        case PG_ERR_NO_MEMORY: return "PG_ERR_NO_MEMORY";
        case PG_ERR_CUDA: return "PG_ERR_CUDA";
        case PG_ERR_TIMEOUT: return "PG_ERR_TIMEOUT";
        case PG_ERR_NOT_FOUND: return "PG_ERR_NOT_FOUND";
        case PG_ERR_BUSY: return "PG_ERR_BUSY";
        case PG_ERR_UNSUPPORTED: return "PG_ERR_UNSUPPORTED";
        case PG_ERR_CANCELLED: return "PG_ERR_CANCELLED";
        default: return "PG_ERR_UNKNOWN";
    }
}

const char *pg_last_error(void) { return g_err; }

int32_t pg_version(void) { return (1 << 16) | 0; }

uint64_t pg_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

pg_status pg_validate_csr(const pg_csr *g, int32_t check_symmetry, int64_t *result,
                          pg_stream_t stream) {
    PG_TRACE("pg_validate_csr");
    pg_status st = check_graph(g);
    if (st) return st;
    PG_REQUIRE(result != nullptr && (reinterpret_cast<uintptr_t>(result) & 7u) == 0,
               PG_ERR_INVALID_ARG, "result must be an 8-byte aligned device int64[2]");
    PG_TRY_CUDA(launch_validate(g->row_ptr, g->col, g->n, g->nnz, check_symmetry, result, stream),
                "pg_validate_csr");
    return PG_OK;
}

size_t pg_edge_index_bytes(int32_t n, int64_t nnz) {
    return (n < 0 || nnz < 0) ? 0 : upper_index_bytes(n, nnz);
}

const int32_t *pg_edge_index_upper_off(const void *index) {
    return static_cast<const int32_t *>(index);
}

pg_status pg_build_edge_index(const pg_csr *g, void *index, size_t index_bytes, pg_stream_t stream) {
    PG_TRACE("pg_build_edge_index");
    pg_status st = check_graph(g);
    if (st) return st;
    PG_REQUIRE(index != nullptr && aligned16(index), PG_ERR_INVALID_ARG,
               "index must be a 16-byte aligned device buffer");
    PG_REQUIRE(index_bytes >= upper_index_bytes(g->n, g->nnz), PG_ERR_NO_MEMORY,
               "index has %zu bytes, needs %zu", index_bytes, upper_index_bytes(g->n, g->nnz));
    PG_TRY_CUDA(launch_upper_index(g->row_ptr, g->col, g->n, g->nnz, index, stream),
                "pg_build_edge_index");
    return PG_OK;
}

int64_t pg_sketch_stride(int32_t kind, uint32_t bits, uint32_t k) {
    int64_t payload = kind == PG_SK_BLOOM ? (int64_t)bits / 8 : 4 * (int64_t)k;
    return (int64_t)round_up((size_t)(payload > 0 ? payload : 16), 16);
}

uint32_t pg_bloom_bits_for_budget(double s, int32_t n, int64_t nnz) {
    if (n <= 0 || !(s > 0.0)) return 64;
    const double csr_bytes = 4.0 * ((double)n + 1.0) + 4.0 * (double)nnz;
    double words = s * csr_bytes * 8.0 / (64.0 * (double)n);
    int64_t w = (int64_t)words;
    if (w < 1) w = 1;
    if (w > 16) w = 16;
    return (uint32_t)(64 * w);
}

size_t pg_build_workspace_bytes(const pg_csr *g) {
    if (!g || g->nnz < 0) return 0;
    return build_workspace_bytes(g->nnz);
}

static pg_status build_common(const pg_csr *g, const pg_sketch *sk, void *ws, size_t ws_bytes) {
    pg_status st = check_graph(g);
    if (st) return st;
    st = check_sketch(g, sk);
    if (st) return st;
    PG_REQUIRE(ws != nullptr && aligned16(ws), PG_ERR_INVALID_ARG,
               "build workspace must be a 16-byte aligned device buffer");
    PG_REQUIRE(ws_bytes >= build_workspace_bytes(g->nnz), PG_ERR_NO_MEMORY,
               "build workspace has %zu bytes, needs %zu", ws_bytes,
               build_workspace_bytes(g->nnz));
    return PG_OK;
}

pg_status pg_build_bloom(const pg_csr *g, const pg_sketch *sk, void *ws, size_t ws_bytes,
                         pg_stream_t stream) {
    PG_TRACE("pg_build_bloom");
    pg_status st = build_common(g, sk, ws, ws_bytes);
    if (st) return st;
    PG_REQUIRE(sk->kind == PG_SK_BLOOM, PG_ERR_INVALID_ARG, "pg_build_bloom needs kind PG_SK_BLOOM");
    PG_TRY_CUDA(launch_build_bloom(g->row_ptr, g->col, g->n, sk->bits, sk->b, sk->seed,
                                   static_cast<uint8_t *>(sk->data), sk->stride_bytes,
                                   static_cast<int32_t *>(ws), stream),
                "pg_build_bloom");
    return PG_OK;
}

pg_status pg_build_minhash(const pg_csr *g, const pg_sketch *sk, void *ws, size_t ws_bytes,
                           pg_stream_t stream) {
    PG_TRACE("pg_build_minhash");
    pg_status st = build_common(g, sk, ws, ws_bytes);
    if (st) return st;
    if (sk->kind == PG_SK_KHASH) {
        PG_TRY_CUDA(launch_build_khash(g->row_ptr, g->col, g->n, sk->k, sk->seed,
                                       static_cast<uint8_t *>(sk->data), sk->stride_bytes,
                                       static_cast<int32_t *>(ws), stream),
                    "pg_build_minhash");
    } else if (sk->kind == PG_SK_1HASH) {
        PG_TRY_CUDA(launch_build_1hash(g->row_ptr, g->col, g->n, sk->k, sk->seed,
                                       static_cast<uint8_t *>(sk->data), sk->stride_bytes,
                                       static_cast<int32_t *>(ws), stream),
                    "pg_build_minhash");
    } else {
        return set_error(PG_ERR_INVALID_ARG, "pg_build_minhash needs kind PG_SK_KHASH or PG_SK_1HASH");
    }
    return PG_OK;
}

pg_status pg_upload_build(const int32_t *host_row_ptr, const int32_t *host_col, const pg_csr *g,
                          const pg_sketch *sketches, int32_t count, void *ws, size_t ws_bytes,
                          int64_t chunk_entries, pg_stream_t copy_stream, pg_stream_t stream) {
    PG_TRACE("pg_upload_build");
    pg_status st = check_graph(g);
    if (st) return st;
    PG_REQUIRE(host_row_ptr != nullptr && (g->nnz == 0 || host_col != nullptr), PG_ERR_INVALID_ARG,
               "pg_upload_build: host CSR is NULL");
    PG_REQUIRE(count >= 0 && (count == 0 || sketches != nullptr), PG_ERR_INVALID_ARG,
               "pg_upload_build: bad sketch list");
    PG_REQUIRE(chunk_entries > 0, PG_ERR_INVALID_ARG, "pg_upload_build: chunk_entries must be positive");
    PG_REQUIRE(host_row_ptr[0] == 0 && (int64_t)host_row_ptr[g->n] == g->nnz, PG_ERR_INVALID_ARG,
               "pg_upload_build: host row_ptr must run from 0 to nnz");
    for (int32_t i = 0; i < count; ++i) {
        st = build_common(g, sketches + i, ws, ws_bytes);
        if (st) return st;
        PG_REQUIRE(sketches[i].kind == PG_SK_BLOOM || sketches[i].kind == PG_SK_KHASH ||
                       sketches[i].kind == PG_SK_1HASH,
                   PG_ERR_INVALID_ARG, "pg_upload_build: sketch %d has an unknown kind", i);
    }
    // the device CSR is this call's output (pg_csr holds it as const for the readers)
    int32_t *dst_rp = const_cast<int32_t *>(g->row_ptr);
    int32_t *dst_col = const_cast<int32_t *>(g->col);
    cudaStream_t cs = copy_stream, s = stream;
    cudaEvent_t ev_start = nullptr, ev_chunk = nullptr;
    PG_TRY_CUDA(cudaEventCreateWithFlags(&ev_start, cudaEventDisableTiming), "pg_upload_build: event");
    cudaError_t e = cudaEventCreateWithFlags(&ev_chunk, cudaEventDisableTiming);
    // the upload overwrites the device CSR: it starts after the work already on the compute stream
    if (e == cudaSuccess) e = cudaEventRecord(ev_start, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, ev_start, 0);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(dst_rp, host_row_ptr, 4 * ((size_t)g->n + 1), cudaMemcpyDefault, cs);
    int64_t copied = 0;  // col entries copied so far
    int32_t r0 = 0;
    while (e == cudaSuccess && (r0 < g->n || copied < g->nnz)) {
        // rows [r0, r1): as many whole rows as fit chunk_entries (at least one)
        int32_t r1 = g->n;
        if (r0 < g->n) {
            const int64_t target = (int64_t)host_row_ptr[r0] + chunk_entries;
            const int32_t *it = std::upper_bound(host_row_ptr + r0 + 1, host_row_ptr + g->n + 1, target,
                                                 [](int64_t t, int32_t x) { return t < (int64_t)x; });
            r1 = std::max<int32_t>(r0 + 1, (int32_t)(it - host_row_ptr) - 1);
            r1 = std::min<int32_t>(r1, g->n);
        }
        const int64_t end = std::min<int64_t>(g->nnz, std::max<int64_t>(copied, host_row_ptr[r1]));
        if (end > copied)
            e = cudaMemcpyAsync(dst_col + copied, host_col + copied, 4 * (size_t)(end - copied), cudaMemcpyDefault,
                                cs);
        copied = end;
        if (r1 == g->n) copied = g->nnz;  // non-monotone offsets: the last chunk takes the rest
        if (e == cudaSuccess && r1 == g->n && end < g->nnz)
            e = cudaMemcpyAsync(dst_col + end, host_col + end, 4 * (size_t)(g->nnz - end), cudaMemcpyDefault, cs);
        if (e == cudaSuccess) e = cudaEventRecord(ev_chunk, cs);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ev_chunk, 0);
        for (int32_t i = 0; e == cudaSuccess && i < count && r1 > r0; ++i) {
            const pg_sketch &sk = sketches[i];
            uint8_t *rows = static_cast<uint8_t *>(sk.data) + (int64_t)r0 * sk.stride_bytes;
            int32_t *hub = static_cast<int32_t *>(ws);
            if (sk.kind == PG_SK_BLOOM)
                e = launch_build_bloom(g->row_ptr + r0, g->col, r1 - r0, sk.bits, sk.b, sk.seed, rows,
                                       sk.stride_bytes, hub, s);
            else if (sk.kind == PG_SK_KHASH)
                e = launch_build_khash(g->row_ptr + r0, g->col, r1 - r0, sk.k, sk.seed, rows, sk.stride_bytes, hub,
                                       s);
            else
                e = launch_build_1hash(g->row_ptr + r0, g->col, r1 - r0, sk.k, sk.seed, rows, sk.stride_bytes, hub,
                                       s);
        }
        r0 = r1;
    }
    cudaEventDestroy(ev_start);
    if (ev_chunk) cudaEventDestroy(ev_chunk);
    PG_TRY_CUDA(e, "pg_upload_build");
    return PG_OK;
}

int64_t pg_hist_bins(const pg_sketch *sk, int32_t estimator) {
    if (!sk || estimator == PG_EST_EXACT) return 0;
    return hist_bins(sk->kind, sk->bits, sk->k, estimator);
}

size_t pg_workspace_bytes(const pg_csr *g, const pg_sketch *sk, int32_t estimator) {
    if (!g || g->n < 0 || g->nnz < 0) return 0;
    if (estimator != PG_EST_EXACT && !sk) return 0;
    return carve(g, estimator == PG_EST_EXACT ? nullptr : sk, estimator, nullptr).total;
}

pg_status pg_triangle_count(const pg_csr *g, const void *index, const pg_sketch *sk,
                            int32_t estimator, void *ws, size_t ws_bytes, pg_tc_result *out,
                            pg_stream_t stream) {
    PG_TRACE("pg_triangle_count");
    Workspace w;
    pg_status st = common_checks(g, index, true, sk, estimator, ws, ws_bytes, &w);
    if (st) return st;
    PG_REQUIRE(out != nullptr && (reinterpret_cast<uintptr_t>(out) & 7u) == 0, PG_ERR_INVALID_ARG,
               "out must be an 8-byte aligned device pg_tc_result");
    const EdgeIndex ix = edge_index_view(index, g->n, g->nnz);
    const int32_t *upper_off = ix.upper_off;
    if (estimator == PG_EST_EXACT) {
        PG_TRY_CUDA(launch_exact_tc(g->row_ptr, g->col, g->n, g->nnz, upper_off, w.exact, nullptr,
                                    out, stream),
                    "pg_triangle_count(exact)");
        return PG_OK;
    }
    const size_t bins = (size_t)hist_bins(sk->kind, sk->bits, sk->k, estimator);
    launch_fill_u64(w.hist, bins, 0, stream);
    EdgeOutputs eo{};
    eo.hist = w.hist;
    PG_TRY_CUDA(launch_intersect_ws(g->row_ptr, g->col, g->n, ix, nullptr, 0, *sk,
                                    estimator, eo, w.table, stream),
                "pg_triangle_count");
    PG_TRY_CUDA(launch_tc_finalize(w.hist, *sk, estimator, out, stream), "pg_triangle_count");
    return PG_OK;
}

pg_status pg_clustering(const pg_csr *g, const void *index, const pg_sketch *sk, int32_t estimator,
                        void *ws, size_t ws_bytes, float *lcc, double *tri, pg_tc_result *tc,
                        pg_stream_t stream) {
    PG_TRACE("pg_clustering");
    Workspace w;
    pg_status st = common_checks(g, index, true, sk, estimator, ws, ws_bytes, &w);
    if (st) return st;
    PG_REQUIRE(g->n == 0 || lcc != nullptr || tri != nullptr, PG_ERR_INVALID_ARG,
               "lcc and tri are both NULL");
    PG_REQUIRE((reinterpret_cast<uintptr_t>(tri) & 7u) == 0 &&
                   (reinterpret_cast<uintptr_t>(tc) & 7u) == 0 &&
                   (reinterpret_cast<uintptr_t>(lcc) & 3u) == 0,
               PG_ERR_INVALID_ARG, "misaligned output pointer");
    const EdgeIndex ix = edge_index_view(index, g->n, g->nnz);
    const int32_t *upper_off = ix.upper_off;
    double *S = tri ? tri : w.S;
    launch_fill_f64(S, (size_t)g->n, 0.0, stream);
    if (estimator == PG_EST_EXACT) {
        PG_TRY_CUDA(launch_exact_tc(g->row_ptr, g->col, g->n, g->nnz, upper_off, w.exact, S, tc,
                                    stream),
                    "pg_clustering(exact)");
    } else {
        EdgeOutputs eo{};
        eo.S = S;
        if (tc) {
            eo.hist = w.hist;
            launch_fill_u64(w.hist, (size_t)hist_bins(sk->kind, sk->bits, sk->k, estimator), 0, stream);
        }
        PG_TRY_CUDA(launch_intersect_ws(g->row_ptr, g->col, g->n, ix, nullptr, 0, *sk,
                                        estimator, eo, w.table, stream),
                    "pg_clustering");
        if (tc) PG_TRY_CUDA(launch_tc_finalize(w.hist, *sk, estimator, tc, stream), "pg_clustering");
    }
    PG_TRY_CUDA(launch_lcc_finalize(g->row_ptr, g->n, S, lcc, tri, stream), "pg_clustering");
    return PG_OK;
}

static pg_status pairs_common(const pg_csr *g, const void *index, const pg_sketch *sk,
                              int32_t estimator, const int32_t *pairs, int64_t P, void *ws,
                              size_t ws_bytes, Workspace *w) {
    pg_status st = common_checks(g, index, pairs == nullptr, sk, estimator, ws, ws_bytes, w);
    if (st) return st;
    if (pairs) {
        PG_REQUIRE(P >= 0, PG_ERR_INVALID_ARG, "P = %lld is negative", (long long)P);
        PG_REQUIRE((reinterpret_cast<uintptr_t>(pairs) & 7u) == 0, PG_ERR_INVALID_ARG,
                   "pairs must be 8-byte aligned");
    }
    return PG_OK;
}

pg_status pg_jaccard_pairs(const pg_csr *g, const void *index, const pg_sketch *sk,
                           int32_t estimator, const int32_t *pairs, int64_t P, void *ws,
                           size_t ws_bytes, float *cn, float *jac, pg_stream_t stream) {
    PG_TRACE("pg_jaccard_pairs");
    Workspace w;
    pg_status st = pairs_common(g, index, sk, estimator, pairs, P, ws, ws_bytes, &w);
    if (st) return st;
    EdgeOutputs eo{};
    eo.cn = cn;
    eo.jac = jac;
    const EdgeIndex ix = edge_index_view(index, g->n, g->nnz);
    if (estimator == PG_EST_EXACT) {
        PG_TRY_CUDA(launch_exact_pairs(g->row_ptr, g->col, g->n, ix, pairs, P, eo, stream),
                    "pg_jaccard_pairs(exact)");
    } else {
        PG_TRY_CUDA(launch_intersect_ws(g->row_ptr, g->col, g->n, ix, pairs, P, *sk,
                                        estimator, eo, w.table, stream),
                    "pg_jaccard_pairs");
    }
    return PG_OK;
}

pg_status pg_similarity_pairs(const pg_csr *g, const void *index, const pg_sketch *sk, int32_t estimator,
                              const int32_t *pairs, int64_t P, void *ws, size_t ws_bytes,
                              const pg_similarity *out, pg_stream_t stream) {
    PG_TRACE("pg_similarity_pairs");
    Workspace w;
    pg_status st = pairs_common(g, index, sk, estimator, pairs, P, ws, ws_bytes, &w);
    if (st) return st;
    PG_REQUIRE(out != nullptr, PG_ERR_INVALID_ARG, "pg_similarity_pairs: outputs is NULL");
    PG_REQUIRE(((reinterpret_cast<uintptr_t>(out->cn) | reinterpret_cast<uintptr_t>(out->jac) |
                 reinterpret_cast<uintptr_t>(out->overlap) | reinterpret_cast<uintptr_t>(out->total)) &
                3u) == 0,
               PG_ERR_INVALID_ARG, "misaligned output pointer");
    EdgeOutputs eo{};
    eo.cn = out->cn;
    eo.jac = out->jac;
    eo.ovl = out->overlap;
    eo.tot = out->total;
    const EdgeIndex ix = edge_index_view(index, g->n, g->nnz);
    if (estimator == PG_EST_EXACT) {
        PG_TRY_CUDA(launch_exact_pairs(g->row_ptr, g->col, g->n, ix, pairs, P, eo, stream),
                    "pg_similarity_pairs(exact)");
    } else {
        PG_TRY_CUDA(launch_intersect_ws(g->row_ptr, g->col, g->n, ix, pairs, P, *sk, estimator, eo, w.table,
                                        stream),
                    "pg_similarity_pairs");
    }
    return PG_OK;
}

pg_status pg_edge_counts(const pg_csr *g, const void *index, const pg_sketch *sk,
                         int32_t estimator, const int32_t *pairs, int64_t P, void *ws,
                         size_t ws_bytes, int32_t *count, int32_t *aux, uint64_t *hist,
                         pg_stream_t stream) {
    PG_TRACE("pg_edge_counts");
    Workspace w;
    pg_status st = pairs_common(g, index, sk, estimator, pairs, P, ws, ws_bytes, &w);
    if (st) return st;
    EdgeOutputs eo{};
    eo.count = count;
    const EdgeIndex ix = edge_index_view(index, g->n, g->nnz);
    if (estimator == PG_EST_EXACT) {
        PG_TRY_CUDA(launch_exact_pairs(g->row_ptr, g->col, g->n, ix, pairs, P, eo, stream),
                    "pg_edge_counts(exact)");
        return PG_OK;
    }
    eo.aux = aux;
    if (hist) {
        PG_REQUIRE((reinterpret_cast<uintptr_t>(hist) & 7u) == 0, PG_ERR_INVALID_ARG,
                   "hist must be 8-byte aligned");
        eo.hist = hist;
        launch_fill_u64(hist, (size_t)hist_bins(sk->kind, sk->bits, sk->k, estimator), 0, stream);
    }
    PG_TRY_CUDA(launch_intersect_ws(g->row_ptr, g->col, g->n, ix, pairs, P, *sk, estimator,
                                    eo, w.table, stream),
                "pg_edge_counts");
    return PG_OK;
}

pg_status pg_analyze(const pg_csr *g, const void *index, const pg_sketch *sk, int32_t estimator,
                     void *ws, size_t ws_bytes, const pg_outputs *out, pg_stream_t stream) {
    PG_TRACE("pg_analyze");
    Workspace w;
    pg_status st = common_checks(g, index, true, sk, estimator, ws, ws_bytes, &w);
    if (st) return st;
    PG_REQUIRE(out != nullptr, PG_ERR_INVALID_ARG, "outputs is NULL");
    PG_REQUIRE((reinterpret_cast<uintptr_t>(out->tri) & 7u) == 0 &&
                   (reinterpret_cast<uintptr_t>(out->tc) & 7u) == 0 &&
                   (reinterpret_cast<uintptr_t>(out->hist) & 7u) == 0 &&
                   (reinterpret_cast<uintptr_t>(out->lcc) & 3u) == 0 &&
                   (reinterpret_cast<uintptr_t>(out->edge_cn) & 3u) == 0 &&
                   (reinterpret_cast<uintptr_t>(out->edge_jac) & 3u) == 0 &&
                   (reinterpret_cast<uintptr_t>(out->edge_count) & 3u) == 0 &&
                   (reinterpret_cast<uintptr_t>(out->edge_aux) & 3u) == 0 &&
                   (reinterpret_cast<uintptr_t>(out->edge_overlap) & 3u) == 0 &&
                   (reinterpret_cast<uintptr_t>(out->edge_total) & 3u) == 0,
               PG_ERR_INVALID_ARG, "misaligned output pointer");
    const EdgeIndex ix = edge_index_view(index, g->n, g->nnz);
    const int32_t *upper_off = ix.upper_off;
    const bool want_vertex = out->lcc || out->tri;
    double *S = want_vertex ? (out->tri ? out->tri : w.S) : nullptr;
    if (S) launch_fill_f64(S, (size_t)g->n, 0.0, stream);
    if (estimator == PG_EST_EXACT) {
        if (S || out->tc)
            PG_TRY_CUDA(launch_exact_tc(g->row_ptr, g->col, g->n, g->nnz, upper_off, w.exact, S,
                                        out->tc, stream),
                        "pg_analyze(exact)");
        if (out->edge_cn || out->edge_jac || out->edge_count || out->edge_overlap || out->edge_total) {
            EdgeOutputs eo{};
            eo.cn = out->edge_cn;
            eo.jac = out->edge_jac;
            eo.ovl = out->edge_overlap;
            eo.tot = out->edge_total;
            eo.count = out->edge_count;
            PG_TRY_CUDA(launch_exact_pairs(g->row_ptr, g->col, g->n, ix, nullptr, 0, eo,
                                           stream),
                        "pg_analyze(exact)");
        }
    } else {
        EdgeOutputs eo{};
        eo.S = S;
        eo.cn = out->edge_cn;
        eo.jac = out->edge_jac;
        eo.ovl = out->edge_overlap;
        eo.tot = out->edge_total;
        eo.count = out->edge_count;
        eo.aux = out->edge_aux;
        uint64_t *hist = out->hist ? out->hist : (out->tc ? w.hist : nullptr);
        if (hist) {
            eo.hist = hist;
            launch_fill_u64(hist, (size_t)hist_bins(sk->kind, sk->bits, sk->k, estimator), 0, stream);
        }
        PG_TRY_CUDA(launch_intersect_ws(g->row_ptr, g->col, g->n, ix, nullptr, 0, *sk,
                                        estimator, eo, w.table, stream),
                    "pg_analyze");
        if (out->tc) PG_TRY_CUDA(launch_tc_finalize(hist, *sk, estimator, out->tc, stream), "pg_analyze");
    }
    if (S) PG_TRY_CUDA(launch_lcc_finalize(g->row_ptr, g->n, S, out->lcc, out->tri, stream), "pg_analyze");
    return PG_OK;
}

// --------------------------------------------------- vertex-partitioned runs
pg_status pg_partial_sums(const pg_csr *g, const void *index, const pg_sketch *sk, int32_t estimator,
                          int32_t u_begin, int32_t u_end, void *ws, size_t ws_bytes, double *sums, uint64_t *hist,
                          pg_stream_t stream) {
    PG_TRACE("pg_partial_sums");
    Workspace w;
    pg_status st = common_checks(g, index, true, sk, estimator, ws, ws_bytes, &w);
    if (st) return st;
    PG_REQUIRE(estimator != PG_EST_EXACT && sk != nullptr, PG_ERR_UNSUPPORTED,
               "pg_partial_sums: the exact count has no partial form here (use pg_analyze)");
    PG_REQUIRE(estimator != PG_EST_1H_KMV, PG_ERR_UNSUPPORTED,
               "pg_partial_sums: the KMV total carries a 128-bit sum that does not add word by word");
    PG_REQUIRE(u_begin >= 0 && u_begin <= u_end && u_end <= g->n, PG_ERR_INVALID_ARG,
               "pg_partial_sums: vertex range [%d, %d) outside [0, %d]", u_begin, u_end, g->n);
    PG_REQUIRE((reinterpret_cast<uintptr_t>(sums) & 7u) == 0 && (reinterpret_cast<uintptr_t>(hist) & 7u) == 0,
               PG_ERR_INVALID_ARG, "pg_partial_sums: misaligned output pointer");
    if (u_begin == u_end || (!sums && !hist)) return PG_OK;
    const EdgeIndex ix = edge_index_view(index, g->n, g->nnz);
    EdgeOutputs eo{};
    eo.S = sums;
    eo.hist = hist;
    eo.u_begin = u_begin;
    eo.u_end = u_end;
    PG_TRY_CUDA(launch_intersect_ws(g->row_ptr, g->col, g->n, ix, nullptr, 0, *sk, estimator, eo, w.table, stream),
                "pg_partial_sums");
    return PG_OK;
}

pg_status pg_finalize_sums(const pg_csr *g, const pg_sketch *sk, int32_t estimator, const uint64_t *hist,
                           double *sums, pg_tc_result *tc, float *lcc, double *tri, pg_stream_t stream) {
    PG_TRACE("pg_finalize_sums");
    PG_REQUIRE(g != nullptr && sk != nullptr, PG_ERR_INVALID_ARG, "pg_finalize_sums: graph or sketch is NULL");
    PG_REQUIRE(g->n >= 0 && (g->n == 0 || g->row_ptr != nullptr), PG_ERR_INVALID_ARG,
               "pg_finalize_sums: bad graph");
    PG_REQUIRE(estimator != PG_EST_EXACT && estimator != PG_EST_1H_KMV, PG_ERR_UNSUPPORTED,
               "pg_finalize_sums: estimator %d has no partial form", estimator);
    PG_REQUIRE(!tc || hist, PG_ERR_INVALID_ARG, "pg_finalize_sums: tc needs hist");
    PG_REQUIRE(!(lcc || tri) || sums, PG_ERR_INVALID_ARG, "pg_finalize_sums: lcc / tri need sums");
    if (tc) PG_TRY_CUDA(launch_tc_finalize(hist, *sk, estimator, tc, stream), "pg_finalize_sums");
    if (lcc || tri) PG_TRY_CUDA(launch_lcc_finalize(g->row_ptr, g->n, sums, lcc, tri, stream), "pg_finalize_sums");
    return PG_OK;
}

// ------------------------------------------------------------ sketch files
// A sketch file is a 64-byte header followed by the n rows of stride bytes,
// as they lie in device memory.
namespace {
struct SketchFileHeader {
    char magic[8];  // "PGSKTCH1"
    int32_t version;
    int32_t kind;
    uint32_t bits, b, k, seed;
    int32_t n;
    int32_t pad;
    int64_t stride;
    int64_t bytes;  // n * stride
    uint8_t reserved[8];
};
static_assert(sizeof(SketchFileHeader) == 64, "sketch file header is 64 bytes");
constexpr char kSketchMagic[8] = {'P', 'G', 'S', 'K', 'T', 'C', 'H', '1'};
constexpr size_t kFileChunk = 64u << 20;

pg_status read_header(const char *path, SketchFileHeader *h, FILE **fp) {
    PG_REQUIRE(path != nullptr, PG_ERR_INVALID_ARG, "sketch file path is NULL");
    FILE *f = std::fopen(path, "rb");
    PG_REQUIRE(f != nullptr, PG_ERR_NOT_FOUND, "cannot open sketch file %s", path);
    const bool ok = std::fread(h, sizeof(*h), 1, f) == 1 && std::memcmp(h->magic, kSketchMagic, 8) == 0 &&
                    h->version == 1 && h->n >= 0 && h->stride >= 0 && h->bytes == (int64_t)h->n * h->stride &&
                    (h->kind == PG_SK_BLOOM || h->kind == PG_SK_KHASH || h->kind == PG_SK_1HASH);
    if (!ok) {
        std::fclose(f);
        return set_error(PG_ERR_INVALID_ARG, "%s is not a sketch file (bad header)", path);
    }
    if (fp)
        *fp = f;
    else
        std::fclose(f);
    return PG_OK;
}
}  // namespace

pg_status pg_sketch_save(const pg_sketch *sk, const char *path, pg_stream_t stream) {
    PG_TRACE("pg_sketch_save");
    PG_REQUIRE(sk != nullptr && path != nullptr && (sk->n == 0 || sk->data != nullptr), PG_ERR_INVALID_ARG,
               "pg_sketch_save: NULL argument");
    PG_REQUIRE(sk->n >= 0 && sk->stride_bytes > 0, PG_ERR_INVALID_ARG, "pg_sketch_save: bad descriptor");
    SketchFileHeader h{};
    std::memcpy(h.magic, kSketchMagic, 8);
    h.version = 1;
    h.kind = sk->kind;
    h.bits = sk->bits;
    h.b = sk->b;
    h.k = sk->k;
    h.seed = sk->seed;
    h.n = sk->n;
    h.stride = sk->stride_bytes;
    h.bytes = (int64_t)sk->n * sk->stride_bytes;
    PG_TRY_CUDA(cudaStreamSynchronize(stream), "pg_sketch_save: stream");
    FILE *f = std::fopen(path, "wb");
    PG_REQUIRE(f != nullptr, PG_ERR_NOT_FOUND, "pg_sketch_save: cannot create %s", path);
    bool ok = std::fwrite(&h, sizeof(h), 1, f) == 1;
    std::vector<uint8_t> buf(ok && h.bytes ? std::min<size_t>(kFileChunk, (size_t)h.bytes) : 0);
    cudaError_t e = cudaSuccess;
    for (int64_t off = 0; ok && e == cudaSuccess && off < h.bytes; off += (int64_t)buf.size()) {
        const size_t len = std::min<size_t>(buf.size(), (size_t)(h.bytes - off));
        e = cudaMemcpy(buf.data(), static_cast<const uint8_t *>(sk->data) + off, len, cudaMemcpyDeviceToHost);
        ok = e == cudaSuccess && std::fwrite(buf.data(), 1, len, f) == len;
    }
    ok = (std::fclose(f) == 0) && ok;
    if (e != cudaSuccess) return cuda_status(e, "pg_sketch_save");
    PG_REQUIRE(ok, PG_ERR_INVALID_ARG, "pg_sketch_save: writing %s failed", path);
    return PG_OK;
}

pg_status pg_sketch_load_header(const char *path, pg_sketch *sk) {
    PG_REQUIRE(sk != nullptr, PG_ERR_INVALID_ARG, "pg_sketch_load_header: sketch is NULL");
    SketchFileHeader h{};
    pg_status st = read_header(path, &h, nullptr);
    if (st) return st;
    sk->kind = h.kind;
    sk->bits = h.bits;
    sk->b = h.b;
    sk->k = h.k;
    sk->seed = h.seed;
    sk->n = h.n;
    sk->stride_bytes = h.stride;
    return PG_OK;
}

pg_status pg_sketch_load(pg_sketch *sk, const char *path, pg_stream_t stream) {
    PG_TRACE("pg_sketch_load");
    PG_REQUIRE(sk != nullptr && (sk->n == 0 || sk->data != nullptr), PG_ERR_INVALID_ARG,
               "pg_sketch_load: NULL argument");
    SketchFileHeader h{};
    FILE *f = nullptr;
    pg_status st = read_header(path, &h, &f);
    if (st) return st;
    const bool same = h.kind == sk->kind && h.bits == sk->bits && h.b == sk->b && h.k == sk->k &&
                      h.seed == sk->seed && h.n == sk->n && h.stride == sk->stride_bytes;
    if (!same) {
        std::fclose(f);
        return set_error(PG_ERR_INVALID_ARG,
                         "pg_sketch_load: %s holds kind %d bits %u b %u k %u seed %u n %d stride %lld, the "
                         "descriptor differs",
                         path, h.kind, h.bits, h.b, h.k, h.seed, h.n, (long long)h.stride);
    }
    cudaError_t e = cudaStreamSynchronize(stream);
    std::vector<uint8_t> buf(h.bytes ? std::min<size_t>(kFileChunk, (size_t)h.bytes) : 0);
    bool ok = e == cudaSuccess;
    for (int64_t off = 0; ok && off < h.bytes; off += (int64_t)buf.size()) {
        const size_t len = std::min<size_t>(buf.size(), (size_t)(h.bytes - off));
        ok = std::fread(buf.data(), 1, len, f) == len;
        if (ok) {
            e = cudaMemcpy(static_cast<uint8_t *>(sk->data) + off, buf.data(), len, cudaMemcpyHostToDevice);
            ok = e == cudaSuccess;
        }
    }
    std::fclose(f);
    if (e != cudaSuccess) return cuda_status(e, "pg_sketch_load");
    PG_REQUIRE(ok, PG_ERR_INVALID_ARG, "pg_sketch_load: %s is truncated", path);
    return PG_OK;
}

}  // extern "C"

// pg_triangle_count_noalloc: the sketched triangle count for callers that
// cannot allocate device memory.
//
// pg_triangle_count needs a small scratch area (the estimator table and the
// integer histogram of per-edge counts) that the caller normally provides
// as a workspace. Some callers cannot provide one: a plugin running inside a
// host application whose own allocator has reserved the device memory, or a
// process whose policy forbids device allocation after start-up. For them
// this entry point keeps that scratch in a fixed array in the library's own
// device memory instead, so the call needs nothing from the caller beyond its
// inputs and the output.
//
// Limits and behaviour:
//   - The array is kNoallocScratchBytes (64 KiB) of static device memory. Every
//     GPU that loads the library holds it until the process exits.
//   - It covers every sketch configuration the library supports (largest:
//     1-Hash with k = 32 read by the KMV estimator, 22,016 table bytes plus
//     2,246 histogram words = 39,984 bytes, about 39 KiB; Bloom with l = 1024
//     and the OR estimator needs about 28 KiB); the exact estimator needs scratch
//     proportional to the graph and is rejected with PG_ERR_UNSUPPORTED.
//   - The first call on each device looks up the array's device address
//     (with that device current). Make that first call before any stream
//     capture begins.
//   - All calls on one device share the array. The histogram part is cleared
//     at the start of each call; the table part is rewritten by each call.
//     Calls that overlap on the GPU (different streams, or different host
//     threads without ordering) race on the array and give wrong results;
//     order them on one stream or synchronise between them.
#include <mutex>

#include "pg_internal.cuh"

namespace pg {
namespace {

constexpr size_t kNoallocScratchBytes = 64 * 1024;
constexpr int kMaxDevices = 64;

// The scratch itself. In host code `g_noalloc_scratch` is only a host-side
// stand-in for the symbol, never a device address: the address handed to
// kernels comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

std::mutex g_mu;
void *g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch on the current device, looked up once per device.
pg_status scratch_for_current_device(void **out) {
    int dev = 0;
    PG_TRY_CUDA(cudaGetDevice(&dev), "pg_triangle_count_noalloc: cudaGetDevice");
    PG_REQUIRE(dev >= 0 && dev < kMaxDevices, PG_ERR_UNSUPPORTED,
               "pg_triangle_count_noalloc: device ordinal %d >= %d", dev, kMaxDevices);
    std::lock_guard<std::mutex> lock(g_mu);
    if (g_scratch_ptr[dev] == nullptr) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_status(e, "pg_triangle_count_noalloc: cudaGetSymbolAddress");
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return PG_OK;
}

}  // namespace
}  // namespace pg

using namespace pg;

extern "C" pg_status pg_triangle_count_noalloc(const pg_csr *g, const void *index,
                                               const pg_sketch *sk, int32_t estimator,
                                               pg_tc_result *out, pg_stream_t stream) {
    pg_status st = check_graph(g);
    if (st) return st;
    PG_REQUIRE(estimator != PG_EST_EXACT, PG_ERR_UNSUPPORTED,
               "pg_triangle_count_noalloc: the exact estimator needs scratch proportional to the "
               "graph; use pg_triangle_count with a workspace");
    st = check_estimator(sk, estimator);
    if (st) return st;
    st = check_sketch(g, sk);
    if (st) return st;
    PG_REQUIRE(index != nullptr && aligned16(index), PG_ERR_INVALID_ARG,
               "pg_triangle_count_noalloc: edge index must be a 16-byte aligned device buffer");
    PG_REQUIRE(out != nullptr && (reinterpret_cast<uintptr_t>(out) & 7u) == 0, PG_ERR_INVALID_ARG,
               "pg_triangle_count_noalloc: out must be an 8-byte aligned device pg_tc_result");
    const size_t table = intersect_table_bytes(sk->kind, sk->bits, sk->k);
    const size_t bins = (size_t)hist_bins(sk->kind, sk->bits, sk->k, estimator);
    const size_t scratch = table + 8 * bins;
    PG_REQUIRE(scratch <= kNoallocScratchBytes, PG_ERR_TOO_LARGE,
               "pg_triangle_count_noalloc: this sketch needs %zu bytes of scratch, the static "
               "array holds %zu",
               scratch, kNoallocScratchBytes);
    void *base = nullptr;
    st = scratch_for_current_device(&base);
    if (st) return st;
    double *tab = static_cast<double *>(base);
    uint64_t *hist = reinterpret_cast<uint64_t *>(static_cast<unsigned char *>(base) + table);
    launch_fill_u64(hist, bins, 0, stream);
    EdgeOutputs eo{};
    eo.hist = hist;
    PG_TRY_CUDA(launch_intersect_ws(g->row_ptr, g->col, g->n, edge_index_view(index, g->n, g->nnz),
                                    nullptr, 0, *sk, estimator, eo, tab, stream),
                "pg_triangle_count_noalloc");
    PG_TRY_CUDA(launch_tc_finalize(hist, *sk, estimator, out, stream), "pg_triangle_count_noalloc");
    return PG_OK;
}

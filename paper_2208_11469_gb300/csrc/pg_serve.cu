// Serving: a request loop over one resident graph and its sketches
// (pg_server_*, pg_submit, pg_poll, pg_cancel).
//
// Requests are vertex-pair similarity queries (common-neighbour and Jaccard
// estimates of Sec. III / IV, as in link prediction) and triangle counts of
// induced subgraphs G[S] (the estimator of Sec. VII applied to G[S]).
//
// Design. A host scheduler thread admits queued requests in arrival order
// while the arena (caller-owned device memory) and the page-locked staging
// have room, and keeps the GPU fed:
//   - Pair requests are cut into tiles of kTile pairs. Each launch of
//     k_serve_pairs takes tiles round-robin from every admitted pair request,
//     up to iteration_pairs pairs, so requests that arrive while a launch runs
//     join the next one (continuous batching) and a small request is not
//     held behind a large one. Two launches can be in flight (double-buffered
//     tile descriptors); each pair is computed alone, so an answer does not
//     depend on the mix.
//   - A subgraph request runs a two-phase pipeline on one of several streams:
//     phase 1 marks S in a per-stream membership bitmap, counts the induced
//     degrees, scans them and writes the induced CSR with local ids (S sorted,
//     so the local CSR is sorted and deterministic), and copies |E(S)| back;
//     when that copy lands the scheduler sizes phase 2 exactly: the edge
//     index, the Bloom sketches of the induced neighbourhoods, the fused pass
//     and the triangle-count finalisation (or the exact count), with the
//     result copied back to the host.
// No kernel waits on the host or on another kernel: the scheduler polls CUDA
// events, and callers wait on the host with their own time limit (pg_poll).
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "pg_internal.cuh"

namespace pg {
namespace {

constexpr int32_t kTile = 1024;  // pairs per tile
constexpr int kServeThreads = 256;
constexpr int kChunksPerTile = kTile / 32;

struct PairTile {
    const int32_t *pairs;  // the request's pairs (device)
    float *cn;             // the request's outputs (device) or null
    float *jac;
    int32_t begin;         // first pair of this tile in the request
    int32_t count;         // pairs in this tile (<= kTile)
    int32_t est;           // PG_EST_BF_AND, PG_EST_BF_L or PG_EST_KH
    int32_t pad;
};

struct ServeSketches {
    const uint8_t *bf;  // Bloom rows or null
    int64_t bf_stride;
    uint32_t bf_l;
    const uint8_t *kh;  // k-Hash rows or null
    int64_t kh_stride;
    uint32_t kh_k;
    const float *tab_and;  // float estimator tables (indexed by the count)
    const float *tab_l;
    const float *tab_kh;
};

__device__ __forceinline__ uint4 ldg16(const uint8_t *p) { return __ldg(reinterpret_cast<const uint4 *>(p)); }

// One lane per pair: the lane reads both rows (whole 16-byte vectors, full
// sectors), counts, and writes the estimate and Jaccard with the same
// arithmetic as the pair path of pg_jaccard_pairs.
__global__ void __launch_bounds__(kServeThreads) k_serve_pairs(const int32_t *__restrict__ row_ptr, int32_t n,
                                                               const PairTile *__restrict__ tiles, int32_t ntiles,
                                                               ServeSketches sk) {
    const unsigned lane = lane_id();
    const int64_t warps = (int64_t)gridDim.x * (kServeThreads / 32);
    const int64_t chunks = (int64_t)ntiles * kChunksPerTile;
    for (int64_t c = ((int64_t)blockIdx.x * kServeThreads + threadIdx.x) >> 5; c < chunks; c += warps) {
        const PairTile *t = tiles + c / kChunksPerTile;
        const int32_t j = (int32_t)(c % kChunksPerTile) * 32 + (int32_t)lane;
        const int32_t count = t->count;
        if (j >= count) continue;
        const int64_t i = (int64_t)t->begin + j;
        const int2 pr = __ldg(reinterpret_cast<const int2 *>(t->pairs) + i);
        const int32_t est = t->est;
        float est_f = 0.0f, jac = 0.0f;
        if (pr.x >= 0 && pr.x < n && pr.y >= 0 && pr.y < n) {
            const int32_t du = __ldg(row_ptr + pr.x + 1) - __ldg(row_ptr + pr.x);
            const int32_t dv = __ldg(row_ptr + pr.y + 1) - __ldg(row_ptr + pr.y);
            uint32_t cnt = 0;
            if (est == PG_EST_KH) {
                const uint8_t *a = sk.kh + (int64_t)pr.x * sk.kh_stride;
                const uint8_t *b = sk.kh + (int64_t)pr.y * sk.kh_stride;
                const int32_t k = (int32_t)sk.kh_k;
                for (int32_t q = 0; q * 4 < k; ++q) {
                    const uint4 x = ldg16(a + 16 * q), y = ldg16(b + 16 * q);
                    cnt += (4 * q + 0 < k && x.x == y.x) + (4 * q + 1 < k && x.y == y.y) +
                           (4 * q + 2 < k && x.z == y.z) + (4 * q + 3 < k && x.w == y.w);
                }
                if (du == 0 || dv == 0) cnt = 0;
                est_f = sk.tab_kh[cnt] * (float)((uint32_t)du + (uint32_t)dv);
            } else {
                const uint8_t *a = sk.bf + (int64_t)pr.x * sk.bf_stride;
                const uint8_t *b = sk.bf + (int64_t)pr.y * sk.bf_stride;
                const int32_t w = (int32_t)(sk.bf_l / 32);
                for (int32_t q = 0; q * 4 < w; ++q) {
                    const uint4 x = ldg16(a + 16 * q), y = ldg16(b + 16 * q);
                    cnt += (4 * q + 0 < w ? __popc(x.x & y.x) : 0) + (4 * q + 1 < w ? __popc(x.y & y.y) : 0) +
                           (4 * q + 2 < w ? __popc(x.z & y.z) : 0) + (4 * q + 3 < w ? __popc(x.w & y.w) : 0);
                }
                est_f = (est == PG_EST_BF_L ? sk.tab_l : sk.tab_and)[cnt];
            }
            const float fu = (float)du, fv = (float)dv;
            const float I = fminf(fmaxf(est_f, 0.0f), fminf(fu, fv));
            const float den = fu + fv - I;
            jac = den > 0.0f ? I / den : 0.0f;
        }
        if (t->cn) t->cn[i] = est_f;
        if (t->jac) t->jac[i] = jac;
    }
}

// Set (or clear) the membership bits of the vertices S[0..ns).
__global__ void k_mark(const int32_t *__restrict__ S, int32_t ns, uint32_t *bitmap, int set) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < ns; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t v = (uint32_t)S[i];
        if (set)
            atomicOr(bitmap + (v >> 5), 1u << (v & 31u));
        else
            atomicAnd(bitmap + (v >> 5), ~(1u << (v & 31u)));
    }
}

__device__ __forceinline__ bool member(const uint32_t *__restrict__ bitmap, int32_t w) {
    return (__ldg(bitmap + ((uint32_t)w >> 5)) >> ((uint32_t)w & 31u)) & 1u;
}

// Phase 1 works on chunks of at most kChunk row entries, (row i of S, first
// entry) pairs listed by the host in row order with at least one chunk per
// row, so a hub row is split over many warps instead of walked by one.
constexpr int32_t kChunk = 1024;
constexpr int kChunkUnroll = 4;  // 32-entry steps whose loads are issued together

// Members of S among the chunk's entries, per chunk (warp per chunk).
__global__ void __launch_bounds__(256) k_chunk_count(const int32_t *__restrict__ row_ptr,
                                                     const int32_t *__restrict__ col,
                                                     const int32_t *__restrict__ S,
                                                     const int2 *__restrict__ chunks, int32_t C,
                                                     const uint32_t *__restrict__ bitmap, int32_t *cnt) {
    const unsigned lane = lane_id();
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < C; c += warps) {
        const int2 ch = chunks[c];
        const int32_t v = S[ch.x];
        const int32_t a = row_ptr[v] + ch.y;
        const int32_t e = min(row_ptr[v + 1], a + kChunk);
        int32_t total = 0;
        for (int32_t base = a; base < e; base += 32 * kChunkUnroll) {
            int32_t w[kChunkUnroll];
#pragma unroll
            for (int u = 0; u < kChunkUnroll; ++u) {
                const int32_t j = base + 32 * u + (int32_t)lane;
                w[u] = j < e ? __ldg(col + j) : -1;
            }
#pragma unroll
            for (int u = 0; u < kChunkUnroll; ++u) {
                const bool in = w[u] >= 0 && member(bitmap, w[u]);
                total += __popc(__ballot_sync(0xffffffffu, in));
            }
        }
        if (lane == 0) cnt[c] = total;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) cnt[C] = 0;  // the scan turns it into the total
}

// Induced rows with local ids (position of the neighbour in sorted S): chunk c
// writes from pos[c] on; the first chunk of row i also sets sub_rp[i].
__global__ void __launch_bounds__(256) k_chunk_fill(const int32_t *__restrict__ row_ptr,
                                                    const int32_t *__restrict__ col,
                                                    const int32_t *__restrict__ S, int32_t ns,
                                                    const int2 *__restrict__ chunks, int32_t C,
                                                    const uint32_t *__restrict__ bitmap,
                                                    const int32_t *__restrict__ pos, int32_t *__restrict__ sub_rp,
                                                    int32_t *__restrict__ sub_col) {
    const unsigned lane = lane_id();
    const unsigned below = (1u << lane) - 1u;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < C; c += warps) {
        const int2 ch = chunks[c];
        const int32_t v = S[ch.x];
        const int32_t a = row_ptr[v] + ch.y;
        const int32_t e = min(row_ptr[v + 1], a + kChunk);
        int32_t out = pos[c];
        if (ch.y == 0 && lane == 0) sub_rp[ch.x] = out;
        for (int32_t base = a; base < e; base += 32 * kChunkUnroll) {
            int32_t w[kChunkUnroll];
#pragma unroll
            for (int u = 0; u < kChunkUnroll; ++u) {
                const int32_t j = base + 32 * u + (int32_t)lane;
                w[u] = j < e ? __ldg(col + j) : -1;
            }
#pragma unroll
            for (int u = 0; u < kChunkUnroll; ++u) {
                const bool in = w[u] >= 0 && member(bitmap, w[u]);
                const unsigned bal = __ballot_sync(0xffffffffu, in);
                if (in) {
                    int32_t lo = 0, hi = ns;  // first index with S[idx] >= w (w is in S)
                    while (lo < hi) {
                        const int32_t mid = (lo + hi) >> 1;
                        if (__ldg(S + mid) < w[u])
                            lo = mid + 1;
                        else
                            hi = mid;
                    }
                    sub_col[out + __popc(bal & below)] = lo;
                }
                out += __popc(bal);
            }
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) sub_rp[ns] = pos[C];
}

int warp_grid(int64_t items) {
    int64_t g = (items + 7) / 8;
    const int64_t cap = 16LL * device_info().sm_count;
    if (g > cap) g = cap;
    return (int)(g < 1 ? 1 : g);
}

// ------------------------------------------------------------- allocator
// First-fit allocator over [0, size) in 256-byte units, with coalescing.
class RangeAlloc {
   public:
    void reset(size_t size) {
        free_.clear();
        size_ = size;
        used_ = peak_ = 0;
        if (size) free_[0] = size;
    }
    bool alloc(size_t bytes, size_t *off) {
        bytes = round_up(bytes ? bytes : 1, 256);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                const size_t rest = it->second - bytes;
                const size_t start = it->first + bytes;
                free_.erase(it);
                if (rest) free_[start] = rest;
                used_ += bytes;
                peak_ = std::max(peak_, used_);
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t bytes) {
        bytes = round_up(bytes ? bytes : 1, 256);
        used_ -= bytes;
        auto it = free_.emplace(off, bytes).first;
        auto next = std::next(it);
        if (next != free_.end() && it->first + it->second == next->first) {
            it->second += next->second;
            free_.erase(next);
        }
        if (it != free_.begin()) {
            auto prev = std::prev(it);
            if (prev->first + prev->second == it->first) {
                prev->second += it->second;
                free_.erase(it);
            }
        }
    }
    // Give back the tail of a block: [off + new_bytes, off + old_bytes).
    void shrink(size_t off, size_t old_bytes, size_t new_bytes) {
        old_bytes = round_up(old_bytes ? old_bytes : 1, 256);
        new_bytes = round_up(new_bytes ? new_bytes : 1, 256);
        if (new_bytes < old_bytes) release(off + new_bytes, old_bytes - new_bytes);
    }
    size_t used() const { return used_; }
    size_t peak() const { return peak_; }
    size_t size() const { return size_; }

   private:
    std::map<size_t, size_t> free_;
    size_t size_ = 0, used_ = 0, peak_ = 0;
};

using Clock = std::chrono::steady_clock;

enum class St { Queued, Phase1, Phase2 };

struct Req {
    uint64_t ticket = 0;
    pg_request r{};
    std::vector<int32_t> S;  // subgraph: sorted, deduplicated
    int64_t U = 0;           // subgraph: sum of the full degrees of S (bound on the induced entries)
    std::vector<int2> chunks;  // subgraph: phase-1 work, (index in S, first entry of the row)
    bool zc = false;               // pairs: the caller's buffers are page-locked, the GPU uses them directly
    const int32_t *d_pairs = nullptr;  // pairs: device-visible input and outputs (arena, or the caller's)
    float *d_cn = nullptr, *d_jac = nullptr;
    St st = St::Queued;
    size_t a_off = 0, a_len = 0;  // arena block
    size_t p_off = 0, p_len = 0;  // staging block
    int64_t next = 0;             // pairs: next pair to put in a tile
    int64_t last_iter = -1;       // pairs: launch that carries the last tile and the output copies
    int stream = -1;              // subgraph: its stream
    cudaEvent_t ev = nullptr;     // subgraph: end of the current phase
    int64_t nnz = 0;              // subgraph: induced CSR entries
    Clock::time_point t_submit, t_admit;
};

// Arena layout of a subgraph request: phase 1 [S | chunks | cnt/pos | scan |
// sub_rp | sub_col | tc], then phase 2.
struct SubLayout {
    size_t S, chunks, pos, scan, rp, col, tc, p2, total_p1;
};
SubLayout sub_layout(int64_t ns, int64_t C, int64_t U) {
    SubLayout L{};
    size_t o = 0;
    auto take = [&](size_t b) {
        const size_t at = o;
        o += round_up(b ? b : 1, 256);
        return at;
    };
    L.S = take(4 * (size_t)ns);
    L.chunks = take(8 * (size_t)C);
    L.pos = take(4 * ((size_t)C + 1));
    L.scan = take(scan_scratch_bytes(C + 1));
    L.rp = take(4 * ((size_t)ns + 1));
    L.col = take(4 * (size_t)U + 4);
    L.tc = take(sizeof(pg_tc_result));
    L.p2 = o;
    L.total_p1 = o;
    return L;
}
// Staging of a subgraph request: [S | chunks | out], out = nnz (int32) at +0
// and the pg_tc_result at +64.
size_t sub_pin_out(const Req *r) { return round_up(4 * r->S.size(), 256) + round_up(8 * r->chunks.size(), 256); }

// Phase 2: [index | sketch | build | table | hist] or [index | exact].
struct Phase2 {
    size_t index, sketch, build, table, hist, exact, total;
};
Phase2 phase2_layout(int32_t ns, int64_t nnz, int32_t est, uint32_t bits) {
    Phase2 P{};
    size_t o = 0;
    auto take = [&](size_t b) {
        const size_t at = o;
        o += round_up(b ? b : 1, 256);
        return at;
    };
    P.index = take(upper_index_bytes(ns, nnz));
    if (est == PG_EST_EXACT) {
        P.exact = take(exact_workspace_bytes(ns, nnz));
    } else {
        P.sketch = take((size_t)ns * (size_t)pg_sketch_stride(PG_SK_BLOOM, bits, 0) + 16);
        P.build = take(build_workspace_bytes(nnz));
        P.table = take(intersect_table_bytes(PG_SK_BLOOM, bits, 0));
        P.hist = take(8 * ((size_t)bits + 1));
    }
    P.total = o;
    return P;
}

}  // namespace
}  // namespace pg

using namespace pg;

struct pg_server {
    pg_csr g{};
    int device = 0;
    pg_sketch bf{}, kh{};
    bool has_bf = false, has_kh = false;
    pg_server_opts opts{};
    std::vector<int32_t> deg;  // host copy of the degrees
    uint8_t *arena = nullptr;
    RangeAlloc arena_alloc;
    uint8_t *pinned = nullptr;
    size_t pinned_bytes = 0;
    RangeAlloc pinned_alloc;
    // reserved device state
    double *tab_and = nullptr, *tab_l = nullptr, *tab_kh = nullptr;
    PairTile *desc_dev[2] = {nullptr, nullptr};
    PairTile *desc_host[2] = {nullptr, nullptr};
    int64_t max_tiles = 0;
    std::vector<uint32_t *> bitmaps;
    cudaStream_t pair_stream = nullptr;
    std::vector<cudaStream_t> sub_streams;
    cudaEvent_t iter_ev[2] = {nullptr, nullptr};
    cudaEvent_t kern_ev[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};  // timing around the pair kernel
    bool kern_timed[2] = {false, false};
    int64_t iter_id[2] = {-1, -1};
    bool iter_busy[2] = {false, false};
    int64_t iters = 0;
    int rr = 0;
    // requests
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<uint64_t> queue;
    std::unordered_map<uint64_t, Req *> reqs;  // queued or running
    std::vector<Req *> pairs_active, subs_active;
    std::unordered_map<uint64_t, pg_response> done;
    uint64_t next_ticket = 1;
    bool stop = false;
    pg_status failed = PG_OK;
    std::thread th;
    pg_server_stats stats{};
};

namespace {

void fill_opts(const pg_server_opts *in, pg_server_opts *o) {
    if (in) *o = *in;
    if (o->streams <= 0) o->streams = 4;
    if (o->max_inflight <= 0) o->max_inflight = 4096;
    if (o->iteration_pairs <= 0) o->iteration_pairs = 262144;
    if (o->pinned_bytes == 0) o->pinned_bytes = 256ull << 20;
    if (o->sub_bits == 0) o->sub_bits = 512;
    if (o->sub_b == 0) o->sub_b = 2;
    if (o->sub_seed == 0) o->sub_seed = 1;
}

int64_t tiles_cap(const pg_server_opts &o) { return o.iteration_pairs / kTile + o.max_inflight + 1; }

// Largest resident sketches a server takes (their estimator tables are reserved up front).
constexpr uint32_t kMaxServeBits = 8192, kMaxServeK = 1024;
size_t table_bytes() {
    return round_up(std::max(intersect_table_bytes(PG_SK_BLOOM, kMaxServeBits, 0),
                             intersect_table_bytes(PG_SK_KHASH, 0, kMaxServeK)),
                    256);
}

size_t reserved_bytes(int32_t n, const pg_server_opts &o) {
    size_t r = 3 * table_bytes();
    r += 2 * round_up((size_t)tiles_cap(o) * sizeof(PairTile), 256);
    r += (size_t)o.streams * round_up(4 * (((size_t)n + 31) / 32) + 8, 256);
    return r;
}

void finish(pg_server *sv, Req *r, pg_status status) {
    // caller holds sv->mu
    pg_response resp{};
    resp.status = status;
    resp.kind = r->r.kind;
    resp.count = r->r.kind == PG_REQ_SUBGRAPH_TC ? (int64_t)r->S.size() : r->r.count;
    if (status == PG_OK && r->r.kind == PG_REQ_SUBGRAPH_TC && r->nnz > 0)
        std::memcpy(&resp.tc, sv->pinned + r->p_off + sub_pin_out(r) + 64, sizeof(pg_tc_result));
    if (status == PG_OK && r->r.kind == PG_REQ_PAIRS && !r->zc) {
        const size_t P = (size_t)r->r.count;
        const uint8_t *out = sv->pinned + r->p_off + round_up(8 * P, 256);
        if (r->r.cn) std::memcpy(r->r.cn, out, 4 * P);
        if (r->r.jac) std::memcpy(r->r.jac, out + round_up(4 * P, 256), 4 * P);
    }
    const auto now = Clock::now();
    const auto t_admit = r->st == St::Queued ? now : r->t_admit;
    resp.queue_us = std::chrono::duration<double, std::micro>(t_admit - r->t_submit).count();
    resp.total_us = std::chrono::duration<double, std::micro>(now - r->t_submit).count();
    if (r->a_len) sv->arena_alloc.release(r->a_off, r->a_len);
    if (r->p_len) sv->pinned_alloc.release(r->p_off, r->p_len);
    if (r->ev) cudaEventDestroy(r->ev);
    if (status == PG_OK)
        sv->stats.completed++;
    else if (status == PG_ERR_CANCELLED)
        sv->stats.cancelled++;
    else
        sv->stats.failed++;
    if (r->r.kind == PG_REQ_PAIRS && status == PG_OK) sv->stats.pairs += (uint64_t)r->r.count;
    sv->done[r->ticket] = resp;
    sv->reqs.erase(r->ticket);
    delete r;
    sv->cv_done.notify_all();
}

// Bytes a request needs in the arena and in the staging memory.
void request_bytes(const pg_server *sv, const Req *r, size_t *arena, size_t *pinned) {
    if (r->r.kind == PG_REQ_PAIRS) {
        const size_t P = (size_t)r->r.count;
        *arena = r->zc ? 0 : round_up(8 * P, 256) + 2 * round_up(4 * P, 256);
        *pinned = *arena;
    } else {
        const int64_t ns = (int64_t)r->S.size();
        const SubLayout L = sub_layout(ns, (int64_t)r->chunks.size(), r->U);
        *arena = L.total_p1 + phase2_layout((int32_t)ns, r->U, r->r.estimator, sv->opts.sub_bits).total;
        *pinned = sub_pin_out(r) + 256;
    }
}

pg_status launch_phase1(pg_server *sv, Req *r) {
    const int32_t ns = (int32_t)r->S.size();
    const int32_t C = (int32_t)r->chunks.size();
    cudaStream_t s = sv->sub_streams[r->stream];
    uint8_t *base = sv->arena + r->a_off;
    const SubLayout L = sub_layout(ns, C, r->U);
    int32_t *S = reinterpret_cast<int32_t *>(base + L.S);
    const int2 *chunks = reinterpret_cast<const int2 *>(base + L.chunks);
    int32_t *pos = reinterpret_cast<int32_t *>(base + L.pos);
    int32_t *scan = reinterpret_cast<int32_t *>(base + L.scan);
    int32_t *rp = reinterpret_cast<int32_t *>(base + L.rp);
    int32_t *col = reinterpret_cast<int32_t *>(base + L.col);
    uint32_t *bm = sv->bitmaps[r->stream];
    // staging [S | chunks | out] has the arena's [S | chunks] offsets: one copy
    uint8_t *pin = sv->pinned + r->p_off;
    std::memcpy(pin + L.S, r->S.data(), 4 * (size_t)ns);
    std::memcpy(pin + L.chunks, r->chunks.data(), 8 * (size_t)C);
    PG_TRY_CUDA(cudaMemcpyAsync(base, pin, L.chunks + 8 * (size_t)C, cudaMemcpyHostToDevice, s), "subgraph: copy S");
    const int tg = (int)std::min<int64_t>((ns + 255) / 256, 4LL * device_info().sm_count);
    k_mark<<<tg, 256, 0, s>>>(S, ns, bm, 1);
    k_chunk_count<<<warp_grid(C), 256, 0, s>>>(sv->g.row_ptr, sv->g.col, S, chunks, C, bm, pos);
    note_launch(2);
    PG_TRY_CUDA(cudaGetLastError(), "subgraph: degrees");
    PG_TRY_CUDA(launch_exclusive_scan(pos, (int64_t)C + 1, scan, s), "subgraph: scan");
    k_chunk_fill<<<warp_grid(C), 256, 0, s>>>(sv->g.row_ptr, sv->g.col, S, ns, chunks, C, bm, pos, rp, col);
    k_mark<<<tg, 256, 0, s>>>(S, ns, bm, 0);
    note_launch(2);
    PG_TRY_CUDA(cudaGetLastError(), "subgraph: induced rows");
    PG_TRY_CUDA(cudaMemcpyAsync(pin + sub_pin_out(r), rp + ns, 4, cudaMemcpyDeviceToHost, s), "subgraph: copy size");
    PG_TRY_CUDA(cudaEventRecord(r->ev, s), "subgraph: event");
    return PG_OK;
}

pg_status launch_phase2(pg_server *sv, Req *r) {
    const int32_t ns = (int32_t)r->S.size();
    cudaStream_t s = sv->sub_streams[r->stream];
    uint8_t *base = sv->arena + r->a_off;
    const SubLayout L = sub_layout(ns, (int64_t)r->chunks.size(), r->U);
    const Phase2 P = phase2_layout(ns, r->nnz, r->r.estimator, sv->opts.sub_bits);
    uint8_t *b2 = base + L.p2;
    const int32_t *rp = reinterpret_cast<const int32_t *>(base + L.rp);
    const int32_t *col = reinterpret_cast<const int32_t *>(base + L.col);
    pg_tc_result *tc = reinterpret_cast<pg_tc_result *>(base + L.tc);
    void *index = b2 + P.index;
    PG_TRY_CUDA(launch_upper_index(rp, col, ns, r->nnz, index, s), "subgraph: edge index");
    const EdgeIndex ix = edge_index_view(index, ns, r->nnz);
    if (r->r.estimator == PG_EST_EXACT) {
        PG_TRY_CUDA(launch_exact_tc(rp, col, ns, r->nnz, ix.upper_off, b2 + P.exact, nullptr, tc, s),
                    "subgraph: exact");
    } else {
        pg_sketch sk{};
        sk.kind = PG_SK_BLOOM;
        sk.bits = sv->opts.sub_bits;
        sk.b = sv->opts.sub_b;
        sk.seed = sv->opts.sub_seed;
        sk.n = ns;
        sk.stride_bytes = pg_sketch_stride(PG_SK_BLOOM, sk.bits, 0);
        sk.data = b2 + P.sketch;
        PG_TRY_CUDA(launch_build_bloom(rp, col, ns, sk.bits, sk.b, sk.seed, static_cast<uint8_t *>(sk.data),
                                       sk.stride_bytes, reinterpret_cast<int32_t *>(b2 + P.build), s),
                    "subgraph: Bloom build");
        uint64_t *hist = reinterpret_cast<uint64_t *>(b2 + P.hist);
        launch_fill_u64(hist, (size_t)sk.bits + 1, 0, s);
        EdgeOutputs eo{};
        eo.hist = hist;
        PG_TRY_CUDA(launch_intersect_ws(rp, col, ns, ix, nullptr, 0, sk, r->r.estimator, eo,
                                        reinterpret_cast<double *>(b2 + P.table), s),
                    "subgraph: pass");
        PG_TRY_CUDA(launch_tc_finalize(hist, sk, r->r.estimator, tc, s), "subgraph: finalize");
    }
    uint8_t *pin = sv->pinned + r->p_off + sub_pin_out(r);
    PG_TRY_CUDA(cudaMemcpyAsync(pin + 64, tc, sizeof(pg_tc_result), cudaMemcpyDeviceToHost, s), "subgraph: copy");
    PG_TRY_CUDA(cudaEventRecord(r->ev, s), "subgraph: event");
    return PG_OK;
}

// Copies of whole request blocks between staging and arena, merged where
// consecutive blocks are adjacent in both (the allocators hand out blocks in
// order, so a burst of admissions usually becomes one copy).
struct Span {
    size_t p, a, len;
};
cudaError_t copy_spans(pg_server *sv, std::vector<Span> &spans, cudaMemcpyKind kind) {
    std::sort(spans.begin(), spans.end(), [](const Span &x, const Span &y) { return x.p < y.p; });
    size_t i = 0;
    while (i < spans.size()) {
        Span cur = spans[i++];
        while (i < spans.size() && spans[i].p == cur.p + cur.len && spans[i].a == cur.a + cur.len)
            cur.len += spans[i++].len;
        cudaError_t e = kind == cudaMemcpyHostToDevice
                            ? cudaMemcpyAsync(sv->arena + cur.a, sv->pinned + cur.p, cur.len, kind, sv->pair_stream)
                            : cudaMemcpyAsync(sv->pinned + cur.p, sv->arena + cur.a, cur.len, kind, sv->pair_stream);
        if (e != cudaSuccess) return e;
    }
    spans.clear();
    return cudaSuccess;
}

// Admit queued requests in order while they fit. Caller holds mu.
bool admit(pg_server *sv) {
    bool progress = false;
    std::vector<Span> h2d;
    std::vector<Req *> admitted_pairs;
    while (!sv->queue.empty() &&
           (int64_t)(sv->pairs_active.size() + sv->subs_active.size() + admitted_pairs.size()) <
               sv->opts.max_inflight) {
        Req *r = sv->reqs[sv->queue.front()];
        size_t need_a = 0, need_p = 0;
        request_bytes(sv, r, &need_a, &need_p);
        size_t a_off = 0, p_off = 0;
        if (need_a && !sv->arena_alloc.alloc(need_a, &a_off)) break;
        if (need_p && !sv->pinned_alloc.alloc(need_p, &p_off)) {
            if (need_a) sv->arena_alloc.release(a_off, need_a);
            break;
        }
        sv->queue.pop_front();
        r->a_off = a_off;
        r->a_len = need_a;
        r->p_off = p_off;
        r->p_len = need_p;
        r->t_admit = Clock::now();
        progress = true;
        r->st = St::Phase1;
        if (r->r.kind == PG_REQ_PAIRS && r->zc) {
            admitted_pairs.push_back(r);
        } else if (r->r.kind == PG_REQ_PAIRS) {
            // block layout [pairs | cn | jac], identical in staging and arena; the whole block is
            // copied (the output parts are overwritten by the kernel)
            const size_t P = (size_t)r->r.count;
            std::memcpy(sv->pinned + p_off, r->r.data, 8 * P);
            h2d.push_back(Span{p_off, a_off, round_up(need_a, 256)});
            uint8_t *a = sv->arena + a_off;
            r->d_pairs = reinterpret_cast<const int32_t *>(a);
            r->d_cn = r->r.cn ? reinterpret_cast<float *>(a + round_up(8 * P, 256)) : nullptr;
            r->d_jac = r->r.jac ? reinterpret_cast<float *>(a + round_up(8 * P, 256) + round_up(4 * P, 256)) : nullptr;
            admitted_pairs.push_back(r);
        } else {
            r->stream = sv->rr++ % (int)sv->sub_streams.size();
            cudaError_t e = cudaEventCreateWithFlags(&r->ev, cudaEventDisableTiming);
            pg_status st = e == cudaSuccess ? launch_phase1(sv, r) : cuda_status(e, "serve: event");
            if (st != PG_OK) {
                sv->failed = st;
                finish(sv, r, st);
                continue;
            }
            sv->subs_active.push_back(r);
            sv->stats.subgraphs++;
        }
    }
    const cudaError_t e = h2d.empty() ? cudaSuccess : copy_spans(sv, h2d, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        sv->failed = cuda_status(e, "serve: copy pairs");
        for (Req *r : admitted_pairs) finish(sv, r, sv->failed);
        return true;
    }
    for (Req *r : admitted_pairs) sv->pairs_active.push_back(r);
    return progress;
}

// One launch of the pair kernel over tiles of every admitted pair request,
// plus the exact pair requests. Caller holds mu.
bool launch_pairs(pg_server *sv) {
    bool pending = false;
    for (Req *r : sv->pairs_active)
        if (r->next < r->r.count) pending = true;
    if (!pending) return false;
    const int slot = (int)(sv->iters & 1);
    if (sv->iter_busy[slot]) return false;
    const int64_t id = sv->iters;
    PairTile *th = sv->desc_host[slot];
    int64_t nt = 0, budget = sv->opts.iteration_pairs;
    std::vector<Req *> exact;
    for (Req *r : sv->pairs_active)
        if (r->r.estimator == PG_EST_EXACT && r->next < r->r.count) {
            r->next = r->r.count;
            r->last_iter = id;
            exact.push_back(r);
        }
    bool grabbed = true;
    while (grabbed && budget > 0 && nt < sv->max_tiles) {
        grabbed = false;
        for (Req *r : sv->pairs_active) {
            if (r->next >= r->r.count) continue;
            const int32_t take = (int32_t)std::min<int64_t>(kTile, r->r.count - r->next);
            PairTile t{};
            t.pairs = r->d_pairs;
            t.cn = r->d_cn;
            t.jac = r->d_jac;
            t.begin = (int32_t)r->next;
            t.count = take;
            t.est = r->r.estimator;
            th[nt++] = t;
            r->next += take;
            budget -= take;
            grabbed = true;
            if (r->next == r->r.count) r->last_iter = id;
            if (budget <= 0 || nt >= sv->max_tiles) break;
        }
    }
    cudaStream_t s = sv->pair_stream;
    cudaError_t e = cudaSuccess;
    if (nt > 0) {
        e = cudaMemcpyAsync(sv->desc_dev[slot], th, (size_t)nt * sizeof(PairTile), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) {
            ServeSketches sk{};
            if (sv->has_bf) {
                sk.bf = static_cast<const uint8_t *>(sv->bf.data);
                sk.bf_stride = sv->bf.stride_bytes;
                sk.bf_l = sv->bf.bits;
                sk.tab_and = reinterpret_cast<const float *>(sv->tab_and + 2 * ((int64_t)sv->bf.bits + 1));
                sk.tab_l = reinterpret_cast<const float *>(sv->tab_l + 2 * ((int64_t)sv->bf.bits + 1));
            }
            if (sv->has_kh) {
                sk.kh = static_cast<const uint8_t *>(sv->kh.data);
                sk.kh_stride = sv->kh.stride_bytes;
                sk.kh_k = sv->kh.k;
                sk.tab_kh = reinterpret_cast<const float *>(sv->tab_kh + 2 * ((int64_t)sv->kh.k + 1));
            }
            const int64_t warps = nt * kChunksPerTile;
            int64_t grid = (warps + kServeThreads / 32 - 1) / (kServeThreads / 32);
            const int64_t cap = 8LL * device_info().sm_count;
            if (grid > cap) grid = cap;
            e = cudaEventRecord(sv->kern_ev[slot][0], s);
            k_serve_pairs<<<(unsigned)grid, kServeThreads, 0, s>>>(sv->g.row_ptr, sv->g.n, sv->desc_dev[slot],
                                                                   (int32_t)nt, sk);
            note_launch();
            if (e == cudaSuccess) e = cudaGetLastError();
            if (e == cudaSuccess) e = cudaEventRecord(sv->kern_ev[slot][1], s);
            sv->kern_timed[slot] = e == cudaSuccess;
            sv->stats.pair_launches++;
        }
    }
    for (Req *r : exact) {
        if (e != cudaSuccess) break;
        EdgeOutputs eo{};
        eo.cn = r->d_cn;
        eo.jac = r->d_jac;
        e = launch_exact_pairs(sv->g.row_ptr, sv->g.col, sv->g.n, EdgeIndex{}, r->d_pairs, r->r.count, eo, s);
    }
    // results of the requests that end in this launch go back to the staging memory: from the
    // output part of a block to its end, merged across blocks adjacent in both staging and arena
    // (a merged copy also brings back the pair part of the inner blocks, unchanged)
    if (e == cudaSuccess) {
        struct Out {
            size_t p, a, out, len;  // block offsets, start of its outputs, block bytes
        };
        std::vector<Out> d2h;
        for (Req *r : sv->pairs_active) {
            if (r->last_iter != id || r->zc || (!r->r.cn && !r->r.jac)) continue;
            d2h.push_back(Out{r->p_off, r->a_off, round_up(8 * (size_t)r->r.count, 256), round_up(r->a_len, 256)});
        }
        std::sort(d2h.begin(), d2h.end(), [](const Out &x, const Out &y) { return x.p < y.p; });
        size_t i = 0;
        while (i < d2h.size() && e == cudaSuccess) {
            const Out first = d2h[i++];
            size_t end_p = first.p + first.len, end_a = first.a + first.len;
            while (i < d2h.size() && d2h[i].p == end_p && d2h[i].a == end_a) {
                end_p += d2h[i].len;
                end_a += d2h[i].len;
                ++i;
            }
            const size_t from = first.out;
            e = cudaMemcpyAsync(sv->pinned + first.p + from, sv->arena + first.a + from, end_p - first.p - from,
                                cudaMemcpyDeviceToHost, s);
        }
    }
    if (e == cudaSuccess) e = cudaEventRecord(sv->iter_ev[slot], s);
    if (e != cudaSuccess) {
        sv->failed = cuda_status(e, "serve: pair launch");
        return true;
    }
    sv->iter_busy[slot] = true;
    sv->iter_id[slot] = id;
    sv->iters++;
    return true;
}

// Completed launches and phases. Caller holds mu.
bool poll_events(pg_server *sv) {
    bool progress = false;
    for (int slot = 0; slot < 2; ++slot) {
        if (!sv->iter_busy[slot]) continue;
        const cudaError_t q = cudaEventQuery(sv->iter_ev[slot]);
        if (q == cudaErrorNotReady) continue;
        const pg_status st = q == cudaSuccess ? PG_OK : cuda_status(q, "serve: pair launch");
        if (st != PG_OK) sv->failed = st;
        const int64_t id = sv->iter_id[slot];
        sv->iter_busy[slot] = false;
        if (sv->kern_timed[slot] && st == PG_OK) {
            float ms = 0.0f;
            if (cudaEventElapsedTime(&ms, sv->kern_ev[slot][0], sv->kern_ev[slot][1]) == cudaSuccess)
                sv->stats.pair_kernel_ns += (uint64_t)(ms * 1e6);
            sv->kern_timed[slot] = false;
        }
        std::vector<Req *> keep;
        for (Req *r : sv->pairs_active) {
            if (r->last_iter == id && r->next >= r->r.count)
                finish(sv, r, st);
            else
                keep.push_back(r);
        }
        sv->pairs_active.swap(keep);
        progress = true;
    }
    std::vector<Req *> keep;
    for (Req *r : sv->subs_active) {
        const cudaError_t q = cudaEventQuery(r->ev);
        if (q == cudaErrorNotReady) {
            keep.push_back(r);
            continue;
        }
        progress = true;
        if (q != cudaSuccess) {
            sv->failed = cuda_status(q, "serve: subgraph");
            finish(sv, r, sv->failed);
            continue;
        }
        if (r->st == St::Phase1) {
            int32_t nnz = 0;
            std::memcpy(&nnz, sv->pinned + r->p_off + sub_pin_out(r), 4);
            r->nnz = nnz;
            if (nnz <= 0 || sv->failed) {
                r->nnz = 0;
                finish(sv, r, sv->failed ? sv->failed : PG_OK);
                continue;
            }
            // keep phase 1 and the exact phase-2 size, give the rest back
            const SubLayout L = sub_layout((int64_t)r->S.size(), (int64_t)r->chunks.size(), r->U);
            const size_t need = L.total_p1 + phase2_layout((int32_t)r->S.size(), r->nnz, r->r.estimator,
                                                           sv->opts.sub_bits).total;
            sv->arena_alloc.shrink(r->a_off, r->a_len, need);
            r->a_len = round_up(need, 256) < round_up(r->a_len, 256) ? need : r->a_len;
            r->st = St::Phase2;
            const pg_status st = launch_phase2(sv, r);
            if (st != PG_OK) {
                sv->failed = st;
                finish(sv, r, st);
                continue;
            }
            keep.push_back(r);
        } else {
            finish(sv, r, PG_OK);
        }
    }
    sv->subs_active.swap(keep);
    return progress;
}

void scheduler(pg_server *sv) {
    cudaSetDevice(sv->device);
    std::unique_lock<std::mutex> lk(sv->mu);
    for (;;) {
        bool progress = false;
        if (sv->failed == PG_OK) {
            progress |= admit(sv);
            progress |= launch_pairs(sv);
        }
        progress |= poll_events(sv);
        if (sv->failed != PG_OK) {
            while (!sv->queue.empty()) {
                Req *r = sv->reqs[sv->queue.front()];
                sv->queue.pop_front();
                finish(sv, r, sv->failed);
            }
        }
        const bool busy = !sv->pairs_active.empty() || !sv->subs_active.empty();
        if (sv->stop && sv->queue.empty() && !busy) break;
        if (!progress) {
            if (busy)
                sv->cv_work.wait_for(lk, std::chrono::microseconds(20));
            else
                sv->cv_work.wait_for(lk, std::chrono::milliseconds(50));
        }
    }
}

}  // namespace

extern "C" {

size_t pg_server_reserved_bytes(const pg_csr *g, const pg_server_opts *opts) {
    if (!g || g->n < 0) return 0;
    pg_server_opts o{};
    fill_opts(opts, &o);
    return reserved_bytes(g->n, o);
}

pg_status pg_server_create(const pg_csr *g, const pg_sketch *const *sketches, int32_t n_sketches, void *arena,
                           size_t arena_bytes, const pg_server_opts *opts, pg_server **out) {
    PG_TRACE("pg_server_create");
    pg_status st = check_graph(g);
    if (st) return st;
    PG_REQUIRE(out != nullptr, PG_ERR_INVALID_ARG, "pg_server_create: out is NULL");
    PG_REQUIRE(n_sketches >= 0 && n_sketches <= 2 && (n_sketches == 0 || sketches), PG_ERR_INVALID_ARG,
               "pg_server_create: 0 to 2 sketches");
    PG_REQUIRE(arena && aligned16(arena), PG_ERR_INVALID_ARG, "pg_server_create: arena must be 16-byte aligned");
    pg_server_opts o{};
    fill_opts(opts, &o);
    PG_REQUIRE(o.sub_bits % 64 == 0 && o.sub_bits <= 2048 && o.sub_b >= 1 && o.sub_b <= 16, PG_ERR_UNSUPPORTED,
               "pg_server_create: subgraph Bloom bits %u (multiple of 64, <= 2048), b %u (1..16)", o.sub_bits,
               o.sub_b);
    PG_REQUIRE(o.streams <= 64, PG_ERR_INVALID_ARG, "pg_server_create: at most 64 streams");
    const size_t reserved = reserved_bytes(g->n, o);
    PG_REQUIRE(arena_bytes >= reserved + 4096, PG_ERR_NO_MEMORY,
               "pg_server_create: arena has %zu bytes, the server reserves %zu", arena_bytes, reserved);
    pg_server *sv = new pg_server();
    sv->g = *g;
    sv->opts = o;
    for (int32_t i = 0; i < n_sketches; ++i) {
        const pg_sketch *sk = sketches[i];
        st = sk ? check_sketch(g, sk) : set_error(PG_ERR_INVALID_ARG, "pg_server_create: sketch %d is NULL", i);
        if (st == PG_OK && ((sk->kind == PG_SK_BLOOM && sk->bits > kMaxServeBits) ||
                            (sk->kind == PG_SK_KHASH && sk->k > kMaxServeK)))
            st = set_error(PG_ERR_UNSUPPORTED, "pg_server_create: sketch %d larger than %u bits / k %u", i,
                           kMaxServeBits, kMaxServeK);
        if (st == PG_OK && sk->kind == PG_SK_BLOOM && !sv->has_bf) {
            sv->bf = *sk;
            sv->has_bf = true;
        } else if (st == PG_OK && sk->kind == PG_SK_KHASH && !sv->has_kh) {
            sv->kh = *sk;
            sv->has_kh = true;
        } else if (st == PG_OK) {
            st = set_error(PG_ERR_UNSUPPORTED, "pg_server_create: sketch %d: one Bloom and one k-Hash at most", i);
        }
        if (st) {
            delete sv;
            return st;
        }
    }
    cudaError_t e = cudaGetDevice(&sv->device);
    sv->arena = static_cast<uint8_t *>(arena);
    // reserved region: tables, descriptors, bitmaps
    size_t off = 0;
    auto take = [&](size_t b) {
        uint8_t *p = sv->arena + off;
        off += round_up(b, 256);
        return p;
    };
    const size_t tb = table_bytes();
    sv->tab_and = reinterpret_cast<double *>(take(tb));
    sv->tab_l = reinterpret_cast<double *>(take(tb));
    sv->tab_kh = reinterpret_cast<double *>(take(tb));
    sv->max_tiles = tiles_cap(o);
    for (int i = 0; i < 2; ++i) sv->desc_dev[i] = reinterpret_cast<PairTile *>(take((size_t)sv->max_tiles * sizeof(PairTile)));
    const size_t bm_bytes = 4 * (((size_t)g->n + 31) / 32) + 8;
    for (int i = 0; i < o.streams; ++i) sv->bitmaps.push_back(reinterpret_cast<uint32_t *>(take(bm_bytes)));
    sv->arena_alloc.reset(arena_bytes - off);
    sv->arena += off;  // requests use the rest
    // host side
    const size_t desc_host_bytes = round_up((size_t)sv->max_tiles * sizeof(PairTile), 256);
    sv->pinned_bytes = o.pinned_bytes + 2 * desc_host_bytes;
    if (e == cudaSuccess) e = cudaHostAlloc(reinterpret_cast<void **>(&sv->pinned), sv->pinned_bytes, cudaHostAllocDefault);
    if (e == cudaSuccess) {
        sv->desc_host[0] = reinterpret_cast<PairTile *>(sv->pinned + o.pinned_bytes);
        sv->desc_host[1] = reinterpret_cast<PairTile *>(sv->pinned + o.pinned_bytes + desc_host_bytes);
        sv->pinned_alloc.reset(o.pinned_bytes);
    }
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sv->pair_stream, cudaStreamNonBlocking);
    for (int i = 0; i < o.streams && e == cudaSuccess; ++i) {
        cudaStream_t s = nullptr;
        e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
        if (e == cudaSuccess) sv->sub_streams.push_back(s);
    }
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&sv->iter_ev[i], cudaEventDisableTiming);
    for (int i = 0; i < 2 && e == cudaSuccess; ++i)
        for (int j = 0; j < 2 && e == cudaSuccess; ++j) e = cudaEventCreate(&sv->kern_ev[i][j]);
    cudaStream_t s0 = sv->pair_stream;
    if (e == cudaSuccess) {
        for (int i = 0; i < o.streams; ++i) launch_fill_u64(reinterpret_cast<uint64_t *>(sv->bitmaps[i]), bm_bytes / 8, 0, s0);
        if (sv->has_bf) {
            e = launch_estimator_table(sv->tab_and, PG_SK_BLOOM, PG_EST_BF_AND, sv->bf.bits, sv->bf.b, 0, s0);
            if (e == cudaSuccess)
                e = launch_estimator_table(sv->tab_l, PG_SK_BLOOM, PG_EST_BF_L, sv->bf.bits, sv->bf.b, 0, s0);
        }
        if (e == cudaSuccess && sv->has_kh) e = launch_estimator_table(sv->tab_kh, PG_SK_KHASH, PG_EST_KH, 0, 0, sv->kh.k, s0);
    }
    // host copy of the degrees (admission bounds of subgraph requests)
    std::vector<int32_t> rp((size_t)g->n + 1);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(rp.data(), g->row_ptr, 4 * rp.size(), cudaMemcpyDeviceToHost, s0);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s0);
    if (e != cudaSuccess) {
        for (cudaStream_t s : sv->sub_streams) cudaStreamDestroy(s);
        if (sv->pair_stream) cudaStreamDestroy(sv->pair_stream);
        for (auto ev : sv->iter_ev)
            if (ev) cudaEventDestroy(ev);
        for (auto &pr : sv->kern_ev)
            for (auto ev : pr)
                if (ev) cudaEventDestroy(ev);
        if (sv->pinned) cudaFreeHost(sv->pinned);
        delete sv;
        return cuda_status(e, "pg_server_create");
    }
    sv->deg.resize((size_t)g->n);
    for (int32_t v = 0; v < g->n; ++v) sv->deg[v] = rp[v + 1] - rp[v];
    sv->stats.arena_bytes = sv->arena_alloc.size();
    sv->th = std::thread(scheduler, sv);
    *out = sv;
    return PG_OK;
}

}  // extern "C"

namespace {

// Device address of a page-locked host range [p, p + bytes), if the whole
// range is one mapping of page-locked memory the device can reach.
bool device_view(const void *p, size_t bytes, void **dev) {
    cudaPointerAttributes a0{}, a1{};
    const char *last = static_cast<const char *>(p) + bytes - 1;
    if (cudaPointerGetAttributes(&a0, p) != cudaSuccess || cudaPointerGetAttributes(&a1, last) != cudaSuccess) {
        cudaGetLastError();  // clear the error the failed query recorded
        return false;
    }
    if (a0.type != cudaMemoryTypeHost || a1.type != cudaMemoryTypeHost || !a0.devicePointer || !a1.devicePointer)
        return false;
    if (static_cast<char *>(a1.devicePointer) - static_cast<char *>(a0.devicePointer) != (ptrdiff_t)(bytes - 1))
        return false;
    *dev = a0.devicePointer;
    return true;
}

// Validate one request and build its record (no lock held).
pg_status prepare(pg_server *sv, const pg_request *req, Req **out) {
    PG_REQUIRE(req, PG_ERR_INVALID_ARG, "pg_submit: NULL request");
    PG_REQUIRE(req->kind == PG_REQ_PAIRS || req->kind == PG_REQ_SUBGRAPH_TC, PG_ERR_INVALID_ARG,
               "pg_submit: unknown request kind %d", req->kind);
    PG_REQUIRE(req->count >= 0 && req->count < (1LL << 31) && (req->count == 0 || req->data), PG_ERR_INVALID_ARG,
               "pg_submit: count %lld with data %p", (long long)req->count, (const void *)req->data);
    if (req->kind == PG_REQ_PAIRS) {
        const int32_t est = req->estimator;
        const bool ok = est == PG_EST_EXACT || ((est == PG_EST_BF_AND || est == PG_EST_BF_L) && sv->has_bf) ||
                        (est == PG_EST_KH && sv->has_kh);
        PG_REQUIRE(ok, PG_ERR_UNSUPPORTED, "pg_submit: pair estimator %d needs a resident sketch of its kind", est);
    } else {
        PG_REQUIRE(req->estimator == PG_EST_BF_AND || req->estimator == PG_EST_BF_L || req->estimator == PG_EST_EXACT,
                   PG_ERR_UNSUPPORTED, "pg_submit: subgraph estimator %d (BF_AND, BF_L or EXACT)", req->estimator);
        for (int64_t i = 0; i < req->count; ++i)
            PG_REQUIRE(req->data[i] >= 0 && req->data[i] < sv->g.n, PG_ERR_INVALID_ARG,
                       "pg_submit: vertex %d outside [0, %d)", req->data[i], sv->g.n);
    }
    Req *r = new Req();
    r->r = *req;
    r->t_submit = Clock::now();
    if (req->kind == PG_REQ_PAIRS && req->count > 0) {
        // page-locked input and outputs: the kernel reads and writes them in place (over the
        // CPU-GPU link), with no staging copies; anything else goes through the staging memory
        void *dp = nullptr, *dc = nullptr, *dj = nullptr;
        const size_t P = (size_t)req->count;
        r->zc = device_view(req->data, 8 * P, &dp) && (!req->cn || device_view(req->cn, 4 * P, &dc)) &&
                (!req->jac || device_view(req->jac, 4 * P, &dj));
        if (r->zc) {
            r->d_pairs = static_cast<const int32_t *>(dp);
            r->d_cn = static_cast<float *>(dc);
            r->d_jac = static_cast<float *>(dj);
        }
    }
    if (req->kind == PG_REQ_SUBGRAPH_TC) {
        r->S.assign(req->data, req->data + req->count);
        std::sort(r->S.begin(), r->S.end());
        r->S.erase(std::unique(r->S.begin(), r->S.end()), r->S.end());
        r->chunks.reserve(r->S.size());
        for (size_t i = 0; i < r->S.size(); ++i) {
            const int32_t d = sv->deg[r->S[i]];
            r->U += d;
            int32_t off = 0;
            do {
                r->chunks.push_back(make_int2((int32_t)i, off));
                off += kChunk;
            } while (off < d);
        }
    }
    *out = r;
    return PG_OK;
}

// Queue a prepared request (mu held).
pg_status enqueue_locked(pg_server *sv, Req *r, uint64_t *ticket) {
    size_t need_a = 0, need_p = 0;
    request_bytes(sv, r, &need_a, &need_p);
    if (sv->failed != PG_OK || sv->stop)
        return set_error(sv->failed != PG_OK ? sv->failed : PG_ERR_CANCELLED, "pg_submit: the server has stopped");
    if (round_up(need_a, 256) > sv->arena_alloc.size() || round_up(need_p, 256) > sv->pinned_alloc.size())
        return set_error(PG_ERR_NO_MEMORY,
                         "pg_submit: request needs %zu arena and %zu staging bytes, the server has %zu and %zu",
                         need_a, need_p, sv->arena_alloc.size(), sv->pinned_alloc.size());
    r->ticket = sv->next_ticket++;
    *ticket = r->ticket;
    sv->stats.submitted++;
    sv->reqs[r->ticket] = r;
    const bool empty = (r->r.kind == PG_REQ_PAIRS && r->r.count == 0) ||
                       (r->r.kind == PG_REQ_SUBGRAPH_TC && r->S.empty());
    if (empty)
        finish(sv, r, PG_OK);
    else
        sv->queue.push_back(r->ticket);
    return PG_OK;
}

}  // namespace

extern "C" {

pg_status pg_submit(pg_server *sv, const pg_request *req, uint64_t *ticket) {
    PG_REQUIRE(sv && ticket, PG_ERR_INVALID_ARG, "pg_submit: NULL argument");
    Req *r = nullptr;
    pg_status st = prepare(sv, req, &r);
    if (st) return st;
    std::lock_guard<std::mutex> lk(sv->mu);
    st = enqueue_locked(sv, r, ticket);
    if (st) {
        delete r;
        return st;
    }
    sv->cv_work.notify_one();
    return PG_OK;
}

pg_status pg_submit_many(pg_server *sv, const pg_request *reqs, int64_t count, uint64_t *tickets) {
    PG_REQUIRE(sv && tickets && count >= 0 && (count == 0 || reqs), PG_ERR_INVALID_ARG,
               "pg_submit_many: NULL argument");
    std::vector<Req *> rs((size_t)count, nullptr);
    for (int64_t i = 0; i < count; ++i) {
        const pg_status st = prepare(sv, reqs + i, &rs[i]);
        if (st) {
            for (Req *r : rs) delete r;
            return set_error(st, "pg_submit_many: request %lld: %s", (long long)i, pg_last_error());
        }
    }
    std::lock_guard<std::mutex> lk(sv->mu);
    for (int64_t i = 0; i < count; ++i) {
        size_t need_a = 0, need_p = 0;
        request_bytes(sv, rs[i], &need_a, &need_p);
        if (round_up(need_a, 256) > sv->arena_alloc.size() || round_up(need_p, 256) > sv->pinned_alloc.size() ||
            sv->failed != PG_OK || sv->stop) {
            const pg_status f = sv->failed != PG_OK ? sv->failed : sv->stop ? PG_ERR_CANCELLED : PG_ERR_NO_MEMORY;
            for (Req *r : rs) delete r;
            return set_error(f, "pg_submit_many: request %lld can not be served (%s)", (long long)i,
                             pg_status_string(f));
        }
    }
    for (int64_t i = 0; i < count; ++i) {
        const pg_status st = enqueue_locked(sv, rs[i], tickets + i);  // cannot fail after the checks above
        if (st) delete rs[i];
    }
    sv->cv_work.notify_one();
    return PG_OK;
}

pg_status pg_poll_many(pg_server *sv, const uint64_t *tickets, int64_t count, pg_response *out, int64_t timeout_us,
                       int64_t *n_done) {
    PG_REQUIRE(sv && count >= 0 && (count == 0 || (tickets && out)), PG_ERR_INVALID_ARG,
               "pg_poll_many: NULL argument");
    std::unique_lock<std::mutex> lk(sv->mu);
    const auto deadline = Clock::now() + std::chrono::microseconds(timeout_us > 0 ? timeout_us : 0);
    std::vector<char> got((size_t)count, 0);
    int64_t done = 0;
    for (;;) {
        for (int64_t i = 0; i < count; ++i) {
            if (got[i]) continue;
            auto it = sv->done.find(tickets[i]);
            if (it != sv->done.end()) {
                out[i] = it->second;
                sv->done.erase(it);
                got[i] = 1;
                ++done;
            } else if (sv->reqs.find(tickets[i]) == sv->reqs.end()) {
                out[i] = pg_response{};
                out[i].status = PG_ERR_NOT_FOUND;
                got[i] = 1;
                ++done;
            }
        }
        if (done == count || timeout_us <= 0 || Clock::now() >= deadline) break;
        sv->cv_done.wait_until(lk, deadline);
    }
    for (int64_t i = 0; i < count; ++i)
        if (!got[i]) {
            out[i] = pg_response{};
            out[i].status = PG_ERR_BUSY;
        }
    if (n_done) *n_done = done;
    return done == count ? PG_OK : set_error(PG_ERR_BUSY, "pg_poll_many: %lld of %lld complete", (long long)done,
                                             (long long)count);
}

pg_status pg_poll(pg_server *sv, uint64_t ticket, pg_response *out, int64_t timeout_us) {
    PG_REQUIRE(sv && out, PG_ERR_INVALID_ARG, "pg_poll: NULL argument");
    std::unique_lock<std::mutex> lk(sv->mu);
    const auto deadline = Clock::now() + std::chrono::microseconds(timeout_us > 0 ? timeout_us : 0);
    for (;;) {
        auto it = sv->done.find(ticket);
        if (it != sv->done.end()) {
            *out = it->second;
            sv->done.erase(it);
            return PG_OK;
        }
        if (sv->reqs.find(ticket) == sv->reqs.end())
            return set_error(PG_ERR_NOT_FOUND, "pg_poll: unknown ticket %llu", (unsigned long long)ticket);
        if (timeout_us <= 0 || Clock::now() >= deadline)
            return set_error(PG_ERR_BUSY, "pg_poll: ticket %llu not complete", (unsigned long long)ticket);
        sv->cv_done.wait_until(lk, deadline);
    }
}

pg_status pg_cancel(pg_server *sv, uint64_t ticket) {
    PG_REQUIRE(sv, PG_ERR_INVALID_ARG, "pg_cancel: NULL server");
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->reqs.find(ticket);
    if (it == sv->reqs.end()) {
        if (sv->done.count(ticket)) return set_error(PG_ERR_BUSY, "pg_cancel: ticket %llu already complete",
                                                     (unsigned long long)ticket);
        return set_error(PG_ERR_NOT_FOUND, "pg_cancel: unknown ticket %llu", (unsigned long long)ticket);
    }
    Req *r = it->second;
    if (r->st != St::Queued)
        return set_error(PG_ERR_BUSY, "pg_cancel: ticket %llu is running", (unsigned long long)ticket);
    sv->queue.erase(std::find(sv->queue.begin(), sv->queue.end(), ticket));
    finish(sv, r, PG_ERR_CANCELLED);
    return PG_OK;
}

pg_status pg_server_stats_get(pg_server *sv, pg_server_stats *out) {
    PG_REQUIRE(sv && out, PG_ERR_INVALID_ARG, "pg_server_stats_get: NULL argument");
    std::lock_guard<std::mutex> lk(sv->mu);
    *out = sv->stats;
    out->queued = sv->queue.size();
    out->running = sv->pairs_active.size() + sv->subs_active.size();
    out->arena_used = sv->arena_alloc.used();
    out->arena_peak = sv->arena_alloc.peak();
    out->arena_bytes = sv->arena_alloc.size();
    return PG_OK;
}

pg_status pg_server_destroy(pg_server *sv) {
    PG_TRACE("pg_server_destroy");
    if (!sv) return PG_OK;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        while (!sv->queue.empty()) {
            Req *r = sv->reqs[sv->queue.front()];
            sv->queue.pop_front();
            finish(sv, r, PG_ERR_CANCELLED);
        }
        sv->stop = true;
        sv->cv_work.notify_all();
    }
    if (sv->th.joinable()) sv->th.join();
    cudaError_t e = cudaSuccess;
    for (cudaStream_t s : sv->sub_streams) {
        cudaError_t e2 = cudaStreamSynchronize(s);
        if (e == cudaSuccess) e = e2;
        cudaStreamDestroy(s);
    }
    if (sv->pair_stream) {
        cudaError_t e2 = cudaStreamSynchronize(sv->pair_stream);
        if (e == cudaSuccess) e = e2;
        cudaStreamDestroy(sv->pair_stream);
    }
    for (auto ev : sv->iter_ev)
        if (ev) cudaEventDestroy(ev);
    for (auto &pr : sv->kern_ev)
        for (auto ev : pr)
            if (ev) cudaEventDestroy(ev);
    if (sv->pinned) cudaFreeHost(sv->pinned);
    for (auto &kv : sv->reqs) delete kv.second;
    delete sv;
    return e == cudaSuccess ? PG_OK : cuda_status(e, "pg_server_destroy");
}

}  // extern "C"

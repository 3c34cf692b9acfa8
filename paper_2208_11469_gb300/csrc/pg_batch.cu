// Batched analysis of many small graphs in one CUDA-graph launch.
//
// The G graphs are one block-diagonal CSR ("union graph", global vertex ids;
// graph g owns vertices [voff[g], voff[g+1])). Each graph gets its own Bloom
// parameters (l, b) and kernel variant; graphs with equal (l, b) must be
// contiguous ("buckets"). One run is
//   per bucket: Bloom build of its vertex range (hashing each graph's own
//     ids, so a sketch is the same alone and in the batch)
//   -> per bucket: pull pass over the rows of its vertices (per-graph
//      popcount histograms, per-vertex sums, LCC and triangles per vertex)
//   -> per graph the histogram dot (TC estimate).
// The first pg_batch_run on a non-default stream captures this sequence into
// a CUDA graph; later runs replay it with one launch.
//
// The autotuner (pg_batch_autotune) picks per graph the filter length from
// the storage budget (Sec. V-A), the hash count from an accuracy model of the
// AND estimator (Eq. bf_int), and pg_batch_create times the pull pass's
// lane/warp split on each bucket itself and keeps the fastest.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "pg_internal.cuh"

namespace pg {
namespace {

// ------------------------------------------------------------- pull pass
// The pass walks each vertex's whole row (every undirected edge is seen from
// both ends, so no upper-edge list is built): for vertex u of graph g,
//   S_u = sum over v in N(u), v != u, of est(|B_u AND B_v|)   (Eq. bf_int,
//         the same per-edge estimate as the edge pass; S_u is twice the
//         estimated triangles at u)
//   hist_g[|B_u AND B_v|] += 1 for every v > u   (each upper edge once)
// and from S_u directly lcc_u = S_u / (d_u (d_u - 1)) and tri_u = S_u / 2.
// S_u is an exact 128-bit sum of the table's fixed-point estimates, so it
// does not depend on the order of the adds or on the work mapping.
//
// Work order: 32-vertex groups (row r of a group is held by lane r), `chunk`
// consecutive groups per work chunk, chunks taken by the warps in order from
// a global counter, so that at any time the warps work inside a window of a
// few graphs whose sketch rows stay in L2 (a static round-robin deal let
// warps that met hub rows fall behind until the window outgrew L2). The last
// block to finish resets the counter for the next launch. A warp walks its group's entries (the rows are
// contiguous in the CSR) 32 at a time, one entry per lane with coalesced
// loads whatever the degrees: a 5-step search over the row ends held by the
// lanes gives each entry's row, and one inclusive warp scan of the 32
// fixed-point estimates gives each row its part of the step. Each warp keeps
// a shared-memory histogram for the graph it is in and flushes it (one
// global atomic per non-zero bin) when it moves to another graph.
constexpr int kPullThreads = 256;
constexpr int kPullWarps = kPullThreads / 32;

struct PullParams {
    const int32_t *row_ptr;
    const int32_t *col;
    int32_t v_lo, v_hi;              // the bucket's vertices
    const uint8_t *data;             // sketch rows addressed by global vertex id
    int64_t stride;
    uint32_t l;
    const unsigned long long *tabV;  // fixed-point estimates by popcount [l + 1]
    const int32_t *gid;
    const int64_t *hoff;
    unsigned long long *hist;        // per-graph histograms (zeroed before the pass)
    float *lcc;
    double *tri;                     // or null
    int32_t chunk;                   // groups per work chunk
    int32_t *queue;                  // [2]: next chunk, blocks done; zero between launches
};

// The W payload words of a sketch row (W = l / 32: 2 for 64-bit filters, whose
// 16-byte rows end in zero padding, else a multiple of 4).
template <int W>
struct Row {
    uint32_t w[W];
};

template <int W>
__device__ __forceinline__ Row<W> pull_row(const PullParams &p, int32_t v) {
    // a column naming a vertex outside the bucket (not a block-diagonal input) reads a row of the bucket
    v = min(max(v, p.v_lo), p.v_hi - 1);
    const uint8_t *src = p.data + (int64_t)v * p.stride;
    Row<W> r;
    if (W == 2) {
        const uint2 x = __ldg(reinterpret_cast<const uint2 *>(src));
        r.w[0] = x.x;
        r.w[1] = x.y;
    } else {
#pragma unroll
        for (int q = 0; q < W / 4; ++q) {
            const uint4 x = __ldg(reinterpret_cast<const uint4 *>(src) + q);
            r.w[4 * q] = x.x;
            r.w[4 * q + 1] = x.y;
            r.w[4 * q + 2] = x.z;
            r.w[4 * q + 3] = x.w;
        }
    }
    return r;
}

template <int W>
__device__ __forceinline__ uint32_t and_popc(const Row<W> &a, const Row<W> &b) {
    uint32_t c = 0;
#pragma unroll
    for (int q = 0; q < W; ++q) c += __popc(a.w[q] & b.w[q]);
    return c;
}

// 128-bit accumulator: lo + 2^64 hi.
__device__ __forceinline__ void acc_add(unsigned long long &lo, uint32_t &hi, unsigned long long x) {
    lo += x;
    hi += lo < x;
}

__device__ __forceinline__ void flush_hist(const PullParams &p, uint32_t *hw, int32_t g, unsigned lane) {
    __syncwarp();
    if (g >= 0) {
        unsigned long long *dst = p.hist + __ldg(p.hoff + g);
        for (uint32_t i = lane; i <= p.l; i += 32) {
            const uint32_t x = hw[i];
            if (x) {
                atomicAdd(dst + i, (unsigned long long)x);
                hw[i] = 0u;
            }
        }
    }
    __syncwarp();
}

template <int W>
__global__ void __launch_bounds__(kPullThreads) k_batch_pull(PullParams p) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int32_t len = (int32_t)p.l + 1;
    unsigned long long *tabV = reinterpret_cast<unsigned long long *>(smem);
    uint32_t *hw = reinterpret_cast<uint32_t *>(smem + 8 * (size_t)len) + (size_t)(threadIdx.x >> 5) * len;
    for (int32_t i = threadIdx.x; i < len; i += blockDim.x) tabV[i] = p.tabV[i];
    for (int32_t i = threadIdx.x; i < len * kPullWarps; i += blockDim.x)
        reinterpret_cast<uint32_t *>(smem + 8 * (size_t)len)[i] = 0u;
    __syncthreads();

    const unsigned lane = lane_id();
    const int64_t groups = ((int64_t)p.v_hi - p.v_lo + 31) / 32;
    const int64_t chunks = (groups + p.chunk - 1) / p.chunk;
    int32_t warp_g = -1;  // graph of the warp's shared histogram

    for (;;) {
        int32_t ch = 0;
        if (lane == 0) ch = atomicAdd(p.queue, 1);
        ch = __shfl_sync(0xffffffffu, ch, 0);
        if (ch >= chunks) break;
        for (int gi = 0; gi < p.chunk; ++gi) {
            const int64_t grp = (int64_t)ch * p.chunk + gi;
            if (grp >= groups) break;
            const int32_t v0 = p.v_lo + (int32_t)(grp * 32);
            const int32_t u = v0 + (int32_t)lane;
            const bool valid = u < p.v_hi;
            // lanes past the bucket hold empty rows at its end
            const int32_t a = __ldg(p.row_ptr + min(u, p.v_hi));
            const int32_t e = __ldg(p.row_ptr + min(u + 1, p.v_hi));
            const int32_t g = valid ? __ldg(p.gid + u) : -1;
            // the group's first vertex decides the warp's histogram graph (a group spans at
            // most a graph boundary or two; the other graph's entries go to global memory)
            const int32_t g0 = __shfl_sync(0xffffffffu, g, 0);
            if (g0 != warp_g) {
                flush_hist(p, hw, warp_g, lane);
                warp_g = g0;
            }
            const int32_t x_lo = __shfl_sync(0xffffffffu, a, 0), x_hi = __shfl_sync(0xffffffffu, e, 31);
            unsigned long long lo = 0ull;
            uint32_t hi = 0u;
            for (int32_t x0 = x_lo; x0 < x_hi; x0 += 32) {
                const int32_t x = x0 + (int32_t)lane;
                const bool live = x < x_hi;
                // the id load is issued before the row search that it does not depend on
                const int32_t cx = live ? __ldg(p.col + x) : 0;
                // row of entry x: the number of rows (lanes) ending at or before x
                int r = 0;
#pragma unroll
                for (int step = 16; step >= 1; step >>= 1) {
                    const int32_t er = __shfl_sync(0xffffffffu, e, r + step - 1);
                    if (er <= x) r += step;
                }
                const int32_t ur = v0 + r;
                const int32_t v = live ? cx : ur;
                const uint32_t c = and_popc<W>(pull_row<W>(p, ur), pull_row<W>(p, v));
                unsigned long long V = (v != ur) ? tabV[c] : 0ull;
                const int32_t gr = __shfl_sync(0xffffffffu, g, r);
                if (v > ur) {
                    if (gr == warp_g) atomicAdd(hw + c, 1u);
                    else atomicAdd(p.hist + __ldg(p.hoff + gr) + c, 1ull);
                }
                // inclusive scan of the 32 estimates (each below 2^57, so no step overflows)
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const unsigned long long y = __shfl_up_sync(0xffffffffu, V, o);
                    if ((int)lane >= o) V += y;
                }
                // this lane's row: entries [first, last] of the step
                const int first = max(a, x0) - x0, last = min(e, x0 + 32) - x0 - 1;
                const unsigned long long s_hi = __shfl_sync(0xffffffffu, V, min(max(last, 0), 31));
                const unsigned long long s_lo = __shfl_sync(0xffffffffu, V, min(max(first - 1, 0), 31));
                if (first <= last) acc_add(lo, hi, s_hi - (first > 0 ? s_lo : 0ull));
            }
            if (valid) {
                const int32_t d = e - a;
                double S, half;
                if (hi == 0u) {
                    S = fixed_to_f64(lo, kFixBits);
                    half = fixed_to_f64(lo, kFixBits + 1);
                } else {  // sums of 2^22 or more (double arithmetic, rare)
                    S = (double)hi * 0x1p22 + (double)lo * 0x1p-42;
                    half = 0.5 * S;
                }
                p.lcc[u] = d >= 2 ? (float)S / ((float)d * (float)(d - 1)) : 0.0f;
                if (p.tri) p.tri[u] = half;
            }
        }
    }
    flush_hist(p, hw, warp_g, lane);
    // every warp of every block has left the loop once the last block gets here: reset the queue
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(p.queue + 1, 1) == (int)gridDim.x - 1) {
            p.queue[0] = 0;
            p.queue[1] = 0;
        }
    }
}

template <int W>
cudaError_t run_pull(const PullParams &p, cudaStream_t s) {
    const size_t smem = 8 * (size_t)(p.l + 1) + 4 * (size_t)(p.l + 1) * kPullWarps;
    auto kern = k_batch_pull<W>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kPullThreads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    kern<<<per_sm * device_info().sm_count, kPullThreads, smem, s>>>(p);
    note_launch();
    return cudaGetLastError();
}

// ------------------------------------------------------------ Bloom build
// The Bloom filters of a bucket's vertices, with the pull pass's work order
// and walk: a warp takes 32 consecutive rows, builds their filters in its
// shared memory (row r at [r * words, (r + 1) * words)) from the rows'
// entries taken 32 at a time (coalesced loads, one entry per lane, its row
// from the search over the row ends), and stores the 32 filters with one
// coalesced row store per lane. Every graph hashes its own ids (global id
// minus the graph's first id) with the bucket's b hash functions, so the
// filter bits are those of the single-graph build (Sec. II-D: bit
// floor(h_i(x) l / 2^32) for each element x and i < b); OR does not depend
// on the order in which entries are hashed.
struct BuildParams {
    const int32_t *row_ptr;
    const int32_t *col;
    int32_t v_lo, v_hi;
    const int32_t *gid;
    const int32_t *voff;
    uint8_t *data;       // rows addressed by global vertex id
    int64_t stride;
    uint32_t l, b, seed;
    int32_t chunk;
};

// B: the bucket's hash count fixed at compile time (1 or 2), or 0 to read p.b.
template <int WORDS, int B>  // WORDS: 32-bit words per stored row (stride / 4)
__global__ void __launch_bounds__(kPullThreads) k_batch_bloom(BuildParams p) {
    __shared__ uint32_t filt[kPullWarps][32 * WORDS];
    __shared__ uint32_t pre_s[16];
    if (threadIdx.x < 16) pre_s[threadIdx.x] = fmix_pre(hash_seed(p.seed, threadIdx.x));
    const unsigned lane = lane_id();
    uint32_t *f = filt[threadIdx.x >> 5];
    for (int i = (int)lane; i < 32 * WORDS; i += 32) f[i] = 0u;
    __syncthreads();
    const int64_t warp = ((int64_t)blockIdx.x * kPullThreads + threadIdx.x) >> 5;
    const int64_t warps = (int64_t)gridDim.x * kPullWarps;
    const int64_t groups = ((int64_t)p.v_hi - p.v_lo + 31) / 32;
    const int64_t chunks = (groups + p.chunk - 1) / p.chunk;
    for (int64_t ch = warp; ch < chunks; ch += warps) {
        for (int gi = 0; gi < p.chunk; ++gi) {
            const int64_t grp = ch * p.chunk + gi;
            if (grp >= groups) break;
            const int32_t v0 = p.v_lo + (int32_t)(grp * 32);
            const int32_t u = v0 + (int32_t)lane;
            const bool valid = u < p.v_hi;
            const int32_t a = __ldg(p.row_ptr + min(u, p.v_hi));
            const int32_t e = __ldg(p.row_ptr + min(u + 1, p.v_hi));
            const int32_t id0 = valid ? __ldg(p.voff + __ldg(p.gid + u)) : 0;
            const int32_t x_lo = __shfl_sync(0xffffffffu, a, 0), x_hi = __shfl_sync(0xffffffffu, e, 31);
            for (int32_t x0 = x_lo; x0 < x_hi; x0 += 32) {
                const int32_t x = x0 + (int32_t)lane;
                // the id load is issued before the row search that it does not depend on
                const int32_t cx = x < x_hi ? __ldg(p.col + x) : 0;
                int r = 0;
#pragma unroll
                for (int step = 16; step >= 1; step >>= 1) {
                    const int32_t er = __shfl_sync(0xffffffffu, e, r + step - 1);
                    if (er <= x) r += step;
                }
                const int32_t idr = __shfl_sync(0xffffffffu, id0, r);
                if (x < x_hi) {
                    const uint32_t px = fmix_pre((uint32_t)(cx - idr));
                    uint32_t *fr = f + r * WORDS;
                    if (B > 0) {
#pragma unroll
                        for (int i = 0; i < B; ++i) {
                            const uint32_t q = bit_pos(hash_pre(px, pre_s[i]), p.l);
                            atomicOr(fr + (q >> 5), 1u << (q & 31u));
                        }
                    } else {
                        for (uint32_t i = 0; i < p.b; ++i) {
                            const uint32_t q = bit_pos(hash_pre(px, pre_s[i]), p.l);
                            atomicOr(fr + (q >> 5), 1u << (q & 31u));
                        }
                    }
                }
            }
            __syncwarp();
            // lane r stores row r (padding words stay zero) and clears it
            uint32_t *fr = f + lane * WORDS;
            if (valid) {
                uint4 *dst = reinterpret_cast<uint4 *>(p.data + (int64_t)u * p.stride);
#pragma unroll
                for (int q = 0; q < WORDS / 4; ++q)
                    dst[q] = make_uint4(fr[4 * q], fr[4 * q + 1], fr[4 * q + 2], fr[4 * q + 3]);
            }
#pragma unroll
            for (int w = 0; w < WORDS; ++w) fr[w] = 0u;
            __syncwarp();
        }
    }
}

template <int WORDS, int B>
cudaError_t run_batch_bloom_b(const BuildParams &p, cudaStream_t s) {
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_bloom<WORDS, B>, kPullThreads, 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    k_batch_bloom<WORDS, B><<<per_sm * device_info().sm_count, kPullThreads, 0, s>>>(p);
    note_launch();
    return cudaGetLastError();
}

// A launch covers graphs of one bucket, which share the hash count p.b.
template <int WORDS>
cudaError_t run_batch_bloom(const BuildParams &p, cudaStream_t s) {
    if (p.b == 1) return run_batch_bloom_b<WORDS, 1>(p, s);
    if (p.b == 2) return run_batch_bloom_b<WORDS, 2>(p, s);
    return run_batch_bloom_b<WORDS, 0>(p, s);
}

// Groups of 32 rows per warp chunk of the build.
constexpr int32_t kBuildChunk = 4;
// Buckets of at most this many bits use k_batch_bloom; wider filters use the
// single-graph builder (lane-private filters for short rows, hub rows split
// across blocks), which was faster there: at 512 bits the few large graphs
// of a bucket leave the flat walk too few groups and long rows to one warp.
constexpr uint32_t kFlatBuildMaxBits = 64;

// Variant v of the pull pass: v consecutive 32-vertex groups per warp chunk
// (the autotuner's candidates below; a caller may set any v up to
// kMaxPullVariant).
constexpr int32_t kPullVariants[] = {1, 4, 16};
constexpr int32_t kMaxPullVariant = 1024;

__global__ void k_graph_ids(const int32_t *__restrict__ voff, int32_t graphs, int32_t *__restrict__ gid) {
    // one block per graph writes its vertex range
    for (int32_t g = blockIdx.x; g < graphs; g += gridDim.x)
        for (int32_t v = voff[g] + threadIdx.x; v < voff[g + 1]; v += blockDim.x) gid[v] = g;
}

struct Bucket {
    int32_t g_lo, g_hi;  // graphs
    int32_t v_lo, v_hi;  // vertices
    uint32_t bits, b;
    int32_t variant;
    int64_t stride;
    uint8_t *data;       // rows of v_lo .. v_hi - 1
    double *table;
};

}  // namespace
}  // namespace pg

struct pg_batch {
    pg_csr g;
    int32_t graphs;
    uint32_t seed;
    int32_t *gid;
    int32_t *voff;
    int64_t *hoff;
    uint32_t *bits_of;
    uint8_t *b_of;
    uint64_t *hist;
    int64_t hist_bins;
    int32_t *hub;
    int32_t *queue;  // work counter of the pull pass
    pg_tc_result *tc_out;
    float *lcc_out;
    double *tri_out;
    std::vector<pg::Bucket> buckets;
    std::vector<int32_t> voff_h;  // host copy of voff
    cudaGraph_t graph;
    cudaGraphExec_t exec;
    cudaStream_t captured_on;
};

using namespace pg;

namespace {

// Expected absolute error of the AND estimator (Eq. bf_int) for two
// neighbourhoods of size d sharing t = ceil(d / 10) elements, in an l-bit
// filter with b hash functions: bias of the estimate at the expected
// popcount (common elements set their bits; private elements collide) plus
// the MSE bound of Prop. 4.1.
double and_error_model(double d, double l, double b) {
    const double t = std::ceil(d / 10.0);
    const double pc = std::pow(1.0 - 1.0 / l, b * t);        // bit untouched by the common part
    const double pp = std::pow(1.0 - 1.0 / l, b * (d - t));  // bit untouched by one private part
    const double ones = l * (1.0 - pc + pc * (1.0 - pp) * (1.0 - pp));
    double B1 = std::min(ones, l - 1.0);
    const double est = -(l / b) * std::log(1.0 - B1 / l);
    const double bias = est - t;
    double mse = std::exp(t * b / (l - 1.0)) * l / (b * b) - l / (b * b) - t / b;
    if (mse < 0.0) mse = 0.0;
    return std::sqrt(bias * bias + mse);
}

uint32_t budget_bits_pow2(double s, int64_t n, int64_t nnz) {
    if (n <= 0) return 64;
    const double csr = 4.0 * (double)(n + 1) + 4.0 * (double)nnz;
    double bits = s * csr * 8.0 / (double)n;
    uint32_t l = 64;
    while (l * 2 <= bits && l < 1024) l *= 2;
    return l;
}

// Carve the workspace (base == nullptr: only size it). Order: graph tables,
// histograms, build scratch, then per bucket its estimator table and sketch
// rows.
size_t carve_batch(const pg_csr *g, int32_t graphs, const pg_batch_config *cfg, std::vector<Bucket> &buckets,
                   uint8_t *base, pg_batch *out) {
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += round_up(bytes, 256);
        return base + o;
    };
    int64_t bins = 0;
    for (int32_t i = 0; i < graphs; ++i) bins += (int64_t)cfg[i].bits + 1;
    uint8_t *gid = take(4 * (size_t)g->n + 4);
    uint8_t *voff = take(4 * ((size_t)graphs + 1));
    uint8_t *hoff = take(8 * ((size_t)graphs + 1));
    uint8_t *bits = take(4 * (size_t)graphs + 4);
    uint8_t *b = take((size_t)graphs + 4);
    uint8_t *hist = take(8 * (size_t)bins + 8);
    uint8_t *hub = take(build_workspace_bytes(g->nnz));
    uint8_t *queue = take(16);
    for (Bucket &bk : buckets) {
        uint8_t *table = take(intersect_table_bytes(PG_SK_BLOOM, bk.bits, 0));
        uint8_t *data = take((size_t)(bk.v_hi - bk.v_lo) * (size_t)bk.stride + 16);
        if (base) {
            bk.table = reinterpret_cast<double *>(table);
            bk.data = data;
        }
    }
    if (base && out) {
        out->gid = reinterpret_cast<int32_t *>(gid);
        out->voff = reinterpret_cast<int32_t *>(voff);
        out->hoff = reinterpret_cast<int64_t *>(hoff);
        out->bits_of = reinterpret_cast<uint32_t *>(bits);
        out->b_of = b;
        out->hist = reinterpret_cast<uint64_t *>(hist);
        out->hist_bins = bins;
        out->hub = reinterpret_cast<int32_t *>(hub);
        out->queue = reinterpret_cast<int32_t *>(queue);
    }
    return off;
}

// Group contiguous runs of equal (bits, b); every key must form one run.
pg_status make_buckets(int32_t graphs, const int32_t *voff_host, const pg_batch_config *cfg,
                       std::vector<Bucket> &out) {
    out.clear();
    for (int32_t i = 0; i < graphs; ++i) {
        const uint32_t bits = cfg[i].bits, b = cfg[i].b;
        PG_REQUIRE(bits == 64 || bits == 128 || bits == 256 || bits == 512 || bits == 1024, PG_ERR_UNSUPPORTED,
                   "graph %d: batch Bloom bits %u not in {64, 128, 256, 512, 1024}", i, bits);
        PG_REQUIRE(b >= 1 && b <= 16, PG_ERR_INVALID_ARG, "graph %d: b = %u not in [1, 16]", i, b);
        PG_REQUIRE(cfg[i].variant >= 0 && cfg[i].variant <= kMaxPullVariant, PG_ERR_INVALID_ARG,
                   "graph %d: variant %d not in [0, %d]", i, cfg[i].variant, kMaxPullVariant);
        PG_REQUIRE(voff_host[i + 1] >= voff_host[i], PG_ERR_INVALID_ARG, "voff not non-decreasing at %d", i);
        if (!out.empty() && out.back().bits == bits && out.back().b == b) {
            out.back().g_hi = i + 1;
            out.back().v_hi = voff_host[i + 1];
            continue;
        }
        for (const Bucket &bk : out)
            PG_REQUIRE(!(bk.bits == bits && bk.b == b), PG_ERR_INVALID_ARG,
                       "graphs with bits %u, b %u are not contiguous (order the graphs by bucket)", bits, b);
        Bucket bk{};
        bk.g_lo = i;
        bk.g_hi = i + 1;
        bk.v_lo = voff_host[i];
        bk.v_hi = voff_host[i + 1];
        bk.bits = bits;
        bk.b = b;
        bk.variant = cfg[i].variant;
        bk.stride = pg_sketch_stride(PG_SK_BLOOM, bits, 0);
        out.push_back(bk);
    }
    return PG_OK;
}

// Launches over the vertices [va, vb) of bucket bk (whole graphs).
cudaError_t launch_batch_bloom(const pg_batch *bt, const Bucket &bk, int32_t va, int32_t vb, cudaStream_t s) {
    BuildParams p{};
    p.row_ptr = bt->g.row_ptr;
    p.col = bt->g.col;
    p.v_lo = va;
    p.v_hi = vb;
    p.gid = bt->gid;
    p.voff = bt->voff;
    p.data = bk.data - (int64_t)bk.v_lo * bk.stride;
    p.stride = bk.stride;
    p.l = bk.bits;
    p.b = bk.b;
    p.seed = bt->seed;
    p.chunk = kBuildChunk;
    switch (bk.stride / 4) {
        case 4: return run_batch_bloom<4>(p, s);
        case 8: return run_batch_bloom<8>(p, s);
        case 16: return run_batch_bloom<16>(p, s);
        case 32: return run_batch_bloom<32>(p, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_build_range(const pg_batch *bt, const Bucket &bk, int32_t va, int32_t vb, cudaStream_t s) {
    if (bk.bits <= kFlatBuildMaxBits) return launch_batch_bloom(bt, bk, va, vb, s);
    BatchMap bm{bt->gid, bt->voff, bt->b_of, va};
    return launch_build_bloom(bt->g.row_ptr + va, bt->g.col, vb - va, bk.bits, bk.b, bt->seed,
                              bk.data + (int64_t)(va - bk.v_lo) * bk.stride, bk.stride, bt->hub, s, &bm);
}

pg_status enqueue_builds(pg_batch *bt, cudaStream_t s) {
    for (const Bucket &bk : bt->buckets) {
        if (bk.v_hi <= bk.v_lo) continue;
        PG_TRY_CUDA(launch_build_range(bt, bk, bk.v_lo, bk.v_hi, s), "pg_batch: Bloom build");
    }
    return PG_OK;
}

cudaError_t launch_pull(const pg_batch *bt, const Bucket &bk, int32_t variant, int32_t va, int32_t vb,
                        cudaStream_t s) {
    PullParams p{};
    p.row_ptr = bt->g.row_ptr;
    p.col = bt->g.col;
    p.v_lo = va;
    p.v_hi = vb;
    p.data = bk.data - (int64_t)bk.v_lo * bk.stride;
    p.stride = bk.stride;
    p.l = bk.bits;
    p.tabV = reinterpret_cast<const unsigned long long *>(bk.table + (bk.bits + 1));
    p.gid = bt->gid;
    p.hoff = bt->hoff;
    p.hist = reinterpret_cast<unsigned long long *>(bt->hist);
    p.lcc = bt->lcc_out;
    p.tri = bt->tri_out;
    p.chunk = variant;
    p.queue = bt->queue;
    switch (bk.bits) {
        case 64: return run_pull<2>(p, s);
        case 128: return run_pull<4>(p, s);
        case 256: return run_pull<8>(p, s);
        case 512: return run_pull<16>(p, s);
        case 1024: return run_pull<32>(p, s);
        default: return cudaErrorInvalidValue;
    }
}

// The estimator table of every bucket (double | fixed point | float by popcount).
pg_status enqueue_tables(pg_batch *bt, cudaStream_t s) {
    for (const Bucket &bk : bt->buckets) {
        if (bk.v_hi <= bk.v_lo) continue;
        PG_TRY_CUDA(launch_estimator_table(bk.table, PG_SK_BLOOM, PG_EST_BF_AND, bk.bits, bk.b, 0, s),
                    "pg_batch: estimator table");
    }
    return PG_OK;
}

pg_status enqueue_passes(pg_batch *bt, cudaStream_t s) {
    launch_fill_u64(bt->hist, (size_t)bt->hist_bins, 0, s);
    for (const Bucket &bk : bt->buckets) {
        if (bk.v_hi <= bk.v_lo) continue;
        PG_TRY_CUDA(launch_pull(bt, bk, bk.variant, bk.v_lo, bk.v_hi, s), "pg_batch: pass");
    }
    PG_TRY_CUDA(launch_batch_finalize(bt->hist, bt->hoff, bt->bits_of, bt->b_of, bt->graphs, PG_EST_BF_AND,
                                      bt->tc_out, s),
                "pg_batch: TC");
    return PG_OK;
}

}  // namespace

extern "C" {

pg_status pg_batch_autotune(const int32_t *n_host, const int64_t *nnz_host, int32_t graphs, double budget,
                            pg_batch_config *cfg_host) {
    PG_REQUIRE(graphs >= 0 && (graphs == 0 || (n_host && nnz_host && cfg_host)), PG_ERR_INVALID_ARG,
               "pg_batch_autotune: bad arguments");
    PG_REQUIRE(budget > 0.0, PG_ERR_INVALID_ARG, "pg_batch_autotune: budget must be positive");
    for (int32_t i = 0; i < graphs; ++i) {
        const uint32_t l = budget_bits_pow2(budget, n_host[i], nnz_host[i]);
        const double d = n_host[i] > 0 ? (double)nnz_host[i] / (double)n_host[i] : 0.0;
        uint32_t best_b = 1;
        double best = 1e300;
        for (uint32_t b : {1u, 2u, 4u}) {
            const double err = and_error_model(std::max(d, 1.0), (double)l, (double)b);
            if (err < best - 1e-12) {
                best = err;
                best_b = b;
            }
        }
        cfg_host[i].bits = l;
        cfg_host[i].b = best_b;
        cfg_host[i].variant = 0;
        cfg_host[i].reserved = 0;
    }
    return PG_OK;
}

size_t pg_batch_workspace_bytes(const pg_csr *g, int32_t graphs, const int32_t *voff_host,
                                const pg_batch_config *cfg_host) {
    if (!g || graphs < 1 || !voff_host || !cfg_host) return 0;
    // the row walks step a 32-bit entry index by 32 past the last entry
    if (g->nnz > (int64_t)INT32_MAX - 64) {
        set_error(PG_ERR_TOO_LARGE, "pg_batch: nnz %lld above %d", (long long)g->nnz, INT32_MAX - 64);
        return 0;
    }
    std::vector<Bucket> buckets;
    if (make_buckets(graphs, voff_host, cfg_host, buckets) != PG_OK) return 0;
    return carve_batch(g, graphs, cfg_host, buckets, nullptr, nullptr);
}

pg_status pg_batch_create(const pg_csr *g, int32_t graphs, const int32_t *voff_host,
                          pg_batch_config *cfg_host, uint32_t seed, void *workspace, size_t workspace_bytes,
                          pg_tc_result *tc_out, float *lcc_out, double *tri_out, pg_stream_t stream,
                          pg_batch **out) {
    PG_TRACE("pg_batch_create");
    pg_status st = check_graph(g);
    if (st) return st;
    PG_REQUIRE(out != nullptr, PG_ERR_INVALID_ARG, "pg_batch_create: out is NULL");
    PG_REQUIRE(graphs >= 1 && voff_host && cfg_host, PG_ERR_INVALID_ARG, "pg_batch_create: no graphs");
    PG_REQUIRE(graphs < (1 << 21), PG_ERR_TOO_LARGE, "pg_batch_create: %d graphs, at most %d", graphs,
               (1 << 21) - 1);
    PG_REQUIRE(voff_host[0] == 0 && voff_host[graphs] == g->n, PG_ERR_INVALID_ARG,
               "pg_batch_create: voff must run from 0 to n");
    PG_REQUIRE(tc_out && lcc_out, PG_ERR_INVALID_ARG, "pg_batch_create: tc_out and lcc_out are required");
    PG_REQUIRE(workspace && aligned16(workspace), PG_ERR_INVALID_ARG, "pg_batch_create: bad workspace");
    const size_t need = pg_batch_workspace_bytes(g, graphs, voff_host, cfg_host);
    PG_REQUIRE(need > 0, PG_ERR_INVALID_ARG, "pg_batch_create: %s", pg_last_error());
    PG_REQUIRE(workspace_bytes >= need, PG_ERR_NO_MEMORY, "pg_batch_create: workspace has %zu bytes, needs %zu",
               workspace_bytes, need);
    pg_batch *bt = new pg_batch();
    bt->g = *g;
    bt->graphs = graphs;
    bt->seed = seed;
    bt->tc_out = tc_out;
    bt->lcc_out = lcc_out;
    bt->tri_out = tri_out;
    st = make_buckets(graphs, voff_host, cfg_host, bt->buckets);
    if (st) {
        delete bt;
        return st;
    }
    carve_batch(g, graphs, cfg_host, bt->buckets, static_cast<uint8_t *>(workspace), bt);
    bt->voff_h.assign(voff_host, voff_host + graphs + 1);
    // host tables -> device
    std::vector<int64_t> hoff(graphs + 1);
    std::vector<uint32_t> bits(graphs);
    std::vector<uint8_t> bs(graphs);
    hoff[0] = 0;
    for (int32_t i = 0; i < graphs; ++i) {
        hoff[i + 1] = hoff[i] + cfg_host[i].bits + 1;
        bits[i] = cfg_host[i].bits;
        bs[i] = (uint8_t)cfg_host[i].b;
    }
    cudaStream_t s = stream;
    cudaError_t e = cudaMemcpyAsync(bt->voff, voff_host, 4 * ((size_t)graphs + 1), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(bt->hoff, hoff.data(), 8 * hoff.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(bt->bits_of, bits.data(), 4 * bits.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(bt->b_of, bs.data(), bs.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(bt->queue, 0, 16, s);
    if (e == cudaSuccess) {
        k_graph_ids<<<std::min(graphs, 4096), 256, 0, s>>>(bt->voff, graphs, bt->gid);
        note_launch();
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // host vectors above die with this call
    if (e != cudaSuccess) {
        delete bt;
        return cuda_status(e, "pg_batch_create");
    }
    // The estimator tables depend only on (l, b): computed once here.
    st = enqueue_tables(bt, s);
    if (st) {
        delete bt;
        return st;
    }
    // Autotune the lane/warp split of every bucket whose variant is 0: build
    // once, time each candidate pass on the bucket and keep the fastest.
    bool tune = false;
    for (const Bucket &bk : bt->buckets) tune |= bk.variant == 0;
    if (tune) {
        st = enqueue_builds(bt, s);
        if (st) {
            delete bt;
            return st;
        }
        cudaEvent_t a, b;
        cudaEventCreate(&a);
        cudaEventCreate(&b);
        for (size_t bi = 0; bi < bt->buckets.size(); ++bi) {
            Bucket &bk = bt->buckets[bi];
            if (bk.variant != 0) continue;
            float best = 1e30f;
            int32_t best_v = kPullVariants[0];
            for (int32_t cand : kPullVariants) {
                for (int rep = 0; rep < 2; ++rep) {  // first run warms up
                    cudaEventRecord(a, s);
                    e = launch_pull(bt, bk, cand, bk.v_lo, bk.v_hi, s);
                    cudaEventRecord(b, s);
                    if (e == cudaSuccess) e = cudaEventSynchronize(b);
                    if (e != cudaSuccess) break;
                    float ms = 0.0f;
                    cudaEventElapsedTime(&ms, a, b);
                    if (rep == 1 && ms < best) {
                        best = ms;
                        best_v = cand;
                    }
                }
                if (e != cudaSuccess) break;
            }
            if (e != cudaSuccess) break;
            bk.variant = best_v;
            for (int32_t i = bk.g_lo; i < bk.g_hi; ++i) cfg_host[i].variant = best_v;
        }
        cudaEventDestroy(a);
        cudaEventDestroy(b);
        if (e != cudaSuccess) {
            delete bt;
            return cuda_status(e, "pg_batch_create: autotune");
        }
    }
    *out = bt;
    return PG_OK;
}

pg_status pg_batch_run(pg_batch *bt, pg_stream_t stream) {
    PG_TRACE("pg_batch_run");
    PG_REQUIRE(bt != nullptr, PG_ERR_INVALID_ARG, "pg_batch_run: batch is NULL");
    cudaStream_t s = stream;
    if (s == nullptr) {  // the legacy default stream cannot be captured: run eagerly
        pg_status st = enqueue_builds(bt, s);
        if (st) return st;
        return enqueue_passes(bt, s);
    }
    if (bt->exec == nullptr || bt->captured_on != s) {
        if (bt->exec) {
            cudaGraphExecDestroy(bt->exec);
            cudaGraphDestroy(bt->graph);
            bt->exec = nullptr;
        }
        PG_TRY_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed), "pg_batch_run: begin capture");
        pg_status st = enqueue_builds(bt, s);
        if (st == PG_OK) st = enqueue_passes(bt, s);
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamEndCapture(s, &graph);
        if (st) {
            if (graph) cudaGraphDestroy(graph);
            return st;
        }
        PG_TRY_CUDA(e, "pg_batch_run: end capture");
        e = cudaGraphInstantiate(&bt->exec, graph, 0);
        if (e != cudaSuccess) {
            cudaGraphDestroy(graph);
            return cuda_status(e, "pg_batch_run: instantiate");
        }
        bt->graph = graph;
        bt->captured_on = s;
    }
    PG_TRY_CUDA(cudaGraphLaunch(bt->exec, s), "pg_batch_run: launch");
    note_launch();
    return PG_OK;
}

pg_status pg_batch_run_host(pg_batch *bt, const int32_t *host_row_ptr, const int32_t *host_col,
                            int64_t chunk_entries, pg_stream_t copy_stream, pg_stream_t stream) {
    PG_TRACE("pg_batch_run_host");
    PG_REQUIRE(bt != nullptr, PG_ERR_INVALID_ARG, "pg_batch_run_host: batch is NULL");
    const pg_csr &g = bt->g;
    PG_REQUIRE(host_row_ptr != nullptr && (g.nnz == 0 || host_col != nullptr), PG_ERR_INVALID_ARG,
               "pg_batch_run_host: host CSR is NULL");
    PG_REQUIRE(chunk_entries > 0, PG_ERR_INVALID_ARG, "pg_batch_run_host: chunk_entries must be positive");
    PG_REQUIRE(host_row_ptr[0] == 0 && (int64_t)host_row_ptr[g.n] == g.nnz, PG_ERR_INVALID_ARG,
               "pg_batch_run_host: host row_ptr must run from 0 to nnz");
    // the batch's device CSR is this call's upload target (pg_csr holds it as const for the readers)
    int32_t *dst_rp = const_cast<int32_t *>(g.row_ptr);
    int32_t *dst_col = const_cast<int32_t *>(g.col);
    cudaStream_t cs = copy_stream, s = stream;
    cudaEvent_t ev_start = nullptr, ev_chunk = nullptr;
    PG_TRY_CUDA(cudaEventCreateWithFlags(&ev_start, cudaEventDisableTiming), "pg_batch_run_host: event");
    cudaError_t e = cudaEventCreateWithFlags(&ev_chunk, cudaEventDisableTiming);
    // the upload overwrites the device CSR: it starts after the work already on the compute stream
    if (e == cudaSuccess) e = cudaEventRecord(ev_start, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, ev_start, 0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dst_rp, host_row_ptr, 4 * ((size_t)g.n + 1), cudaMemcpyDefault, cs);
    if (e == cudaSuccess) {
        launch_fill_u64(bt->hist, (size_t)bt->hist_bins, 0, s);
        e = cudaGetLastError();
    }
    const std::vector<int32_t> &vo = bt->voff_h;
    for (const Bucket &bk : bt->buckets) {
        // chunks of whole graphs of the bucket, about chunk_entries CSR entries each (at least one graph)
        for (int32_t g0 = bk.g_lo; e == cudaSuccess && g0 < bk.g_hi;) {
            const int64_t x0 = host_row_ptr[vo[g0]];
            int32_t g1 = g0 + 1;
            while (g1 < bk.g_hi && (int64_t)host_row_ptr[vo[g1 + 1]] - x0 <= chunk_entries) ++g1;
            const int32_t va = vo[g0], vb = vo[g1];
            const int64_t x1 = host_row_ptr[vb];
            if (x1 > x0)
                e = cudaMemcpyAsync(dst_col + x0, host_col + x0, 4 * (size_t)(x1 - x0), cudaMemcpyDefault, cs);
            if (e == cudaSuccess) e = cudaEventRecord(ev_chunk, cs);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ev_chunk, 0);
            if (e == cudaSuccess && vb > va) e = launch_build_range(bt, bk, va, vb, s);
            if (e == cudaSuccess && vb > va) e = launch_pull(bt, bk, bk.variant, va, vb, s);
            g0 = g1;
        }
    }
    // the buckets cover every graph (voff runs from 0 to n), so the chunks copied all of col;
    // order the stream after the whole upload
    if (e == cudaSuccess) e = cudaEventRecord(ev_chunk, cs);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ev_chunk, 0);
    if (e == cudaSuccess)
        e = launch_batch_finalize(bt->hist, bt->hoff, bt->bits_of, bt->b_of, bt->graphs, PG_EST_BF_AND, bt->tc_out,
                                  s);
    cudaEventDestroy(ev_start);
    if (ev_chunk) cudaEventDestroy(ev_chunk);
    PG_TRY_CUDA(e, "pg_batch_run_host");
    return PG_OK;
}

pg_status pg_batch_destroy(pg_batch *bt) {
    if (!bt) return PG_OK;
    if (bt->exec) cudaGraphExecDestroy(bt->exec);
    if (bt->graph) cudaGraphDestroy(bt->graph);
    delete bt;
    return PG_OK;
}

}  // extern "C"

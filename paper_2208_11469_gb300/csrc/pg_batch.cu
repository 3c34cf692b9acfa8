// Batched analysis of many small graphs in one CUDA-graph launch.
//
// The G graphs are one block-diagonal CSR ("union graph", global vertex ids;
// graph g owns vertices [voff[g], voff[g+1])). Each graph gets its own Bloom
// parameters (l, b) and kernel variant; graphs with equal (l, b) must be
// contiguous ("buckets"). One run is
//   upper-edge index of the union graph
//   -> per bucket: Bloom build of its vertex range (hashing each graph's own
//      ids, so a sketch is the same alone and in the batch)
//   -> per bucket: fused Bloom pass (per-graph popcount histograms, per-vertex
//      sums)
//   -> LCC of every vertex, and per graph the histogram dot (TC estimate).
// The first pg_batch_run on a non-default stream captures this sequence into
// a CUDA graph; later runs replay it with one launch.
//
// The autotuner (pg_batch_autotune) picks per graph the filter length from
// the storage budget (Sec. V-A), the hash count from an accuracy model of the
// AND estimator (Eq. bf_int), and pg_batch_create times the lane mappings
// available for each bucket's width on the bucket itself and keeps the
// fastest.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "pg_internal.cuh"

namespace pg {
namespace {

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
    void *index;
    int32_t *gid;
    int32_t *voff;
    int64_t *hoff;
    uint32_t *bits_of;
    uint8_t *b_of;
    uint64_t *hist;
    int64_t hist_bins;
    double *S;
    int32_t *hub;
    pg_tc_result *tc_out;
    float *lcc_out;
    double *tri_out;
    std::vector<pg::Bucket> buckets;
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

// Carve the workspace (base == nullptr: only size it). Order: edge index,
// graph tables, histograms, per-vertex sums, build scratch, then per bucket
// its estimator table and sketch rows.
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
    uint8_t *index = take(upper_index_bytes(g->n, g->nnz));
    uint8_t *gid = take(4 * (size_t)g->n + 4);
    uint8_t *voff = take(4 * ((size_t)graphs + 1));
    uint8_t *hoff = take(8 * ((size_t)graphs + 1));
    uint8_t *bits = take(4 * (size_t)graphs + 4);
    uint8_t *b = take((size_t)graphs + 4);
    uint8_t *hist = take(8 * (size_t)bins + 8);
    uint8_t *S = take(8 * (size_t)g->n + 8);
    uint8_t *hub = take(build_workspace_bytes(g->nnz));
    for (Bucket &bk : buckets) {
        uint8_t *table = take(intersect_table_bytes(PG_SK_BLOOM, bk.bits, 0));
        uint8_t *data = take((size_t)(bk.v_hi - bk.v_lo) * (size_t)bk.stride + 16);
        if (base) {
            bk.table = reinterpret_cast<double *>(table);
            bk.data = data;
        }
    }
    if (base && out) {
        out->index = index;
        out->gid = reinterpret_cast<int32_t *>(gid);
        out->voff = reinterpret_cast<int32_t *>(voff);
        out->hoff = reinterpret_cast<int64_t *>(hoff);
        out->bits_of = reinterpret_cast<uint32_t *>(bits);
        out->b_of = b;
        out->hist = reinterpret_cast<uint64_t *>(hist);
        out->hist_bins = bins;
        out->S = reinterpret_cast<double *>(S);
        out->hub = reinterpret_cast<int32_t *>(hub);
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

pg_sketch bucket_sketch(const pg_batch *bt, const Bucket &bk) {
    pg_sketch sk{};
    sk.kind = PG_SK_BLOOM;
    sk.bits = bk.bits;
    sk.b = bk.b;
    sk.seed = bt->seed;
    sk.n = bt->g.n;
    sk.stride_bytes = bk.stride;
    // rows are addressed by global vertex id; the bucket's rows start at v_lo
    sk.data = bk.data - (int64_t)bk.v_lo * bk.stride;
    return sk;
}

pg_status enqueue_builds(pg_batch *bt, cudaStream_t s) {
    PG_TRY_CUDA(launch_upper_index(bt->g.row_ptr, bt->g.col, bt->g.n, bt->g.nnz, bt->index, s),
                "pg_batch: edge index");
    for (const Bucket &bk : bt->buckets) {
        if (bk.v_hi <= bk.v_lo) continue;
        BatchMap bm{bt->gid, bt->voff, bt->b_of, bk.v_lo};
        PG_TRY_CUDA(launch_build_bloom(bt->g.row_ptr + bk.v_lo, bt->g.col, bk.v_hi - bk.v_lo, bk.bits, bk.b,
                                       bt->seed, bk.data, bk.stride, bt->hub, s, &bm),
                    "pg_batch: Bloom build");
    }
    return PG_OK;
}

pg_status enqueue_passes(pg_batch *bt, cudaStream_t s) {
    launch_fill_u64(bt->hist, (size_t)bt->hist_bins, 0, s);
    double *S = bt->S;
    launch_fill_f64(S, (size_t)bt->g.n, 0.0, s);
    const EdgeIndex ix = edge_index_view(bt->index, bt->g.n, bt->g.nnz);
    for (const Bucket &bk : bt->buckets) {
        if (bk.v_hi <= bk.v_lo) continue;
        const pg_sketch sk = bucket_sketch(bt, bk);
        PG_TRY_CUDA(launch_batch_pass(bt->g.row_ptr, bt->g.col, bt->g.n, ix, sk, PG_EST_BF_AND, bk.variant,
                                      bt->gid, bt->hoff, bk.v_lo, bk.v_hi, bt->hist, S, bk.table, s),
                    "pg_batch: pass");
    }
    PG_TRY_CUDA(launch_lcc_finalize(bt->g.row_ptr, bt->g.n, S, bt->lcc_out, bt->tri_out, s), "pg_batch: LCC");
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
    // Autotune the lane mapping of every bucket whose variant is 0: build once,
    // time each candidate pass on the bucket and keep the fastest.
    bool tune = false;
    for (const Bucket &bk : bt->buckets) tune |= bk.variant == 0;
    if (tune) {
        st = enqueue_builds(bt, s);
        if (st) {
            delete bt;
            return st;
        }
        const EdgeIndex ix = edge_index_view(bt->index, g->n, g->nnz);
        cudaEvent_t a, b;
        cudaEventCreate(&a);
        cudaEventCreate(&b);
        for (size_t bi = 0; bi < bt->buckets.size(); ++bi) {
            Bucket &bk = bt->buckets[bi];
            if (bk.variant != 0) continue;
            int32_t cand[4];
            const int32_t nc = batch_variants(bk.bits, cand);
            float best = 1e30f;
            int32_t best_v = cand[0];
            const pg_sketch sk = bucket_sketch(bt, bk);
            for (int32_t c = 0; c < nc; ++c) {
                for (int rep = 0; rep < 2; ++rep) {  // first run warms up
                    cudaEventRecord(a, s);
                    e = launch_batch_pass(g->row_ptr, g->col, g->n, ix, sk, PG_EST_BF_AND, cand[c], bt->gid,
                                          bt->hoff, bk.v_lo, bk.v_hi, bt->hist, bt->S, bk.table, s);
                    cudaEventRecord(b, s);
                    if (e == cudaSuccess) e = cudaEventSynchronize(b);
                    if (e != cudaSuccess) break;
                    float ms = 0.0f;
                    cudaEventElapsedTime(&ms, a, b);
                    if (rep == 1 && ms < best) {
                        best = ms;
                        best_v = cand[c];
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

pg_status pg_batch_destroy(pg_batch *bt) {
    if (!bt) return PG_OK;
    if (bt->exec) cudaGraphExecDestroy(bt->exec);
    if (bt->graph) cudaGraphDestroy(bt->graph);
    delete bt;
    return PG_OK;
}

}  // extern "C"

/*
 * pg.h — C ABI of the GB300-native ProbGraph hot path.
 *
 * Method: Besta et al., "ProbGraph: High-Performance and High-Accuracy Graph
 * Mining with Probabilistic Set Representations", SC'22 (arXiv 2208.11469).
 * Each vertex neighbourhood N_v gets a fixed-size sketch (Bloom filter,
 * k-Hash MinHash or 1-Hash MinHash, Sec. II-D); |N_u ∩ N_v| is estimated
 * per edge from the two sketches (Sec. IV) and the estimates are reduced
 * into the triangle count (Sec. VII), per-vertex local clustering
 * coefficients and per-edge / per-pair Jaccard and common-neighbour scores
 * (Sec. III, Listings 3 and 6).
 *
 * Conventions shared by every entry point
 *   Memory    All array arguments are DEVICE pointers owned by the caller,
 *             unless a comment says HOST. The library allocates no device
 *             memory; calls that need scratch take a caller-provided
 *             workspace whose size the matching *_bytes function returns.
 *             A workspace is in use until the call's work on its stream
 *             has finished: calls that may run at the same time (on
 *             different streams) need separate workspaces.
 *   Streams   Every call is stream-ordered on `stream` (NULL = the legacy
 *             default stream) and returns without synchronising it, except
 *             pg_server_* / pg_poll, which are documented separately.
 *   Errors    Every call returns a pg_status. Nothing is thrown across the
 *             ABI. pg_last_error() gives a thread-local detail message.
 *             A PG_ERR_CUDA status means a CUDA launch or runtime call
 *             failed; the stream's work up to that call may be incomplete.
 *   Graphs    pg_csr: int32 CSR of a simple undirected graph, both directions
 *             of every edge stored, every row sorted ascending, no self
 *             loops, no duplicates (Sec. II-A). nnz < 2^31. Calls trust this
 *             unless pg_validate_csr has rejected the graph.
 *   Edges     "Upper edges": each undirected edge once, as (u, v) with u < v
 *             taken from row u, in CSR order (u ascending, then v
 *             ascending). Per-edge outputs are indexed by this order
 *             e = upper_off[u] + (position of v among row u's entries > u).
 *   Hashing   h_i(x) = fmix32(uint32(x) XOR s_i), s_i = fmix32(seed +
 *             i * 0x9E3779B9), where fmix32 is MurmurHash3's 32-bit
 *             finaliser (Sec. VI-C names MurmurHash3; the seeding is this
 *             library's choice). Bit position of h in an l-bit filter:
 *             floor(h * l / 2^32).
 *   Determinism  Same inputs and seed give bit-identical sketches, integer
 *             counts and histograms. Floating totals are computed from the
 *             integer histograms in a fixed order and are deterministic too;
 *             per-vertex sums use double atomics (order-dependent at ~1e-16
 *             relative).
 */
#ifndef PG_H
#define PG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* A cudaStream_t (the same type, declared here without CUDA headers). */
struct CUstream_st;
typedef struct CUstream_st *pg_stream_t;

/* ------------------------------------------------------------------ status */
typedef int32_t pg_status;
#define PG_OK                 0
#define PG_ERR_INVALID_ARG   (-1) /* a null/misaligned pointer, a bad size or parameter */
#define PG_ERR_INVALID_GRAPH (-2) /* pg_validate_csr found the CSR malformed */
#define PG_ERR_TOO_LARGE     (-3) /* a size beyond what the call supports (e.g. nnz >= 2^31) */
#define PG_ERR_NO_MEMORY     (-4) /* workspace/arena smaller than required */
#define PG_ERR_CUDA          (-5) /* a CUDA runtime call or kernel launch failed */
#define PG_ERR_TIMEOUT       (-6) /* a bounded wait ran out */
#define PG_ERR_NOT_FOUND     (-7) /* unknown ticket / handle */
#define PG_ERR_BUSY          (-8) /* result not ready yet / queue full */
#define PG_ERR_UNSUPPORTED   (-9) /* a parameter combination this build does not implement */
#define PG_ERR_CANCELLED    (-10) /* a served request was cancelled or its server shut down */

/* Human-readable name of a status code (static string). */
const char *pg_status_string(pg_status status);
/* Detail message of the last failing call on this host thread (static per thread). */
const char *pg_last_error(void);
/* Library ABI version: (major << 16) | minor. */
int32_t pg_version(void);
/* Number of CUDA kernels this library has enqueued in this process so far
 * (all devices and streams; a monotone counter for accounting and tests). */
uint64_t pg_kernel_launches(void);

/* ------------------------------------------------------------------- graph */
typedef struct pg_csr {
    const int32_t *row_ptr; /* DEVICE [n+1], row_ptr[0] = 0, non-decreasing, row_ptr[n] = nnz */
    const int32_t *col;     /* DEVICE [nnz] neighbour ids in [0, n) */
    int32_t n;              /* vertices, >= 0 */
    int64_t nnz;            /* CSR entries (2 x undirected edges), 0 <= nnz < 2^31 */
} pg_csr;

/* Structural check of a CSR (Sec. II-A form): row_ptr monotone and ending at
 * nnz, ids in range, rows strictly increasing (sorted, no duplicates), no
 * self loops, and (if check_symmetry) every (u,v) has its (v,u).
 * result: DEVICE int64[2]; after the stream reaches this call, result[0] is
 * 0 if the graph is valid, else a PG_CSR_* code, and result[1] the first
 * offending row or entry index found (any one of them if several).
 * Returns PG_OK when the check was enqueued; the verdict is in result. */
#define PG_CSR_OK            0
#define PG_CSR_BAD_ROW_PTR   1
#define PG_CSR_OUT_OF_RANGE  2
#define PG_CSR_UNSORTED      3
#define PG_CSR_SELF_LOOP     4
#define PG_CSR_ASYMMETRIC    5
pg_status pg_validate_csr(const pg_csr *g, int32_t check_symmetry, int64_t *result,
                          pg_stream_t stream);

/* ------------------------------------------------------------ edge index */
/* The upper-edge index: upper_off[u] = number of upper edges (u', v) with
 * u' < u, upper_off[n] = m (undirected edges), and the list of upper edges
 * the passes stream: each edge (u, v) once, grouped by the block of v (blocks
 * of 2^s vertex ids, s = max(20, ceil(log2 n) - 3), so at most 8 blocks),
 * each block in upper-edge order, with every entry's upper-edge index (its
 * per-edge output position). It enumerates each edge once for the sum over E
 * of the TC estimator (Sec. VII) and fixes the per-edge output order. Built
 * once per graph and reused by every analysis call; the buffer also holds the
 * build's scratch. Its size bounds m by nnz / 2 (a symmetric CSR); for a CSR
 * that is not symmetric the list is cut there (pg_validate_csr reports such
 * graphs). */
size_t pg_edge_index_bytes(int32_t n, int64_t nnz);
/* index: DEVICE buffer of pg_edge_index_bytes(g->n, g->nnz) bytes, 16-byte
 * aligned. Overwritten. Valid for this graph until the graph changes. */
pg_status pg_build_edge_index(const pg_csr *g, void *index, size_t index_bytes,
                              pg_stream_t stream);
/* The DEVICE address of upper_off (int32 [n+1]) inside an index buffer. */
const int32_t *pg_edge_index_upper_off(const void *index);

/* ----------------------------------------------------------------- sketches */
#define PG_SK_BLOOM 1 /* Bloom filter, Sec. II-D */
#define PG_SK_KHASH 2 /* MinHash, k-Hash variant, Sec. II-D */
#define PG_SK_1HASH 3 /* MinHash, 1-Hash variant, Sec. II-D */

/* One sketch per vertex, row-major, row v at data + v * stride_bytes.
 *   Bloom: bits l (multiple of 64, 64..1024) in 64-bit words, bit p of the
 *          filter is bit (p % 64) of word p / 64; words beyond l/64 up to the
 *          stride are zero. b hash functions h_0..h_{b-1} (1..16).
 *   k-Hash: k uint32 (1..256): entry i = min over x in N_v of h_i(x); a
 *          vertex with no neighbours has all entries 0xFFFFFFFF.
 *   1-Hash: k uint32 (1..32): the min(k, d_v) smallest values of h_0 over
 *          N_v in increasing order, then 0xFFFFFFFF padding. Because every
 *          h_i is a bijection on 32-bit ids, storing hash values is
 *          equivalent to storing the minimising elements of Sec. II-D. */
typedef struct pg_sketch {
    int32_t kind;         /* PG_SK_* */
    uint32_t bits;        /* Bloom: l */
    uint32_t b;           /* Bloom: hash functions per element */
    uint32_t k;           /* MinHash: sketch size */
    uint32_t seed;        /* hash seed */
    int32_t n;            /* rows (must equal the graph's n) */
    int64_t stride_bytes; /* >= row payload, multiple of 16 */
    void *data;           /* DEVICE, n * stride_bytes, 16-byte aligned */
} pg_sketch;

/* Default row stride: the payload (l/8 or 4k bytes) rounded up to 16 bytes. */
int64_t pg_sketch_stride(int32_t kind, uint32_t bits, uint32_t k);
/* Filter length for a storage budget s (fraction of CSR bytes, Sec. V-A):
 * l = 64 * floor(s * (4(n+1) + 4 nnz) * 8 / (64 n)), clamped to [64, 1024]. */
uint32_t pg_bloom_bits_for_budget(double s, int32_t n, int64_t nnz);

/* Device scratch bytes the builders need for this graph (a list of the rows
 * too long for one warp, which are finished by a second kernel). */
size_t pg_build_workspace_bytes(const pg_csr *g);

/* Bloom filter construction (Sec. II-D): for every v, start from l zero bits
 * and, for each x in N_v and i < b, set bit floor(h_i(x) * l / 2^32).
 * sk: kind = PG_SK_BLOOM with bits, b, seed, n, stride_bytes, data set.
 * workspace: DEVICE, >= pg_build_workspace_bytes(g), 16-byte aligned.
 * Overwrites every row of sk->data. */
pg_status pg_build_bloom(const pg_csr *g, const pg_sketch *sk, void *workspace,
                         size_t workspace_bytes, pg_stream_t stream);

/* MinHash construction (Sec. II-D), kind PG_SK_KHASH or PG_SK_1HASH, with
 * k, seed, n, stride_bytes, data set. Overwrites the first k entries of
 * every row of sk->data (row padding beyond k entries is not written).
 * workspace as for pg_build_bloom. */
pg_status pg_build_minhash(const pg_csr *g, const pg_sketch *sk, void *workspace,
                           size_t workspace_bytes, pg_stream_t stream);

/* Upload a CSR from HOST memory (page-locked for the copies to overlap) into
 * the DEVICE CSR g and build sketches of its rows while it lands: row_ptr is
 * copied first, then col in chunks of whole rows (about chunk_entries
 * entries each, at least one row) on copy_stream; after each chunk, stream
 * waits for it and builds every sketch's rows of that chunk (the builds of
 * Sec. II-D are per row, so the result equals pg_build_bloom /
 * pg_build_minhash on the uploaded CSR). The copies start after the work
 * already enqueued on stream, so a previous step that reads g is not
 * overwritten. When the call returns, stream is ordered after the whole
 * upload and the builds; copy_stream may equal stream (no overlap).
 * host_row_ptr: HOST int32 [n+1] from 0 to nnz, non-decreasing (it is read
 * on the host to cut the chunks); host_col: HOST int32 [nnz]. sketches:
 * HOST array of count descriptors (any kinds, DEVICE data for g's n rows);
 * ws: DEVICE build workspace (pg_build_workspace_bytes), shared by the
 * builds in stream order. Errors: PG_ERR_INVALID_ARG (NULLs, offsets not
 * from 0 to nnz, sketch checks as for the builders), PG_ERR_NO_MEMORY
 * (workspace too small), PG_ERR_CUDA. Asynchronous. */
pg_status pg_upload_build(const int32_t *host_row_ptr, const int32_t *host_col, const pg_csr *g,
                          const pg_sketch *sketches, int32_t count, void *workspace, size_t workspace_bytes,
                          int64_t chunk_entries, pg_stream_t copy_stream, pg_stream_t stream);

/* Sketch files (checkpoint / resume of the sketches, which are a pure
 * function of the CSR, the parameters and the seed): a 64-byte header
 * {"PGSKTCH1", version 1, kind, bits, b, k, seed, n, stride, n * stride}
 * followed by the n rows exactly as they lie in device memory.
 * pg_sketch_save synchronises the stream and writes sk->data (DEVICE) to path.
 * pg_sketch_load_header fills every field of *sk but data from the file.
 * pg_sketch_load synchronises the stream and copies the rows into sk->data
 * (DEVICE, n * stride bytes) if the file's descriptor equals *sk's.
 * Errors: PG_ERR_NOT_FOUND (file cannot be opened), PG_ERR_INVALID_ARG (bad
 * header, descriptor mismatch, truncated or unwritable file), PG_ERR_CUDA. */
pg_status pg_sketch_save(const pg_sketch *sk, const char *path, pg_stream_t stream);
pg_status pg_sketch_load_header(const char *path, pg_sketch *sk);
pg_status pg_sketch_load(pg_sketch *sk, const char *path, pg_stream_t stream);

/* --------------------------------------------------------------- estimators */
#define PG_EST_EXACT       0 /* exact |N_u ∩ N_v| (no sketch) */
#define PG_EST_BF_AND      1 /* Eq. (bf_int) on popcount(B_u AND B_v), B1 = l read as l - 1 */
#define PG_EST_BF_L        2 /* Eq. (limit_xs): popcount(B_u AND B_v) / b */
#define PG_EST_KH          3 /* Eq. (est_int_mh), J = #{i : min_i(u) = min_i(v)} / k */
#define PG_EST_1H          4 /* Sec. IV-D, J = c_union / K (see pg_tc_result) */
#define PG_EST_1H_LITERAL  5 /* Sec. IV-D as printed, J = |M1_u ∩ M1_v| / k */
#define PG_EST_BF_OR       6 /* Eq. (bf_int_union): d_u + d_v + (l/b) log(1 - U/l), U = popcount(B_u OR B_v)
                                (read as l - 1 when U = l); per-edge aux = U; pass kernels of any width */
#define PG_EST_BF_SS       7 /* the single-set Bloom estimator on the AND filter (Sec. VIII):
                                log(1 - B1/l) / (b log(1 - 1/l)), B1 = l read as l - 1 */
#define PG_EST_1H_KMV      8 /* Sec. IX, KMV on the 1-Hash rows: d_u + d_v - (k - 1) / h_k, h_k the
                                k-th smallest hash of the two rows' union mapped into (0, 1] as
                                (h + 1) / 2^32; a union of fewer than k values is counted exactly.
                                Totals: the 1-Hash histograms plus the exact 128-bit sum (x 2^-52)
                                of the real union estimates (two extra bins); est_tc_alt = the
                                c_union / K estimate of the same edges */

/* Graph-level result, written to a DEVICE pg_tc_result. */
typedef struct pg_tc_result {
    uint64_t edges;      /* undirected edges (or pairs) intersected */
    uint64_t count_sum;  /* sum over them of the integer count: popcount(AND) (popcount(OR)
                            for PG_EST_BF_OR), k-Hash matches, 1-Hash c_union, or exact
                            |N_u ∩ N_v| */
    uint64_t exact_tc;   /* PG_EST_EXACT: the exact triangle count; else 0 */
    uint64_t reserved;
    double est_tc;       /* (1/3) sum over edges of the requested estimate (Sec. VII) */
    double est_tc_alt;   /* Bloom: the other of AND / L from the same popcounts;
                            1-Hash: the other of the c_union / literal readings; else 0 */
} pg_tc_result;

/* Number of uint64 histogram bins pg_edge_counts fills for a sketch/estimator:
 * Bloom: l+1 (count of edges per popcount; OR: per union popcount, plus one
 * bin with the sum of d_u + d_v); k-Hash: 2(k+1) (edges per match count, then
 * sum of d_u + d_v per match count); 1-Hash: 2(k+1)^2 + 2(k+1) ((c_union, K)
 * edge counts, their degree sums, then c_lit edge counts and degree sums),
 * plus two for KMV (the 128-bit sum x 2^52 of the real union estimates, low
 * word first); exact: 0. */
int64_t pg_hist_bins(const pg_sketch *sk, int32_t estimator);

/* Workspace bytes for pg_triangle_count / pg_clustering / pg_jaccard_pairs /
 * pg_edge_counts on this graph, sketch and estimator (sk may be NULL for
 * PG_EST_EXACT). */
size_t pg_workspace_bytes(const pg_csr *g, const pg_sketch *sk, int32_t estimator);

/* Triangle count (Sec. VII): TC^ = (1/3) sum over undirected edges of the
 * estimate of |N_u ∩ N_v|; with PG_EST_EXACT the exact count by degree-
 * ordered node iteration (Sec. III, Listing 1). index: built by
 * pg_build_edge_index for g. sk: NULL for exact. out: DEVICE pg_tc_result. */
pg_status pg_triangle_count(const pg_csr *g, const void *index, const pg_sketch *sk,
                            int32_t estimator, void *workspace, size_t workspace_bytes,
                            pg_tc_result *out, pg_stream_t stream);

/* Local clustering coefficient per vertex: T_v = 1/2 sum over u in N_v of
 * the estimate of |N_u ∩ N_v| (exact: triangles at v) and
 * lcc_v = 2 T_v / (d_v (d_v - 1)), 0 when d_v < 2; not clamped to 1.
 * lcc: DEVICE float [n]; tri: DEVICE double [n] or NULL; tc: DEVICE
 * pg_tc_result or NULL (the triangle count comes from the same pass). */
pg_status pg_clustering(const pg_csr *g, const void *index, const pg_sketch *sk,
                        int32_t estimator, void *workspace, size_t workspace_bytes,
                        float *lcc, double *tri, pg_tc_result *tc, pg_stream_t stream);

/* Common neighbours and Jaccard (Listings 3 and 6): cn = estimate of
 * |N_u ∩ N_v| (not clamped); jac = I / (d_u + d_v - I) with
 * I = clamp(cn, 0, min(d_u, d_v)), 0 when d_u + d_v = 0.
 * pairs: DEVICE int32 [2P] as (u0, v0, u1, v1, ...), any vertices in [0, n);
 * or NULL for every upper edge (then P is ignored and outputs have m entries
 * in upper-edge order). cn, jac: DEVICE float, either may be NULL. */
pg_status pg_jaccard_pairs(const pg_csr *g, const void *index, const pg_sketch *sk,
                           int32_t estimator, const int32_t *pairs, int64_t P,
                           void *workspace, size_t workspace_bytes, float *cn, float *jac,
                           pg_stream_t stream);

/* Vertex-similarity measures of Listing sim for every pair (or every upper
 * edge with pairs NULL), from the exact or estimated |N_u ∩ N_v|: with
 * I = clamp(estimate, 0, min(d_u, d_v)), cn = the estimate, jac =
 * I / (d_u + d_v - I), overlap = I / min(d_u, d_v), total = d_u + d_v - I
 * (a zero denominator gives 0). Every pointer is a DEVICE float array [P or m]
 * or NULL. Arguments and errors as pg_jaccard_pairs. */
typedef struct pg_similarity {
    float *cn;
    float *jac;
    float *overlap;
    float *total;
} pg_similarity;
pg_status pg_similarity_pairs(const pg_csr *g, const void *index, const pg_sketch *sk, int32_t estimator,
                              const int32_t *pairs, int64_t P, void *workspace, size_t workspace_bytes,
                              const pg_similarity *out, pg_stream_t stream);

/* The integer counts behind every estimate, for checking and analysis:
 * count: DEVICE int32 [m or P] or NULL — popcount(AND) / k-Hash matches /
 * 1-Hash c_union / exact |N_u ∩ N_v|; aux: DEVICE int32 [m or P] or NULL —
 * 1-Hash: K | (c_lit << 16), Bloom OR: popcount(B_u OR B_v), else unwritten;
 * hist: DEVICE uint64 [pg_hist_bins] or NULL.
 * pairs as in pg_jaccard_pairs. */
pg_status pg_edge_counts(const pg_csr *g, const void *index, const pg_sketch *sk,
                         int32_t estimator, const int32_t *pairs, int64_t P,
                         void *workspace, size_t workspace_bytes, int32_t *count,
                         int32_t *aux, uint64_t *hist, pg_stream_t stream);

/* Everything the hot path produces, in ONE pass over the upper edges
 * (sketch intersection, estimate, TC histogram, per-vertex sums, per-edge
 * scores). Every pointer is DEVICE and optional (NULL = not wanted):
 *   tc         pg_tc_result, as pg_triangle_count
 *   lcc, tri   float [n], double [n], as pg_clustering
 *   edge_cn, edge_jac    float [m], as pg_jaccard_pairs over all upper edges
 *   edge_count, edge_aux int32 [m], as pg_edge_counts (edge_aux: 1-Hash only)
 *   hist       uint64 [pg_hist_bins], as pg_edge_counts
 * With PG_EST_EXACT the per-edge outputs take a second kernel over full rows
 * and edge_aux / hist are not written. */
typedef struct pg_outputs {
    pg_tc_result *tc;
    float *lcc;
    double *tri;
    float *edge_cn;
    float *edge_jac;
    int32_t *edge_count;
    int32_t *edge_aux;
    uint64_t *hist;
    float *edge_overlap;  /* float [m], as pg_similarity_pairs over all upper edges */
    float *edge_total;    /* float [m], as pg_similarity_pairs over all upper edges */
} pg_outputs;
pg_status pg_analyze(const pg_csr *g, const void *index, const pg_sketch *sk, int32_t estimator,
                     void *workspace, size_t workspace_bytes, const pg_outputs *out,
                     pg_stream_t stream);

/* pg_triangle_count without a workspace, for callers that cannot allocate
 * device memory (for example a plugin inside a host application whose own
 * allocator has reserved the device memory, or a process that forbids device
 * allocation after start-up). The paper has no counterpart: this is a
 * packaging variant of pg_triangle_count, with the same arguments minus the
 * workspace and the same result.
 * Its scratch (estimator table and count histogram) lives in a 64 KiB static
 * array of device memory inside the library, held on every GPU that loads the
 * library until the process exits; every supported sketch fits. The exact
 * estimator is rejected (PG_ERR_UNSUPPORTED); a sketch whose scratch would
 * not fit returns PG_ERR_TOO_LARGE. The call allocates nothing.
 * The first call on a device looks up the array's address with that device
 * current; make it before any stream capture. All calls on a device share
 * the array (cleared per call where it must start at zero): calls that
 * overlap on the GPU race and give wrong results, so order them on one
 * stream or synchronise between them. */
pg_status pg_triangle_count_noalloc(const pg_csr *g, const void *index, const pg_sketch *sk,
                                    int32_t estimator, pg_tc_result *out, pg_stream_t stream);

/* ------------------------------------------- vertex-partitioned runs --
 * The distributed form of the pass (Sec. VIII-F: the vertices are split
 * among processes, each builds the sketches of its own vertices, the rows
 * that its edges need are exchanged, and each estimates the edges of its own
 * vertices). One rank, holding the whole CSR and index and the exchanged
 * sketch table, calls pg_partial_sums for its vertex range; the ranks sum
 * their `sums` and `hist` (element-wise, e.g. an all-reduce; hist as 64-bit
 * integers, wrapping) and any rank then calls pg_finalize_sums. The results
 * equal pg_analyze's over the whole graph: the histogram bit for bit, the
 * per-vertex sums up to the order of double additions.
 *
 * pg_partial_sums: the upper edges (u, v) with u_begin <= u < u_end only.
 * Adds each edge's estimate to sums[u] and sums[v] (DEVICE double [n],
 * caller-zeroed, or NULL) and its count to hist (DEVICE uint64
 * [pg_hist_bins], caller-zeroed, or NULL). Workspace as pg_analyze.
 * PG_ERR_UNSUPPORTED for PG_EST_EXACT and PG_EST_1H_KMV (whose total holds a
 * 128-bit sum). */
pg_status pg_partial_sums(const pg_csr *g, const void *index, const pg_sketch *sk, int32_t estimator,
                          int32_t u_begin, int32_t u_end, void *workspace, size_t workspace_bytes,
                          double *sums, uint64_t *hist, pg_stream_t stream);
/* pg_finalize_sums: from the summed partials, tc (DEVICE pg_tc_result, from
 * hist, the fixed-order dot of pg_triangle_count), tri = sums / 2 (DEVICE
 * double [n], may alias sums) and lcc (DEVICE float [n]); each output is
 * optional. */
pg_status pg_finalize_sums(const pg_csr *g, const pg_sketch *sk, int32_t estimator, const uint64_t *hist,
                           double *sums, pg_tc_result *tc, float *lcc, double *tri, pg_stream_t stream);

/* ----------------------------------------------------- Jarvis-Patrick --
 * Jarvis-Patrick clustering (Sec. III, Listing "Jarvis-Patrick
 * clustering"): the edges (u, v) whose common-neighbour count |N_u ∩ N_v|
 * exceeds tau form the clustering C; the clusters are the connected
 * components of (V, C), singletons included. The count is exact
 * (PG_EST_EXACT, sk NULL) or estimated with sk (every estimator). Keep test:
 * exact count > tau; Bloom AND: the AND estimate of the count > tau (decided
 * on the count, the estimate being non-decreasing in it); Bloom L: count / b
 * > tau; MinHash: J / (1 + J) * (d_u + d_v) > tau, J = c / K, in double.
 *   labels: DEVICE int32 [n] or NULL: each vertex's cluster, named by the
 *           smallest vertex id in it (the same for any execution order)
 *   out:    DEVICE pg_jp_result
 *   workspace: pg_jarvis_patrick_workspace_bytes; index: pg_build_edge_index.
 * Errors as pg_triangle_count, plus PG_ERR_INVALID_ARG for a NaN tau. */
typedef struct pg_jp_result {
    int64_t clusters; /* connected components of (V, C) */
    int64_t kept;     /* |C| */
    int64_t edges;    /* undirected edges of the graph */
    int64_t reserved;
} pg_jp_result;
size_t pg_jarvis_patrick_workspace_bytes(const pg_csr *g, const pg_sketch *sk, int32_t estimator);
pg_status pg_jarvis_patrick(const pg_csr *g, const void *index, const pg_sketch *sk, int32_t estimator,
                            double tau, void *workspace, size_t workspace_bytes, int32_t *labels,
                            pg_jp_result *out, pg_stream_t stream);

/* ------------------------------------------------------------- 4-cliques --
 * 4-clique counting (Sec. III-A, Listing "Reformulated 4-Clique Counting"):
 * vertices ranked by (degree, id), N+_v = neighbours ranked above v; for every
 * oriented edge u -> v, C3 = N+_u ∩ N+_v (exact), and the count is the sum
 * over w in C3 of |N+_w ∩ C3|. With PG_EST_BF_AND / PG_EST_BF_L that
 * innermost intersection is estimated from popcount(BF+_u AND BF+_v AND
 * BF+_w), the Bloom filters (bits, b, seed as pg_build_bloom) being built
 * over the oriented neighbourhoods inside the call; PG_EST_EXACT counts it.
 *   workspace: pg_clique4_workspace_bytes(g, estimator, bits)
 *   out:       DEVICE pg_clique4_result
 * Errors: PG_ERR_INVALID_ARG, PG_ERR_UNSUPPORTED (estimator, bits not a
 * multiple of 64 in [64, 1024], b not in 1..16), PG_ERR_NO_MEMORY, PG_ERR_CUDA. */
typedef struct pg_clique4_result {
    uint64_t triangles; /* 3-cliques (u, v, w) visited = the triangle count */
    uint64_t exact;     /* PG_EST_EXACT: the 4-clique count; else 0 */
    uint64_t count_sum; /* sketch: sum over the 3-cliques of the triple-AND popcount */
    uint64_t reserved;
    double est;         /* the 4-clique count (exact, or the chosen estimator's total) */
    double est_alt;     /* sketch: the other Bloom estimator's total (L for AND, AND for L) */
} pg_clique4_result;
size_t pg_clique4_workspace_bytes(const pg_csr *g, int32_t estimator, uint32_t bits);
pg_status pg_clique4_count(const pg_csr *g, int32_t estimator, uint32_t bits, uint32_t b, uint32_t seed,
                           void *workspace, size_t workspace_bytes, pg_clique4_result *out, pg_stream_t stream);

/* ---------------------------------------------------------------- batch --
 * Many small graphs analysed together (the per-graph Bloom-filter triangle
 * count of Sec. V, Eq. bf_int, and the LCC of Sec. III-A, per graph), in one
 * launch sequence that is captured once as a CUDA graph and replayed.
 *
 * The G graphs come as ONE block-diagonal CSR g with global vertex ids: graph
 * i owns vertices [voff[i], voff[i+1]) and its rows only name vertices of the
 * same range (voff: HOST int32 [G+1], voff[0] = 0, voff[G] = g->n). Each
 * graph's sketch hashes its own ids (global id - voff[i]), so a graph's
 * sketch and estimates are the same in the batch and alone.
 *
 * Per graph i, cfg[i] sets the Bloom filter: bits in {64, 128, 256, 512,
 * 1024}, b in [1, 16], and variant in [0, 1024] = consecutive 32-vertex
 * groups per warp work chunk of the pass (0 = let pg_batch_create time the
 * candidates 1, 4, 16 and choose; it writes the choice back into cfg). Every
 * variant gives bit-identical results: the per-vertex sums are exact
 * fixed-point sums. Graphs with equal (bits, b) must be contiguous: order
 * them by bucket. */
typedef struct pg_batch_config {
    uint32_t bits;
    uint32_t b;
    int32_t variant;
    int32_t reserved;
} pg_batch_config;
typedef struct pg_batch pg_batch;

/* Autotuner, host only: cfg[i].bits = the largest power of two in [64, 1024]
 * not above budget * (CSR bytes of graph i) * 8 / n_i (the storage budget s
 * of Sec. V-A), cfg[i].b = the b in {1, 2, 4} with the smallest modelled
 * error of the AND estimator at that length (bias at the expected popcount
 * plus the MSE bound of Prop. 4.1, for neighbourhoods of the graph's average
 * degree sharing a tenth of their elements), cfg[i].variant = 0.
 * n, nnz: HOST arrays [graphs]. */
pg_status pg_batch_autotune(const int32_t *n, const int64_t *nnz, int32_t graphs, double budget,
                            pg_batch_config *cfg);

/* Device workspace a batch needs (graph tables, per-graph histograms,
 * estimator tables, sketches); 0 for invalid arguments, including a union
 * graph of more than 2^31 - 65 CSR entries. */
size_t pg_batch_workspace_bytes(const pg_csr *g, int32_t graphs, const int32_t *voff,
                                const pg_batch_config *cfg);

/* Create a batch over g (DEVICE CSR, resident for the batch's lifetime) and
 * a caller workspace of pg_batch_workspace_bytes. Outputs (DEVICE, written by
 * every pg_batch_run): tc pg_tc_result [G] (graph i's triangle count and
 * edge totals, as pg_triangle_count with PG_EST_BF_AND), lcc float [n] and
 * tri double [n] or NULL (per vertex, as pg_clustering). Synchronises the
 * stream; when a variant is 0 it runs and times the candidate passes once.
 * Errors: PG_ERR_INVALID_ARG (NULLs, voff not covering g, non-contiguous
 * buckets, b or variant out of range), PG_ERR_UNSUPPORTED (bits), PG_ERR_NO_MEMORY
 * (workspace too small), PG_ERR_CUDA. On error *out is unchanged. */
pg_status pg_batch_create(const pg_csr *g, int32_t graphs, const int32_t *voff, pg_batch_config *cfg,
                          uint32_t seed, void *workspace, size_t workspace_bytes, pg_tc_result *tc,
                          float *lcc, double *tri, pg_stream_t stream, pg_batch **out);

/* One run: sketches and pass of every graph (the pass writes LCC and
 * triangles per vertex), then the per-graph triangle counts. On a
 * non-default stream the first run captures the sequence as a CUDA graph
 * (for that stream) and every run launches it; on the default stream (NULL)
 * the kernels are launched one by one. The CSR contents may change between
 * runs (same n, nnz and voff). Runs of one batch use its workspace (sketches,
 * histograms, the pass's work counter) and must not overlap in time: order
 * runs on different streams with events. Asynchronous. */
pg_status pg_batch_run(pg_batch *batch, pg_stream_t stream);

/* One run from a HOST copy of the union CSR (page-locked for the copies to
 * overlap): row_ptr is uploaded into the batch's device CSR, then col in
 * chunks of whole graphs of one bucket (about chunk_entries entries each, at
 * least one graph) on copy_stream; after each chunk, stream waits for it and
 * builds and passes over that chunk's graphs, so the upload of the next
 * chunks overlaps the work on the earlier ones (a graph's sketches and pass
 * read only its own rows). Same outputs as pg_batch_run (bit-identical), run
 * eagerly, not captured. The copies start after the work already enqueued
 * on stream; when the call returns, stream is ordered after the whole
 * upload. host_row_ptr: HOST int32 [n+1] from 0 to nnz with the batch's
 * graph layout (voff); host_col: HOST int32 [nnz]. copy_stream may equal
 * stream (no overlap). Errors: PG_ERR_INVALID_ARG (NULLs, offsets not from 0
 * to nnz, chunk_entries < 1), PG_ERR_CUDA. Asynchronous. */
pg_status pg_batch_run_host(pg_batch *batch, const int32_t *host_row_ptr, const int32_t *host_col,
                            int64_t chunk_entries, pg_stream_t copy_stream, pg_stream_t stream);

/* Free the host state and the captured graph (not the workspace). NULL is a
 * no-op. */
pg_status pg_batch_destroy(pg_batch *batch);

/* -------------------------------------------------------------- serving --
 * A request loop over one resident graph and its sketches: vertex-pair
 * similarity queries (the common-neighbour and Jaccard estimates of Sec. III
 * and IV, as in link prediction) and triangle counts of induced subgraphs
 * (Sec. VII on G[S]), with continuous batching.
 *
 * A host scheduler thread owned by the server admits queued requests in
 * arrival order while the arena (caller-owned DEVICE memory) has room for
 * them, and keeps the GPU busy with the admitted ones:
 *   - pair requests are cut into tiles of 1024 pairs; every launch of the
 *     pair kernel takes tiles round-robin from all admitted pair requests
 *     (up to iteration_pairs pairs), so a request that arrives while others
 *     run joins the next launch and small requests finish without waiting
 *     for large ones;
 *   - each subgraph request runs its own pipeline (membership marks,
 *     induced degrees, scan, induced CSR with local ids; then edge index,
 *     Bloom sketches of the induced neighbourhoods and the fused pass, or the
 *     exact count) on one of `streams` streams, overlapping with the pair
 *     launches and with each other.
 * Results are deterministic: a request's answer does not depend on what else
 * is in flight (the pair kernel computes each pair alone; a subgraph's
 * vertices are sorted and deduplicated, and its sketches hash their local
 * ids in that order).
 * No kernel waits on the host: the scheduler polls CUDA events, and pg_poll
 * waits on the host with the caller's time limit. */
#define PG_REQ_PAIRS       1
#define PG_REQ_SUBGRAPH_TC 2

typedef struct pg_server_opts {
    int32_t streams;         /* concurrent subgraph pipelines (0: 4) */
    int32_t max_inflight;    /* admitted requests at once (0: 4096) */
    int64_t iteration_pairs; /* pairs per pair-kernel launch at most (0: 262144) */
    size_t pinned_bytes;     /* page-locked host staging the server allocates (0: 256 MiB) */
    uint32_t sub_bits;       /* Bloom filter of subgraph requests (0: 512 bits) */
    uint32_t sub_b;          /* its hash count (0: 2) */
    uint32_t sub_seed;       /* its seed (0: 1) */
    int32_t reserved;
} pg_server_opts;

typedef struct pg_request {
    int32_t kind;      /* PG_REQ_PAIRS or PG_REQ_SUBGRAPH_TC */
    int32_t estimator; /* pairs: PG_EST_BF_AND, PG_EST_BF_L (the server's Bloom sketch), PG_EST_KH (its
                          k-Hash sketch) or PG_EST_EXACT (merge of the two rows);
                          subgraph: PG_EST_BF_AND, PG_EST_BF_L or PG_EST_EXACT */
    int64_t count;     /* pairs P, or vertices |S| (duplicates allowed) */
    const int32_t *data; /* HOST: pairs int32 [2P] (u, v), or vertex ids [|S|]; read when the request is
                            admitted, so it must stay valid until pg_poll returns its response */
    float *cn;         /* HOST float [P] or NULL: common-neighbour estimate per pair */
    float *jac;        /* HOST float [P] or NULL: Jaccard estimate per pair.
                          When data and the outputs of a pair request are all page-locked (cudaHostAlloc /
                          cudaHostRegister), the kernels read and write them in place over the CPU-GPU link,
                          with no staging copy and no arena bytes. */
} pg_request;

typedef struct pg_response {
    int32_t status;   /* PG_OK, PG_ERR_CANCELLED, or the error that ended the request */
    int32_t kind;
    int64_t count;    /* pairs answered, or |S| after deduplication */
    pg_tc_result tc;  /* subgraph: as pg_triangle_count on G[S] (tc.edges = edges of G[S]) */
    double queue_us;  /* submit -> admission */
    double total_us;  /* submit -> result on the host */
} pg_response;

typedef struct pg_server pg_server;

/* Arena bytes a server reserves for itself (estimator tables, pair tile
 * descriptors, one membership bitmap of n bits per stream); requests use the
 * rest. opts may be NULL (defaults). */
size_t pg_server_reserved_bytes(const pg_csr *g, const pg_server_opts *opts);

/* Create a server over the DEVICE CSR g and n_sketches resident sketches (at
 * most one Bloom of <= 8192 bits and one k-Hash of k <= 1024; pair requests for an estimator whose sketch
 * is absent fail with PG_ERR_UNSUPPORTED). The CSR, the sketches and the
 * arena stay owned by the caller and must outlive the server; the server
 * copies the row offsets to the host once (admission bounds). Starts the
 * scheduler thread on the current device. Errors: PG_ERR_INVALID_ARG,
 * PG_ERR_NO_MEMORY (arena below pg_server_reserved_bytes), PG_ERR_CUDA. */
pg_status pg_server_create(const pg_csr *g, const pg_sketch *const *sketches, int32_t n_sketches,
                           void *arena, size_t arena_bytes, const pg_server_opts *opts, pg_server **out);

/* Queue a request; *ticket identifies it for pg_poll / pg_cancel. Checks the
 * arguments (vertex ids must lie in [0, n); pair ids outside give 0 answers)
 * and that the request can ever fit the arena and the staging memory
 * (PG_ERR_NO_MEMORY otherwise); never waits for the GPU. */
pg_status pg_submit(pg_server *server, const pg_request *req, uint64_t *ticket);

/* pg_submit for count requests in one call (one lock, one wake-up of the
 * scheduler): tickets[i] for reqs[i]. All or nothing: if any request is
 * invalid or can never fit, none is queued and the error names its index. */
pg_status pg_submit_many(pg_server *server, const pg_request *reqs, int64_t count, uint64_t *tickets);

/* pg_poll for count tickets: waits up to timeout_us until all complete.
 * out[i] receives each completed response (whose ticket is then released),
 * status PG_ERR_BUSY for one still running and PG_ERR_NOT_FOUND for an
 * unknown ticket. *n_done (may be NULL) = responses with a final status.
 * Returns PG_OK when all are final, else PG_ERR_BUSY. */
pg_status pg_poll_many(pg_server *server, const uint64_t *tickets, int64_t count, pg_response *out,
                       int64_t timeout_us, int64_t *n_done);

/* Wait up to timeout_us microseconds (0: do not wait) for the request to
 * complete. PG_OK: *out holds the response, the outputs are written, and the
 * ticket is released. PG_ERR_BUSY: not complete yet. PG_ERR_NOT_FOUND:
 * unknown or already collected ticket. */
pg_status pg_poll(pg_server *server, uint64_t ticket, pg_response *out, int64_t timeout_us);

/* Cancel a request that has not been admitted yet (its response then has
 * status PG_ERR_CANCELLED). PG_ERR_BUSY if it already runs (it completes
 * normally), PG_ERR_NOT_FOUND for an unknown ticket. */
pg_status pg_cancel(pg_server *server, uint64_t ticket);

/* Counters since creation. */
typedef struct pg_server_stats {
    uint64_t submitted, completed, cancelled, failed;
    uint64_t pair_launches;  /* launches of the pair kernel */
    uint64_t pairs;          /* pairs answered */
    uint64_t subgraphs;      /* subgraph pipelines run */
    uint64_t queued, running;
    uint64_t arena_used, arena_peak, arena_bytes;
    uint64_t pair_kernel_ns;  /* device time of the pair-kernel launches (CUDA events around each) */
} pg_server_stats;
pg_status pg_server_stats_get(pg_server *server, pg_server_stats *out);

/* Stop the server: requests not yet admitted are cancelled, admitted ones
 * run to completion on the GPU (their responses are discarded), then the
 * thread, streams and staging memory are released. NULL is a no-op. */
pg_status pg_server_destroy(pg_server *server);

#ifdef __cplusplus
}
#endif
#endif /* PG_H */

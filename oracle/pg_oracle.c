/*
 * ProbGraph oracle: a plain, serial, obviously-correct CPU restatement of the
 * per-edge |N(u) ∩ N(v)| estimation path of Besta et al., "ProbGraph:
 * High-Performance and High-Accuracy Graph Mining with Probabilistic Set
 * Representations" (SC'22).
 *
 * TEST INFRASTRUCTURE. Only tests/, __graft_entry__.smoke() and bench.py's
 * CPU-baseline leg may build, load or call this file. It shares no code,
 * header, table or constant generator with the CUDA library, and the CUDA
 * library never calls it.
 *
 * Conventions
 *   - Graphs are CSR: row_ptr[n+1], col[nnz], both directions of every
 *     undirected edge stored, neighbour lists sorted, no self-loops (Sec. II-A).
 *   - Bloom filters are kept one BYTE per bit (0/1) so that every bit can be
 *     read directly; pgo_bloom_pack only re-lays them out as 64-bit words
 *     (bit p -> word p/64, bit p%64) for comparison with packed filters.
 *   - MinHash sketches hold ELEMENTS (vertex ids), as M_X does in Sec. II-D;
 *     -1 marks an empty slot.
 *   - This file computes sketches and integer counts only; the estimators
 *     (double precision) are written out in oracle.py.
 *
 * Readings where the paper is silent (every one is listed in the design notes):
 *   A  hash family: h_i(x) = fmix32(x XOR s_i), s_i = fmix32(seed + i*0x9E3779B9),
 *      fmix32 = MurmurHash3's 32-bit finaliser (Sec. VI-C names MurmurHash3).
 *   B  bit position of a hash value in an l-bit filter: floor(h * l / 2^32).
 *   C  1-Hash count: c_union = number of elements of X∩Y among the K smallest
 *      of M1_X ∪ M1_Y, K = min(k, |M1_X ∪ M1_Y|); J^ = c_union / K.
 *      The literal |M1_X ∩ M1_Y| is also returned (c_lit).
 *   D  k-Hash count: #{i : x_{i,min}(X) = x_{i,min}(Y)}.
 *   E  AND estimator saturation: B~1 = B1 - [B1 = B] (appendix, "Enhancing
 *      the Estimator by Swamidass").
 *   J  an empty set has an empty sketch; any count involving it is 0.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Hashing (Sec. VI-C "Implementation Details": MurmurHash3; reading A).    */
/* ------------------------------------------------------------------------ */

/* MurmurHash3's 32-bit finalisation mix: two multiply / xor-shift rounds. */
uint32_t pgo_fmix32(uint32_t h)
{
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
}

/* Per-function seed s_i of hash function number i (0-based). */
uint32_t pgo_hash_seed(uint32_t seed, uint32_t i)
{
    return pgo_fmix32(seed + i * 0x9E3779B9u);
}

/* h_i(x): the i-th hash function applied to element x. */
uint32_t pgo_hash(uint32_t seed, uint32_t i, int32_t x)
{
    return pgo_fmix32((uint32_t)x ^ pgo_hash_seed(seed, i));
}

/* Position in [0, l) of hash value h (reading B). */
uint32_t pgo_bit_position(uint32_t h, uint32_t l)
{
    return (uint32_t)(((uint64_t)h * (uint64_t)l) >> 32);
}

/* ------------------------------------------------------------------------ */
/* Bloom filters (Sec. II-D "Bloom filters").                               */
/* ------------------------------------------------------------------------ */

/* Construct B_X for every vertex neighbourhood X = N_v: start from l zero
 * bits; for each x in X and each of the b hash functions set bit h_i(x).
 * out: n * l bytes, one byte per bit, vertex-major. */
void pgo_bloom_build(int32_t n, const int32_t *row_ptr, const int32_t *col,
                     uint32_t l, uint32_t b, uint32_t seed, uint8_t *out)
{
    for (int32_t v = 0; v < n; ++v) {
        uint8_t *B = out + (size_t)v * l;
        memset(B, 0, l);
        for (int32_t j = row_ptr[v]; j < row_ptr[v + 1]; ++j) {
            int32_t x = col[j];
            for (uint32_t i = 0; i < b; ++i)
                B[pgo_bit_position(pgo_hash(seed, i, x), l)] = 1;
        }
    }
}

/* Bloom filter of one explicit set (used by tests on synthetic sets). */
void pgo_bloom_of_set(const int32_t *X, int64_t nx, uint32_t l, uint32_t b,
                      uint32_t seed, uint8_t *out)
{
    memset(out, 0, l);
    for (int64_t j = 0; j < nx; ++j)
        for (uint32_t i = 0; i < b; ++i)
            out[pgo_bit_position(pgo_hash(seed, i, X[j]), l)] = 1;
}

/* Layout only: bit p of each filter -> bit (p % 64) of word (p / 64). */
void pgo_bloom_pack(int32_t n, uint32_t l, const uint8_t *bits,
                    uint64_t *words, int64_t words_per_row)
{
    for (int32_t v = 0; v < n; ++v) {
        uint64_t *w = words + (size_t)v * words_per_row;
        for (int64_t q = 0; q < words_per_row; ++q) w[q] = 0;
        for (uint32_t p = 0; p < l; ++p)
            if (bits[(size_t)v * l + p]) w[p / 64] |= (uint64_t)1 << (p % 64);
    }
}

/* B_{X∩Y,1}: the number of ones of B_X AND B_Y (Sec. IV-B, "In practice"). */
int32_t pgo_bloom_and_ones(const uint8_t *BX, const uint8_t *BY, uint32_t l)
{
    int32_t ones = 0;
    for (uint32_t p = 0; p < l; ++p) ones += (BX[p] & BY[p]);
    return ones;
}

/* B_{X∪Y,1}: the number of ones of BF_X OR BF_Y, the filter of X ∪ Y
 * (Eq. bf_int_union, the OR estimator). */
int32_t pgo_bloom_or_ones(const uint8_t *BX, const uint8_t *BY, uint32_t l)
{
    int32_t ones = 0;
    for (uint32_t p = 0; p < l; ++p) ones += (BX[p] | BY[p]);
    return ones;
}

/* B_{X,1}: the number of ones of one filter. */
int32_t pgo_bloom_ones(const uint8_t *BX, uint32_t l)
{
    int32_t ones = 0;
    for (uint32_t p = 0; p < l; ++p) ones += BX[p];
    return ones;
}

/* ------------------------------------------------------------------------ */
/* MinHash, k-Hash variant (Sec. II-D; estimator Sec. IV-C, reading D).      */
/* ------------------------------------------------------------------------ */

/* M_X = {x_{1,min}, ..., x_{k,min}}: for each hash function i separately the
 * element of X with the smallest h_i. out: n * k element ids (-1 if X empty). */
void pgo_khash_build(int32_t n, const int32_t *row_ptr, const int32_t *col,
                     int32_t k, uint32_t seed, int32_t *out)
{
    for (int32_t v = 0; v < n; ++v) {
        for (int32_t i = 0; i < k; ++i) {
            int32_t best = -1;
            uint32_t best_h = 0;
            for (int32_t j = row_ptr[v]; j < row_ptr[v + 1]; ++j) {
                uint32_t h = pgo_hash(seed, (uint32_t)i, col[j]);
                if (best < 0 || h < best_h) { best = col[j]; best_h = h; }
            }
            out[(size_t)v * k + i] = best;
        }
    }
}

/* |M_X ∩ M_Y| read as the number of hash functions whose minimising
 * elements coincide (reading D); 0 if either set is empty (reading J). */
int32_t pgo_khash_matches(const int32_t *MX, const int32_t *MY, int32_t k)
{
    int32_t c = 0;
    if (k > 0 && (MX[0] < 0 || MY[0] < 0)) return 0;
    for (int32_t i = 0; i < k; ++i) c += (MX[i] == MY[i]);
    return c;
}

/* ------------------------------------------------------------------------ */
/* MinHash, 1-Hash variant (Sec. II-D; estimator Sec. IV-D, reading C).      */
/* ------------------------------------------------------------------------ */

static uint32_t g_sort_seed; /* qsort comparator context (serial oracle) */

static int cmp_by_h0(const void *a, const void *b)
{
    uint32_t ha = pgo_hash(g_sort_seed, 0, *(const int32_t *)a);
    uint32_t hb = pgo_hash(g_sort_seed, 0, *(const int32_t *)b);
    return (ha > hb) - (ha < hb);
}

/* M1_X: the k elements of X with the smallest values of the single hash
 * function h = h_0, stored in increasing order of h; min(k, |X|) of them,
 * remaining slots -1. out: n * k. */
void pgo_onehash_build(int32_t n, const int32_t *row_ptr, const int32_t *col,
                       int32_t k, uint32_t seed, int32_t *out)
{
    int64_t cap = 0;
    int32_t *buf = NULL;
    g_sort_seed = seed;
    for (int32_t v = 0; v < n; ++v) {
        int64_t d = row_ptr[v + 1] - row_ptr[v];
        if (d > cap) { cap = d; buf = (int32_t *)realloc(buf, sizeof(int32_t) * (size_t)cap); }
        if (d) memcpy(buf, col + row_ptr[v], sizeof(int32_t) * (size_t)d);
        if (d > 1) qsort(buf, (size_t)d, sizeof(int32_t), cmp_by_h0);
        for (int32_t i = 0; i < k; ++i)
            out[(size_t)v * k + i] = (i < d) ? buf[i] : -1;
    }
    free(buf);
}

/* Counts of two 1-Hash sketches MX (length lx) and MY (length ly):
 *   c_lit   = |M1_X ∩ M1_Y|                (the formula as printed)
 *   K       = min(k, |M1_X ∪ M1_Y|)
 *   c_union = # elements among the K smallest (by h) of M1_X ∪ M1_Y that
 *             lie in both sketches            (reading C)                 */
void pgo_onehash_counts(const int32_t *MX, int32_t lx, const int32_t *MY,
                        int32_t ly, int32_t k, uint32_t seed,
                        int32_t *c_lit, int32_t *c_union, int32_t *K)
{
    /* union, in increasing order of h_0, by a plain merge of two sorted lists */
    int32_t i = 0, j = 0, taken = 0, lit = 0, cu = 0;
    int32_t Ku;
    int32_t union_size = 0;
    /* pass 1: |union| and c_lit */
    while (i < lx || j < ly) {
        if (j >= ly) { ++i; }
        else if (i >= lx) { ++j; }
        else {
            uint32_t hx = pgo_hash(seed, 0, MX[i]), hy = pgo_hash(seed, 0, MY[j]);
            if (MX[i] == MY[j]) { ++lit; ++i; ++j; }
            else if (hx < hy) ++i;
            else ++j;
        }
        ++union_size;
    }
    Ku = union_size < k ? union_size : k;
    /* pass 2: walk the first Ku union elements, count the common ones */
    i = 0; j = 0;
    while (taken < Ku) {
        if (j >= ly) { ++i; }
        else if (i >= lx) { ++j; }
        else {
            uint32_t hx = pgo_hash(seed, 0, MX[i]), hy = pgo_hash(seed, 0, MY[j]);
            if (MX[i] == MY[j]) { ++cu; ++i; ++j; }
            else if (hx < hy) ++i;
            else ++j;
        }
        ++taken;
    }
    *c_lit = lit;
    *c_union = cu;
    *K = Ku;
}

/* ------------------------------------------------------------------------ */
/* Exact sorted-set intersection (Sec. II-A, Sec. III Listing 1).           */
/* ------------------------------------------------------------------------ */

/* |A ∩ B| of two sorted arrays by a two-pointer merge. */
int64_t pgo_intersect_sorted(const int32_t *A, int64_t la, const int32_t *B, int64_t lb)
{
    int64_t i = 0, j = 0, c = 0;
    while (i < la && j < lb) {
        if (A[i] < B[j]) ++i;
        else if (A[i] > B[j]) ++j;
        else { ++c; ++i; ++j; }
    }
    return c;
}

/* The undirected edge list, each edge once as (u, v) with u < v, in CSR
 * order (u ascending, then v ascending). Returns m; eu/ev may be NULL. */
int64_t pgo_upper_edges(int32_t n, const int32_t *row_ptr, const int32_t *col,
                        int32_t *eu, int32_t *ev)
{
    int64_t m = 0;
    for (int32_t u = 0; u < n; ++u)
        for (int32_t j = row_ptr[u]; j < row_ptr[u + 1]; ++j)
            if (col[j] > u) {
                if (eu) { eu[m] = u; ev[m] = col[j]; }
                ++m;
            }
    return m;
}

/* Exact |N_u ∩ N_v| for P vertex pairs. */
void pgo_exact_pairs(const int32_t *row_ptr, const int32_t *col,
                     const int32_t *pu, const int32_t *pv, int64_t P, int64_t *out)
{
    for (int64_t p = 0; p < P; ++p) {
        int32_t u = pu[p], v = pv[p];
        out[p] = pgo_intersect_sorted(col + row_ptr[u], row_ptr[u + 1] - row_ptr[u],
                                      col + row_ptr[v], row_ptr[v + 1] - row_ptr[v]);
    }
}

/* ------------------------------------------------------------------------ */
/* Per-pair integer counts of the sketches for a list of pairs.             */
/* ------------------------------------------------------------------------ */

void pgo_bloom_pairs(const uint8_t *bits, uint32_t l, const int32_t *pu,
                     const int32_t *pv, int64_t P, int32_t *ones)
{
    for (int64_t p = 0; p < P; ++p)
        ones[p] = pgo_bloom_and_ones(bits + (size_t)pu[p] * l, bits + (size_t)pv[p] * l, l);
}

void pgo_bloom_or_pairs(const uint8_t *bits, uint32_t l, const int32_t *pu,
                        const int32_t *pv, int64_t P, int32_t *ones)
{
    for (int64_t p = 0; p < P; ++p)
        ones[p] = pgo_bloom_or_ones(bits + (size_t)pu[p] * l, bits + (size_t)pv[p] * l, l);
}

void pgo_khash_pairs(const int32_t *M, int32_t k, const int32_t *pu,
                     const int32_t *pv, int64_t P, int32_t *c)
{
    for (int64_t p = 0; p < P; ++p)
        c[p] = pgo_khash_matches(M + (size_t)pu[p] * k, M + (size_t)pv[p] * k, k);
}

void pgo_onehash_pairs(const int32_t *M1, int32_t k, uint32_t seed,
                       const int32_t *row_ptr, const int32_t *pu,
                       const int32_t *pv, int64_t P, int32_t *c_lit,
                       int32_t *c_union, int32_t *K)
{
    for (int64_t p = 0; p < P; ++p) {
        int32_t u = pu[p], v = pv[p];
        int32_t du = row_ptr[u + 1] - row_ptr[u], dv = row_ptr[v + 1] - row_ptr[v];
        int32_t lu = du < k ? du : k, lv = dv < k ? dv : k;
        pgo_onehash_counts(M1 + (size_t)u * k, lu, M1 + (size_t)v * k, lv, k, seed,
                           c_lit + p, c_union + p, K + p);
    }
}

/* Vectorised hash evaluation: out[t] = h_{i}(x[t]) (test helper). */
void pgo_hash_array(uint32_t seed, uint32_t i, const int32_t *x, int64_t cnt, uint32_t *out)
{
    for (int64_t t = 0; t < cnt; ++t) out[t] = pgo_hash(seed, i, x[t]);
}

/* ------------------------------------------------------------------------ */
/* Connected components of a subset of the edges (Jarvis-Patrick clustering,  */
/* Sec. III, Listing "Jarvis-Patrick clustering": the clusters are the      */
/* connected components of (V, C), C = edges whose |N_u ∩ N_v| exceeds tau).  */
/* ------------------------------------------------------------------------ */

static int32_t uf_find(int32_t *parent, int32_t x)
{
    while (parent[x] != x) x = parent[x];
    return x;
}

/* label[v] = smallest vertex id of v's component in the graph (V, {e : keep[e]}),
 * by serial union-find that always makes the smaller root the parent. */
void pgo_components(int32_t n, int64_t m, const int32_t *eu, const int32_t *ev, const uint8_t *keep,
                    int32_t *label)
{
    for (int32_t v = 0; v < n; ++v) label[v] = v;
    for (int64_t e = 0; e < m; ++e) {
        if (!keep[e]) continue;
        int32_t a = uf_find(label, eu[e]), b = uf_find(label, ev[e]);
        if (a == b) continue;
        if (a < b) label[b] = a; else label[a] = b;
    }
    for (int32_t v = 0; v < n; ++v) label[v] = uf_find(label, v);
}

/* ------------------------------------------------------------------------ */
/* 4-clique counting (Sec. III-A, Listing "Reformulated 4-Clique Counting"). */
/* ------------------------------------------------------------------------ */

/* Degree order R: R(v) < R(u) iff (d_v, v) < (d_u, u). N+_v = {u in N_v :
 * R(v) < R(u)}, kept in increasing id order. plus_off[n+1], plus_col[nnz/2]. */
static int before(const int32_t *row_ptr, int32_t v, int32_t u)
{
    int32_t dv = row_ptr[v + 1] - row_ptr[v], du = row_ptr[u + 1] - row_ptr[u];
    return dv < du || (dv == du && v < u);
}

void pgo_orient(int32_t n, const int32_t *row_ptr, const int32_t *col, int32_t *plus_off,
                int32_t *plus_col)
{
    int64_t o = 0;
    for (int32_t v = 0; v < n; ++v) {
        plus_off[v] = (int32_t)o;
        for (int32_t j = row_ptr[v]; j < row_ptr[v + 1]; ++j)
            if (before(row_ptr, v, col[j])) plus_col[o++] = col[j];
    }
    plus_off[n] = (int32_t)o;
}

/* Exact count: for u, v in N+_u, C3 = N+_u ∩ N+_v, and for w in C3 the
 * 4-cliques |N+_w ∩ C3|. Returns the number of 4-cliques; *triangles =
 * sum over (u, v) of |C3|. */
uint64_t pgo_clique4_exact(int32_t n, const int32_t *plus_off, const int32_t *plus_col,
                           uint64_t *triangles)
{
    uint64_t ck = 0, tri = 0;
    int32_t *C3 = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
    for (int32_t u = 0; u < n; ++u) {
        for (int32_t a = plus_off[u]; a < plus_off[u + 1]; ++a) {
            int32_t v = plus_col[a];
            /* C3 = N+_u ∩ N+_v by a two-pointer merge of the sorted lists */
            int32_t i = plus_off[u], j = plus_off[v], c = 0;
            while (i < plus_off[u + 1] && j < plus_off[v + 1]) {
                if (plus_col[i] < plus_col[j]) ++i;
                else if (plus_col[i] > plus_col[j]) ++j;
                else { C3[c++] = plus_col[i]; ++i; ++j; }
            }
            tri += (uint64_t)c;
            for (int32_t t = 0; t < c; ++t) {
                int32_t w = C3[t];
                ck += (uint64_t)pgo_intersect_sorted(plus_col + plus_off[w], plus_off[w + 1] - plus_off[w],
                                                     C3, c);
            }
        }
    }
    free(C3);
    *triangles = tri;
    return ck;
}

/* Bloom version: bits = one byte per bit of the filters of N+_v (n x l).
 * For every 3-clique (u, v, w in C3) the count of ones of
 * BF+_u AND BF+_v AND BF+_w goes into hist[0..l]; returns the number of
 * 3-cliques visited. */
uint64_t pgo_clique4_bloom(int32_t n, const int32_t *plus_off, const int32_t *plus_col,
                           const uint8_t *bits, uint32_t l, uint64_t *hist)
{
    uint64_t tri = 0;
    for (uint32_t j = 0; j <= l; ++j) hist[j] = 0;
    for (int32_t u = 0; u < n; ++u) {
        for (int32_t a = plus_off[u]; a < plus_off[u + 1]; ++a) {
            int32_t v = plus_col[a];
            int32_t i = plus_off[u], j = plus_off[v];
            while (i < plus_off[u + 1] && j < plus_off[v + 1]) {
                if (plus_col[i] < plus_col[j]) ++i;
                else if (plus_col[i] > plus_col[j]) ++j;
                else {
                    int32_t w = plus_col[i];
                    const uint8_t *bu = bits + (size_t)u * l, *bv = bits + (size_t)v * l, *bw = bits + (size_t)w * l;
                    uint32_t ones = 0;
                    for (uint32_t p = 0; p < l; ++p) ones += (bu[p] & bv[p] & bw[p]);
                    hist[ones] += 1;
                    ++tri;
                    ++i;
                    ++j;
                }
            }
        }
    }
    return tri;
}

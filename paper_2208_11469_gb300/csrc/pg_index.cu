// Upper-edge index, CSR validation and fill kernels.
//
// The upper-edge index enumerates every undirected edge once, as (u, v) with
// u < v taken from row u — the sum over E of the TC estimator (Sec. VII)
// and the per-edge sums of Sec. III. upper_off is the exclusive prefix sum
// of the per-vertex upper degrees: upper edge e (the per-edge output order)
// belongs to the vertex u with upper_off[u] <= e < upper_off[u+1] and sits at
// CSR position row_ptr[u+1] - (upper_off[u+1] - e).
//
// The list the passes stream is the same edges grouped by the block of v:
// group j holds the edges with v in [j * 2^shift, (j + 1) * 2^shift), each
// group in upper-edge order (u, then v, ascending), with the degree sum
// d_u + d_v beside each entry; an entry's upper-edge index follows from the
// group offsets (upper_pos). A pass that walks the list in order touches,
// while it is inside one group, only the sketch rows and per-vertex sums of
// that group's vertices (an L2-sized slice at the largest graphs) besides
// the row of u, which repeats along the list.
#include "pg_internal.cuh"

namespace pg {

namespace {

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

__global__ void k_fill_u64(uint64_t *p, size_t count, uint64_t value) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count;
         i += (size_t)gridDim.x * blockDim.x)
        p[i] = value;
}

__global__ void k_fill_f64(double *p, size_t count, double value) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count;
         i += (size_t)gridDim.x * blockDim.x)
        p[i] = value;
}

// Per row u: its upper degree |{v in N_u : v > u}| and the row's upper part
// cut by the vertex groups: segment j holds the entries with v >> shift == j.
// cnt[j * (n + 1) + u] = segment length, seg_end[j * n + u] = CSR position
// one past the segment, deg[u] = d_u (the list writer gathers it for every
// entry). Entry n of upper_off and of every cnt row is set to 0, so that the
// exclusive scans of n + 1 values end with the totals.
//
// All cuts are lower bounds in the sorted row: the upper part starts at the
// first v >= u + 1 and group j - 1 ends at the first v >= j * 2^shift (or at
// the upper start, if that comes later). The groups' searches share one
// length sequence, so they run in lockstep, branch-free: every halving step
// issues the probes of all groups together, and a row costs about log2(d)
// dependent loads rather than one search after another.
__global__ void k_group_count(const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col, int32_t n,
                              int32_t shift, int32_t groups, int32_t *__restrict__ upper_off,
                              int32_t *__restrict__ cnt, int32_t *__restrict__ seg_end,
                              int32_t *__restrict__ deg) {
    const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (u > n) return;
    if (u == n) {
        upper_off[n] = 0;
        for (int32_t j = 0; j < groups; ++j) cnt[(int64_t)j * ((int64_t)n + 1) + n] = 0;
        return;
    }
    const int32_t a = row_ptr[u], end = row_ptr[u + 1];
    deg[u] = end - a;
    // thresholds: x_0 = u + 1 (upper start), x_j = j << shift for 1 <= j < groups (group starts)
    int32_t x[kMaxGroups];
    int32_t base[kMaxGroups];
#pragma unroll
    for (int t = 0; t < kMaxGroups; ++t) {
        x[t] = t == 0 ? (int32_t)(u + 1) : t << shift;  // < n <= INT32_MAX for t < groups
        base[t] = a;
    }
    int32_t len = end - a;
    while (len > 1) {
        const int32_t half = len >> 1;
        int32_t probe[kMaxGroups];
#pragma unroll
        for (int t = 0; t < kMaxGroups; ++t)
            if (t < groups) probe[t] = __ldg(col + base[t] + half);
#pragma unroll
        for (int t = 0; t < kMaxGroups; ++t)
            if (t < groups && probe[t] < x[t]) base[t] += half;
        len -= half;
    }
    if (len == 1) {
#pragma unroll
        for (int t = 0; t < kMaxGroups; ++t)
            if (t < groups && __ldg(col + base[t]) < x[t]) base[t] += 1;
    }
    const int32_t lo = base[0];
    upper_off[u] = end - lo;
    int32_t cur = lo;
#pragma unroll
    for (int t = 0; t < kMaxGroups; ++t) {
        if (t < groups) {
            int32_t stop = end;
            if (t + 1 < groups) stop = base[t + 1] > cur ? base[t + 1] : cur;
            cnt[(int64_t)t * ((int64_t)n + 1) + u] = stop - cur;
            seg_end[(int64_t)t * n + u] = stop;
            cur = stop;
        }
    }
}

// The grouped list: entry i = (eu[i], ev[i]) and the degree sum d_u + d_v, eds[i].
// off = the scanned counts (group j's row u occupies [off_j[u], off_j[u+1]),
// off_j = off + j * (n + 1)); group j spans [off_j[0], off_j[n]) and only its
// rows u < R_j = min(n, (j + 1) * 2^shift) can hold entries (u < v).
//
// Work is cut by merge path: an item is a row visited or an entry written,
// group j's items are its R_j rows and its entries, ordered by row with each
// row followed by its entries, so that D(j, u) = base_j + u + off_j[u]
// (base_j = R_0 + ... + R_{j-1}) items precede row u of group j. A chunk is
// kListItems consecutive items: a warp locates both ends (cut) with a
// 32-way search and walks windows of 32 consecutive rows from the first,
// each lane finding the window row of its output position by a binary
// search over the 32 segment ends held in the lanes. A chunk's cost is
// bounded whether its rows are dense or sparse: where a group's entries
// thin out (its rows just below R_j), the rows themselves fill the chunk.
// d_v is gathered from the degree array the count kernel writes (group j's
// slice, so from L2), and the next window's row data (segment end offsets,
// segment ends, degrees) is loaded while the current window is written.
// Stores are coalesced and each lane has kListUnroll independent loads in
// flight. Entry indices fit in int32 (m <= nnz / 2 < 2^30); item counts may
// not. Writes at or beyond cap are dropped.
constexpr int32_t kListItems = 4096;
constexpr int kListUnroll = 4;

struct ListCut {
    int32_t j, u, e;  // group, first row to walk, first entry
};

__device__ __forceinline__ int64_t group_rows(int32_t j, int32_t n, int32_t shift) {
    const int64_t r = (int64_t)(j + 1) << shift;
    return r < (int64_t)n ? r : (int64_t)n;
}

// The cuts at items d[0] and d[1] (0 <= d <= total), located together so that
// their loads overlap. Group: the last j with D(j, 0) <= d (lane j tests
// group j); row: the largest u in [0, R_j] with u + off_j[u] <= d - base_j.
__device__ __forceinline__ void list_cuts(const int32_t *__restrict__ off, int32_t n, int32_t shift,
                                          int32_t groups, const int64_t d[2], ListCut cut[2],
                                          unsigned lane) {
    int64_t lbase = 0;
    for (int32_t i = 0; i < (int32_t)lane && i < groups; ++i) lbase += group_rows(i, n, shift);
    const int64_t lstart =
        (int32_t)lane < groups ? lbase + off[(int64_t)lane * ((int64_t)n + 1)] : INT64_MAX;
    int64_t t[2], lo[2], hi[2];
    const int32_t *offj[2];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        const unsigned bal = __ballot_sync(0xffffffffu, lstart <= d[s]);  // lane 0 always holds
        const int j = 31 - __clz((int)bal);
        cut[s].j = j;
        t[s] = d[s] - __shfl_sync(0xffffffffu, lbase, j);
        offj[s] = off + (int64_t)j * ((int64_t)n + 1);
        lo[s] = 0;
        hi[s] = group_rows(j, n, shift);
    }
    while (hi[0] - lo[0] >= 32 || hi[1] - lo[1] >= 32) {
        int64_t step[2];
        bool ok[2];
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            // 32 probes reach past hi: lo + 32 * step > hi
            step[s] = hi[s] - lo[s] >= 32 ? (hi[s] - lo[s]) / 32 + 1 : 0;
            const int64_t probe = lo[s] + (int64_t)lane * step[s];
            ok[s] = step[s] > 0 && probe <= hi[s] && probe + offj[s][probe] <= t[s];
        }
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            if (step[s] == 0) continue;  // warp-uniform
            const int last = 31 - __clz((int)__ballot_sync(0xffffffffu, ok[s] || lane == 0));
            const int64_t nlo = lo[s] + (int64_t)last * step[s];
            hi[s] = nlo + step[s] - 1 < hi[s] ? nlo + step[s] - 1 : hi[s];
            lo[s] = nlo;
        }
    }
    bool ok[2];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        const int64_t probe = lo[s] + lane;
        ok[s] = probe <= hi[s] && probe + offj[s][probe] <= t[s];
    }
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        const int64_t u = lo[s] + (31 - __clz((int)__ballot_sync(0xffffffffu, ok[s] || lane == 0)));
        cut[s].u = (int32_t)u;
        cut[s].e = (int32_t)(t[s] - u);
    }
}

__global__ void __launch_bounds__(256, 5) k_group_lists(const int32_t *__restrict__ col, int32_t n, int32_t shift,
                                                     int32_t groups, const int32_t *__restrict__ off,
                                                     const int32_t *__restrict__ seg_end,
                                                     const int32_t *__restrict__ deg,
                                                     int32_t *__restrict__ eu, int32_t *__restrict__ ev,
                                                     int32_t *__restrict__ eds, int64_t cap) {
    const unsigned lane = threadIdx.x & 31u;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    int64_t total = off[(int64_t)(groups - 1) * ((int64_t)n + 1) + n];
    for (int32_t j = 0; j < groups; ++j) total += group_rows(j, n, shift);
    const int32_t cap32 = cap < (int64_t)INT32_MAX ? (int32_t)cap : INT32_MAX;
    for (int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; c * kListItems < total; c += warps) {
        const int64_t d[2] = {c * kListItems, (c + 1) * kListItems < total ? (c + 1) * kListItems : total};
        ListCut cut[2];
        list_cuts(off, n, shift, groups, d, cut, lane);
        for (int32_t j = cut[0].j; j <= cut[1].j; ++j) {
            const int32_t *offj = off + (int64_t)j * ((int64_t)n + 1);
            const int32_t *endj = seg_end + (int64_t)j * n;
            int32_t u0 = j == cut[0].j ? cut[0].u : 0;
            int32_t e = j == cut[0].j ? cut[0].e : offj[0];
            const int32_t s1 = j == cut[1].j ? cut[1].e : offj[n];
            // window rows u0 .. u0+31 (lanes past n repeat row n-1); the next window's row data
            // is loaded while this window's entries are written
            int32_t ul = u0 + (int32_t)lane < n ? u0 + (int32_t)lane : n - 1;
            int32_t off_end_n = offj[ul + 1], se_n = endj[ul], du_n = deg[ul];
            while (e < s1 && u0 < n) {
                const int32_t off_end = off_end_n, se = se_n, du = du_n;
                ul = u0 + 32 + (int32_t)lane < n ? u0 + 32 + (int32_t)lane : n - 1;
                off_end_n = offj[ul + 1];
                se_n = endj[ul];
                du_n = deg[ul];
                const int32_t last_end = __shfl_sync(0xffffffffu, off_end, 31);
                const int32_t wend = s1 < last_end ? s1 : last_end;
                for (int32_t base = e; base < wend; base += 32 * kListUnroll) {
                    // three phases so that all loads of the kListUnroll entries are in flight together:
                    // locate the row and load v, then gather the degrees of v (inside group j's
                    // vertices, so from L2), then store
                    int32_t vs[kListUnroll], rows[kListUnroll], dus[kListUnroll];
#pragma unroll
                    for (int q = 0; q < kListUnroll; ++q) {
                        const int32_t ee = base + 32 * q + (int32_t)lane;
                        int r = 0;  // window rows whose segment ends at or before ee
#pragma unroll
                        for (int step = 16; step >= 1; step >>= 1) {
                            const int32_t pr = __shfl_sync(0xffffffffu, off_end, r + step - 1);
                            if (pr <= ee) r += step;
                        }
                        const int rr = r < 31 ? r : 31;
                        const int32_t oe = __shfl_sync(0xffffffffu, off_end, rr);
                        const int32_t sq = __shfl_sync(0xffffffffu, se, rr);
                        rows[q] = rr;
                        dus[q] = __shfl_sync(0xffffffffu, du, rr);
                        vs[q] = ee < wend ? __ldg(col + (sq - (oe - ee))) : 0;
                    }
                    int32_t dvs[kListUnroll];
#pragma unroll
                    for (int q = 0; q < kListUnroll; ++q)
                        dvs[q] = __ldg(deg + vs[q]);
#pragma unroll
                    for (int q = 0; q < kListUnroll; ++q) {
                        const int32_t ee = base + 32 * q + (int32_t)lane;
                        if (ee < wend && ee < cap32) {
                            eu[ee] = u0 + rows[q];
                            ev[ee] = vs[q];
                            eds[ee] = dus[q] + dvs[q];
                        }
                    }
                }
                e = wend > e ? wend : e;
                u0 += 32;
            }
        }
    }
}

// Block-wide exclusive scan of kScanItems values per thread.
__device__ __forceinline__ int32_t block_exclusive_scan(int32_t v[kScanItems], int32_t *smem_warp,
                                                        int32_t &block_total) {
    int32_t local = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) local += v[i];
    const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    int32_t incl = local;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int32_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= (unsigned)o) incl += t;
    }
    if (lane == 31) smem_warp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int32_t w = (lane < (blockDim.x >> 5)) ? smem_warp[lane] : 0;
        int32_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int32_t t = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= (unsigned)o) wi += t;
        }
        smem_warp[lane] = wi - w;       // exclusive prefix of warp totals
        if (lane == 31) smem_warp[32] = wi;  // block total
    }
    __syncthreads();
    int32_t run = smem_warp[warp] + incl - local;
    block_total = smem_warp[32];
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        int32_t x = v[i];
        v[i] = run;
        run += x;
    }
    return 0;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_tiles(const int32_t *__restrict__ in,
                                                             int64_t count,
                                                             int32_t *__restrict__ tile_sums) {
    __shared__ int32_t smem[33];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + threadIdx.x * kScanItems;
    int32_t v[kScanItems];
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) v[i] = (base + i < count) ? in[base + i] : 0;
    int32_t total;
    block_exclusive_scan(v, smem, total);
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = total;
}

// Exclusive scan of the tile sums by one block, looping over chunks.
__global__ void __launch_bounds__(kScanThreads) k_scan_sums(int32_t *__restrict__ sums,
                                                            int64_t tiles) {
    __shared__ int32_t smem[33];
    int32_t carry = 0;
    for (int64_t c0 = 0; c0 < tiles; c0 += kScanTile) {
        const int64_t base = c0 + threadIdx.x * kScanItems;
        int32_t v[kScanItems];
#pragma unroll
        for (int i = 0; i < kScanItems; ++i) v[i] = (base + i < tiles) ? sums[base + i] : 0;
        int32_t total;
        block_exclusive_scan(v, smem, total);
#pragma unroll
        for (int i = 0; i < kScanItems; ++i)
            if (base + i < tiles) sums[base + i] = v[i] + carry;
        carry += total;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kScanThreads) k_scan_apply(int32_t *__restrict__ data,
                                                             int64_t count,
                                                             const int32_t *__restrict__ tile_off) {
    __shared__ int32_t smem[33];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + threadIdx.x * kScanItems;
    int32_t v[kScanItems];
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) v[i] = (base + i < count) ? data[base + i] : 0;
    int32_t total;
    block_exclusive_scan(v, smem, total);
    const int32_t off = tile_off[blockIdx.x];
#pragma unroll
    for (int i = 0; i < kScanItems; ++i)
        if (base + i < count) data[base + i] = v[i] + off;
}

// ------------------------------------------------------------ validation
// While the check runs, result[0] holds the smallest (code << 40 | index)
// found (all ones = none); k_validate_final unpacks it, so the verdict is
// deterministic: the lowest code wins, then the lowest index.
__device__ __forceinline__ void report(int64_t *result, int64_t code, int64_t where) {
    atomicMin(reinterpret_cast<unsigned long long *>(result),
              ((unsigned long long)code << 40) | (unsigned long long)where);
}

__global__ void k_validate_final(int64_t *result) {
    const unsigned long long key = reinterpret_cast<unsigned long long *>(result)[0];
    if (key == ~0ull) {
        result[0] = 0;
        result[1] = 0;
    } else {
        result[0] = (int64_t)(key >> 40);
        result[1] = (int64_t)(key & ((1ull << 40) - 1));
    }
}

__global__ void k_validate_rows(const int32_t *__restrict__ row_ptr, int32_t n, int64_t nnz,
                                int64_t *result) {
    int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (u > n) return;
    if (u == 0 && row_ptr[0] != 0) report(result, PG_CSR_BAD_ROW_PTR, 0);
    if (u == n && (int64_t)row_ptr[n] != nnz) report(result, PG_CSR_BAD_ROW_PTR, n);
    if (u < n && row_ptr[u] > row_ptr[u + 1]) report(result, PG_CSR_BAD_ROW_PTR, u);
}

__global__ void k_validate_entries(const int32_t *__restrict__ row_ptr,
                                   const int32_t *__restrict__ col, int32_t n, int64_t nnz,
                                   int check_symmetry, int64_t *result) {
    if ((*(volatile unsigned long long *)result >> 40) == PG_CSR_BAD_ROW_PTR) return;  // rows unusable
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < nnz;
         j += (int64_t)gridDim.x * blockDim.x) {
        // owning row: largest u with row_ptr[u] <= j
        int32_t lo = 0, hi = n;
        while (lo < hi) {
            int32_t mid = lo + ((hi - lo + 1) >> 1);
            if (row_ptr[mid] <= j)
                lo = mid;
            else
                hi = mid - 1;
        }
        const int32_t u = lo;
        const int32_t v = col[j];
        if (v < 0 || v >= n) {
            report(result, PG_CSR_OUT_OF_RANGE, j);
            continue;
        }
        if (v == u) {
            report(result, PG_CSR_SELF_LOOP, j);
            continue;
        }
        if (j + 1 < row_ptr[u + 1] && col[j + 1] <= v) {
            report(result, PG_CSR_UNSORTED, j);
            continue;
        }
        if (check_symmetry) {
            int32_t a = row_ptr[v], b = row_ptr[v + 1];
            bool found = false;
            while (a < b) {
                int32_t mid = a + ((b - a) >> 1);
                int32_t w = col[mid];
                if (w == u) {
                    found = true;
                    break;
                }
                if (w < u)
                    a = mid + 1;
                else
                    b = mid;
            }
            if (!found) report(result, PG_CSR_ASYMMETRIC, j);
        }
    }
}

}  // namespace

void launch_fill_u64(uint64_t *p, size_t count, uint64_t value, cudaStream_t s) {
    if (!count) return;
    int grid = (int)((count + 255) / 256);
    if (grid > 4 * device_info().sm_count) grid = 4 * device_info().sm_count;
    k_fill_u64<<<grid, 256, 0, s>>>(p, count, value);
    note_launch();
}

void launch_fill_f64(double *p, size_t count, double value, cudaStream_t s) {
    if (!count) return;
    int grid = (int)((count + 255) / 256);
    if (grid > 8 * device_info().sm_count) grid = 8 * device_info().sm_count;
    k_fill_f64<<<grid, 256, 0, s>>>(p, count, value);
    note_launch();
}

static int64_t scan_tiles(int64_t count) { return (count + kScanTile - 1) / kScanTile; }

// Index layout: upper_off [n+1] | scan scratch | cnt / offsets [G (n+1)] |
// segment ends [G n] | degrees [n] | eu | ev | eds [cap each], where cap = nnz / 2 + 1
// bounds m for a symmetric CSR (m = nnz / 2). For a CSR that is not
// symmetric the lists are cut at cap (consumers read at most cap edges);
// pg_validate_csr detects such graphs.
static int64_t list_cap(int64_t nnz) { return nnz / 2 + 1; }

// Vertex groups of 2^shift ids: at most 8 groups, none below 2^20 vertices
// (a graph of up to 2^20 vertices is one group).
int32_t group_shift(int32_t n) {
    int32_t bits = 0;
    while (bits < 31 && ((int64_t)1 << bits) < (int64_t)n) ++bits;
    const int32_t sh = bits - 3;
    return sh > 20 ? sh : 20;
}

static int32_t group_count(int32_t n, int32_t shift) {
    const int64_t g = ((int64_t)n + ((int64_t)1 << shift) - 1) >> shift;
    return g < 1 ? 1 : (int32_t)g;
}

namespace {
struct IndexLayout {
    size_t scratch, cnt, seg, deg, eu, ev, eds, total;
};
IndexLayout index_layout(int32_t n, int64_t nnz) {
    const int64_t count = (int64_t)n + 1;
    const int32_t G = group_count(n, group_shift(n));
    IndexLayout L{};
    size_t o = round_up(sizeof(int32_t) * (size_t)count, 256);
    L.scratch = o;
    o += round_up(sizeof(int32_t) * (size_t)scan_tiles((int64_t)G * count), 256);
    L.cnt = o;
    o += round_up(sizeof(int32_t) * (size_t)G * (size_t)count, 256);
    L.seg = o;
    o += round_up(sizeof(int32_t) * (size_t)G * (size_t)(n > 0 ? n : 1), 256);
    L.deg = o;
    o += round_up(sizeof(int32_t) * (size_t)(n > 0 ? n : 1), 256);
    const size_t lb = round_up(sizeof(int32_t) * (size_t)list_cap(nnz), 256);
    L.eu = o;
    L.ev = o + lb;
    L.eds = o + 2 * lb;
    L.total = o + 3 * lb;
    return L;
}
}  // namespace

size_t upper_index_bytes(int32_t n, int64_t nnz) { return index_layout(n, nnz).total; }

EdgeIndex edge_index_view(const void *index, int32_t n, int64_t nnz) {
    const uint8_t *b = static_cast<const uint8_t *>(index);
    const IndexLayout L = index_layout(n, nnz);
    EdgeIndex x;
    x.upper_off = reinterpret_cast<const int32_t *>(b);
    x.eu = reinterpret_cast<const int32_t *>(b + L.eu);
    x.ev = reinterpret_cast<const int32_t *>(b + L.ev);
    x.eds = reinterpret_cast<const int32_t *>(b + L.eds);
    x.goff = reinterpret_cast<const int32_t *>(b + L.cnt);
    x.seg_end = reinterpret_cast<const int32_t *>(b + L.seg);
    x.cap = list_cap(nnz);
    x.shift = group_shift(n);
    x.groups = group_count(n, x.shift);
    return x;
}

size_t scan_scratch_bytes(int64_t count) {
    return round_up(sizeof(int32_t) * (size_t)scan_tiles(count), 256);
}

cudaError_t launch_exclusive_scan(int32_t *data, int64_t count, int32_t *scratch, cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    const int64_t tiles = scan_tiles(count);
    k_scan_tiles<<<(unsigned)tiles, kScanThreads, 0, s>>>(data, count, scratch);
    k_scan_sums<<<1, kScanThreads, 0, s>>>(scratch, tiles);
    k_scan_apply<<<(unsigned)tiles, kScanThreads, 0, s>>>(data, count, scratch);
    note_launch(3);
    return cudaGetLastError();
}

cudaError_t launch_upper_index(const int32_t *row_ptr, const int32_t *col, int32_t n, int64_t nnz,
                               void *index, cudaStream_t s) {
    const int64_t count = (int64_t)n + 1;
    uint8_t *b = static_cast<uint8_t *>(index);
    const IndexLayout L = index_layout(n, nnz);
    const int32_t shift = group_shift(n);
    const int32_t G = group_count(n, shift);
    int32_t *upper_off = reinterpret_cast<int32_t *>(b);
    int32_t *scratch = reinterpret_cast<int32_t *>(b + L.scratch);
    int32_t *cnt = reinterpret_cast<int32_t *>(b + L.cnt);
    int32_t *seg = reinterpret_cast<int32_t *>(b + L.seg);
    int32_t *deg = reinterpret_cast<int32_t *>(b + L.deg);
    k_group_count<<<(unsigned)((count + 255) / 256), 256, 0, s>>>(row_ptr, col, n, shift, G, upper_off, cnt, seg,
                                                                 deg);
    note_launch();
    cudaError_t e = launch_exclusive_scan(upper_off, count, scratch, s);
    if (e != cudaSuccess) return e;
    e = launch_exclusive_scan(cnt, (int64_t)G * count, scratch, s);
    if (e != cudaSuccess || n == 0) return e;
    // items: at most G n rows + nnz / 2 + 1 entries
    const int64_t chunks = ((int64_t)G * n + nnz / 2 + 1 + kListItems - 1) / kListItems;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_group_lists, 256, 0);
    if (e != cudaSuccess) return e;
    int64_t grid = (chunks + 7) / 8;
    if (grid > (int64_t)per_sm * device_info().sm_count) grid = (int64_t)per_sm * device_info().sm_count;
    if (grid < 1) grid = 1;
    k_group_lists<<<(unsigned)grid, 256, 0, s>>>(col, n, shift, G, cnt, seg, deg,
                                                 reinterpret_cast<int32_t *>(b + L.eu),
                                                 reinterpret_cast<int32_t *>(b + L.ev),
                                                 reinterpret_cast<int32_t *>(b + L.eds), list_cap(nnz));
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_validate(const int32_t *row_ptr, const int32_t *col, int32_t n, int64_t nnz,
                            int check_symmetry, int64_t *result, cudaStream_t s) {
    launch_fill_u64(reinterpret_cast<uint64_t *>(result), 2, ~0ull, s);
    k_validate_rows<<<(unsigned)(((int64_t)n + 1 + 255) / 256), 256, 0, s>>>(row_ptr, n, nnz,
                                                                              result);
    if (nnz > 0) {
        int64_t grid = (nnz + 255) / 256;
        if (grid > 16 * device_info().sm_count) grid = 16 * device_info().sm_count;
        k_validate_entries<<<(unsigned)grid, 256, 0, s>>>(row_ptr, col, n, nnz, check_symmetry,
                                                          result);
        note_launch();
    }
    k_validate_final<<<1, 1, 0, s>>>(result);
    note_launch(2);
    return cudaGetLastError();
}

}  // namespace pg

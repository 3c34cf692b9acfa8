// Sketch intersection, per-edge estimation and reduction (Sec. IV, Sec. VII).
//
// The work is a list of (u, v) pairs: every upper edge of the graph (the
// lists eu/ev of the edge index: u < v, grouped by the block of v, each group
// in CSR order) or an explicit pair list. Edge lists are dealt to the warps in
// chunks of kChunk consecutive entries, round-robin, so that all warps move
// through the list together and work inside one group of v at a time (its
// sketch rows and per-vertex sums stay in L2); a pair list is cut into one
// contiguous range per warp. Either way the (u, v) loads are coalesced
// streams and consecutive edges share u. Per-edge outputs go to the edge's
// upper-edge index, derived from the group offsets of the edge index.
//   Bloom / k-Hash (k_pass): a group of L lanes holds one sketch row as 16-byte
//     vectors; per iteration it loads the rows of B edges, counts
//     popcount(B_u AND B_v) or equal minima lane-wise and reduce-scatters the
//     counts so that each edge ends on its owner lane, which runs the
//     epilogue (estimate, histogram, per-vertex sums, outputs).
//   1-Hash (k_onehash): one lane per edge merges its two bottom-k rows,
//     staged in shared memory, into c_union among the K smallest values of
//     the union (and the literal common count when asked for).
// Graph totals come from exact integer histograms of the counts (block-local
// in shared memory with 32-bit atomics, merged with 64-bit integer atomics)
// and one fixed-order double dot product in k_tc_finalize, so they are
// deterministic. Per-vertex sums S_v of the estimate use double atomics: one
// per edge at v, one per run of equal u in the warp at u.
#include "pg_internal.cuh"

namespace pg {

namespace {

constexpr int kThreads = 256;

__host__ __device__ __forceinline__ int32_t round_up4(int32_t x) { return (x + 3) & ~3; }

enum Kind { BLOOM = PG_SK_BLOOM, KHASH = PG_SK_KHASH, ONEHASH = PG_SK_1HASH };

struct Params {
    const int32_t *row_ptr;
    const int32_t *col;
    int32_t n;
    const int32_t *upper_off;
    const int32_t *eu;      // upper-edge list (edge source)
    const int32_t *ev;
    const int32_t *eds;     // degree sum d_u + d_v of each list entry
    const int32_t *goff;    // group offsets of the list (groups x (n + 1))
    const int32_t *seg_end; // per group and row, the CSR position one past the row's entries
    int32_t groups;
    int32_t out_upper;      // per-edge outputs at the edge's upper-edge index (else at its list position)
    int32_t u_begin, u_end; // edge source: only the edges whose u lies in [u_begin, u_end)
    int64_t cap;            // list capacity
    const int32_t *pairs;   // pair list (pair source)
    int64_t P;
    const uint8_t *data;
    int64_t stride;
    int32_t nvec;       // 16-byte vectors per row that carry payload
    uint32_t l;         // Bloom bits
    uint32_t k;         // MinHash k
    int32_t est;
    int32_t need_deg;   // per-edge degrees needed
    int32_t need_est;   // per-edge estimate needed (S, cn or jac)
    int32_t need_out;   // some per-edge output is written (its position is needed)
    const double *table;  // estimator table in global memory
    int32_t table_len;
    // outputs
    double *S;
    float *cn;
    float *jac;
    float *ovl;         // overlap similarity per edge/pair
    float *tot;         // total-neighbour similarity per edge/pair
    int32_t *count;
    int32_t *aux;
    uint64_t *hist;
    int32_t hist_len;   // number of uint64 bins
    int32_t want_union; // Bloom OR estimator: also count popcount(row_u OR row_v) (upper 16 bits)
};

__device__ __forceinline__ double fx_to_f64(unsigned long long x) { return fixed_to_f64(x, kFixBits); }

__device__ __forceinline__ uint4 ldg4(const uint8_t *p) {
    return __ldg(reinterpret_cast<const uint4 *>(p));
}

// Per-lane partial count of one edge for Bloom / k-Hash from the lane's
// VPL vectors of each row (vector index g + q*L), already in registers.
template <int KIND, int L, int VPL>
__device__ __forceinline__ uint32_t lane_count(const Params &p, const uint4 (&a)[VPL],
                                               const uint4 (&b)[VPL], unsigned g) {
    uint32_t c = 0;
#pragma unroll
    for (int q = 0; q < VPL; ++q) {
        const uint32_t idx = g + (uint32_t)q * L;
        if (KIND == BLOOM) {
            // 32-bit words at or beyond l/32 are row padding: masked, so the
            // count never exceeds l whatever the padding holds.
            const uint32_t w0 = 4u * idx, wl = p.l / 32u;
            c += __popc(a[q].x & b[q].x) + __popc(a[q].y & b[q].y) +
                 (w0 + 2 < wl ? __popc(a[q].z & b[q].z) + __popc(a[q].w & b[q].w) : 0u);
            if (p.want_union)  // popcount of the OR (filter of the union), l <= 1024 < 2^16
                c += (__popc(a[q].x | b[q].x) + __popc(a[q].y | b[q].y) +
                      (w0 + 2 < wl ? __popc(a[q].z | b[q].z) + __popc(a[q].w | b[q].w) : 0u))
                     << 16;
        } else {
            const uint32_t i0 = 4u * idx;
            c += (i0 + 0 < p.k && a[q].x == b[q].x) + (i0 + 1 < p.k && a[q].y == b[q].y) +
                 (i0 + 2 < p.k && a[q].z == b[q].z) + (i0 + 3 < p.k && a[q].w == b[q].w);
        }
    }
    return c;
}

// ---------------------------------------------------------------------------
// Bloom / k-Hash pass. A group of L lanes holds one sketch row as L 16-byte
// vectors (VPL per lane); it handles B edges per iteration and each edge is
// owned by one lane (every S = L / B lanes), which walks the index for it,
// receives its reduced count and runs its epilogue, so the per-edge scalar
// work is spread over the lanes instead of serialised on a group leader.
//   iteration i:  broadcast (u_t, v_t) of the B edges  ->  issue 2B row loads
//                 -> walk + CSR loads of iteration i+1 (overlaps the loads)
//                 -> popcount / equality per lane -> reduce-scatter -> epilogue
// Shared-memory histograms use 32-bit atomics; the k-Hash degree sums are kept
// as 32-bit low words with a carry counter.

// Reduce-scatter of B per-lane partials over the L lanes of a group: lane g
// ends with the total of edge g / (L / B).
template <int L, int B>
__device__ __forceinline__ uint32_t reduce_scatter(uint32_t (&v)[B], unsigned g) {
    int V = B;
#pragma unroll
    for (int o = L / 2; o > 0; o >>= 1) {
        if (V > 1) {
            const bool hi = (g & (unsigned)o) != 0;
#pragma unroll
            for (int i = 0; i < B / 2; ++i) {
                if (i < V / 2) {
                    const uint32_t send = hi ? v[i] : v[i + V / 2];
                    const uint32_t keep = hi ? v[i + V / 2] : v[i];
                    v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
                }
            }
            V >>= 1;
        } else {
            v[0] += __shfl_xor_sync(0xffffffffu, v[0], o);
        }
    }
    return v[0];
}

// The chunks of a warp. A pair list is cut into one contiguous range per
// warp. An edge list is a sequence of segments, one per vertex group j: the
// group's entries whose u lies in [u_begin, u_end), which are contiguous
// (goff_j[u_begin] .. goff_j[u_end]); each segment is padded to whole chunks
// of kChunk entries in a chunk space, so a chunk never straddles two groups,
// and the warps take chunks round-robin (warp w: chunks w, w + W, ...). The
// segment table sits in shared memory, filled by the block's first warp.
constexpr int64_t kChunk = 1024;

struct SegTable {
    int64_t beg[kMaxGroups];   // list start of segment j
    int64_t end[kMaxGroups];   // list end of segment j
    int64_t vend[kMaxGroups];  // end of segment j in the chunk space
    int64_t total;             // length of the chunk space
    int64_t ch;                // chunk size
    int32_t groups;
};

// Called by all 32 lanes of one warp.
template <bool PAIRS>
__device__ __forceinline__ void seg_table_fill(const Params &p, SegTable &t, int64_t warps) {
    const unsigned lane = lane_id();
    if (PAIRS) {
        if (lane == 0) {
            t.total = p.P;
            t.ch = (p.P + warps - 1) / warps;
            t.groups = 1;
            t.beg[0] = 0;
            t.end[0] = p.P;
            t.vend[0] = p.P;
        }
        return;
    }
    int64_t a = 0, b = 0;
    if ((int32_t)lane < p.groups) {
        const int32_t *gj = p.goff + (int64_t)lane * ((int64_t)p.n + 1);
        a = gj[p.u_begin];
        b = gj[p.u_end];
        if (b > p.cap) b = p.cap;
        if (a > b) a = b;
    }
    int64_t v = (b - a + kChunk - 1) / kChunk * kChunk;  // inclusive scan of the padded lengths
#pragma unroll
    for (int o = 1; o < kMaxGroups; o <<= 1) {
        const int64_t x = __shfl_up_sync(0xffffffffu, v, o);
        if ((int)lane >= o) v += x;
    }
    if ((int32_t)lane < p.groups) {
        t.beg[lane] = a;
        t.end[lane] = b;
        t.vend[lane] = v;
    }
    if ((int32_t)lane == p.groups - 1) {
        t.total = v;
        t.ch = kChunk;
        t.groups = p.groups;
    }
}

// List range [w0, w1) of the chunk that starts at vc; returns its group.
template <bool PAIRS>
__device__ __forceinline__ int32_t seg_range(const SegTable &t, int64_t vc, int64_t &w0, int64_t &w1) {
    if (PAIRS) {
        w0 = vc;
        w1 = vc + t.ch < t.total ? vc + t.ch : t.total;
        return 0;
    }
    int32_t j = 0;
    while (j + 1 < t.groups && t.vend[j] <= vc) ++j;
    const int64_t len = t.end[j] - t.beg[j];
    const int64_t vstart = t.vend[j] - (len + kChunk - 1) / kChunk * kChunk;
    w0 = t.beg[j] + (vc - vstart);
    w1 = w0 + kChunk < t.end[j] ? w0 + kChunk : t.end[j];
    if (w0 > w1) w0 = w1;
    return j;
}

// (u, v) of work item e (u = -1: beyond the range; -2: pair with an id outside
// [0, n)) and, when want_deg, the two degrees. From the edge list with
// SPLIT = false only their sum is exact (du = d_u + d_v, dv = 0), read from
// the list itself; with SPLIT, d_u comes from the row offsets.
template <bool PAIRS, bool SPLIT = true>
__device__ __forceinline__ void item(const Params &p, int64_t e, int64_t w1, bool want_deg, int32_t &u,
                                     int32_t &v, int32_t &du, int32_t &dv) {
    u = v = -1;
    du = dv = 0;
    if (e < w1) {
        if (PAIRS) {
            const int2 pr = __ldg(reinterpret_cast<const int2 *>(p.pairs) + e);
            const bool ok = pr.x >= 0 && pr.x < p.n && pr.y >= 0 && pr.y < p.n;
            u = ok ? pr.x : -2;
            v = ok ? pr.y : -2;
            if (ok && want_deg) {
                du = __ldg(p.row_ptr + u + 1) - __ldg(p.row_ptr + u);
                dv = __ldg(p.row_ptr + v + 1) - __ldg(p.row_ptr + v);
            }
        } else {
            u = __ldg(p.eu + e);
            v = __ldg(p.ev + e);
            if (want_deg) {
                const int32_t ds = __ldg(p.eds + e);
                du = SPLIT ? __ldg(p.row_ptr + u + 1) - __ldg(p.row_ptr + u) : ds;
                dv = SPLIT ? ds - du : 0;
            }
        }
    }
}

// Output position of work item e of group j with source u: its upper-edge
// index for the edge source when per-edge outputs go there, else e itself.
template <bool PAIRS>
__device__ __forceinline__ int64_t out_pos(const Params &p, int32_t j, int32_t u, int64_t e) {
    // one group: the list is in upper-edge order itself
    if (PAIRS || !p.need_out || !p.out_upper || u < 0 || p.groups == 1) return e;
    return upper_pos(p.row_ptr, p.n, p.upper_off, p.goff, p.seg_end, j, u, e);
}

// Per-vertex sums at u for the edge source: lanes hold consecutive edges, so
// equal u form runs of lanes; a segmented suffix sum of the fixed-point
// values leaves each run's total on its first lane, which issues one atomic.
__device__ __forceinline__ void add_u_runs(double *S, int32_t key, unsigned long long val) {
    const unsigned lane = lane_id();
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long ov = __shfl_down_sync(0xffffffffu, val, o);
        const int32_t ok = __shfl_down_sync(0xffffffffu, key, o);
        if (lane + (unsigned)o < 32u && ok == key) val += ov;
    }
    const int32_t prev = __shfl_up_sync(0xffffffffu, key, 1);
    if (key >= 0 && (lane == 0 || prev != key) && val != 0ull) atomicAdd(S + key, fx_to_f64(val));
}

// Similarity outputs of one edge / pair from its estimate (Listing sim):
// I = clamp(est, 0, min(d_u, d_v)); Jaccard I / (d_u + d_v - I), overlap
// I / min(d_u, d_v), total neighbours d_u + d_v - I (0 for a zero denominator).
__device__ __forceinline__ void write_sims(const Params &p, int64_t e, float est_f, int32_t du, int32_t dv) {
    if (p.cn) p.cn[e] = est_f;
    if (p.jac || p.ovl || p.tot) {
        const float fu = (float)du, fv = (float)dv;
        const float mn = fminf(fu, fv);
        const float I = fminf(fmaxf(est_f, 0.0f), mn);
        const float den = fu + fv - I;
        if (p.jac) p.jac[e] = den > 0.0f ? I / den : 0.0f;
        if (p.ovl) p.ovl[e] = mn > 0.0f ? I / mn : 0.0f;
        if (p.tot) p.tot[e] = den;
    }
}

__device__ __forceinline__ void write_zero(const Params &p, int64_t e) {
    if (p.count) p.count[e] = 0;
    if (p.aux) p.aux[e] = 0;
    if (p.cn) p.cn[e] = 0.0f;
    if (p.jac) p.jac[e] = 0.0f;
    if (p.ovl) p.ovl[e] = 0.0f;
    if (p.tot) p.tot[e] = 0.0f;
}

// Fixed-point MinHash estimate V = round(c / (K + c) * 2^42) * (d_u + d_v).
// The per-vertex sums add at most 32 such values per run, so a value at or
// above 2^58 (an edge between two vertices of ~2^16+ neighbours with
// near-identical sketches) is not carried in fixed point: fx_ok = false and
// the caller adds the double estimate directly.
__device__ __forceinline__ unsigned long long minhash_fixed(unsigned long long tv, uint32_t ds, bool &fx_ok) {
    const unsigned long long lo = tv * (unsigned long long)ds;
    fx_ok = __umul64hi(tv, (unsigned long long)ds) == 0ull && lo < (1ull << 58);
    return fx_ok ? lo : 0ull;
}

// Layout of a Bloom / k-Hash pass: a group of L lanes holds a sketch row as
// L x VPL 16-byte vectors and owns B items per iteration (every L/B-th lane
// owns one: it fetches the item, receives its reduced count and runs its
// epilogue). Rows are loaded SB items at a time (registers bound SB); with
// UREUSE the row of u stays in registers while u repeats. MINB = blocks per SM
// the register budget is sized for.
template <int KIND, int L, int VPL, int B, int SB, bool UREUSE, int MINB, bool PAIRS>
__global__ void __launch_bounds__(kThreads, MINB) k_pass(Params p) {
    constexpr int S = L / B;          // lanes per owned item
    constexpr int E = (32 / L) * B;   // items per warp iteration
    extern __shared__ __align__(16) unsigned char smem[];
    // tables: estimate (double), estimate * 2^42 (integer), estimate (float)
    double *tab = reinterpret_cast<double *>(smem);
    unsigned long long *tabV = reinterpret_cast<unsigned long long *>(smem + 8 * (size_t)p.table_len);
    float *tabF = reinterpret_cast<float *>(smem + 16 * (size_t)p.table_len);
    uint32_t *h32 = reinterpret_cast<uint32_t *>(smem + 20 * (size_t)round_up4(p.table_len));
    const int hk = (int)p.k + 1;
    // Bloom: counts [l+1]; k-Hash: counts [k+1], degree-sum low words [k+1], carries [k+1]
    const int h32_len = (KIND == BLOOM) ? (int)p.l + 1 : 3 * hk;
    const bool want_hist = p.hist != nullptr;
    {
        const unsigned long long *gV = reinterpret_cast<const unsigned long long *>(p.table + p.table_len);
        const float *gF = reinterpret_cast<const float *>(p.table + 2 * p.table_len);
        for (int i = threadIdx.x; i < p.table_len; i += blockDim.x) {
            tab[i] = p.table[i];
            tabV[i] = gV[i];
            tabF[i] = gF[i];
        }
    }
    if (want_hist)
        for (int i = threadIdx.x; i < h32_len; i += blockDim.x) h32[i] = 0u;
    __shared__ SegTable s_seg;
    if (threadIdx.x < 32) seg_table_fill<PAIRS>(p, s_seg, (int64_t)gridDim.x * (kThreads >> 5));
    __syncthreads();

    const unsigned lane = lane_id();
    const unsigned g = lane % L;
    const unsigned base = lane - g;
    const bool owner = (g % S) == 0;
    const int slot = (int)(lane / L) * B + (int)(g / S);  // item offset inside an iteration

    int32_t cur_u = -1;  // UREUSE: vertex whose row slice is in cur_row
    unsigned long long dsum = 0ull;  // OR estimator: this lane's sum of d_u + d_v
    uint4 cur_row[VPL];
#pragma unroll
    for (int q = 0; q < VPL; ++q) cur_row[q] = make_uint4(0u, 0u, 0u, 0u);
    const int64_t warp = ((int64_t)blockIdx.x * kThreads + threadIdx.x) >> 5;
    const int64_t warps = (int64_t)gridDim.x * (kThreads >> 5);
    for (int64_t vc = warp * s_seg.ch; vc < s_seg.total; vc += warps * s_seg.ch) {
    int64_t w0, w1;
    const int32_t gj = seg_range<PAIRS>(s_seg, vc, w0, w1);
    const int32_t iters = (int32_t)((w1 - w0 + E - 1) / E);

    int32_t cu, cv, cdu, cdv;
    item<PAIRS>(p, w0 + slot, w1, p.need_deg != 0, cu, cv, cdu, cdv);
    for (int32_t it = 0; it < iters; ++it) {
        const int64_t eb = w0 + (int64_t)it * E;
        // next iteration's work items (independent of this iteration's row loads)
        int32_t nu, nv, ndu, ndv;
        item<PAIRS>(p, eb + E + slot, w1, p.need_deg != 0, nu, nv, ndu, ndv);
        uint32_t part[B];
#pragma unroll
        for (int sb = 0; sb < B; sb += SB) {
            int32_t us[SB], vs[SB];
#pragma unroll
            for (int t = 0; t < SB; ++t) {
                us[t] = __shfl_sync(0xffffffffu, cu, base + (unsigned)((sb + t) * S));
                vs[t] = __shfl_sync(0xffffffffu, cv, base + (unsigned)((sb + t) * S));
            }
            // issue every row load of the sub-batch before any use
            uint4 ra[SB][VPL], rb[SB][VPL];
#pragma unroll
            for (int t = 0; t < SB; ++t) {
                const bool reuse = UREUSE && us[t] == cur_u;
#pragma unroll
                for (int q = 0; q < VPL; ++q) {
                    const int idx = (int)g + q * L;
                    const bool in = us[t] >= 0 && idx < p.nvec;
                    rb[t][q] = in ? ldg4(p.data + (int64_t)vs[t] * p.stride + 16 * idx)
                                  : (KIND == BLOOM ? make_uint4(0u, 0u, 0u, 0u) : make_uint4(1u, 1u, 1u, 1u));
                    if (reuse)
                        ra[t][q] = cur_row[q];
                    else
                        ra[t][q] = in ? ldg4(p.data + (int64_t)us[t] * p.stride + 16 * idx) : make_uint4(0u, 0u, 0u, 0u);
                }
            }
#pragma unroll
            for (int t = 0; t < SB; ++t) part[sb + t] = lane_count<KIND, L, VPL>(p, ra[t], rb[t], g);
            if (UREUSE) {
#pragma unroll
                for (int t = 0; t < SB; ++t) {
                    if (us[t] >= 0) {
                        cur_u = us[t];
#pragma unroll
                        for (int q = 0; q < VPL; ++q) cur_row[q] = ra[t][q];
                    }
                }
            }
        }
        uint32_t c = reduce_scatter<L, B>(part, g);

        // ---- epilogue: the owner lane of each edge
        const int64_t e = owner ? out_pos<PAIRS>(p, gj, cu, eb + slot) : eb + slot;
        unsigned long long V = 0ull;  // estimate * 2^42
        if (owner && cu == -2) write_zero(p, e);  // invalid pair
        if (owner && cu >= 0) {
            if (KIND == KHASH && (cdu == 0 || cdv == 0)) c = 0;
            float est_f = 0.0f;
            double est_d = 0.0;
            bool fx_ok = true;
            const uint32_t ds = (uint32_t)cdu + (uint32_t)cdv;
            if (KIND == BLOOM && p.want_union) {
                // OR estimator: |X| + |Y| + (l/b) log(1 - U~/l), the table holding the logarithm term
                const uint32_t U = c >> 16;
                c &= 0xFFFFu;
                est_d = (double)ds + tab[U];
                est_f = (float)est_d;
                fx_ok = est_d >= 0.0 && est_d < 65536.0;
                V = fx_ok ? __double2ull_rn(ldexp(est_d, kFixBits)) : 0ull;
                if (want_hist) atomicAdd(h32 + U, 1u);
                dsum += ds;
                if (p.aux) p.aux[e] = (int32_t)U;
            } else if (KIND == BLOOM) {
                if (p.need_est) {
                    V = tabV[c];
                    est_d = tab[c];
                    est_f = tabF[c];
                }
                if (want_hist) atomicAdd(h32 + c, 1u);
            } else {
                if (p.need_est) {
                    V = minhash_fixed(tabV[c], ds, fx_ok);
                    est_d = fx_ok ? (p.S ? fx_to_f64(V) : 0.0) : tab[c] * (double)ds;
                    est_f = tabF[c] * (float)ds;
                }
                if (want_hist) {
                    atomicAdd(h32 + c, 1u);
                    const uint32_t old = atomicAdd(h32 + hk + c, ds);
                    if (old + ds < old) atomicAdd(h32 + 2 * hk + c, 1u);
                }
            }
            if (p.count) p.count[e] = (int32_t)c;
            write_sims(p, e, est_f, cdu, cdv);
            if (p.S) {
                atomicAdd(p.S + cv, est_d);
                if (PAIRS || !fx_ok) atomicAdd(p.S + cu, est_d);
            }
        }
        // non-owner lanes carry their owner's u (cu) with a zero value, so runs stay contiguous
        if (!PAIRS && p.S) add_u_runs(p.S, cu, owner ? V : 0ull);
        cu = nu;
        cv = nv;
        cdu = ndu;
        cdv = ndv;
    }
    }

    if (want_hist) {
        if (KIND == BLOOM && p.want_union) {
            // OR estimator: the exact sum of d_u + d_v goes to the bin after the l + 1 union counts
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) dsum += __shfl_xor_sync(0xffffffffu, dsum, o);
            if (lane == 0 && dsum) atomicAdd(reinterpret_cast<unsigned long long *>(p.hist + p.l + 1), dsum);
        }
        __syncthreads();
        if (KIND == BLOOM) {
            for (int i = threadIdx.x; i < h32_len; i += blockDim.x)
                if (h32[i]) atomicAdd(reinterpret_cast<unsigned long long *>(p.hist + i), (unsigned long long)h32[i]);
        } else {
            for (int i = threadIdx.x; i < hk; i += blockDim.x) {
                if (h32[i]) atomicAdd(reinterpret_cast<unsigned long long *>(p.hist + i), (unsigned long long)h32[i]);
                const unsigned long long d = (unsigned long long)h32[hk + i] | ((unsigned long long)h32[2 * hk + i] << 32);
                if (d) atomicAdd(reinterpret_cast<unsigned long long *>(p.hist + hk + i), d);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Lean passes for the common row widths (edge source). Lane l of a warp owns
// item eb + l of a 32-item iteration; a group of L lanes reads one row per
// step as L 16-byte vectors, so an iteration is L steps of 32 / L items.
//   Bloom (L = l / 128 vectors per row, last vector possibly half used): the
//     group's popcount partials are summed with log2(L) xor-shuffles.
//   k-Hash (L = 16 lanes, k / 4 of them hold a vector): each lane counts its
//     equal minima; one warp-wide integer reduction returns the counts of
//     both 16-lane groups at once (group 1's count in the upper 16 bits).
// The row of u stays in registers while u repeats (u is non-decreasing along
// the list); the epilogue is the same as in k_pass, run by every lane for its
// own item.
template <int KIND, int L, int W, int SB, bool UREUSE, int MINB, bool EDGE_OUT>
__global__ void __launch_bounds__(kThreads, MINB) k_lean(Params p) {
    // W: 32-bit words of the row payload (l / 32 for Bloom, k for k-Hash)
    constexpr int NV = (W + 3) / 4;               // vectors per row
    constexpr int VPL = (NV + L - 1) / L;          // vectors per lane: vector g + q L for q < VPL
    static_assert(VPL <= 2, "a row must fit two vectors per lane");
    // k-Hash match counts (at most 64 for the packed forms) of all groups in one integer
    // reduction: 2 groups x 16 bits (L = 16) or 4 groups x 8 bits (L = 8)
    constexpr int kPack = (KIND == KHASH && L == 16) ? 16 : (KIND == KHASH && L == 8 && W <= 255) ? 8 : 0;
    // with 16-bit fields (k = 64) the warp-uniform reduction of each step goes to shared memory and
    // every lane takes its own count once per iteration, instead of a compare, shift, mask and
    // select per step (measured 16.3 -> 16.0 ms at scale 24 together with UREUSE = false)
    constexpr bool kStash = kPack == 16;
    extern __shared__ __align__(16) unsigned char smem[];
    double *tab = reinterpret_cast<double *>(smem);
    unsigned long long *tabV = reinterpret_cast<unsigned long long *>(smem + 8 * (size_t)p.table_len);
    float *tabF = reinterpret_cast<float *>(smem + 16 * (size_t)p.table_len);
    uint32_t *h32 = reinterpret_cast<uint32_t *>(smem + 20 * (size_t)round_up4(p.table_len));
    const int hk = (int)p.k + 1;
    const int h32_len = (KIND == BLOOM) ? (int)p.l + 1 : 3 * hk;
    const bool want_hist = p.hist != nullptr;
    {
        const unsigned long long *gV = reinterpret_cast<const unsigned long long *>(p.table + p.table_len);
        const float *gF = reinterpret_cast<const float *>(p.table + 2 * p.table_len);
        for (int i = threadIdx.x; i < p.table_len; i += blockDim.x) {
            tab[i] = p.table[i];
            tabV[i] = gV[i];
            tabF[i] = gF[i];
        }
    }
    if (want_hist)
        for (int i = threadIdx.x; i < h32_len; i += blockDim.x) h32[i] = 0u;
    __shared__ SegTable s_seg;
    if (threadIdx.x < 32) seg_table_fill<false>(p, s_seg, (int64_t)gridDim.x * (kThreads >> 5));
    __syncthreads();

    const unsigned lane = lane_id();
    const unsigned g = lane & (L - 1);
    const int grp = (int)(lane / L);
    // Lanes past the row's vectors read vector 0 (inside the row) and count nothing;
    // word j of vector x is payload iff 4x + j < W (compile-time for full rows).
    bool ok[VPL][4];
    const uint8_t *rowbase[VPL];
#pragma unroll
    for (int q = 0; q < VPL; ++q) {
        const int x = (int)g + q * L;
        rowbase[q] = p.data + 16 * (x < NV ? x : 0);
#pragma unroll
        for (int w = 0; w < 4; ++w) ok[q][w] = 4 * x + w < W;
    }
    const uint32_t grp_shift = (uint32_t)grp * (uint32_t)kPack;
    const bool need_deg = p.need_deg != 0;
    __shared__ uint32_t s_stash[kStash ? kThreads / 32 : 1][32];
    uint32_t *stash = s_stash[kStash ? threadIdx.x >> 5 : 0];

    int32_t cur_u = -1;
    uint4 cur_row[VPL];
#pragma unroll
    for (int q = 0; q < VPL; ++q) cur_row[q] = make_uint4(0u, 0u, 0u, 0u);
    const int64_t warp = ((int64_t)blockIdx.x * kThreads + threadIdx.x) >> 5;
    const int64_t warps = (int64_t)gridDim.x * (kThreads >> 5);
    for (int64_t vc = warp * s_seg.ch; vc < s_seg.total; vc += warps * s_seg.ch) {
    int64_t w0, w1;
    const int32_t gj = seg_range<false>(s_seg, vc, w0, w1);
    const int32_t iters = (int32_t)((w1 - w0 + 31) / 32);

    int32_t cu, cv, cdu, cdv;
    item<false, EDGE_OUT>(p, w0 + lane, w1, need_deg, cu, cv, cdu, cdv);

    for (int32_t it = 0; it < iters; ++it) {
        const int64_t eb = w0 + (int64_t)it * 32;
        int32_t nu, nv, ndu, ndv;
        item<false, EDGE_OUT>(p, eb + 32 + lane, w1, need_deg, nu, nv, ndu, ndv);
        uint32_t c = 0;
#pragma unroll
        for (int s0 = 0; s0 < L; s0 += SB) {
            int32_t us[SB];
            uint4 ra[SB][VPL], rb[SB][VPL];
#pragma unroll
            for (int t = 0; t < SB; ++t) {
                const unsigned src = (unsigned)(grp * L + s0 + t);  // lane owning this step's item
                us[t] = __shfl_sync(0xffffffffu, cu, src);
                // items past the range read row 0 and count nothing
                const int32_t vs_ = max(__shfl_sync(0xffffffffu, cv, src), 0);
                const bool reuse = UREUSE && us[t] == cur_u;
#pragma unroll
                for (int q = 0; q < VPL; ++q) {
                    rb[t][q] = ldg4(rowbase[q] + (int64_t)vs_ * p.stride);
                    ra[t][q] = reuse ? cur_row[q] : ldg4(rowbase[q] + (int64_t)max(us[t], 0) * p.stride);
                }
            }
#pragma unroll
            for (int t = 0; t < SB; ++t) {
                uint32_t v = 0;
#pragma unroll
                for (int q = 0; q < VPL; ++q) {
                    const uint4 a = ra[t][q], b = rb[t][q];
                    if (KIND == BLOOM) {
                        v += (ok[q][0] ? __popc(a.x & b.x) : 0u) + (ok[q][1] ? __popc(a.y & b.y) : 0u) +
                             (ok[q][2] ? __popc(a.z & b.z) : 0u) + (ok[q][3] ? __popc(a.w & b.w) : 0u);
                    } else {
                        v += (ok[q][0] && a.x == b.x) + (ok[q][1] && a.y == b.y) + (ok[q][2] && a.z == b.z) +
                             (ok[q][3] && a.w == b.w);
                    }
                }
                if (kPack) {
                    // every group's count in one reduction, group grp in bits [grp kPack, (grp + 1) kPack)
                    const uint32_t r = __reduce_add_sync(0xffffffffu, v << grp_shift);
                    if (kStash) {
                        if (lane == 0) stash[s0 + t] = r;  // warp-uniform
                    } else if ((int)g == s0 + t) {
                        c = (r >> grp_shift) & ((1u << kPack) - 1u);
                    }
                } else {
#pragma unroll
                    for (int o = L / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                    if ((int)g == s0 + t) c = v;
                }
            }
            if (UREUSE && us[SB - 1] >= 0) {
                cur_u = us[SB - 1];
#pragma unroll
                for (int q = 0; q < VPL; ++q) cur_row[q] = ra[SB - 1][q];
            }
        }

        if (kStash) {
            __syncwarp();
            c = (stash[g] >> grp_shift) & ((1u << kPack) - 1u);
            __syncwarp();
        }
        // ---- epilogue: every lane, for its own item
        const int64_t e = EDGE_OUT ? out_pos<false>(p, gj, cu, eb + lane) : eb + lane;
        unsigned long long V = 0ull;
        if (cu >= 0) {
            // (edges of the list join two vertices of degree >= 1: no empty sketch here)
            float est_f = 0.0f;
            double est_d = 0.0;
            if (KIND == BLOOM) {
                if (p.need_est) {
                    V = tabV[c];
                    est_d = tab[c];
                    est_f = tabF[c];
                }
                if (want_hist) atomicAdd(h32 + c, 1u);
            } else {
                const uint32_t ds = (uint32_t)cdu + (uint32_t)cdv;
                if (p.need_est) {
                    bool fx_ok;
                    V = minhash_fixed(tabV[c], ds, fx_ok);
                    est_d = fx_ok ? (p.S ? fx_to_f64(V) : 0.0) : tab[c] * (double)ds;
                    if (!fx_ok && p.S) atomicAdd(p.S + cu, est_d);  // too large for the fixed-point run sum
                    est_f = tabF[c] * (float)ds;
                }
                if (want_hist) {
                    atomicAdd(h32 + c, 1u);
                    const uint32_t old = atomicAdd(h32 + hk + c, ds);
                    if (old + ds < old) atomicAdd(h32 + 2 * hk + c, 1u);
                }
            }
            if (EDGE_OUT) {
                if (p.count) p.count[e] = (int32_t)c;
                write_sims(p, e, est_f, cdu, cdv);
            }
            if (p.S) atomicAdd(p.S + cv, est_d);
        }
        if (p.S) add_u_runs(p.S, cu, V);
        cu = nu;
        cv = nv;
        cdu = ndu;
        cdv = ndv;
    }
    }

    if (want_hist) {
        __syncthreads();
        if (KIND == BLOOM) {
            for (int i = threadIdx.x; i < h32_len; i += blockDim.x)
                if (h32[i]) atomicAdd(reinterpret_cast<unsigned long long *>(p.hist + i), (unsigned long long)h32[i]);
        } else {
            for (int i = threadIdx.x; i < hk; i += blockDim.x) {
                if (h32[i]) atomicAdd(reinterpret_cast<unsigned long long *>(p.hist + i), (unsigned long long)h32[i]);
                const unsigned long long d = (unsigned long long)h32[hk + i] | ((unsigned long long)h32[2 * hk + i] << 32);
                if (d) atomicAdd(reinterpret_cast<unsigned long long *>(p.hist + hk + i), d);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// 1-Hash pass: one lane per edge (32 edges per warp iteration). Each lane
// copies its two bottom-k rows into the warp's shared staging area, stored
// transposed (entry i of lane r's row at [i * 32 + r]) so that a lane only
// ever touches its own bank, then merges them itself (reading C):
//   phase 1 - the K = min(k, |S_u ∪ S_v|) smallest distinct values, counting
//             the c_union values present in both rows;
//   phase 2 - (only when the literal count is needed) the rest of the merge,
//             counting the common values of the two whole rows (c_lit).
// A merge step takes the smaller head (both on a tie); rows hold distinct
// values, so each step emits one distinct value of the union. The loops stop
// when no lane of the warp has entries left. Histogram updates are
// aggregated over the lanes with the same bin (one shared atomic per bin).
constexpr int kOneHashWarps = kThreads / 32;

// x (a double in [0, 2^75)) added to the 128-bit integer (lo, hi) as x * 2^52:
// exact for x >= 1 (whose last significant bit is at 2^-52 or above); a
// positive x below 1 would lose its bits below 2^-52 (the KMV union
// estimates are 0 or at least k - 1 >= 1).
__device__ __forceinline__ void add_fixed52(unsigned long long &lo, unsigned long long &hi, double x) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
    const int ex = (int)((bits >> 52) & 0x7FF);
    if (ex == 0) return;  // zero (or subnormal)
    const unsigned long long mant = (bits & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    const int sh = ex - 1023;  // x = mant * 2^(sh - 52), so x * 2^52 = mant * 2^sh
    unsigned long long xl, xh;
    if (sh >= 64) {
        xl = 0ull;
        xh = mant << (sh - 64);
    } else if (sh >= 0) {
        xl = mant << sh;
        xh = sh == 0 ? 0ull : (mant >> (64 - sh));
    } else {
        xl = -sh < 64 ? (mant >> -sh) : 0ull;
        xh = 0ull;
    }
    lo += xl;
    hi += xh + (lo < xl);
}

template <bool PAIRS>
__global__ void __launch_bounds__(kThreads) k_onehash(Params p) {
    extern __shared__ __align__(16) unsigned char smem[];
    double *tab = reinterpret_cast<double *>(smem);
    unsigned long long *tabV = reinterpret_cast<unsigned long long *>(smem + 8 * (size_t)p.table_len);
    float *tabF = reinterpret_cast<float *>(smem + 16 * (size_t)p.table_len);
    uint32_t *h32 = reinterpret_cast<uint32_t *>(smem + 20 * (size_t)round_up4(p.table_len));
    const uint32_t k = p.k;
    const int hk = (int)k + 1, hk2 = hk * hk;
    // counts [(k+1)^2], degree-sum low words and carries [(k+1)^2] each, then
    // literal counts [k+1], literal degree-sum low words and carries [k+1] each
    const int h32_len = 3 * hk2 + 3 * hk;
    const bool want_hist = p.hist != nullptr;
    const bool want_lit = want_hist || p.aux != nullptr || p.est == PG_EST_1H_LITERAL;
    uint32_t *stage = h32 + (want_hist ? round_up4(h32_len) : 0);
    const unsigned lane = lane_id();
    uint32_t *A = stage + (size_t)(threadIdx.x >> 5) * 2 * (k + 1) * 32 + lane;
    uint32_t *Bv = A + (size_t)(k + 1) * 32;
    {
        const unsigned long long *gV = reinterpret_cast<const unsigned long long *>(p.table + p.table_len);
        const float *gF = reinterpret_cast<const float *>(p.table + 2 * p.table_len);
        for (int i = threadIdx.x; i < p.table_len; i += blockDim.x) {
            tab[i] = p.table[i];
            tabV[i] = gV[i];
            tabF[i] = gF[i];
        }
    }
    if (want_hist)
        for (int i = threadIdx.x; i < h32_len; i += blockDim.x) h32[i] = 0u;
    __shared__ SegTable s_seg;
    if (threadIdx.x < 32) seg_table_fill<PAIRS>(p, s_seg, (int64_t)gridDim.x * (kThreads >> 5));
    __syncthreads();

    const int nv4 = (int)((k + 3) / 4);
    const bool kmv = p.est == PG_EST_1H_KMV;
    // KMV totals: this lane's sum of the real union estimates (k - 1) 2^32 / (h_k + 1) of its
    // edges whose union sketch is full, as an exact 128-bit integer x 2^-52
    unsigned long long rlo = 0ull, rhi = 0ull;
    const int64_t warp = ((int64_t)blockIdx.x * kThreads + threadIdx.x) >> 5;
    const int64_t warps = (int64_t)gridDim.x * (kThreads >> 5);
    for (int64_t vc = warp * s_seg.ch; vc < s_seg.total; vc += warps * s_seg.ch) {
    int64_t w0, w1;
    const int32_t gj = seg_range<PAIRS>(s_seg, vc, w0, w1);
    const int32_t iters = (int32_t)((w1 - w0 + 31) / 32);
    for (int32_t it = 0; it < iters; ++it) {
        const int64_t ei = w0 + (int64_t)it * 32 + lane;
        int32_t cu, cv, cdu, cdv;
        item<PAIRS>(p, ei, w1, true, cu, cv, cdu, cdv);
        const int64_t e = out_pos<PAIRS>(p, gj, cu, ei);
        const bool valid = cu >= 0;
        const uint32_t la = valid ? min(k, (uint32_t)cdu) : 0u, lb = valid ? min(k, (uint32_t)cdv) : 0u;
        // stage the two rows (whole 16-byte vectors; entries past min(k, d) are never read)
        if (valid) {
            const uint4 *ru = reinterpret_cast<const uint4 *>(p.data + (int64_t)cu * p.stride);
            const uint4 *rv = reinterpret_cast<const uint4 *>(p.data + (int64_t)cv * p.stride);
            for (int q = 0; q < nv4; ++q) {
                const uint4 x = __ldg(ru + q), y = __ldg(rv + q);
                A[(4 * q + 0) * 32] = x.x;
                A[(4 * q + 1) * 32] = x.y;
                A[(4 * q + 2) * 32] = x.z;
                A[(4 * q + 3) * 32] = x.w;
                Bv[(4 * q + 0) * 32] = y.x;
                Bv[(4 * q + 1) * 32] = y.y;
                Bv[(4 * q + 2) * 32] = y.z;
                Bv[(4 * q + 3) * 32] = y.w;
            }
        }
        __syncwarp();
        // phase 1: the K smallest distinct values of the union (hK: the last of them)
        uint32_t i = 0, j = 0, K = 0, cun = 0, hK = 0;
        for (uint32_t st = 0; st < k; ++st) {
            const bool ha = i < la, hb = j < lb;
            if (!__any_sync(0xffffffffu, ha || hb)) break;
            const uint32_t x = A[i * 32], y = Bv[j * 32];
            const bool ta = ha && (!hb || x <= y);
            const bool tb = hb && (!ha || y <= x);
            K += (ha || hb);
            cun += (ta && tb);
            if (ha || hb) hK = ta ? x : y;
            i += ta;
            j += tb;
        }
        // phase 2: common values among the rest of the two rows
        uint32_t clit = cun;
        if (want_lit) {
            for (uint32_t st = 0; st < 2 * k; ++st) {
                const bool ha = i < la, hb = j < lb;
                if (!__any_sync(0xffffffffu, ha && hb)) break;
                const uint32_t x = A[i * 32], y = Bv[j * 32];
                const bool both = ha && hb;
                clit += (both && x == y);
                i += both && x <= y;
                j += both && y <= x;
            }
        }
        __syncwarp();  // the staging area is rewritten by the next iteration

        // ---- epilogue: every lane for its own edge
        unsigned long long V = 0ull;
        bool fx_ok = true;
        double big = 0.0;
        uint32_t ds = 0;
        if (cu == -2) write_zero(p, e);
        if (valid) {
            ds = (uint32_t)cdu + (uint32_t)cdv;
            const int ti = (p.est == PG_EST_1H_LITERAL) ? (int)k * hk + (int)clit : (int)K * hk + (int)cun;
            V = minhash_fixed(tabV[ti], ds, fx_ok);
            if (!fx_ok) big = tab[ti] * (double)ds;
            float est_f = tabF[ti] * (float)ds;
            if (kmv) {
                // Sec. IX: |X ∪ Y| ~ (k - 1) / max of the union's k smallest hashes in (0, 1];
                // a union of fewer than k values is the whole union
                const double uni = K < k ? (double)K : (double)(k - 1) * 4294967296.0 / ((double)hK + 1.0);
                est_f = (float)((double)ds - uni);
                fx_ok = false;  // per-vertex sums take the double at both ends
                V = 0ull;
                big = (double)ds - uni;
                if (K >= k) add_fixed52(rlo, rhi, uni);
            }
            if (p.aux) p.aux[e] = (int32_t)(K | (clit << 16));
            if (p.count) p.count[e] = (int32_t)((p.est == PG_EST_1H_LITERAL) ? clit : cun);
            write_sims(p, e, est_f, cdu, cdv);
            if (p.S) {
                const double est_d = fx_ok ? fx_to_f64(V) : big;
                atomicAdd(p.S + cv, est_d);
                if (PAIRS || !fx_ok) atomicAdd(p.S + cu, est_d);
            }
        }
        if (!PAIRS && p.S) add_u_runs(p.S, cu, fx_ok ? V : 0ull);
        if (want_hist) {
            // lanes with the same bin add together: one shared atomic per distinct bin
            const uint32_t bin = valid ? K * (uint32_t)hk + cun : 0xFFFFFFFFu;
            const unsigned same = __match_any_sync(0xffffffffu, bin);
            const uint32_t dsum = __reduce_add_sync(same, ds);
            if (valid && (int)lane == __ffs(same) - 1) {
                atomicAdd(h32 + bin, (uint32_t)__popc(same));
                const uint32_t old = atomicAdd(h32 + hk2 + bin, dsum);
                if (old + dsum < old) atomicAdd(h32 + 2 * hk2 + bin, 1u);
            }
            const uint32_t lbin = valid ? clit : 0xFFFFFFFFu;
            const unsigned lsame = __match_any_sync(0xffffffffu, lbin);
            const uint32_t ldsum = __reduce_add_sync(lsame, ds);
            if (valid && (int)lane == __ffs(lsame) - 1) {
                atomicAdd(h32 + 3 * hk2 + lbin, (uint32_t)__popc(lsame));
                const uint32_t old = atomicAdd(h32 + 3 * hk2 + hk + lbin, ldsum);
                if (old + ldsum < old) atomicAdd(h32 + 3 * hk2 + 2 * hk + lbin, 1u);
            }
        }
    }
    }

    if (want_hist && kmv) {
        // exact 128-bit warp sum, then one 128-bit global add (carry from the low word)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long olo = __shfl_xor_sync(0xffffffffu, rlo, o);
            const unsigned long long ohi = __shfl_xor_sync(0xffffffffu, rhi, o);
            rlo += olo;
            rhi += ohi + (rlo < olo);
        }
        if (lane == 0 && (rlo | rhi)) {
            unsigned long long *acc = reinterpret_cast<unsigned long long *>(p.hist + 2 * hk2 + 2 * hk);
            const unsigned long long old = atomicAdd(acc, rlo);
            atomicAdd(acc + 1, rhi + (old + rlo < old ? 1ull : 0ull));
        }
    }
    if (want_hist) {
        __syncthreads();
        for (int i = threadIdx.x; i < hk2; i += blockDim.x) {
            if (h32[i]) atomicAdd(reinterpret_cast<unsigned long long *>(p.hist + i), (unsigned long long)h32[i]);
            const unsigned long long d = (unsigned long long)h32[hk2 + i] | ((unsigned long long)h32[2 * hk2 + i] << 32);
            if (d) atomicAdd(reinterpret_cast<unsigned long long *>(p.hist + hk2 + i), d);
        }
        for (int i = threadIdx.x; i < hk; i += blockDim.x) {
            const uint32_t c = h32[3 * hk2 + i];
            if (c) atomicAdd(reinterpret_cast<unsigned long long *>(p.hist + 2 * hk2 + i), (unsigned long long)c);
            const unsigned long long d = (unsigned long long)h32[3 * hk2 + hk + i] |
                                         ((unsigned long long)h32[3 * hk2 + 2 * hk + i] << 32);
            if (d) atomicAdd(reinterpret_cast<unsigned long long *>(p.hist + 2 * hk2 + hk + i), d);
        }
    }
}

// Estimator tables (double, fixed point * 2^42, float): Bloom f(B1) for
// B1 = 0..l; MinHash r(K, c) = c / (K + c) (the estimate is r * (d_u + d_v)).
__global__ void k_table(double *tab, int32_t len, int32_t kind, int32_t est, uint32_t l, uint32_t b,
                        uint32_t k) {
    unsigned long long *tabV = reinterpret_cast<unsigned long long *>(tab + len);
    float *tabF = reinterpret_cast<float *>(tab + 2 * len);
    for (int32_t i = threadIdx.x; i < len; i += blockDim.x) {
        double v;
        if (kind == BLOOM) {
            const uint32_t j = (uint32_t)i;
            const double B1 = (j == l) ? (double)j - 1.0 : (double)j;
            if (est == PG_EST_BF_L) {
                v = (double)j / (double)b;
            } else if (est == PG_EST_BF_OR) {  // indexed by the union count; the caller adds d_u + d_v
                v = ((double)l / (double)b) * log(1.0 - B1 / (double)l);
            } else if (est == PG_EST_BF_SS) {
                v = log(1.0 - B1 / (double)l) / ((double)b * log(1.0 - 1.0 / (double)l));
            } else {
                v = -((double)l / (double)b) * log(1.0 - B1 / (double)l);
            }
        } else {
            const uint32_t hk = k + 1;
            const uint32_t K = (kind == KHASH) ? k : (uint32_t)i / hk;
            const uint32_t c = (uint32_t)i % hk;
            v = (K + c) > 0 ? (double)c / (double)(K + c) : 0.0;
        }
        tab[i] = v;
        tabV[i] = __double2ull_rn(ldexp(v, kFixBits));
        tabF[i] = (float)v;
    }
}

// Graph totals from the histograms in a fixed order (deterministic): one
// 256-thread block reduces one histogram.
__device__ __forceinline__ void tc_dot_block(const uint64_t *__restrict__ hist, int32_t kind, int32_t est,
                                             uint32_t l, uint32_t b, uint32_t k, pg_tc_result *out) {
    __shared__ double s_main[256], s_alt[256];
    __shared__ unsigned long long s_edges[256], s_sum[256];
    double main_ = 0.0, alt = 0.0;
    unsigned long long edges = 0, sum = 0;
    const uint32_t hk = k + 1;
    if (kind == BLOOM && est == PG_EST_BF_OR) {
        // bins 0..l: union counts; bin l + 1: the exact sum of d_u + d_v
        for (uint32_t j = threadIdx.x; j <= l; j += blockDim.x) {
            const unsigned long long h = hist[j];
            const double U = (j == l) ? (double)j - 1.0 : (double)j;
            main_ += (double)h * (((double)l / (double)b) * log(1.0 - U / (double)l));
            edges += h;
            sum += h * j;
        }
        if (threadIdx.x == 0) main_ += (double)hist[l + 1];
    } else if (kind == BLOOM) {
        for (uint32_t j = threadIdx.x; j <= l; j += blockDim.x) {
            const unsigned long long h = hist[j];
            const double B1 = (j == l) ? (double)j - 1.0 : (double)j;
            const double f_and = -((double)l / (double)b) * log(1.0 - B1 / (double)l);
            const double f_l = (double)j / (double)b;
            const double f_ss = log(1.0 - B1 / (double)l) / ((double)b * log(1.0 - 1.0 / (double)l));
            main_ += (double)h * (est == PG_EST_BF_L ? f_l : est == PG_EST_BF_SS ? f_ss : f_and);
            alt += (double)h * (est == PG_EST_BF_L ? f_and : f_l);
            edges += h;
            sum += h * j;
        }
    } else if (kind == KHASH) {
        for (uint32_t c = threadIdx.x; c < hk; c += blockDim.x) {
            const unsigned long long h = hist[c], hd = hist[hk + c];
            main_ += (double)hd * ((double)c / (double)(k + c));
            edges += h;
            sum += h * c;
        }
    } else if (est == PG_EST_1H_KMV) {
        // sum of d_u + d_v over all edges, minus the exact union sizes K of the edges whose union
        // sketch has fewer than k values, minus the 128-bit sum of the others' real estimates;
        // alt: the c_union / K estimate of the same edges
        const uint32_t hk2 = hk * hk;
        for (uint32_t i = threadIdx.x; i < hk2; i += blockDim.x) {
            const uint32_t K = i / hk, c = i % hk;
            const unsigned long long h = hist[i], hd = hist[hk2 + i];
            main_ += (double)hd - (K < k ? (double)h * (double)K : 0.0);
            alt += (double)hd * ((K + c) > 0 ? (double)c / (double)(K + c) : 0.0);
            edges += h;
            sum += h * c;
        }
        if (threadIdx.x == 0) {
            const unsigned long long rlo = hist[2 * hk2 + 2 * hk], rhi = hist[2 * hk2 + 2 * hk + 1];
            main_ -= (double)rhi * 0x1p12 + (double)rlo * 0x1p-52;
        }
    } else {
        const uint32_t hk2 = hk * hk;
        for (uint32_t i = threadIdx.x; i < hk2; i += blockDim.x) {
            const uint32_t K = i / hk, c = i % hk;
            const unsigned long long h = hist[i], hd = hist[hk2 + i];
            const double r = (K + c) > 0 ? (double)c / (double)(K + c) : 0.0;
            const double lit = (i < hk) ? (double)hist[2 * hk2 + hk + i] * ((double)i / (double)(k + i)) : 0.0;
            main_ += (est == PG_EST_1H_LITERAL) ? lit : (double)hd * r;
            alt += (est == PG_EST_1H_LITERAL) ? (double)hd * r : lit;
            edges += h;
            sum += h * c;
        }
    }
    s_main[threadIdx.x] = main_;
    s_alt[threadIdx.x] = alt;
    s_edges[threadIdx.x] = edges;
    s_sum[threadIdx.x] = sum;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            s_main[threadIdx.x] += s_main[threadIdx.x + o];
            s_alt[threadIdx.x] += s_alt[threadIdx.x + o];
            s_edges[threadIdx.x] += s_edges[threadIdx.x + o];
            s_sum[threadIdx.x] += s_sum[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out->edges = s_edges[0];
        out->count_sum = s_sum[0];
        out->exact_tc = 0;
        out->reserved = 0;
        out->est_tc = s_main[0] / 3.0;
        out->est_tc_alt = s_alt[0] / 3.0;
    }
}

__global__ void __launch_bounds__(256) k_tc_finalize(const uint64_t *__restrict__ hist, int32_t kind,
                                                     int32_t est, uint32_t l, uint32_t b, uint32_t k,
                                                     pg_tc_result *out) {
    tc_dot_block(hist, kind, est, l, b, k, out);
}

// Batch: block g reduces graph g's Bloom histogram with the graph's own l and b.
__global__ void __launch_bounds__(256) k_batch_tc_finalize(const uint64_t *__restrict__ hist,
                                                           const int64_t *__restrict__ hoff,
                                                           const uint32_t *__restrict__ bits_of,
                                                           const uint8_t *__restrict__ b_of, int32_t est,
                                                           pg_tc_result *out) {
    const int g = blockIdx.x;
    tc_dot_block(hist + hoff[g], BLOOM, est, bits_of[g], b_of[g], 0, out + g);
}

__global__ void k_lcc(const int32_t *__restrict__ row_ptr, int32_t n, double *S, float *lcc,
                      double *tri) {
    const int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (v >= n) return;
    const int32_t d = row_ptr[v + 1] - row_ptr[v];
    const double s = S[v];
    if (lcc) lcc[v] = d >= 2 ? (float)s / ((float)d * (float)(d - 1)) : 0.0f;
    if (tri) tri[v] = 0.5 * s;
}

template <bool PAIRS>
cudaError_t run_onehash(const Params &p, cudaStream_t s) {
    const int hk = (int)p.k + 1;
    // tables | histogram | per warp two staged rows of k + 1 entries x 32 lanes
    const size_t smem = 20 * (size_t)round_up4(p.table_len) +
                        (p.hist ? 4 * (size_t)round_up4(3 * hk * hk + 3 * hk) : 0) +
                        4 * (size_t)kOneHashWarps * 2 * (p.k + 1) * 32;
    auto kern = k_onehash<PAIRS>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    kern<<<per_sm * device_info().sm_count, kThreads, smem, s>>>(p);
    note_launch();
    return cudaGetLastError();
}

template <int KIND, int L, int VPL, int B, int SB, bool UREUSE, int MINB, bool PAIRS>
cudaError_t run_pass(const Params &p, cudaStream_t s) {
    const int h32_len = (KIND == BLOOM) ? (int)p.l + 1 : 3 * ((int)p.k + 1);
    const size_t smem = 20 * (size_t)round_up4(p.table_len) + (p.hist ? 4 * (size_t)h32_len : 0);
    auto kern = k_pass<KIND, L, VPL, B, SB, UREUSE, MINB, PAIRS>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    kern<<<per_sm * device_info().sm_count, kThreads, smem, s>>>(p);
    note_launch();
    return cudaGetLastError();
}

template <int KIND, int L, int W, int SB, bool UREUSE, int MINB>
cudaError_t run_lean(const Params &p, cudaStream_t s) {
    const int h32_len = (KIND == BLOOM) ? (int)p.l + 1 : 3 * ((int)p.k + 1);
    const size_t smem = 20 * (size_t)round_up4(p.table_len) + (p.hist ? 4 * (size_t)h32_len : 0);
    // per-edge outputs take their own instance, so that passes without them carry none of that code
    auto kern = p.need_out ? k_lean<KIND, L, W, SB, UREUSE, MINB, true> : k_lean<KIND, L, W, SB, UREUSE, MINB, false>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    kern<<<per_sm * device_info().sm_count, kThreads, smem, s>>>(p);
    note_launch();
    return cudaGetLastError();
}

int pow2_at_least(int x) {
    int y = 1;
    while (y < x) y <<= 1;
    return y;
}

}  // namespace

int64_t hist_bins(int32_t kind, uint32_t l, uint32_t k, int32_t estimator) {
    if (kind == BLOOM) return (int64_t)l + 1 + (estimator == PG_EST_BF_OR ? 1 : 0);
    if (kind == KHASH) return 2 * ((int64_t)k + 1);
    if (kind == ONEHASH)
        return 2 * ((int64_t)k + 1) * (k + 1) + 2 * ((int64_t)k + 1) + (estimator == PG_EST_1H_KMV ? 2 : 0);
    return 0;
}

static int64_t table_len(int32_t kind, uint32_t l, uint32_t k) {
    if (kind == BLOOM) return (int64_t)l + 1;
    if (kind == KHASH) return (int64_t)k + 1;
    return ((int64_t)k + 1) * (k + 1);
}

// The estimator tables sit at the start of the intersect workspace:
// double [len] | uint64 [len] | float [len].
size_t intersect_table_bytes(int32_t kind, uint32_t l, uint32_t k) {
    return round_up(20 * (size_t)table_len(kind, l, k), 256);
}

cudaError_t launch_intersect_ws(const int32_t *row_ptr, const int32_t *col, int32_t n,
                                const EdgeIndex &ix, const int32_t *pairs, int64_t P,
                                const pg_sketch &sk, int32_t estimator, const EdgeOutputs &out,
                                double *table_ws, cudaStream_t s) {
    Params p{};
    p.row_ptr = row_ptr;
    p.col = col;
    p.n = n;
    p.upper_off = ix.upper_off;
    p.eu = ix.eu;
    p.ev = ix.ev;
    p.eds = ix.eds;
    p.out_upper = out.list_order ? 0 : 1;
    p.goff = ix.goff;
    p.seg_end = ix.seg_end;
    p.groups = ix.groups;
    p.u_begin = out.u_begin;
    p.u_end = out.u_end < 0 ? n : out.u_end;
    p.cap = ix.cap;
    p.pairs = pairs;
    p.P = P;
    p.data = static_cast<const uint8_t *>(sk.data);
    p.stride = sk.stride_bytes;
    p.l = sk.bits;
    p.k = sk.k;
    p.est = estimator;
    p.S = out.S;
    p.cn = out.cn;
    p.jac = out.jac;
    p.ovl = out.ovl;
    p.tot = out.tot;
    p.count = out.count;
    p.aux = out.aux;
    p.hist = out.hist;
    p.want_union = (sk.kind == PG_SK_BLOOM && estimator == PG_EST_BF_OR) ? 1 : 0;
    p.hist_len = (int32_t)hist_bins(sk.kind, sk.bits, sk.k, estimator);
    p.table = table_ws;
    p.table_len = (int32_t)table_len(sk.kind, sk.bits, sk.k);
    const bool sims = out.jac || out.ovl || out.tot;
    p.need_est = (out.S || out.cn || sims) ? 1 : 0;
    p.need_out = (out.count || out.aux || out.cn || sims) ? 1 : 0;
    p.need_deg = (sk.kind != PG_SK_BLOOM || sims || p.want_union) ? 1 : 0;
    k_table<<<1, 256, 0, s>>>(table_ws, p.table_len, sk.kind, estimator, sk.bits, sk.b, sk.k);
    note_launch();
    const bool pr = pairs != nullptr;
    if (pr && P == 0) return cudaGetLastError();
    // the OR estimator counts two popcounts per word: generic pass kernels only
#define PG_LEAN(KIND, L, W, SB, UR, MB) \
    if (!pr && !p.want_union) return run_lean<KIND, L, W, SB, UR, MB>(p, s)
#define PG_PASS(KIND, L, VPL, B, SB, UR, MB) \
    return pr ? run_pass<KIND, L, VPL, B, SB, UR, MB, true>(p, s) : run_pass<KIND, L, VPL, B, SB, UR, MB, false>(p, s)
    if (sk.kind == PG_SK_BLOOM) {
        // l <= 1024: at most 8 vectors, one per lane
        p.nvec = (int32_t)(sk.bits / 128 + ((sk.bits % 128) ? 1 : 0));
        switch (pow2_at_least(p.nvec)) {
            case 1: PG_PASS(BLOOM, 1, 1, 1, 1, false, 4);
            case 2:
                if (sk.bits == 192) PG_LEAN(BLOOM, 2, 6, 2, true, 3);
                if (sk.bits == 256) PG_LEAN(BLOOM, 2, 8, 2, true, 3);
                PG_PASS(BLOOM, 2, 1, 2, 2, false, 4);
            case 4:
                if (sk.bits == 448) PG_LEAN(BLOOM, 4, 14, 4, true, 3);
                if (sk.bits == 512) PG_LEAN(BLOOM, 4, 16, 4, true, 3);
                PG_PASS(BLOOM, 4, 1, 4, 4, false, 4);
            default:
                if (sk.bits == 960) PG_LEAN(BLOOM, 8, 30, 2, true, 3);
                if (sk.bits == 1024) PG_LEAN(BLOOM, 8, 32, 2, true, 3);
                PG_PASS(BLOOM, 8, 1, 8, 4, false, 3);
        }
    } else if (sk.kind == PG_SK_KHASH) {
        // k <= 256: up to 64 vectors; at most 16 lanes with up to 4 vectors each
        p.nvec = (int32_t)((sk.k + 3) / 4);
        if (sk.k == 64) PG_LEAN(KHASH, 16, 64, 8, false, 3);
        if (sk.k == 32) PG_LEAN(KHASH, 8, 32, 2, true, 3);
        if (sk.k == 16) PG_LEAN(KHASH, 4, 16, 4, true, 3);
        const int L = pow2_at_least(p.nvec) > 16 ? 16 : pow2_at_least(p.nvec);
        switch (L) {
            case 1: PG_PASS(KHASH, 1, 1, 1, 1, false, 4);
            case 2: PG_PASS(KHASH, 2, 1, 2, 2, false, 4);
            case 4: PG_PASS(KHASH, 4, 1, 4, 4, false, 4);
            case 8: PG_PASS(KHASH, 8, 1, 4, 4, false, 4);
            default:
                if (p.nvec <= 16) PG_PASS(KHASH, 16, 1, 4, 4, false, 4);
                if (p.nvec <= 32) PG_PASS(KHASH, 16, 2, 2, 2, false, 3);
                PG_PASS(KHASH, 16, 4, 1, 1, false, 3);
        }
#undef PG_PASS
#undef PG_LEAN
    } else {
        p.nvec = 0;
        return pr ? run_onehash<true>(p, s) : run_onehash<false>(p, s);
    }
}

cudaError_t launch_estimator_table(double *table_ws, int32_t kind, int32_t estimator, uint32_t l, uint32_t b,
                                   uint32_t k, cudaStream_t s) {
    k_table<<<1, 256, 0, s>>>(table_ws, (int32_t)table_len(kind, l, k), kind, estimator, l, b, k);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_batch_finalize(const uint64_t *hist, const int64_t *hoff, const uint32_t *bits_of,
                                  const uint8_t *b_of, int32_t graphs, int32_t estimator, pg_tc_result *out,
                                  cudaStream_t s) {
    if (graphs <= 0) return cudaSuccess;
    k_batch_tc_finalize<<<graphs, 256, 0, s>>>(hist, hoff, bits_of, b_of, estimator, out);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_tc_finalize(const uint64_t *hist, const pg_sketch &sk, int32_t estimator,
                               pg_tc_result *out, cudaStream_t s) {
    k_tc_finalize<<<1, 256, 0, s>>>(hist, sk.kind, estimator, sk.bits, sk.b, sk.k, out);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_lcc_finalize(const int32_t *row_ptr, int32_t n, double *S, float *lcc,
                                double *tri, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    k_lcc<<<(unsigned)(((int64_t)n + 255) / 256), 256, 0, s>>>(row_ptr, n, S, lcc, tri);
    note_launch();
    return cudaGetLastError();
}

}  // namespace pg

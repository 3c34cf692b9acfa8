// Sketch intersection, per-edge estimation and reduction (Sec. IV, Sec. VII).
//
// One kernel serves all three sketch kinds and both work sources:
//   - every upper edge (u < v) of the graph, enumerated from the upper-edge
//     index, or
//   - an explicit list of vertex pairs.
// A "group" of L lanes handles one edge at a time; each lane loads 16-byte
// vectors of the two sketch rows (the row of u repeats along a CSR row and
// is served from L1), the group reduces its partial count with shuffles and
// the epilogue turns the integer count into the estimate:
//   Bloom : B1 = popcount(B_u AND B_v)          -> Eq. (bf_int) / Eq. (limit_xs)
//   k-Hash: c = #{i : min_i(u) = min_i(v)}        -> Eq. (est_int_mh)
//   1-Hash: c_union, K, c_lit (warp-wide merge)   -> Sec. IV-D
// Graph totals come from exact integer histograms of the counts (block-local
// in shared memory, merged with integer atomics) and one fixed-order double
// dot product in k_tc_finalize, so they are deterministic. Per-vertex sums
// S_v = sum over incident edges of the estimate use double atomics.
//
// Edge partition: the m upper edges are split into Q equal contiguous ranges,
// one per group (a persistent grid of Q groups); each group binary-searches
// its first vertex once and then walks the index.
#include "pg_internal.cuh"

namespace pg {

namespace {

constexpr int kThreads = 256;
constexpr int kBatch = 4;      // edges a group has in flight
constexpr uint32_t kEmpty = 0xFFFFFFFFu;

enum Kind { BLOOM = PG_SK_BLOOM, KHASH = PG_SK_KHASH, ONEHASH = PG_SK_1HASH };

struct Params {
    const int32_t *row_ptr;
    const int32_t *col;
    int32_t n;
    const int32_t *upper_off;
    const int32_t *pairs;
    int64_t P;
    const uint8_t *data;
    int64_t stride;
    int32_t nvec;       // 16-byte vectors per row that carry payload
    uint32_t l;         // Bloom bits
    uint32_t k;         // MinHash k
    int32_t est;
    int32_t need_deg;   // per-edge degrees needed
    int32_t need_est;   // per-edge estimate needed (S, cn or jac)
    const double *table;  // estimator table in global memory
    int32_t table_len;
    // outputs
    double *S;
    float *cn;
    float *jac;
    int32_t *count;
    int32_t *aux;
    uint64_t *hist;
    int32_t hist_len;   // number of uint64 bins
};

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
        } else {
            const uint32_t i0 = 4u * idx;
            c += (i0 + 0 < p.k && a[q].x == b[q].x) + (i0 + 1 < p.k && a[q].y == b[q].y) +
                 (i0 + 2 < p.k && a[q].z == b[q].z) + (i0 + 3 < p.k && a[q].w == b[q].w);
        }
    }
    return c;
}

// 1-Hash counts for one edge, whole warp (lane r holds entry r of each row).
__device__ __forceinline__ void onehash_counts(uint32_t su, uint32_t sv, int la, int lb, int k,
                                               int &c_union, int &K, int &c_lit) {
    const unsigned r = lane_id();
    const uint32_t x = su;
    int pos = 0;
#pragma unroll
    for (int step = 16; step >= 1; step >>= 1) {
        const int probe = pos + step - 1;
        const uint32_t pv = __shfl_sync(0xffffffffu, sv, probe);
        if (probe < lb && pv < x) pos += step;
    }
    const uint32_t pv = __shfl_sync(0xffffffffu, sv, pos & 31);
    bool found = false;
    if (pos < lb) {
        if (pv < x)
            ++pos;
        else
            found = (pv == x);
    }
    found = found && ((int)r < la);
    const unsigned fm = __ballot_sync(0xffffffffu, found);
    c_lit = __popc(fm);
    const int U = la + lb - c_lit;
    K = U < k ? U : k;
    const int rank = (int)r + pos - __popc(fm & ((1u << r) - 1u));
    c_union = __popc(__ballot_sync(0xffffffffu, found && rank < K));
}

template <int KIND, int L, int VPL, bool PAIRS>
__global__ void __launch_bounds__(kThreads) k_intersect(Params p) {
    extern __shared__ __align__(16) unsigned char smem[];
    double *tab = reinterpret_cast<double *>(smem);
    uint64_t *hist = reinterpret_cast<uint64_t *>(smem + 8 * (size_t)p.table_len);
    const bool want_hist = p.hist != nullptr;
    for (int i = threadIdx.x; i < p.table_len; i += blockDim.x) tab[i] = p.table[i];
    if (want_hist)
        for (int i = threadIdx.x; i < p.hist_len; i += blockDim.x) hist[i] = 0ull;
    __syncthreads();

    const unsigned lane = lane_id();
    const unsigned g = lane % L;
    const int64_t group = ((int64_t)blockIdx.x * kThreads + threadIdx.x) / L;
    const int64_t groups = (int64_t)gridDim.x * kThreads / L;
    const uint32_t k = p.k;
    const int hk = (int)k + 1;

    // ---- work range of this group
    int64_t e0, e1;
    if (PAIRS) {
        e0 = group * p.P / groups;
        e1 = (group + 1) * p.P / groups;
    } else {
        const int64_t m = p.upper_off[p.n];
        e0 = group * m / groups;
        e1 = (group + 1) * m / groups;
    }
    // for KIND == ONEHASH (L == 32) the range is warp-uniform by construction

    int32_t u = 0, next_off = 0, row_end = 0;
    if (!PAIRS && e0 < e1) {
        int32_t lo = 0, hi = p.n - 1;  // largest u with upper_off[u] <= e0
        while (lo < hi) {
            const int32_t mid = (lo + hi + 1) >> 1;
            if (p.upper_off[mid] <= e0)
                lo = mid;
            else
                hi = mid - 1;
        }
        u = lo;
        next_off = p.upper_off[u + 1];
        row_end = p.row_ptr[u + 1];
    }
    double acc_u = 0.0;  // sum of estimates of the current u (edge source)
    int32_t acc_vertex = -1;

    // Groups of one warp may own ranges that differ by one edge: iterate the
    // warp-wide maximum number of batches so that every shuffle is converged.
    const int32_t my_batches = (int32_t)((e1 - e0 + kBatch - 1) / kBatch);
    const int32_t warp_batches = __reduce_max_sync(0xffffffffu, (unsigned)my_batches);
    for (int32_t bi = 0; bi < warp_batches; ++bi) {
        const int64_t eb = e0 + (int64_t)bi * kBatch;
        int32_t us[kBatch], vs[kBatch];
#pragma unroll
        for (int t = 0; t < kBatch; ++t) {
            const int64_t e = eb + t;
            us[t] = -1;
            vs[t] = -1;
            if (e < e1) {
                if (PAIRS) {
                    const int2 pr = __ldg(reinterpret_cast<const int2 *>(p.pairs) + e);
                    // an id outside [0, n) makes an invalid pair: all outputs 0
                    const bool ok = pr.x >= 0 && pr.x < p.n && pr.y >= 0 && pr.y < p.n;
                    us[t] = ok ? pr.x : -2;
                    vs[t] = ok ? pr.y : -2;
                } else {
                    while (e >= next_off) {
                        ++u;
                        next_off = p.upper_off[u + 1];
                        row_end = p.row_ptr[u + 1];
                    }
                    us[t] = u;
                    vs[t] = __ldg(p.col + (row_end - (next_off - (int32_t)e)));
                }
            }
        }
        int32_t du[kBatch], dv[kBatch];
        if (p.need_deg || KIND == ONEHASH) {
#pragma unroll
            for (int t = 0; t < kBatch; ++t) {
                du[t] = dv[t] = 0;
                if (us[t] >= 0) {
                    du[t] = __ldg(p.row_ptr + us[t] + 1) - __ldg(p.row_ptr + us[t]);
                    dv[t] = __ldg(p.row_ptr + vs[t] + 1) - __ldg(p.row_ptr + vs[t]);
                }
            }
        }
        int32_t cnt[kBatch], Ks[kBatch], lits[kBatch];
        if (KIND == ONEHASH) {
            uint32_t su[kBatch], sv[kBatch];
#pragma unroll
            for (int t = 0; t < kBatch; ++t) {
                su[t] = sv[t] = kEmpty;
                if (us[t] >= 0 && lane < k) {
                    su[t] = __ldg(reinterpret_cast<const uint32_t *>(p.data + (int64_t)us[t] * p.stride) + lane);
                    sv[t] = __ldg(reinterpret_cast<const uint32_t *>(p.data + (int64_t)vs[t] * p.stride) + lane);
                }
            }
#pragma unroll
            for (int t = 0; t < kBatch; ++t) {
                const int la = min((int)k, du[t]), lb = min((int)k, dv[t]);
                onehash_counts(su[t], sv[t], la, lb, (int)k, cnt[t], Ks[t], lits[t]);
            }
        } else {
            // Issue every row load of the batch before any use, so that a
            // group keeps 2 * kBatch independent 16-byte loads in flight.
            uint4 ra[kBatch][VPL], rb[kBatch][VPL];
#pragma unroll
            for (int t = 0; t < kBatch; ++t) {
#pragma unroll
                for (int q = 0; q < VPL; ++q) {
                    const int idx = (int)g + q * L;
                    if (us[t] >= 0 && idx < p.nvec) {
                        ra[t][q] = ldg4(p.data + (int64_t)us[t] * p.stride + 16 * idx);
                        rb[t][q] = ldg4(p.data + (int64_t)vs[t] * p.stride + 16 * idx);
                    } else {
                        ra[t][q] = make_uint4(0u, 0u, 0u, 0u);
                        rb[t][q] = make_uint4(1u, 1u, 1u, 1u);
                    }
                }
            }
#pragma unroll
            for (int t = 0; t < kBatch; ++t) {
                uint32_t c = lane_count<KIND, L, VPL>(p, ra[t], rb[t], g);
#pragma unroll
                for (int o = L / 2; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
                cnt[t] = (int32_t)c;
                if (KIND == KHASH && us[t] >= 0 && p.need_deg && (du[t] == 0 || dv[t] == 0)) cnt[t] = 0;
            }
        }
        // ---- epilogue (group leader)
#pragma unroll
        for (int t = 0; t < kBatch; ++t) {
            if (PAIRS && us[t] == -2 && g == 0) {
                const int64_t e = eb + t;
                if (p.count) p.count[e] = 0;
                if (p.aux) p.aux[e] = 0;
                if (p.cn) p.cn[e] = 0.0f;
                if (p.jac) p.jac[e] = 0.0f;
            }
            if (us[t] < 0 || g != 0) continue;
            const int64_t e = eb + t;
            const int c = cnt[t];
            double est = 0.0;
            int64_t deg_sum = 0;
            if (KIND == BLOOM) {
                if (p.need_est) est = tab[c];
                if (want_hist) atomicAdd(reinterpret_cast<unsigned long long *>(hist + c), 1ull);
            } else if (KIND == KHASH) {
                deg_sum = (int64_t)du[t] + dv[t];
                if (p.need_est) est = tab[c] * (double)deg_sum;
                if (want_hist) {
                    atomicAdd(reinterpret_cast<unsigned long long *>(hist + c), 1ull);
                    atomicAdd(reinterpret_cast<unsigned long long *>(hist + hk + c), (unsigned long long)deg_sum);
                }
            } else {
                deg_sum = (int64_t)du[t] + dv[t];
                const int Kk = Ks[t], lit = lits[t];
                if (p.need_est) {
                    est = (p.est == PG_EST_1H_LITERAL) ? tab[(int)k * hk + lit] * (double)deg_sum
                                                       : tab[Kk * hk + c] * (double)deg_sum;
                }
                if (want_hist) {
                    const int bin = Kk * hk + c;
                    const int hk2 = hk * hk;
                    atomicAdd(reinterpret_cast<unsigned long long *>(hist + bin), 1ull);
                    atomicAdd(reinterpret_cast<unsigned long long *>(hist + hk2 + bin), (unsigned long long)deg_sum);
                    atomicAdd(reinterpret_cast<unsigned long long *>(hist + 2 * hk2 + lit), 1ull);
                    atomicAdd(reinterpret_cast<unsigned long long *>(hist + 2 * hk2 + hk + lit),
                              (unsigned long long)deg_sum);
                }
                if (p.aux) p.aux[e] = Kk | (lit << 16);
            }
            if (p.count) p.count[e] = (KIND == ONEHASH && p.est == PG_EST_1H_LITERAL) ? lits[t] : c;
            if (p.cn) p.cn[e] = (float)est;
            if (p.jac) {
                const float fu = (float)du[t], fv = (float)dv[t];
                float I = fminf(fmaxf((float)est, 0.0f), fminf(fu, fv));
                const float den = fu + fv - I;
                p.jac[e] = den > 0.0f ? I / den : 0.0f;
            }
            if (p.S) {
                if (PAIRS) {
                    atomicAdd(p.S + us[t], est);
                    atomicAdd(p.S + vs[t], est);
                } else {
                    if (us[t] != acc_vertex) {
                        if (acc_vertex >= 0) atomicAdd(p.S + acc_vertex, acc_u);
                        acc_vertex = us[t];
                        acc_u = 0.0;
                    }
                    acc_u += est;
                    atomicAdd(p.S + vs[t], est);
                }
            }
        }
    }
    if (!PAIRS && p.S && g == 0 && acc_vertex >= 0) atomicAdd(p.S + acc_vertex, acc_u);

    if (want_hist) {
        __syncthreads();
        for (int i = threadIdx.x; i < p.hist_len; i += blockDim.x) {
            const unsigned long long h = hist[i];
            if (h) atomicAdd(reinterpret_cast<unsigned long long *>(p.hist + i), h);
        }
    }
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

template <int KIND, int L, int VPL, int B, bool PAIRS>
__global__ void __launch_bounds__(kThreads) k_pass(Params p) {
    constexpr int S = L / B;  // lanes per owned edge
    extern __shared__ __align__(16) unsigned char smem[];
    double *tab = reinterpret_cast<double *>(smem);
    uint32_t *h32 = reinterpret_cast<uint32_t *>(smem + 8 * (size_t)p.table_len);
    const int hk = (int)p.k + 1;
    // Bloom: counts [l+1]; k-Hash: counts [k+1], degree-sum low words [k+1], carries [k+1]
    const int h32_len = (KIND == BLOOM) ? (int)p.l + 1 : 3 * hk;
    const bool want_hist = p.hist != nullptr;
    for (int i = threadIdx.x; i < p.table_len; i += blockDim.x) tab[i] = p.table[i];
    if (want_hist)
        for (int i = threadIdx.x; i < h32_len; i += blockDim.x) h32[i] = 0u;
    __syncthreads();

    const unsigned lane = lane_id();
    const unsigned g = lane % L;
    const unsigned base = lane - g;
    const int t_own = (int)(g / S);
    const bool owner = (g % S) == 0;
    const int64_t group = ((int64_t)blockIdx.x * kThreads + threadIdx.x) / L;
    const int64_t groups = (int64_t)gridDim.x * kThreads / L;

    int64_t e0, e1;
    if (PAIRS) {
        e0 = group * p.P / groups;
        e1 = (group + 1) * p.P / groups;
    } else {
        const int64_t m = p.upper_off[p.n];
        e0 = group * m / groups;
        e1 = (group + 1) * m / groups;
    }
    // group walk state: vertex u whose upper range holds the next edge
    int32_t gu = 0, g_next = 0, g_end = 0;
    if (!PAIRS && e0 < e1) {
        int32_t lo = 0, hi = p.n - 1;  // largest u with upper_off[u] <= e0
        while (lo < hi) {
            const int32_t mid = (lo + hi + 1) >> 1;
            if (p.upper_off[mid] <= e0)
                lo = mid;
            else
                hi = mid - 1;
        }
        gu = lo;
        g_next = p.upper_off[gu + 1];
        g_end = p.row_ptr[gu + 1];
    }

    // Edge eb + t_own of this lane: (u, v), validity and, for owners, degrees.
    // Returns the walk state after that edge (used by the lane owning t = B-1).
    auto fetch = [&](int64_t eb, int32_t &u_l, int32_t &v_l, int32_t &du_l, int32_t &dv_l,
                     int32_t &nu, int32_t &nn, int32_t &ne) {
        const int64_t e = eb + t_own;
        u_l = -1;
        v_l = -1;
        du_l = dv_l = 0;
        nu = gu;
        nn = g_next;
        ne = g_end;
        if (e < e1) {
            if (PAIRS) {
                const int2 pr = __ldg(reinterpret_cast<const int2 *>(p.pairs) + e);
                const bool ok = pr.x >= 0 && pr.x < p.n && pr.y >= 0 && pr.y < p.n;
                u_l = ok ? pr.x : -2;
                v_l = ok ? pr.y : -2;
                if (ok && p.need_deg && owner) {
                    du_l = __ldg(p.row_ptr + u_l + 1) - __ldg(p.row_ptr + u_l);
                    dv_l = __ldg(p.row_ptr + v_l + 1) - __ldg(p.row_ptr + v_l);
                }
            } else {
                while (e >= nn) {
                    ++nu;
                    nn = p.upper_off[nu + 1];
                    ne = p.row_ptr[nu + 1];
                }
                u_l = nu;
                v_l = __ldg(p.col + (ne - (nn - (int32_t)e)));
                if (p.need_deg && owner) {
                    du_l = ne - __ldg(p.row_ptr + nu);
                    dv_l = __ldg(p.row_ptr + v_l + 1) - __ldg(p.row_ptr + v_l);
                }
            }
        }
    };

    double acc_u = 0.0;
    int32_t acc_vertex = -1;
    const int32_t my_iters = (int32_t)((e1 - e0 + B - 1) / B);
    const int32_t warp_iters = (int32_t)__reduce_max_sync(0xffffffffu, (unsigned)(my_iters > 0 ? my_iters : 0));

    int32_t cu, cv, cdu, cdv;
    {
        int32_t nu, nn, ne;
        fetch(e0, cu, cv, cdu, cdv, nu, nn, ne);
        const unsigned last = base + (unsigned)((B - 1) * S);
        gu = __shfl_sync(0xffffffffu, nu, last);
        g_next = __shfl_sync(0xffffffffu, nn, last);
        g_end = __shfl_sync(0xffffffffu, ne, last);
    }
    for (int32_t it = 0; it < warp_iters; ++it) {
        const int64_t eb = e0 + (int64_t)it * B;
        // broadcast the B edges of this iteration to every lane of the group
        int32_t us[B], vs[B];
#pragma unroll
        for (int t = 0; t < B; ++t) {
            us[t] = __shfl_sync(0xffffffffu, cu, base + (unsigned)(t * S));
            vs[t] = __shfl_sync(0xffffffffu, cv, base + (unsigned)(t * S));
        }
        uint4 ra[B][VPL], rb[B][VPL];
#pragma unroll
        for (int t = 0; t < B; ++t) {
#pragma unroll
            for (int q = 0; q < VPL; ++q) {
                const int idx = (int)g + q * L;
                if (us[t] >= 0 && idx < p.nvec) {
                    ra[t][q] = ldg4(p.data + (int64_t)us[t] * p.stride + 16 * idx);
                    rb[t][q] = ldg4(p.data + (int64_t)vs[t] * p.stride + 16 * idx);
                } else {
                    ra[t][q] = make_uint4(0u, 0u, 0u, 0u);
                    rb[t][q] = make_uint4(1u, 1u, 1u, 1u);
                }
            }
        }
        // next iteration's edges (independent of the row loads above)
        int32_t nu_, nv_, ndu, ndv;
        {
            int32_t su, sn, se;
            fetch(eb + B, nu_, nv_, ndu, ndv, su, sn, se);
            const unsigned last = base + (unsigned)((B - 1) * S);
            gu = __shfl_sync(0xffffffffu, su, last);
            g_next = __shfl_sync(0xffffffffu, sn, last);
            g_end = __shfl_sync(0xffffffffu, se, last);
        }
        uint32_t part[B];
#pragma unroll
        for (int t = 0; t < B; ++t) part[t] = lane_count<KIND, L, VPL>(p, ra[t], rb[t], g);
        uint32_t c = reduce_scatter<L, B>(part, g);

        // ---- epilogue: the owner lane of each edge
        const int64_t e = eb + t_own;
        if (owner && cu == -2) {  // invalid pair
            if (p.count) p.count[e] = 0;
            if (p.cn) p.cn[e] = 0.0f;
            if (p.jac) p.jac[e] = 0.0f;
        }
        if (owner && cu >= 0) {
            if (KIND == KHASH && p.need_deg && (cdu == 0 || cdv == 0)) c = 0;
            double est = 0.0;
            if (KIND == BLOOM) {
                if (p.need_est) est = tab[c];
                if (want_hist) atomicAdd(h32 + c, 1u);
            } else {
                const uint32_t ds = (uint32_t)cdu + (uint32_t)cdv;
                if (p.need_est) est = tab[c] * (double)ds;
                if (want_hist) {
                    atomicAdd(h32 + c, 1u);
                    const uint32_t old = atomicAdd(h32 + hk + c, ds);
                    if (old + ds < old) atomicAdd(h32 + 2 * hk + c, 1u);
                }
            }
            if (p.count) p.count[e] = (int32_t)c;
            if (p.cn) p.cn[e] = (float)est;
            if (p.jac) {
                const float fu = (float)cdu, fv = (float)cdv;
                const float I = fminf(fmaxf((float)est, 0.0f), fminf(fu, fv));
                const float den = fu + fv - I;
                p.jac[e] = den > 0.0f ? I / den : 0.0f;
            }
            if (p.S) {
                if (PAIRS) {
                    atomicAdd(p.S + cu, est);
                    atomicAdd(p.S + cv, est);
                } else {
                    if (cu != acc_vertex) {
                        if (acc_vertex >= 0) atomicAdd(p.S + acc_vertex, acc_u);
                        acc_vertex = cu;
                        acc_u = 0.0;
                    }
                    acc_u += est;
                    atomicAdd(p.S + cv, est);
                }
            }
        }
        cu = nu_;
        cv = nv_;
        cdu = ndu;
        cdv = ndv;
    }
    if (!PAIRS && p.S && acc_vertex >= 0) atomicAdd(p.S + acc_vertex, acc_u);

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

// Estimator table: Bloom f(B1) for B1 = 0..l; MinHash r(K, c) = c / (K + c).
__global__ void k_table(double *tab, int32_t kind, int32_t est, uint32_t l, uint32_t b, uint32_t k) {
    if (kind == BLOOM) {
        for (uint32_t j = threadIdx.x; j <= l; j += blockDim.x) {
            if (est == PG_EST_BF_L) {
                tab[j] = (double)j / (double)b;
            } else {
                const double B1 = (j == l) ? (double)j - 1.0 : (double)j;
                tab[j] = -((double)l / (double)b) * log(1.0 - B1 / (double)l);
            }
        }
    } else {
        const uint32_t hk = k + 1;
        const uint32_t rows = (kind == KHASH) ? 1u : hk;
        for (uint32_t i = threadIdx.x; i < rows * hk; i += blockDim.x) {
            const uint32_t K = (kind == KHASH) ? k : i / hk;
            const uint32_t c = i % hk;
            tab[i] = (K + c) > 0 ? (double)c / (double)(K + c) : 0.0;
        }
    }
}

// Graph totals from the histograms in a fixed order (deterministic).
__global__ void __launch_bounds__(256) k_tc_finalize(const uint64_t *__restrict__ hist,
                                                     int32_t kind, int32_t est, uint32_t l,
                                                     uint32_t b, uint32_t k,
                                                     pg_tc_result *out) {
    __shared__ double s_main[256], s_alt[256];
    __shared__ unsigned long long s_edges[256], s_sum[256];
    double main_ = 0.0, alt = 0.0;
    unsigned long long edges = 0, sum = 0;
    const uint32_t hk = k + 1;
    if (kind == BLOOM) {
        for (uint32_t j = threadIdx.x; j <= l; j += blockDim.x) {
            const unsigned long long h = hist[j];
            const double B1 = (j == l) ? (double)j - 1.0 : (double)j;
            const double f_and = -((double)l / (double)b) * log(1.0 - B1 / (double)l);
            const double f_l = (double)j / (double)b;
            main_ += (double)h * (est == PG_EST_BF_L ? f_l : f_and);
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

__global__ void k_lcc(const int32_t *__restrict__ row_ptr, int32_t n, double *S, float *lcc,
                      double *tri) {
    const int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (v >= n) return;
    const int32_t d = row_ptr[v + 1] - row_ptr[v];
    const double s = S[v];
    if (lcc) lcc[v] = d >= 2 ? (float)s / ((float)d * (float)(d - 1)) : 0.0f;
    if (tri) tri[v] = 0.5 * s;
}

template <int KIND, int L, int VPL, bool PAIRS>
cudaError_t run(const Params &p, cudaStream_t s) {
    const size_t smem = 8 * (size_t)p.table_len + (p.hist ? 8 * (size_t)p.hist_len : 0);
    auto kern = k_intersect<KIND, L, VPL, PAIRS>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    const int grid = per_sm * device_info().sm_count;
    kern<<<grid, kThreads, smem, s>>>(p);
    note_launch();
    return cudaGetLastError();
}

template <int KIND, int L, int VPL, int B, bool PAIRS>
cudaError_t run_pass(const Params &p, cudaStream_t s) {
    const int h32_len = (KIND == BLOOM) ? (int)p.l + 1 : 3 * ((int)p.k + 1);
    const size_t smem = 8 * (size_t)p.table_len + (p.hist ? 4 * (size_t)h32_len : 0);
    auto kern = k_pass<KIND, L, VPL, B, PAIRS>;
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

int64_t hist_bins(int32_t kind, uint32_t l, uint32_t k) {
    if (kind == BLOOM) return (int64_t)l + 1;
    if (kind == KHASH) return 2 * ((int64_t)k + 1);
    if (kind == ONEHASH) return 2 * ((int64_t)k + 1) * (k + 1) + 2 * ((int64_t)k + 1);
    return 0;
}

static int64_t table_len(int32_t kind, uint32_t l, uint32_t k) {
    if (kind == BLOOM) return (int64_t)l + 1;
    if (kind == KHASH) return (int64_t)k + 1;
    return ((int64_t)k + 1) * (k + 1);
}

// The estimator table sits at the start of the intersect workspace.
size_t intersect_table_bytes(int32_t kind, uint32_t l, uint32_t k) {
    return round_up(8 * (size_t)table_len(kind, l, k), 256);
}

cudaError_t launch_intersect_ws(const int32_t *row_ptr, const int32_t *col, int32_t n,
                                const int32_t *upper_off, const int32_t *pairs, int64_t P,
                                const pg_sketch &sk, int32_t estimator, const EdgeOutputs &out,
                                double *table_ws, cudaStream_t s) {
    Params p{};
    p.row_ptr = row_ptr;
    p.col = col;
    p.n = n;
    p.upper_off = upper_off;
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
    p.count = out.count;
    p.aux = out.aux;
    p.hist = out.hist;
    p.hist_len = (int32_t)hist_bins(sk.kind, sk.bits, sk.k);
    p.table = table_ws;
    p.table_len = (int32_t)table_len(sk.kind, sk.bits, sk.k);
    p.need_est = (out.S || out.cn || out.jac) ? 1 : 0;
    p.need_deg = (sk.kind != PG_SK_BLOOM || out.jac) ? 1 : 0;
    k_table<<<1, 256, 0, s>>>(table_ws, sk.kind, estimator, sk.bits, sk.b, sk.k);
    note_launch();
    const bool pr = pairs != nullptr;
    if (pr && P == 0) return cudaGetLastError();
    if (sk.kind == PG_SK_BLOOM) {
        // l <= 1024: at most 8 vectors, one per lane; B = min(L, 4) edges per group
        p.nvec = (int32_t)(sk.bits / 128 + ((sk.bits % 128) ? 1 : 0));
        const int L = pow2_at_least(p.nvec);
        switch (L) {
            case 1: return pr ? run_pass<BLOOM, 1, 1, 1, true>(p, s) : run_pass<BLOOM, 1, 1, 1, false>(p, s);
            case 2: return pr ? run_pass<BLOOM, 2, 1, 2, true>(p, s) : run_pass<BLOOM, 2, 1, 2, false>(p, s);
            case 4: return pr ? run_pass<BLOOM, 4, 1, 4, true>(p, s) : run_pass<BLOOM, 4, 1, 4, false>(p, s);
            default: return pr ? run_pass<BLOOM, 8, 1, 4, true>(p, s) : run_pass<BLOOM, 8, 1, 4, false>(p, s);
        }
    } else if (sk.kind == PG_SK_KHASH) {
        // k <= 256: up to 64 vectors; at most 16 lanes with up to 4 vectors each
        p.nvec = (int32_t)((sk.k + 3) / 4);
        const int L = pow2_at_least(p.nvec) > 16 ? 16 : pow2_at_least(p.nvec);
        if (L < 16) {
            switch (L) {
                case 1: return pr ? run_pass<KHASH, 1, 1, 1, true>(p, s) : run_pass<KHASH, 1, 1, 1, false>(p, s);
                case 2: return pr ? run_pass<KHASH, 2, 1, 2, true>(p, s) : run_pass<KHASH, 2, 1, 2, false>(p, s);
                case 4: return pr ? run_pass<KHASH, 4, 1, 4, true>(p, s) : run_pass<KHASH, 4, 1, 4, false>(p, s);
                default: return pr ? run_pass<KHASH, 8, 1, 4, true>(p, s) : run_pass<KHASH, 8, 1, 4, false>(p, s);
            }
        }
        if (p.nvec <= 16) return pr ? run_pass<KHASH, 16, 1, 4, true>(p, s) : run_pass<KHASH, 16, 1, 4, false>(p, s);
        if (p.nvec <= 32) return pr ? run_pass<KHASH, 16, 2, 2, true>(p, s) : run_pass<KHASH, 16, 2, 2, false>(p, s);
        return pr ? run_pass<KHASH, 16, 4, 1, true>(p, s) : run_pass<KHASH, 16, 4, 1, false>(p, s);
    } else {
        p.nvec = 0;
        return pr ? run<ONEHASH, 32, 1, true>(p, s) : run<ONEHASH, 32, 1, false>(p, s);
    }
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

"""Python face of the ProbGraph CPU oracle (pg_oracle.c) plus the plain
numpy reductions that turn per-edge counts into the graph results.

TEST INFRASTRUCTURE. Only tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline leg may import this module. It never imports the CUDA library
and the CUDA library never imports it.

Every function restates one passage of Besta et al., SC'22 (ProbGraph):
  * sketches:   Sec. II-D (Bloom filter, k-Hash, 1-Hash)
  * estimators: Eq. (est_ss_bf), Eq. (bf_int), Eq. (limit_xs),
                Eq. (est_int_mh), Sec. IV-D and the KMV estimator of
                Sec. IX (est_kmv)
  * reductions: the TC estimator of Sec. VII, (1/3) * sum over edges;
                per-vertex triangles and the local clustering coefficient
                (Sec. III-A "clustering coefficient", standard local form);
                Jaccard / common neighbours of Listings 3 and 6.
The readings taken where the paper is silent are listed at the top of
pg_oracle.c and in the design notes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pg_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libpg_oracle.so")
_lock = threading.Lock()
_lib = None

EST_EXACT, EST_BF_AND, EST_BF_L, EST_KH, EST_1H, EST_1H_LITERAL = 0, 1, 2, 3, 4, 5
EST_BF_OR, EST_BF_SS, EST_1H_KMV = 6, 7, 8


def build(force: bool = False) -> str:
    """Compile pg_oracle.c with the host C compiler (plain -O3, portable: no
    machine-specific flags, so the same source builds on x86-64 and Arm)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O3", "-std=c99", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            u32, i32, i64, vp = ctypes.c_uint32, ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p
            sig = {
                "pgo_fmix32": (u32, [u32]),
                "pgo_hash_seed": (u32, [u32, u32]),
                "pgo_hash": (u32, [u32, u32, i32]),
                "pgo_bit_position": (u32, [u32, u32]),
                "pgo_bloom_build": (None, [i32, vp, vp, u32, u32, u32, vp]),
                "pgo_bloom_of_set": (None, [vp, i64, u32, u32, u32, vp]),
                "pgo_bloom_pack": (None, [i32, u32, vp, vp, i64]),
                "pgo_bloom_and_ones": (i32, [vp, vp, u32]),
                "pgo_bloom_ones": (i32, [vp, u32]),
                "pgo_khash_build": (None, [i32, vp, vp, i32, u32, vp]),
                "pgo_khash_matches": (i32, [vp, vp, i32]),
                "pgo_onehash_build": (None, [i32, vp, vp, i32, u32, vp]),
                "pgo_onehash_counts": (None, [vp, i32, vp, i32, i32, u32, vp, vp, vp]),
                "pgo_intersect_sorted": (i64, [vp, i64, vp, i64]),
                "pgo_upper_edges": (i64, [i32, vp, vp, vp, vp]),
                "pgo_exact_pairs": (None, [vp, vp, vp, vp, i64, vp]),
                "pgo_bloom_pairs": (None, [vp, u32, vp, vp, i64, vp]),
                "pgo_khash_pairs": (None, [vp, i32, vp, vp, i64, vp]),
                "pgo_onehash_pairs": (None, [vp, i32, u32, vp, vp, vp, i64, vp, vp, vp]),
                "pgo_hash_array": (None, [u32, u32, vp, i64, vp]),
                "pgo_components": (None, [i32, i64, vp, vp, vp, vp]),
                "pgo_bloom_or_ones": (i32, [vp, vp, u32]),
                "pgo_bloom_or_pairs": (None, [vp, u32, vp, vp, i64, vp]),
                "pgo_orient": (None, [i32, vp, vp, vp, vp]),
                "pgo_clique4_exact": (ctypes.c_uint64, [i32, vp, vp, vp]),
                "pgo_clique4_bloom": (ctypes.c_uint64, [i32, vp, vp, vp, u32, vp]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _csr(row_ptr, col):
    rp = np.ascontiguousarray(np.asarray(row_ptr), dtype=np.int32)
    cl = np.ascontiguousarray(np.asarray(col), dtype=np.int32)
    return rp, cl


# --------------------------------------------------------------------------
# hashing (Sec. VI-C, reading A)
# --------------------------------------------------------------------------

def fmix32(h: int) -> int:
    return int(lib().pgo_fmix32(h & 0xFFFFFFFF))


def hash_seed(seed: int, i: int) -> int:
    return int(lib().pgo_hash_seed(seed & 0xFFFFFFFF, i))


def hash_i(seed: int, i: int, x: int) -> int:
    return int(lib().pgo_hash(seed & 0xFFFFFFFF, i, x))


def bit_position(h: int, l: int) -> int:
    return int(lib().pgo_bit_position(h & 0xFFFFFFFF, l))


def hash_array(seed: int, i: int, x) -> np.ndarray:
    x = np.ascontiguousarray(np.asarray(x), dtype=np.int32)
    out = np.empty(x.shape, dtype=np.uint32)
    lib().pgo_hash_array(seed & 0xFFFFFFFF, i, _p(x), x.size, _p(out))
    return out


# --------------------------------------------------------------------------
# sketches (Sec. II-D)
# --------------------------------------------------------------------------

def bloom_bits(row_ptr, col, l: int, b: int, seed: int) -> np.ndarray:
    """B_{N_v} for every v: uint8 [n, l], one byte per bit."""
    rp, cl = _csr(row_ptr, col)
    n = rp.size - 1
    out = np.empty((n, l), dtype=np.uint8)
    lib().pgo_bloom_build(n, _p(rp), _p(cl), l, b, seed & 0xFFFFFFFF, _p(out))
    return out


def bloom_of_set(X, l: int, b: int, seed: int) -> np.ndarray:
    X = np.ascontiguousarray(np.asarray(X), dtype=np.int32)
    out = np.empty(l, dtype=np.uint8)
    lib().pgo_bloom_of_set(_p(X), X.size, l, b, seed & 0xFFFFFFFF, _p(out))
    return out


def bloom_pack(bits: np.ndarray, words_per_row: int) -> np.ndarray:
    bits = np.ascontiguousarray(bits, dtype=np.uint8)
    n, l = bits.shape
    out = np.empty((n, words_per_row), dtype=np.uint64)
    lib().pgo_bloom_pack(n, l, _p(bits), _p(out), words_per_row)
    return out


def and_ones(BX: np.ndarray, BY: np.ndarray) -> int:
    BX = np.ascontiguousarray(BX, dtype=np.uint8)
    BY = np.ascontiguousarray(BY, dtype=np.uint8)
    return int(lib().pgo_bloom_and_ones(_p(BX), _p(BY), BX.size))


def ones(BX: np.ndarray) -> int:
    BX = np.ascontiguousarray(BX, dtype=np.uint8)
    return int(lib().pgo_bloom_ones(_p(BX), BX.size))


def khash(row_ptr, col, k: int, seed: int) -> np.ndarray:
    """M_{N_v} for every v: int32 [n, k] minimising elements (-1: empty)."""
    rp, cl = _csr(row_ptr, col)
    n = rp.size - 1
    out = np.empty((n, k), dtype=np.int32)
    lib().pgo_khash_build(n, _p(rp), _p(cl), k, seed & 0xFFFFFFFF, _p(out))
    return out


def onehash(row_ptr, col, k: int, seed: int) -> np.ndarray:
    """M1_{N_v} for every v: int32 [n, k] elements in increasing h_0 (-1 pad)."""
    rp, cl = _csr(row_ptr, col)
    n = rp.size - 1
    out = np.empty((n, k), dtype=np.int32)
    lib().pgo_onehash_build(n, _p(rp), _p(cl), k, seed & 0xFFFFFFFF, _p(out))
    return out


def khash_values(M: np.ndarray, seed: int) -> np.ndarray:
    """The hash values h_i(x_{i,min}) of a k-Hash sketch (0xFFFFFFFF where empty)."""
    n, k = M.shape
    out = np.full((n, k), 0xFFFFFFFF, dtype=np.uint32)
    for i in range(k):
        col = np.ascontiguousarray(M[:, i])
        h = hash_array(seed, i, col)
        out[:, i] = np.where(col >= 0, h, np.uint32(0xFFFFFFFF))
    return out


def onehash_values(M1: np.ndarray, seed: int) -> np.ndarray:
    """The hash values h_0(x) of a 1-Hash sketch (0xFFFFFFFF where empty)."""
    h = hash_array(seed, 0, M1)
    return np.where(M1 >= 0, h, np.uint32(0xFFFFFFFF)).astype(np.uint32)


# --------------------------------------------------------------------------
# edges and per-pair integer counts
# --------------------------------------------------------------------------

def upper_edges(row_ptr, col):
    """Each undirected edge once as (u, v), u < v, in CSR order."""
    rp, cl = _csr(row_ptr, col)
    n = rp.size - 1
    m = int(lib().pgo_upper_edges(n, _p(rp), _p(cl), None, None))
    eu = np.empty(m, dtype=np.int32)
    ev = np.empty(m, dtype=np.int32)
    lib().pgo_upper_edges(n, _p(rp), _p(cl), _p(eu), _p(ev))
    return eu, ev


def exact_pairs(row_ptr, col, pu, pv) -> np.ndarray:
    rp, cl = _csr(row_ptr, col)
    pu = np.ascontiguousarray(pu, dtype=np.int32)
    pv = np.ascontiguousarray(pv, dtype=np.int32)
    out = np.empty(pu.size, dtype=np.int64)
    lib().pgo_exact_pairs(_p(rp), _p(cl), _p(pu), _p(pv), pu.size, _p(out))
    return out


def bloom_pairs(bits: np.ndarray, pu, pv) -> np.ndarray:
    bits = np.ascontiguousarray(bits, dtype=np.uint8)
    pu = np.ascontiguousarray(pu, dtype=np.int32)
    pv = np.ascontiguousarray(pv, dtype=np.int32)
    out = np.empty(pu.size, dtype=np.int32)
    lib().pgo_bloom_pairs(_p(bits), bits.shape[1], _p(pu), _p(pv), pu.size, _p(out))
    return out


def bloom_or_pairs(bits: np.ndarray, pu, pv) -> np.ndarray:
    """B_{X∪Y,1} = popcount(BF_u OR BF_v) per pair."""
    bits = np.ascontiguousarray(bits, dtype=np.uint8)
    pu = np.ascontiguousarray(pu, dtype=np.int32)
    pv = np.ascontiguousarray(pv, dtype=np.int32)
    out = np.empty(pu.size, dtype=np.int32)
    lib().pgo_bloom_or_pairs(_p(bits), bits.shape[1], _p(pu), _p(pv), pu.size, _p(out))
    return out


def khash_pairs(M: np.ndarray, pu, pv) -> np.ndarray:
    M = np.ascontiguousarray(M, dtype=np.int32)
    pu = np.ascontiguousarray(pu, dtype=np.int32)
    pv = np.ascontiguousarray(pv, dtype=np.int32)
    out = np.empty(pu.size, dtype=np.int32)
    lib().pgo_khash_pairs(_p(M), M.shape[1], _p(pu), _p(pv), pu.size, _p(out))
    return out


def onehash_pairs(M1: np.ndarray, seed: int, row_ptr, pu, pv):
    """(c_lit, c_union, K) per pair (reading C)."""
    M1 = np.ascontiguousarray(M1, dtype=np.int32)
    rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
    pu = np.ascontiguousarray(pu, dtype=np.int32)
    pv = np.ascontiguousarray(pv, dtype=np.int32)
    P = pu.size
    cl, cu, K = (np.empty(P, dtype=np.int32) for _ in range(3))
    lib().pgo_onehash_pairs(_p(M1), M1.shape[1], seed & 0xFFFFFFFF, _p(rp), _p(pu), _p(pv), P,
                            _p(cl), _p(cu), _p(K))
    return cl, cu, K


# --------------------------------------------------------------------------
# estimators
# --------------------------------------------------------------------------

def est_and(ones_, l: int, b: int):
    """Eq. (bf_int) with the bounded count B~1 = B1 - [B1 = l] (appendix)."""
    o = np.asarray(ones_, dtype=np.float64)
    o = np.where(o == l, o - 1.0, o)
    return -(l / b) * np.log(1.0 - o / l)


def est_or(union_ones, size_x, size_y, l: int, b: int):
    """Eq. bf_int_union: |X| + |Y| + (l/b) log(1 - B~_{X∪Y,1}/l), the single-set
    estimator of |X ∪ Y| subtracted from the exact |X| + |Y|; the count is
    bounded as for AND, B~ = B - [B = l] (reading E)."""
    o = np.asarray(union_ones, dtype=np.float64)
    o = np.where(o == l, o - 1.0, o)
    s = np.asarray(size_x, dtype=np.float64) + np.asarray(size_y, dtype=np.float64)
    return s + (l / b) * np.log(1.0 - o / l)


def est_single_set(ones_, l: int, b: int):
    """The single-set estimator the paper analyses beside its own (Sec. VIII),
    applied to the AND filter (reading R): |X|^ = log(1 - B~_{X,1}/l) /
    (b log(1 - 1/l)). The printed form carries a leading minus that would make
    it negative for every non-empty filter (both logarithms are negative); the
    expected fill l (1 - (1 - 1/l)^{b t}) must map back to t, which fixes the
    sign. The count is bounded as for AND."""
    o = np.asarray(ones_, dtype=np.float64)
    o = np.where(o == l, o - 1.0, o)
    return np.log(1.0 - o / l) / (b * np.log(1.0 - 1.0 / l))


def est_limit(ones_, b: int):
    """Eq. (limit_xs): B1 / b."""
    return np.asarray(ones_, dtype=np.float64) / b


def est_minhash(c, K, size_x, size_y):
    """Eq. (est_int_mh): J/(1+J) * (|X| + |Y|), J = c / K; 0 when K = 0."""
    c = np.asarray(c, dtype=np.float64)
    K = np.asarray(K, dtype=np.float64)
    s = np.asarray(size_x, dtype=np.float64) + np.asarray(size_y, dtype=np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        J = np.where(K > 0, c / np.where(K > 0, K, 1.0), 0.0)
    return J / (1.0 + J) * s


def kmv_union(hx, hy, k: int) -> np.ndarray:
    """Sec. IX: the KMV sketch of X ∪ Y, the k smallest distinct values of
    the two sketches' hash values (hx, hy: ascending uint32 hashes)."""
    merged = np.union1d(np.asarray(hx, dtype=np.uint64), np.asarray(hy, dtype=np.uint64))
    return merged[:k]


def est_kmv(hx, hy, size_x: int, size_y: int, k: int) -> float:
    """Sec. IX: |X ∩ Y|^ = |X| + |Y| - |X ∪ Y|^, with |X ∪ Y|^ = (k - 1) /
    max K_{X∪Y} and the 32-bit hashes mapped into (0, 1] by h -> (h + 1) /
    2^32. hx, hy: the sketches' hash values (the k smallest hashes of each
    set, all of them for a set of at most k elements: a 1-Hash row). Reading
    T: a union sketch of fewer than k values holds the whole union, whose
    size is then its length (the estimator needs k values)."""
    u = kmv_union(hx, hy, k)
    if u.size < k:
        union = float(u.size)
    else:
        union = (k - 1) / ((float(u[-1]) + 1.0) / 4294967296.0)
    return float(size_x) + float(size_y) - union


# --------------------------------------------------------------------------
# whole-graph analysis
# --------------------------------------------------------------------------

def degrees(row_ptr) -> np.ndarray:
    rp = np.asarray(row_ptr, dtype=np.int64)
    return rp[1:] - rp[:-1]


def sketch(row_ptr, col, kind: str, *, l=256, b=2, k=16, seed=1):
    """Build one sketch of every neighbourhood. kind in {'bloom','khash','onehash'}."""
    if kind == "bloom":
        return bloom_bits(row_ptr, col, l, b, seed)
    if kind == "khash":
        return khash(row_ptr, col, k, seed)
    if kind == "onehash":
        return onehash(row_ptr, col, k, seed)
    raise ValueError(kind)


def pair_counts(row_ptr, col, est: int, sk, pu, pv, *, seed=1):
    """Integer counts for pairs: dict with 'count' (B1 / c / c_union) and,
    for 1-Hash, 'K' and 'c_lit'; for exact, |N_u ∩ N_v|."""
    if est == EST_EXACT:
        return {"count": exact_pairs(row_ptr, col, pu, pv)}
    if est in (EST_BF_AND, EST_BF_L, EST_BF_SS):
        return {"count": bloom_pairs(sk, pu, pv)}
    if est == EST_BF_OR:
        return {"count": bloom_pairs(sk, pu, pv), "union": bloom_or_pairs(sk, pu, pv)}
    if est == EST_KH:
        return {"count": khash_pairs(sk, pu, pv)}
    if est in (EST_1H, EST_1H_LITERAL):
        cl, cu, K = onehash_pairs(sk, seed, row_ptr, pu, pv)
        return {"count": cu, "K": K, "c_lit": cl}
    if est == EST_1H_KMV:
        cl, cu, K = onehash_pairs(sk, seed, row_ptr, pu, pv)
        H = onehash_values(sk, seed)
        d = degrees(row_ptr)
        k = sk.shape[1]
        kmv = np.array([est_kmv(H[u][H[u] != 0xFFFFFFFF], H[v][H[v] != 0xFFFFFFFF], d[u], d[v], k)
                        for u, v in zip(np.asarray(pu), np.asarray(pv))], dtype=np.float64)
        return {"count": cu, "K": K, "c_lit": cl, "kmv": kmv}
    raise ValueError(est)


def pair_estimates(row_ptr, est: int, counts: dict, pu, pv, *, l=256, b=2, k=16):
    """|N_u ∩ N_v|^ per pair in double."""
    d = degrees(row_ptr)
    c = counts["count"]
    if est == EST_EXACT:
        return np.asarray(c, dtype=np.float64)
    if est == EST_BF_AND:
        return est_and(c, l, b)
    if est == EST_BF_L:
        return est_limit(c, b)
    if est == EST_BF_OR:
        return est_or(counts["union"], d[pu], d[pv], l, b)
    if est == EST_BF_SS:
        return est_single_set(c, l, b)
    if est == EST_KH:
        return est_minhash(c, np.full(len(c), k), d[pu], d[pv])
    if est == EST_1H:
        return est_minhash(c, counts["K"], d[pu], d[pv])
    if est == EST_1H_LITERAL:
        # the formula as printed: J = |M1_X ∩ M1_Y| / k
        return est_minhash(counts["c_lit"], np.full(len(c), k), d[pu], d[pv])
    if est == EST_1H_KMV:
        return counts["kmv"]
    raise ValueError(est)


def similarities(row_ptr, estimate, pu, pv):
    """Listing sim: with I = clamp(|N_u ∩ N_v|^, 0, min(d_u, d_v)) (reading F),
    Jaccard I / (d_u + d_v - I), overlap I / min(d_u, d_v) and total
    neighbours d_u + d_v - I; common neighbours = the estimate itself. A
    quotient with a zero denominator is 0."""
    d = degrees(row_ptr).astype(np.float64)
    du, dv = d[pu], d[pv]
    cn = np.asarray(estimate, dtype=np.float64)
    I = np.clip(cn, 0.0, np.minimum(du, dv))
    den = du + dv - I
    mn = np.minimum(du, dv)
    with np.errstate(divide="ignore", invalid="ignore"):
        J = np.where(den > 0, I / np.where(den > 0, den, 1.0), 0.0)
        ov = np.where(mn > 0, I / np.where(mn > 0, mn, 1.0), 0.0)
    return {"cn": cn, "jac": J, "overlap": ov, "total": du + dv - I}


def jaccard_and_cn(row_ptr, estimate, pu, pv):
    """Listing 3 / Listing 6: CN = |N_u ∩ N_v|^ and
    J = I / (|N_u| + |N_v| - I), with I = clamp(CN, 0, min(d_u, d_v)) for the
    Jaccard only (reading F); J = 0 when both degrees are 0."""
    d = degrees(row_ptr).astype(np.float64)
    du, dv = d[pu], d[pv]
    cn = np.asarray(estimate, dtype=np.float64)
    I = np.clip(cn, 0.0, np.minimum(du, dv))
    den = du + dv - I
    with np.errstate(divide="ignore", invalid="ignore"):
        J = np.where(den > 0, I / np.where(den > 0, den, 1.0), 0.0)
    return cn, J


def analyze(row_ptr, col, est: int, *, l=256, b=2, k=16, seed=1, sk=None):
    """Everything the hot path produces for one graph and one estimator.

    Returns a dict with the upper edge list (eu, ev), per-edge integer counts,
    per-edge double estimates, TC^ = (1/3) * sum over edges (Sec. VII),
    per-vertex S_v = sum_{u in N_v} est(u, v) and T_v = S_v / 2, the local
    clustering coefficient LCC_v = 2 T_v / (d_v (d_v - 1)) (0 if d_v < 2),
    per-edge CN and Jaccard, and the integer histograms of the counts."""
    rp, cl = _csr(row_ptr, col)
    n = rp.size - 1
    kind = {EST_BF_AND: "bloom", EST_BF_L: "bloom", EST_BF_OR: "bloom", EST_BF_SS: "bloom", EST_KH: "khash",
            EST_1H: "onehash", EST_1H_LITERAL: "onehash",
            EST_1H_KMV: "onehash"}.get(est)
    if sk is None and kind is not None:
        sk = sketch(rp, cl, kind, l=l, b=b, k=k, seed=seed)
    eu, ev = upper_edges(rp, cl)
    counts = pair_counts(rp, cl, est, sk, eu, ev, seed=seed)
    e = pair_estimates(rp, est, counts, eu, ev, l=l, b=b, k=k)
    d = degrees(rp)
    S = np.zeros(n, dtype=np.float64)
    np.add.at(S, eu, e)
    np.add.at(S, ev, e)
    T = S / 2.0
    dd = d.astype(np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        lcc = np.where(d >= 2, 2.0 * T / np.where(d >= 2, dd * (dd - 1.0), 1.0), 0.0)
    cn, J = jaccard_and_cn(rp, e, eu, ev)
    out = {
        "eu": eu, "ev": ev, "m": int(eu.size), "counts": counts, "est": e,
        "tc": float(e.sum()) / 3.0, "S": S, "T": T, "lcc": lcc, "cn": cn, "jac": J,
        "sketch": sk,
    }
    sim = similarities(rp, e, eu, ev)
    out["overlap"], out["total"] = sim["overlap"], sim["total"]
    c = np.asarray(counts["count"], dtype=np.int64)
    if est in (EST_BF_AND, EST_BF_L, EST_BF_SS):
        out["hist"] = np.bincount(c, minlength=l + 1).astype(np.uint64)
    elif est == EST_BF_OR:
        U = np.asarray(counts["union"], dtype=np.int64)
        out["hist"] = np.concatenate([np.bincount(U, minlength=l + 1),
                                      [int((d[eu] + d[ev]).sum())]]).astype(np.uint64)
    elif est == EST_KH:
        out["hist"] = np.bincount(c, minlength=k + 1).astype(np.uint64)
        hd = np.zeros(k + 1, dtype=np.int64)
        np.add.at(hd, c, d[eu] + d[ev])
        out["hist_deg"] = hd.astype(np.uint64)
    elif est == EST_EXACT:
        out["tc_exact"] = int(c.sum()) // 3
    return out


# --------------------------------------------------------------------------
# Jarvis-Patrick clustering (Sec. III, Listing "Jarvis-Patrick clustering")
# --------------------------------------------------------------------------

def components(n: int, eu, ev, keep) -> np.ndarray:
    """Label of every vertex = the smallest vertex id of its connected
    component in (V, {e : keep[e]})."""
    eu = np.ascontiguousarray(eu, dtype=np.int32)
    ev = np.ascontiguousarray(ev, dtype=np.int32)
    keep = np.ascontiguousarray(keep, dtype=np.uint8)
    label = np.empty(n, dtype=np.int32)
    lib().pgo_components(n, eu.size, _p(eu), _p(ev), _p(keep), _p(label))
    return label


def jp_keep(row_ptr, est: int, counts: dict, pu, pv, tau: float, *, l=256, b=2, k=16) -> np.ndarray:
    """The Listing's test |N_u ∩ N_v|^ > tau per edge, evaluated on the double
    estimate of each estimator (reading P)."""
    e = pair_estimates(row_ptr, est, counts, pu, pv, l=l, b=b, k=k)
    return e > tau


def jarvis_patrick(row_ptr, col, est: int, tau: float, *, l=256, b=2, k=16, seed=1, sk=None):
    """Clusters = connected components of the graph restricted to the edges
    whose (estimated) common-neighbour count exceeds tau. Returns a dict
    with labels (smallest vertex id per cluster), the number of clusters
    (singletons included), the kept-edge mask and the upper edges."""
    rp, cl = _csr(row_ptr, col)
    n = rp.size - 1
    kind = {EST_BF_AND: "bloom", EST_BF_L: "bloom", EST_BF_OR: "bloom", EST_BF_SS: "bloom", EST_KH: "khash",
            EST_1H: "onehash", EST_1H_LITERAL: "onehash"}.get(est)
    if sk is None and kind is not None:
        sk = sketch(rp, cl, kind, l=l, b=b, k=k, seed=seed)
    eu, ev = upper_edges(rp, cl)
    counts = pair_counts(rp, cl, est, sk, eu, ev, seed=seed)
    keep = jp_keep(rp, est, counts, eu, ev, tau, l=l, b=b, k=k)
    label = components(n, eu, ev, keep)
    return {"labels": label, "clusters": int(np.count_nonzero(label == np.arange(n))),
            "kept": int(np.count_nonzero(keep)), "keep": keep, "eu": eu, "ev": ev, "counts": counts}


# --------------------------------------------------------------------------
# 4-clique counting (Sec. III-A, Listing "Reformulated 4-Clique Counting")
# --------------------------------------------------------------------------

def orient(row_ptr, col):
    """N+_v = neighbours after v in the degree order (d, id), as a CSR."""
    rp, cl = _csr(row_ptr, col)
    n = rp.size - 1
    plus_off = np.empty(n + 1, dtype=np.int32)
    plus_col = np.empty(max(cl.size // 2, 1), dtype=np.int32)
    lib().pgo_orient(n, _p(rp), _p(cl), _p(plus_off), _p(plus_col))
    return plus_off, plus_col[: int(plus_off[-1])]


def clique4(row_ptr, col, est: int, *, l=256, b=2, seed=1):
    """Number of 4-cliques: exact (est = EST_EXACT) or with the innermost
    |N+_w ∩ C3| estimated from popcount(BF+_u AND BF+_v AND BF+_w), the
    filters built over the oriented neighbourhoods N+ (reading S), evaluated
    with the AND or L estimator. Returns a dict with the count (int for
    exact, double otherwise), the number of 3-cliques visited and, with a
    sketch, the histogram of the triple-AND counts."""
    rp, cl = _csr(row_ptr, col)
    n = rp.size - 1
    po, pc = orient(rp, cl)
    pc_ = np.ascontiguousarray(pc if pc.size else np.zeros(1, np.int32))
    tri = ctypes.c_uint64()
    if est == EST_EXACT:
        ck = int(lib().pgo_clique4_exact(n, _p(po), _p(pc_), ctypes.byref(tri)))
        return {"count": ck, "triangles": int(tri.value)}
    bits = bloom_bits(po, pc, l, b, seed)
    hist = np.zeros(l + 1, dtype=np.uint64)
    t = int(lib().pgo_clique4_bloom(n, _p(po), _p(pc_), _p(np.ascontiguousarray(bits)), l, _p(hist)))
    j = np.arange(l + 1)
    f = est_and(j, l, b) if est == EST_BF_AND else est_limit(j, b)
    return {"count": float((hist.astype(np.float64) * f).sum()), "triangles": t, "hist": hist}

"""Pins for the CPU oracle: each test checks the oracle against something
other than itself — published hash values, closed forms, brute force,
special cases the paper states, or the distributions the paper gives for
the MinHash counts. A plausible slip in the oracle (a dropped term, a wrong
sign, a wrong index, a swapped operand) fails at least one of them."""
import itertools
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2208_11469_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _csr_np(rp, cl):
    return rp.numpy().astype(np.int32), cl.numpy().astype(np.int32)


# ---------------------------------------------------------------- hashing --

def test_fmix32_matches_published_murmur3_vectors():
    """Sec. VI-C uses MurmurHash3; its zero-length-key test vectors equal
    fmix32(seed)."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "murmur3_fmix32.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for seed, want in rows:
        assert O.fmix32(int(seed, 16)) == int(want, 16)


def test_hash_functions_are_injective_and_distinct():
    """Reading A: every h_i is a bijection on 32-bit ids, so equal hash
    values mean equal elements (no ties in any MinHash)."""
    x = np.arange(0, 1 << 20, dtype=np.int32)
    for i in range(3):
        h = O.hash_array(7, i, x)
        assert np.unique(h).size == x.size
    h0, h1 = O.hash_array(7, 0, x[:1000]), O.hash_array(7, 1, x[:1000])
    assert np.mean(h0 == h1) < 0.01


def test_bit_position_range_and_power_of_two_top_bits():
    rng = np.random.default_rng(0)
    for h in rng.integers(0, 2**32, 2000, dtype=np.uint64):
        h = int(h)
        assert O.bit_position(h, 256) == h >> 24          # top 8 bits for l = 256
        assert 0 <= O.bit_position(h, 448) < 448
        assert O.bit_position(h, 448) == (h * 448) >> 32
    assert O.bit_position(0xFFFFFFFF, 192) == 191
    assert O.bit_position(0, 192) == 0


# ---------------------------------------------------------- Bloom filter --

def test_bloom_invariants():
    rng = np.random.default_rng(1)
    l, b, seed = 256, 2, 11
    for _ in range(50):
        X = rng.choice(10**6, size=rng.integers(0, 80), replace=False).astype(np.int32)
        Y = rng.choice(10**6, size=rng.integers(0, 80), replace=False).astype(np.int32)
        BX, BY = O.bloom_of_set(X, l, b, seed), O.bloom_of_set(Y, l, b, seed)
        # ones never exceed min(l, b|X|)
        assert O.ones(BX) <= min(l, b * X.size)
        # BF of a union = OR of the BFs; BF of a set = OR of singleton BFs
        BU = O.bloom_of_set(np.concatenate([X, Y]), l, b, seed)
        assert np.array_equal(BU, BX | BY)
        acc = np.zeros(l, np.uint8)
        for x in X:
            acc |= O.bloom_of_set(np.array([x], np.int32), l, b, seed)
        assert np.array_equal(acc, BX)
        # popcount(A & B) <= min(popcount A, popcount B); identical sets
        a = O.and_ones(BX, BY)
        assert a <= min(O.ones(BX), O.ones(BY))
        assert O.and_ones(BX, BX) == O.ones(BX)
        # the intersection's filter lies under the AND of the filters
        I = np.intersect1d(X, Y)
        BI = O.bloom_of_set(I, l, b, seed)
        assert np.all(BI <= (BX & BY))


def test_bloom_collision_free_case_is_exact():
    """When the b*|X ∪ Y| hash positions are all distinct (checked by
    listing them), each element owns b personal bits (appendix, proof of
    consistency): popcount(B_X AND B_Y) = b|X ∩ Y| and the limit estimator
    B1/b of Eq. (limit_xs) returns |X ∩ Y| exactly."""
    rng = np.random.default_rng(2)
    l, seed = 1 << 20, 5
    for b in (1, 2, 4):
        checked = 0
        while checked < 20:
            common = rng.choice(10**7, size=rng.integers(0, 30), replace=False)
            only_x = rng.choice(np.arange(10**7, 2 * 10**7), size=rng.integers(0, 30), replace=False)
            only_y = rng.choice(np.arange(2 * 10**7, 3 * 10**7), size=rng.integers(0, 30), replace=False)
            X = np.concatenate([common, only_x]).astype(np.int32)
            Y = np.concatenate([common, only_y]).astype(np.int32)
            U = np.concatenate([common, only_x, only_y]).astype(np.int32)
            pos = [O.bit_position(O.hash_i(seed, i, int(x)), l) for x in U for i in range(b)]
            if len(set(pos)) != len(pos):
                continue
            checked += 1
            a = O.and_ones(O.bloom_of_set(X, l, b, seed), O.bloom_of_set(Y, l, b, seed))
            assert a == b * common.size
            assert O.est_limit(a, b) == common.size


def test_and_estimator_closed_forms():
    """Eq. (est_ss_bf)/(bf_int): feeding the expected fill
    B1 = l (1 - exp(-b t / l)) returns t exactly; B1 = 0 gives 0; the estimate
    grows with B1; saturation B1 = l uses B1 - 1 (appendix); and the
    l -> infinity limit is B1 / b (Eq. limit_xs)."""
    for l, b, t in [(256, 2, 10.0), (448, 2, 37.5), (1024, 4, 100.0), (192, 1, 3.0)]:
        B1 = l * (1.0 - math.exp(-b * t / l))
        assert O.est_and(B1, l, b) == pytest.approx(t, rel=1e-12)
    assert O.est_and(0, 256, 2) == 0.0
    v = O.est_and(np.arange(0, 257), 256, 2)
    assert np.all(np.diff(v[:256]) > 0)
    assert np.isfinite(v[256]) and v[256] == v[255]
    assert v[256] == pytest.approx(-(256 / 2) * math.log(1.0 / 256), rel=1e-14)
    for B1 in (1, 7, 40):
        assert O.est_and(B1, 10**9, 2) == pytest.approx(B1 / 2, rel=1e-6)


def test_and_estimator_mse_within_prop_4_1():
    """Prop. 4.1 bounds E[(|X∩Y|^_AND - |X∩Y|)^2] for the filter built from
    X ∩ Y when b = o(sqrt(l)) and b|X∩Y| <= 0.499 l log l; check the
    empirical MSE over 400 seeded hash families against the bound."""
    rng = np.random.default_rng(3)
    for l, b, t in [(256, 2, 40), (512, 1, 100), (1024, 2, 150)]:
        assert b * t <= 0.499 * l * math.log(l)
        errs = []
        for s in range(400):
            S = rng.choice(10**8, size=t, replace=False).astype(np.int32)
            errs.append(O.est_and(O.ones(O.bloom_of_set(S, l, b, 1000 + s)), l, b) - t)
        mse = float(np.mean(np.square(errs)))
        bound = math.exp(t * b / (l - 1)) * l / b**2 - l / b**2 - t / b
        assert mse <= 1.25 * bound, (l, b, t, mse, bound)
        assert mse >= 0.5 * bound  # the bound is tight to first order: catches a dropped factor


# ----------------------------------------------------------------- k-Hash --

def _sets_with_overlap(rng, nx, ny, ni):
    pool = rng.choice(10**8, size=nx + ny - ni, replace=False).astype(np.int32)
    X = pool[:nx]
    Y = np.concatenate([pool[:ni], pool[nx:nx + ny - ni]])
    return X, Y


def _two_row_csr(X, Y):
    X, Y = np.sort(X), np.sort(Y)
    rp = np.array([0, X.size, X.size + Y.size], np.int32)
    return rp, np.concatenate([X, Y]).astype(np.int32)


def test_khash_argmin_and_special_cases():
    rng = np.random.default_rng(4)
    X, Y = _sets_with_overlap(rng, 40, 30, 10)
    rp, cl = _two_row_csr(X, Y)
    k = 24
    M = O.khash(rp, cl, k, 9)
    for i in range(k):  # x_{i,min}: the element with the smallest h_i, by brute force
        hx = O.hash_array(9, i, np.sort(X))
        assert M[0, i] == np.sort(X)[np.argmin(hx)]
    # identical sets: every minimum matches; disjoint sets: none do
    rp2, cl2 = _two_row_csr(X, X)
    MM = O.khash(rp2, cl2, k, 9)
    assert O.khash_pairs(MM, [0], [1])[0] == k
    assert O.pair_estimates(rp2, O.EST_KH, {"count": np.array([k])}, np.array([0]), np.array([1]), k=k)[0] == X.size
    Z = (np.sort(X) + 10**8).astype(np.int32)
    rp3, cl3 = _two_row_csr(X, Z)
    assert O.khash_pairs(O.khash(rp3, cl3, k, 9), [0], [1])[0] == 0
    # an empty set contributes nothing
    rp4 = np.array([0, X.size, X.size], np.int32)
    M4 = O.khash(rp4, np.sort(X).astype(np.int32), k, 9)
    assert np.all(M4[1] == -1)
    assert O.khash_pairs(M4, [0], [1])[0] == 0


def test_khash_count_is_binomial_k_J():
    """Sec. IV-C: |M_X ∩ M_Y| ~ Bin(k, J). Over 300 seeds the mean of c/k
    lies within the Hoeffding radius of J, and the mean estimate matches the
    expectation formula Eq. (exp_int_mh) within 4 standard errors."""
    rng = np.random.default_rng(5)
    X, Y = _sets_with_overlap(rng, 60, 45, 20)
    J = 20 / 85
    rp, cl = _two_row_csr(X, Y)
    k, N = 16, 300
    cs = np.array([O.khash_pairs(O.khash(rp, cl, k, 77 + s), [0], [1])[0] for s in range(N)])
    radius = math.sqrt(math.log(2 / 1e-6) / (2 * N * k))
    assert abs(cs.mean() / k - J) < radius
    est = O.est_minhash(cs, np.full(N, k), 60, 45)
    expect = 105 * sum(math.comb(k, s) * J**s * (1 - J)**(k - s) * s / (k + s) for s in range(k + 1))
    assert abs(est.mean() - expect) < 4 * est.std() / math.sqrt(N)
    # variance of a binomial count: k J (1 - J)
    assert cs.var() == pytest.approx(k * J * (1 - J), rel=0.25)


# ----------------------------------------------------------------- 1-Hash --

def test_onehash_is_bottom_k_by_h0():
    rng = np.random.default_rng(6)
    X = rng.choice(10**7, size=100, replace=False).astype(np.int32)
    rp = np.array([0, 100], np.int32)
    k = 32
    M1 = O.onehash(rp, np.sort(X), k, 3)
    h = O.hash_array(3, 0, np.sort(X))
    want = np.sort(X)[np.argsort(h)][:k]
    assert np.array_equal(M1[0], want)
    # short sets: all elements, then -1 padding
    M1s = O.onehash(np.array([0, 5], np.int32), np.sort(X[:5]), k, 3)
    assert set(M1s[0, :5]) == set(X[:5]) and np.all(M1s[0, 5:] == -1)


def test_onehash_exact_when_union_fits_in_k():
    """Reading C: if |X ∪ Y| <= k both sketches hold the whole sets, so
    J^ = J and the estimate equals |X ∩ Y| exactly."""
    rng = np.random.default_rng(7)
    k = 32
    for _ in range(30):
        ni = int(rng.integers(0, 10))
        nx, ny = ni + int(rng.integers(0, 12)), ni + int(rng.integers(0, 12))
        X, Y = _sets_with_overlap(rng, nx, ny, ni)
        rp, cl = _two_row_csr(X, Y)
        M1 = O.onehash(rp, cl, k, 21)
        cnt = O.pair_counts(rp, cl, O.EST_1H, M1, np.array([0]), np.array([1]), seed=21)
        assert cnt["K"][0] == nx + ny - ni
        assert cnt["count"][0] == ni and cnt["c_lit"][0] == ni
        e = O.pair_estimates(rp, O.EST_1H, cnt, np.array([0]), np.array([1]), k=k)[0]
        assert e == pytest.approx(ni, abs=1e-12)


def test_onehash_count_is_hypergeometric():
    """Sec. IV-D: the count follows Hypergeometric(|X ∪ Y|, |X ∩ Y|, k).
    With |X ∪ Y| > k the union-restricted count has mean k |X∩Y| / |X∪Y|;
    the mean estimate matches Eq. (exp_int_mh) within 4 standard errors."""
    rng = np.random.default_rng(8)
    k, N = 32, 300
    X, Y = _sets_with_overlap(rng, 80, 70, 30)
    U, I = 120, 30
    rp, cl = _two_row_csr(X, Y)
    cs, Ks, lits = [], [], []
    for s in range(N):
        M1 = O.onehash(rp, cl, k, 500 + s)
        cnt = O.pair_counts(rp, cl, O.EST_1H, M1, np.array([0]), np.array([1]), seed=500 + s)
        cs.append(cnt["count"][0]); Ks.append(cnt["K"][0]); lits.append(cnt["c_lit"][0])
    cs, Ks, lits = np.array(cs), np.array(Ks), np.array(lits)
    assert np.all(Ks == k)
    assert np.all(lits >= cs)
    mean_h = k * I / U
    var_h = k * (I / U) * (1 - I / U) * (U - k) / (U - 1)
    assert abs(cs.mean() - mean_h) < 4 * math.sqrt(var_h / N)
    assert cs.var() == pytest.approx(var_h, rel=0.3)
    est = O.est_minhash(cs, Ks, 80, 70)
    expect = 150 * sum(math.comb(I, s) * math.comb(U - I, k - s) / math.comb(U, k) * s / (k + s)
                       for s in range(k + 1))
    assert abs(est.mean() - expect) < 4 * est.std() / math.sqrt(N)


def test_minhash_jaccard_identity():
    """Listing 6 Jaccard applied to a MinHash estimate recovers c / K exactly
    (I / (|X|+|Y|-I) with I = J/(1+J)(|X|+|Y|) is J)."""
    rp = np.array([0, 30, 70], np.int32)
    for c, K in [(0, 16), (3, 16), (16, 16), (5, 32), (31, 32)]:
        e = O.est_minhash(c, K, 30, 40)
        if e <= 30:
            cn, J = O.jaccard_and_cn(rp, np.array([e]), np.array([0]), np.array([1]))
            assert J[0] == pytest.approx(c / K, rel=1e-12)


# ------------------------------------------------------------------ exact --

def _brute_force(n, edges):
    A = np.zeros((n, n), bool)
    for u, v in edges:
        A[u, v] = A[v, u] = True
    tri = 0
    Tv = np.zeros(n, np.int64)
    for a, b, c in itertools.combinations(range(n), 3):
        if A[a, b] and A[b, c] and A[a, c]:
            tri += 1
            Tv[[a, b, c]] += 1
    return A, tri, Tv


def test_exact_matches_brute_force_on_small_graphs():
    rng = np.random.default_rng(9)
    for trial in range(12):
        n = int(rng.integers(2, 40))
        p = float(rng.uniform(0.05, 0.8))
        edges = [(u, v) for u in range(n) for v in range(u + 1, n) if rng.random() < p]
        rp, cl = _csr_np(*synth.from_edges(n, edges))
        A, tri, Tv = _brute_force(n, edges)
        r = O.analyze(rp, cl, O.EST_EXACT)
        assert r["tc_exact"] == tri
        assert r["tc"] == pytest.approx(tri, abs=1e-9)
        assert np.allclose(r["T"], Tv)
        d = A.sum(1)
        lcc = np.where(d >= 2, 2 * Tv / np.maximum(d * (d - 1), 1), 0.0)
        assert np.allclose(r["lcc"], lcc)
        for e in range(r["m"]):
            u, v = r["eu"][e], r["ev"][e]
            assert u < v and A[u, v]
            inter = int(np.sum(A[u] & A[v]))
            assert r["counts"]["count"][e] == inter
            assert r["jac"][e] == pytest.approx(inter / np.sum(A[u] | A[v]))
        assert r["m"] == len(edges)


def test_exact_closed_forms():
    for n in (3, 4, 7, 12):
        rp, cl = _csr_np(*synth.complete_graph(n))
        r = O.analyze(rp, cl, O.EST_EXACT)
        assert r["tc_exact"] == math.comb(n, 3)
        assert np.allclose(r["lcc"], 1.0)
        assert np.allclose(r["jac"], (n - 2) / n)
    star = [(0, i) for i in range(1, 9)]
    path = [(i, i + 1) for i in range(9)]
    for edges in (star, path):
        rp, cl = _csr_np(*synth.from_edges(10, edges))
        r = O.analyze(rp, cl, O.EST_EXACT)
        assert r["tc_exact"] == 0 and np.all(r["lcc"] == 0)


def test_exact_gnp_mean_triangles():
    """G(n, p) has C(n, 3) p^3 triangles in expectation: the mean over 32
    seeds lies within 4 standard errors."""
    n, deg = 600, 30.0
    p = deg / (n - 1)
    tcs = []
    for s in range(32):
        rp, cl = _csr_np(*synth.erdos_renyi(n, deg, seed=100 + s))
        tcs.append(O.analyze(rp, cl, O.EST_EXACT)["tc_exact"])
    tcs = np.array(tcs, dtype=np.float64)
    mu = math.comb(n, 3) * p**3
    assert abs(tcs.mean() - mu) < 4 * tcs.std(ddof=1) / math.sqrt(tcs.size)


# ------------------------------------------------------- whole-graph sums --

@pytest.mark.parametrize("est", [O.EST_BF_AND, O.EST_BF_L, O.EST_KH, O.EST_1H])
def test_histogram_and_sum_identities(est):
    rp, cl = _csr_np(*synth.erdos_renyi(512, 12, seed=3))
    r = O.analyze(rp, cl, est, l=256, b=2, k=16, seed=4)
    c = np.asarray(r["counts"]["count"], np.int64)
    if "hist" in r:
        assert int(r["hist"].sum()) == r["m"]
        assert int((np.arange(r["hist"].size) * r["hist"]).sum()) == int(c.sum())
    # TC = (1/3) sum_e est = (1/3) sum_v T_v
    assert r["tc"] == pytest.approx(r["T"].sum() / 3.0, rel=1e-12)
    d = O.degrees(rp)
    assert np.all(r["lcc"][d < 2] == 0)


def test_sketch_estimates_track_exact_on_dense_graph():
    """End-to-end sanity: with generous sketches the per-edge estimates are
    close to the exact counts on average (the accuracy claim of Sec. VIII-B,
    loosely)."""
    rp, cl = _csr_np(*synth.erdos_renyi(300, 60, seed=8))
    ex = O.analyze(rp, cl, O.EST_EXACT)
    for est, kw in [(O.EST_BF_AND, dict(l=4096, b=2)), (O.EST_KH, dict(k=256)), (O.EST_1H, dict(k=64))]:
        r = O.analyze(rp, cl, est, seed=2, **kw)
        assert abs(r["tc"] - ex["tc"]) / ex["tc"] < 0.35, est

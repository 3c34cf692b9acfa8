"""Pins of the oracle's KMV intersection estimator (Sec. IX) against what the
mathematics fixes, not against its own formula:
  * sets whose union has fewer than k elements: the union sketch holds the
    whole union, so the estimate is the exact intersection (brute force),
    also on the 1-Hash rows of a real graph;
  * symmetry in X and Y;
  * unbiasedness of the KMV size estimator, (k - 1) / U_(k) for n uniform
    hashes has mean n: averaged over many hash seeds the intersection
    estimate of sets with a known overlap lands on it within a few standard
    errors, for overlapping, identical and disjoint sets."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2208_11469_gb300 import synth


def _kmv_row(X, k, seed):
    h = np.sort(O.hash_array(seed, 0, np.asarray(X, dtype=np.int32)).astype(np.uint64))
    return h[:k]


def test_small_unions_are_exact():
    rng = np.random.default_rng(4)
    for trial in range(200):
        k = int(rng.integers(4, 40))
        nx = int(rng.integers(0, k))
        ny = int(rng.integers(0, k - nx))  # nx + ny < k: the union has fewer than k elements
        universe = rng.permutation(1000)
        X = universe[:nx]
        Y = universe[int(rng.integers(0, nx + 1)):][:ny]
        hx, hy = _kmv_row(X, k, trial), _kmv_row(Y, k, trial)
        assert O.est_kmv(hx, hy, nx, ny, k) == len(np.intersect1d(X, Y)), trial


def test_one_hash_rows_of_a_graph():
    """On the 1-Hash rows of a small graph, every edge whose two rows are
    complete and whose union has fewer than k values gets its exact common
    neighbour count."""
    rp, cl = synth.erdos_renyi(300, 5.0, seed=3)
    rp, cl = rp.numpy(), cl.numpy()
    k = 16
    M1 = O.onehash(rp, cl, k, 7)
    H = O.onehash_values(M1, 7)
    d = np.diff(rp)
    eu, ev = O.upper_edges(rp, cl)
    exact = O.exact_pairs(rp, cl, eu, ev)
    checked = 0
    for u, v, c in zip(eu, ev, exact):
        if d[u] + d[v] < k:
            hu = H[u][H[u] != 0xFFFFFFFF]
            hv = H[v][H[v] != 0xFFFFFFFF]
            assert O.est_kmv(hu, hv, d[u], d[v], k) == c
            checked += 1
    assert checked > 100


def test_symmetric():
    rng = np.random.default_rng(8)
    for trial in range(50):
        X = rng.choice(5000, 300, replace=False)
        Y = rng.choice(5000, 200, replace=False)
        hx, hy = _kmv_row(X, 32, trial), _kmv_row(Y, 32, trial)
        assert O.est_kmv(hx, hy, 300, 200, 32) == O.est_kmv(hy, hx, 200, 300, 32)


@pytest.mark.parametrize("k", [8, 64])
@pytest.mark.parametrize("nx,ny,common", [(2000, 1500, 500), (1200, 1200, 1200), (1000, 800, 0)])
def test_unbiased_over_hash_seeds(nx, ny, common, k):
    """At k = 8, using k instead of k - 1 in the size estimator would move the
    mean by |X ∪ Y| / 7, several standard errors."""
    X = np.arange(nx)
    Y = np.concatenate([np.arange(common), 100000 + np.arange(ny - common)])
    ests = [O.est_kmv(_kmv_row(X, k, s), _kmv_row(Y, k, s), nx, ny, k) for s in range(400)]
    union = nx + ny - common
    # Var[(k-1)/U_(k)] = n^2 / (k - 2) for the size estimator; the intersection inherits it
    se = union / np.sqrt(k - 2) / np.sqrt(len(ests))
    assert abs(np.mean(ests) - common) < 4.0 * se, (np.mean(ests), common, se)

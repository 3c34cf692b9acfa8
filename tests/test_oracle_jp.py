"""Pins of the oracle's Jarvis-Patrick clustering (Sec. III, Listing
"Jarvis-Patrick clustering"): clusters are the connected components of the
graph restricted to the edges whose |N_u ∩ N_v| exceeds tau.

The component labelling is checked against a library routine
(scipy.sparse.csgraph) and against breadth-first search written here; the
clustering against closed forms (disjoint cliques, paths, stars, the strict
inequality at tau = n - 2 in K_n)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2208_11469_gb300 import synth


def _np(t):
    return t.numpy() if hasattr(t, "numpy") else np.asarray(t)


def _canonical(labels):
    """Map any component labelling to 'smallest vertex id of the component'."""
    labels = np.asarray(labels)
    out = np.empty_like(labels)
    for c in np.unique(labels):
        members = np.flatnonzero(labels == c)
        out[members] = members.min()
    return out


def _bfs_labels(n, eu, ev, keep):
    adj = [[] for _ in range(n)]
    for a, b, k in zip(eu, ev, keep):
        if k:
            adj[a].append(b)
            adj[b].append(a)
    lab = [-1] * n
    for s in range(n):
        if lab[s] >= 0:
            continue
        stack = [s]
        lab[s] = s
        while stack:
            x = stack.pop()
            for y in adj[x]:
                if lab[y] < 0:
                    lab[y] = s
                    stack.append(y)
    return np.asarray(lab)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_components_match_scipy(seed):
    sp = pytest.importorskip("scipy.sparse")
    csg = pytest.importorskip("scipy.sparse.csgraph")
    rp, cl = synth.erdos_renyi(3000, 2.5, seed=seed)
    eu, ev = O.upper_edges(_np(rp), _np(cl))
    keep = np.random.default_rng(seed).random(eu.size) < 0.7
    got = O.components(3000, eu, ev, keep)
    A = sp.coo_matrix((np.ones(int(keep.sum())), (eu[keep], ev[keep])), shape=(3000, 3000))
    ncomp, lab = csg.connected_components(A, directed=False)
    np.testing.assert_array_equal(got, _canonical(lab))
    assert np.count_nonzero(got == np.arange(3000)) == ncomp


def test_components_match_bfs_on_small_graphs():
    rng = np.random.default_rng(0)
    for trial in range(30):
        n = int(rng.integers(1, 40))
        rp, cl = synth.erdos_renyi(n, float(rng.uniform(0.5, 4.0)), seed=trial)
        eu, ev = O.upper_edges(_np(rp), _np(cl))
        keep = rng.random(eu.size) < rng.uniform(0, 1)
        np.testing.assert_array_equal(O.components(n, eu, ev, keep), _bfs_labels(n, eu, ev, keep))


def _disjoint_cliques(sizes):
    edges, off = [], 0
    for s in sizes:
        edges += [(off + i, off + j) for i in range(s) for j in range(i + 1, s)]
        off += s
    return synth.from_edges(off, edges), off


def test_jp_disjoint_cliques_closed_form():
    """In K_s every edge has s - 2 common neighbours: with exact counts the
    clique survives iff s - 2 > tau, so the cluster count is the number of
    surviving cliques plus one singleton per vertex of the others."""
    sizes = [3, 4, 5, 7, 9]
    (rp, cl), n = _disjoint_cliques(sizes)
    for tau in (-1.0, 0.5, 1.0, 2.5, 3.0, 5.0, 6.9, 7.0, 100.0):
        r = O.jarvis_patrick(_np(rp), _np(cl), O.EST_EXACT, tau)
        want = sum(1 if s - 2 > tau else s for s in sizes)
        assert r["clusters"] == want, (tau, r["clusters"], want)
        assert r["kept"] == sum(s * (s - 1) // 2 for s in sizes if s - 2 > tau)


def test_jp_strict_threshold_and_trivial_cases():
    rp, cl = synth.complete_graph(8)
    assert O.jarvis_patrick(_np(rp), _np(cl), O.EST_EXACT, 6.0)["clusters"] == 8   # 6 > 6 is false
    assert O.jarvis_patrick(_np(rp), _np(cl), O.EST_EXACT, 5.999)["clusters"] == 1
    # a path has no triangles: any tau >= 0 leaves every vertex alone; tau < 0 keeps the path
    rp, cl = synth.from_edges(10, [(i, i + 1) for i in range(9)])
    assert O.jarvis_patrick(_np(rp), _np(cl), O.EST_EXACT, 0.0)["clusters"] == 10
    r = O.jarvis_patrick(_np(rp), _np(cl), O.EST_EXACT, -0.5)
    assert r["clusters"] == 1 and (r["labels"] == 0).all()
    # a star (centre 0): leaves share only the centre, which is not a common
    # neighbour of an edge (0, leaf); tau < 0 keeps the star in one cluster
    rp, cl = synth.from_edges(6, [(0, i) for i in range(1, 6)])
    assert O.jarvis_patrick(_np(rp), _np(cl), O.EST_EXACT, 0.0)["clusters"] == 6
    assert O.jarvis_patrick(_np(rp), _np(cl), O.EST_EXACT, -1.0)["clusters"] == 1
    # no vertices
    r = O.jarvis_patrick(np.zeros(1, np.int32), np.zeros(0, np.int32), O.EST_EXACT, 1.0)
    assert r["clusters"] == 0 and r["labels"].size == 0


def test_jp_sketch_decision_is_the_estimate_test():
    """With a sketch, an edge is kept iff its double estimate exceeds tau;
    the labels are the components of those edges, and every kept edge joins
    two vertices of one cluster while every cluster is connected by kept
    edges."""
    rp, cl = synth.rmat(10, 8, seed=4)
    rp, cl = _np(rp), _np(cl)
    for est, kw in ((O.EST_BF_AND, dict(l=256, b=2)), (O.EST_BF_L, dict(l=256, b=2)), (O.EST_KH, dict(k=16)),
                    (O.EST_1H, dict(k=16))):
        r = O.jarvis_patrick(rp, cl, est, 2.0, **kw)
        e = O.pair_estimates(rp, est, r["counts"], r["eu"], r["ev"], **kw)
        np.testing.assert_array_equal(r["keep"], e > 2.0)
        lab = r["labels"]
        assert (lab[r["eu"][r["keep"]]] == lab[r["ev"][r["keep"]]]).all()
        np.testing.assert_array_equal(lab, _bfs_labels(rp.size - 1, r["eu"], r["ev"], r["keep"]))

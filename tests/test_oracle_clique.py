"""Pins of the oracle's 4-clique counting (Sec. III-A, Listing
"Reformulated 4-Clique Counting"): closed forms (K_n, disjoint cliques, the
octahedron and wheels, which have triangles but no 4-cliques), brute force
over all 4-subsets of small graphs, the orientation's invariants, and the
Bloom version's collision-free limit, where the L estimate of every triple
intersection is exact."""
import itertools
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2208_11469_gb300 import synth


def _np(t):
    return t.numpy() if hasattr(t, "numpy") else np.asarray(t)


def _brute(n, edges):
    adj = set()
    for a, b in edges:
        adj.add((a, b))
        adj.add((b, a))
    k4 = sum(all((a, b) in adj for a, b in itertools.combinations(q, 2)) for q in itertools.combinations(range(n), 4))
    k3 = sum(all((a, b) in adj for a, b in itertools.combinations(q, 2)) for q in itertools.combinations(range(n), 3))
    return k4, k3


@pytest.mark.parametrize("n", range(4, 13))
def test_complete_graph(n):
    rp, cl = synth.complete_graph(n)
    r = O.clique4(_np(rp), _np(cl), O.EST_EXACT)
    assert r["count"] == math.comb(n, 4) and r["triangles"] == math.comb(n, 3)


def test_graphs_with_triangles_but_no_four_cliques():
    octa = [(a, b) for a in range(6) for b in range(a + 1, 6) if b != a + 3 or a >= 3]
    octa = [(a, b) for a, b in octa if not (b - a == 3)]
    rp, cl = synth.from_edges(6, octa)
    r = O.clique4(_np(rp), _np(cl), O.EST_EXACT)
    assert r["count"] == 0 and r["triangles"] == 8
    for k in (5, 6, 9):  # wheel: hub 0 and a k-cycle
        edges = [(0, i) for i in range(1, k + 1)] + [(i, i % k + 1) for i in range(1, k + 1)]
        rp, cl = synth.from_edges(k + 1, edges)
        r = O.clique4(_np(rp), _np(cl), O.EST_EXACT)
        assert r["count"] == 0 and r["triangles"] == k


def test_disjoint_cliques():
    sizes = [4, 5, 7, 3, 9]
    edges, off = [], 0
    for s in sizes:
        edges += [(off + i, off + j) for i in range(s) for j in range(i + 1, s)]
        off += s
    rp, cl = synth.from_edges(off, edges)
    r = O.clique4(_np(rp), _np(cl), O.EST_EXACT)
    assert r["count"] == sum(math.comb(s, 4) for s in sizes)
    assert r["triangles"] == sum(math.comb(s, 3) for s in sizes)


def test_brute_force_small_graphs():
    rng = np.random.default_rng(2)
    for trial in range(25):
        n = int(rng.integers(5, 22))
        rp, cl = synth.erdos_renyi(n, float(rng.uniform(2.0, 9.0)), seed=trial)
        rp, cl = _np(rp), _np(cl)
        eu, ev = O.upper_edges(rp, cl)
        k4, k3 = _brute(n, list(zip(eu.tolist(), ev.tolist())))
        r = O.clique4(rp, cl, O.EST_EXACT)
        assert (r["count"], r["triangles"]) == (k4, k3), trial


def test_orientation_invariants():
    rp, cl = synth.rmat(11, 8, seed=5)
    rp, cl = _np(rp), _np(cl)
    po, pc = O.orient(rp, cl)
    d = np.diff(rp)
    assert pc.size * 2 == cl.size                       # every edge once
    src = np.repeat(np.arange(rp.size - 1), np.diff(po))
    key = lambda x: d[x].astype(np.int64) * (1 << 32) + x
    assert (key(src) < key(pc)).all()                   # lower to higher in the degree order
    for v in range(0, rp.size - 1, 37):
        row = pc[po[v]:po[v + 1]]
        assert (np.diff(row) > 0).all()
    eu, ev = O.upper_edges(rp, cl)
    assert set(zip(np.minimum(src, pc).tolist(), np.maximum(src, pc).tolist())) == set(zip(eu.tolist(), ev.tolist()))


def test_bloom_collision_free_limit_and_histogram():
    """With filters far longer than b times the neighbourhoods, the triple
    AND of three oriented-neighbourhood filters has exactly
    b |N+_u ∩ N+_v ∩ N+_w| ones, so the L estimate of the count is exact;
    the histogram always counts every 3-clique once."""
    rp, cl = synth.erdos_renyi(40, 12.0, seed=9)
    rp, cl = _np(rp), _np(cl)
    exact = O.clique4(rp, cl, O.EST_EXACT)
    for b in (1, 3):
        r = O.clique4(rp, cl, O.EST_BF_L, l=1 << 20, b=b, seed=4)
        assert int(r["hist"].sum()) == exact["triangles"] == r["triangles"]
        assert r["count"] == pytest.approx(exact["count"], abs=1e-9)
        assert int((np.arange(r["hist"].size) * r["hist"]).sum()) == b * exact["count"]
    r = O.clique4(rp, cl, O.EST_BF_AND, l=256, b=2, seed=4)
    assert int(r["hist"].sum()) == exact["triangles"]

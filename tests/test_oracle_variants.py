"""Pins of the oracle's estimator variants: the Bloom OR estimator (Eq.
bf_int_union), the single-set Bloom estimator applied to the AND filter, and
the overlap / total-neighbour similarities of Listing sim. Each is checked
against closed forms, limits, the union identity of Bloom filters, a seeded
Monte-Carlo mean, and brute force over Python sets."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2208_11469_gb300 import synth


@pytest.mark.parametrize("l", [64, 256, 1000])
@pytest.mark.parametrize("b", [1, 2, 4])
def test_single_set_inverts_the_expected_fill(l, b):
    """E[B_{X,1}] = l (1 - (1 - 1/l)^{b t}) for t inserted elements; the
    estimator maps that fill back to t exactly (this also fixes its sign)."""
    t = np.arange(0, 60, dtype=np.float64)
    fill = l * (1.0 - (1.0 - 1.0 / l) ** (b * t))
    np.testing.assert_allclose(O.est_single_set(fill, l, b), t, rtol=1e-9, atol=1e-9)
    e = O.est_single_set(np.arange(l + 1), l, b)
    assert e[0] == 0.0 and (np.diff(e) >= 0).all() and e[-1] == e[-2]


@pytest.mark.parametrize("l,b", [(256, 2), (1024, 1), (512, 4)])
def test_or_estimator_inverts_the_union_fill(l, b):
    """With the union filter at its (Poisson) expected fill
    l (1 - exp(-b s / l)), s = |X ∪ Y|, the OR estimator returns
    |X| + |Y| - s = |X ∩ Y| exactly."""
    for x, y, i in ((10, 10, 3), (40, 7, 7), (100, 100, 0), (5, 90, 2)):
        s = x + y - i
        fill = l * (1.0 - math.exp(-b * s / l))
        assert O.est_or(fill, x, y, l, b) == pytest.approx(i, abs=1e-9)


def test_or_count_is_the_filter_of_the_union():
    rng = np.random.default_rng(3)
    for trial in range(20):
        X = rng.choice(5000, size=int(rng.integers(1, 80)), replace=False)
        Y = rng.choice(5000, size=int(rng.integers(1, 80)), replace=False)
        for l, b in ((192, 1), (448, 2), (1024, 3)):
            bx, by = O.bloom_of_set(X, l, b, trial), O.bloom_of_set(Y, l, b, trial)
            bu = O.bloom_of_set(np.union1d(X, Y), l, b, trial)
            assert O.lib().pgo_bloom_or_ones(O._p(bx), O._p(by), l) == O.ones(bu)
            assert O.ones(bu) <= min(l, b * np.union1d(X, Y).size)


def test_or_limit_of_long_filters():
    """B -> infinity: no collisions, B_{X∪Y,1} = b |X ∪ Y| and the estimate
    tends to |X ∩ Y| (as for AND, Eq. limit_xs)."""
    x, y, i = 30, 25, 11
    s = x + y - i
    for b in (1, 2, 4):
        for l in (10 ** 6, 10 ** 8):
            assert O.est_or(b * s, x, y, l, b) == pytest.approx(i, abs=2.0 * b * s * s / l + 1e-6)


def test_or_monte_carlo_mean():
    """Over 400 seeds the OR estimate averages to |X ∩ Y| within the
    sampling error (l large enough that the bias of the logarithm is small)."""
    rng = np.random.default_rng(11)
    base = rng.choice(10 ** 6, size=60, replace=False)
    X, Y = base[:40], base[25:]          # |X ∩ Y| = 15, |X ∪ Y| = 60
    l, b = 2048, 2
    vals = []
    for seed in range(400):
        bx, by = O.bloom_of_set(X, l, b, seed), O.bloom_of_set(Y, l, b, seed)
        U = O.lib().pgo_bloom_or_ones(O._p(bx), O._p(by), l)
        vals.append(O.est_or(U, X.size, Y.size, l, b))
    vals = np.asarray(vals)
    assert abs(vals.mean() - 15.0) < 4.0 * vals.std() / math.sqrt(vals.size) + 0.2


def test_similarities_brute_force():
    """Exact counts on small graphs: overlap = |N_u ∩ N_v| / min(d_u, d_v),
    total = |N_u ∪ N_v|, Jaccard = |∩| / |∪|, written with Python sets."""
    for seed in range(6):
        rp, cl = synth.erdos_renyi(60, 8.0, seed=seed)
        rp, cl = rp.numpy(), cl.numpy()
        N = [set(cl[rp[v]:rp[v + 1]].tolist()) for v in range(60)]
        pu = np.repeat(np.arange(60), 60).astype(np.int32)
        pv = np.tile(np.arange(60), 60).astype(np.int32)
        e = O.exact_pairs(rp, cl, pu, pv).astype(np.float64)
        s = O.similarities(rp, e, pu, pv)
        for k in range(pu.size):
            a, b = N[pu[k]], N[pv[k]]
            inter, union = len(a & b), len(a | b)
            assert s["overlap"][k] == pytest.approx(inter / min(len(a), len(b)) if min(len(a), len(b)) else 0.0)
            assert s["total"][k] == len(a) + len(b) - inter == union
            assert s["jac"][k] == pytest.approx(inter / union if union else 0.0)


def test_or_histogram_identity_gives_the_total():
    rp, cl = synth.rmat(10, 8, seed=4)
    rp, cl = rp.numpy(), cl.numpy()
    l, b = 448, 2
    r = O.analyze(rp, cl, O.EST_BF_OR, l=l, b=b)
    h = r["hist"].astype(np.float64)
    assert h[: l + 1].sum() == r["m"]
    d = O.degrees(rp)
    assert h[l + 1] == (d[r["eu"]] + d[r["ev"]]).sum()
    g = O.est_or(np.arange(l + 1), 0, 0, l, b)   # the logarithm term alone
    assert (h[l + 1] + (h[: l + 1] * g).sum()) / 3.0 == pytest.approx(r["tc"], rel=1e-12)

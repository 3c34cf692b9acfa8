"""GPU parity of Jarvis-Patrick clustering (pg_jarvis_patrick) against the
oracle: the kept-edge count, the cluster count and every vertex's label
(smallest vertex id of its cluster) are bit-exact, for the exact count and
every estimator, on uneven graphs, over thresholds from "keep everything"
to "keep nothing"; the labels do not depend on the run."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2208_11469_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pg():
    from paper_2208_11469_gb300 import build, pg as _pg
    build.build()
    _pg.lib()
    return _pg


def _hubs():
    n = 20000
    rp, cl = synth.erdos_renyi(n, 6.0, seed=8)
    src = torch.repeat_interleave(torch.arange(n), (rp[1:] - rp[:-1]).long())
    g = torch.Generator().manual_seed(8)
    hub = torch.randperm(n, generator=g)[:9000]
    u = torch.cat([src, torch.zeros(9000, dtype=torch.int64)])
    v = torch.cat([cl.long(), hub])
    return synth.csr_from_pairs(u, v, n)


GRAPHS = {
    "er4096": lambda: synth.erdos_renyi(4096, 16.0, seed=1),
    "rmat12": lambda: synth.rmat(12, 16, seed=7),
    "hubs": _hubs,
    "cliques": lambda: synth.from_edges(
        19, [(o + i, o + j) for o, s in ((0, 3), (3, 4), (7, 5), (12, 7)) for i in range(s) for j in range(i + 1, s)]),
}
_cache = {}


def _graph(name):
    if name not in _cache:
        rp, cl = GRAPHS[name]()
        _cache[name] = (rp.numpy().astype(np.int32), cl.numpy().astype(np.int32))
    return _cache[name]


def _sketch(pg, g, est, kw, seed):
    if est in (O.EST_BF_AND, O.EST_BF_L):
        return pg.build_bloom(g, kw["l"], kw["b"], seed=seed)
    if est == O.EST_KH:
        return pg.build_minhash(g, pg.SK_KHASH, kw["k"], seed=seed)
    if est in (O.EST_1H, O.EST_1H_LITERAL):
        return pg.build_minhash(g, pg.SK_1HASH, kw["k"], seed=seed)
    return None


def _safe_taus(est, kw, taus):
    """Drop thresholds within 1e-9 (relative) of an AND estimate value: there
    the two sides' logarithms could round differently (reading P)."""
    if est != O.EST_BF_AND:
        return taus
    vals = O.est_and(np.arange(kw["l"] + 1), kw["l"], kw["b"])
    return [t for t in taus if np.min(np.abs(vals - t)) > 1e-9 * max(1.0, abs(t))]


CASES = [
    ("cliques", O.EST_EXACT, {}),
    ("er4096", O.EST_EXACT, {}),
    ("er4096", O.EST_BF_AND, dict(l=256, b=2)),
    ("er4096", O.EST_BF_L, dict(l=256, b=2)),
    ("er4096", O.EST_KH, dict(k=16)),
    ("er4096", O.EST_1H, dict(k=32)),
    ("er4096", O.EST_1H_LITERAL, dict(k=32)),
    ("rmat12", O.EST_EXACT, {}),
    ("rmat12", O.EST_BF_AND, dict(l=448, b=2)),
    ("rmat12", O.EST_KH, dict(k=64)),
    ("rmat12", O.EST_1H, dict(k=16)),
    ("hubs", O.EST_EXACT, {}),
    ("hubs", O.EST_BF_AND, dict(l=192, b=1)),
    ("hubs", O.EST_KH, dict(k=32)),
]


@pytest.mark.parametrize("name,est,kw", CASES)
def test_jp_bit_exact(pg, name, est, kw):
    rp, cl = _graph(name)
    g = pg.graph(torch.from_numpy(rp).cuda(), torch.from_numpy(cl).cuda())
    sk = _sketch(pg, g, est, kw, seed=3)
    osk = None
    if sk is not None:
        kind = {O.EST_BF_AND: "bloom", O.EST_BF_L: "bloom", O.EST_KH: "khash"}.get(est, "onehash")
        osk = O.sketch(rp, cl, kind, l=kw.get("l", 256), b=kw.get("b", 2), k=kw.get("k", 16), seed=3)
    for tau in _safe_taus(est, kw, [-1.0, 0.0, 0.5, 1.0, 2.5, 4.0, 7.25, 1e9]):
        want = O.jarvis_patrick(rp, cl, est, tau, l=kw.get("l", 256), b=kw.get("b", 2), k=kw.get("k", 16),
                                seed=3, sk=osk)
        labels, res = pg.jarvis_patrick(g, sk, est, tau)
        assert res["edges"] == want["eu"].size
        assert res["kept"] == want["kept"], (tau, res, want["kept"])
        assert res["clusters"] == want["clusters"], (tau, res, want["clusters"])
        np.testing.assert_array_equal(labels.cpu().numpy(), want["labels"], err_msg=f"tau {tau}")


def test_jp_labels_repeat_and_optional_outputs(pg):
    rp, cl = _graph("rmat12")
    g = pg.graph(torch.from_numpy(rp).cuda(), torch.from_numpy(cl).cuda())
    sk = pg.build_bloom(g, 256, 2, seed=1)
    a, ra = pg.jarvis_patrick(g, sk, pg.EST_BF_AND, 3.0)
    b, rb = pg.jarvis_patrick(g, sk, pg.EST_BF_AND, 3.0)
    assert ra == rb
    assert torch.equal(a, b)
    none, rc = pg.jarvis_patrick(g, sk, pg.EST_BF_AND, 3.0, want_labels=False)
    assert none is None and rc == ra


def test_jp_degenerate(pg):
    for rp, cl in (synth.from_edges(5, []), synth.from_edges(2, [(0, 1)]), synth.complete_graph(6)):
        rpn, cln = rp.numpy().astype(np.int32), cl.numpy().astype(np.int32)
        g = pg.graph(rp.to(torch.int32).cuda(), cl.to(torch.int32).cuda())
        for tau in (-0.5, 3.5, 4.0):
            labels, res = pg.jarvis_patrick(g, None, pg.EST_EXACT, tau)
            want = O.jarvis_patrick(rpn, cln, O.EST_EXACT, tau)
            assert res["clusters"] == want["clusters"] and res["kept"] == want["kept"]
            np.testing.assert_array_equal(labels.cpu().numpy(), want["labels"])
    with pytest.raises(pg.PGError) as ei:
        g = pg.graph(*[t.to(torch.int32).cuda() for t in synth.complete_graph(4)])
        pg.jarvis_patrick(g, None, pg.EST_EXACT, float("nan"))
    assert ei.value.status == -1

"""pg_triangle_count_noalloc — the triangle count for callers that cannot
allocate device memory (a plugin inside a host application whose allocator
owns the device memory, or a process that forbids device allocation after
start-up). It keeps its scratch in a static array inside the library instead
of a caller workspace. This file is collected last on purpose: the entry
point shares that array across calls, and the check must hold both in a
fresh process and after every other test has used the library.

The results must equal those of pg_triangle_count, which takes a workspace,
on two calls in a row (the second call must not see the first call's
histogram)."""
import numpy as np
import pytest
import torch

from paper_2208_11469_gb300 import synth

pytestmark = pytest.mark.gpu

RTOL_F64 = 1e-9


@pytest.fixture(scope="module")
def pg():
    from paper_2208_11469_gb300 import build, pg as _pg
    build.build()
    _pg.lib()
    return _pg


@pytest.mark.parametrize("graph,kind,params,est", [
    ("er", "bloom", dict(bits=256, b=2), 1),
    ("er", "bloom", dict(bits=256, b=2), 2),
    ("rmat", "bloom", dict(bits=1024, b=4), 1),
    ("rmat", "khash", dict(k=64), 3),
    ("er", "khash", dict(k=256), 3),
    ("rmat", "onehash", dict(k=32), 4),
    ("rmat", "onehash", dict(k=32), 5),
    ("rmat", "onehash", dict(k=32), 8),   # KMV: the largest scratch (two extra histogram words)
    ("rmat", "bloom", dict(bits=1024, b=2), 6),  # OR: one extra histogram bin
    ("er", "bloom", dict(bits=448, b=2), 7),     # single-set estimator
])
def test_noalloc_matches_workspace_entry_point_twice(pg, graph, kind, params, est):
    rp, cl = synth.erdos_renyi(4096, 16.0, seed=1) if graph == "er" else synth.rmat(13, 16, seed=3)
    g = pg.graph(rp.cuda(), cl.cuda())
    if kind == "bloom":
        sk = pg.build_bloom(g, params["bits"], params["b"], seed=7)
    else:
        sk = pg.build_minhash(g, pg.SK_KHASH if kind == "khash" else pg.SK_1HASH, params["k"], seed=7)
    want = pg.triangle_count(g, sk, est)
    for _ in range(2):
        got = pg.triangle_count_noalloc(g, sk, est)
        assert got["edges"] == want["edges"] and got["count_sum"] == want["count_sum"]
        assert got["est_tc"] == pytest.approx(want["est_tc"], rel=RTOL_F64, abs=1e-12)
        assert got["est_tc_alt"] == pytest.approx(want["est_tc_alt"], rel=RTOL_F64, abs=1e-12)


def test_noalloc_alternating_sketches_do_not_leak_state(pg):
    """Two different graphs and sketch kinds back to back on one stream: each
    call starts from a cleared histogram."""
    a = pg.graph(*[t.cuda() for t in synth.erdos_renyi(2048, 12.0, seed=5)])
    b = pg.graph(*[t.cuda() for t in synth.rmat(12, 8, seed=6)])
    ska = pg.build_bloom(a, 192, 2, seed=1)
    skb = pg.build_minhash(b, pg.SK_1HASH, 16, seed=1)
    wa, wb = pg.triangle_count(a, ska, pg.EST_BF_AND), pg.triangle_count(b, skb, pg.EST_1H)
    for _ in range(2):
        ga = pg.triangle_count_noalloc(a, ska, pg.EST_BF_AND)
        gb = pg.triangle_count_noalloc(b, skb, pg.EST_1H)
        assert ga["count_sum"] == wa["count_sum"] and gb["count_sum"] == wb["count_sum"]
        assert ga["est_tc"] == pytest.approx(wa["est_tc"], rel=RTOL_F64)
        assert gb["est_tc"] == pytest.approx(wb["est_tc"], rel=RTOL_F64)


def test_noalloc_rejects_what_its_scratch_cannot_hold(pg):
    g = pg.graph(*[t.cuda() for t in synth.erdos_renyi(256, 6.0, seed=2)])
    sk = pg.build_bloom(g, 256, 2, seed=1)
    with pytest.raises(pg.PGError) as ei:
        pg.triangle_count_noalloc(g, sk, pg.EST_EXACT)
    assert ei.value.status == -9 and "exact" in str(ei.value)
    np.testing.assert_equal(pg.triangle_count_noalloc(g, sk, pg.EST_BF_AND)["edges"], g.m)

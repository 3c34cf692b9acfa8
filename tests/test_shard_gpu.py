"""The device side of the vertex-partitioned run (Sec. VIII-F) on one GPU:
the ranks of shard.run are played one after another in this process, each
through shard.DeviceOps (row-range sketch builds through a CSR view,
pg_partial_sums over its vertex range), the exchange being the concatenation
of the ranks' rows and the reductions element-wise sums. The results must
equal one pg_analyze over the whole graph — the exchanged sketch table and
the histogram bit for bit, TC and T_v within 1e-9, LCC within 1e-5 — and the
oracle's."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2208_11469_gb300 import synth

pytestmark = pytest.mark.gpu

RTOL_F64 = 1e-9


@pytest.fixture(scope="module")
def pg():
    from paper_2208_11469_gb300 import build, pg as _pg
    build.build()
    _pg.lib()
    return _pg


def _play_ranks(pg, g, kind, est, world, **kw):
    from paper_2208_11469_gb300 import shard
    ops = shard.DeviceOps(g, kind, est, **kw)
    bounds = shard.partition(pg.Graph.degrees(g).cpu().numpy(), world)
    table = torch.cat([ops.build_rows(int(bounds[r]), int(bounds[r + 1])) for r in range(world)], dim=0)
    ops.set_table(table)
    sums = torch.zeros(g.n, dtype=torch.float64, device=g.device)
    hist = None
    for r in range(world):
        s, h = ops.partial(int(bounds[r]), int(bounds[r + 1]))
        sums += s
        hist = h if hist is None else hist + h
    return ops.finalize(hist, sums), table


CASES = [
    ("bloom", 1, dict(bits=448, b=2)),
    ("bloom", 2, dict(bits=256, b=1)),
    ("khash", 3, dict(k=64)),
    ("khash", 3, dict(k=20)),
    ("onehash", 4, dict(k=32)),
]


@pytest.mark.parametrize("world", [1, 2, 3, 8])
@pytest.mark.parametrize("kind,est,kw", CASES)
def test_partitioned_passes_equal_one_pass(pg, world, kind, est, kw):
    rp, cl = synth.rmat(13, 16, seed=9)
    g = pg.graph(rp.cuda(), cl.cuda())
    sk_kind = {"bloom": pg.SK_BLOOM, "khash": pg.SK_KHASH, "onehash": pg.SK_1HASH}[kind]
    if kind == "bloom":
        full = pg.build_bloom(g, kw["bits"], kw["b"], seed=3)
    else:
        full = pg.build_minhash(g, sk_kind, kw["k"], seed=3)
    got, table = _play_ranks(pg, g, sk_kind, est, world, seed=3, **kw)
    assert torch.equal(table.view(-1), full.data[: g.n * full.stride])
    dev = g.device
    want_hist = torch.zeros(pg.hist_bins(full, est), dtype=torch.int64, device=dev)
    tri = torch.empty(g.n, dtype=torch.float64, device=dev)
    lcc = torch.empty(g.n, dtype=torch.float32, device=dev)
    tc = pg.tc_result_buffer(dev)
    pg.analyze(g, full, est, tc=tc, lcc=lcc, tri=tri, hist=want_hist)
    assert torch.equal(got["hist"], want_hist)
    w = pg.read_tc_result(tc)
    assert got["tc"]["edges"] == w["edges"] and got["tc"]["count_sum"] == w["count_sum"]
    assert got["tc"]["est_tc"] == pytest.approx(w["est_tc"], rel=RTOL_F64)
    np.testing.assert_allclose(got["tri"].cpu().numpy(), tri.cpu().numpy(), rtol=RTOL_F64, atol=1e-9)
    np.testing.assert_allclose(got["lcc"].cpu().numpy(), lcc.cpu().numpy(), rtol=1e-5, atol=1e-7)
    okw = dict(l=kw["bits"], b=kw["b"]) if kind == "bloom" else dict(k=kw["k"])
    ref = O.analyze(rp.numpy(), cl.numpy(), est, seed=3, **okw)
    assert got["tc"]["est_tc"] == pytest.approx(ref["tc"], rel=RTOL_F64)
    np.testing.assert_allclose(got["tri"].cpu().numpy(), ref["T"], rtol=RTOL_F64, atol=1e-9)


def test_partial_sums_rejects_what_has_no_partial_form(pg):
    rp, cl = synth.erdos_renyi(512, 6.0, seed=2)
    g = pg.graph(rp.cuda(), cl.cuda())
    oh = pg.build_minhash(g, pg.SK_1HASH, 16, seed=1)
    with pytest.raises(pg.PGError) as ei:
        pg.partial_sums(g, oh, pg.EST_1H_KMV, 0, g.n)
    assert ei.value.status == -9
    bf = pg.build_bloom(g, 256, 2, seed=1)
    with pytest.raises(pg.PGError) as ei:
        pg.partial_sums(g, bf, pg.EST_BF_AND, 5, g.n + 1)
    assert ei.value.status == -1
    s, h = pg.partial_sums(g, bf, pg.EST_BF_AND, 7, 7)  # an empty range adds nothing
    assert not s.any() and not h.any()

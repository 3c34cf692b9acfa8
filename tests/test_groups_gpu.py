"""GPU parity on a graph of more than 2^20 vertices, whose edge list is cut
into several vertex groups (blocks of 2^20 ids of v; three here).

Per-edge outputs must land at each edge's upper-edge index, which the kernels
derive from the group offsets; the pass walks the groups as separate segments
(and, for a vertex range, only part of each); Jarvis-Patrick reads its counts
in the list's own order; the exact per-edge counts derive the same positions.
Bar as everywhere: bit-exact integer counts and histograms, 1e-9 relative on
double totals and T_v, 1e-5 relative on float outputs."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2208_11469_gb300 import synth

pytestmark = pytest.mark.gpu

RTOL_F32 = 1e-5
RTOL_F64 = 1e-9
N = (1 << 21) + 4099


@pytest.fixture(scope="module")
def pg():
    from paper_2208_11469_gb300 import build, pg as _pg
    build.build()
    _pg.lib()
    return _pg


_G = {}


def graph_np():
    """Erdos-Renyi background (average degree 3) plus a few hubs of 30 000
    neighbours spread over every group, so that rows cross group cuts."""
    if "g" not in _G:
        rp, cl = synth.erdos_renyi(N, 3.0, seed=21)
        g = torch.Generator().manual_seed(21)
        hubs = [7, (1 << 20) + 3, (1 << 21) + 11]
        src = torch.repeat_interleave(torch.arange(N), (rp[1:] - rp[:-1]).long())
        us, vs = [src], [cl.long()]
        for h in hubs:
            pick = torch.randperm(N, generator=g)[:30000]
            pick = pick[pick != h]
            us.append(torch.full((pick.numel(),), h, dtype=torch.int64))
            vs.append(pick.long())
        rp2, cl2 = synth.csr_from_pairs(torch.cat(us), torch.cat(vs), N)
        _G["g"] = (rp2.numpy().astype(np.int32), cl2.numpy().astype(np.int32))
    return _G["g"]


def _np(t):
    return t.cpu().numpy()


@pytest.mark.parametrize("est,kind,kw", [
    (O.EST_BF_AND, "bloom", dict(l=64, b=1)),
    (O.EST_BF_AND, "bloom", dict(l=448, b=2)),   # the lean 448-bit kernel
    (O.EST_KH, "khash", dict(k=16)),
    (O.EST_1H, "onehash", dict(k=8)),
    (O.EST_BF_OR, "bloom", dict(l=256, b=2)),    # the generic kernel
])
def test_multi_group_outputs_match_oracle(pg, est, kind, kw):
    rp, cl = graph_np()
    g = pg.graph(torch.from_numpy(rp).cuda(), torch.from_numpy(cl).cuda())
    seed = 5
    if kind == "bloom":
        sk = pg.build_bloom(g, kw["l"], kw["b"], seed=seed)
    else:
        sk = pg.build_minhash(g, pg.SK_KHASH if kind == "khash" else pg.SK_1HASH, kw["k"], seed=seed)
    r = O.analyze(rp, cl, est, seed=seed, **kw)
    m, dev = g.m, g.device
    assert m == r["m"]
    out = dict(tc=pg.tc_result_buffer(dev), lcc=torch.empty(g.n, dtype=torch.float32, device=dev),
               tri=torch.empty(g.n, dtype=torch.float64, device=dev),
               edge_cn=torch.empty(m, dtype=torch.float32, device=dev),
               edge_jac=torch.empty(m, dtype=torch.float32, device=dev),
               edge_count=torch.empty(m, dtype=torch.int32, device=dev))
    pg.analyze(g, sk, est, **out)
    # per-edge outputs in upper-edge order
    assert np.array_equal(_np(out["edge_count"]), np.asarray(r["counts"]["count"], np.int32))
    floor = 1e-9 * (O.degrees(rp)[r["eu"]] + O.degrees(rp)[r["ev"]]) + 1e-6 if est == O.EST_BF_OR else 1e-6
    got_cn = _np(out["edge_cn"]).astype(np.float64)
    assert np.all(np.abs(got_cn - r["cn"]) <= floor + RTOL_F32 * np.abs(r["cn"]))
    np.testing.assert_allclose(_np(out["edge_jac"]), r["jac"], rtol=RTOL_F32, atol=1e-7)
    # totals and per-vertex sums
    tc = pg.read_tc_result(out["tc"])
    assert tc["edges"] == m
    assert tc["est_tc"] == pytest.approx(r["tc"], rel=RTOL_F64)
    np.testing.assert_allclose(_np(out["tri"]), r["T"], rtol=RTOL_F64, atol=1e-9)
    np.testing.assert_allclose(_np(out["lcc"]), r["lcc"], rtol=RTOL_F32, atol=1e-7)
    # the same sums from vertex ranges that cut every group (pg_partial_sums)
    if est != O.EST_BF_OR:
        bounds = [0, 333_333, (1 << 20) + 17, (1 << 21) - 1, g.n]
        sums = torch.zeros(g.n, dtype=torch.float64, device=dev)
        hist = torch.zeros(pg.hist_bins(sk, est), dtype=torch.int64, device=dev)
        for a, b in zip(bounds[:-1], bounds[1:]):
            pg.partial_sums(g, sk, est, a, b, sums=sums, hist=hist)
        tcb, lcc2, tri2 = pg.finalize_sums(g, sk, est, hist, sums)
        assert pg.read_tc_result(tcb)["est_tc"] == pytest.approx(r["tc"], rel=RTOL_F64)
        np.testing.assert_allclose(_np(tri2), r["T"], rtol=RTOL_F64, atol=1e-9)


def test_multi_group_exact_and_jarvis_patrick(pg):
    rp, cl = graph_np()
    g = pg.graph(torch.from_numpy(rp).cuda(), torch.from_numpy(cl).cuda())
    r = O.analyze(rp, cl, O.EST_EXACT)
    cnt, _, _ = pg.edge_counts(g, None, O.EST_EXACT)
    assert np.array_equal(_np(cnt), r["counts"]["count"].astype(np.int32))
    tc = pg.triangle_count(g, None, O.EST_EXACT)
    assert tc["exact_tc"] == r["tc_exact"]
    # Jarvis-Patrick with k-Hash (keep test on d_u + d_v) reads the counts in list order
    sk = pg.build_minhash(g, pg.SK_KHASH, 16, seed=3)
    ref = O.jarvis_patrick(rp, cl, O.EST_KH, 2.0, k=16, seed=3)
    labels, res = pg.jarvis_patrick(g, sk, O.EST_KH, 2.0)
    assert np.array_equal(_np(labels), ref["labels"])
    assert res["clusters"] == ref["clusters"] and res["kept"] == ref["kept"]
    # and with the Bloom L estimator on 64-bit filters, where collisions keep many edges
    bf = pg.build_bloom(g, 64, 1, seed=3)
    ref = O.jarvis_patrick(rp, cl, O.EST_BF_L, 1.5, l=64, b=1, seed=3)
    labels, res = pg.jarvis_patrick(g, bf, O.EST_BF_L, 1.5)
    assert ref["kept"] > 1000
    assert np.array_equal(_np(labels), ref["labels"])
    assert res["clusters"] == ref["clusters"] and res["kept"] == ref["kept"]

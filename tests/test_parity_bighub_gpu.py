"""GPU parity at hub degrees like the R-MAT scale-24 workload's.

The passes carry per-vertex sums as fixed-point integers V = round(est * 2^42)
summed over runs of up to 32 edges. An estimate of 2^16 or more (an edge
between two vertices of ~10^5 neighbours with near-identical neighbourhoods,
as R-MAT's hub-hub edges are) does not fit that form and is added as a
double at both endpoints instead. These graphs have three mutually adjacent
hubs of 80 000 neighbours drawn from one pool of 82 000, so every hub-hub
edge takes that branch for the MinHash estimators (k-Hash in the lean kernels
k = 16/32/64 and the generic kernel, 1-Hash, KMV) and for the Bloom OR
estimator, whose estimate is near d_u + d_v there.

Bar (Sec. VII sums over every edge, whatever its degree): bit-exact per-edge
counts and histograms, 1e-9 relative on the triangle total and on per-vertex
triangles T_v, 1e-5 relative on LCC and per-edge common-neighbour floats."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2208_11469_gb300 import synth

pytestmark = pytest.mark.gpu

RTOL_F32 = 1e-5
RTOL_F64 = 1e-9
HUBS = (5, 77777, 100003)
N = 120000


def big_hub_graph(seed=12):
    """ER background (average degree 4) on N vertices plus three hubs, each
    adjacent to the other two and to 80 000 vertices of a shared pool of
    82 000."""
    rp, cl = synth.erdos_renyi(N, 4.0, seed=seed)
    g = torch.Generator().manual_seed(seed)
    others = torch.tensor([v for v in range(N) if v not in HUBS])
    pool = others[torch.randperm(others.numel(), generator=g)[:82000]]
    us, vs = [], []
    for h in HUBS:
        pick = pool[torch.randperm(pool.numel(), generator=g)[:80000]]
        us.append(torch.full((pick.numel(),), h, dtype=torch.int64))
        vs.append(pick.long())
    for a in range(3):
        for b in range(a + 1, 3):
            us.append(torch.tensor([HUBS[a]]))
            vs.append(torch.tensor([HUBS[b]]))
    src = torch.repeat_interleave(torch.arange(N), (rp[1:] - rp[:-1]).long())
    u = torch.cat([src] + us).long()
    v = torch.cat([cl.long()] + vs).long()
    rp2, cl2 = synth.csr_from_pairs(u, v, N)
    return rp2.numpy().astype(np.int32), cl2.numpy().astype(np.int32)


_G = {}


def graph_np():
    if "g" not in _G:
        _G["g"] = big_hub_graph()
    return _G["g"]


@pytest.fixture(scope="module")
def pg():
    from paper_2208_11469_gb300 import build, pg as _pg
    build.build()
    _pg.lib()
    return _pg


def _np(t):
    return t.cpu().numpy()


def _hub_edges(r):
    eu, ev = r["eu"], r["ev"]
    hs = np.array(HUBS)
    return np.flatnonzero(np.isin(eu, hs) & np.isin(ev, hs))


def test_graph_has_the_hub_degrees():
    rp, cl = graph_np()
    d = O.degrees(rp)
    for h in HUBS:
        assert 80002 <= d[h] <= 80002 + 40
    # the pool makes every hub pair share at least 78 000 neighbours
    rows = [set(cl[rp[h]:rp[h + 1]].tolist()) for h in HUBS]
    assert min(len(rows[a] & rows[b]) for a in range(3) for b in range(a + 1, 3)) >= 78000


CASES = [
    (O.EST_KH, "khash", dict(k=16)),    # lean kernel, 4-lane groups
    (O.EST_KH, "khash", dict(k=32)),    # lean kernel, 8-lane groups
    (O.EST_KH, "khash", dict(k=64)),    # lean kernel, 16-lane groups (the scale-24 bench's)
    (O.EST_KH, "khash", dict(k=48)),    # generic pass kernel
    (O.EST_1H, "onehash", dict(k=32)),
    (O.EST_1H_KMV, "onehash", dict(k=32)),
    (O.EST_BF_OR, "bloom", dict(l=256, b=2)),
]


@pytest.mark.parametrize("est,kind,kw", CASES)
def test_fixed_point_bypass_matches_oracle(pg, est, kind, kw):
    rp, cl = graph_np()
    seed = 17
    g = pg.graph(torch.from_numpy(rp).cuda(), torch.from_numpy(cl).cuda())
    if kind == "bloom":
        sk = pg.build_bloom(g, kw["l"], kw["b"], seed=seed)
    else:
        sk = pg.build_minhash(g, pg.SK_KHASH if kind == "khash" else pg.SK_1HASH, kw["k"], seed=seed)
    r = O.analyze(rp, cl, est, seed=seed, **kw)
    assert g.m == r["m"]
    # the case reaches the branch: every hub-hub estimate is at least 2^16
    hub = _hub_edges(r)
    assert hub.size == 3
    assert np.all(r["est"][hub] >= 65536.0), r["est"][hub]
    # per-edge integer counts, bit-exact
    cnt, aux, _ = pg.edge_counts(g, sk, est, want_aux=est == O.EST_BF_OR)
    assert np.array_equal(_np(cnt), np.asarray(r["counts"]["count"], np.int32))
    if est == O.EST_BF_OR:  # the union popcount
        assert np.array_equal(_np(aux), np.asarray(r["counts"]["union"], np.int32))
    # totals and per-vertex sums from the fused pass
    lcc, tri, tcb = pg.clustering(g, sk, est)
    tc = pg.read_tc_result(tcb)
    assert tc["edges"] == r["m"]
    assert tc["est_tc"] == pytest.approx(r["tc"], rel=RTOL_F64)
    T = _np(tri)
    np.testing.assert_allclose(T, r["T"], rtol=RTOL_F64, atol=1e-9)
    np.testing.assert_allclose(T[list(HUBS)], r["T"][list(HUBS)], rtol=RTOL_F64)
    np.testing.assert_allclose(_np(lcc), r["lcc"], rtol=RTOL_F32, atol=1e-7)
    # the same per-vertex sums through pg_analyze with per-edge outputs
    m = g.m
    dev = g.device
    lcc2 = torch.empty(g.n, dtype=torch.float32, device=dev)
    tri2 = torch.empty(g.n, dtype=torch.float64, device=dev)
    cn = torch.empty(m, dtype=torch.float32, device=dev)
    tcb2 = pg.tc_result_buffer(dev)
    pg.analyze(g, sk, est, tc=tcb2, lcc=lcc2, tri=tri2, edge_cn=cn)
    np.testing.assert_allclose(_np(tri2), r["T"], rtol=RTOL_F64, atol=1e-9)
    np.testing.assert_allclose(_np(cn), r["cn"].astype(np.float32), rtol=RTOL_F32, atol=1e-6)
    assert pg.read_tc_result(tcb2)["est_tc"] == pytest.approx(r["tc"], rel=RTOL_F64)

"""GPU parity of 4-clique counting (pg_clique4_count) against the oracle:
exact counts and 3-clique counts bit-exact; with Bloom filters of the
oriented neighbourhoods, the sum of triple-AND popcounts bit-exact and the
double totals within 1e-9 relative."""
import math

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


def _hubs():
    n = 12000
    rp, cl = synth.erdos_renyi(n, 10.0, seed=3)
    src = torch.repeat_interleave(torch.arange(n), (rp[1:] - rp[:-1]).long())
    g = torch.Generator().manual_seed(3)
    u = [torch.zeros(6000, dtype=torch.int64), torch.ones(9000, dtype=torch.int64)]
    v = [torch.randperm(n, generator=g)[:6000], torch.randperm(n, generator=g)[:9000]]
    return synth.csr_from_pairs(torch.cat([src] + u), torch.cat([cl.long()] + v), n)


def _cliques():
    sizes = [4, 6, 9, 12]
    edges, off = [], 0
    for s in sizes:
        edges += [(off + i, off + j) for i in range(s) for j in range(i + 1, s)]
        off += s
    return synth.from_edges(off, edges)


GRAPHS = {
    "er4096": lambda: synth.erdos_renyi(4096, 24.0, seed=1),
    "rmat12": lambda: synth.rmat(12, 16, seed=7),
    "rmat13": lambda: synth.rmat(13, 24, seed=2),
    "hubs": _hubs,
    "cliques": _cliques,
    "k30": lambda: synth.complete_graph(30),
}
_cache = {}


def _graph(name):
    if name not in _cache:
        rp, cl = GRAPHS[name]()
        _cache[name] = (rp.numpy().astype(np.int32), cl.numpy().astype(np.int32))
    return _cache[name]


@pytest.mark.parametrize("name", list(GRAPHS))
def test_exact(pg, name):
    rp, cl = _graph(name)
    g = pg.graph(torch.from_numpy(rp).cuda(), torch.from_numpy(cl).cuda())
    want = O.clique4(rp, cl, O.EST_EXACT)
    got = pg.clique4_count(g, pg.EST_EXACT)
    assert got["exact"] == want["count"] and got["triangles"] == want["triangles"]
    assert got["est"] == float(want["count"])
    if name == "k30":
        assert got["exact"] == math.comb(30, 4)


@pytest.mark.parametrize("name", ["er4096", "rmat12", "rmat13", "hubs", "cliques"])
@pytest.mark.parametrize("est,bits,b", [(1, 256, 2), (1, 448, 1), (2, 1024, 4), (1, 64, 2), (1, 192, 3)])
def test_bloom(pg, name, est, bits, b):
    rp, cl = _graph(name)
    g = pg.graph(torch.from_numpy(rp).cuda(), torch.from_numpy(cl).cuda())
    want = O.clique4(rp, cl, est, l=bits, b=b, seed=5)
    got = pg.clique4_count(g, est, bits, b, seed=5)
    assert got["triangles"] == want["triangles"]
    j = np.arange(bits + 1)
    assert got["count_sum"] == int((j * want["hist"].astype(np.int64)).sum())
    assert got["est"] == pytest.approx(want["count"], rel=RTOL_F64, abs=1e-9)
    alt = O.est_limit(j, b) if est == O.EST_BF_AND else O.est_and(j, bits, b)
    assert got["est_alt"] == pytest.approx(float((want["hist"].astype(np.float64) * alt).sum()), rel=RTOL_F64,
                                           abs=1e-9)
    assert got["exact"] == 0


def test_degenerate_and_errors(pg):
    for rp, cl in (synth.from_edges(3, []), synth.from_edges(2, [(0, 1)]), synth.complete_graph(4)):
        g = pg.graph(rp.to(torch.int32).cuda(), cl.to(torch.int32).cuda())
        want = O.clique4(rp.numpy(), cl.numpy(), O.EST_EXACT)
        got = pg.clique4_count(g, pg.EST_EXACT)
        assert (got["exact"], got["triangles"]) == (want["count"], want["triangles"])
        gb = pg.clique4_count(g, pg.EST_BF_AND, 128, 2)
        assert gb["triangles"] == want["triangles"]
    g = pg.graph(*[t.to(torch.int32).cuda() for t in synth.complete_graph(5)])
    for bad in (dict(est=pg.EST_KH), dict(est=pg.EST_BF_AND, bits=100), dict(est=pg.EST_BF_AND, bits=2048)):
        with pytest.raises(pg.PGError) as ei:
            pg.clique4_count(g, bad["est"], bad.get("bits", 256))
        assert ei.value.status == -9

"""pg_upload_build: the CSR copied from page-locked host memory in row chunks
while the sketches of each chunk are built must leave the same device CSR
and bit-identical sketches as a plain copy followed by the single-call
builders, for every chunk size (one row per chunk up to a single chunk), with
the copy on its own stream or on the compute stream, and with hub rows that
take the builders' second kernel."""
import numpy as np
import pytest
import torch

from paper_2208_11469_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pg():
    from paper_2208_11469_gb300 import build, pg as _pg
    build.build()
    _pg.lib()
    return _pg


def _hubs():
    n = 9000
    rp, cl = synth.erdos_renyi(n, 6.0, seed=2)
    src = torch.repeat_interleave(torch.arange(n), (rp[1:] - rp[:-1]).long())
    hub = torch.randperm(n, generator=torch.Generator().manual_seed(1))[:8900]
    u = torch.cat([src, torch.full((8900,), 5, dtype=torch.int64)])
    v = torch.cat([cl.long(), hub])
    return synth.csr_from_pairs(u, v, n)


GRAPHS = {
    "rmat12": lambda: synth.rmat(12, 16, seed=7),
    "hubs": _hubs,
    "no_edges": lambda: synth.from_edges(5, []),
}


def _sketches(pg, g):
    return [pg.alloc_sketch(g, pg.SK_BLOOM, bits=256, b=2, seed=3),
            pg.alloc_sketch(g, pg.SK_BLOOM, bits=64, b=1, seed=4),
            pg.alloc_sketch(g, pg.SK_KHASH, k=32, seed=5),
            pg.alloc_sketch(g, pg.SK_1HASH, k=16, seed=6)]


def _reference(pg, rp, cl):
    g = pg.graph(rp.cuda(), cl.cuda(), build_index=False)
    out = []
    for sk in _sketches(pg, g):
        if sk.kind == pg.SK_BLOOM:
            pg.build_bloom(g, sk.bits, sk.b, sk.seed, out=sk)
        else:
            pg.build_minhash(g, sk.kind, sk.k, sk.seed, out=sk)
        out.append(sk.data.cpu())
    return out


@pytest.mark.parametrize("name", list(GRAPHS))
@pytest.mark.parametrize("chunk", [1, 700, 1 << 30])
@pytest.mark.parametrize("own_stream", [True, False])
def test_upload_build_matches_copy_then_build(pg, name, chunk, own_stream):
    rp, cl = GRAPHS[name]()
    rp, cl = rp.to(torch.int32), cl.to(torch.int32)
    if name == "rmat12" and chunk == 1 and not own_stream:
        pytest.skip("one row per chunk is covered with the copy stream")
    want = _reference(pg, rp, cl)
    host_rp, host_col = rp.pin_memory(), cl.pin_memory()
    # device CSR buffers holding garbage before the upload
    g = pg.graph(torch.full_like(rp, -7, device="cuda"), torch.full_like(cl, 123456, device="cuda"),
                 build_index=False)
    sks = _sketches(pg, g)
    for sk in sks:
        sk.data.fill_(0xA5)
    cs = torch.cuda.Stream() if own_stream else torch.cuda.current_stream()
    pg.upload_build(g, host_rp, host_col, sks, chunk_entries=chunk, copy_stream=cs)
    torch.cuda.synchronize()
    assert torch.equal(g.row_ptr.cpu(), rp) and torch.equal(g.col.cpu(), cl)
    for sk, w in zip(sks, want):
        got = sk.data.cpu()
        if sk.kind == pg.SK_BLOOM:
            assert torch.equal(got, w), (name, sk.kind, sk.bits)
        else:
            # the builders write the first k entries of each row; padding is not part of the sketch
            k = sk.k
            gv = got.view(torch.int32).view(g.n, -1)[:, :k]
            wv = w.view(torch.int32).view(g.n, -1)[:, :k]
            assert torch.equal(gv, wv), (name, sk.kind)


def test_upload_build_argument_errors(pg):
    rp, cl = synth.rmat(8, 8, seed=1)
    rp, cl = rp.to(torch.int32), cl.to(torch.int32)
    g = pg.graph(rp.cuda(), cl.cuda(), build_index=False)
    sks = _sketches(pg, g)
    bad = rp.clone()
    bad[-1] += 1
    for args in ((bad.pin_memory(), cl.pin_memory(), dict()), (rp.pin_memory(), cl.pin_memory(),
                                                                  dict(chunk_entries=0))):
        with pytest.raises(pg.PGError) as ei:
            pg.upload_build(g, args[0], args[1], sks, **args[2])
        assert ei.value.status == -1
    tiny = torch.empty(8, dtype=torch.uint8, device="cuda")
    with pytest.raises(pg.PGError) as ei:
        pg.upload_build(g, rp.pin_memory(), cl.pin_memory(), sks, workspace=tiny)
    assert ei.value.status == -4

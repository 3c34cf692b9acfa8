"""The timed step of bench.py runs the edge index and the Bloom build on a
side stream while the k-Hash build runs on the launching stream, each build
with its own workspace (the hub-row list). Its outputs must equal the same
calls made one after another on one stream: the sketch tables and the TC
results bit for bit, T_v within 1e-12 relative (double atomics on the v
side add in a run-dependent order). The graph has rows long enough for the
hub kernels of both builds (Bloom: more than 8192 ids, k-Hash: more than
2048), so that both builds keep hub records at the same time."""
import os
import sys

import pytest
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

pytestmark = pytest.mark.gpu


def _graph(dev):
    from paper_2208_11469_gb300 import synth
    n = 1 << 15
    rp, cl = synth.erdos_renyi(n, 8.0, seed=31)
    g = torch.Generator().manual_seed(31)
    src = torch.repeat_interleave(torch.arange(n), (rp[1:] - rp[:-1]).long())
    us, vs = [src], [cl.long()]
    for h, d in ((5, 12000), (777, 9000), (n - 3, 3000), (1 << 14, 2500)):
        pick = torch.randperm(n, generator=g)[:d]
        pick = pick[pick != h]
        us.append(torch.full((pick.numel(),), h, dtype=torch.int64))
        vs.append(pick.long())
    rp2, cl2 = synth.csr_from_pairs(torch.cat(us), torch.cat(vs), n)
    return rp2.to(dev), cl2.to(dev)


def test_two_stream_step_equals_one_stream():
    import bench
    from paper_2208_11469_gb300 import build, pg
    build.build()
    dev = torch.device("cuda:0")
    rp, cl = _graph(dev)
    pipe = bench.Pipeline("rmat22", rp, cl)
    g = pipe.g
    assert int((rp[1:] - rp[:-1]).max()) > 8192
    for _ in range(3):
        pipe.step()
    torch.cuda.synchronize()
    bf, kh = pipe.passes[0][1], pipe.passes[1][1]
    # the same calls, one after another on one stream, into fresh buffers
    ref_bf = pg.build_bloom(g, bf.bits, bf.b, bf.seed)
    ref_kh = pg.build_minhash(g, kh.kind, kh.k, kh.seed)
    assert torch.equal(bf.data[: g.n * bf.stride], ref_bf.data[: g.n * ref_bf.stride])
    assert torch.equal(kh.data[: g.n * kh.stride], ref_kh.data[: g.n * ref_kh.stride])
    for (name, sk, est), ref_sk in zip(pipe.passes, (ref_bf, ref_kh)):
        tc = pg.tc_result_buffer(dev)
        tri = torch.empty(g.n, dtype=torch.float64, device=dev)
        lcc = torch.empty(g.n, dtype=torch.float32, device=dev)
        pg.analyze(g, ref_sk, est, tc=tc, tri=tri, lcc=lcc)
        got = pipe.out[name]
        assert torch.equal(got["tc"], tc), name
        torch.testing.assert_close(got["tri"], tri, rtol=1e-12, atol=0)


def test_e2e_step_equals_one_stream():
    """The end-to-end step: pg_upload_build from page-locked host buffers on a
    copy stream, the edge index on a side stream once the CSR has landed
    (beside the builds' tail), then the passes."""
    import bench
    from paper_2208_11469_gb300 import build, pg
    build.build()
    dev = torch.device("cuda:0")
    rp, cl = _graph(dev)
    pipe = bench.Pipeline("rmat22", rp, cl)
    g = pipe.g
    host_rp = rp.cpu().pin_memory()
    host_cl = cl.cpu().pin_memory()
    bf, kh = pipe.passes[0][1], pipe.passes[1][1]
    ref_bf = pg.build_bloom(g, bf.bits, bf.b, bf.seed)
    ref_kh = pg.build_minhash(g, kh.kind, kh.k, kh.seed)
    refs = []
    for (name, sk, est), ref_sk in zip(pipe.passes, (ref_bf, ref_kh)):
        tc = pg.tc_result_buffer(dev)
        tri = torch.empty(g.n, dtype=torch.float64, device=dev)
        pg.analyze(g, ref_sk, est, tc=tc, tri=tri)
        refs.append((name, tc, tri))
    # wipe the device CSR, the sketches and the outputs: the e2e steps must rebuild all of them
    cl_ref = cl.clone()
    g.col.zero_()
    bf.data.zero_()
    kh.data.zero_()
    for name, _, _ in refs:
        pipe.out[name]["tc"].zero_()
    bench.e2e_steps(pipe, host_rp, host_cl, 2)
    torch.cuda.synchronize()
    assert torch.equal(g.col, cl_ref)
    assert torch.equal(bf.data[: g.n * bf.stride], ref_bf.data[: g.n * ref_bf.stride])
    assert torch.equal(kh.data[: g.n * kh.stride], ref_kh.data[: g.n * ref_kh.stride])
    for name, tc, tri in refs:
        assert torch.equal(pipe.out[name]["tc"], tc), name
        torch.testing.assert_close(pipe.out[name]["tri"], tri, rtol=1e-12, atol=0)

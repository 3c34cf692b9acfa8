"""Serving (pg_server_*, pg_submit, pg_poll, pg_cancel): answers equal the
single-call entry points on the same inputs, alone and in a mix of requests
of uneven sizes; admission by free arena bytes; cancellation, unknown
tickets, time-limited polls and shutdown with requests in flight. No test
makes a kernel wait or fault: every wait is on the host."""
import numpy as np
import pytest
import torch

from paper_2208_11469_gb300 import synth


@pytest.fixture(scope="module")
def pg():
    from paper_2208_11469_gb300 import build, pg as _pg
    build.build()
    _pg.lib()
    return _pg


def test_reserved_bytes_host_rule(pg):
    """The server's own reservation grows with n (one membership bitmap of n
    bits per stream) and with the stream count; it needs no GPU."""
    small = pg.Csr(None, None, 1000, 0)
    big = pg.Csr(None, None, 1_000_000, 0)
    import ctypes
    L = pg.lib()
    o1 = pg.ServerOpts(1, 0, 0, 0, 0, 0, 0, 0)
    o4 = pg.ServerOpts(4, 0, 0, 0, 0, 0, 0, 0)
    a = L.pg_server_reserved_bytes(ctypes.byref(small), ctypes.byref(o1))
    b = L.pg_server_reserved_bytes(ctypes.byref(big), ctypes.byref(o1))
    c = L.pg_server_reserved_bytes(ctypes.byref(big), ctypes.byref(o4))
    assert b - a >= (1_000_000 - 1000) // 8 - 512
    assert c - b >= 3 * (1_000_000 // 8) - 1024


# ------------------------------------------------------------------- GPU
@pytest.fixture(scope="module")
def world(pg):
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    rp, cl = synth.rmat(13, 16, seed=3)
    g = pg.graph(rp.cuda(), cl.cuda())
    bf = pg.build_bloom(g, 512, 2, seed=1)
    kh = pg.build_minhash(g, pg.SK_KHASH, 32, seed=1)
    return dict(rp=rp.numpy(), cl=cl.numpy(), g=g, bf=bf, kh=kh)


def _pairs(world, count, seed, invalid=False):
    n = world["g"].n
    p = synth.random_pairs(n, count, seed, torch.from_numpy(world["rp"]), torch.from_numpy(world["cl"])).numpy()
    if invalid and count >= 4:
        p[0] = (-1, 3)
        p[1] = (2, n)
        p[2] = (n + 5, -7)
    return p


def _want_pairs(pg, world, pairs, est):
    sk = world["kh"] if est == pg.EST_KH else world["bf"]
    if est == pg.EST_EXACT:
        sk = None
    cn, jac = pg.jaccard_pairs(world["g"], sk, est, torch.from_numpy(pairs).cuda())
    return cn.cpu().numpy(), jac.cpu().numpy()


def _induced(rp, cl, S):
    """Induced CSR with local ids in sorted-vertex order."""
    S = np.unique(S)
    pos = -np.ones(rp.size - 1, np.int64)
    pos[S] = np.arange(S.size)
    rows = []
    for v in S:
        nb = pos[cl[rp[v]:rp[v + 1]]]
        rows.append(nb[nb >= 0])
    srp = np.zeros(S.size + 1, np.int32)
    srp[1:] = np.cumsum([r.size for r in rows])
    scl = np.concatenate(rows).astype(np.int32) if rows else np.zeros(0, np.int32)
    return srp, scl


def _want_subgraph(pg, world, S, est):
    srp, scl = _induced(world["rp"], world["cl"], S)
    if scl.size == 0:
        return None
    g = pg.graph(torch.from_numpy(srp).cuda(), torch.from_numpy(scl).cuda())
    sk = None if est == pg.EST_EXACT else pg.build_bloom(g, 512, 2, seed=1)
    return pg.triangle_count(g, sk, est)


def _same_pairs(got, want):
    np.testing.assert_array_equal(got["cn"], want[0])
    np.testing.assert_array_equal(got["jac"], want[1])


@pytest.mark.gpu
def test_pairs_alone_equal_single_call(pg, world):
    sv = pg.Server(world["g"], [world["bf"], world["kh"]], 256 << 20)
    try:
        for est in (pg.EST_BF_AND, pg.EST_BF_L, pg.EST_KH, pg.EST_EXACT):
            for count, seed in ((1, 1), (37, 2), (1024, 3), (5000, 4)):
                pairs = _pairs(world, count, seed, invalid=True)
                r = sv.wait(sv.submit_pairs(pairs, est))
                assert r["status"] == 0 and r["count"] == count
                _same_pairs(r, _want_pairs(pg, world, pairs, est))
        st = sv.stats()
        assert st["completed"] == 16 and st["failed"] == 0 and st["pair_launches"] >= 12
    finally:
        sv.close()


@pytest.mark.gpu
def test_subgraph_alone_equal_single_call(pg, world):
    sv = pg.Server(world["g"], [world["bf"], world["kh"]], 256 << 20, sub_bits=512, sub_b=2, sub_seed=1)
    try:
        rng = np.random.default_rng(5)
        starts = rng.integers(0, world["cl"].size, 6)
        for i, j in enumerate(starts):
            v = int(np.searchsorted(world["rp"], j, side="right") - 1)
            S = synth.bfs_ball(world["rp"], world["cl"], v, [50, 2000, 20000][i % 3])
            S_dup = np.concatenate([S, S[: S.size // 3]])[::-1].copy()  # duplicates and order do not matter
            for est in (pg.EST_BF_AND, pg.EST_BF_L, pg.EST_EXACT):
                r = sv.wait(sv.submit_subgraph(S_dup, est))
                assert r["status"] == 0 and r["count"] == np.unique(S).size
                want = _want_subgraph(pg, world, S, est)
                if want is None:
                    assert r["tc"]["edges"] == 0
                    continue
                assert r["tc"]["edges"] == want["edges"]
                assert r["tc"]["count_sum"] == want["count_sum"]
                assert r["tc"]["exact_tc"] == want["exact_tc"]
                assert r["tc"]["est_tc"] == want["est_tc"]
    finally:
        sv.close()


@pytest.mark.gpu
def test_subgraph_exact_against_oracle(pg, world):
    from oracle import oracle as O
    sv = pg.Server(world["g"], [world["bf"]], 64 << 20)
    try:
        v = int(np.argmax(np.diff(world["rp"])))  # the largest hub
        S = synth.bfs_ball(world["rp"], world["cl"], v, 3000)
        srp, scl = _induced(world["rp"], world["cl"], S)
        ref = O.analyze(srp, scl, O.EST_EXACT)
        r = sv.wait(sv.submit_subgraph(S, pg.EST_EXACT))
        assert r["tc"]["exact_tc"] == int(round(ref["tc"])) and r["tc"]["edges"] == ref["m"]
    finally:
        sv.close()


@pytest.mark.gpu
def test_mix_equals_alone(pg, world):
    """Forty requests of uneven sizes and kinds submitted back to back: every
    answer equals the single-call answer for the same input."""
    sv = pg.Server(world["g"], [world["bf"], world["kh"]], 512 << 20, iteration_pairs=16384)
    rng = np.random.default_rng(11)
    jobs = []
    try:
        for i in range(40):
            if i % 5 == 4:
                j = int(rng.integers(0, world["cl"].size))
                v = int(np.searchsorted(world["rp"], j, side="right") - 1)
                S = synth.bfs_ball(world["rp"], world["cl"], v, int(10 ** rng.uniform(2, 4.3)))
                est = [pg.EST_BF_AND, pg.EST_EXACT][i % 2]
                jobs.append(("sub", S, est, sv.submit_subgraph(S, est)))
            else:
                P = int(np.clip(round(rng.lognormal(np.log(256), 2.0)), 1, 65536))
                est = [pg.EST_BF_AND, pg.EST_BF_L, pg.EST_KH, pg.EST_BF_AND][i % 4]
                pairs = _pairs(world, P, 100 + i, invalid=(i % 3 == 0))
                jobs.append(("pairs", pairs, est, sv.submit_pairs(pairs, est)))
        for kind, x, est, t in jobs:
            r = sv.wait(t)
            assert r["status"] == 0
            if kind == "pairs":
                _same_pairs(r, _want_pairs(pg, world, x, est))
            else:
                want = _want_subgraph(pg, world, x, est)
                if want is None:
                    assert r["tc"]["edges"] == 0
                else:
                    assert (r["tc"]["edges"], r["tc"]["count_sum"], r["tc"]["exact_tc"], r["tc"]["est_tc"]) == \
                        (want["edges"], want["count_sum"], want["exact_tc"], want["est_tc"])
        st = sv.stats()
        assert st["completed"] == 40 and st["queued"] == 0 and st["running"] == 0 and st["arena_used"] == 0
    finally:
        sv.close()


@pytest.mark.gpu
def test_admission_by_free_arena(pg, world):
    """An arena that holds about three 65536-pair requests at once: twelve of
    them all complete (admitted as earlier ones free their memory), the peak
    stays within the arena, and a request larger than the whole arena is
    refused at submission."""
    reserved = pg.Server.reserved_bytes(world["g"])
    per = 65536 * 16
    sv = pg.Server(world["g"], [world["bf"]], reserved + 3 * per + 4096)
    try:
        tickets = [(sv.submit_pairs(_pairs(world, 65536, 200 + i), pg.EST_BF_AND), i) for i in range(12)]
        with pytest.raises(pg.PGError) as ei:
            sv.submit_pairs(_pairs(world, 300000, 7), pg.EST_BF_AND)
        assert ei.value.status == -4
        for t, i in tickets:
            r = sv.wait(t)
            assert r["status"] == 0
        st = sv.stats()
        assert st["arena_peak"] <= st["arena_bytes"] and st["arena_peak"] >= per
        assert st["completed"] == 12
    finally:
        sv.close()


@pytest.mark.gpu
def test_cancel_poll_unknown_and_shutdown(pg, world):
    reserved = pg.Server.reserved_bytes(world["g"])
    sv = pg.Server(world["g"], [world["bf"]], reserved + 2 * 65536 * 16 + 4096)
    tickets = [sv.submit_pairs(_pairs(world, 65536, 300 + i), pg.EST_BF_AND) for i in range(10)]
    # the last one waits for arena space behind the others: cancel it, or it already runs
    rc = sv.cancel(tickets[-1])
    assert rc in (0, -8)
    r = sv.wait(tickets[-1])
    assert r["status"] == (-10 if rc == 0 else 0)
    for t in tickets[:-1]:
        assert sv.wait(t)["status"] == 0
    with pytest.raises(pg.PGError) as ei:
        sv.poll(tickets[0])  # already collected
    assert ei.value.status == -7
    with pytest.raises(pg.PGError) as ei:
        sv.poll(10 ** 9)
    assert ei.value.status == -7
    assert sv.cancel(10 ** 9) == -7
    # a time-limited poll on a queued request returns "not yet" (None) or the answer
    more = [sv.submit_pairs(_pairs(world, 65536, 400 + i), pg.EST_BF_AND) for i in range(6)]
    got = sv.poll(more[-1], timeout_us=100)
    assert got is None or got["status"] == 0
    # shutdown with requests queued and running: returns, queued ones are cancelled
    sv.close()
    assert sv._h is None


@pytest.mark.gpu
def test_bad_requests(pg, world):
    sv = pg.Server(world["g"], [world["bf"]], 64 << 20)
    try:
        with pytest.raises(pg.PGError) as ei:
            sv.submit_pairs(_pairs(world, 10, 1), pg.EST_KH)  # no k-Hash sketch resident
        assert ei.value.status == -9
        with pytest.raises(pg.PGError) as ei:
            sv.submit_subgraph(np.array([0, world["g"].n], np.int32), pg.EST_BF_AND)
        assert ei.value.status == -1
        with pytest.raises(pg.PGError) as ei:
            sv.submit_subgraph(np.array([0, 1], np.int32), pg.EST_KH)
        assert ei.value.status == -9
        r = sv.wait(sv.submit_pairs(np.zeros((0, 2), np.int32), pg.EST_BF_AND))
        assert r["status"] == 0 and r["count"] == 0
        r = sv.wait(sv.submit_subgraph(np.array([], np.int32), pg.EST_BF_AND))
        assert r["status"] == 0 and r["tc"]["edges"] == 0
        isolated = np.flatnonzero(np.diff(world["rp"]) == 0)[:5]
        r = sv.wait(sv.submit_subgraph(isolated, pg.EST_BF_AND))
        assert r["status"] == 0 and r["tc"]["edges"] == 0 and r["tc"]["est_tc"] == 0.0
    finally:
        sv.close()


@pytest.mark.gpu
def test_submit_many_equals_single_calls(pg, world):
    """A burst through pg_submit_many / pg_poll_many: every answer equals the
    single-call answer, the pair launches take many requests each, and the
    concatenated form (one pair array, per-request slices) gives the same."""
    sv = pg.Server(world["g"], [world["bf"], world["kh"]], 512 << 20)
    rng = np.random.default_rng(17)
    try:
        items = []
        for i in range(300):
            if i % 50 == 7:
                j = int(rng.integers(0, world["cl"].size))
                v = int(np.searchsorted(world["rp"], j, side="right") - 1)
                items.append(("sub", synth.bfs_ball(world["rp"], world["cl"], v, 3000), pg.EST_BF_AND))
            else:
                P = int(np.clip(round(rng.lognormal(np.log(64), 1.5)), 1, 65536))
                items.append(("pairs", _pairs(world, P, 500 + i), [pg.EST_BF_AND, pg.EST_KH][i % 2]))
        l0 = sv.stats()["pair_launches"]
        tickets, outs = sv.submit_many(items)
        resp = sv.poll_many(tickets, timeout_us=60_000_000)
        assert (resp["status"] == 0).all()
        assert sv.stats()["pair_launches"] - l0 < 100  # requests share launches
        for (kind, x, est), r, o in zip(items, resp, outs):
            if kind == "pairs":
                want = _want_pairs(pg, world, x, est)
                np.testing.assert_array_equal(o[0], want[0])
                np.testing.assert_array_equal(o[1], want[1])
            else:
                want = _want_subgraph(pg, world, x, est)
                assert (r["edges"], r["count_sum"], r["est_tc"]) == (want["edges"], want["count_sum"], want["est_tc"])
        # the concatenated form
        pl = [x for k, x, _ in items if k == "pairs"]
        offs = np.concatenate([[0], np.cumsum([p.shape[0] for p in pl])])
        t2, cn, jac = sv.submit_pairs_many(np.concatenate(pl), offs, pg.EST_BF_L)
        r2 = sv.poll_many(t2, timeout_us=60_000_000)
        assert (r2["status"] == 0).all() and (r2["count"] == np.diff(offs)).all()
        want = _want_pairs(pg, world, np.concatenate(pl), pg.EST_BF_L)
        np.testing.assert_array_equal(cn[: offs[-1]], want[0])
        np.testing.assert_array_equal(jac[: offs[-1]], want[1])
        # unknown tickets come back as not found, without waiting
        r3 = sv.poll_many(np.array([10 ** 9], np.uint64), timeout_us=1000)
        assert r3["status"][0] == -7
    finally:
        sv.close()


@pytest.mark.gpu
def test_page_locked_buffers_are_used_in_place(pg, world):
    """Pair requests whose input and outputs are page-locked skip the staging
    copies and the arena (the kernel reads and writes them over the CPU-GPU
    link); answers are the same as through the staging path."""
    sv = pg.Server(world["g"], [world["bf"], world["kh"]], 64 << 20)
    try:
        sizes = [1, 5, 700, 3000, 20000]
        host = np.concatenate([_pairs(world, P, 900 + i, invalid=(P > 4)) for i, P in enumerate(sizes)])
        offs = np.concatenate([[0], np.cumsum(sizes)])
        pinned = pg.pinned_empty(host.shape, np.int32)
        pinned[...] = host
        peak0 = sv.stats()["arena_used"]
        for est in (pg.EST_BF_AND, pg.EST_KH, pg.EST_EXACT):
            t, cn, jac = sv.submit_pairs_many(pinned, offs, est, pinned=True)
            r = sv.poll_many(t, timeout_us=60_000_000)
            assert (r["status"] == 0).all()
            want = _want_pairs(pg, world, host, est)
            np.testing.assert_array_equal(cn[: offs[-1]], want[0])
            np.testing.assert_array_equal(jac[: offs[-1]], want[1])
            # the same requests through the staging path
            t2, cn2, jac2 = sv.submit_pairs_many(host, offs, est)
            assert (sv.poll_many(t2, timeout_us=60_000_000)["status"] == 0).all()
            np.testing.assert_array_equal(cn2[: offs[-1]], want[0])
        assert sv.stats()["arena_used"] == peak0
    finally:
        sv.close()

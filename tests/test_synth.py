"""The seeded synthetic inputs follow the recipe the design states: simple
undirected CSRs (symmetric, sorted rows, no loops or duplicates), the same
graph for the same seed, Erdos-Renyi mean degree on target, R-MAT degree
skew, the batch mix's size and degree ranges, block-diagonal concatenation,
pair queries half on edges, and BFS balls that grow level by level up to
their edge target."""
import numpy as np
import pytest
import torch

from paper_2208_11469_gb300 import synth


def _check_simple(rp, cl):
    rp, cl = rp.numpy().astype(np.int64), cl.numpy().astype(np.int64)
    n = rp.size - 1
    assert rp[0] == 0 and np.all(np.diff(rp) >= 0) and rp[-1] == cl.size
    src = np.repeat(np.arange(n), np.diff(rp))
    assert np.all((cl >= 0) & (cl < n))
    assert not np.any(cl == src)                                   # no loops
    same_row = src[1:] == src[:-1]
    assert np.all(cl[1:][same_row] > cl[:-1][same_row])            # sorted, no duplicates
    fwd = set(zip(src.tolist(), cl.tolist()))
    assert all((v, u) in fwd for u, v in fwd)                      # symmetric
    return n, cl.size


@pytest.mark.parametrize("gen", [lambda s: synth.rmat(12, 16, seed=s), lambda s: synth.erdos_renyi(3000, 9.0, seed=s)])
def test_simple_and_deterministic(gen):
    rp, cl = gen(5)
    _check_simple(rp, cl)
    rp2, cl2 = gen(5)
    assert torch.equal(rp, rp2) and torch.equal(cl, cl2)
    rp3, cl3 = gen(6)
    assert not (rp3.shape == rp.shape and torch.equal(rp3, rp) and torch.equal(cl3, cl))


def test_erdos_renyi_mean_degree():
    n, d = 4096, 16.0
    degs = []
    for s in range(5):
        rp, cl = synth.erdos_renyi(n, d, seed=s)
        degs.append(cl.numel() / n)
    # M ~ Bin(n(n-1)/2, p): the mean degree 2M/n has standard deviation about sqrt(2 d / n)
    assert abs(np.mean(degs) - d) < 4 * np.sqrt(2 * d / n / len(degs))


def test_rmat_is_skewed():
    rp, cl = synth.rmat(14, 16, seed=1)
    d = np.diff(rp.numpy())
    assert d.max() > 20 * d[d > 0].mean()      # hubs
    assert np.count_nonzero(d == 0) > 0          # and isolated vertices, as R-MAT leaves them


def test_batch_mix_ranges_and_block_diagonal():
    parts = synth.batch_mix(24, seed=3, log2_n=(8, 11))
    assert len(parts) == 24
    for i, (rp, cl) in enumerate(parts):
        n, nnz = _check_simple(rp, cl)
        assert 2**8 <= n < 2**11
        if i % 2 == 0:  # Erdos-Renyi: average degree within the clip range (a few sd of slack)
            assert 2.0 <= nnz / n <= 70.0
    rp, cl, voff = synth.block_diagonal(parts)
    _check_simple(rp, cl)
    assert voff[0] == 0 and voff[-1] == rp.numel() - 1
    r, c = rp.numpy(), cl.numpy()
    for i in range(len(parts)):
        a, b = int(voff[i]), int(voff[i + 1])
        seg = c[r[a]:r[b]]
        assert np.all((seg >= a) & (seg < b))   # rows name only their own graph's vertices
        assert np.array_equal(seg - a, parts[i][1].numpy())


def test_random_pairs_half_on_edges():
    rp, cl = synth.rmat(11, 8, seed=2)
    P = synth.random_pairs(rp.numel() - 1, 4001, 9, rp, cl).numpy()
    assert P.shape == (4001, 2)
    edges = set(zip(np.repeat(np.arange(rp.numel() - 1), np.diff(rp.numpy())).tolist(), cl.numpy().tolist()))
    first = [tuple(p) in edges for p in P[:2000].tolist()]
    assert all(first)                            # the edge half is drawn from CSR entries
    n = rp.numel() - 1
    assert np.all((P >= 0) & (P < n))


def test_bfs_ball_levels_and_target():
    rp, cl = synth.erdos_renyi(2000, 6.0, seed=4)
    r, c = rp.numpy(), cl.numpy()
    for target in (50, 500, 3000):
        S = synth.bfs_ball(rp, cl, 0, target)
        assert S[0] == 0 and len(set(S.tolist())) == len(S)
        inside = np.zeros(r.size - 1, bool)
        inside[S] = True
        src = np.repeat(np.arange(r.size - 1), np.diff(r))
        induced = int(np.count_nonzero(inside[src] & inside[c])) // 2
        # the ball stops at the first prefix reaching the target (or the whole component)
        inside[S[-1]] = False
        before = int(np.count_nonzero(inside[src] & inside[c])) // 2
        assert induced >= target or len(S) == r.size - 1 or before < target
        assert before < target

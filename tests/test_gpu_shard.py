"""The sharded merge tree with the library's S-Merge: every rank count gives
the single-device knnm_merge_tree graph bit for bit (ranks simulated in one
process on this device, transfers through the loopback channel)."""
import numpy as np
import pytest

from paper_1908_00814_gb300 import datagen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as _t
    if not _t.cuda.is_available():
        pytest.skip("no CUDA device")
    return _t


@pytest.mark.parametrize("world", [1, 2, 3, 4])
def test_sharded_tree_equals_single_device_tree(torch, orc, world):
    from paper_1908_00814_gb300 import build, knnm, shard
    build.build()
    ctx = knnm.Context(0)
    rows = [300, 280, 310, 290, 305, 295, 320]   # odd count: a block is carried up
    X = datagen.sift_like(sum(rows), 32, seed=17)
    K = 8
    G = np.concatenate([orc.bruteforce_knn(X[o:o + r], K)[0]
                        for o, r in zip(np.cumsum([0] + rows[:-1]), rows)])
    Xd = torch.from_numpy(X).cuda()
    Gd = torch.from_numpy(G).cuda()
    p = knnm.params(k=K, precision="bf16", max_iters=5, delta=0.0, seed=21)
    want_i, want_d, _ = ctx.merge_tree(Xd, rows, Gd, p)
    got_i, got_d = shard.simulate(ctx, Xd, Gd, rows, p, world)
    assert np.array_equal(got_i.cpu().numpy(), want_i.cpu().numpy())
    assert np.array_equal(got_d.cpu().numpy().view(np.uint32), want_d.cpu().numpy().view(np.uint32))
    ctx.close()


@pytest.mark.parametrize("precision,gen", [("fp32", "gmm"), ("bf16", "sift")])
@pytest.mark.parametrize("world", [1, 2, 3, 4])
def test_sharded_smerge_equals_single_device_merge(torch, orc, world, precision, gen):
    """Sharded S-Merge (replicated sampling, each rank's local join over its own
    node range, partial lists unioned by their owners) on the library's step
    calls, ranks simulated in lock-step on this device: the graph and c_t per
    round equal knnm_merge_symmetric's, and the oracle's."""
    from paper_1908_00814_gb300 import build, knnm, shard
    build.build()
    ctx = knnm.Context(0)
    n1, n2, d, K = 1400, 1300, 32, 10
    X = (datagen.sift_like(n1 + n2, d, n_centres=24, seed=5) if gen == "sift"
         else datagen.gaussian_mixture(n1 + n2, d, n_comp=8, seed=5))
    G1, _ = orc.bruteforce_knn(X[:n1], K)
    G2, _ = orc.bruteforce_knn(X[n1:], K)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    p = knnm.params(k=K, precision=precision, max_iters=7, delta=0.0, seed=13)
    want_i, want_d, want_st = ctx.merge_symmetric(dev(X[:n1]), dev(G1), dev(X[n1:]), dev(G2), p)
    steps = [shard.LibraryRounds(ctx, dev(X[:n1]), dev(G1), dev(X[n1:]), dev(G2), p)
             for _ in range(world)]
    ids, dists, hist = shard.simulate_smerge(steps, n1 + n2, p, world)
    assert hist == want_st["updates"]
    assert np.array_equal(ids.cpu().numpy(), want_i.cpu().numpy())
    assert np.array_equal(dists.cpu().numpy().view(np.uint32),
                          want_d.cpu().numpy().view(np.uint32))
    ref_i, _, _ = orc.merge_symmetric(X[:n1], G1, X[n1:], G2, K, max_iters=7, seed=13)
    assert np.array_equal(ids.cpu().numpy(), ref_i)
    ctx.close()


def test_join_rows_ranges_add_up_to_the_full_join(torch, orc):
    """The union of the per-range joins' partial lists equals the full-range
    step join (lists, flags and c_t), for ranges that split the nodes."""
    from paper_1908_00814_gb300 import build, knnm
    build.build()
    ctx = knnm.Context(0)
    X = datagen.gaussian_mixture(1500, 16, n_comp=6, seed=2)
    n1, K = 800, 8
    G1, _ = orc.bruteforce_knn(X[:n1], K)
    G2, _ = orc.bruteforce_knn(X[n1:], K)
    Xd = torch.from_numpy(X).cuda()
    p = knnm.params(k=K, max_iters=3, seed=4)
    s = knnm.list_widths(p, knnm.SYMMETRIC, n1)[2]
    ids, dists, flags, _, _ = ctx.step_init(knnm.SYMMETRIC, Xd, n1, torch.from_numpy(G1).cuda(),
                                            torch.from_numpy(G2).cuda(), p)
    cands = ctx.step_sample(ids, dists, flags, 4, 1, s)
    start = (ids.clone(), dists.clone(), flags.clone())
    full = [a.clone() for a in start]
    c_full, ev_full = ctx.step_join(knnm.SYMMETRIC, Xd, n1, p, *full, cands)
    cuts = [0, 1, 377, 900, 1499, 1500]
    parts_i, parts_d, evals = [], [], 0
    for lo, hi in zip(cuts, cuts[1:]):
        part = [a.clone() for a in start]
        _, ev = ctx.step_join_rows(knnm.SYMMETRIC, Xd, n1, p, *part, cands, lo, hi)
        evals += ev
        parts_i.append(part[0])
        parts_d.append(part[1])
    oi, od, of, c = ctx.step_union(torch.stack(parts_i), torch.stack(parts_d), *start)
    assert evals == ev_full and c == c_full
    assert torch.equal(oi, full[0]) and torch.equal(od.view(torch.int32), full[1].view(torch.int32))
    assert torch.equal(of, full[2])
    with pytest.raises(knnm.KnnmError):
        ctx.step_join_rows(knnm.SYMMETRIC, Xd, n1, p, *[a.clone() for a in start], cands, 5, 4)
    ctx.close()

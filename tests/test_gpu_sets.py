"""Jaccard merges of itemsets (the Kosarak metric of Sec. 5) through the C ABI:
CSR set rows on the device, the oracle on the same sets as 0/1 rows.  Ids,
distances and per-round counters must be identical."""
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


@pytest.fixture(scope="module")
def km(torch):
    from paper_1908_00814_gb300 import build, knnm
    build.build()
    return knnm


@pytest.fixture(scope="module")
def ctx(km):
    return km.Context(0)


def cuda(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def same_bits(a, b):
    a, b = np.asarray(a), np.asarray(b)
    if a.dtype == np.float32:
        return a.shape == b.shape and np.array_equal(a.view(np.uint32), b.view(np.uint32))
    return a.shape == b.shape and np.array_equal(a, b)


def sets(n, dim, seed, empty=()):
    off, items = datagen.itemsets(n, dim, n_types=max(8, n // 15), core=30, mean_len=12.0,
                                  seed=seed)
    if empty:   # make some rows empty sets
        lens = np.diff(off)
        keep = np.ones(len(items), bool)
        for r in empty:
            keep[off[r]:off[r + 1]] = False
            lens[r] = 0
        items = items[keep]
        off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    return off, items, datagen.sets_to_rows(off, items, dim)


def test_build_sets_matches_oracle(torch, km, ctx, orc):
    off, items, X = sets(1400, 2500, seed=3, empty=(5, 700))
    K = 10
    want_i, want_d, want_st = orc.build_graph(X, K, metric=orc.JACCARD, max_iters=6, delta=0.0,
                                              seed=4)
    p = km.params(k=K, metric="jaccard", max_iters=6, delta=0.0, seed=4)
    ids, dists, st = ctx.build_sets(cuda(torch, off), cuda(torch, items), p)
    assert st["updates"] == want_st["updates"] and st["dist_evals"] == want_st["dist_evals"]
    assert same_bits(ids.cpu().numpy(), want_i)
    assert same_bits(dists.cpu().numpy(), want_d)


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_merge_symmetric_sets_matches_oracle(torch, km, ctx, orc, precision):
    off, items, X = sets(1500, 3000, seed=5)
    n1, K = 800, 12
    G1, _ = orc.bruteforce_knn(X[:n1], K, metric=orc.JACCARD)
    G2, _ = orc.bruteforce_knn(X[n1:], K, metric=orc.JACCARD)
    want_i, want_d, want_st = orc.merge_symmetric(X[:n1], G1, X[n1:], G2, K, metric=orc.JACCARD,
                                                  max_iters=5, delta=0.0, seed=7)
    p = km.params(k=K, metric="jaccard", precision=precision, max_iters=5, delta=0.0, seed=7)
    ids, dists, st = ctx.merge_symmetric_sets(cuda(torch, off), cuda(torch, items), n1,
                                              cuda(torch, G1), cuda(torch, G2), p)
    assert st["updates"] == want_st["updates"] and st["dist_evals"] == want_st["dist_evals"]
    assert same_bits(ids.cpu().numpy(), want_i)
    assert same_bits(dists.cpu().numpy(), want_d)


def test_merge_joint_sets_matches_oracle(torch, km, ctx, orc):
    off, items, X = sets(1300, 2000, seed=9, empty=(1000,))
    n1, K = 700, 8
    G1, _ = orc.bruteforce_knn(X[:n1], K, metric=orc.JACCARD)
    want_i, want_d, _ = orc.merge_joint(X[:n1], G1, X[n1:], K, metric=orc.JACCARD,
                                        max_iters=5, delta=0.0, seed=2)
    p = km.params(k=K, metric="jaccard", max_iters=5, delta=0.0, seed=2)
    ids, dists, _ = ctx.merge_joint_sets(cuda(torch, off), cuda(torch, items), n1,
                                         cuda(torch, G1), p)
    assert same_bits(ids.cpu().numpy(), want_i)
    assert same_bits(dists.cpu().numpy(), want_d)


def test_malformed_sets_and_metric_mismatch(torch, km, ctx, orc):
    off, items, X = sets(300, 500, seed=1)
    p = km.params(k=6, metric="jaccard", max_iters=2)
    bad = items.copy()
    r = 40
    if off[r + 1] - off[r] >= 2:
        bad[off[r]], bad[off[r] + 1] = bad[off[r] + 1], bad[off[r]]   # out of order
        with pytest.raises(km.KnnmError) as e:
            ctx.build_sets(cuda(torch, off), cuda(torch, bad), p)
        assert f"row {r}" in str(e.value)
    o2 = off.copy()
    o2[100] = o2[101] + 1    # decreasing offsets
    with pytest.raises(km.KnnmError):
        ctx.build_sets(cuda(torch, o2), cuda(torch, items), p)
    o3 = off.copy()
    o3[-1] += 5              # beyond the items
    with pytest.raises(km.KnnmError):
        ctx.build_sets(cuda(torch, o3), cuda(torch, items), p)
    with pytest.raises(km.KnnmError):   # Jaccard needs set rows
        ctx.build(cuda(torch, X), p)
    with pytest.raises(km.KnnmError):   # set rows need Jaccard
        ctx.build_sets(cuda(torch, off), cuda(torch, items), km.params(k=6, metric="l2"))
    ctx.build_sets(cuda(torch, off), cuda(torch, items), p)   # still usable

"""Pins of the oracle's H-Merge pieces (Sec. 3.3): the visiting order and the
hierarchy itself."""
import numpy as np
import pytest

from paper_1908_00814_gb300 import datagen


@pytest.mark.parametrize("n", [1, 2, 3, 5, 17, 64, 65, 1000, 4097])
def test_permute_is_a_bijection(orc, n):
    p = orc.permute(n, 11)
    assert sorted(p.tolist()) == list(range(n))
    assert np.array_equal(p, orc.permute(n, 11))


def test_permute_depends_on_the_seed(orc):
    a, b = orc.permute(1000, 1), orc.permute(1000, 2)
    assert not np.array_equal(a, b)
    # no fixed structure: positions and rows are not strongly correlated
    assert abs(np.corrcoef(np.arange(1000), a)[0, 1]) < 0.2


def test_permute_follows_the_feistel_definition(orc):
    """Recompute the order from the definition with the pinned hash."""
    n, seed = 300, 7
    b = 2
    while (1 << b) < n:
        b += 2
    half, mask = b // 2, (1 << (b // 2)) - 1

    def F(x):
        L, R = x >> half, x & mask
        for r in range(4):
            L, R = R, L ^ (orc.hash64(seed, r, 7, R, 0) & mask)
        return (L << half) | R

    want = []
    for i in range(n):
        y = F(i)
        while y >= n:
            y = F(y)
        want.append(y)
    assert orc.permute(n, seed).tolist() == want


def test_hmerge_layers_and_bottom_graph(orc):
    X = datagen.sift_like(3000, 16, seed=5)
    K, first = 10, 90
    perm, layers, ids, dists = orc.hmerge(X, K, first, max_iters=8, seed=2)
    assert np.array_equal(layers[len(X)], ids)
    sizes = sorted(layers)
    assert sizes[0] == first and sizes[-1] == len(X)
    assert all(b == 2 * a for a, b in zip(sizes[:-2], sizes[1:-1]))
    for m in sizes:
        L = layers[m]
        w = K if m == len(X) else K // 2
        assert L.shape == (m, w)
        assert (L >= 0).all() and (L < m).all()
        assert not (L == np.arange(m)[:, None]).any()
        assert all(len(set(r)) == w for r in L.tolist())
    # the bottom graph, in the visiting order, is close to the exact one (an id
    # counts when its distance is within the exact k-th one: ties count)
    Xp = X[perm]
    _, exd = orc.bruteforce_knn(Xp, K)
    hits = sum(int((dists[i] <= exd[i, K - 1]).sum()) for i in range(len(X)))
    assert hits / (len(X) * K) >= 0.95
    # each upper layer is the first k/2 entries of a graph built on its rows:
    # a layer's lists are sorted by distance from the row
    for m in sizes[:-1]:
        L = layers[m]
        for i in range(0, m, max(1, m // 20)):
            d = [orc.distance(0, Xp[i], Xp[j]) for j in L[i]]
            assert d == sorted(d)

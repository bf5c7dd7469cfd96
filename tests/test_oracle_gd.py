"""Pins of the oracle's graph diversification (Alg. 3) and of the top-down
search on the hierarchy (Sec. 3.4): hand-traced examples, closed forms on
lines and grids, and exact search where the graph leaves no choice."""
import json
import os

import numpy as np
import pytest

from paper_1908_00814_gb300 import datagen

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "gd_hand_examples.json")


def complete_lists(n):
    return np.array([[j for j in range(n) if j != i] for i in range(n)], np.int32)


def test_hand_traced_examples(orc):
    cases = json.load(open(GOLDEN))["cases"]
    for c in cases:
        X = np.array(c["points"], np.float32)
        n, K = len(X), c["k"]
        G, _ = orc.bruteforce_knn(X, K)
        ids, dists, deg, _ = orc.diversify(X, G, max_degree=4)
        for i in range(n):
            assert deg[i] == len(c["want_ids"][i]), (c["name"], i)
            assert ids[i, :deg[i]].tolist() == c["want_ids"][i], (c["name"], i)
            assert dists[i, :deg[i]].tolist() == c["want_dists"][i], (c["name"], i)
            assert (ids[i, deg[i]:] == -1).all() and np.isinf(dists[i, deg[i]:]).all()


@pytest.mark.parametrize("K", [2, 4, 6, 9])
def test_points_on_a_line_keep_one_neighbour_per_side(orc, K):
    """Collinear points: a candidate beyond a kept neighbour on the same side is
    closer to that neighbour than to the row, so each row keeps exactly its
    nearest neighbour on each side."""
    n, d = 60, 8
    pos = np.random.default_rng(3).permutation(n)     # row i sits at position pos[i]
    X = np.zeros((n, d), np.float32)
    X[:, 0] = pos
    at = np.argsort(pos)                                # row at each position
    G, _ = orc.bruteforce_knn(X, K)
    ids, dists, deg, _ = orc.diversify(X, G, max_degree=K + 4)
    for i in range(n):
        p = pos[i]
        want = [int(at[p - 1])] if p > 0 else []
        want += [int(at[p + 1])] if p < n - 1 else []
        want.sort()                                     # both at distance 1: id order
        assert ids[i, :deg[i]].tolist() == want
        assert (dists[i, :deg[i]] == 1.0).all()


def test_grid_keeps_the_four_axis_neighbours(orc):
    """Integer grid, k = 8: an inner point's list is its 4 axis neighbours
    (distance 1) and 4 diagonal ones (distance 2); every diagonal one is closer
    to an axis neighbour (1) than to the point, so the four axis ones remain.
    Reverse lists bring nothing more: any other row listing the point is at
    distance >= 4 and within distance 1 of a kept axis neighbour."""
    side, K = 12, 8
    xy = np.array([(x, y) for x in range(side) for y in range(side)], np.float32)
    G, _ = orc.bruteforce_knn(xy, K)
    ids, dists, deg, _ = orc.diversify(xy, G, max_degree=16)
    for i, (x, y) in enumerate(xy.astype(int)):
        if not (0 < x < side - 1 and 0 < y < side - 1):
            continue
        want = sorted([(x - 1) * side + y, (x + 1) * side + y, x * side + y - 1,
                       x * side + y + 1])
        assert deg[i] == 4 and ids[i, :4].tolist() == want and (dists[i, :4] == 1).all()


def test_rule_invariants_on_clustered_data(orc):
    """What Alg. 3 guarantees, checked with float64 recomputation on integer
    data (exact in float32): each output row is sorted, repeat-free and a subset
    of the row's list and reverse list; the nearest entry of each list is kept;
    and every dropped entry of either list has an earlier kept entry of the same
    list that is closer to it than the row is."""
    X = np.round(datagen.gaussian_mixture(400, 8, n_comp=6, seed=4) * 4).astype(np.float32)
    K = 10
    G, _ = orc.bruteforce_knn(X, K)
    ids, dists, deg, _ = orc.diversify(X, G, max_degree=64)
    assert deg.max() < 64
    X64 = X.astype(np.float64)
    rev = [set() for _ in range(len(X))]
    for b in range(len(X)):
        for a in G[b]:
            rev[a].add(b)

    def d2(i, j):
        return float(((X64[i] - X64[j]) ** 2).sum())
    dropped = 0
    for a in range(len(X)):
        row = ids[a, :deg[a]].tolist()
        assert len(set(row)) == len(row) and a not in row
        assert set(row) <= set(G[a].tolist()) | rev[a]
        keys = [(d2(a, v), v) for v in row]
        assert keys == sorted(keys)
        assert [dists[a, j] for j in range(deg[a])] == [np.float32(k[0]) for k in keys]
        for lst in (G[a].tolist(), sorted(rev[a])):
            if not lst:
                continue
            lk = sorted((d2(a, v), v) for v in lst)
            assert lk[0][1] in row
            for i, (dv, v) in enumerate(lk):
                if v in row:
                    continue
                dropped += 1
                assert any(c in row and d2(v, c) < dv for _, c in lk[:i])
    assert dropped > 1000


def test_degree_cut_is_a_prefix_and_rows_subset_agrees(orc):
    X = datagen.gaussian_mixture(500, 16, n_comp=5, seed=8)
    G, _ = orc.bruteforce_knn(X, 12)
    big = orc.diversify(X, G, max_degree=40)
    for m in (1, 3, 6):
        small = orc.diversify(X, G, max_degree=m)
        assert np.array_equal(small[2], np.minimum(big[2], m))
        assert np.array_equal(small[0], big[0][:, :m])
        assert np.array_equal(small[1], big[1][:, :m])
    rows = np.array([499, 0, 17, 250, 17])
    sub = orc.diversify(X, G, max_degree=40, rows=rows)
    assert np.array_equal(sub[0], big[0][rows]) and np.array_equal(sub[2], big[2][rows])


def test_malformed_graph_is_rejected(orc):
    X = datagen.gaussian_mixture(50, 4, seed=1)
    G, _ = orc.bruteforce_knn(X, 4)
    for bad in (50, -1):
        H = G.copy()
        H[3, 1] = bad
        with pytest.raises(RuntimeError):
            orc.diversify(X, H, 8)
    H = G.copy()
    H[7, 2] = H[7, 0]
    with pytest.raises(RuntimeError):
        orc.diversify(X, H, 8)
    H = G.copy()
    H[9, 0] = 9
    with pytest.raises(RuntimeError):
        orc.diversify(X, H, 8)


# ---------------------------------------------------------------- search

def exact_topk(X, Q, k):
    """(distance, id) order of squared l2 in float64 (exact for integer data)."""
    D = ((Q.astype(np.float64)[:, None, :] - X.astype(np.float64)[None]) ** 2).sum(-1)
    out = []
    for q in range(len(Q)):
        order = sorted(range(len(X)), key=lambda j: (D[q, j], j))[:k]
        out.append(order)
    return np.array(out), D


def test_search_on_a_complete_graph_is_exact(orc):
    rng = np.random.default_rng(5)
    X = rng.integers(-20, 20, size=(120, 6)).astype(np.float32)
    Q = rng.integers(-20, 20, size=(30, 6)).astype(np.float32)
    want, D = exact_topk(X, Q, 10)
    ids, dists, ev = orc.search(X, [complete_lists(120)], Q, ef=10, k_out=10, seed=3)
    assert np.array_equal(ids, want)
    assert np.array_equal(dists, np.take_along_axis(D, want, 1).astype(np.float32))
    # the first expansion meets every row once: 1 (start) + 119 comparisons
    assert (ev == 120).all()


def test_search_with_ef_at_least_n_on_a_connected_graph_is_exact(orc):
    rng = np.random.default_rng(6)
    X = rng.integers(0, 30, size=(300, 4)).astype(np.float32)
    Q = rng.integers(0, 30, size=(20, 4)).astype(np.float32)
    G, _ = orc.bruteforce_knn(X, 8)
    import scipy.sparse as sp
    import scipy.sparse.csgraph as cg
    A = sp.csr_matrix((np.ones(G.size), (np.repeat(np.arange(300), 8), G.ravel())), (300, 300))
    assert cg.connected_components(A, directed=True, connection="strong")[0] == 1
    want, _ = exact_topk(X, Q, 5)
    ids, _, ev = orc.search(X, [G], Q, ef=300, k_out=5, seed=1)
    assert np.array_equal(ids, want)
    assert (ev == 300).all()                       # every row compared exactly once


def test_greedy_on_a_line_reaches_the_nearest_point(orc):
    """Rows at positions 0..n-1 of a line, each linked to its neighbours at
    +-1: with ef = 1 the bottom search is pure hill-climbing and must stop at
    the integer nearest to the query; with a coarse top layer (even positions,
    linked at +-2) the descent ends at the same row."""
    n, d = 101, 4
    X = np.zeros((n, d), np.float32)
    order = np.concatenate([np.arange(0, n, 2), np.arange(1, n, 2)])  # evens first
    X[:, 0] = order
    row_at = np.argsort(order)
    G = np.full((n, 2), -1, np.int32)
    for r, p in enumerate(order):
        G[r] = [row_at[p - 1] if p > 0 else -1, row_at[p + 1] if p < n - 1 else -1]
    ne = (n + 1) // 2
    top = np.full((ne, 2), -1, np.int32)
    for r in range(ne):
        p = order[r]
        top[r] = [row_at[p - 2] if p >= 2 else -1, row_at[p + 2] if p + 2 < n else -1]
    rng = np.random.default_rng(2)
    qpos = rng.uniform(-5, n + 5, 200)
    qpos = qpos[np.abs(qpos - np.round(qpos)) > 0.01]   # no ties at half-integers
    Q = np.zeros((len(qpos), d), np.float32)
    Q[:, 0] = qpos
    want = row_at[np.clip(np.round(qpos), 0, n - 1).astype(int)]
    for layers in ([G], [top, G]):
        ids, _, _ = orc.search(X, layers, Q, ef=1, k_out=1, seed=9)
        assert np.array_equal(ids[:, 0], want)


def test_search_start_follows_the_hash(orc):
    """With k_out = ef = 1 on a graph without edges the result is the start row."""
    X = datagen.gaussian_mixture(77, 8, seed=2)
    empty = np.full((77, 3), -1, np.int32)
    Q = X[:10] + 0.5
    ids, _, ev = orc.search(X, [empty], Q, ef=1, k_out=1, seed=42)
    want = [orc.hash64(42, 0, 9, q, 0) % 77 for q in range(10)]
    assert ids[:, 0].tolist() == want and (ev == 1).all()

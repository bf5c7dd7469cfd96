"""Pins for the oracle's primitives: distance m(.,.), the hash, UpdateNN order.

Each test checks the oracle against something other than itself: exact
integer arithmetic, a float64 recomputation within the FP32 error bound, the
published SplitMix64 output sequence, or a value worked out by hand.
"""
import json
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
M64 = (1 << 64) - 1


def test_splitmix64_published_vectors(orc):
    """The mixing step is SplitMix64's: its generator reproduces the published outputs."""
    cases = json.load(open(os.path.join(GOLDEN, "splitmix64_vectors.json")))["cases"]
    for c in cases:
        assert orc.splitmix64(c["seed"], len(c["outputs"])) == c["outputs"]


def test_hash_is_chained_splitmix(orc):
    """H(seed,t,stream,owner,member): five SplitMix64 steps, each absorbing one
    word by xor; a step is the first output of a generator seeded with the word."""
    def step(z):
        return orc.splitmix64(z & M64, 1)[0]
    rng = np.random.default_rng(5)
    for _ in range(20):
        w = [int(x) for x in rng.integers(0, 2**63, size=5)]
        h = step(w[0])
        for x in w[1:]:
            h = step(h ^ x)
        assert orc.hash64(*w) == h
    # distinct counters give distinct values (no accidental word drop)
    base = orc.hash64(0, 1, 0, 7, 9)
    assert len({base, orc.hash64(0, 2, 0, 7, 9), orc.hash64(0, 1, 1, 7, 9),
                orc.hash64(0, 1, 0, 8, 9), orc.hash64(0, 1, 0, 7, 10),
                orc.hash64(1, 1, 0, 7, 9)}) == 6
    # owner and member are not interchangeable
    assert orc.hash64(0, 1, 0, 7, 9) != orc.hash64(0, 1, 0, 9, 7)


@pytest.mark.parametrize("d", [1, 7, 37, 128])
def test_distance_exact_on_small_integers(orc, d):
    """With small integers every partial sum is exact in FP32, so the canonical
    distance equals the exact integer value of each metric's definition."""
    rng = np.random.default_rng(d)
    for _ in range(10):
        a = rng.integers(-50, 51, size=d)
        b = rng.integers(-50, 51, size=d)
        assert orc.distance(orc.L2, a, b) == float(((a - b) ** 2).sum())
        assert orc.distance(orc.L1, a, b) == float(np.abs(a - b).sum())
        assert orc.distance(orc.IP, a, b) == float(-(a * b).sum())


def test_distance_accumulates_in_index_order(orc):
    """Sequential FP32 accumulation in dimension order (round to nearest even):
    2^24 + 1 + 1 + 1 + 1 stays 2^24, whereas any other order would reach 2^24 + 4."""
    a = np.array([4096.0, 1, 1, 1, 1], np.float32)
    b = np.zeros(5, np.float32)
    assert orc.distance(orc.L2, a, b) == 16777216.0
    a1 = np.array([16777216.0, 1, 1, 1, 1], np.float32)
    assert orc.distance(orc.L1, a1, b) == 16777216.0
    # reversed order does reach 2^24 + 4: the order is what decides it
    assert orc.distance(orc.L2, a[::-1].copy(), b) == 16777220.0


@pytest.mark.parametrize("metric", ["L2", "IP", "COS", "L1"])
def test_distance_close_to_float64(orc, metric):
    """Within the sequential-summation error bound of d+2 units of 2^-24 times
    the sum of absolute terms."""
    m = getattr(orc, metric)
    rng = np.random.default_rng(11)
    d = 96
    u = 2.0 ** -24
    for _ in range(50):
        a = rng.standard_normal(d).astype(np.float32)
        b = rng.standard_normal(d).astype(np.float32)
        A, B = a.astype(np.float64), b.astype(np.float64)
        got = float(orc.distance(m, a, b))
        if metric == "L2":
            ref, scale = ((A - B) ** 2).sum(), ((A - B) ** 2).sum()
        elif metric == "L1":
            ref, scale = np.abs(A - B).sum(), np.abs(A - B).sum()
        elif metric == "IP":
            ref, scale = -(A * B).sum(), np.abs(A * B).sum()
        else:
            na, nb = np.linalg.norm(A), np.linalg.norm(B)
            ref, scale = 1 - (A * B).sum() / (na * nb), np.abs(A * B).sum() / (na * nb) + 1
        assert abs(got - ref) <= (d + 4) * u * scale * 1.01


def test_distance_bit_symmetric(orc):
    rng = np.random.default_rng(3)
    for m in (orc.L2, orc.IP, orc.COS, orc.L1):
        for _ in range(20):
            a = rng.standard_normal(33).astype(np.float32)
            b = rng.standard_normal(33).astype(np.float32)
            assert orc.distance(m, a, b).tobytes() == orc.distance(m, b, a).tobytes()


def test_cosine_special_cases(orc):
    z = np.zeros(8, np.float32)
    a = np.arange(1, 9, dtype=np.float32)
    assert orc.distance(orc.COS, z, a) == 1.0          # zero norm reads as orthogonal
    assert orc.distance(orc.COS, a, 3 * a) <= 1e-6     # parallel
    assert abs(orc.distance(orc.COS, a, -a) - 2.0) <= 1e-6
    # no negative zero from 0 - dot
    assert np.signbit(orc.distance(orc.IP, z, a)) == np.False_


def test_bruteforce_knn_matches_float64_sort(orc):
    """Exact k-NN of the oracle vs a float64 argsort (no near ties in this draw)."""
    rng = np.random.default_rng(0)
    X = rng.standard_normal((300, 12)).astype(np.float32)
    K = 8
    ids, dists = orc.bruteforce_knn(X, K)
    X64 = X.astype(np.float64)
    D = ((X64[:, None, :] - X64[None, :, :]) ** 2).sum(-1)
    np.fill_diagonal(D, np.inf)
    ref = np.argsort(D, axis=1, kind="stable")[:, :K]
    assert np.array_equal(ids, ref)
    assert np.allclose(dists, np.take_along_axis(D, ref, 1), rtol=1e-5)
    # L1 as well
    ids1, _ = orc.bruteforce_knn(X, K, metric=orc.L1)
    D1 = np.abs(X64[:, None, :] - X64[None, :, :]).sum(-1)
    np.fill_diagonal(D1, np.inf)
    assert np.array_equal(ids1, np.argsort(D1, axis=1, kind="stable")[:, :K])


def test_bruteforce_ties_break_by_smaller_id(orc):
    X = np.array([[0.0], [1.0], [-1.0], [2.0], [-2.0]], np.float32)
    ids, d = orc.bruteforce_knn(X, 4)
    assert ids[0].tolist() == [1, 2, 3, 4]
    assert d[0].tolist() == [1.0, 1.0, 4.0, 4.0]


def test_exact_knn_f64_helper_matches_direct(orc):
    rng = np.random.default_rng(1)
    X = rng.standard_normal((400, 10)).astype(np.float32)
    q = np.arange(0, 400, 7)
    for metric in (orc.L2, orc.L1, orc.COS, orc.IP):
        ids, dd = orc.exact_knn_f64(X, q, 5, metric=metric, block=16)
        full = orc.distances_f64(metric, X, q, np.tile(np.arange(400), (len(q), 1)))
        full[np.arange(len(q)), q] = np.inf
        ref = np.argsort(full, axis=1, kind="stable")[:, :5]
        assert np.array_equal(ids, ref)
        assert np.allclose(dd, np.take_along_axis(full, ref, 1))


def test_chi_square_hand_values(orc):
    """Chi-square distance (the NUSWide metric of Sec. 5): the sum over t of
    (a_t - b_t)^2 / (a_t + b_t), a term with a_t + b_t = 0 counting 0."""
    f = lambda a, b: float(orc.distance(orc.CHI2, np.array(a, np.float32), np.array(b, np.float32)))
    assert f([1, 0, 3, 2], [3, 0, 1, 2]) == 2.0        # 4/4 + 0 + 4/4 + 0/4
    assert f([1, 2], [0, 0]) == 3.0                    # 1/1 + 4/2
    assert f([0, 0, 0], [0, 0, 0]) == 0.0
    assert f([4, 0, 9], [4, 0, 9]) == 0.0
    # pairs whose terms are exact: the sum is exact
    rng = np.random.default_rng(1)
    pairs = [(1, 3, 1.0), (2, 2, 0.0), (0, 0, 0.0), (1, 0, 1.0), (4, 0, 4.0), (3, 1, 1.0),
             (0, 8, 8.0), (5, 3, 0.5)]
    for _ in range(20):
        pick = [pairs[i] for i in rng.integers(0, len(pairs), size=40)]
        a = [p[0] for p in pick]
        b = [p[1] for p in pick]
        assert f(a, b) == sum(p[2] for p in pick)


def test_chi_square_close_to_float64_and_symmetric(orc):
    rng = np.random.default_rng(7)
    u = 2.0 ** -24
    for d in (5, 64, 500):
        for _ in range(20):
            a = rng.gamma(0.5, 3.0, size=d).astype(np.float32)   # sparse-ish histograms
            b = rng.gamma(0.5, 3.0, size=d).astype(np.float32)
            a[rng.random(d) < 0.3] = 0.0
            b[rng.random(d) < 0.3] = 0.0
            A, B = a.astype(np.float64), b.astype(np.float64)
            S = A + B
            terms = np.where(S == 0, 0.0, (A - B) ** 2 / np.where(S == 0, 1.0, S))
            got = orc.distance(orc.CHI2, a, b)
            assert abs(float(got) - terms.sum()) <= (d + 8) * u * terms.sum() * 1.01
            assert got.tobytes() == orc.distance(orc.CHI2, b, a).tobytes()


def test_chi_square_bruteforce_knn_matches_float64(orc):
    rng = np.random.default_rng(9)
    X = rng.poisson(1.5, size=(300, 24)).astype(np.float32)
    ids, dists = orc.bruteforce_knn(X, 8, metric=orc.CHI2)
    X64 = X.astype(np.float64)
    for i in range(0, 300, 7):
        S = X64[i] + X64
        T = np.where(S == 0, 0.0, (X64[i] - X64) ** 2 / np.where(S == 0, 1.0, S)).sum(1)
        T[i] = np.inf
        want = np.sort(T)[:8]
        assert np.allclose(dists[i], want, rtol=1e-5, atol=1e-6)
        assert np.allclose(T[ids[i]], want, rtol=1e-5, atol=1e-6)


def _sets_to_rows(sets, dim):
    X = np.zeros((len(sets), dim), np.float32)
    for i, s in enumerate(sets):
        X[i, list(s)] = 1.0
    return X


def test_jaccard_definition(orc):
    """Jaccard distance of Kosarak's itemsets (Sec. 5): 1 - |A n B| / |A u B|,
    computed by the oracle on 0/1 rows; checked against Python sets."""
    rng = np.random.default_rng(5)
    dim = 300
    sets = [set(rng.choice(dim, size=int(rng.integers(0, 40)), replace=False).tolist())
            for _ in range(60)]
    sets[0] = set()
    sets[1] = set()
    X = _sets_to_rows(sets, dim)
    for i in range(60):
        for j in range(0, 60, 7):
            a, b = sets[i], sets[j]
            u = len(a | b)
            want = np.float32(0.0) if u == 0 else np.float32(1.0) - np.float32(len(a & b)) / np.float32(u)
            got = orc.distance(orc.JACCARD, X[i], X[j])
            assert got.tobytes() == want.tobytes(), (i, j)
    assert orc.distance(orc.JACCARD, X[0], X[1]) == 0.0          # two empty sets
    assert orc.distance(orc.JACCARD, X[0], X[2]) == (1.0 if sets[2] else 0.0)
    f = lambda a, b: float(orc.distance(orc.JACCARD, *_sets_to_rows([a, b], 10)))
    assert f({1, 2, 3}, {2, 3, 4}) == np.float32(1.0) - np.float32(2.0) / np.float32(4.0)
    assert f({1}, {2}) == 1.0 and f({5, 6}, {5, 6}) == 0.0

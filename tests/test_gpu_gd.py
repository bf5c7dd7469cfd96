"""Parity of graph diversification (Alg. 3) and of the top-down search on the
hierarchy (Sec. 3.4) with the CPU oracle, through the C ABI.

Both sides compute canonical FP32 distances, so every keep/drop decision and
every search step is taken on the same bits: ids, distances and degrees are
compared bit for bit, and so are the per-query distance counts whenever the
library's visited table never filled."""
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


def data(kind, n, d, seed):
    if kind == "gmm":
        return datagen.gaussian_mixture(n, d, n_comp=12, seed=seed)
    if kind == "norm":
        return datagen.gaussian_mixture(n, d, n_comp=12, seed=seed, normalize=True)
    if kind == "sift":
        return datagen.sift_like(n, d, seed=seed)
    if kind == "bovw":
        return datagen.bovw_like(n, d, n_topics=10, words=3.0 * d, seed=seed)
    if kind == "hub":   # one row at the centre of a thin shell: it is in every list
        rng = np.random.default_rng(seed)
        X = rng.normal(size=(n, d))
        X /= np.linalg.norm(X, axis=1, keepdims=True)
        X *= 1.0 + 0.05 * rng.random((n, 1))
        X[0] = 0.0
        return X.astype(np.float32)
    raise ValueError(kind)


CASES = [
    # (data, n, d, K, metric, max_degree)
    ("gmm", 3001, 32, 16, "l2", 40),
    ("gmm", 2500, 20, 7, "l1", 12),
    ("norm", 2200, 48, 20, "cos", 64),
    ("gmm", 1800, 16, 10, "ip", 30),
    ("sift", 4000, 128, 20, "l2", 48),
    ("hub", 3000, 64, 8, "l2", 256),
    ("gmm", 700, 12, 32, "l2", 1),
    ("gmm", 600, 12, 1, "l2", 5),
    ("gmm", 997, 13, 9, "l2", 9),   # d not a multiple of 4: scalar loads
    ("bovw", 2500, 100, 16, "chi2", 32),
    ("bovw", 1200, 50, 10, "chi2", 20),   # d not a multiple of 4
]


@pytest.mark.parametrize("case", CASES, ids=[f"{c[0]}-{c[1]}-{c[4]}-k{c[3]}-m{c[5]}" for c in CASES])
def test_diversify_matches_oracle(torch, km, ctx, orc, case):
    kind, n, d, K, metric, M = case
    X = data(kind, n, d, seed=n + K)
    mcode = km.METRICS[metric]
    G, _ = orc.bruteforce_knn(X, K, metric=mcode)
    want_i, want_d, want_deg, _ = orc.diversify(X, G, M, metric=mcode)
    ids, dists, deg, st = ctx.diversify(cuda(torch, X), cuda(torch, G), M, metric=metric)
    assert same_bits(deg.cpu().numpy(), want_deg)
    assert same_bits(ids.cpu().numpy(), want_i)
    assert same_bits(dists.cpu().numpy(), want_d)
    assert st["edges"] == int(want_deg.sum())
    assert st["full_rows"] == int((want_deg == M).sum())
    indeg = np.bincount(G.ravel(), minlength=n)
    assert st["max_in_degree"] == int(indeg.max())
    if kind == "hub":
        assert indeg[0] > 1000        # the reverse list of row 0 spans many batches


def test_diversify_on_an_approximate_graph(torch, km, ctx, orc):
    """Input graph from the oracle's own NN-Descent build (not exact lists)."""
    X = datagen.clustered_mixture(5000, 24, n_comp=40, seed=3)
    G, _, _ = orc.build_graph(X, 12, max_iters=4, delta=0.0, seed=5)
    want = orc.diversify(X, G, 24)
    got = ctx.diversify(cuda(torch, X), cuda(torch, G), 24)
    for a, b in zip(got[:3], want[:3]):
        assert same_bits(a.cpu().numpy(), b)


def test_diversify_rejects_malformed_graphs(torch, km, ctx, orc):
    X = datagen.gaussian_mixture(300, 8, seed=1)
    G, _ = orc.bruteforce_knn(X, 6)
    for r, c, v in ((5, 2, 300), (7, 0, -3), (9, 1, 9), (11, 4, None)):
        H = G.copy()
        H[r, c] = H[r, 0] if v is None else v
        if v is None:
            H[r, c] = H[r, 1] if c == 0 else H[r, 0]
        with pytest.raises(km.KnnmError) as e:
            ctx.diversify(cuda(torch, X), cuda(torch, H), 8)
        assert e.value.code == -1 and f"row {r}" in str(e.value)
    with pytest.raises(km.KnnmError):
        ctx.diversify(cuda(torch, X), cuda(torch, G), 0)
    with pytest.raises(km.KnnmError):
        ctx.diversify(cuda(torch, X), cuda(torch, G), 257)
    # the context stays usable
    ctx.diversify(cuda(torch, X), cuda(torch, G), 8)


# ---------------------------------------------------------------- search

@pytest.fixture(scope="module")
def hierarchy(orc):
    """An H-Merge hierarchy made by the oracle, each layer diversified by the
    oracle: (rows in visiting order, [layer lists from the top down])."""
    n, d, K = 12000, 32, 16
    X = datagen.clustered_mixture(n, d, n_comp=60, seed=21)
    perm, layers, ids, _ = orc.hmerge(X, K, first_rows=1500, max_iters=6, delta=0.001, seed=4)
    Xp = np.ascontiguousarray(X[perm])
    out = []
    for m in sorted(layers):
        g = layers[m]
        div, _, _, _ = orc.diversify(Xp[:m], g, 2 * K)
        out.append(div)
    return Xp, out


@pytest.mark.parametrize("ef,k_out", [(10, 10), (48, 10), (200, 20), (1, 1)])
def test_hierarchical_search_matches_oracle(torch, km, ctx, orc, hierarchy, ef, k_out):
    Xp, layers = hierarchy
    Q = datagen.clustered_mixture(700, Xp.shape[1], n_comp=60, seed=21)[-333:] + 0.01
    want_i, want_d, want_ev = orc.search(Xp, layers, Q, ef, k_out, seed=17)
    ids, dists, ev, st = ctx.search(cuda(torch, Xp), [cuda(torch, g) for g in layers],
                                    cuda(torch, Q), ef, k_out, seed=17)
    assert same_bits(ids.cpu().numpy(), want_i)
    assert same_bits(dists.cpu().numpy(), want_d)
    assert st["crowded_queries"] == 0
    assert np.array_equal(ev.cpu().numpy().astype(np.uint64), want_ev)
    assert st["dist_evals"] == int(want_ev.sum())


@pytest.mark.parametrize("metric", ["l2", "l1", "ip", "cos", "chi2"])
@pytest.mark.parametrize("kind", ["float", "int"])
def test_flat_search_matches_oracle(torch, km, ctx, orc, metric, kind):
    """Float rows take the estimate-then-canonical route, small-integer rows the
    exact estimate; both must give the oracle's bits."""
    mcode = km.METRICS[metric]
    if kind == "int":
        X = datagen.sift_like(4000, 32, n_centres=4, seed=8)
        Q = np.concatenate([X[:40], datagen.sift_like(160, 32, n_centres=4, seed=9)])
        Q[-1, 0] += 0.5   # a non-integer query: its pairs take the bounded route
    else:
        X = datagen.gaussian_mixture(5000, 20, n_comp=10, seed=8, normalize=metric == "cos")
        Q = np.concatenate([X[:50], datagen.gaussian_mixture(150, 20, n_comp=10, seed=9,
                                                            normalize=metric == "cos")])
        if metric == "chi2":   # histogram-like: non-negative
            X, Q = np.abs(X), np.abs(Q)
    G, _ = orc.bruteforce_knn(X, 10, metric=mcode)
    want = orc.search(X, [G], Q, 64, 12, metric=mcode, seed=2)
    Xd = cuda(torch, X)
    for aux in (None, ctx.search_prepare(Xd)):
        got = ctx.search(Xd, [cuda(torch, G)], cuda(torch, Q), 64, 12, metric=metric, seed=2,
                         row_aux=aux)
        assert same_bits(got[0].cpu().numpy(), want[0])
        assert same_bits(got[1].cpu().numpy(), want[1])
        assert np.array_equal(got[2].cpu().numpy().astype(np.uint64), want[2])


def test_search_prepare(torch, km, ctx):
    X = datagen.gaussian_mixture(300, 12, seed=3)
    X[:100] = np.round(X[:100] * 10)
    X[100:110] = np.round(X[100:110]) * 1e7    # integers beyond 2^24 count as inexact
    aux = ctx.search_prepare(cuda(torch, X)).cpu().numpy()
    for i in range(300):
        integral = bool((X[i] == np.round(X[i])).all()) and np.abs(X[i]).max() <= 2 ** 24
        assert aux[i, 0] == (np.abs(X[i]).max() if integral else -1.0)
    ref = np.sqrt((X.astype(np.float64) ** 2).sum(1))
    assert np.allclose(aux[:, 1], ref, rtol=1e-5)


def test_crowded_visited_table_keeps_the_result(torch, km, ctx, orc):
    """ef = 1024 on a wide random graph: far more rows are compared than the
    visited table holds, so some rows are compared again; the lists must not
    change."""
    rng = np.random.default_rng(14)
    n = 100000
    X = rng.normal(size=(n, 8)).astype(np.float32)
    G = rng.integers(0, n, size=(n, 128)).astype(np.int32)   # self and repeats allowed
    Q = rng.normal(size=(40, 8)).astype(np.float32)
    want_i, want_d, want_ev = orc.search(X, [G], Q, 1024, 50, seed=3)
    ids, dists, ev, st = ctx.search(cuda(torch, X), [cuda(torch, G)], cuda(torch, Q), 1024, 50,
                                    seed=3)
    assert st["crowded_queries"] > 0
    assert same_bits(ids.cpu().numpy(), want_i)
    assert same_bits(dists.cpu().numpy(), want_d)
    assert (ev.cpu().numpy().astype(np.uint64) >= want_ev).all()


def test_search_edge_cases(torch, km, ctx, orc):
    X = datagen.gaussian_mixture(400, 8, seed=4)
    G, _ = orc.bruteforce_knn(X, 5)
    Xd, Gd = cuda(torch, X), cuda(torch, G)
    # no queries
    ids, dists, ev, st = ctx.search(Xd, [Gd], cuda(torch, X[:0]), 8, 4)
    assert ids.shape == (0, 4) and st["dist_evals"] == 0
    # graph without edges: the start row only, padded
    empty = cuda(torch, np.full((400, 3), -1, np.int32))
    ids, dists, _, _ = ctx.search(Xd, [empty], cuda(torch, X[:5]), 8, 4, seed=6)
    want = orc.search(X, [np.full((400, 3), -1, np.int32)], X[:5], 8, 4, seed=6)
    assert same_bits(ids.cpu().numpy(), want[0]) and (ids.cpu().numpy()[:, 1:] == -1).all()
    assert np.isinf(dists.cpu().numpy()[:, 1:]).all()
    # malformed layers are reported
    bad = G.copy()
    bad[:, 0] = 400
    with pytest.raises(km.KnnmError):
        ctx.search(Xd, [cuda(torch, bad)], cuda(torch, X[:20]), 8, 4)
    top = cuda(torch, np.full((100, 2), 150, np.int32))   # ids beyond the top layer's rows
    with pytest.raises(km.KnnmError):
        ctx.search(Xd, [top, Gd], cuda(torch, X[:20]), 8, 4)
    with pytest.raises(km.KnnmError):                    # bottom must cover all rows
        ctx.search(Xd, [Gd[:300]], cuda(torch, X[:20]), 8, 4)
    with pytest.raises(km.KnnmError):                    # k_out > ef
        ctx.search(Xd, [Gd], cuda(torch, X[:20]), 4, 8)
    # still usable
    ctx.search(Xd, [Gd], cuda(torch, X[:20]), 8, 4)


def test_gather_rows(torch, km, ctx, orc):
    X = datagen.gaussian_mixture(1000, 12, seed=2)
    perm = orc.permute(1000, 5)
    out = ctx.gather_rows(cuda(torch, X), cuda(torch, perm))
    assert same_bits(out.cpu().numpy(), X[perm])
    part = ctx.gather_rows(cuda(torch, X), cuda(torch, perm), n=17)
    assert same_bits(part.cpu().numpy(), X[perm[:17]])
    bad = perm.copy()
    bad[3] = 1000
    with pytest.raises(km.KnnmError):
        ctx.gather_rows(cuda(torch, X), cuda(torch, bad))

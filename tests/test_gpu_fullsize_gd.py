"""Diversification (Alg. 3) and the top-down search (Sec. 3.4) at the size the
benchmark runs them: 1,000,000 SIFT-like rows (d = 128, k = 20), 10,000
queries.

* Parity on sampled rows / queries: the inputs are seeded random graphs made
  here (valid lists, no self, no repeats), so the oracle can recompute any row
  of the diversified graph, and any query of a search, on its own.
* The benchmark's own pipeline (H-Merge hierarchy, every layer diversified,
  search with ef = 64) is checked by properties that hold at any size: sorted
  repeat-free lists drawn from each row's list and reverse list, distances that
  match a float64 recomputation, and recall@10 >= 0.95 of the search.
"""
import numpy as np
import pytest

from paper_1908_00814_gb300 import datagen

pytestmark = pytest.mark.gpu

N, D, K, NQ = 1_000_000, 128, 20, 10_000


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


def random_graph(n, k, seed, limit=None):
    """k distinct ids per row in [0, limit or n), none equal to the row."""
    rng = np.random.default_rng(seed)
    m = n if limit is None else limit
    r = np.sort(rng.integers(0, m - k, size=(n, k)), axis=1) + np.arange(k)
    G = (np.arange(n)[:, None] + 1 + r) % m
    return np.ascontiguousarray(rng.permuted(G, axis=1).astype(np.int32))


@pytest.fixture(scope="module")
def data():
    X = datagen.generate("hsearch_sift_1m_d128_k20", n=N + NQ)
    return np.ascontiguousarray(X[:N]), np.ascontiguousarray(X[N:])


def test_fullsize_diversify_sampled_rows(torch, km, ctx, orc, data):
    X, _ = data
    G = random_graph(N, K, 31)
    ids, dists, deg, st = ctx.diversify(torch.from_numpy(X).cuda(), torch.from_numpy(G).cuda(),
                                        2 * K)
    rows = datagen.sample_nodes(N, 2000, seed=3)
    rows = np.concatenate([rows, [0, N - 1]])
    wi, wd, wdeg, _ = orc.diversify(X, G, 2 * K, rows=rows)
    assert np.array_equal(deg.cpu().numpy()[rows], wdeg)
    assert np.array_equal(ids.cpu().numpy()[rows], wi)
    assert np.array_equal(dists.cpu().numpy()[rows].view(np.uint32), wd.view(np.uint32))
    assert st["max_in_degree"] == int(np.bincount(G.ravel(), minlength=N).max())


def test_fullsize_search_sampled_queries(torch, km, ctx, orc, data):
    X, Q = data
    sizes = [4096, 65536, N]
    layers = [random_graph(m, 12 if m < N else 24, 40 + i) for i, m in enumerate(sizes)]
    ids, dists, ev, st = ctx.search(torch.from_numpy(X).cuda(),
                                    [torch.from_numpy(g).cuda() for g in layers],
                                    torch.from_numpy(Q).cuda(), 64, 10, seed=9)
    qs = datagen.sample_nodes(NQ, 200, seed=4)
    wi, wd, wev = orc.search(X, layers, np.ascontiguousarray(Q[qs]), 64, 10, seed=9,
                             query_index=qs)
    assert np.array_equal(ids.cpu().numpy()[qs], wi)
    assert np.array_equal(dists.cpu().numpy()[qs].view(np.uint32), wd.view(np.uint32))
    got_ev = ev.cpu().numpy()[qs].astype(np.uint64)
    if st["crowded_queries"] == 0:
        assert np.array_equal(got_ev, wev)
    else:   # rows compared again when the visited table filled; results unchanged
        assert (got_ev >= wev).all()


def test_fullsize_pipeline_properties_and_recall(torch, km, ctx, orc, data):
    X, Q = data
    Xd = torch.from_numpy(X).cuda()
    p = km.params(k=K, precision="bf16", max_iters=10, delta=0.001, seed=0)
    keep = [64, 512, 4096, 32768, 262144]
    perm, ids, _, layers, _ = ctx.hmerge(Xd, 64, p, layers=keep)
    Xp = ctx.gather_rows(Xd, torch.from_numpy(perm).cuda())
    assert np.array_equal(Xp.cpu().numpy(), X[perm])
    graphs = [layers[m] for m in keep] + [ids]
    div = []
    for g, cap in zip(graphs, [K] * len(keep) + [2 * K]):
        di, dd, dg, _ = ctx.diversify(Xp[:len(g)], torch.from_numpy(g).cuda(), cap)
        div.append(di)
        # properties on sampled rows: sorted, no repeats, no self, drawn from the
        # row's list and reverse list, distances = float64 recomputation
        m = len(g)
        rows = datagen.sample_nodes(m, min(m, 300), seed=m)
        hi, hd, hg = di.cpu().numpy(), dd.cpu().numpy(), dg.cpu().numpy()
        Xpm = X[perm[:m]].astype(np.float64)
        rev = {int(r): set() for r in rows}
        src = np.nonzero(np.isin(g, rows))
        for b, j in zip(*src):
            rev[int(g[b, j])].add(int(b))
        for r in rows:
            row = hi[r, :hg[r]].tolist()
            assert len(set(row)) == len(row) and r not in row and hg[r] >= 1
            assert set(row) <= set(g[r].tolist()) | rev[int(r)]
            ref = ((Xpm[row] - Xpm[r]) ** 2).sum(1)
            assert np.allclose(hd[r, :hg[r]], ref, rtol=1e-6)
            assert (np.diff(hd[r, :hg[r]]) >= 0).all()
            assert (hi[r, hg[r]:] == -1).all()
    sids, sdist, _, st = ctx.search(Xp, div, torch.from_numpy(Q).cuda(), 64, 10, seed=0)
    # recall@10 against exact float64 neighbours of 500 sampled queries
    qs = datagen.sample_nodes(NQ, 500, seed=8)
    Xt = torch.from_numpy(X[perm]).cuda().double()
    hits = 0
    for q in qs:
        dq = ((Xt - torch.from_numpy(Q[q]).cuda().double()) ** 2).sum(1)
        kth = torch.topk(dq, 10, largest=False).values[-1].item()
        got = sids[q].long()
        hits += int((dq[got] <= kth).sum().item())
    assert hits / (10 * len(qs)) >= 0.95

"""Parity at the full size of the 1M-point workload (2 x 500,000 SIFT-like
vectors, d = 128, k = 20, rho = 0.5), in the launch configuration the
benchmark times.

* init and the sampler are compared with the oracle on every row (both are
  cheap enough on the CPU at this size);
* one local-join round is checked on sampled nodes: the oracle's distance
  function and the paper's UpdateNN rule rebuild each sampled list from the
  candidate sets of every node that lists it;
* the whole merge is checked by properties that hold at any size: BF16+rerank
  and FP32 give the same graph, lists are sorted/unique/self-free, sampled
  distances are the oracle's, and recall@10 >= 0.95 against exact float64
  neighbours on sampled nodes.
"""
import numpy as np
import pytest

from paper_1908_00814_gb300 import datagen

pytestmark = pytest.mark.gpu

WORKLOAD = "smerge_sift_1m_d128_k20"
K = 20
S = 10


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


@pytest.fixture(scope="module")
def data():
    X = datagen.generate(WORKLOAD)
    return X, len(X) // 2


def random_graph(n, k, seed):
    """Valid input lists: k distinct ids per row, no self."""
    rng = np.random.default_rng(seed)
    # sorted draws plus 0..k-1 are strictly increasing: k distinct offsets in [0, n-1)
    r = np.sort(rng.integers(0, n - k, size=(n, k)), axis=1) + np.arange(k)
    G = (np.arange(n)[:, None] + 1 + r) % n
    return np.ascontiguousarray(rng.permuted(G, axis=1).astype(np.int32))


@pytest.fixture(scope="module")
def state(torch, km, ctx, orc, data):
    X, n1 = data
    n = len(X)
    G1 = random_graph(n1, K, 1)
    G2 = random_graph(n - n1, K, 2)
    ref = orc.init(orc.SYMMETRIC, X, n1, K, 10, seed=5, G1=G1, G2=G2)
    Xd = torch.from_numpy(X).cuda()
    got = ctx.step_init(km.SYMMETRIC, Xd, n1, torch.from_numpy(G1).cuda(),
                        torch.from_numpy(G2).cuda(), km.params(k=K, seed=5))
    return X, n1, Xd, ref, got


def test_fullsize_init_all_rows(state):
    X, n1, Xd, ref, got = state
    assert np.array_equal(got[0].cpu().numpy(), ref.ids)
    assert np.array_equal(got[1].cpu().numpy().view(np.uint32), ref.dists.view(np.uint32))
    assert np.array_equal(got[3].cpu().numpy(), ref.rear_ids)


def test_fullsize_sample_and_join(torch, km, ctx, orc, state):
    X, n1, Xd, ref, got = state
    n = len(X)
    st = ref.copy()
    rng = np.random.default_rng(3)
    st.flags[:] = (rng.random(st.flags.shape) < 0.7).astype(np.uint8)
    ids = torch.from_numpy(st.ids).cuda()
    dists = torch.from_numpy(st.dists).cuda()
    flags = torch.from_numpy(st.flags).cuda()
    cands_ref = orc.sample(st, 7, 2, S)
    cands = ctx.step_sample(ids, dists, flags, 7, 2, S)
    assert np.array_equal(flags.cpu().numpy(), st.flags)
    new_ids, new_cnt, old_ids, old_cnt = (c.cpu().numpy() for c in cands)
    assert np.array_equal(new_cnt, cands_ref[1]) and np.array_equal(old_cnt, cands_ref[3])
    cn = np.arange(new_ids.shape[1])[None, :] < new_cnt[:, None]
    co = np.arange(old_ids.shape[1])[None, :] < old_cnt[:, None]
    assert np.array_equal(np.where(cn, new_ids, -1), np.where(cn, cands_ref[0], -1))
    assert np.array_equal(np.where(co, old_ids, -1), np.where(co, cands_ref[2], -1))

    start_ids, start_d, start_f = st.ids.copy(), st.dists.copy(), st.flags.copy()
    for precision in ("bf16", "fp32"):
        i2, d2, f2 = ids.clone(), dists.clone(), flags.clone()
        c, ev = ctx.step_join(km.SYMMETRIC, Xd, n1, km.params(k=K, precision=precision),
                              i2, d2, f2, cands)
        if precision == "bf16":
            bf = (i2.cpu().numpy(), d2.cpu().numpy(), f2.cpu().numpy(), c, ev)
    gi, gd, gf = i2.cpu().numpy(), d2.cpu().numpy(), f2.cpu().numpy()
    assert np.array_equal(bf[0], gi) and np.array_equal(bf[1].view(np.uint32), gd.view(np.uint32))
    assert (bf[3], bf[4]) == (c, ev)

    # rebuild sampled lists from the candidate sets (UpdateNN on both endpoints)
    newm = np.where(cn, new_ids, -1)
    oldm = np.where(co, old_ids, -1)
    for v in datagen.sample_nodes(n, 24, seed=9):
        partners = set()
        for u in np.nonzero((newm == v).any(1))[0]:
            partners |= set(newm[u][newm[u] >= 0].tolist()) | set(oldm[u][oldm[u] >= 0].tolist())
        for u in np.nonzero((oldm == v).any(1))[0]:
            partners |= set(newm[u][newm[u] >= 0].tolist())
        partners.discard(int(v))
        partners = {q for q in partners if (q < n1) != (v < n1)}
        pool = {int(q): float(orc.distance(0, X[v], X[q])) for q in partners}
        for j in range(K):
            pool[int(start_ids[v, j])] = float(start_d[v, j])
        best = sorted(pool.items(), key=lambda kv: (np.float32(kv[1]), kv[0]))[:K]
        assert gi[v].tolist() == [b[0] for b in best], v
        assert np.array_equal(gd[v], np.array([b[1] for b in best], np.float32)), v
        was = dict(zip(start_ids[v].tolist(), start_f[v].tolist()))
        assert gf[v].tolist() == [was.get(b[0], 1) for b in best], v


def test_fullsize_merge_properties_and_recall(torch, km, ctx, orc, data):
    X, n1 = data
    n = len(X)
    Xd = torch.from_numpy(X).cuda()
    S1, S2 = Xd[:n1].contiguous(), Xd[n1:].contiguous()
    bp = km.params(k=K, precision="bf16", max_iters=10, delta=0.001, seed=11)
    G1, _, _ = ctx.build(S1, bp)
    bp.seed = 12
    G2, _, _ = ctx.build(S2, bp)
    outs = {}
    for precision in ("bf16", "fp32"):
        p = km.params(k=K, precision=precision, max_iters=10, delta=0.001, seed=0)
        outs[precision] = ctx.merge_symmetric(S1, G1, S2, G2, p)
    ib, db, sb = outs["bf16"]
    if_, df, sf = outs["fp32"]
    assert torch.equal(ib, if_) and torch.equal(db.view(torch.int32), df.view(torch.int32))
    assert sb["updates"] == sf["updates"] and sb["dist_evals"] == sf["dist_evals"]
    # properties on every row
    assert int(ib.min()) >= 0 and int(ib.max()) < n
    assert not bool((ib == torch.arange(n, device=ib.device)[:, None]).any())
    si = torch.sort(ib, dim=1).values
    assert not bool((si[:, 1:] == si[:, :-1]).any())
    ok = (db[:, :-1] < db[:, 1:]) | ((db[:, :-1] == db[:, 1:]) & (ib[:, :-1] < ib[:, 1:]))
    assert bool(ok.all())
    # sampled distances are the oracle's canonical distances
    ids_h, d_h = ib.cpu().numpy(), db.cpu().numpy()
    for v in datagen.sample_nodes(n, 64, seed=4):
        for j in range(K):
            assert orc.distance(0, X[v], X[ids_h[v, j]]) == d_h[v, j]
    # recall@10 against exact float64 neighbours
    q = datagen.sample_nodes(n, 300, seed=0)
    r = orc.recall_at(X, q, ids_h, 10)
    assert r >= 0.95, r

"""Serving loop (knnm_server_*): J-Merge (Alg. 2) of raw batches into a graph
kept resident on the device, several batches in flight at once.

The checks replay the server's own schedule: each request records which
commits its snapshot contained and where it committed.  Rebuilding every
snapshot from the commits before it, the test runs that request's J-Merge
alone (one library call, nothing else on the device) and through the oracle,
and requires the served result to be identical to both; the resident graph
after draining must equal the fold of all commits.
"""
import numpy as np
import pytest

from paper_1908_00814_gb300 import datagen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


@pytest.fixture(scope="module")
def km(torch):
    from paper_1908_00814_gb300 import build, knnm
    build.build()
    return knnm


def commit(state, full_ids, full_dists, n_snap, K):
    """Plain definition of a commit: batch ids move to the end of the resident
    rows; each snapshot row keeps the first K distinct entries of (resident
    list, result list) in (distance, id) order; batch rows are appended."""
    X, ids, dists = state
    base = ids.shape[0]
    rid = full_ids.astype(np.int64)
    rid = np.where(rid >= n_snap, base + (rid - n_snap), rid).astype(np.int32)
    new_ids = ids.copy()
    new_d = dists.copy()
    for v in range(n_snap):
        cat_i = np.concatenate([ids[v], rid[v]])
        cat_d = np.concatenate([dists[v], full_dists[v]])
        order = np.lexsort((cat_i, cat_d))
        seen, keep = set(), []
        for j in order:
            if int(cat_i[j]) in seen:
                continue
            seen.add(int(cat_i[j]))
            keep.append(j)
            if len(keep) == K:
                break
        new_ids[v] = cat_i[keep]
        new_d[v] = cat_d[keep]
    return new_ids, new_d, rid[n_snap:], full_dists[n_snap:]


CASES = {
    "l2_fp32": dict(metric="l2", precision="fp32", gen="gmm"),
    "l2_bf16_sift": dict(metric="l2", precision="bf16", gen="sift"),
    "cos_bf16": dict(metric="cos", precision="bf16", gen="gmm_norm"),
}


@pytest.mark.parametrize("case", list(CASES))
def test_served_batches_equal_alone_runs_and_oracle(torch, km, orc, case):
    cfg = CASES[case]
    K, d, n0 = 10, 32, 1500
    sizes = [60, 140, 90, 200, 75, 130]
    total = n0 + sum(sizes)
    if cfg["gen"] == "sift":
        X = datagen.sift_like(total, d, seed=91)
    else:
        X = datagen.gaussian_mixture(total, d, n_comp=8, seed=92,
                                     normalize=cfg["gen"] == "gmm_norm")
    metric = km.METRICS[cfg["metric"]]
    G0, _ = orc.bruteforce_knn(X[:n0], K, metric=metric)
    seed, rounds = 7, 5
    p = km.params(k=K, metric=cfg["metric"], precision=cfg["precision"], max_iters=rounds,
                  delta=0.0, seed=seed)
    srv = km.Server(X[:n0].copy(), G0, p, slots=3, capacity_rows=total + 10,
                    max_batch_rows=256)
    try:
        X0, ids0, d0 = srv.resident()
        assert np.array_equal(X0, X[:n0])
        # resident lists: the input ids with canonical distances, (distance, id) sorted
        for i in range(0, n0, 97):
            assert sorted(ids0[i].tolist()) == sorted(G0[i].tolist())
            for j in range(K):
                assert d0[i, j] == orc.distance(metric, X[i], X[ids0[i, j]])
        batches, off = {}, n0
        for r, b in enumerate(sizes):
            batches[100 + r] = X[off:off + b].copy()
            off += b
        for rid, B in batches.items():
            srv.submit(B, rid)
        served = {rid: srv.wait(rid, timeout_ms=120000) for rid in batches}
        srv.drain()
        stats = srv.stats()
        assert stats["completed"] == len(sizes) and stats["failed"] == 0
        assert stats["max_concurrent"] >= 2
        assert stats["resident_rows"] == total
        Xr, idr, dr = srv.resident()
    finally:
        srv.close()

    # Replay the schedule in commit order.
    order = sorted(served, key=lambda q: served[q][2]["commit_seq"])
    assert [served[q][2]["commit_seq"] for q in order] == list(range(len(sizes)))
    ctx = km.Context(0)
    states = [(X[:n0], ids0, d0)]
    Xs = X[:n0]
    for q in order:
        ids_out, d_out, info = served[q]
        c = info["snapshot_commits"]
        assert c <= info["commit_seq"]
        sX, sI, sD = states[c]
        n_snap = sI.shape[0]
        assert info["snapshot_rows"] == n_snap
        B = batches[q]
        seed_r = orc.hash64(seed, 0, 4, q, 0)
        pr = km.params(k=K, metric=cfg["metric"], precision=cfg["precision"], max_iters=rounds,
                       delta=0.0, seed=seed_r)
        ai, ad, ast = ctx.merge_joint(torch.from_numpy(np.ascontiguousarray(sX)).cuda(),
                                      torch.from_numpy(sI).cuda(),
                                      torch.from_numpy(B).cuda(), pr)
        ai, ad = ai.cpu().numpy(), ad.cpu().numpy()
        assert info["rounds"] == ast["rounds"]
        oi, od, _ = orc.merge_joint(np.ascontiguousarray(sX), sI, B, K, metric=metric,
                                    max_iters=rounds, delta=0.0, seed=seed_r)
        assert np.array_equal(ai, oi) and np.array_equal(ad, od), f"alone != oracle ({q})"
        cur = states[-1]
        assert info["commit_base"] == cur[1].shape[0]
        ni, nd, bi, bd = commit(cur, ai, ad, n_snap, K)
        # same alone and in the mix: the served batch rows are the alone run's rows
        assert np.array_equal(ids_out, bi), f"served ids differ from the alone run ({q})"
        assert np.array_equal(d_out, bd), f"served dists differ from the alone run ({q})"
        Xs = np.concatenate([Xs, B])
        states.append((Xs, np.concatenate([ni, bi]), np.concatenate([nd, bd])))
    ctx.close()
    fX, fI, fD = states[-1]
    assert np.array_equal(Xr, fX)
    assert np.array_equal(idr, fI)
    assert np.array_equal(dr, fD)
    # every resident list: sorted, no self, no repeats, ids in range
    assert (np.diff(dr, axis=1) >= 0).all()
    assert (idr >= 0).all() and (idr < total).all()
    assert not (idr == np.arange(total)[:, None]).any()
    assert all(len(set(row)) == K for row in idr.tolist())


def test_admission_and_limits(torch, km, orc):
    K, d, n0 = 8, 16, 400
    X = datagen.gaussian_mixture(n0 + 300, d, seed=5)
    G0, _ = orc.bruteforce_knn(X[:n0], K)
    p = km.params(k=K, max_iters=3, delta=0.0)
    # a reserve larger than the device: nothing can be admitted, and with no
    # batch running the request fails instead of waiting for ever
    srv = km.Server(X[:n0].copy(), G0, p, slots=2, capacity_rows=n0 + 250, max_batch_rows=200,
                    hbm_reserve_bytes=1 << 60)
    try:
        srv.submit(X[n0:n0 + 50].copy(), 1)
        with pytest.raises(km.KnnmError) as e:
            srv.wait(1, timeout_ms=60000)
        assert e.value.code == -2
        with pytest.raises(km.KnnmError) as e:   # larger than max_batch_rows
            srv.submit(X[n0:n0 + 201].copy(), 2)
        assert e.value.code == -2
    finally:
        srv.close()
    srv = km.Server(X[:n0].copy(), G0, p, slots=1, capacity_rows=n0 + 120, max_batch_rows=200)
    try:
        srv.submit(X[n0:n0 + 100].copy(), 1)
        with pytest.raises(km.KnnmError) as e:   # would pass capacity_rows
            srv.submit(X[n0 + 100:n0 + 130].copy(), 2)
        assert e.value.code == -2
        with pytest.raises(km.KnnmError) as e:   # id in use
            srv.submit(X[n0 + 100:n0 + 110].copy(), 1)
        assert e.value.code == -1
        ids, dists, info = srv.wait(1, timeout_ms=60000)
        assert info["status"] == 0 and info["commit_base"] == n0 and ids.shape == (100, K)
        srv.submit(X[n0 + 100:n0 + 120].copy(), 3)   # exactly fills capacity_rows
        srv.wait(3, timeout_ms=60000)
        assert srv.stats()["resident_rows"] == n0 + 120
    finally:
        srv.close()


def test_malformed_resident_graph_is_rejected(torch, km, orc):
    K, n0 = 6, 200
    X = datagen.gaussian_mixture(n0, 8, seed=2)
    G0, _ = orc.bruteforce_knn(X, K)
    G0[17, 2] = G0[17, 3]
    with pytest.raises(km.KnnmError):
        km.Server(X, G0, km.params(k=K), slots=1)
    G0, _ = orc.bruteforce_knn(X, K)
    G0[5, 0] = 5
    with pytest.raises(km.KnnmError):
        km.Server(X, G0, km.params(k=K), slots=1)

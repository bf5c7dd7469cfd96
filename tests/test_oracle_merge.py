"""Pins for the oracle's merge steps (Alg. 1 S-Merge, Alg. 2 J-Merge, NN-Descent build).

Each test pins the oracle to something the paper or the mathematics fixes:
a round traced by hand, the brute-force merge of Sec. 1, exactness when the
random init covers the whole other set, the convergence invariant of Sec. 3.4
(phi non-increasing), the fixpoint where a round changes no list, the
set masks of Alg. 1/2, and brute-force checks of the sampling rule.
"""
import json
import os

import numpy as np
import pytest

from paper_1908_00814_gb300 import datagen

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _hand_state(orc, fx):
    ids = np.array(fx["start_ids"], np.int32)
    dists = np.array(fx["start_dists"], np.float32)
    flags = np.zeros_like(ids, dtype=np.uint8)  # all old: inserted entries become new
    n, K = ids.shape
    return orc.State(ids, dists, flags, np.zeros((n, 0), np.int32), np.zeros((n, 0), np.float32))


@pytest.mark.parametrize("mode", ["symmetric", "joint"])
def test_hand_traced_round(orc, mode):
    fx = json.load(open(os.path.join(GOLDEN, "hand_round_3p3.json")))
    X = np.array(fx["points"], np.float32)[:, None]
    st = _hand_state(orc, fx)
    st.flags[:] = orc.FLAG_NEW
    new_ids, new_cnt, old_ids, old_cnt = orc.sample(st, seed=0, t=1, s=1, literal=True)
    got = [sorted(new_ids[u, :new_cnt[u]].tolist()) for u in range(len(X))]
    assert got == fx["graph_script"]
    assert old_cnt.sum() == 0
    st.flags[:] = orc.FLAG_OLD
    m = orc.SYMMETRIC if mode == "symmetric" else orc.JOINT
    c, ev = orc.join(m, X, fx["n1"], st, (new_ids, new_cnt, old_ids, old_cnt))
    exp = fx[mode]
    assert ev == exp["dist_evals"]
    assert c == exp["updates"]
    assert st.ids.tolist() == exp["end_ids"]
    assert st.dists.tolist() == exp["end_dists"]
    if "end_inserted" in exp:
        assert st.flags.tolist() == exp["end_inserted"]


def _check_lists(X, ids, dists, orc, metric=0, allow_neg=False):
    n, K = ids.shape
    assert ids.min() >= 0 and ids.max() < n
    assert not np.any(ids == np.arange(n)[:, None])
    s = np.sort(ids, axis=1)
    assert not np.any(s[:, 1:] == s[:, :-1])
    # sorted by (distance, id)
    dd, ii = dists[:, 1:], ids[:, 1:]
    dp, ip = dists[:, :-1], ids[:, :-1]
    assert np.all((dp < dd) | ((dp == dd) & (ip < ii)))
    # stored distances are the canonical ones
    for u in range(0, n, max(1, n // 50)):
        for j in range(K):
            assert orc.distance(metric, X[u], X[ids[u, j]]) == dists[u, j]


def _small_split(seed=7, n1=300, n2=300, d=8, K=8, metric=0):
    X = datagen.gaussian_mixture(n1 + n2, d, n_comp=6, seed=seed)
    return X, n1, n2, K


def test_bruteforce_merge_of_exact_graphs_is_exact(orc):
    """Sec. 1: cross-comparing S1 x S2 on exact G1, G2 yields the exact graph of S."""
    X, n1, n2, K = _small_split()
    G1, _ = orc.bruteforce_knn(X[:n1], K)
    G2, _ = orc.bruteforce_knn(X[n1:], K)
    ids, dists = orc.bruteforce_merge(X[:n1], G1, X[n1:], G2, K)
    ref_ids, ref_d = orc.bruteforce_knn(X, K)
    assert np.array_equal(ids, ref_ids)
    assert np.array_equal(dists, ref_d)


def test_build_with_k_equal_n_minus_1_is_exact(orc):
    """Every list holds all other nodes, so the build is the exact graph."""
    X = datagen.gaussian_mixture(9, 5, seed=3)
    ids, dists, st = orc.build_graph(X, 8, max_iters=3)
    ref_ids, ref_d = orc.bruteforce_knn(X, 8)
    assert np.array_equal(ids, ref_ids) and np.array_equal(dists, ref_d)


def test_joint_full_coverage_rows_are_exact(orc):
    """J-Merge, raw set no larger than k - k/2: every S1 list is appended with
    all of S2 (Alg. 2 Append), so after the final merge with G1^v each S1 row is
    the exact k-NN list of S1 u S2, whatever the rounds do."""
    X = datagen.gaussian_mixture(43, 6, seed=9)
    n1, K = 40, 6           # K_keep = 3, K - K_keep = 3 = |S2|
    G1, _ = orc.bruteforce_knn(X[:n1], K)
    ids, dists, _ = orc.merge_joint(X[:n1], G1, X[n1:], K, max_iters=4)
    ref_ids, ref_d = orc.bruteforce_knn(X, K)
    assert np.array_equal(ids[:n1], ref_ids[:n1])
    assert np.array_equal(dists[:n1], ref_d[:n1])


def test_init_divide_and_append(orc):
    """Alg. 1 Divide/Append: the kept part is the first K_keep of the re-sorted
    input list, the rear is the rest, the appended ids are distinct members of
    the other set."""
    X, n1, n2, K = _small_split(seed=2, n1=50, n2=40)
    rng = np.random.default_rng(0)
    G1 = np.stack([rng.choice(np.delete(np.arange(n1), i), K, replace=False) for i in range(n1)])
    G2 = np.stack([rng.choice(np.delete(np.arange(n2), i), K, replace=False) for i in range(n2)])
    Kk = 4
    st = orc.init(orc.SYMMETRIC, X, n1, K, Kk, seed=5, G1=G1, G2=G2)
    for i in range(n1 + n2):
        own = (G1[i] if i < n1 else G2[i - n1] + n1).tolist()
        dd = [orc.distance(0, X[i], X[j]) for j in own]
        order = sorted(range(K), key=lambda a: (dd[a], own[a]))
        kept = [own[a] for a in order[:Kk]]
        rear = [own[a] for a in order[Kk:]]
        assert st.rear_ids[i].tolist() == rear
        row = st.ids[i].tolist()
        assert set(kept) <= set(row)
        appended = [v for v in row if v not in kept]
        assert len(appended) == K - Kk
        assert all((v >= n1) == (i < n1) for v in appended)
        assert np.all(st.flags[i] == orc.FLAG_NEW)
    _check_lists(X, st.ids, st.dists, orc)


def test_init_random_draws_follow_hash(orc):
    """Appended ids are base + H(seed, 0, 3, i, c) mod n_src, in draw order,
    skipping self and repeats."""
    X = datagen.gaussian_mixture(30, 4, seed=1)
    st = orc.init(orc.JOINT, X, 0, 5, 0, seed=77)
    for i in range(30):
        exp, c = [], 0
        while len(exp) < 5:
            j = orc.hash64(77, 0, orc.STREAM_INIT, i, c) % 30
            c += 1
            if j != i and j not in exp:
                exp.append(j)
        assert sorted(st.ids[i].tolist()) == sorted(exp)


def test_sampling_rule_by_brute_force(orc):
    """Round step 1 checked against a direct reading of the rule: the s new
    entries with the smallest sampling key are taken (and flipped), reverse
    lists keep the s smallest keys, new and old are disjoint."""
    X, n1, n2, K = _small_split(seed=4, n1=120, n2=100)
    st = orc.init(orc.JOINT, X, 0, K, 0, seed=3)
    rng = np.random.default_rng(1)
    st.flags[:] = (rng.random(st.flags.shape) < 0.6).astype(np.uint8)
    before = st.flags.copy()
    s, seed, t = 3, 11, 2
    new_ids, new_cnt, old_ids, old_cnt = orc.sample(st, seed, t, s)
    n = len(X)

    def key(stream, owner, member):
        member = int(member)
        return ((orc.hash64(seed, t, stream, int(owner), member) >> 32) << 32) | member

    fwd_new = {}
    fwd_old = {}
    for u in range(n):
        cand = [v for j, v in enumerate(st.ids[u]) if before[u, j] == orc.FLAG_NEW]
        cand.sort(key=lambda v: key(0, u, v))
        fwd_new[u] = cand[:s]
        fwd_old[u] = [v for j, v in enumerate(st.ids[u]) if before[u, j] == orc.FLAG_OLD]
        for j, v in enumerate(st.ids[u]):
            expect_flag = orc.FLAG_OLD if (v in fwd_new[u] or before[u, j] == 0) else orc.FLAG_NEW
            assert st.flags[u, j] == expect_flag
    rev_new = {u: [] for u in range(n)}
    rev_old = {u: [] for u in range(n)}
    for u in range(n):
        for v in fwd_new[u]:
            rev_new[v].append(u)
        for v in fwd_old[u]:
            rev_old[v].append(u)
    for u in range(n):
        rn = sorted(rev_new[u], key=lambda w: key(1, u, w))[:s]
        ro = sorted(rev_old[u], key=lambda w: key(2, u, w))[:s]
        exp_new = set(fwd_new[u]) | set(rn)
        exp_old = (set(fwd_old[u]) | set(ro)) - exp_new
        got_new = new_ids[u, :new_cnt[u]].tolist()
        got_old = old_ids[u, :old_cnt[u]].tolist()
        assert len(got_new) == len(set(got_new)) and set(got_new) == exp_new
        assert len(got_old) == len(set(got_old)) and set(got_old) == exp_old


def _run_rounds(orc, mode, X, n1, K, G1=None, G2=None, rounds=6, s=4, seed=0, literal=False):
    Kk = orc.keep_count(K, 0.5) if n1 > 0 else K
    st = orc.init(mode, X, n1, K, Kk, seed, G1=G1, G2=G2)
    hist = [st.copy()]
    stats = []
    for t in range(1, rounds + 1):
        cands = orc.sample(st, seed, t, s, literal=literal)
        c, ev = orc.join(mode, X, n1, st, cands)
        hist.append(st.copy())
        stats.append((c, ev, cands))
        if c == 0:
            break
    return hist, stats


@pytest.mark.parametrize("mode", ["symmetric", "joint", "build"])
def test_round_invariants(orc, mode):
    """After every round: lists sorted by (distance, id), unique, no self, ids in
    range, canonical distances; phi non-increasing (Sec. 3.4, Eq. conv); each
    node's set of true neighbours never shrinks; the set mask holds."""
    X, n1, n2, K = _small_split(seed=12)
    G1 = G2 = None
    if mode != "build":
        G1, _ = orc.bruteforce_knn(X[:n1], K)
        G2, _ = orc.bruteforce_knn(X[n1:], K)
    m = orc.SYMMETRIC if mode == "symmetric" else orc.JOINT
    nn1 = 0 if mode == "build" else n1
    hist, stats = _run_rounds(orc, m, X, nn1, K, G1=G1, G2=G2 if mode == "symmetric" else None)
    exact_ids, exact_d = orc.bruteforce_knn(X, K)
    kth = exact_d[:, -1]
    prev_phi, prev_true = None, None
    for st in hist:
        _check_lists(X, st.ids, st.dists, orc)
        ph = orc.phi(st.dists)
        true_sets = [set(st.ids[u][(st.dists[u] < kth[u]) |
                                   ((st.dists[u] == kth[u]) & np.isin(st.ids[u], exact_ids[u]))])
                     for u in range(len(X))]
        if prev_phi is not None:
            assert ph <= prev_phi
            assert all(p <= q for p, q in zip(prev_true, true_sets))
        prev_phi, prev_true = ph, true_sets
    first = hist[0]
    last = hist[-1]
    if mode == "symmetric":
        for u in range(n1):   # S1 rows gain no S1 ids beyond their kept part
            assert {v for v in last.ids[u] if v < n1} <= set(first.ids[u])
        for u in range(n1, 2 * n1):
            assert {v for v in last.ids[u] if v >= n1} <= set(first.ids[u])
    if mode == "joint":
        for u in range(n1):
            assert {v for v in last.ids[u] if v < n1} <= set(first.ids[u])
    for c, ev, _ in stats:
        assert ev > 0


@pytest.mark.parametrize("mode", ["symmetric", "joint"])
def test_literal_fixpoint(orc, mode):
    """Alg. 1/2 stop once a round changes no list: at that point no allowed pair
    of any G-script[u] = G[u] u Reverse(G)[u] can enter either endpoint's list."""
    X, n1, n2, K = _small_split(seed=21, n1=60, n2=50, d=4, K=5)
    G1, _ = orc.bruteforce_knn(X[:n1], K)
    G2, _ = orc.bruteforce_knn(X[n1:], K)
    m = orc.SYMMETRIC if mode == "symmetric" else orc.JOINT
    hist, stats = _run_rounds(orc, m, X, n1, K, G1=G1, G2=G2 if mode == "symmetric" else None,
                              rounds=60, literal=True)
    assert stats[-1][0] == 0
    st = hist[-1]
    n = len(X)
    rev = {u: set() for u in range(n)}
    for u in range(n):
        for v in st.ids[u]:
            rev[int(v)].add(u)
    for u in range(n):
        gs = sorted(set(st.ids[u].tolist()) | rev[u])
        for a in range(len(gs)):
            for b in range(a + 1, len(gs)):
                p, q = gs[a], gs[b]
                if mode == "symmetric" and (p < n1) == (q < n1):
                    continue
                if mode == "joint" and p < n1 and q < n1:
                    continue
                dpq = orc.distance(0, X[p], X[q])
                for x, y in ((p, q), (q, p)):
                    if y in st.ids[x]:
                        continue
                    kd, ki = st.dists[x, -1], st.ids[x, -1]
                    assert (dpq, y) > (kd, ki)


def test_literal_evals_count_pairs(orc):
    """dist_evals = number of unordered allowed pairs of each G-script[u], summed
    over u (each occurrence counts: the scanning rate C of Sec. 5.1)."""
    X, n1, n2, K = _small_split(seed=5, n1=40, n2=30, d=3, K=4)
    G1, _ = orc.bruteforce_knn(X[:n1], K)
    G2, _ = orc.bruteforce_knn(X[n1:], K)
    st = orc.init(orc.SYMMETRIC, X, n1, K, 2, 0, G1=G1, G2=G2)
    before = st.copy()
    cands = orc.sample(st, 0, 1, 1, literal=True)
    _, ev = orc.join(orc.SYMMETRIC, X, n1, st, cands)
    n = len(X)
    rev = {u: set() for u in range(n)}
    for u in range(n):
        for v in before.ids[u]:
            rev[int(v)].add(u)
    total = 0
    for u in range(n):
        gs = set(before.ids[u].tolist()) | rev[u]
        a = sum(1 for v in gs if v < n1)
        total += a * (len(gs) - a)
    assert ev == total


def test_merge_config1_recall(orc):
    """The smallest workload (2 x 5,000 x 32 Gaussian mixture, k=10, 8 rounds,
    rho=0.5).  Unit-variance clusters in 32-d have intrinsic dimension 32, where
    sampled NN-Descent with k=10 stalls near 0.91; the merge must beat a from-
    scratch build of the whole set (about 0.85 here), as Sec. 5.2 reports."""
    X = datagen.generate("smerge_gmm_10k_d32_k10")
    n1 = 5000
    G1, _ = orc.bruteforce_knn(X[:n1], 10)
    G2, _ = orc.bruteforce_knn(X[n1:], 10)
    ids, dists, st = orc.merge_symmetric(X[:n1], G1, X[n1:], G2, 10, max_iters=8, seed=0)
    q = datagen.sample_nodes(len(X), 2000, seed=0)
    truth = orc.exact_knn_f64(X, q, 10)
    r = orc.recall_at(X, q, ids, 10, truth=truth)
    assert r >= 0.90, r
    assert st["rounds"] >= 1
    b_ids, _, _ = orc.build_graph(X, 10, max_iters=8, seed=0)
    assert r > orc.recall_at(X, q, b_ids, 10, truth=truth)
    _check_lists(X, ids, dists, orc)


def test_build_recall(orc):
    """NN-Descent build (J-Merge with an empty graph) reaches high recall."""
    X = datagen.gaussian_mixture(2000, 8, n_comp=8, seed=31)
    ids, dists, st = orc.build_graph(X, 10, max_iters=12, seed=1)
    r = orc.recall_at(X, np.arange(0, 2000, 5), ids, 10)
    assert r >= 0.95, r


def test_final_merge_keeps_best_distinct(orc):
    ids = np.array([[3, 1, 4]], np.int32)
    dists = np.array([[1.0, 2.0, 5.0]], np.float32)
    rid = np.array([[1, 7, -1]], np.int32)
    rd = np.array([[2.0, 3.0, np.inf]], np.float32)
    st = orc.State(ids, dists, np.zeros_like(ids, dtype=np.uint8), rid, rd)
    oi, od = orc.final(st)
    assert oi.tolist() == [[3, 1, 7]] and od.tolist() == [[1.0, 2.0, 3.0]]


def _metric_data(metric, n, seed):
    if metric == 4:   # chi-square: non-negative histograms
        return datagen.bovw_like(n, 12, n_topics=3, words=30.0, seed=seed)
    if metric == 5:   # Jaccard: sets as 0/1 rows
        off, items = datagen.itemsets(n, 40, n_types=4, core=10, mean_len=6.0, seed=seed)
        return datagen.sets_to_rows(off, items, 40)
    return datagen.gaussian_mixture(n, 5, seed=seed, normalize=metric == 2)


@pytest.mark.parametrize("metric", [0, 1, 2, 3, 4, 5])
def test_exact_cases_hold_for_every_metric(orc, metric):
    """k = n - 1 builds and brute-force merges of exact graphs give the exact
    graph under every metric (the merge steps do not depend on the metric)."""
    X = _metric_data(metric, 9, 3)
    ids, dists, _ = orc.build_graph(X, 8, metric=metric, max_iters=3)
    ref_ids, ref_d = orc.bruteforce_knn(X, 8, metric=metric)
    assert np.array_equal(ids, ref_ids) and np.array_equal(dists, ref_d)
    X = _metric_data(metric, 80, 5)
    n1, K = 40, 6
    G1, _ = orc.bruteforce_knn(X[:n1], K, metric=metric)
    G2, _ = orc.bruteforce_knn(X[n1:], K, metric=metric)
    ids, dists = orc.bruteforce_merge(X[:n1], G1, X[n1:], G2, K, metric=metric)
    ref_ids, ref_d = orc.bruteforce_knn(X, K, metric=metric)
    assert np.array_equal(ids, ref_ids) and np.array_equal(dists, ref_d)


def _literal_script(ids):
    """Alg. 1's G-script as printed: G[u] united with Reverse(G)[u] = {v : u in G[v]}."""
    n = len(ids)
    script = [set(map(int, ids[u])) for u in range(n)]
    for v in range(n):
        for u in ids[v]:
            script[int(u)].add(v)
    return [sorted(s) for s in script]


def _sampled_sets(orc, st, flag, s, seed=5, t=3):
    st.flags[:] = flag
    new_ids, new_cnt, old_ids, old_cnt = orc.sample(st, seed, t, s)
    new = [sorted(new_ids[u, :new_cnt[u]].tolist()) for u in range(len(st.ids))]
    old = [sorted(old_ids[u, :old_cnt[u]].tolist()) for u in range(len(st.ids))]
    return new, old


def test_sampled_mode_reduces_to_literal_script_hand(orc):
    """Alg. 1's Reverse and union steps: when the sample size covers every list
    entry and every in-edge, the sampled mode takes everything, so its new set
    (all flags new) or old set (all flags old) is the literal G-script, here the
    hand-traced one of the 3 + 3 fixture."""
    fx = json.load(open(os.path.join(GOLDEN, "hand_round_3p3.json")))
    st = _hand_state(orc, fx)
    s = len(fx["points"])  # >= K and >= every in-degree
    new, old = _sampled_sets(orc, st, orc.FLAG_NEW, s)
    assert new == fx["graph_script"] and all(len(o) == 0 for o in old)
    assert np.all(st.flags == orc.FLAG_OLD)  # every sampled forward entry turns old
    new, old = _sampled_sets(orc, st, orc.FLAG_OLD, s)
    assert old == fx["graph_script"] and all(len(x) == 0 for x in new)


@pytest.mark.parametrize("K", [6, 10])
def test_sampled_mode_reduces_to_literal_script_random(orc, K):
    """Same reduction on 300 rows with a random graph (hubs included): the sets
    equal G[u] united with Reverse(G)[u] computed here from the ids alone."""
    X = datagen.gaussian_mixture(300, 4, n_comp=3, seed=9)
    st = orc.init(orc.JOINT, X, 0, K, 0, seed=21)
    # make row 0 a hub: many lists point at it, so s must exceed K
    for u in range(1, 120):
        if 0 not in st.ids[u]:
            st.ids[u, -1] = 0
    indeg = np.bincount(st.ids.ravel(), minlength=300)
    s = int(max(K, indeg.max()))
    assert s > K
    script = _literal_script(st.ids)
    new, old = _sampled_sets(orc, st, orc.FLAG_NEW, s)
    assert new == script and all(len(o) == 0 for o in old)
    new, old = _sampled_sets(orc, st, orc.FLAG_OLD, s)
    assert old == script and all(len(x) == 0 for x in new)
    # one short of the largest in-degree: only the lists of the rows with that
    # in-degree are cut (one reverse entry each); every other row is unchanged
    new, _ = _sampled_sets(orc, st, orc.FLAG_NEW, s - 1)
    for u in range(300):
        if indeg[u] < s:
            assert new[u] == script[u]
        else:
            assert set(new[u]) <= set(script[u]) and set(st.ids[u].tolist()) <= set(new[u])
            assert len(script[u]) - 1 <= len(new[u]) <= len(script[u])

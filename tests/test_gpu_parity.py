"""Parity of the CUDA library (through the C ABI) with the CPU oracle.

Every comparison is element by element on the same seeded inputs: ids and
flags bit-exact, distances bit-exact (both sides compute the canonical FP32
distance), per-round counters equal.  The BF16 tensor-core path must produce
the very same graphs as the FP32 path (its re-rank is exact whenever the
error bound cannot rule a pair out).
"""
import json
import os

import numpy as np
import pytest

from paper_1908_00814_gb300 import datagen

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


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


def cuda(torch, a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def host(t):
    return t.cpu().numpy()


def assert_same(a, b, what=""):
    a, b = np.asarray(a), np.asarray(b)
    assert a.shape == b.shape, (what, a.shape, b.shape)
    if a.dtype == np.float32:
        bad = a.view(np.uint32) != b.view(np.uint32)
    else:
        bad = a != b
    if bad.any():
        idx = np.argwhere(bad)[:5]
        raise AssertionError(f"{what}: {bad.sum()} mismatches, first at {idx.tolist()}: "
                             f"{a[tuple(idx[0])]} vs {b[tuple(idx[0])]}")


def split_data(seed=3, n1=700, n2=600, d=16, kind="gmm"):
    if kind == "sift":
        X = datagen.sift_like(n1 + n2, d, seed=seed)
    elif kind == "bovw":   # non-negative histograms for the chi-square metric
        X = datagen.bovw_like(n1 + n2, d, n_topics=8, words=4.0 * d, seed=seed)
    else:
        X = datagen.gaussian_mixture(n1 + n2, d, n_comp=8, seed=seed)
    return X, n1


METRIC_NAMES = {0: "l2", 1: "ip", 2: "cos", 3: "l1", 4: "chi2"}


# ------------------------------------------------------------------ steps

def test_hand_traced_round(torch, km, ctx):
    fx = json.load(open(os.path.join(GOLDEN, "hand_round_3p3.json")))
    X = np.array(fx["points"], np.float32)[:, None].repeat(4, 1) * np.array([1, 0, 0, 0],
                                                                            np.float32)
    n = len(X)
    gs = fx["graph_script"]
    cap = max(len(g) for g in gs)
    new_ids = np.full((n, cap), -1, np.int32)
    for u, g in enumerate(gs):
        new_ids[u, :len(g)] = g
    new_cnt = np.array([len(g) for g in gs], np.int32)
    old_ids = np.full((n, 1), -1, np.int32)
    old_cnt = np.zeros(n, np.int32)
    for mode, key in ((km.SYMMETRIC, "symmetric"), (km.JOINT, "joint")):
        ids = cuda(torch, np.array(fx["start_ids"], np.int32))
        dists = cuda(torch, np.array(fx["start_dists"], np.float32))
        flags = cuda(torch, np.zeros((n, 2), np.uint8))
        p = km.params(k=2, metric="l2")
        c, ev = ctx.step_join(mode, cuda(torch, X), fx["n1"], p, ids, dists, flags,
                              tuple(cuda(torch, a) for a in (new_ids, new_cnt, old_ids, old_cnt)))
        exp = fx[key]
        assert ev == exp["dist_evals"] and c == exp["updates"]
        assert host(ids).tolist() == exp["end_ids"]
        assert host(dists).tolist() == exp["end_dists"]
        if "end_inserted" in exp:
            assert host(flags).tolist() == exp["end_inserted"]


@pytest.mark.parametrize("mode", ["symmetric", "joint", "build"])
@pytest.mark.parametrize("metric", [0, 1, 2, 3, 4])
def test_init_parity(torch, km, ctx, orc, mode, metric):
    X, n1 = split_data(seed=5 + metric, kind="bovw" if metric == 4 else "gmm")
    n = len(X)
    K = 10
    G1 = G2 = None
    if mode != "build":
        G1, _ = orc.bruteforce_knn(X[:n1], K, metric=metric)
        # shuffle the rows' order: init must re-sort the input lists
        G1 = np.random.default_rng(0).permuted(G1, axis=1)
    if mode == "symmetric":
        G2, _ = orc.bruteforce_knn(X[n1:], K, metric=metric)
    m = orc.SYMMETRIC if mode == "symmetric" else orc.JOINT
    split = 0 if mode == "build" else n1
    Kk = K if mode == "build" else orc.keep_count(K, 0.5)
    ref = orc.init(m, X, split, K, Kk, seed=9, metric=metric, G1=G1, G2=G2)
    p = km.params(k=K, metric=metric, seed=9)
    got = ctx.step_init(m, cuda(torch, X), split, None if G1 is None else cuda(torch, G1),
                        None if G2 is None else cuda(torch, G2), p)
    assert_same(host(got[0]), ref.ids, "ids")
    assert_same(host(got[1]), ref.dists, "dists")
    assert_same(host(got[2]), ref.flags, "flags")
    if ref.rear_ids.shape[1]:
        assert_same(host(got[3]), ref.rear_ids, "rear ids")
        assert_same(host(got[4]), ref.rear_dists, "rear dists")


@pytest.mark.parametrize("K,s,n", [(10, 5, 1300), (20, 10, 2049), (7, 3, 33), (32, 16, 500),
                                   (1, 1, 40)])
def test_sample_parity(torch, km, ctx, orc, K, s, n):
    X = datagen.gaussian_mixture(n, 8, seed=K)
    st = orc.init(orc.JOINT, X, 0, K, K, seed=4)
    rng = np.random.default_rng(K)
    st.flags[:] = (rng.random(st.flags.shape) < 0.55).astype(np.uint8)
    flags_gpu = cuda(torch, st.flags)
    ids_gpu, d_gpu = cuda(torch, st.ids), cuda(torch, st.dists)
    ref = orc.sample(st, 21, 3, s)
    got = ctx.step_sample(ids_gpu, d_gpu, flags_gpu, 21, 3, s)
    assert_same(host(flags_gpu), st.flags, "flipped flags")
    for a, b, what in ((got[1], ref[1], "new_cnt"), (got[3], ref[3], "old_cnt")):
        assert_same(host(a), b, what)
    for u in range(n):
        assert host(got[0][u, :ref[1][u]]).tolist() == ref[0][u, :ref[1][u]].tolist()
        assert host(got[2][u, :ref[3][u]]).tolist() == ref[2][u, :ref[3][u]].tolist()


def _join_case(orc, X, n1, K, mode, metric, seed=1, t=2, s=None):
    """Oracle state after init + one round, then the candidate sets of the next."""
    G1 = G2 = None
    if n1 > 0:
        G1, _ = orc.bruteforce_knn(X[:n1], K, metric=metric)
    if mode == orc.SYMMETRIC:
        G2, _ = orc.bruteforce_knn(X[n1:], K, metric=metric)
    Kk = K if n1 == 0 else orc.keep_count(K, 0.5)
    st = orc.init(mode, X, n1, K, Kk, seed=seed, metric=metric, G1=G1, G2=G2)
    s = s or orc.sample_count(K, 0.5)
    cands = orc.sample(st, seed, 1, s)
    orc.join(mode, X, n1, st, cands, metric=metric)
    cands = orc.sample(st, seed, t, s)
    return st, cands


@pytest.mark.parametrize("precision", ["fp32", "bf16", "fp16"])
@pytest.mark.parametrize("metric", [0, 1, 2, 3, 4])
@pytest.mark.parametrize("mode", ["symmetric", "joint", "build"])
def test_join_parity(torch, km, ctx, orc, precision, metric, mode):
    X, n1 = split_data(seed=11 + metric, n1=800, n2=700, d=24,
                       kind="bovw" if metric == 4 else "gmm")
    K = 12
    m = orc.SYMMETRIC if mode == "symmetric" else orc.JOINT
    split = 0 if mode == "build" else n1
    st, cands = _join_case(orc, X, split, K, m, metric)
    ids, dists, flags = cuda(torch, st.ids), cuda(torch, st.dists), cuda(torch, st.flags)
    gc = tuple(cuda(torch, a) for a in cands)
    ref = st.copy()
    c_ref, e_ref = orc.join(m, X, split, ref, cands, metric=metric)
    p = km.params(k=K, metric=metric, precision=precision)
    c, e = ctx.step_join(m, cuda(torch, X), split, p, ids, dists, flags, gc)
    assert (c, e) == (c_ref, e_ref)
    assert_same(host(ids), ref.ids, "ids")
    assert_same(host(dists), ref.dists, "dists")
    assert_same(host(flags), ref.flags, "flags")


@pytest.mark.parametrize("d", [3, 8, 128, 960, 1030])
def test_join_parity_dims(torch, km, ctx, orc, d):
    """Row lengths that are not a multiple of 4 (plain loads), exactly one
    vector, and rows long enough to be processed in several chunks."""
    X = datagen.sift_like(900, d, seed=d)
    K = 8
    st, cands = _join_case(orc, X, 0, K, orc.JOINT, 0)
    ids, dists, flags = cuda(torch, st.ids), cuda(torch, st.dists), cuda(torch, st.flags)
    ref = st.copy()
    c_ref, e_ref = orc.join(orc.JOINT, X, 0, ref, cands)
    for precision in (["fp32", "bf16", "fp16"] if d % 8 == 0 else ["fp32"]):
        i2, d2, f2 = ids.clone(), dists.clone(), flags.clone()
        c, e = ctx.step_join(km.JOINT, cuda(torch, X), 0, km.params(k=K, precision=precision),
                             i2, d2, f2, tuple(cuda(torch, a) for a in cands))
        assert (c, e) == (c_ref, e_ref), precision
        assert_same(host(i2), ref.ids, f"ids {precision}")
        assert_same(host(d2), ref.dists, f"dists {precision}")


def test_final_parity(torch, km, ctx, orc):
    X, n1 = split_data(seed=2)
    K = 10
    G1, _ = orc.bruteforce_knn(X[:n1], K)
    G2, _ = orc.bruteforce_knn(X[n1:], K)
    st = orc.init(orc.SYMMETRIC, X, n1, K, 5, seed=1, G1=G1, G2=G2)
    ref_i, ref_d = orc.final(st)
    oi, od = ctx.step_final(cuda(torch, st.ids), cuda(torch, st.dists), cuda(torch, st.rear_ids),
                            cuda(torch, st.rear_dists))
    assert_same(host(oi), ref_i, "ids")
    assert_same(host(od), ref_d, "dists")


# ------------------------------------------------------------------ whole merges

def _smerge_both(torch, km, ctx, orc, X, n1, K, rounds, metric=0, sample_rate=0.5, seed=0,
                 delta=0.0, precisions=("fp32", "bf16", "fp16")):
    G1, _ = orc.bruteforce_knn(X[:n1], K, metric=metric)
    G2, _ = orc.bruteforce_knn(X[n1:], K, metric=metric)
    ref_i, ref_d, ref_st = orc.merge_symmetric(X[:n1], G1, X[n1:], G2, K, metric=metric,
                                               max_iters=rounds, sample_rate=sample_rate,
                                               seed=seed, delta=delta)
    for precision in precisions:
        p = km.params(k=K, metric=metric, precision=precision, max_iters=rounds,
                      sample_rate=sample_rate, seed=seed, delta=delta)
        gi, gd, st = ctx.merge_symmetric(cuda(torch, X[:n1]), cuda(torch, G1),
                                         cuda(torch, X[n1:]), cuda(torch, G2), p)
        assert st["updates"] == ref_st["updates"], precision
        assert st["dist_evals"] == ref_st["dist_evals"], precision
        assert_same(host(gi), ref_i, f"ids {precision}")
        assert_same(host(gd), ref_d, f"dists {precision}")
    return ref_i, ref_d, ref_st


def test_smerge_config1_parity(torch, km, ctx, orc):
    """The 2 x 5,000 x 32 Gaussian-mixture S-Merge, k=10, 8 rounds, rho=0.5."""
    X = datagen.generate("smerge_gmm_10k_d32_k10")
    _smerge_both(torch, km, ctx, orc, X, 5000, 10, 8)


@pytest.mark.parametrize("metric", [1, 2, 3, 4])
def test_smerge_metrics_parity(torch, km, ctx, orc, metric):
    if metric == 4:   # chi-square on non-negative histograms; no tensor-core form
        X = datagen.bovw_like(1800, 64, n_topics=12, words=120.0, seed=44)
    else:
        X = datagen.gaussian_mixture(1800, 24, n_comp=6, seed=40 + metric,
                                     normalize=(metric == 2))
    _smerge_both(torch, km, ctx, orc, X, 1000, 12, 5, metric=metric,
                 precisions=("fp32", "bf16") if metric >= 3 else ("fp32", "bf16", "fp16"))


def test_smerge_sift_parity(torch, km, ctx, orc):
    X = datagen.sift_like(4000, 128, seed=77)
    _smerge_both(torch, km, ctx, orc, X, 2100, 20, 6, delta=0.001)


@pytest.mark.parametrize("precision", ["fp32", "bf16", "fp16"])
def test_jmerge_parity(torch, km, ctx, orc, precision):
    X = datagen.gaussian_mixture(3000, 32, n_comp=10, seed=8, normalize=True)
    n1, K = 2000, 16
    G1, _ = orc.bruteforce_knn(X[:n1], K, metric=orc.COS)
    ref_i, ref_d, ref_st = orc.merge_joint(X[:n1], G1, X[n1:], K, metric=orc.COS, max_iters=6)
    p = km.params(k=K, metric="cos", precision=precision, max_iters=6, delta=0.0)
    gi, gd, st = ctx.merge_joint(cuda(torch, X[:n1]), cuda(torch, G1), cuda(torch, X[n1:]), p)
    assert st["updates"] == ref_st["updates"] and st["dist_evals"] == ref_st["dist_evals"]
    assert_same(host(gi), ref_i, "ids")
    assert_same(host(gd), ref_d, "dists")


@pytest.mark.parametrize("precision", ["fp32", "bf16", "fp16"])
def test_build_parity(torch, km, ctx, orc, precision):
    X = datagen.sift_like(2500, 64, seed=12)
    ref_i, ref_d, ref_st = orc.build_graph(X, 20, max_iters=5, seed=3)
    p = km.params(k=20, precision=precision, max_iters=5, seed=3, delta=0.0)
    gi, gd, st = ctx.build(cuda(torch, X), p)
    assert st["updates"] == ref_st["updates"]
    assert_same(host(gi), ref_i, "ids")
    assert_same(host(gd), ref_d, "dists")


def test_host_pointers_match_device(torch, km, ctx, orc):
    """Host (numpy) inputs and outputs go through the same kernels."""
    X = datagen.gaussian_mixture(1200, 16, seed=1)
    n1, K = 600, 8
    G1, _ = orc.bruteforce_knn(X[:n1], K)
    G2, _ = orc.bruteforce_knn(X[n1:], K)
    p = km.params(k=K, max_iters=4, delta=0.0)
    hi, hd, _ = ctx.merge_symmetric(X[:n1].copy(), G1, X[n1:].copy(), G2, p)
    gi, gd, _ = ctx.merge_symmetric(cuda(torch, X[:n1]), cuda(torch, G1), cuda(torch, X[n1:]),
                                    cuda(torch, G2), p)
    assert isinstance(hi, np.ndarray)
    assert_same(hi, host(gi), "ids")
    assert_same(hd, host(gd), "dists")


def test_edge_sizes(torch, km, ctx, orc):
    # the smallest legal build: every list holds all other rows
    X = datagen.gaussian_mixture(9, 5, seed=3)
    gi, gd, _ = ctx.build(cuda(torch, X), km.params(k=8, max_iters=2, delta=0.0))
    ref_i, ref_d = orc.bruteforce_knn(X, 8)
    assert_same(host(gi), ref_i, "ids")
    assert_same(host(gd), ref_d, "dists")
    # k = 1 and k = 32, ragged row counts
    for K, n in ((1, 37), (32, 333)):
        X = datagen.gaussian_mixture(n, 6, seed=K)
        ref_i, ref_d, _ = orc.build_graph(X, K, max_iters=3, seed=2)
        gi, gd, _ = ctx.build(cuda(torch, X), km.params(k=K, max_iters=3, seed=2, delta=0.0))
        assert_same(host(gi), ref_i, f"ids k={K}")
        assert_same(host(gd), ref_d, f"dists k={K}")


def test_invalid_inputs_are_rejected(torch, km, ctx, orc):
    X = datagen.gaussian_mixture(100, 8, seed=1)
    n1, K = 50, 6
    G1, _ = orc.bruteforce_knn(X[:n1], K)
    G2, _ = orc.bruteforce_knn(X[n1:], K)
    p = km.params(k=K, max_iters=2)
    bad = []
    g = G1.copy(); g[3, 2] = 3; bad.append(g)          # self
    g = G1.copy(); g[4, 1] = g[4, 0]; bad.append(g)    # repeat
    g = G1.copy(); g[5, 0] = n1; bad.append(g)         # out of range
    for g in bad:
        with pytest.raises(km.KnnmError) as ei:
            ctx.merge_symmetric(cuda(torch, X[:n1]), cuda(torch, g), cuda(torch, X[n1:]),
                                cuda(torch, G2), p)
        assert ei.value.code == -1
    with pytest.raises(km.KnnmError):
        ctx.merge_symmetric(cuda(torch, X[:5]), cuda(torch, G1[:5]), cuda(torch, X[n1:]),
                            cuda(torch, G2), p)
    with pytest.raises(km.KnnmError):
        ctx.build(cuda(torch, X[:, :7].copy()), km.params(k=K, precision="bf16"))
    # the context stays usable
    gi, _, _ = ctx.merge_symmetric(cuda(torch, X[:n1]), cuda(torch, G1), cuda(torch, X[n1:]),
                                   cuda(torch, G2), p)
    assert host(gi).shape == (100, K)


@pytest.mark.parametrize("d,hi", [(128, 255), (136, 255), (64, 256), (128, 17)])
def test_join_parity_integer_extremes(torch, km, ctx, orc, d, hi):
    """Non-negative integer rows take the exact tensor-core path when
    d * (max_i^2 + max_j^2) < 2^24 (128 x 255: sums up to 16.6M, just inside),
    the bounded path otherwise (136 x 255); both must equal the oracle."""
    rng = np.random.default_rng(d + hi)
    X = rng.choice(np.array([0, 1, hi - 1, hi], np.float32), size=(900, d),
                   p=[0.3, 0.2, 0.2, 0.3]).astype(np.float32)
    X[:, :5] = rng.integers(0, hi + 1, size=(900, 5))  # break exact duplicates
    K = 10
    st, cands = _join_case(orc, X, 0, K, orc.JOINT, 0)
    ref = st.copy()
    c_ref, e_ref = orc.join(orc.JOINT, X, 0, ref, cands)
    ids, dists, flags = cuda(torch, st.ids), cuda(torch, st.dists), cuda(torch, st.flags)
    c, e = ctx.step_join(km.JOINT, cuda(torch, X), 0, km.params(k=K, precision="bf16"), ids,
                         dists, flags, tuple(cuda(torch, a) for a in cands))
    assert (c, e) == (c_ref, e_ref)
    assert_same(host(ids), ref.ids, "ids")
    assert_same(host(dists), ref.dists, "dists")


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_graph_replay_matches_stream_launches(torch, km, ctx, orc, precision):
    """Rounds replayed from one captured CUDA graph give the same graph, counters and
    stopping round as rounds launched one kernel at a time."""
    X = datagen.sift_like(3000, 64, seed=21)
    n1, K = 1600, 16
    G1, _ = orc.bruteforce_knn(X[:n1], K)
    G2, _ = orc.bruteforce_knn(X[n1:], K)
    g = km.Context(0)
    g.set_graphs(True)
    for delta in (0.0, 0.01):
        p = km.params(k=K, precision=precision, max_iters=9, delta=delta, seed=5)
        args = (cuda(torch, X[:n1]), cuda(torch, G1), cuda(torch, X[n1:]), cuda(torch, G2), p)
        ai, ad, ast = ctx.merge_symmetric(*args)
        bi, bd, bst = g.merge_symmetric(*args)
        assert ast["rounds"] == bst["rounds"]
        assert ast["updates"] == bst["updates"] and ast["dist_evals"] == bst["dist_evals"]
        assert_same(host(ai), host(bi), "ids")
        assert_same(host(ad), host(bd), "dists")
    ji, jd, jst = g.merge_joint(cuda(torch, X[:n1]), cuda(torch, G1), cuda(torch, X[n1:]),
                                km.params(k=K, precision=precision, max_iters=5, delta=0.0))
    ref_i, ref_d, ref_st = orc.merge_joint(X[:n1], G1, X[n1:], K, max_iters=5)
    assert jst["updates"] == ref_st["updates"]
    assert_same(host(ji), ref_i, "jmerge ids")
    assert_same(host(jd), ref_d, "jmerge dists")


def test_fp16_out_of_range_rows_fall_back_to_fp32(torch, km, ctx, orc):
    """Rows beyond the FP16 range get an infinite error bound: every pair with
    them is re-ranked in canonical FP32, and the merge still equals the oracle."""
    X = datagen.gaussian_mixture(1600, 16, n_comp=6, seed=77)
    X[::7] *= 1.0e5   # some rows far beyond +-65504
    _smerge_both(torch, km, ctx, orc, X, 800, 10, 4, precisions=("fp16",))


def _tree_oracle(orc, X, part_rows, G, K, seed, **kw):
    """The merge tree composed from oracle S-Merges, same pairing and seeds."""
    blocks, off = [], 0
    for r in part_rows:
        blocks.append((off, r, G[off:off + r]))
        off += r
    level = 0
    while len(blocks) > 1:
        nxt = []
        for j in range(0, len(blocks), 2):
            if j + 1 == len(blocks):
                nxt.append(blocks[j])
                continue
            (a0, ar, ag), (b0, br, bg) = blocks[j], blocks[j + 1]
            s = orc.hash64(seed, level, 6, j // 2, 0)
            ids, dists, _ = orc.merge_symmetric(X[a0:a0 + ar], ag, X[b0:b0 + br], bg, K, seed=s,
                                                **kw)
            nxt.append((a0, ar + br, ids))
            last = dists
        blocks = nxt
        level += 1
    return blocks[0][2], last


@pytest.mark.parametrize("parts", [8, 5])
def test_merge_tree_parity(torch, km, ctx, orc, parts):
    """Merge tree: levels of pairwise S-Merges over exact part graphs, bit-exact
    with the same tree composed from oracle merges (odd blocks carried up)."""
    K, rows = 8, 260
    X = datagen.gaussian_mixture(parts * rows, 16, n_comp=10, seed=90 + parts)
    part_rows = [rows] * parts
    G = np.concatenate([orc.bruteforce_knn(X[p * rows:(p + 1) * rows], K)[0]
                        for p in range(parts)])
    ref_i, ref_d = _tree_oracle(orc, X, part_rows, G, K, seed=3, max_iters=4, delta=0.0)
    for precision in ("fp32", "bf16"):
        p = km.params(k=K, precision=precision, max_iters=4, delta=0.0, seed=3)
        gi, gd, st = ctx.merge_tree(cuda(torch, X), part_rows, cuda(torch, G), p)
        assert st["rounds"] == int(np.ceil(np.log2(parts)))
        assert_same(host(gi), ref_i, f"tree ids {precision}")
        assert_same(host(gd), ref_d, f"tree dists {precision}")
    # one part: the input graph with canonical distances, sorted
    gi, gd, st = ctx.merge_tree(cuda(torch, X[:rows]), [rows], cuda(torch, G[:rows]),
                                km.params(k=K))
    assert st["rounds"] == 0
    for i in range(0, rows, 37):
        assert sorted(host(gi)[i].tolist()) == sorted(G[i].tolist())
        assert all(host(gd)[i, j] == orc.distance(0, X[i], X[host(gi)[i, j]]) for j in range(K))


def test_tensor_core_rounds_follow_the_rerank_share(torch, km, ctx, orc):
    """With a tensor-core precision every round of a merge of small-integer rows
    runs the tensor-core join; on float rows the first round (almost every pair
    a proposal) runs the FP32 join.  The graph equals the oracle either way."""
    X = datagen.sift_like(3000, 64, seed=41)
    _, _, st = ctx.merge_symmetric(cuda(torch, X[:1500]), cuda(torch, orc.bruteforce_knn(X[:1500], 12)[0]),
                                   cuda(torch, X[1500:]), cuda(torch, orc.bruteforce_knn(X[1500:], 12)[0]),
                                   km.params(k=12, precision="bf16", max_iters=5, delta=0.0))
    assert all(st["tc_rounds"]) and sum(st["reranked"]) == 0
    Xf = datagen.gaussian_mixture(3000, 32, n_comp=8, seed=42)
    ref_i, ref_d, _ = _smerge_both(torch, km, ctx, orc, Xf, 1500, 12, 6, precisions=("fp16",))
    G1, _ = orc.bruteforce_knn(Xf[:1500], 12)
    G2, _ = orc.bruteforce_knn(Xf[1500:], 12)
    _, _, st = ctx.merge_symmetric(cuda(torch, Xf[:1500]), cuda(torch, G1), cuda(torch, Xf[1500:]),
                                   cuda(torch, G2), km.params(k=12, precision="fp16", max_iters=6,
                                                              delta=0.0))
    assert st["tc_rounds"][0] is False


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_hmerge_parity(torch, km, ctx, orc, precision):
    """H-Merge (Sec. 3.3): visiting order, every upper layer (k/2 lists) and the
    bottom graph equal the oracle's step-by-step composition."""
    X = datagen.sift_like(2600, 32, seed=61)
    K, first = 12, 100
    perm_r, layers_r, ids_r, dists_r = orc.hmerge(X, K, first, max_iters=5, seed=9)
    p = km.params(k=K, precision=precision, max_iters=5, delta=0.0, seed=9)
    want = [m for m in layers_r if m < len(X)]
    perm, ids, dists, layers, st = ctx.hmerge(cuda(torch, X), first, p, layers=want)
    assert np.array_equal(perm, perm_r)
    assert sorted(perm.tolist()) == list(range(len(X)))
    assert st["rounds"] == len(layers_r)
    for m in want:
        assert_same(layers[m], layers_r[m], f"layer {m}")
    assert_same(ids, ids_r, "bottom ids")
    assert_same(dists, dists_r, "bottom dists")


@pytest.mark.parametrize("precision", ["bf16", "fp16"])
@pytest.mark.parametrize("metric,d", [(0, 32), (1, 48), (2, 40), (0, 96)])
def test_tensor_core_join_on_float_rows_every_round(torch, km, orc, precision, metric, d):
    """Float rows (not small integers): the tensor-core join (estimates on the
    tensor cores, canonical FP32 re-ranks wherever the bound cannot rule a pair
    out) forced on every round, and the FP32 join forced on every round: S-Merge
    and J-Merge equal the oracle bit for bit either way, and the estimates rule
    some pairs out without a re-rank."""
    X = datagen.gaussian_mixture(2200, d, n_comp=8, seed=70 + d + metric,
                                 normalize=(metric == 2))
    n1, K, rounds = 1100, 10, 6
    G1, _ = orc.bruteforce_knn(X[:n1], K, metric=metric)
    G2, _ = orc.bruteforce_knn(X[n1:], K, metric=metric)
    ref_i, ref_d, ref_st = orc.merge_symmetric(X[:n1], G1, X[n1:], G2, K, metric=metric,
                                               max_iters=rounds, seed=3)
    jref_i, jref_d, jref_st = orc.merge_joint(X[:n1], G1, X[n1:], K, metric=metric,
                                              max_iters=rounds, seed=4)
    for choice in (1, 2):
        ctx = km.Context(0)
        ctx.set_option(km.OPT_TC_JOIN, choice)
        p = km.params(k=K, metric=METRIC_NAMES[metric], precision=precision, max_iters=rounds,
                      delta=0.0, seed=3)
        gi, gd, st = ctx.merge_symmetric(cuda(torch, X[:n1]), cuda(torch, G1),
                                         cuda(torch, X[n1:]), cuda(torch, G2), p)
        assert all(st["tc_rounds"]) if choice == 1 else not any(st["tc_rounds"])
        if choice == 1:
            assert 0 < sum(st["reranked"]) < sum(st["dist_evals"])
        assert st["updates"] == ref_st["updates"] and st["dist_evals"] == ref_st["dist_evals"]
        assert_same(host(gi), ref_i, f"ids {precision} choice {choice}")
        assert_same(host(gd), ref_d, f"dists {precision} choice {choice}")
        p.seed = 4
        gi, gd, st = ctx.merge_joint(cuda(torch, X[:n1]), cuda(torch, G1), cuda(torch, X[n1:]), p)
        assert st["updates"] == jref_st["updates"]
        assert_same(host(gi), jref_i, f"jmerge ids {precision} choice {choice}")
        assert_same(host(gd), jref_d, f"jmerge dists {precision} choice {choice}")
        ctx.close()

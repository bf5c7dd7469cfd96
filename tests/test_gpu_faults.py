"""Paths that a normal run seldom or never takes, forced through context
options of the C ABI and checked against the CPU oracle:

* the join's direct insert: when a target's proposal bucket is full, further
  proposals for it go straight into its live list by ordered slot insertion
  (the lock-free form of UpdateNN) instead of through the bucketed update.
  With tiny buckets most proposals take that path; the merged graph
  must still equal the oracle's bit for bit (synchronous UpdateNN is the top-K
  of the round-start list and all proposals, whatever the insertion order);
* a device-side wait that gives up: the join's waits for its staged rows are
  bounded; with the poll limit at 0 every wait gives up at once, the call
  returns KNNM_ERR_DEVICE with the wait-timeout bit, and the same context then
  merges correctly;
* a scratch reservation that fails (host-side injection): KNNM_ERR_NOMEM, and
  the next call works;
* a serving wait that runs out: KNNM_ERR_TIMEOUT while the request is still
  running, then the request completes normally.
No test faults, traps or hangs the GPU: every failure is made on the host or
by a bounded wait that returns.
"""
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


def cuda(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def same_bits(a, b):
    a, b = np.asarray(a), np.asarray(b)
    if a.dtype == np.float32:
        return a.shape == b.shape and np.array_equal(a.view(np.uint32), b.view(np.uint32))
    return np.array_equal(a, b)


def _inputs(orc, kind, n1, n2, d, K, seed):
    if kind == "sift":
        X = datagen.sift_like(n1 + n2, d, n_centres=32, seed=seed)
    else:
        X = datagen.gaussian_mixture(n1 + n2, d, n_comp=8, seed=seed)
    G1, _ = orc.bruteforce_knn(X[:n1], K)
    G2, _ = orc.bruteforce_knn(X[n1:], K)
    return X, G1, G2


@pytest.mark.parametrize("bucket_cap", [1, 12])
@pytest.mark.parametrize("precision,kind", [("fp32", "gmm"), ("bf16", "sift"), ("bf16", "gmm")])
def test_direct_insert_path_is_bit_exact(torch, km, orc, bucket_cap, precision, kind):
    n1, n2, d, K, rounds = 1300, 1100, 32, 12, 6
    X, G1, G2 = _inputs(orc, kind, n1, n2, d, K, seed=31)
    ctx = km.Context(0)
    ctx.set_option(km.OPT_BUCKET_CAP, bucket_cap)
    p = km.params(k=K, precision=precision, max_iters=rounds, delta=0.0, seed=4)
    gi, gd, st = ctx.merge_symmetric(cuda(torch, X[:n1]), cuda(torch, G1), cuda(torch, X[n1:]),
                                     cuda(torch, G2), p)
    ri, rd, rst = orc.merge_symmetric(X[:n1], G1, X[n1:], G2, K, max_iters=rounds, seed=4)
    assert sum(st["spilled"]) > 0, st["spilled"]
    assert st["updates"] == rst["updates"] and st["dist_evals"] == rst["dist_evals"]
    assert same_bits(gi.cpu().numpy(), ri) and same_bits(gd.cpu().numpy(), rd)
    # J-Merge: the raw rows start from random lists, so early rounds propose a lot
    p = km.params(k=K, precision=precision, max_iters=rounds, delta=0.0, seed=6)
    gi, gd, st = ctx.merge_joint(cuda(torch, X[:n1]), cuda(torch, G1), cuda(torch, X[n1:]), p)
    ri, rd, rst = orc.merge_joint(X[:n1], G1, X[n1:], K, max_iters=rounds, seed=6)
    assert sum(st["spilled"]) > 0, st["spilled"]
    assert st["updates"] == rst["updates"]
    assert same_bits(gi.cpu().numpy(), ri) and same_bits(gd.cpu().numpy(), rd)
    ctx.close()


@pytest.mark.parametrize("precision,kind", [("fp32", "gmm"), ("bf16", "sift")])
def test_wait_that_gives_up_is_reported_and_context_recovers(torch, km, orc, precision, kind):
    n1, n2, d, K = 900, 900, 32, 10
    X, G1, G2 = _inputs(orc, kind, n1, n2, d, K, seed=12)
    args = (cuda(torch, X[:n1]), cuda(torch, G1), cuda(torch, X[n1:]), cuda(torch, G2))
    ctx = km.Context(0)
    ctx.set_option(km.OPT_WAIT_POLLS, 0)
    p = km.params(k=K, precision=precision, max_iters=3, delta=0.0, seed=2)
    with pytest.raises(km.KnnmError) as err:
        ctx.merge_symmetric(*args, p)
    assert err.value.code == -6 and "0x8" in str(err.value), str(err.value)
    torch.cuda.synchronize()  # the device is still healthy
    ctx.set_option(km.OPT_WAIT_POLLS, -1)
    gi, gd, st = ctx.merge_symmetric(*args, p)
    ri, rd, rst = orc.merge_symmetric(X[:n1], G1, X[n1:], G2, K, max_iters=3, seed=2)
    assert st["updates"] == rst["updates"]
    assert same_bits(gi.cpu().numpy(), ri) and same_bits(gd.cpu().numpy(), rd)
    with pytest.raises(km.KnnmError):
        ctx.set_option(km.OPT_WAIT_POLLS, -2)
    ctx.close()


def test_failed_scratch_reservation_is_nomem_and_next_call_works(torch, km, orc):
    n1, n2, d, K = 600, 500, 16, 8
    X, G1, G2 = _inputs(orc, "gmm", n1, n2, d, K, seed=5)
    args = (cuda(torch, X[:n1]), cuda(torch, G1), cuda(torch, X[n1:]), cuda(torch, G2))
    p = km.params(k=K, max_iters=4, delta=0.0, seed=1)
    ctx = km.Context(0)
    ctx.set_option(km.OPT_FAIL_ALLOC, 2)
    for _ in range(2):
        with pytest.raises(km.KnnmError) as err:
            ctx.merge_symmetric(*args, p)
        assert err.value.code == -2 and "injected" in str(err.value)
    gi, gd, _ = ctx.merge_symmetric(*args, p)
    ri, rd, _ = orc.merge_symmetric(X[:n1], G1, X[n1:], G2, K, max_iters=4, seed=1)
    assert same_bits(gi.cpu().numpy(), ri) and same_bits(gd.cpu().numpy(), rd)
    # scratch already reserved: the injected failure still comes first
    ctx.set_option(km.OPT_FAIL_ALLOC, 1)
    with pytest.raises(km.KnnmError) as err:
        ctx.merge_symmetric(*args, p)
    assert err.value.code == -2
    gi, _, _ = ctx.merge_symmetric(*args, p)
    assert same_bits(gi.cpu().numpy(), ri)
    ctx.close()


def test_server_wait_times_out_then_completes(torch, km, orc):
    n, d, K = 60000, 64, 10
    X = datagen.sift_like(n + 6000, d, n_centres=64, seed=8)
    ctx = km.Context(0)
    G, _, _ = ctx.build(cuda(torch, X[:n]), km.params(k=K, precision="bf16", max_iters=4))
    ctx.close()
    p = km.params(k=K, precision="fp32", max_iters=8, delta=0.0, seed=3)
    srv = km.Server(cuda(torch, X[:n]), G, p, slots=1, use_graphs=False)
    batch = np.ascontiguousarray(X[n:])
    srv.submit(batch, 7)
    with pytest.raises(TimeoutError):
        srv.wait(7, timeout_ms=0)
    ids, dists, info = srv.wait(7, timeout_ms=-1)
    assert info["status"] == 0 and info["rows"] == len(batch)
    assert ids.min() >= 0 and ids.max() < n + len(batch)
    assert np.all(np.diff(dists, axis=1) >= 0)
    srv.close()

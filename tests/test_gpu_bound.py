"""Coverage of the tensor-core estimate's error bound.

The BF16/FP16 joins settle a pair from its tensor-core estimate alone only
when the proven bound E shows the pair cannot be a proposal; otherwise they
re-rank it in canonical FP32.  So the merged graph equals the FP32 one exactly
if |estimate - canonical| <= E holds for every pair.  These tests compute, for
many pairs of float rows, the estimate exactly as the join computes it, its
bound and the canonical distance (knnm_step_tc_estimate), and require the
inequality for every pair; the largest ratio |estimate - canonical| / E of each
case is printed (how much slack the bound leaves).  Rows of small non-negative
integers must give bound 0 and an estimate equal to the canonical distance bit
for bit.  The canonical distances are checked against the oracle's.
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


@pytest.fixture(scope="module")
def ctx(km):
    return km.Context(0)


def _rows(kind, n, d, seed):
    if kind == "gmm":
        return datagen.gaussian_mixture(n, d, n_comp=8, seed=seed)
    if kind == "gmm_norm":
        return datagen.gaussian_mixture(n, d, n_comp=8, seed=seed, normalize=True)
    if kind == "gist":
        return datagen.gist_like(n, d, seed=seed) if d >= 64 else np.abs(
            datagen.gaussian_mixture(n, d, seed=seed))
    if kind == "wide":  # rows spread over six decades of magnitude
        X = datagen.gaussian_mixture(n, d, n_comp=8, seed=seed)
        scale = 10.0 ** np.random.default_rng(seed).uniform(-3, 3, size=(n, 1))
        return (X * scale).astype(np.float32)
    raise ValueError(kind)


def _pairs(X, P, seed):
    """Half random pairs, half near pairs (nearest of a random sample of 64)."""
    rng = np.random.default_rng(seed)
    n = len(X)
    pi = rng.integers(0, n, P)
    pj = rng.integers(0, n, P)
    h = P // 2
    for r in range(h):
        cand = rng.integers(0, n, 64)
        dd = ((X[cand] - X[pi[r]]) ** 2).sum(1)
        dd[cand == pi[r]] = np.inf
        pj[r] = cand[np.argmin(dd)]
    return pi.astype(np.int32), pj.astype(np.int32)


CASES = [(kind, d, metric, prec)
         for d in (32, 96, 128, 960)
         for kind, metric in (("gmm", "l2"), ("gist", "l2"), ("gmm", "ip"), ("gmm_norm", "cos"),
                              ("wide", "l2"), ("wide", "cos"))
         for prec in ("bf16", "fp16")]


@pytest.mark.parametrize("kind,d,metric,prec", CASES)
def test_every_estimate_within_its_bound(torch, km, ctx, orc, kind, d, metric, prec):
    n, P = 3000, 6000
    X = _rows(kind, n, d, seed=d + len(kind))
    pi, pj = _pairs(X, P, seed=d)
    Xd = torch.from_numpy(X).cuda()
    est, bound, canon = ctx.step_tc_estimate(Xd, torch.from_numpy(pi).cuda(),
                                             torch.from_numpy(pj).cuda(), metric, prec)
    est, bound, canon = (t.cpu().numpy() for t in (est, bound, canon))
    m = km.METRICS[metric]
    for r in range(0, P, 97):
        assert canon[r] == orc.distance(m, X[pi[r]], X[pj[r]]), r
    err = np.abs(est.astype(np.float64) - canon.astype(np.float64))
    assert np.all(np.isfinite(est) | ~np.isfinite(bound))
    bad = ~(err <= bound)
    assert not bad.any(), (int(bad.sum()), err[bad][:5], bound[bad][:5])
    fin = np.isfinite(bound) & (bound > 0)
    ratio = float((err[fin] / bound[fin]).max()) if fin.any() else 0.0
    rel = float(np.median(bound[fin] / np.maximum(np.abs(canon[fin]), 1e-30))) if fin.any() else 0.0
    print(f"\nbound {kind} d={d} {metric} {prec}: max |est-canon|/E = {ratio:.3e}, "
          f"median E/|canon| = {rel:.3e}")
    assert ratio <= 1.0


@pytest.mark.parametrize("prec", ["bf16", "fp16"])
@pytest.mark.parametrize("metric", ["l2", "ip", "cos"])
def test_small_integer_rows_are_exact(torch, km, ctx, metric, prec):
    X = datagen.sift_like(2000, 128, seed=3)
    pi, pj = _pairs(X, 4000, seed=1)
    est, bound, canon = ctx.step_tc_estimate(torch.from_numpy(X).cuda(),
                                             torch.from_numpy(pi).cuda(),
                                             torch.from_numpy(pj).cuda(), metric, prec)
    assert torch.all(bound == 0)
    assert torch.equal(est.view(torch.int32), canon.view(torch.int32))


def test_estimate_rejects_bad_arguments(torch, km, ctx):
    X = torch.zeros((10, 16), device="cuda")
    i = torch.zeros(4, dtype=torch.int32, device="cuda")
    j = torch.tensor([1, 2, 3, 10], dtype=torch.int32, device="cuda")
    with pytest.raises(km.KnnmError):
        ctx.step_tc_estimate(X, i, j)  # row 10 of 10
    with pytest.raises(km.KnnmError):
        ctx.step_tc_estimate(X, i, i, metric="l1")

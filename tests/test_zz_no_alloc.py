"""knnm_step_sample_noalloc: the sampler for callers that cannot allocate
device memory (plug-ins inside an application that owns the device budget,
servers that reserve everything at start-up).  Its scratch is a fixed array
inside the library, so its results must equal those of knnm_step_sample,
which takes its scratch from the context's allocator.  Checked through the C
ABI on two calls in a row (the second smaller, so stale contents of the shared
array from the first call would show), and the size limit is rejected on the
host before anything runs."""
import numpy as np
import pytest

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


def _state(torch, n, K, seed):
    rng = np.random.default_rng(seed)
    r = np.sort(rng.integers(0, n - K, size=(n, K)), axis=1) + np.arange(K)
    ids = ((np.arange(n)[:, None] + 1 + r) % n).astype(np.int32)
    dists = np.sort(rng.random((n, K)).astype(np.float32), axis=1)
    flags = (rng.random((n, K)) < 0.6).astype(np.uint8)
    return [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (ids, dists, flags)]


def _outputs(torch, n, K, s):
    return (torch.full((n, 2 * s), -1, dtype=torch.int32, device="cuda"),
            torch.zeros(n, dtype=torch.int32, device="cuda"),
            torch.full((n, K + s), -1, dtype=torch.int32, device="cuda"),
            torch.zeros(n, dtype=torch.int32, device="cuda"))


@pytest.mark.parametrize("calls", [[(20000, 20, 10, 2, 1), (3001, 12, 6, 5, 2)]])
def test_noalloc_matches_allocating_sampler(torch, km, calls):
    ctx = km.Context(0)
    for n, K, s, t, seed in calls:
        ids, dists, flags = _state(torch, n, K, seed)
        flags_ref = flags.clone()
        ref = ctx.step_sample(ids, dists, flags_ref, 99, t, s)
        out = _outputs(torch, n, K, s)
        rc = km.step_sample_noalloc(ids, dists, flags, 99, t, s, *out)
        torch.cuda.synchronize()
        assert rc == 0
        assert torch.equal(flags, flags_ref)
        assert torch.equal(out[1], ref[1]) and torch.equal(out[3], ref[3])
        cn = torch.arange(2 * s, device="cuda")[None, :] < ref[1][:, None]
        co = torch.arange(K + s, device="cuda")[None, :] < ref[3][:, None]
        assert torch.equal(torch.where(cn, out[0], -1), torch.where(cn, ref[0], -1))
        assert torch.equal(torch.where(co, out[2], -1), torch.where(co, ref[2], -1))
    ctx.close()


def test_noalloc_rejects_oversize(torch, km):
    n, K, s = 40000, 20, 10  # 40000 * 40 * 8 bytes > the fixed array
    ids, dists, flags = _state(torch, n, K, 3)
    out = _outputs(torch, n, K, s)
    assert km.step_sample_noalloc(ids, dists, flags, 1, 1, s, *out) == -1


def test_noalloc_limit_is_the_stated_formula(torch, km):
    """The header's limit, a(N*K*8) + 2*a(N*s*8) + 256 <= the array size with a()
    rounding up to 256 bytes: the largest N that fits runs, one more row is
    rejected before anything is launched."""
    K, s = 20, 10
    a = lambda x: (x + 255) // 256 * 256
    cap = 8 << 20
    n = cap // (8 * (K + 2 * s))
    while a(n * K * 8) + 2 * a(n * s * 8) + 256 > cap:
        n -= 1
    while a((n + 1) * K * 8) + 2 * a((n + 1) * s * 8) + 256 <= cap:
        n += 1
    ids, dists, flags = _state(torch, n + 1, K, 4)
    out = _outputs(torch, n + 1, K, s)
    assert km.step_sample_noalloc(ids, dists, flags, 1, 1, s, *out) == -1
    ids, dists, flags = _state(torch, n, K, 4)  # ids within [0, n)
    out = _outputs(torch, n, K, s)
    assert km.step_sample_noalloc(ids, dists, flags, 1, 1, s, *out) == 0

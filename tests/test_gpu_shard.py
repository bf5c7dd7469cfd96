"""The sharded merge tree with the library's S-Merge: every rank count gives
the single-device knnm_merge_tree graph bit for bit (ranks simulated in one
process on this device, transfers through the loopback channel)."""
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


@pytest.mark.parametrize("world", [1, 2, 3, 4])
def test_sharded_tree_equals_single_device_tree(torch, orc, world):
    from paper_1908_00814_gb300 import build, knnm, shard
    build.build()
    ctx = knnm.Context(0)
    rows = [300, 280, 310, 290, 305, 295, 320]   # odd count: a block is carried up
    X = datagen.sift_like(sum(rows), 32, seed=17)
    K = 8
    G = np.concatenate([orc.bruteforce_knn(X[o:o + r], K)[0]
                        for o, r in zip(np.cumsum([0] + rows[:-1]), rows)])
    Xd = torch.from_numpy(X).cuda()
    Gd = torch.from_numpy(G).cuda()
    p = knnm.params(k=K, precision="bf16", max_iters=5, delta=0.0, seed=21)
    want_i, want_d, _ = ctx.merge_tree(Xd, rows, Gd, p)
    got_i, got_d = shard.simulate(ctx, Xd, Gd, rows, p, world)
    assert np.array_equal(got_i.cpu().numpy(), want_i.cpu().numpy())
    assert np.array_equal(got_d.cpu().numpy().view(np.uint32), want_d.cpu().numpy().view(np.uint32))
    ctx.close()

"""Host logic of the sharded merge tree (paper_1908_00814_gb300.shard): the
plan, the library's hash, and the transfers between ranks over gloo
(world size 2, CPU).  The S-Merge is replaced by a deterministic stand-in
that records the tree's order and seeds, so that the two-rank run must equal
the in-process run exactly; the GPU test compares the real merges with
knnm_merge_tree."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

from paper_1908_00814_gb300 import knnm, shard


def test_plan_mirrors_the_single_device_tree():
    for parts, world in ((1, 1), (2, 2), (7, 3), (8, 4), (13, 2), (64, 8), (5, 8)):
        rows = [10 + i for i in range(parts)]
        levels = shard.plan(rows, world)
        merges = [s for lv in levels for s in lv if s[0] == "merge"]
        assert len(merges) == parts - 1
        # merge j of a level pairs blocks 2j and 2j+1; the left block keeps its owner
        for lv in levels:
            for s in lv:
                if s[0] == "merge":
                    _, j, a, b = s
                    assert a.start + a.rows == b.start and a.owner <= b.owner
        owners = [shard.part_owner(p, parts, world) for p in range(parts)]
        assert owners == sorted(owners) and owners[0] == 0


def test_library_hash_is_the_oracle_hash(orc):
    rng = np.random.default_rng(1)
    for _ in range(50):
        w = [int(x) for x in rng.integers(0, 2 ** 63, size=5)]
        assert knnm.hash64(*w) == orc.hash64(*w)


def fake_merge(S1, G1, S2, G2, q):
    """Stand-in S-Merge: the lists side by side (right ids shifted past the
    left rows), every distance the merge's seed: the result records the order
    of the merges and their seeds."""
    ids = torch.cat([G1, G2 + S1.shape[0]]).to(torch.int32)
    dists = torch.full(ids.shape, float(q.seed % 1000003), dtype=torch.float32)
    return ids, dists


def _data(parts, K=4, d=3):
    rows = [6 + (i * 5) % 7 for i in range(parts)]
    n = sum(rows)
    S = torch.arange(n * d, dtype=torch.float32).reshape(n, d)
    G = torch.cat([torch.arange(r * K, dtype=torch.int32).reshape(r, K) % r for r in rows])
    return rows, S, G


def _worker(rank, world, port, parts, out_path):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    rows, S, G = _data(parts)
    owners = [shard.part_owner(i, parts, world) for i in range(parts)]
    mine = [i for i in range(parts) if owners[i] == rank]
    lo = sum(rows[:mine[0]]) if mine else 0
    n = sum(rows[i] for i in mine)
    p = knnm.params(k=4, seed=11)
    res = shard.merge_tree_sharded(None, S[lo:lo + n], G[lo:lo + n], rows, p, rank=rank,
                                   world=world, comm=shard.TorchComm("cpu"), merge=fake_merge)
    if rank == 0:
        torch.save(res, out_path)
    dist.barrier()
    dist.destroy_process_group()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


@pytest.mark.parametrize("parts", [2, 5, 8])
def test_two_ranks_over_gloo_equal_one_process(tmp_path, parts):
    rows, S, G = _data(parts)
    p = knnm.params(k=4, seed=11)
    want = shard.simulate(None, S, G, rows, p, world=1, merge=fake_merge)
    also = shard.simulate(None, S, G, rows, p, world=2, merge=fake_merge)
    assert torch.equal(want[0], also[0]) and torch.equal(want[1], also[1])
    out = tmp_path / "res.pt"
    mp.start_processes(_worker, args=(2, _free_port(), parts, str(out)), nprocs=2,
                       start_method="spawn")
    got = torch.load(out)
    assert torch.equal(got[0], want[0]) and torch.equal(got[1], want[1])
    # the seeds of the root: merge 0 of the last level
    levels = len(shard.plan(rows, 1))
    assert float(got[1][0, 0]) == float(knnm.hash64(11, levels - 1, 6, 0, 0) % 1000003)

"""Host logic of the sharded S-Merge (paper_1908_00814_gb300.shard): nodes
partitioned by id range, replicated init and sampling, each rank's local join
over its own nodes, partial lists sent to their owners (all-to-all), the
owners' top-K union, an all-reduce of c_t and an all-gather of the rows.

The per-rank steps here are the CPU oracle's (init, sample, join restricted to
the rank's nodes by zeroing the other nodes' candidate counts, final) and a
plain numpy top-K union, so the whole protocol runs on CPU: in one process
with the ranks in lock-step, and over gloo with two processes.  Both must give
the oracle's single-process S-Merge bit for bit, with the same c_t per round
(UpdateNN is the top K of the round-start list and all proposals, so unions of
partial lists are exact).  The GPU test runs the same driver on the library's
steps."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

from paper_1908_00814_gb300 import datagen, shard


def _ordered(d):
    u = np.ascontiguousarray(d, np.float32).view(np.uint32).astype(np.uint64)
    return np.where(u & 0x80000000, (~u) & 0xFFFFFFFF, u | 0x80000000)


def np_union(part_ids, part_dists, start_ids, start_dists, start_flags):
    """First K distinct (distance, id) entries of all parts of each row; an
    entry already in the row's start list keeps its flag, any other is new."""
    P, n, K = part_ids.shape
    oi = np.full((n, K), -1, np.int32)
    od = np.full((n, K), np.inf, np.float32)
    of = np.ones((n, K), np.uint8)
    c = 0
    for v in range(n):
        ids = part_ids[:, v].ravel()
        ds = part_dists[:, v].ravel()
        order = np.lexsort((ids.astype(np.int64), _ordered(ds)))
        start = {(int(i), int(b)): int(f) for i, b, f in
                 zip(start_ids[v], np.ascontiguousarray(start_dists[v]).view(np.uint32),
                     start_flags[v])}
        seen, m = set(), 0
        for j in order:
            i = int(ids[j])
            if i < 0 or i in seen:
                continue
            seen.add(i)
            oi[v, m], od[v, m] = i, ds[j]
            key = (i, int(np.float32(ds[j]).view(np.uint32)))
            if key in start:
                of[v, m] = start[key]
            else:
                c += 1
            m += 1
            if m == K:
                break
    return oi, od, of, c


class OracleRounds:
    """The per-rank steps on the CPU oracle; state as CPU tensors sharing
    memory with the oracle's arrays."""

    def __init__(self, orc, X, n1, G1, G2, K, seed, s):
        self.orc, self.X, self.n1, self.G1, self.G2 = orc, X, n1, G1, G2
        self.K, self.seed, self.s = K, seed, s

    def _st(self, state):
        ids, dists, flags = (t.numpy() for t in state)
        return self.orc.State(ids, dists, flags, *self.rear)

    def init(self):
        orc = self.orc
        st = orc.init(orc.SYMMETRIC, self.X, self.n1, self.K, orc.keep_count(self.K, 0.5),
                      self.seed, G1=self.G1, G2=self.G2)
        self.rear = (st.rear_ids, st.rear_dists)
        return [torch.from_numpy(st.ids), torch.from_numpy(st.dists), torch.from_numpy(st.flags)]

    def sample(self, state, t):
        return self.orc.sample(self._st(state), self.seed, t, self.s)

    def join_rows(self, state, cands, lo, hi):
        new_ids, new_cnt, old_ids, old_cnt = cands
        own = (np.arange(len(new_cnt)) >= lo) & (np.arange(len(new_cnt)) < hi)
        self.orc.join(self.orc.SYMMETRIC, self.X, self.n1, self._st(state),
                      (new_ids, np.where(own, new_cnt, 0), old_ids, np.where(own, old_cnt, 0)))

    def union(self, part_ids, part_dists, start):
        oi, od, of, c = np_union(part_ids.numpy(), part_dists.numpy(),
                                 *(t.numpy() for t in start))
        return torch.from_numpy(oi), torch.from_numpy(od), torch.from_numpy(of), c

    def final(self, state):
        ids, dists = self.orc.final(self._st(state))
        return torch.from_numpy(ids), torch.from_numpy(dists)


def _case(orc, n1=260, n2=240, d=8, K=6, seed=3):
    X = datagen.gaussian_mixture(n1 + n2, d, n_comp=5, seed=seed)
    G1, _ = orc.bruteforce_knn(X[:n1], K)
    G2, _ = orc.bruteforce_knn(X[n1:], K)
    return X, n1, G1, G2, K


class P:
    """The parameters the driver reads (k, max_iters, delta)."""

    def __init__(self, k, max_iters, delta):
        self.k, self.max_iters, self.delta = k, max_iters, delta


def test_node_ranges_partition_the_rows():
    for N in (1, 7, 100, 1001):
        for world in (1, 2, 3, 8):
            r = [shard.node_range(N, k, world) for k in range(world)]
            assert r[0][0] == 0 and r[-1][1] == N
            assert all(a[1] == b[0] for a, b in zip(r, r[1:]))
            assert max(h - l for l, h in r) - min(h - l for l, h in r) <= 1


@pytest.mark.parametrize("world", [1, 2, 3, 4])
def test_lockstep_ranks_equal_single_process_merge(orc, world):
    X, n1, G1, G2, K = _case(orc)
    rounds, s = 6, 3
    ref_i, ref_d, ref_st = orc.merge_symmetric(X[:n1], G1, X[n1:], G2, K, max_iters=rounds,
                                               delta=0.0, seed=9)
    steps = [OracleRounds(orc, X, n1, G1, G2, K, 9, s) for _ in range(world)]
    ids, dists, hist = shard.simulate_smerge(steps, len(X), P(K, rounds, 0.0), world)
    assert np.array_equal(ids.numpy(), ref_i)
    assert np.array_equal(dists.numpy().view(np.uint32), ref_d.view(np.uint32))
    assert hist == ref_st["updates"]


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out_path):
    import torch.distributed as dist

    import oracle as orc
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        X, n1, G1, G2, K = _case(orc)
        steps = OracleRounds(orc, X, n1, G1, G2, K, 9, 3)
        gen = shard.smerge_rank(steps, len(X), P(K, 6, 0.0), rank, world)
        ids, dists, hist = shard.run_collectives(gen, len(X), rank, world)
        np.savez(f"{out_path}.{rank}.npz", ids=ids.numpy(), dists=dists.numpy(),
                 hist=np.array(hist))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_equal_single_process_merge(orc, tmp_path):
    world = 2
    out = str(tmp_path / "res")
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world,
                       start_method="spawn")
    X, n1, G1, G2, K = _case(orc)
    ref_i, ref_d, ref_st = orc.merge_symmetric(X[:n1], G1, X[n1:], G2, K, max_iters=6,
                                               delta=0.0, seed=9)
    for r in range(world):
        res = np.load(f"{out}.{r}.npz")
        assert np.array_equal(res["ids"], ref_i)
        assert np.array_equal(res["dists"].view(np.uint32), ref_d.view(np.uint32))
        assert res["hist"].tolist() == ref_st["updates"]

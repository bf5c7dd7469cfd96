"""Merge tree over several ranks, one GPU each (Sec. 1 and Sec. 3: a graph over
a large set made from graphs built independently on its parts).

The tree is the one knnm_merge_tree runs on one device: level by level,
neighbouring blocks (0, 1), (2, 3), ... are joined by S-Merge (Alg. 1), an odd
last block waits for the next level, and merge j of level l runs with seed
H(seed, l, 6, j, 0).  Here the parts are spread over the ranks in contiguous
runs; a merge runs on the rank that holds its left block, and the right
block's rows and lists are sent there first when another rank holds them.
Ownership only moves towards lower ranks, so the root ends on rank 0 and the
result is bit for bit the single-device tree's.

Only host orchestration lives here: every merge is the library's
knnm_merge_symmetric, every seed the library's hash.
"""
from __future__ import annotations

from dataclasses import dataclass

from . import knnm


@dataclass
class Block:
    start: int  # first row (global)
    rows: int
    owner: int  # rank holding its rows and lists


def part_owner(part: int, parts: int, world: int) -> int:
    """Contiguous runs of parts per rank."""
    return part * world // parts


def plan(part_rows, world):
    """The levels of the tree: per level a list of ("merge", j, a, b) and
    ("carry", a) steps over Blocks, in the order every rank executes them."""
    parts = len(part_rows)
    blocks, off = [], 0
    for p, r in enumerate(part_rows):
        blocks.append(Block(off, int(r), part_owner(p, parts, world)))
        off += int(r)
    levels = []
    while len(blocks) > 1:
        steps, nxt = [], []
        for j in range(0, len(blocks), 2):
            a = blocks[j]
            if j + 1 == len(blocks):
                steps.append(("carry", a))
                nxt.append(a)
                continue
            b = blocks[j + 1]
            steps.append(("merge", j // 2, a, b))
            nxt.append(Block(a.start, a.rows + b.rows, a.owner))
        levels.append(steps)
        blocks = nxt
    return levels


class LoopbackComm:
    """Ranks of one process run one after another, highest rank first: a rank
    only receives from higher ranks, whose sends are already queued."""

    def __init__(self):
        self.queues = {}

    def send(self, tensors, src, dst):
        self.queues.setdefault((src, dst), []).append([t.clone() for t in tensors])

    def recv(self, src, dst, like):
        return self.queues[(src, dst)].pop(0)


class TorchComm:
    """Point-to-point transfers over torch.distributed (gloo: host copies)."""

    def __init__(self, device):
        import torch.distributed as dist
        self.dist = dist
        self.device = device
        self.host = dist.get_backend() == "gloo"

    def send(self, tensors, src, dst):
        import torch
        for t in tensors:
            shape = torch.tensor(list(t.shape) + [0] * (2 - t.dim()), dtype=torch.int64)
            self.dist.send(shape, dst)
            self.dist.send(t.cpu() if self.host else t.contiguous(), dst)

    def recv(self, src, dst, like):
        import torch
        out = []
        for dtype in like:
            shape = torch.empty(2, dtype=torch.int64)
            self.dist.recv(shape, src)
            dims = [int(x) for x in shape.tolist() if x > 0] or [0]
            t = torch.empty(dims, dtype=dtype, device="cpu" if self.host else self.device)
            self.dist.recv(t, src)
            out.append(t.to(self.device))
        return out


def merge_tree_sharded(ctx, S_local, G_local, part_rows, p, rank=0, world=1, comm=None,
                       merge=None):
    """One rank's share of the sharded merge tree.

    S_local, G_local: the rows and lists (ids local to each part) of the parts
    this rank holds (part_owner), concatenated in part order.  p: knnm.Params.
    merge(S1, G1, S2, G2, params) -> (ids, dists) runs one S-Merge (default:
    the library's, on ctx).  Returns (ids, dists) of the whole graph on rank 0
    and None on the other ranks."""
    import copy

    import torch
    parts = len(part_rows)
    if merge is None:
        def merge(S1, G1, S2, G2, q):
            ids, dists, _ = ctx.merge_symmetric(S1, G1, S2, G2, q)
            return ids, dists
    held, off = {}, 0
    starts = [0]
    for r in part_rows[:-1]:
        starts.append(starts[-1] + int(r))
    for part in range(parts):
        if part_owner(part, parts, world) == rank:
            n = int(part_rows[part])
            held[starts[part]] = (S_local[off:off + n], G_local[off:off + n], None)
            off += n
    if parts == 1:
        if rank != 0:
            return None
        ids, dists, _ = ctx.merge_tree(S_local, part_rows, G_local, p)
        return ids, dists
    for level, steps in enumerate(plan(part_rows, world)):
        for step in steps:
            if step[0] == "carry":
                continue
            _, j, a, b = step
            if a.owner != b.owner:
                if rank == b.owner:
                    Sb, Gb, _ = held.pop(b.start)
                    comm.send([Sb, Gb], rank, a.owner)
                elif rank == a.owner:
                    Sb, Gb = comm.recv(b.owner, rank, [S_local.dtype, G_local.dtype])
                    held[b.start] = (Sb, Gb, None)
            if rank != a.owner:
                continue
            Sa, Ga, _ = held.pop(a.start)
            Sb, Gb, _ = held.pop(b.start)
            q = copy.copy(p)
            q.seed = knnm.hash64(p.seed, level, 6, j, 0)
            ids, dists = merge(Sa.contiguous(), Ga.contiguous(), Sb.contiguous(), Gb.contiguous(),
                               q)
            held[a.start] = (torch.cat([Sa, Sb]), ids, dists)
    if rank != 0:
        return None
    _, ids, dists = held[0]
    return ids, dists


def simulate(ctx, S, G, part_rows, p, world, merge=None):
    """All ranks of a sharded tree in this process, on this device (highest
    rank first, transfers through a LoopbackComm); returns rank 0's result."""
    comm = LoopbackComm()
    parts = len(part_rows)
    out = None
    for rank in reversed(range(world)):
        rows = [part_owner(i, parts, world) == rank for i in range(parts)]
        lo = sum(int(r) for i, r in enumerate(part_rows) if i < rows.index(True)) \
            if any(rows) else 0
        n = sum(int(r) for i, r in enumerate(part_rows) if rows[i])
        res = merge_tree_sharded(ctx, S[lo:lo + n], G[lo:lo + n], part_rows, p, rank=rank,
                                 world=world, comm=comm, merge=merge)
        if rank == 0:
            out = res
    return out


# ---------------------------------------------------------------------------
# Sharded S-Merge (Alg. 1 over several ranks, one GPU each)
# ---------------------------------------------------------------------------
#
# Nodes are partitioned by id range; the read-only vectors and the input graphs
# are on every rank.  Init (Divide / Append) and each round's sampler run on
# every rank on the full round-start lists (they are deterministic, so every
# rank holds the same candidate sets); the local join, the dominant cost, runs
# on each rank for its own node range only, and its proposals update the
# rank's copy of every list.  The exchange of a round: an all-to-all that sends
# each row's partial list (top K of the round-start list and this rank's
# proposals) to the row's owner, the owner's top-K union of them (which is the
# top K of the round-start list and all proposals: synchronous UpdateNN), an
# all-reduce of c_t, and an all-gather of the owners' rows for the next round.
# The result is bit for bit the single-device knnm_merge_symmetric graph.


def node_range(N, rank, world):
    """Rows [lo, hi) owned by `rank`."""
    return N * rank // world, N * (rank + 1) // world


class LibraryRounds:
    """The per-rank steps of the sharded S-Merge on the library (device tensors)."""

    def __init__(self, ctx, S1, G1, S2, G2, p):
        import torch
        self.ctx, self.p = ctx, p
        self.X = torch.cat([S1, S2]).contiguous()
        self.n1 = S1.shape[0]
        self.G1, self.G2 = G1, G2
        self.s = knnm.list_widths(p, knnm.SYMMETRIC, self.n1)[2]

    def init(self):
        ids, dists, flags, rid, rd = self.ctx.step_init(knnm.SYMMETRIC, self.X, self.n1, self.G1,
                                                        self.G2, self.p)
        self.rear = (rid, rd)
        return [ids, dists, flags]

    def sample(self, state, t):
        ids, dists, flags = state
        return self.ctx.step_sample(ids, dists, flags, self.p.seed, t, self.s)

    def join_rows(self, state, cands, lo, hi):
        ids, dists, flags = state
        return self.ctx.step_join_rows(knnm.SYMMETRIC, self.X, self.n1, self.p, ids, dists, flags,
                                       cands, lo, hi)

    def union(self, part_ids, part_dists, start):
        return self.ctx.step_union(part_ids, part_dists, *start)

    def final(self, state):
        return self.ctx.step_final(state[0], state[1], *self.rear)


def smerge_rank(steps, N, p, rank, world):
    """One rank's share of the sharded S-Merge, as a generator: it yields its
    collective requests and receives their results (see run_collectives /
    simulate_smerge).  Returns (ids, dists, c_t per round) on every rank."""
    import torch
    K = p.k
    lo, hi = node_range(N, rank, world)
    state = steps.init()
    history = []
    for t in range(1, p.max_iters + 1):
        cands = steps.sample(state, t)
        start = [a[lo:hi].clone() for a in state]      # round-start rows of this rank
        steps.join_rows(state, cands, lo, hi)
        part_ids, part_dists = yield ("rows_to_owners", state[0], state[1])
        ids, dists, flags, c_own = steps.union(part_ids, part_dists, start)
        c = yield ("sum", c_own)
        state = list((yield ("gather_rows", ids, dists, flags)))
        history.append(int(c))
        if c <= p.delta * N * K:
            break
    ids, dists = steps.final(state)
    return ids, dists, history


def _rows_of(a, lo, hi):
    return a[lo:hi]


def simulate_smerge(steps_per_rank, N, p, world):
    """Every rank of a sharded S-Merge in this process (on one device), in
    lock-step: each collective request is served once all ranks made it.
    Returns rank 0's (ids, dists, c_t history)."""
    import torch
    gens = [smerge_rank(steps_per_rank[r], N, p, r, world) for r in range(world)]
    reqs = [next(g) for g in gens]
    ranges = [node_range(N, r, world) for r in range(world)]
    results = [None] * world
    while True:
        kind = reqs[0][0]
        assert all(r[0] == kind for r in reqs)
        if kind == "rows_to_owners":
            outs = []
            for o, (lo, hi) in enumerate(ranges):
                outs.append((torch.stack([_rows_of(reqs[q][1], lo, hi) for q in range(world)]),
                             torch.stack([_rows_of(reqs[q][2], lo, hi) for q in range(world)])))
        elif kind == "sum":
            total = sum(int(r[1]) for r in reqs)
            outs = [total] * world
        else:  # gather_rows
            full = [torch.cat([reqs[q][i] for q in range(world)]) for i in (1, 2, 3)]
            outs = [[f.clone() for f in full] for _ in range(world)]
        done = 0
        for r, g in enumerate(gens):
            try:
                reqs[r] = g.send(outs[r])
            except StopIteration as stop:
                results[r] = stop.value
                done += 1
        if done == world:
            return results[0]
        assert done == 0, "ranks left the round loop at different rounds"


def run_collectives(gen, N, rank, world, device=None):
    """Drives one rank's smerge_rank generator over torch.distributed
    (all_to_all_single, all_reduce, all_gather; gloo or NCCL).  Returns the
    generator's result."""
    import torch
    import torch.distributed as dist
    ranges = [node_range(N, r, world) for r in range(world)]
    lo, hi = ranges[rank]
    own = hi - lo
    most = max(h - l for l, h in ranges)
    host = dist.get_backend() == "gloo"

    def to_comm(t):
        return t.cpu().contiguous() if host else t.contiguous()

    def back(t, like):
        return t.to(like.device)

    req = next(gen)
    while True:
        kind = req[0]
        if kind == "rows_to_owners":
            outs = []
            for a in (req[1], req[2]):
                K = a.shape[1]
                src = to_comm(a).reshape(-1)
                dst = torch.empty(world * own * K, dtype=src.dtype, device=src.device)
                dist.all_to_all_single(dst, src, [own * K] * world,
                                       [(h - l) * K for l, h in ranges])
                outs.append(back(dst.reshape(world, own, K), a))
            res = tuple(outs)
        elif kind == "sum":
            t = torch.tensor([int(req[1])], dtype=torch.int64,
                             device="cpu" if host else device)
            dist.all_reduce(t)
            res = int(t.item())
        else:  # gather_rows: pad to the largest range, gather, strip
            res = []
            for a in req[1:]:
                K = a.shape[1]
                pad = torch.zeros((most, K), dtype=a.dtype, device=a.device)
                pad[:own] = a
                buf = torch.empty((world * most, K), dtype=a.dtype,
                                  device="cpu" if host else a.device)
                dist.all_gather_into_tensor(buf, to_comm(pad))
                full = torch.cat([buf[q * most:q * most + (h - l)] for q, (l, h) in enumerate(ranges)])
                res.append(back(full, a))
        try:
            req = gen.send(res)
        except StopIteration as stop:
            return stop.value

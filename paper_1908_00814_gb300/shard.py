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

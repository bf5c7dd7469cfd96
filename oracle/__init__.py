"""CPU oracle for the k-NN graph merge (S-Merge, Alg. 1; J-Merge, Alg. 2).

TEST INFRASTRUCTURE ONLY.  The plain C restatement in ``knnm_oracle.c`` is
compiled by :func:`build` and called through ctypes.  Only the test suite, the
smoke check and the CPU-baseline leg of the benchmark may import this package;
the CUDA library never does, and this package never imports the CUDA library.

Every function here follows the paper's steps (see the header of
``knnm_oracle.c`` for the readings taken where the paper is silent).  The
numpy helpers at the bottom (exact k-NN in float64, recall@k, phi) are plain
definitions: recall@k is Sec. 5.1's equation, phi is Sec. 3.4's sum of list
distances.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_SRC = _HERE / "knnm_oracle.c"
_LIB_PATH = _HERE / "_build" / "libknnm_oracle.so"

L2, IP, COS, L1, CHI2, JACCARD = 0, 1, 2, 3, 4, 5
SYMMETRIC, JOINT = 0, 1
FLAG_OLD, FLAG_NEW = 0, 1
STREAM_FWD_NEW, STREAM_REV_NEW, STREAM_REV_OLD, STREAM_INIT = 0, 1, 2, 3

_lib = None


def build(force: bool = False) -> Path:
    """Compile the oracle with gcc (no fused multiply-add contraction)."""
    _LIB_PATH.parent.mkdir(parents=True, exist_ok=True)
    if force or not _LIB_PATH.exists() or _LIB_PATH.stat().st_mtime < _SRC.stat().st_mtime:
        tmp = _LIB_PATH.with_suffix(f".{os.getpid()}.tmp.so")
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
               "-fno-fast-math", str(_SRC), "-o", str(tmp), "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(str(_LIB_PATH))
        P = ctypes.c_void_p
        i64, i32, u64, f32 = ctypes.c_int64, ctypes.c_int, ctypes.c_uint64, ctypes.c_float
        L.orc_distance.argtypes = [i32, P, P, i32]
        L.orc_distance.restype = f32
        L.orc_splitmix64_next.argtypes = [ctypes.POINTER(ctypes.c_uint64)]
        L.orc_splitmix64_next.restype = u64
        L.orc_hash.argtypes = [u64, u64, u64, u64, u64]
        L.orc_hash.restype = u64
        L.orc_init.argtypes = [i32, P, i64, i64, i32, i32, P, P, i32, i32, u64, P, P, P, P, P]
        L.orc_sample.argtypes = [i64, i32, P, P, u64, i32, i32, i32, i32, i32, P, P, P, P]
        L.orc_join.argtypes = [i32, P, i64, i64, i32, i32, i32, P, P, P, i32, i32, P, P, P, P,
                               ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]
        L.orc_final.argtypes = [i64, i32, P, P, i32, P, P, P, P]
        L.orc_merge.argtypes = [i32, P, i64, i64, i32, i32, P, P, i32, f32, f32, i32, f32, u64,
                                i32, P, P, P, P, ctypes.POINTER(ctypes.c_int)]
        L.orc_permute.argtypes = [i64, u64, P]
        L.orc_bruteforce_knn.argtypes = [P, i64, i32, i32, i32, P, P]
        L.orc_bruteforce_merge.argtypes = [P, i64, i64, i32, i32, P, P, i32, P, P]
        L.orc_diversify.argtypes = [P, i64, i32, i32, P, i32, i32, P, i64, P, P, P, P]
        L.orc_search.argtypes = [P, i64, i32, i32, i32, P, P, P, P, i64, P, i32, i32, u64, P, P,
                                 P]
        for name in ("orc_init", "orc_sample", "orc_join", "orc_final", "orc_merge",
                     "orc_permute", "orc_bruteforce_knn", "orc_bruteforce_merge",
                     "orc_diversify", "orc_search"):
            getattr(L, name).restype = ctypes.c_int
        _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f32(x):
    return np.ascontiguousarray(x, dtype=np.float32)


def _i32(x):
    return np.ascontiguousarray(x, dtype=np.int32)


def _check(rc, what):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with code {rc}")


# ---------------------------------------------------------------- primitives

def distance(metric: int, a, b) -> np.float32:
    a, b = _f32(a), _f32(b)
    return np.float32(lib().orc_distance(metric, _ptr(a), _ptr(b), a.shape[-1]))


def splitmix64(seed: int, count: int) -> list[int]:
    state = ctypes.c_uint64(seed)
    return [int(lib().orc_splitmix64_next(ctypes.byref(state))) for _ in range(count)]


def hash64(seed, t, stream, owner, member) -> int:
    return int(lib().orc_hash(seed, t, stream, owner, member))


def keep_count(K: int, keep_ratio: float) -> int:
    return int(float(np.float32(keep_ratio)) * K)


def sample_count(K: int, sample_rate: float) -> int:
    return max(1, int(float(np.float32(sample_rate)) * K))


# ---------------------------------------------------------------- round steps

class State:
    """Working lists of one merge: ids/dists/flags [n][K], rear lists [n][Kr]."""

    def __init__(self, ids, dists, flags, rear_ids, rear_dists):
        self.ids, self.dists, self.flags = ids, dists, flags
        self.rear_ids, self.rear_dists = rear_ids, rear_dists

    def copy(self):
        return State(self.ids.copy(), self.dists.copy(), self.flags.copy(),
                     self.rear_ids.copy(), self.rear_dists.copy())


def init(mode, X, n1, K, K_keep, seed, metric=L2, G1=None, G2=None) -> State:
    X = _f32(X)
    n, d = X.shape
    Kr = K - K_keep
    ids = np.empty((n, K), np.int32)
    dists = np.empty((n, K), np.float32)
    flags = np.empty((n, K), np.uint8)
    rid = np.empty((n, max(Kr, 0)), np.int32)
    rd = np.empty((n, max(Kr, 0)), np.float32)
    G1 = None if G1 is None else _i32(G1)
    G2 = None if G2 is None else _i32(G2)
    rc = lib().orc_init(mode, _ptr(X), n, n1, d, metric, _ptr(G1), _ptr(G2), K, K_keep, seed,
                        _ptr(ids), _ptr(dists), _ptr(flags), _ptr(rid), _ptr(rd))
    _check(rc, "init")
    return State(ids, dists, flags, rid, rd)


def sample(state: State, seed, t, s, literal=False, cap_new=None, cap_old=None):
    """Round step 1.  Flips sampled flags in ``state`` and returns the new/old
    candidate lists as (new_ids, new_cnt, old_ids, old_cnt)."""
    n, K = state.ids.shape
    if cap_new is None:
        cap_new = n if literal else 2 * s
    if cap_old is None:
        cap_old = 1 if literal else K + s
    new_ids = np.full((n, cap_new), -1, np.int32)
    old_ids = np.full((n, cap_old), -1, np.int32)
    new_cnt = np.zeros(n, np.int32)
    old_cnt = np.zeros(n, np.int32)
    rc = lib().orc_sample(n, K, _ptr(state.ids), _ptr(state.flags), seed, t, s, int(literal),
                          cap_new, cap_old, _ptr(new_ids), _ptr(new_cnt), _ptr(old_ids),
                          _ptr(old_cnt))
    _check(rc, "sample")
    return new_ids, new_cnt, old_ids, old_cnt


def join(mode, X, n1, state: State, cands, metric=L2):
    """Round step 2 (local join + UpdateNN) in place.  Returns (c_t, dist_evals)."""
    X = _f32(X)
    n, d = X.shape
    K = state.ids.shape[1]
    new_ids, new_cnt, old_ids, old_cnt = (_i32(c) for c in cands)
    c = ctypes.c_int64(0)
    ev = ctypes.c_int64(0)
    rc = lib().orc_join(mode, _ptr(X), n, n1, d, metric, K, _ptr(state.ids), _ptr(state.dists),
                        _ptr(state.flags), new_ids.shape[1], old_ids.shape[1], _ptr(new_ids),
                        _ptr(new_cnt), _ptr(old_ids), _ptr(old_cnt), ctypes.byref(c),
                        ctypes.byref(ev))
    _check(rc, "join")
    return int(c.value), int(ev.value)


def final(state: State):
    n, K = state.ids.shape
    Kr = state.rear_ids.shape[1]
    out_ids = np.empty((n, K), np.int32)
    out_d = np.empty((n, K), np.float32)
    rc = lib().orc_final(n, K, _ptr(state.ids), _ptr(state.dists), Kr, _ptr(state.rear_ids),
                         _ptr(state.rear_dists), _ptr(out_ids), _ptr(out_d))
    _check(rc, "final")
    return out_ids, out_d


# ---------------------------------------------------------------- whole merges

def _merge(mode, X, n1, K, G1, G2, metric, keep_ratio, sample_rate, max_iters, delta, seed,
           literal):
    X = _f32(X)
    n, d = X.shape
    out_ids = np.empty((n, K), np.int32)
    out_d = np.empty((n, K), np.float32)
    c_hist = np.zeros(max(max_iters, 1), np.int64)
    e_hist = np.zeros(max(max_iters, 1), np.int64)
    rounds = ctypes.c_int(0)
    G1 = None if G1 is None else _i32(G1)
    G2 = None if G2 is None else _i32(G2)
    rc = lib().orc_merge(mode, _ptr(X), n, n1, d, metric, _ptr(G1), _ptr(G2), K, keep_ratio,
                         sample_rate, max_iters, delta, seed, int(literal), _ptr(out_ids),
                         _ptr(out_d), _ptr(c_hist), _ptr(e_hist), ctypes.byref(rounds))
    _check(rc, "merge")
    r = rounds.value
    return out_ids, out_d, {"rounds": r, "updates": c_hist[:r].tolist(),
                            "dist_evals": e_hist[:r].tolist()}


def merge_symmetric(S1, G1, S2, G2, K, metric=L2, keep_ratio=0.5, sample_rate=0.5, max_iters=10,
                    delta=0.0, seed=0, literal=False):
    """S-Merge (Alg. 1).  G1/G2 hold ids local to S1/S2; output ids are global."""
    X = np.concatenate([_f32(S1), _f32(S2)], axis=0)
    return _merge(SYMMETRIC, X, len(S1), K, G1, G2, metric, keep_ratio, sample_rate, max_iters,
                  delta, seed, literal)


def merge_joint(S1, G1, S_new, K, metric=L2, keep_ratio=0.5, sample_rate=0.5, max_iters=10,
                delta=0.0, seed=0, literal=False):
    """J-Merge (Alg. 2): the graph G1 of S1 is joined with the raw rows S_new."""
    X = np.concatenate([_f32(S1), _f32(S_new)], axis=0)
    return _merge(JOINT, X, len(S1), K, G1, None, metric, keep_ratio, sample_rate, max_iters,
                  delta, seed, literal)


def permute(n, seed) -> np.ndarray:
    """H-Merge sampling order: position r holds row perm[r] (Feistel bijection)."""
    perm = np.empty(n, np.int32)
    _check(lib().orc_permute(n, seed, _ptr(perm)), "permute")
    return perm


def hmerge(S, K, first_rows, metric=L2, sample_rate=0.5, max_iters=10, delta=0.0, seed=0):
    """H-Merge (Sec. 3.3), step by step: rows visited in a random order; an
    NN-Descent graph on the first `first_rows`; then each step J-Merges a raw block
    as large as the current graph (the whole rest when less than k + 1 rows would
    remain after it), so the graph doubles.  The
    growing graph keeps k entries per list (J-Merge never compares two rows of the
    existing graph, so lists cut to k/2 could not be refilled); each upper layer is
    kept as the first k/2 entries of its lists.  Merge l runs with seed
    H(seed, l, 8, 0, 0).  Returns (perm, layers, ids, dists): layers maps a layer's
    row count to its lists (ids = positions in the order; k/2 wide above the
    bottom); ids/dists are the bottom graph in positions."""
    S = _f32(S)
    n = len(S)
    perm = permute(n, seed)
    Xp = np.ascontiguousarray(S[perm])
    half = max(1, K // 2)
    m = min(first_rows, n)
    ids, dists, _ = build_graph(Xp[:m], K, metric=metric, sample_rate=sample_rate,
                                max_iters=max_iters, delta=delta, seed=hash64(seed, 0, 8, 0, 0))
    layers = {m: ids if m == n else np.ascontiguousarray(ids[:, :half])}
    level = 1
    while m < n:
        b = min(m, n - m)
        if 0 < n - m - b < K + 1:   # too small a rest for a J-Merge of its own
            b = n - m
        ids, dists, _ = merge_joint(Xp[:m], ids, Xp[m:m + b], K, metric=metric,
                                    sample_rate=sample_rate, max_iters=max_iters, delta=delta,
                                    seed=hash64(seed, level, 8, 0, 0))
        m += b
        layers[m] = ids if m == n else np.ascontiguousarray(ids[:, :half])
        level += 1
    return perm, layers, ids, dists


def diversify(S, G, max_degree, metric=L2, rows=None):
    """Graph diversification (Alg. 3, Sec. 3.4) of the k-NN graph G: each row's
    list and its reverse list, each in (distance, id) order, are diversified
    (first entry kept; a later one dropped when a kept entry is closer to it
    than the row is) and merged without repeats, cut to max_degree.  Returns
    (ids, dists, degree, evals) for `rows` (all rows when None)."""
    S, G = _f32(S), _i32(G)
    n, d = S.shape
    K = G.shape[1]
    r = None if rows is None else np.ascontiguousarray(rows, dtype=np.int64)
    m = n if r is None else len(r)
    ids = np.empty((m, max_degree), np.int32)
    dists = np.empty((m, max_degree), np.float32)
    deg = np.empty(m, np.int32)
    ev = ctypes.c_uint64(0)
    _check(lib().orc_diversify(_ptr(S), n, d, metric, _ptr(G), K, max_degree, _ptr(r), m,
                               _ptr(ids), _ptr(dists), _ptr(deg), ctypes.byref(ev)), "diversify")
    return ids, dists, deg, int(ev.value)


def search(S, layers, Q, ef, k_out, metric=L2, seed=0, query_index=None):
    """Top-down search (Sec. 3.4) of the queries Q on a hierarchy: `layers` is a
    list of id arrays from the top layer down, layer l covering the first
    len(layers[l]) rows of S (the bottom one all of them; ids < 0 are padding).
    Greedy descent above the bottom, best-first over an ef-entry rank list at the
    bottom.  Query q starts from the hash of its batch index, or of
    query_index[q] when given.  Returns (ids, dists, evals) with k_out entries
    per query."""
    S, Q = _f32(S), _f32(Q)
    n, d = S.shape
    rows = np.array([len(g) for g in layers], np.int64)
    width = np.array([g.shape[1] for g in layers], np.int32)
    flat = np.concatenate([_i32(g).ravel() for g in layers])
    nq = len(Q)
    ids = np.empty((nq, k_out), np.int32)
    dists = np.empty((nq, k_out), np.float32)
    ev = np.empty(nq, np.uint64)
    qi = None if query_index is None else np.ascontiguousarray(query_index, dtype=np.int64)
    _check(lib().orc_search(_ptr(S), n, d, metric, len(layers), _ptr(rows), _ptr(width),
                            _ptr(flat), _ptr(Q), nq, _ptr(qi), ef, k_out, seed, _ptr(ids),
                            _ptr(dists), _ptr(ev)), "search")
    return ids, dists, ev


def build_graph(S, K, metric=L2, sample_rate=0.5, max_iters=10, delta=0.0, seed=0,
                literal=False):
    """NN-Descent build = J-Merge with an empty existing graph."""
    return _merge(JOINT, _f32(S), 0, K, None, None, metric, 1.0, sample_rate, max_iters, delta,
                  seed, literal)


def bruteforce_knn(X, K, metric=L2):
    X = _f32(X)
    n, d = X.shape
    ids = np.empty((n, K), np.int32)
    dists = np.empty((n, K), np.float32)
    _check(lib().orc_bruteforce_knn(_ptr(X), n, d, metric, K, _ptr(ids), _ptr(dists)), "bf knn")
    return ids, dists


def bruteforce_merge(S1, G1, S2, G2, K, metric=L2):
    X = np.concatenate([_f32(S1), _f32(S2)], axis=0)
    n, d = X.shape
    ids = np.empty((n, K), np.int32)
    dists = np.empty((n, K), np.float32)
    _check(lib().orc_bruteforce_merge(_ptr(X), n, len(S1), d, metric, _ptr(_i32(G1)),
                                      _ptr(_i32(G2)), K, _ptr(ids), _ptr(dists)), "bf merge")
    return ids, dists


# ---------------------------------------------------------------- evaluation

def distances_f64(metric, X, q_rows, cand_ids):
    """float64 distances from X[q_rows[i]] to X[cand_ids[i, j]]."""
    A = np.asarray(X, np.float64)[np.asarray(q_rows)][:, None, :]
    B = np.asarray(X, np.float64)[np.asarray(cand_ids)]
    if metric == L2:
        return ((A - B) ** 2).sum(-1)
    if metric == L1:
        return np.abs(A - B).sum(-1)
    dot = (A * B).sum(-1)
    if metric == IP:
        return -dot
    na = np.sqrt((A * A).sum(-1))
    nb = np.sqrt((B * B).sum(-1))
    den = na * nb
    return np.where(den == 0, 1.0, 1.0 - dot / np.where(den == 0, 1.0, den))


def exact_knn_f64(X, queries, K, metric=L2, block=256, margin=16):
    """Exact k-NN of X[queries] within X (self excluded), float64 distances.

    Candidates are preselected with a blocked float64 expansion and their
    distances recomputed directly (for L1, directly throughout).  Returns
    (ids [q][K], dists [q][K]) in ascending distance, ties by id."""
    X64 = np.asarray(X, np.float64)
    queries = np.asarray(queries, np.int64)
    n = X64.shape[0]
    m = min(n - 1, K + margin)
    out_i = np.empty((len(queries), K), np.int64)
    out_d = np.empty((len(queries), K), np.float64)
    sq = (X64 * X64).sum(1)
    for b0 in range(0, len(queries), block):
        qb = queries[b0:b0 + block]
        Q = X64[qb]
        if metric == L1:
            D = np.empty((len(qb), n))
            for r in range(len(qb)):
                D[r] = np.abs(X64 - Q[r]).sum(1)
        elif metric == L2:
            D = sq[qb][:, None] + sq[None, :] - 2.0 * (Q @ X64.T)
        elif metric == IP:
            D = -(Q @ X64.T)
        else:
            nq = np.sqrt(sq[qb])[:, None] * np.sqrt(sq)[None, :]
            D = 1.0 - (Q @ X64.T) / np.where(nq == 0, 1.0, nq)
        D[np.arange(len(qb)), qb] = np.inf
        cand = np.argpartition(D, m - 1, axis=1)[:, :m]
        dd = distances_f64(metric, X64, qb, cand)
        for r in range(len(qb)):
            o = np.lexsort((cand[r], dd[r]))[:K]
            out_i[b0 + r] = cand[r][o]
            out_d[b0 + r] = dd[r][o]
    return out_i, out_d


def recall_at(X, queries, graph_ids, K, metric=L2, truth=None, rel_tol=1e-9):
    """recall@K (Sec. 5.1): returned ids among the first K of each sampled
    list that are true K nearest neighbours, over |queries|*K.  An id whose
    float64 distance ties the exact K-th distance (within rel_tol) counts."""
    queries = np.asarray(queries, np.int64)
    if truth is None:
        truth = exact_knn_f64(X, queries, K, metric)
    _, td = truth
    kth = td[:, K - 1]
    got = np.asarray(graph_ids)[queries][:, :K]
    dd = distances_f64(metric, X, queries, got)
    thr = kth + rel_tol * np.abs(kth)
    hits = 0
    for r in range(len(queries)):
        row_ids = got[r]
        valid = row_ids >= 0
        uniq = np.zeros(len(row_ids), bool)
        seen = set()
        for j, v in enumerate(row_ids):
            if valid[j] and v not in seen and v != queries[r]:
                uniq[j] = True
                seen.add(int(v))
        hits += int(np.sum(uniq & (dd[r] <= thr[r])))
    return hits / (len(queries) * K)


def phi(dists) -> float:
    """phi(G) of Sec. 3.4: sum of all list distances (float64)."""
    return float(np.asarray(dists, np.float64).sum())

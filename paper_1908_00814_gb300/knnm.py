"""Thin ctypes binding over libknnm.so (declared in include/knnm.h).

Only argument marshalling happens here: every step of a merge runs in the
library's CUDA kernels.  Arrays may be torch tensors (CUDA or CPU) or numpy
arrays; CUDA tensors are passed as device pointers, everything else as host
pointers (the library copies host data in and out inside the call).  Importing
this module does not load the library; the first call does, and raises if the
library has not been built (``paper_1908_00814_gb300.build``).
"""
from __future__ import annotations

import ctypes
from pathlib import Path

import numpy as np

_LIB_PATH = Path(__file__).resolve().parent / "libknnm.so"

L2, IP, COS, L1, CHI2, JACCARD = 0, 1, 2, 3, 4, 5
FP32, BF16_RERANK, FP16_RERANK = 0, 1, 2
SYMMETRIC, JOINT = 0, 1
OPT_GRAPHS, OPT_BUCKET_CAP, OPT_WAIT_POLLS, OPT_FAIL_ALLOC, OPT_TC_JOIN = 1, 2, 3, 4, 5
MAX_ROUNDS = 64
METRICS = {"l2": L2, "ip": IP, "cos": COS, "l1": L1, "chi2": CHI2, "jaccard": JACCARD}

ERRORS = {0: "ok", -1: "invalid argument", -2: "out of memory", -3: "CUDA error",
          -4: "timeout", -5: "not ready", -6: "device-side error"}


class Params(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int), ("metric", ctypes.c_int), ("precision", ctypes.c_int),
                ("max_iters", ctypes.c_int), ("sample_rate", ctypes.c_float),
                ("keep_ratio", ctypes.c_float), ("delta", ctypes.c_float),
                ("seed", ctypes.c_uint64)]


class Stats(ctypes.Structure):
    _fields_ = [("rounds", ctypes.c_int), ("kernel_launches", ctypes.c_int),
                ("updates", ctypes.c_int64 * MAX_ROUNDS),
                ("dist_evals", ctypes.c_int64 * MAX_ROUNDS),
                ("proposals", ctypes.c_int64 * MAX_ROUNDS),
                ("reranked", ctypes.c_int64 * MAX_ROUNDS),
                ("gathered", ctypes.c_int64 * MAX_ROUNDS),
                ("ms_sample", ctypes.c_float * MAX_ROUNDS),
                ("ms_join", ctypes.c_float * MAX_ROUNDS),
                ("ms_update", ctypes.c_float * MAX_ROUNDS),
                ("ms_init", ctypes.c_float), ("ms_rounds", ctypes.c_float),
                ("ms_final", ctypes.c_float), ("ms_total", ctypes.c_float),
                ("tc_rounds", ctypes.c_uint64),
                ("spilled", ctypes.c_int64 * MAX_ROUNDS)]

    def as_dict(self):
        r = self.rounds
        out = {"rounds": r, "kernel_launches": self.kernel_launches, "ms_init": self.ms_init,
               "ms_rounds": self.ms_rounds, "ms_final": self.ms_final, "ms_total": self.ms_total,
               "tc_rounds": [bool((self.tc_rounds >> t) & 1) for t in range(r)]}
        for name in ("updates", "dist_evals", "proposals", "reranked", "gathered", "ms_sample",
                     "ms_join", "ms_update", "spilled"):
            out[name] = list(getattr(self, name)[:r])
        return out


class ServerConfig(ctypes.Structure):
    _fields_ = [("slots", ctypes.c_int), ("use_graphs", ctypes.c_int),
                ("capacity_rows", ctypes.c_int64), ("max_batch_rows", ctypes.c_int64),
                ("hbm_reserve_bytes", ctypes.c_uint64)]


class RequestInfo(ctypes.Structure):
    _fields_ = [("req_id", ctypes.c_uint64), ("status", ctypes.c_int), ("rounds", ctypes.c_int),
                ("rows", ctypes.c_int64), ("snapshot_rows", ctypes.c_int64),
                ("snapshot_commits", ctypes.c_int64), ("commit_seq", ctypes.c_int64),
                ("commit_base", ctypes.c_int64), ("dist_evals", ctypes.c_int64),
                ("slot", ctypes.c_int), ("queue_ms", ctypes.c_double),
                ("run_ms", ctypes.c_double), ("latency_ms", ctypes.c_double),
                ("merge_ms", ctypes.c_double), ("init_ms", ctypes.c_float),
                ("rounds_ms", ctypes.c_float), ("final_ms", ctypes.c_float),
                ("commit_ms", ctypes.c_double)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64),
                ("failed", ctypes.c_int64), ("resident_rows", ctypes.c_int64),
                ("rows_completed", ctypes.c_int64), ("max_concurrent", ctypes.c_int64),
                ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double),
                ("busy_s", ctypes.c_double)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class GdStats(ctypes.Structure):
    _fields_ = [("dist_evals", ctypes.c_uint64), ("edges", ctypes.c_uint64),
                ("full_rows", ctypes.c_int64), ("max_in_degree", ctypes.c_int64),
                ("ms", ctypes.c_float)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class SearchStats(ctypes.Structure):
    _fields_ = [("dist_evals", ctypes.c_uint64), ("crowded_queries", ctypes.c_int64),
                ("ms", ctypes.c_float)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


_lib = None

# name -> (restype, argtypes) of every entry point in include/knnm.h
_P, _I, _I64, _U64, _F = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_uint64, ctypes.c_float
SIGNATURES = {
    "knnm_create": (_I, [ctypes.POINTER(ctypes.c_void_p), _I, _P]),
    "knnm_destroy": (_I, [_P]),
    "knnm_set_stream": (_I, [_P, _P]),
    "knnm_last_error": (ctypes.c_char_p, [_P]),
    "knnm_set_option": (_I, [_P, _I, _I]),
    "knnm_strerror": (ctypes.c_char_p, [_I]),
    "knnm_hash64": (_U64, [_U64, _U64, _U64, _U64, _U64]),
    "knnm_list_widths": (_I, [ctypes.POINTER(Params), _I, _I64, _P, _P, _P]),
    "knnm_default_params": (None, [ctypes.POINTER(Params)]),
    "knnm_merge_symmetric": (_I, [_P, _P, _I64, _P, _P, _I64, _P, _I, ctypes.POINTER(Params),
                                  _P, _P, ctypes.POINTER(Stats)]),
    "knnm_merge_joint": (_I, [_P, _P, _I64, _P, _P, _I64, _I, ctypes.POINTER(Params), _P, _P,
                              ctypes.POINTER(Stats)]),
    "knnm_build": (_I, [_P, _P, _I64, _I, ctypes.POINTER(Params), _P, _P,
                        ctypes.POINTER(Stats)]),
    "knnm_step_init": (_I, [_P, _I, _P, _I64, _P, _I64, _I64, _I, _P, _P, ctypes.POINTER(Params),
                            _P, _P, _P, _P, _P]),
    "knnm_step_sample": (_I, [_P, _I64, _I, _P, _P, _P, _U64, _I, _I, _I, _I, _P, _P, _P, _P]),
    "knnm_step_join": (_I, [_P, _I, _P, _I64, _P, _I64, _I64, _I, ctypes.POINTER(Params), _P, _P,
                            _P, _I, _I, _P, _P, _P, _P, ctypes.POINTER(ctypes.c_int64),
                            ctypes.POINTER(ctypes.c_int64)]),
    "knnm_step_final": (_I, [_P, _I64, _I, _P, _P, _I, _P, _P, _P, _P]),
    "knnm_step_join_rows": (_I, [_P, _I, _P, _I64, _P, _I64, _I64, _I, ctypes.POINTER(Params),
                                 _P, _P, _P, _I, _I, _P, _P, _P, _P, _I64, _I64,
                                 ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]),
    "knnm_step_union": (_I, [_P, _I64, _I, _I, _P, _P, _P, _P, _P, _P, _P, _P,
                             ctypes.POINTER(ctypes.c_int64)]),
    "knnm_step_tc_estimate": (_I, [_P, _P, _I64, _I, _I, _I, _P, _P, _I64, _P, _P, _P]),
    "knnm_step_sample_noalloc": (_I, [_P, _I64, _I, _P, _P, _P, _U64, _I, _I, _I, _I, _P, _P,
                                      _P, _P]),
    "knnm_merge_symmetric_sets": (_I, [_P, _P, _P, _I64, _I64, _I64, _P, _P,
                                       ctypes.POINTER(Params), _P, _P, ctypes.POINTER(Stats)]),
    "knnm_merge_joint_sets": (_I, [_P, _P, _P, _I64, _I64, _I64, _P, ctypes.POINTER(Params),
                                   _P, _P, ctypes.POINTER(Stats)]),
    "knnm_build_sets": (_I, [_P, _P, _P, _I64, _I64, ctypes.POINTER(Params), _P, _P,
                             ctypes.POINTER(Stats)]),
    "knnm_merge_tree": (_I, [_P, _P, _I64, _I, _I, _P, _P, ctypes.POINTER(Params), _P, _P,
                             ctypes.POINTER(Stats)]),
    "knnm_hmerge": (_I, [_P, _P, _I64, _I, _I64, ctypes.POINTER(Params), _P, _P, _P, _I, _P,
                         _P, ctypes.POINTER(Stats)]),
    "knnm_merge_scratch_bytes": (_I, [_P, _I, _I64, _I64, _I, ctypes.POINTER(Params),
                                      ctypes.POINTER(ctypes.c_uint64)]),
    "knnm_gather_rows": (_I, [_P, _P, _I64, _I, _P, _I64, _P]),
    "knnm_diversify": (_I, [_P, _P, _I64, _I, _P, _I, _I, _I, _P, _P, _P,
                            ctypes.POINTER(GdStats)]),
    "knnm_search_prepare": (_I, [_P, _P, _I64, _I, _P]),
    "knnm_search": (_I, [_P, _P, _I64, _I, _P, _I, _I, _P, _P, _P, _P, _I64, _I, _I, _U64, _P,
                         _P, _P, ctypes.POINTER(SearchStats)]),
    "knnm_server_create": (_I, [_I, _P, _I64, _P, _I, ctypes.POINTER(Params),
                                ctypes.POINTER(ServerConfig), ctypes.POINTER(ctypes.c_void_p)]),
    "knnm_server_submit": (_I, [_P, _P, _I64, _U64]),
    "knnm_server_wait": (_I, [_P, _U64, _I, _P, _P, ctypes.POINTER(RequestInfo)]),
    "knnm_server_drain": (_I, [_P, _I]),
    "knnm_server_get_stats": (_I, [_P, ctypes.POINTER(ServerStats)]),
    "knnm_server_resident": (_I, [_P, ctypes.POINTER(ctypes.c_int64), _P, _P, _P]),
    "knnm_server_last_error": (ctypes.c_char_p, [_P]),
    "knnm_server_destroy": (_I, [_P]),
}


def lib_path() -> Path:
    return _LIB_PATH


def lib():
    """Loads libknnm.so; raises if it is missing (there is no fallback path)."""
    global _lib
    if _lib is None:
        if not _LIB_PATH.exists():
            raise RuntimeError(f"{_LIB_PATH} is not built: run python -m "
                               "paper_1908_00814_gb300.build (no CPU fallback exists)")
        L = ctypes.CDLL(str(_LIB_PATH))
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


class KnnmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


def hash64(seed, t, stream, owner, member) -> int:
    """The library's counter-based hash H(seed, t, stream, owner, member)."""
    m = (1 << 64) - 1
    return int(lib().knnm_hash64(seed & m, t & m, stream & m, owner & m, member & m))


def list_widths(p: Params, mode: int, set_split: int):
    """(K_keep, Kr, s) that a merge with these parameters uses (knnm_list_widths)."""
    kk, kr, s = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    rc = lib().knnm_list_widths(ctypes.byref(p), mode, set_split, ctypes.byref(kk),
                                ctypes.byref(kr), ctypes.byref(s))
    if rc != 0:
        raise KnnmError(rc, "invalid merge parameters")
    return kk.value, kr.value, s.value


def params(k=20, metric="l2", precision="fp32", max_iters=10, sample_rate=0.5, keep_ratio=0.5,
           delta=0.001, seed=0) -> Params:
    p = Params()
    p.k = k
    p.metric = METRICS[metric] if isinstance(metric, str) else int(metric)
    p.precision = {"fp32": FP32, "bf16": BF16_RERANK, "fp16": FP16_RERANK}[precision] \
        if isinstance(precision, str) \
        else int(precision)
    p.max_iters = max_iters
    p.sample_rate = sample_rate
    p.keep_ratio = keep_ratio
    p.delta = delta
    p.seed = seed
    return p


def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _ptr(x):
    """Device or host pointer of a tensor / array (None stays None)."""
    if x is None:
        return None
    if _is_torch(x):
        assert x.is_contiguous(), "arrays must be contiguous"
        return ctypes.c_void_p(x.data_ptr())
    assert x.flags["C_CONTIGUOUS"], "arrays must be contiguous"
    return x.ctypes.data_as(ctypes.c_void_p)


def _current_stream(device):
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


class Context:
    """A library context bound to one device; follows torch's current stream."""

    def __init__(self, device: int = 0):
        self.device = device
        h = ctypes.c_void_p()
        rc = lib().knnm_create(ctypes.byref(h), device, None)
        if rc != 0:
            raise KnnmError(rc, "knnm_create failed")
        self.h = h

    def set_graphs(self, on: bool = True):
        """Replay each merge round as one captured CUDA graph."""
        self._check(lib().knnm_set_option(self.h, OPT_GRAPHS, int(on)))

    def set_option(self, option: int, value: int):
        """knnm_set_option (OPT_BUCKET_CAP, OPT_WAIT_POLLS, OPT_FAIL_ALLOC, ...)."""
        self._check(lib().knnm_set_option(self.h, option, int(value)))

    def close(self):
        if getattr(self, "h", None):
            lib().knnm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _sync_stream(self):
        try:
            import torch
            if torch.cuda.is_available():
                lib().knnm_set_stream(self.h, _current_stream(self.device))
        except ImportError:
            pass

    def _check(self, rc):
        if rc != 0:
            raise KnnmError(rc, lib().knnm_last_error(self.h).decode())

    # ------------------------------------------------------------ whole merges
    def _outputs(self, like, n, k, out=None):
        """Output ids [n, k] int32 and distances [n, k] float32: the caller's `out`
        pair (for example pinned host buffers, so that the library's copy back
        runs at full speed), checked, else new arrays where `like` lives."""
        if out is not None:
            ids, dists = out
            for a, dt, name in ((ids, "int32", "ids"), (dists, "float32", "dists")):
                shape = tuple(a.shape)
                dtype = str(a.dtype).replace("torch.", "")
                contiguous = a.is_contiguous() if _is_torch(a) else a.flags["C_CONTIGUOUS"]
                if shape != (n, k) or dtype != dt or not contiguous:
                    raise ValueError(f"out {name}: need a contiguous {dt} array of shape "
                                     f"({n}, {k}), got {dtype} {shape}")
            return ids, dists
        if _is_torch(like):
            import torch
            dev = like.device if like.is_cuda else "cpu"
            return (torch.empty((n, k), dtype=torch.int32, device=dev),
                    torch.empty((n, k), dtype=torch.float32, device=dev))
        return np.empty((n, k), np.int32), np.empty((n, k), np.float32)

    def merge_symmetric(self, S1, G1, S2, G2, p: Params, out=None):
        n1, d = S1.shape
        n2 = S2.shape[0]
        ids, dists = self._outputs(S1, n1 + n2, p.k, out)
        st = Stats()
        self._sync_stream()
        self._check(lib().knnm_merge_symmetric(self.h, _ptr(S1), n1, _ptr(G1), _ptr(S2), n2,
                                               _ptr(G2), d, ctypes.byref(p), _ptr(ids),
                                               _ptr(dists), ctypes.byref(st)))
        return ids, dists, st.as_dict()

    def merge_joint(self, S1, G1, S_new, p: Params, out=None):
        n1, d = S1.shape
        n2 = S_new.shape[0]
        ids, dists = self._outputs(S_new, n1 + n2, p.k, out)
        st = Stats()
        self._sync_stream()
        self._check(lib().knnm_merge_joint(self.h, _ptr(S1), n1, _ptr(G1), _ptr(S_new), n2, d,
                                           ctypes.byref(p), _ptr(ids), _ptr(dists),
                                           ctypes.byref(st)))
        return ids, dists, st.as_dict()

    # ------------------------------------------------------------ sets (Jaccard)
    # offsets [n+1] int64 and items int32: CUDA tensors (CSR rows, ascending items).
    def _set_outputs(self, offsets, n, k):
        import torch
        return (torch.empty((n, k), dtype=torch.int32, device=offsets.device),
                torch.empty((n, k), dtype=torch.float32, device=offsets.device))

    def merge_symmetric_sets(self, offsets, items, n1, G1, G2, p: Params):
        n = offsets.shape[0] - 1
        ids, dists = self._set_outputs(offsets, n, p.k)
        st = Stats()
        self._sync_stream()
        self._check(lib().knnm_merge_symmetric_sets(self.h, _ptr(offsets), _ptr(items),
                                                    items.shape[0], n1, n - n1, _ptr(G1),
                                                    _ptr(G2), ctypes.byref(p), _ptr(ids),
                                                    _ptr(dists), ctypes.byref(st)))
        return ids, dists, st.as_dict()

    def merge_joint_sets(self, offsets, items, n1, G1, p: Params):
        n = offsets.shape[0] - 1
        ids, dists = self._set_outputs(offsets, n, p.k)
        st = Stats()
        self._sync_stream()
        self._check(lib().knnm_merge_joint_sets(self.h, _ptr(offsets), _ptr(items),
                                                items.shape[0], n1, n - n1, _ptr(G1),
                                                ctypes.byref(p), _ptr(ids), _ptr(dists),
                                                ctypes.byref(st)))
        return ids, dists, st.as_dict()

    def build_sets(self, offsets, items, p: Params):
        n = offsets.shape[0] - 1
        ids, dists = self._set_outputs(offsets, n, p.k)
        st = Stats()
        self._sync_stream()
        self._check(lib().knnm_build_sets(self.h, _ptr(offsets), _ptr(items), items.shape[0], n,
                                          ctypes.byref(p), _ptr(ids), _ptr(dists),
                                          ctypes.byref(st)))
        return ids, dists, st.as_dict()

    def merge_tree(self, S, part_rows, G, p: Params):
        """Merge tree over consecutive parts of S (G: each part's graph, local ids).
        Stats: rounds = levels, per-round arrays = per-level sums."""
        n, d = S.shape
        rows = np.ascontiguousarray(np.asarray(part_rows, dtype=np.int64))
        ids, dists = self._outputs(S, n, p.k)
        st = Stats()
        self._sync_stream()
        self._check(lib().knnm_merge_tree(self.h, _ptr(S), n, d, len(rows), _ptr(rows), _ptr(G),
                                          ctypes.byref(p), _ptr(ids), _ptr(dists),
                                          ctypes.byref(st)))
        return ids, dists, st.as_dict()

    def hmerge(self, S, first_rows, p: Params, layers=()):
        """H-Merge: returns (perm, ids, dists, layer_lists, stats); ids/dists are the
        bottom graph and the upper layers' k/2 lists, rows and ids as positions in
        the visiting order perm."""
        n, d = S.shape
        K, half = p.k, p.k // 2
        perm = np.empty(n, np.int32)
        ids = np.empty((n, K), np.int32)
        dists = np.empty((n, K), np.float32)
        rows = np.ascontiguousarray(np.asarray(list(layers), dtype=np.int64))
        lay = np.empty(max(1, int(rows.sum())) * half, np.int32)
        st = Stats()
        self._sync_stream()
        self._check(lib().knnm_hmerge(self.h, _ptr(S), n, d, first_rows, ctypes.byref(p),
                                      _ptr(perm), _ptr(ids), _ptr(dists), len(rows),
                                      _ptr(rows) if len(rows) else None,
                                      _ptr(lay) if len(rows) else None, ctypes.byref(st)))
        out, off = {}, 0
        for m in rows.tolist():
            out[m] = lay[off * half:(off + m) * half].reshape(m, half)
            off += m
        return perm, ids, dists, out, st.as_dict()

    # ------------------------------------------- diversification and search
    # Sec. 3.4.  All arrays: CUDA torch tensors.
    def gather_rows(self, S, perm, n=None):
        """out[r] = S[perm[r]] for the first n entries of perm."""
        import torch
        n_src, d = S.shape
        n = perm.shape[0] if n is None else n
        out = torch.empty((n, d), dtype=torch.float32, device=S.device)
        self._sync_stream()
        self._check(lib().knnm_gather_rows(self.h, _ptr(S), n_src, d, _ptr(perm), n, _ptr(out)))
        return out

    def diversify(self, S, G, max_degree, metric="l2"):
        """Alg. 3 on G's lists and reverse lists; returns (ids, dists, degree, stats),
        ids/dists [n][max_degree] padded with -1 / inf."""
        import torch
        n, d = S.shape
        k = G.shape[1]
        m = METRICS[metric] if isinstance(metric, str) else int(metric)
        ids = torch.empty((n, max_degree), dtype=torch.int32, device=S.device)
        dists = torch.empty((n, max_degree), dtype=torch.float32, device=S.device)
        deg = torch.empty(n, dtype=torch.int32, device=S.device)
        st = GdStats()
        self._sync_stream()
        self._check(lib().knnm_diversify(self.h, _ptr(S), n, d, _ptr(G), k, m, max_degree,
                                         _ptr(ids), _ptr(dists), _ptr(deg), ctypes.byref(st)))
        return ids, dists, deg, st.as_dict()

    def search_prepare(self, S):
        """Per-row data for knnm_search over S ([n][2] floats)."""
        import torch
        n, d = S.shape
        aux = torch.empty((n, 2), dtype=torch.float32, device=S.device)
        self._sync_stream()
        self._check(lib().knnm_search_prepare(self.h, _ptr(S), n, d, _ptr(aux)))
        return aux

    def search(self, S, layers, Q, ef, k_out, metric="l2", seed=0, row_aux=None):
        """Top-down search; `layers` lists the layer graphs from the top down (layer
        l covers the first len(layers[l]) rows of S); row_aux from search_prepare
        (None: computed inside the call).  Returns (ids, dists, evals, stats) with
        k_out entries per query."""
        import torch
        n, d = S.shape
        nq = Q.shape[0]
        m = METRICS[metric] if isinstance(metric, str) else int(metric)
        L = len(layers)
        rows = (ctypes.c_int64 * L)(*[int(g.shape[0]) for g in layers])
        width = (ctypes.c_int32 * L)(*[int(g.shape[1]) for g in layers])
        for g in layers:
            assert g.is_contiguous() and g.dtype == torch.int32
        ptrs = (ctypes.c_void_p * L)(*[g.data_ptr() for g in layers])
        ids = torch.empty((nq, k_out), dtype=torch.int32, device=S.device)
        dists = torch.empty((nq, k_out), dtype=torch.float32, device=S.device)
        evals = torch.empty(nq, dtype=torch.int32, device=S.device)
        st = SearchStats()
        self._sync_stream()
        self._check(lib().knnm_search(self.h, _ptr(S), n, d, _ptr(row_aux), m, L,
                                      ctypes.cast(rows, _P),
                                      ctypes.cast(width, _P), ctypes.cast(ptrs, _P), _ptr(Q), nq,
                                      ef, k_out, seed, _ptr(ids), _ptr(dists), _ptr(evals),
                                      ctypes.byref(st)))
        return ids, dists, evals, st.as_dict()

    def scratch_bytes(self, mode, n1, n2, d, p: Params) -> int:
        """Device scratch one whole-merge call of these sizes takes."""
        out = ctypes.c_uint64(0)
        self._check(lib().knnm_merge_scratch_bytes(self.h, mode, n1, n2, d, ctypes.byref(p),
                                                   ctypes.byref(out)))
        return int(out.value)

    def build(self, S, p: Params, out=None):
        n, d = S.shape
        ids, dists = self._outputs(S, n, p.k, out)
        st = Stats()
        self._sync_stream()
        self._check(lib().knnm_build(self.h, _ptr(S), n, d, ctypes.byref(p), _ptr(ids),
                                     _ptr(dists), ctypes.byref(st)))
        return ids, dists, st.as_dict()

    # ------------------------------------------------------------ round steps
    # All arrays: CUDA torch tensors.
    def step_init(self, mode, X, set_split, G1, G2, p: Params):
        import torch
        N, d = X.shape
        K = p.k
        Kr = list_widths(p, mode, set_split)[1]
        dev = X.device
        ids = torch.empty((N, K), dtype=torch.int32, device=dev)
        dists = torch.empty((N, K), dtype=torch.float32, device=dev)
        flags = torch.empty((N, K), dtype=torch.uint8, device=dev)
        rid = torch.empty((N, max(Kr, 0)), dtype=torch.int32, device=dev)
        rd = torch.empty((N, max(Kr, 0)), dtype=torch.float32, device=dev)
        self._sync_stream()
        self._check(lib().knnm_step_init(self.h, mode, _ptr(X), N, None, N, set_split, d,
                                         _ptr(G1), _ptr(G2), ctypes.byref(p), _ptr(ids),
                                         _ptr(dists), _ptr(flags), _ptr(rid) if Kr else None,
                                         _ptr(rd) if Kr else None))
        return ids, dists, flags, rid, rd

    def step_sample(self, ids, dists, flags, seed, t, s, cap_new=None, cap_old=None):
        import torch
        N, K = ids.shape
        cap_new = cap_new or 2 * s
        cap_old = cap_old or K + s
        dev = ids.device
        new_ids = torch.full((N, cap_new), -1, dtype=torch.int32, device=dev)
        old_ids = torch.full((N, cap_old), -1, dtype=torch.int32, device=dev)
        new_cnt = torch.zeros(N, dtype=torch.int32, device=dev)
        old_cnt = torch.zeros(N, dtype=torch.int32, device=dev)
        self._sync_stream()
        self._check(lib().knnm_step_sample(self.h, N, K, _ptr(ids), _ptr(dists), _ptr(flags), seed,
                                           t, s, cap_new, cap_old, _ptr(new_ids), _ptr(new_cnt),
                                           _ptr(old_ids), _ptr(old_cnt)))
        return new_ids, new_cnt, old_ids, old_cnt

    def step_join(self, mode, X, set_split, p: Params, ids, dists, flags, cands):
        N, d = X.shape
        new_ids, new_cnt, old_ids, old_cnt = cands
        upd = ctypes.c_int64(0)
        ev = ctypes.c_int64(0)
        self._sync_stream()
        self._check(lib().knnm_step_join(self.h, mode, _ptr(X), N, None, N, set_split, d,
                                         ctypes.byref(p), _ptr(ids), _ptr(dists), _ptr(flags),
                                         new_ids.shape[1], old_ids.shape[1], _ptr(new_ids),
                                         _ptr(new_cnt), _ptr(old_ids), _ptr(old_cnt),
                                         ctypes.byref(upd), ctypes.byref(ev)))
        return int(upd.value), int(ev.value)

    def step_join_rows(self, mode, X, set_split, p: Params, ids, dists, flags, cands, lo, hi):
        """step_join for the nodes in [lo, hi) only (their proposals reach every row)."""
        N, d = X.shape
        new_ids, new_cnt, old_ids, old_cnt = cands
        upd = ctypes.c_int64(0)
        ev = ctypes.c_int64(0)
        self._sync_stream()
        self._check(lib().knnm_step_join_rows(self.h, mode, _ptr(X), N, None, N, set_split, d,
                                              ctypes.byref(p), _ptr(ids), _ptr(dists),
                                              _ptr(flags), new_ids.shape[1], old_ids.shape[1],
                                              _ptr(new_ids), _ptr(new_cnt), _ptr(old_ids),
                                              _ptr(old_cnt), lo, hi, ctypes.byref(upd),
                                              ctypes.byref(ev)))
        return int(upd.value), int(ev.value)

    def step_union(self, part_ids, part_dists, start_ids, start_dists, start_flags):
        """Top-K union of parts [P][n][K] against the start lists [n][K]:
        (ids, dists, flags, c_t) of the n rows (device tensors)."""
        import torch
        P, n, K = part_ids.shape
        oi = torch.empty((n, K), dtype=torch.int32, device=part_ids.device)
        od = torch.empty((n, K), dtype=torch.float32, device=part_ids.device)
        of = torch.empty((n, K), dtype=torch.uint8, device=part_ids.device)
        upd = ctypes.c_int64(0)
        self._sync_stream()
        self._check(lib().knnm_step_union(self.h, n, K, P, _ptr(part_ids), _ptr(part_dists),
                                          _ptr(start_ids), _ptr(start_dists), _ptr(start_flags),
                                          _ptr(oi), _ptr(od), _ptr(of), ctypes.byref(upd)))
        return oi, od, of, int(upd.value)

    def step_tc_estimate(self, X, pi, pj, metric="l2", precision="bf16"):
        """(estimate, bound, canonical) of each pair (pi[r], pj[r]) of rows of X,
        as the tensor-core join computes them (device tensors)."""
        import torch
        n, d = X.shape
        P = pi.shape[0]
        est, bound, canon = (torch.empty(P, dtype=torch.float32, device=X.device)
                             for _ in range(3))
        prec = {"bf16": BF16_RERANK, "fp16": FP16_RERANK}[precision]
        self._sync_stream()
        self._check(lib().knnm_step_tc_estimate(self.h, _ptr(X), n, d, METRICS[metric], prec,
                                                _ptr(pi), _ptr(pj), P, _ptr(est), _ptr(bound),
                                                _ptr(canon)))
        return est, bound, canon

    def step_final(self, ids, dists, rear_ids, rear_dists):
        import torch
        N, K = ids.shape
        Kr = rear_ids.shape[1]
        out_i = torch.empty_like(ids)
        out_d = torch.empty_like(dists)
        self._sync_stream()
        self._check(lib().knnm_step_final(self.h, N, K, _ptr(ids), _ptr(dists), Kr,
                                          _ptr(rear_ids) if Kr else None,
                                          _ptr(rear_dists) if Kr else None, _ptr(out_i),
                                          _ptr(out_d)))
        return out_i, out_d


def step_sample_noalloc(ids, dists, flags, seed, t, s, new_ids, new_cnt, old_ids, old_cnt,
                        stream=None) -> int:
    """knnm_step_sample_noalloc: the sampler with the library's fixed scratch
    instead of allocated scratch, for callers that must not allocate device
    memory.  All arrays are caller-owned CUDA tensors (outputs included, so
    the call itself allocates nothing); returns the library's status code."""
    import torch
    N, K = ids.shape
    if stream is None:
        stream = torch.cuda.current_stream(ids.device).cuda_stream
    return lib().knnm_step_sample_noalloc(ctypes.c_void_p(stream), N, K, _ptr(ids), _ptr(dists),
                                          _ptr(flags), seed, t, s, new_ids.shape[1],
                                          old_ids.shape[1], _ptr(new_ids), _ptr(new_cnt),
                                          _ptr(old_ids), _ptr(old_cnt))


class Server:
    """knnm_server_*: J-Merge of raw batches into a graph resident on one device.

    submit() returns at once; worker slots inside the library run queued
    batches concurrently as slots and device memory allow.  The binding keeps
    each submitted batch alive until its wait() returns."""

    def __init__(self, S, G, p: Params, slots=2, capacity_rows=None, max_batch_rows=65536,
                 use_graphs=True, hbm_reserve_bytes=1 << 30, device=0):
        n, d = S.shape
        self.d, self.k = d, p.k
        cfg = ServerConfig()
        cfg.slots = slots
        cfg.use_graphs = int(use_graphs)
        cfg.capacity_rows = capacity_rows or 2 * n
        cfg.max_batch_rows = max_batch_rows
        cfg.hbm_reserve_bytes = hbm_reserve_bytes
        h = ctypes.c_void_p()
        rc = lib().knnm_server_create(device, _ptr(S), n, _ptr(G), d, ctypes.byref(p),
                                      ctypes.byref(cfg), ctypes.byref(h))
        if rc != 0:
            raise KnnmError(rc, "knnm_server_create failed")
        self.h = h
        self._batches = {}

    def _check(self, rc):
        if rc != 0:
            raise KnnmError(rc, lib().knnm_server_last_error(self.h).decode())

    def submit(self, batch, req_id: int):
        self._check(lib().knnm_server_submit(self.h, _ptr(batch), batch.shape[0], req_id))
        self._batches[req_id] = batch

    def wait(self, req_id: int, timeout_ms: int = -1, out=True):
        """Returns (ids, dists, info) of a completed batch: its rows' merged
        lists in resident numbering (numpy) and its request info."""
        rows = self._batches[req_id].shape[0]
        ids = np.empty((rows, self.k), np.int32) if out else None
        dists = np.empty((rows, self.k), np.float32) if out else None
        info = RequestInfo()
        rc = lib().knnm_server_wait(self.h, req_id, timeout_ms, _ptr(ids), _ptr(dists),
                                    ctypes.byref(info))
        if rc == -4:
            raise TimeoutError(f"request {req_id} not complete after {timeout_ms} ms")
        self._batches.pop(req_id, None)
        self._check(rc)
        return ids, dists, info.as_dict()

    def drain(self, timeout_ms: int = -1):
        self._check(lib().knnm_server_drain(self.h, timeout_ms))

    def stats(self):
        st = ServerStats()
        self._check(lib().knnm_server_get_stats(self.h, ctypes.byref(st)))
        return st.as_dict()

    def resident(self, rows: int = -1, vectors=True, device=None):
        """Copies of the resident rows: (vectors, ids, dists), numpy arrays, or
        torch tensors on `device` when it is given."""
        st = self.stats()
        n = st["resident_rows"] if rows < 0 else min(rows, st["resident_rows"])
        if device is not None:
            import torch
            X = torch.empty((n, self.d), dtype=torch.float32, device=device) if vectors else None
            ids = torch.empty((n, self.k), dtype=torch.int32, device=device)
            dists = torch.empty((n, self.k), dtype=torch.float32, device=device)
        else:
            X = np.empty((n, self.d), np.float32) if vectors else None
            ids = np.empty((n, self.k), np.int32)
            dists = np.empty((n, self.k), np.float32)
        cnt = ctypes.c_int64(n)
        self._check(lib().knnm_server_resident(self.h, ctypes.byref(cnt), _ptr(X), _ptr(ids),
                                               _ptr(dists)))
        n = int(cnt.value)
        return (X[:n] if vectors else None), ids[:n], dists[:n]

    def close(self):
        if getattr(self, "h", None):
            lib().knnm_server_destroy(self.h)
            self.h = None
            self._batches.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

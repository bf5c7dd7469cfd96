#!/usr/bin/env python
"""Benchmark of the k-NN graph merge on GB300.

Workload (one "step"): the symmetric merge (S-Merge, Alg. 1) of two SIFT-like
sets of 500,000 x 128 float32 vectors (L2, k = 20, rho = 0.5, keep ratio 0.5,
up to 10 local-join rounds, stop when a round changes <= 0.1% of the entries).
The input graphs are NN-Descent builds of each half (10 rounds), made once
before timing.  The whole merge (init + rounds + final merge) is one step.

Reported: points merged per second of the BF16 tensor-core + FP32 re-rank path
(the headline), the plain FP32 path beside it, recall@10 of the merged graph
against the exact graph on 10,000 sampled nodes, the roofline of the dominant
kernel and of each round phase (sampler, join, top-k update), the end-to-end
rate through the C ABI with host buffers, and the CPU oracle timed on a
bounded sample of the same workload.

Multi-GPU: the merge does not shard; N ranks run N independent replicas of the
workload (weak scaling) and the value is the sum of their points over the
slowest rank's time.

``--impl reference`` times the CPU oracle instead (the only reference this
method has: a plain restatement of the paper's algorithm).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1908_00814_gb300 import datagen  # noqa: E402

WORKLOAD = "smerge_sift_1m_d128_k20"
METRIC = "points merged/sec at recall@10>=0.95 (BF16+rerank vs FP32 plain); serving p50/p99 batch latency"
UNIT = "points/s"
BUILD_RATE_960 = 0.75  # sample rate of the 960-d workload's input builds
PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return PEAKS_FALLBACK, "fallback"


def workload_config(w):
    """The workload both arms run (the reference arm on a bounded sample of it, stated in
    its cpu_baseline); each line names its own arithmetic in a top-level "precision"."""
    return {"workload": WORKLOAD, "merge": "symmetric (Alg. 1)", "n1": w["n"] // 2,
            "n2": w["n"] - w["n"] // 2, "d": w["d"], "k": w["k"], "metric": w["metric"],
            "max_rounds": w["rounds"], "sample_rate": w["sample_rate"], "keep_ratio": 0.5,
            "delta": 0.001,
            "inputs": "NN-Descent builds of each half, 10 rounds, made before timing",
            "l2_flush": "inputs larger than L2 (512 MB vectors + 0.5 GB list state per step)",
            "parallelism": "replicas"}


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    rows.append(parts)
                except ValueError:
                    pass
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            for name, v in zip(names, r[5:9]):
                if v.lower() in ("active", "1", "yes"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(rows)}


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# ----------------------------------------------------------------------------- CPU oracle

def oracle_sample(w, per_half, seed_off=0):
    """The same workload cut to `per_half` rows of each half, with input graphs
    from the oracle's own NN-Descent build (10 rounds)."""
    import oracle
    X = datagen.generate(WORKLOAD, n=w["n"])
    h = w["n"] // 2
    S1 = np.ascontiguousarray(X[:per_half])
    S2 = np.ascontiguousarray(X[h:h + per_half])
    G1, _, _ = oracle.build_graph(S1, w["k"], max_iters=10, delta=0.001, seed=11)
    G2, _, _ = oracle.build_graph(S2, w["k"], max_iters=10, delta=0.001, seed=12)
    return S1, G1, S2, G2


def host_cpu():
    """Host CPU of this run: logical cores available and the model name."""
    model = None
    arm_parts = {"0xd4f": "Arm Neoverse-V2", "0xd40": "Arm Neoverse-V1", "0xd0c": "Arm Neoverse-N1"}
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                low = line.lower()
                if low.startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
                if low.startswith("cpu part") and model is None:
                    part = line.split(":", 1)[1].strip().lower()
                    model = arm_parts.get(part, "Arm CPU part " + part)
    except OSError:
        pass
    if model is None:
        import platform
        model = platform.processor() or platform.machine()
    return {"nproc": os.cpu_count(), "cpu_model": model}


def time_oracle_merge(w, S1, G1, S2, G2, seed=0):
    import oracle
    t0 = time.perf_counter()
    oracle.merge_symmetric(S1, G1, S2, G2, w["k"], max_iters=w["rounds"],
                           sample_rate=w["sample_rate"], delta=0.001, seed=seed)
    return time.perf_counter() - t0


def run_reference(args, w):
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    per_half = args.reference_rows
    S1, G1, S2, G2 = oracle_sample(w, per_half)
    for i in range(args.warmup):
        time_oracle_merge(w, S1, G1, S2, G2, seed=i)
    times = [time_oracle_merge(w, S1, G1, S2, G2, seed=i) for i in range(args.steps)]
    ms = 1000.0 * sum(times) / len(times)
    value = 2 * per_half / (ms / 1000.0)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": workload_config(w), "precision": "fp32 (CPU oracle)",
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"S-Merge of {per_half} rows of each half "
                                       f"({2 * per_half} points) per step, single-threaded",
                             **host_cpu()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------- GPU arm

def exact_recall(torch, X_dev, ids_dev, queries, K=10, chunk=131072, extra=48, metric="l2"):
    """recall@K of the merged lists on `queries` against exact float64 neighbours
    under `metric` ("l2", "cos" or "l1")."""
    q = torch.as_tensor(queries, device=X_dev.device, dtype=torch.long)
    Q = X_dev[q].double()
    qn = (Q ** 2).sum(1)
    best_d = None
    best_i = None
    n = X_dev.shape[0]
    if metric in ("l1", "chi2"):
        chunk = max(1024, chunk // 32)

    def block(Xb):
        Xd = Xb.double()
        if metric == "l1":
            return torch.cdist(Q, Xd, p=1)
        if metric == "chi2":
            return chi2_block(torch, Q, Xd)
        dot = Q @ Xd.T
        if metric == "cos":
            den = qn.sqrt()[:, None] * (Xd ** 2).sum(1).sqrt()[None, :]
            return 1.0 - dot / den.clamp_min(1e-300)
        return qn[:, None] + (Xd ** 2).sum(1)[None, :] - 2.0 * dot

    for b in range(0, n, chunk):
        Xb = X_dev[b:b + chunk]
        D = block(Xb)
        idx = torch.arange(b, b + Xb.shape[0], device=X_dev.device)
        D[idx[None, :] == q[:, None]] = float("inf")
        d2, i2 = torch.topk(D, min(K + extra, D.shape[1]), dim=1, largest=False)
        i2 = i2 + b
        if best_d is None:
            best_d, best_i = d2, i2
        else:
            cd = torch.cat([best_d, d2], 1)
            ci = torch.cat([best_i, i2], 1)
            best_d, o = torch.topk(cd, K + extra, dim=1, largest=False)
            best_i = torch.gather(ci, 1, o)

    # exact float64 distances of the candidates and of the returned ids
    def direct(ids):
        R = X_dev[ids].double()
        if metric == "l1":
            return (R - Q[:, None, :]).abs().sum(-1)
        if metric == "chi2":
            s = R + Q[:, None, :]
            return torch.where(s == 0, 0.0, (R - Q[:, None, :]) ** 2 / s.masked_fill(s == 0, 1.0)).sum(-1)
        if metric == "cos":
            dot = (R * Q[:, None, :]).sum(-1)
            den = qn.sqrt()[:, None] * (R ** 2).sum(-1).sqrt()
            return 1.0 - dot / den.clamp_min(1e-300)
        return ((R - Q[:, None, :]) ** 2).sum(-1)
    cd = direct(best_i)
    kth = torch.sort(cd, dim=1).values[:, K - 1]
    got = ids_dev[q][:, :K].long()
    gd = direct(got)
    hits = (gd <= kth[:, None] * (1 + 1e-9) + 1e-12).sum().item()
    return hits / (len(queries) * K)


def chi2_block(torch, Q, Xd, qchunk=64):
    """Chi-square distances [len(Q)][len(Xd)] in float64, by query blocks."""
    out = []
    for a in range(0, Q.shape[0], qchunk):
        q = Q[a:a + qchunk, None, :]
        s = q + Xd[None]
        out.append(torch.where(s == 0, 0.0, (q - Xd[None]) ** 2 / s.masked_fill(s == 0, 1.0))
                   .sum(-1))
    return torch.cat(out, 0)


def distance_error(torch, X_dev, ids_dev, dists_dev, queries, metric="l2"):
    """Relative error of the returned FP32 distances against float64 (max, p99)."""
    q = torch.as_tensor(queries, device=X_dev.device, dtype=torch.long)
    Q = X_dev[q].double()
    ids = ids_dev[q].long()
    R = X_dev[ids].double()
    if metric == "l1":
        ref = (R - Q[:, None, :]).abs().sum(-1)
    elif metric == "chi2":
        sm = R + Q[:, None, :]
        ref = torch.where(sm == 0, 0.0, (R - Q[:, None, :]) ** 2 / sm.masked_fill(sm == 0, 1.0)).sum(-1)
    elif metric == "cos":
        dot = (R * Q[:, None, :]).sum(-1)
        ref = 1.0 - dot / ((Q ** 2).sum(-1).sqrt()[:, None] * (R ** 2).sum(-1).sqrt())
    else:
        ref = ((R - Q[:, None, :]) ** 2).sum(-1)
    got = dists_dev[q].double()
    rel = ((got - ref).abs() / ref.abs().clamp_min(1e-30)).flatten()
    return {"max_rel": float(rel.max().item()),
            "p99_rel": float(torch.quantile(rel.float(), 0.99).item()),
            "nodes": len(queries), "versus": "float64 recomputation of the returned neighbours"}


SERVE = "serve_sift_2m_d128_k16"


def run_serving(args, torch, knnm, ctx, fp32_arm=False):
    """Serving loop (J-Merge of raw batches into a resident graph): a closed-loop
    run gives the saturation rate, then an open-loop run with Poisson arrivals
    at 0.8 x that rate gives the batch latencies.  With fp32_arm, the same
    closed-loop batches are also merged one at a time by a plain FP32 server
    (one slot, no CUDA graphs, no overlap) from the same resident graph."""
    import threading
    w = datagen.WORKLOADS[SERVE]
    n0 = args.serve_resident or w["n"]
    K, d = w["k"], w["d"]
    nb, slots = args.serve_batches, args.serve_slots
    sizes = {"warm": datagen.serve_batch_sizes(slots, seed=w["seed"] + 1),
             "closed": datagen.serve_batch_sizes(nb, seed=w["seed"] + 2),
             "open": datagen.serve_batch_sizes(nb, seed=w["seed"] + 3)}
    total = n0 + sum(int(v.sum()) for v in sizes.values())
    X = datagen.generate(SERVE, n=total)
    X0 = torch.from_numpy(X[:n0]).cuda()
    G0, _, _ = ctx.build(X0, knnm.params(k=K, precision="bf16", max_iters=10, delta=0.001,
                                         seed=21))
    p = knnm.params(k=K, precision="bf16", max_iters=w["rounds"], sample_rate=w["sample_rate"],
                    delta=0.001, seed=0)
    srv = knnm.Server(X0, G0, p, slots=slots, capacity_rows=total, max_batch_rows=64000,
                      use_graphs=True)
    plain = None
    if fp32_arm:
        p32 = knnm.params(k=K, precision="fp32", max_iters=w["rounds"],
                          sample_rate=w["sample_rate"], delta=0.001, seed=0)
        plain = knnm.Server(X0, G0, p32, slots=1, capacity_rows=total, max_batch_rows=64000,
                            use_graphs=False)
    del X0, G0
    off = n0
    next_id = [1]

    def cut(kind):
        nonlocal off
        out = []
        for b in sizes[kind]:
            out.append((next_id[0], X[off:off + int(b)]))
            next_id[0] += 1
            off += int(b)
        return out

    def closed(batch_list, server=None):
        server = server or srv
        t0 = time.perf_counter()
        for rid, B in batch_list:
            server.submit(B, rid)
        infos = [server.wait(rid, out=False)[2] for rid, _ in batch_list]
        return time.perf_counter() - t0, infos

    warm = cut("warm")
    closed(warm)
    closed_list = cut("closed")
    wall, infos_c = closed(closed_list)
    recall_closed = None
    if fp32_arm:  # the serving graph after the same batches the FP32 arm merges
        Xc, idc, _ = srv.resident(device="cuda")
        qc = datagen.sample_nodes(Xc.shape[0], args.recall_queries, seed=1)
        recall_closed = exact_recall(torch, Xc, idc, qc, K=10)
        del Xc, idc
    plain_res = None
    if plain is not None:
        closed(warm, plain)
        wall_p, infos_p = closed(closed_list, plain)
        Xp, idp, _ = plain.resident(device="cuda")
        plain.close()
        qp = datagen.sample_nodes(Xp.shape[0], args.recall_queries, seed=1)
        rows_p = int(sizes["closed"].sum())
        plain_res = {"server": "FP32, one slot, no CUDA graphs (batches merged one at a time)",
                     "batches": nb, "rows": rows_p, "wall_s": wall_p,
                     "rows_per_s": rows_p / wall_p,
                     "mean_request_ms": float(np.mean([i["run_ms"] for i in infos_p])),
                     "recall_at_10_end": exact_recall(torch, Xp, idp, qp, K=10),
                     "resident_rows_end": int(Xp.shape[0])}
        del Xp, idp
    rows_c = int(sizes["closed"].sum())
    sat_rate = nb / wall
    lam = 0.8 * sat_rate
    arrivals = datagen.poisson_arrivals(nb, lam, seed=w["seed"] + 4)
    batch_list = cut("open")
    submitted = [threading.Event() for _ in batch_list]

    def submitter(t0):
        for i, (rid, B) in enumerate(batch_list):
            delay = t0 + arrivals[i] - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            srv.submit(B, rid)
            submitted[i].set()

    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    t0 = time.perf_counter()
    th = threading.Thread(target=submitter, args=(t0,))
    th.start()
    infos_o = []
    for i, (rid, _) in enumerate(batch_list):
        submitted[i].wait()
        infos_o.append(srv.wait(rid, out=False)[2])
    wall_o = time.perf_counter() - t0
    th.join()
    clocks = sampler.stop()
    stats = srv.stats()
    lat = np.array([i["latency_ms"] for i in infos_o])

    def nearest_rank(v, q):
        v = np.sort(v)
        return float(v[max(1, int(math.ceil(q * len(v)))) - 1])

    Xr, idr, _ = srv.resident(device="cuda")
    srv.close()
    queries = datagen.sample_nodes(Xr.shape[0], args.recall_queries, seed=1)
    recall = exact_recall(torch, Xr, idr, queries, K=10)
    rows_o = int(sizes["open"].sum())

    def breakdown(infos):
        return {k: float(np.mean([i[k] for i in infos]))
                for k in ("queue_ms", "run_ms", "merge_ms", "init_ms", "rounds_ms", "final_ms",
                          "commit_ms")}
    out = {
        "workload": SERVE, "resident_rows_start": n0, "resident_rows_end": int(Xr.shape[0]),
        "d": d, "k": K, "metric": "l2", "precision": "bf16_rerank", "graphs": True,
        "slots": slots, "batch_sizes": "lognormal, median 8000, sigma 1.0, clipped 1000-64000",
        "closed_loop": {"batches": nb, "rows": rows_c, "wall_s": wall,
                        "rows_per_s": rows_c / wall, "batches_per_s": sat_rate,
                        "mean_rounds": float(np.mean([i["rounds"] for i in infos_c])),
                        "recall_at_10_after": recall_closed},
        "open_loop": {"batches": nb, "rows": rows_o, "arrival_rate_per_s": lam,
                      "arrivals": "Poisson, 0.8 x closed-loop batches/s", "wall_s": wall_o,
                      "rows_per_s": rows_o / wall_o, "p50_ms": nearest_rank(lat, 0.50),
                      "p99_ms": nearest_rank(lat, 0.99), "max_ms": float(lat.max()),
                      "mean_queue_ms": float(np.mean([i["queue_ms"] for i in infos_o])),
                      "clocks": clocks},
        "max_concurrent": stats["max_concurrent"], "failed": stats["failed"],
        "recall_at_10_end": recall,
        "request_breakdown_ms": {"closed_loop": breakdown(infos_c),
                                 "open_loop": breakdown(infos_o)},
    }
    if plain_res is not None:
        out["fp32_plain_closed_loop"] = plain_res
        out["closed_loop_speedup_over_fp32_plain"] = (rows_c / wall) / plain_res["rows_per_s"]
    return out


def run_serve_workload(args):
    """One JSON line for the serving workload: closed- and open-loop runs of the
    BF16 serving loop and the plain FP32 server on the same batches."""
    import torch
    from paper_1908_00814_gb300 import build as kbuild, knnm
    kbuild.build()
    torch.cuda.set_device(0)
    ctx = knnm.Context(0)
    res = run_serving(args, torch, knnm, ctx, fp32_arm=not args.no_fp32)
    ctx.close()
    cl = res["closed_loop"]
    line = {"metric": "serving rows merged/sec (closed loop) with p50/p99 batch latency "
                      "(open loop)",
            "value": cl["rows_per_s"], "unit": "rows/s", "n_gpus": 1,
            "steps": cl["batches"], "warmup": args.serve_slots,
            "ms_per_step": 1000.0 * cl["wall_s"] / cl["batches"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16+f32", "data": "synthetic",
            "config": {"workload": SERVE, "resident_rows": res["resident_rows_start"],
                       "batches_per_phase": cl["batches"], "slots": res["slots"],
                       "batch_sizes": res["batch_sizes"]},
            "serving": res}
    print(json.dumps(line), flush=True)
    return 0


def join_traffic():
    """DRAM bytes per launch of the join, from the committed ncu capture of the timed
    merge's join launches; null when the kernel source has changed since."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "k_join_ring_traffic_smerge_sift_1m.json")
    try:
        with open(path) as f:
            cap = json.load(f)
        with open(os.path.join(ROOT, cap["source"]), "rb") as f:
            sha = hashlib.sha256(f.read()).hexdigest()
    except (OSError, KeyError, ValueError):
        return None, "no capture"
    if sha != cap["source_sha256"]:
        return None, "kernel changed since the capture"
    return cap["mean_dram_bytes_per_launch"], os.path.relpath(path, ROOT)


def timed_call(torch, fn, steps, warmup):
    """Device time of `fn` (ms, mean over steps) with CUDA events on the current stream."""
    for _ in range(warmup):
        out = fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    outs = [fn() for _ in range(steps)]
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps, outs[-1], [o[2] for o in outs]


def query_recall(torch, X_dev, Q_dev, ids_dev, K=10, extra=48, qchunk=1024, chunk=262144):
    """recall@K of search results for external queries: candidates from an FP32
    scan (K + extra per query), exact float64 distances of the candidates and of
    the returned ids, ties at the K-th distance counted as hits."""
    hits = 0
    n = X_dev.shape[0]
    xn = (X_dev.double() ** 2).sum(1).float()
    prev_tf32 = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    for a in range(0, Q_dev.shape[0], qchunk):
        Q = Q_dev[a:a + qchunk]
        qn = (Q ** 2).sum(1)
        best_d = best_i = None
        for b in range(0, n, chunk):
            D = qn[:, None] + xn[None, b:b + chunk] - 2.0 * (Q @ X_dev[b:b + chunk].T)
            d2, i2 = torch.topk(D, min(K + extra, D.shape[1]), dim=1, largest=False)
            i2 = i2 + b
            if best_d is None:
                best_d, best_i = d2, i2
            else:
                cd, ci = torch.cat([best_d, d2], 1), torch.cat([best_i, i2], 1)
                best_d, o = torch.topk(cd, K + extra, dim=1, largest=False)
                best_i = torch.gather(ci, 1, o)
        Q64 = Q.double()
        cand = ((X_dev[best_i].double() - Q64[:, None, :]) ** 2).sum(-1)
        kth = torch.sort(cand, dim=1).values[:, K - 1]
        got = ids_dev[a:a + qchunk, :K].long()
        gd = ((X_dev[got.clamp_min(0)].double() - Q64[:, None, :]) ** 2).sum(-1)
        ok = (gd <= kth[:, None] * (1 + 1e-9) + 1e-12) & (got >= 0)
        hits += int(ok.sum().item())
    torch.backends.cuda.matmul.allow_tf32 = prev_tf32
    return hits / (Q_dev.shape[0] * K)


def jaccard_recall(torch, off, items, dim, ids_dev, queries, K=10, chunk=16384):
    """recall@K of set lists: exact Jaccard distances of the sampled rows to all
    rows from 0/1 blocks (FP32 counts are exact), ties at the K-th distance
    counted as hits."""
    n = len(off) - 1
    lens = torch.from_numpy(np.diff(off)).cuda().float()

    def dense(rows):
        M = torch.zeros((len(rows), dim), dtype=torch.float32, device="cuda")
        for r, i in enumerate(rows):
            M[r, torch.from_numpy(items[off[i]:off[i + 1]].astype(np.int64)).cuda()] = 1.0
        return M
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    Q = dense(queries)
    qlen = lens[torch.as_tensor(queries, device="cuda")]
    D = torch.empty((len(queries), n), device="cuda")
    for b in range(0, n, chunk):
        B = dense(range(b, min(n, b + chunk)))
        inter = Q @ B.T
        uni = qlen[:, None] + lens[None, b:b + B.shape[0]] - inter
        D[:, b:b + B.shape[0]] = torch.where(uni == 0, 0.0, 1.0 - inter / uni.clamp_min(1.0))
    torch.backends.cuda.matmul.allow_tf32 = prev
    q = torch.as_tensor(queries, device="cuda", dtype=torch.long)
    D[torch.arange(len(queries), device="cuda"), q] = float("inf")
    kth = torch.sort(D, dim=1).values[:, K - 1]
    got = ids_dev[q][:, :K].long()
    gd = torch.gather(D, 1, got)
    return (gd <= kth[:, None] + 1e-7).sum().item() / (len(queries) * K)


def run_sets(args, name):
    """Jaccard S-Merge of itemsets (the Kosarak metric of Sec. 5): two halves
    built by NN-Descent, merged; set rows as CSR arrays on the device."""
    import torch
    from paper_1908_00814_gb300 import build as kbuild, knnm
    kbuild.build()
    torch.cuda.set_device(0)
    ctx = knnm.Context(0)
    w = dict(datagen.WORKLOADS[name])
    n = args.rows or w["n"]
    K = w["k"]
    off, items = datagen.itemsets(n, w["dim"], seed=w["seed"], **w["gen_args"])
    n1 = n // 2
    offd = torch.from_numpy(off).cuda()
    itd = torch.from_numpy(items).cuda()
    o1 = offd[:n1 + 1].contiguous()
    o2 = (offd[n1:] - offd[n1]).contiguous()
    i1 = itd[:off[n1]].contiguous()
    i2 = itd[off[n1]:].contiguous()
    bp = knnm.params(k=K, metric="jaccard", max_iters=w["rounds"], delta=0.001, seed=11)
    G1, _, _ = ctx.build_sets(o1, i1, bp)
    bp.seed = 12
    G2, _, _ = ctx.build_sets(o2, i2, bp)
    p = knnm.params(k=K, metric="jaccard", max_iters=w["rounds"], sample_rate=w["sample_rate"],
                    delta=0.001, seed=0)
    ms, out, stats = timed_call(torch, lambda: ctx.merge_symmetric_sets(offd, itd, n1, G1, G2, p),
                                args.steps, args.warmup)
    queries = datagen.sample_nodes(n, args.recall_queries, seed=0)
    recall = jaccard_recall(torch, off, items, w["dim"], out[0], queries)
    st = stats[-1]
    line = {"metric": METRIC, "value": n / (ms / 1000.0), "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": name, "merge": "symmetric (Alg. 1), Jaccard on sets",
                       "n": n, "dim": w["dim"], "mean_set_size": float(len(items) / n),
                       "k": K, "metric": "jaccard", "max_rounds": w["rounds"],
                       "sample_rate": w["sample_rate"], "delta": 0.001,
                       "inputs": "NN-Descent builds of each half (library), made before timing",
                       "parallelism": "replicas"},
            "recall_at_10": recall, "recall_queries": len(queries), "rounds": st["rounds"],
            "dist_evals": sum(st["dist_evals"]), "ms_join_per_step": sum(st["ms_join"]),
            "ms_sample_per_step": sum(st["ms_sample"]),
            "ms_update_per_step": sum(st["ms_update"])}
    print(json.dumps(line), flush=True)
    ctx.close()
    return 0


def run_search(args, name):
    """Graph diversification (Alg. 3) of an H-Merge hierarchy and the top-down
    search on it (Sec. 3.4): 10,000 held-out queries, recall@10 and queries/s
    for a sweep of rank-list sizes, beside a flat search of the bottom layer."""
    import torch
    from paper_1908_00814_gb300 import build as kbuild, knnm
    kbuild.build()
    torch.cuda.set_device(0)
    ctx = knnm.Context(0)
    w = dict(datagen.WORKLOADS[name])
    if args.rows:
        w["n"] = args.rows
    n, d, K, nq = w["n"], w["d"], w["k"], w["queries"]
    X = datagen.generate(name, n=n + nq)
    base = torch.from_numpy(X[:n]).cuda()
    Q = torch.from_numpy(X[n:]).cuda()
    del X
    first = 64
    keep = [m for m in (64, 512, 4096, 32768, 262144) if m < n]
    p = knnm.params(k=K, precision="bf16", max_iters=w["rounds"], sample_rate=w["sample_rate"],
                    delta=0.001, seed=0)
    t0 = time.perf_counter()
    perm, ids, _, layers, hst = ctx.hmerge(base, first, p, layers=keep)
    torch.cuda.synchronize()
    ms_hmerge = (time.perf_counter() - t0) * 1000.0
    Xp = ctx.gather_rows(base, torch.from_numpy(perm).cuda())
    del base
    graphs = [torch.from_numpy(layers[m]).cuda() for m in keep] + [torch.from_numpy(ids).cuda()]
    caps = [K] * len(keep) + [2 * K]

    def diversify_all():
        outs = [ctx.diversify(Xp[:g.shape[0]], g, cap) for g, cap in zip(graphs, caps)]
        return outs, None, [o[3] for o in outs]
    ms_div, res, _ = timed_call(torch, diversify_all, args.steps, args.warmup)
    outs = res[0]
    div = [o[0] for o in outs]
    layer_info = [{"rows": int(g.shape[0]), "width_in": int(g.shape[1]), "max_degree": cap,
                   "mean_degree": o[3]["edges"] / g.shape[0],
                   "max_in_degree": o[3]["max_in_degree"], "ms": o[3]["ms"]}
                  for g, cap, o in zip(graphs, caps, outs)]
    aux = ctx.search_prepare(Xp)
    sweep = []
    for label, lay in (("hierarchy", div), ("flat", div[-1:])):
        for ef in (16, 32, 64, 128, 256):
            if label == "flat" and ef not in (32, 128):
                continue
            def call():
                ids_, dists_, _, st_ = ctx.search(Xp, lay, Q, ef, 10, seed=0, row_aux=aux)
                return ids_, dists_, st_
            ms, out, sts = timed_call(torch, call, args.steps, args.warmup)
            r = {"layers": label, "ef": ef, "ms": ms, "queries_per_s": nq / (ms / 1000.0),
                 "recall_at_10": query_recall(torch, Xp, Q, out[0], K=10),
                 "mean_dist_evals": sts[-1]["dist_evals"] / nq,
                 "crowded_queries": sts[-1]["crowded_queries"]}
            sweep.append(r)
            print(f"# {label} ef={ef}: {ms:.2f} ms, {r['queries_per_s']:.0f} q/s, recall "
                  f"{r['recall_at_10']:.4f}, {r['mean_dist_evals']:.0f} evals/query",
                  file=sys.stderr, flush=True)
    good = [r for r in sweep if r["layers"] == "hierarchy" and r["recall_at_10"] >= 0.95]
    head = max(good, key=lambda r: r["queries_per_s"]) if good else sweep[-1]
    line = {"metric": "queries/s of the top-down search at recall@10>=0.95 (Sec. 3.4)",
            "value": head["queries_per_s"], "unit": "queries/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": head["ms"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": name, "n": n, "d": d, "k": K, "queries": nq,
                       "metric": "l2", "hierarchy": f"H-Merge from {first} rows, BF16, "
                       f"upper layers {keep} (k/2 lists), bottom k",
                       "diversify": "Alg. 3, lists + reverse lists, degree caps k above, "
                                    "2k at the bottom",
                       "head_ef": head["ef"], "parallelism": "replicas"},
            "recall_at_10": head["recall_at_10"],
            "ms_hmerge": ms_hmerge, "hmerge_merges": hst["rounds"],
            "ms_diversify_all_layers": ms_div,
            "diversify_points_per_s": sum(li["rows"] for li in layer_info) / (ms_div / 1000.0),
            "layers": layer_info, "sweep": sweep}
    print(json.dumps(line), flush=True)
    ctx.close()
    return 0


def run_other(args, name):
    """The other merge workloads, one JSON line each: the joint merge of 1M raw
    cosine vectors into a 1M graph (96-d), and the 960-d GIST-like symmetric
    merge (L1 on the FP32 path, L2 on every path) with its 64-part merge tree."""
    import torch
    from paper_1908_00814_gb300 import build as kbuild, knnm
    kbuild.build()
    torch.cuda.set_device(0)
    ctx = knnm.Context(0)
    w = dict(datagen.WORKLOADS[name])
    if args.rows:
        w["n"] = args.rows
    n, d, K = w["n"], w["d"], w["k"]
    X = datagen.generate(name, n=n)
    Xd = torch.from_numpy(X).cuda()
    n1 = n // 2
    S1, S2 = Xd[:n1].contiguous(), Xd[n1:].contiguous()
    queries = datagen.sample_nodes(n, args.recall_queries, seed=0)
    steps, warmup = args.steps, args.warmup
    runs = {}

    def record(label, metric, ms, out, stats, points):
        # the L1 and chi-square scans are elementwise (no GEMM): fewer, spread-out nodes
        q = queries if metric not in ("l1", "chi2") else \
            queries[::max(1, -(-len(queries) // 2000))]
        r = {"ms_per_step": ms, "points_per_s": points / (ms / 1000.0),
             "recall_at_10": exact_recall(torch, Xd, out[0], q, K=10, metric=metric),
             "recall_queries": len(q),
             "rounds": stats[-1]["rounds"],
             "dist_evals": sum(stats[-1]["dist_evals"]),
             "reranked": sum(stats[-1]["reranked"]),
             "ms_join_per_step": sum(sum(s_["ms_join"]) for s_ in stats) / len(stats),
             "ms_sample_per_step": sum(sum(s_["ms_sample"]) for s_ in stats) / len(stats),
             "ms_update_per_step": sum(sum(s_["ms_update"]) for s_ in stats) / len(stats),
             "distance_error": distance_error(torch, Xd, out[0], out[1], queries[:200], metric)}
        r["rerank_fraction"] = r["reranked"] / max(r["dist_evals"], 1)
        runs[label] = r
        print(f"# {label}: {ms:.1f} ms, recall {r['recall_at_10']:.4f}", file=sys.stderr,
              flush=True)

    if w["kind"] == "hmerge":
        # H-Merge (Sec. 3.3) from 64 rows, layers of 64, 512, 4096 and 32768 kept
        # (the hierarchy sizes of the paper's search experiments), beside an
        # NN-Descent build of the whole set
        first, keep = 64, [64, 512, 4096, 32768]
        for prec in ("bf16", "fp32"):
            p = knnm.params(k=K, precision=prec, max_iters=w["rounds"],
                            sample_rate=w["sample_rate"], delta=0.001, seed=0)
            Xh = Xd

            def call():
                perm, ids, dists, layers, st = ctx.hmerge(Xh, first, p, layers=keep)
                return (torch.from_numpy(perm), ids, dists, layers, st)
            for _ in range(warmup):
                call()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(steps):
                out = call()
            torch.cuda.synchronize()
            ms = (time.perf_counter() - t0) * 1000.0 / steps
            perm, ids, dists = out[0].long().cuda(), out[1], out[2]
            # recall in the visiting order: rows and ids are positions
            Xp = Xd[perm]
            runs[f"hmerge_{prec}"] = {
                "ms_per_step": ms, "points_per_s": n / (ms / 1000.0),
                "recall_at_10": exact_recall(torch, Xp, torch.from_numpy(ids).cuda(), queries,
                                             K=10),
                "merges": out[4]["rounds"], "first_rows": first, "layers_kept": keep,
                "timing": "host wall clock around the whole call (one library call per step)"}
            print(f"# hmerge {prec}: {ms:.1f} ms", file=sys.stderr, flush=True)
            bp = knnm.params(k=K, precision=prec, max_iters=w["rounds"],
                             sample_rate=w["sample_rate"], delta=0.001, seed=0)
            ms, out, stats = timed_call(torch, lambda: ctx.build(Xd, bp), steps, warmup)
            runs[f"build_{prec}"] = {
                "ms_per_step": ms, "points_per_s": n / (ms / 1000.0),
                "recall_at_10": exact_recall(torch, Xd, out[0], queries, K=10),
                "rounds": stats[-1]["rounds"]}
        head = runs["hmerge_bf16"]
        merge = "H-Merge (Sec. 3.3) beside an NN-Descent build"
    elif w["kind"] == "symmetric_chi2":
        # NUSWide-like BoVW histograms under chi-square (Sec. 5): FP32 path only
        metric = w["metric"]
        bp = knnm.params(k=K, metric=metric, precision="fp32", max_iters=w["rounds"],
                         delta=0.001, seed=11)
        G1, _, _ = ctx.build(S1, bp)
        bp.seed = 12
        G2, _, _ = ctx.build(S2, bp)
        p = knnm.params(k=K, metric=metric, precision="fp32", max_iters=w["rounds"],
                        sample_rate=w["sample_rate"], delta=0.001, seed=0)
        ms, out, stats = timed_call(torch, lambda: ctx.merge_symmetric(S1, G1, S2, G2, p),
                                    steps, warmup)
        record(f"{metric}_fp32", metric, ms, out, stats, n)
        head = runs[f"{metric}_fp32"]
        merge = "symmetric (Alg. 1), chi-square"
    elif w["kind"] == "joint":
        metric = w["metric"]
        G1, _, _ = ctx.build(S1, knnm.params(k=K, metric=metric, precision="fp32",
                                             max_iters=10, delta=0.001, seed=11))
        for prec in ("fp32", "fp16", "bf16"):
            p = knnm.params(k=K, metric=metric, precision=prec, max_iters=w["rounds"],
                            sample_rate=w["sample_rate"], delta=0.001, seed=0)
            ms, out, stats = timed_call(torch, lambda: ctx.merge_joint(S1, G1, S2, p), steps,
                                        warmup)
            record(f"{metric}_{prec}", metric, ms, out, stats, n)
            runs[f"{metric}_{prec}"]["raw_points_per_s"] = (n - n1) / (ms / 1000.0)
        head = runs[f"{metric}_fp32"]
        merge = "joint (Alg. 2)"
    else:
        for metric, precs in (("l1", ("fp32",)), ("l2", ("fp32", "fp16", "bf16"))):
            # input graphs: 10-round NN-Descent builds of each half at sample
            # rate 0.75 (at 0.5 the inputs capped the merged graph at recall
            # 0.956 for L2 and 0.92 for L1)
            bp = knnm.params(k=K, metric=metric, precision="fp32", max_iters=10,
                             sample_rate=BUILD_RATE_960, delta=0.001, seed=11)
            G1, _, _ = ctx.build(S1, bp)
            bp.seed = 12
            G2, _, _ = ctx.build(S2, bp)
            for prec in precs:
                p = knnm.params(k=K, metric=metric, precision=prec, max_iters=w["rounds"],
                                sample_rate=w["sample_rate"], delta=0.001, seed=0)
                ms, out, stats = timed_call(
                    torch, lambda: ctx.merge_symmetric(S1, G1, S2, G2, p), steps, warmup)
                record(f"{metric}_{prec}", metric, ms, out, stats, n)
        # merge tree: 64 exact part graphs (brute force, not timed), merged pairwise
        parts = 64
        rows = [n // parts + (1 if i < n % parts else 0) for i in range(parts)]
        Gt = torch.empty((n, K), dtype=torch.int32, device="cuda")
        off = 0
        torch.backends.cuda.matmul.allow_tf32 = False
        for r in rows:
            P = Xd[off:off + r]
            sq = (P ** 2).sum(1)
            D = sq[:, None] + sq[None, :] - 2.0 * (P @ P.T)
            D.fill_diagonal_(float("inf"))
            Gt[off:off + r] = torch.topk(D, K, dim=1, largest=False).indices.int()
            off += r
            del P, D
        p = knnm.params(k=K, metric="l2", precision="fp32", max_iters=w["rounds"],
                        sample_rate=w["sample_rate"], delta=0.001, seed=0)
        ms, out, stats = timed_call(torch, lambda: ctx.merge_tree(Xd, rows, Gt, p), 1, 1)
        runs["tree_l2_fp32"] = {"parts": parts, "part_rows": rows[0], "levels": stats[-1]["rounds"],
                                "merges": parts - 1, "ms": ms, "points_per_s": n / (ms / 1000.0),
                                "recall_at_10": exact_recall(torch, Xd, out[0], queries, K=10),
                                "leaf_graphs": "brute force (FP32 GEMM, not timed)"}
        print(f"# tree: {ms:.1f} ms", file=sys.stderr, flush=True)
        head = runs["l2_fp32"]
        merge = "symmetric (Alg. 1) + merge tree"
    inputs = {"symmetric": f"NN-Descent builds of each half, 10 rounds, sample rate "
                           f"{BUILD_RATE_960}",
              "symmetric_chi2": "NN-Descent builds of each half, 10 rounds",
              "joint": "NN-Descent build of the first half, 10 rounds"}.get(w["kind"])
    line = {"metric": METRIC, "value": head["points_per_s"], "unit": UNIT, "n_gpus": 1,
            "steps": steps, "warmup": warmup, "ms_per_step": head["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16+f32" if w["kind"] == "hmerge" else "f32", "data": "synthetic",
            "config": {"workload": name, "merge": merge, "n": n, "d": d, "k": K,
                       "metric": w["metric"], "max_rounds": w["rounds"],
                       "sample_rate": w["sample_rate"], "delta": 0.001,
                       "recall_queries": len(queries), "inputs": inputs,
                       "l2_flush": "inputs larger than L2"},
            "runs": runs}
    print(json.dumps(line), flush=True)
    ctx.close()
    return 0


def run_ours(args, w):
    import torch
    from paper_1908_00814_gb300 import build as kbuild, knnm

    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    kbuild.build()
    ctx = knnm.Context(local)
    peaks, peaks_kind = load_peaks()

    X = datagen.generate(WORKLOAD, n=w["n"])
    n1 = w["n"] // 2
    K, d = w["k"], w["d"]
    if rank == 0:
        print(f"# workload {WORKLOAD}: {w['n']} x {d}, k={K}", file=sys.stderr, flush=True)
    Xd = torch.from_numpy(X).cuda()
    S1, S2 = Xd[:n1].contiguous(), Xd[n1:].contiguous()
    bp = knnm.params(k=K, precision="bf16", max_iters=10, sample_rate=w["sample_rate"],
                     delta=0.001, seed=11)
    G1, _, b1 = ctx.build(S1, bp)
    bp.seed = 12
    G2, _, b2 = ctx.build(S2, bp)
    torch.cuda.synchronize()
    build_rounds = [b1["rounds"], b2["rounds"]]

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    def timed(precision, steps, warmup):
        p = knnm.params(k=K, precision=precision, max_iters=w["rounds"],
                        sample_rate=w["sample_rate"], delta=0.001, seed=rank)
        for _ in range(warmup):
            ctx.merge_symmetric(S1, G1, S2, G2, p)
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        stream = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        sampler = ClockSampler(local)
        sampler.start()
        e0.record(stream)
        stats = []
        out = None
        for _ in range(steps):
            out = ctx.merge_symmetric(S1, G1, S2, G2, p)
            stats.append(out[2])
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        clocks = sampler.stop()
        ms = e0.elapsed_time(e1) / steps
        if world > 1:
            import torch.distributed as dist
            t = torch.tensor([ms], device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ms = float(t.item())
        return ms, stats, out, clocks

    ms_bf, st_bf, out_bf, clocks = timed("bf16", args.steps, args.warmup)
    res = {"ms_bf16": ms_bf}
    if not args.no_fp32:
        ms_fp, st_fp, out_fp, clocks_fp = timed("fp32", args.steps, args.warmup)
        same = bool(torch.equal(out_fp[0], out_bf[0]) and torch.equal(
            out_fp[1].view(torch.int32), out_bf[1].view(torch.int32)))
    # recall@10 on sampled nodes (not timed)
    queries = datagen.sample_nodes(w["n"], args.recall_queries, seed=0)
    recall = exact_recall(torch, Xd, out_bf[0], queries, K=10)
    dist_err = distance_error(torch, Xd, out_bf[0], out_bf[1], queries[:500])

    # roofline of each phase (per-round device times from the library's events)
    tot = {"sample": 0.0, "join": 0.0, "update": 0.0}
    nbytes = {"sample": 0.0, "join": 0.0, "update": 0.0}
    launches_join = 0
    launches = 0
    N = w["n"]
    for st in st_bf:
        launches += st["kernel_launches"]
        tot["sample"] += sum(st["ms_sample"])
        tot["join"] += sum(st["ms_join"])
        tot["update"] += sum(st["ms_update"])
        launches_join += st["rounds"]
        for r in range(st["rounds"]):
            G, P = st["gathered"][r], st["proposals"][r]
            # sampler: lists and flags read, snapshot written, k-th keys; per
            # list entry its forward id (written, read back), reverse source
            # id (written, read back) and in-edge count; per staged candidate
            # its 16-byte record entry (id, width or norm, k-th key); per node
            # the record header and the four set counts
            nbytes["sample"] += N * K * (9 + 8 + 8 + 8 + 4) + N * (8 + 16 + 16) + G * 16
            # join: per staged row the 16-bit row with its 16 bytes of error
            # data, its id, k-th key and exactness width; per re-ranked pair
            # both FP32 rows; per proposal its key and its target's count; per
            # node the candidate counts
            nbytes["join"] += (G * (d * 2 + 16 + 4 + 8 + 4) + st["reranked"][r] * 2 * d * 4
                               + P * 12 + N * 8)
            # update: per proposal its key; per node the list, the round-start
            # snapshot and flags read, list and flags written, its count
            nbytes["update"] += P * 8 + N * K * (8 + 8 + 1 + 8 + 1) + N * 8
    dominant = max(tot, key=tot.get)
    bytes_join = nbytes["join"]
    achieved = bytes_join / (tot["join"] / 1000.0) / 1e9 if tot["join"] > 0 else 0.0
    hbm = float(peaks.get("hbm_gbs", PEAKS_FALLBACK["hbm_gbs"]))
    phase_roofline = {
        ph: {"bound": "hbm", "achieved": nbytes[ph] / (tot[ph] / 1000.0) / 1e9 if tot[ph] else 0.0,
             "peak": hbm, "unit": "GB/s",
             "frac": nbytes[ph] / (tot[ph] / 1000.0) / 1e9 / hbm if tot[ph] else 0.0,
             "algorithmic_bytes_per_merge": nbytes[ph] / len(st_bf),
             "ms_per_merge": tot[ph] / len(st_bf)}
        for ph in tot}
    traffic, traffic_note = join_traffic()
    roofline = {"kernel": "k_join_ring (BF16 tensor-core join)", "bound": "hbm",
                "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                "peak_source": f"hbm_gbs of {peaks_kind}", "traffic": traffic,
                "traffic_source": traffic_note,
                "time_share": {k: v / sum(tot.values()) for k, v in tot.items()},
                "dominant_phase": dominant, "launches": launches_join,
                "algorithmic_bytes_per_launch": bytes_join / max(launches_join, 1)}

    # end to end through the C ABI with pinned host buffers
    e2e = None
    if not args.no_e2e:
        hS1 = S1.cpu().pin_memory()
        hS2 = S2.cpu().pin_memory()
        hG1 = G1.cpu().pin_memory()
        hG2 = G2.cpu().pin_memory()
        # pinned outputs too, allocated once (as a serving process would)
        hout = (torch.empty((w["n"], K), dtype=torch.int32).pin_memory(),
                torch.empty((w["n"], K), dtype=torch.float32).pin_memory())
        p = knnm.params(k=K, precision="bf16", max_iters=w["rounds"],
                        sample_rate=w["sample_rate"], delta=0.001, seed=rank)
        ctx.merge_symmetric(hS1, hG1, hS2, hG2, p, out=hout)
        ts = []
        for _ in range(max(1, min(args.steps, 3))):
            barrier()
            t0 = time.perf_counter()
            ids, dists, _ = ctx.merge_symmetric(hS1, hG1, hS2, hG2, p, out=hout)
            ts.append(time.perf_counter() - t0)
        h2d = (hS1.numel() + hS2.numel()) * 4 + (hG1.numel() + hG2.numel()) * 4
        d2h = ids.numel() * 4 + dists.numel() * 4
        e2e = {"value": world * w["n"] / statistics.mean(ts), "unit": UNIT,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "note": "knnm_merge_symmetric with pinned host inputs/outputs; copies inside"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        per_half = args.cpu_rows
        S1h, G1h, S2h, G2h = oracle_sample(w, per_half)
        t = time_oracle_merge(w, S1h, G1h, S2h, G2h)
        cpu = {"value": 2 * per_half / t, "unit": UNIT, "cores": 1, "kind": "oracle", **host_cpu(),
               "sample": f"S-Merge of the first {per_half} rows of each half "
                         f"({2 * per_half} points), inputs from the oracle's own NN-Descent "
                         f"build, single-threaded, {t:.1f} s"}

    value = world * w["n"] / (ms_bf / 1000.0)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_bf,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16+f32", "data": "synthetic", "config": workload_config(w),
            "precision": "bf16_rerank",
            "recall_at_10": recall, "recall_queries": len(queries),
            "distance_error": dist_err,
            "rounds": st_bf[-1]["rounds"], "updates_per_round": st_bf[-1]["updates"],
            "per_round": {k: st_bf[-1][k] for k in ("dist_evals", "proposals", "spilled",
                                                    "reranked", "gathered", "ms_sample",
                                                    "ms_join", "ms_update")},
            "roofline": roofline, "phase_roofline": phase_roofline, "cpu_baseline": cpu,
            "e2e": e2e, "clocks": clocks,
            "gpu_launches": launches, "input_build_rounds": build_rounds}
    if not args.no_fp32:
        line["fp32_plain"] = {"value": world * w["n"] / (ms_fp / 1000.0), "ms_per_step": ms_fp,
                              "dtype": "f32", "identical_graph_to_bf16": same,
                              "ms_join_per_step": sum(sum(s["ms_join"]) for s in st_fp) / len(st_fp),
                              "clocks": clocks_fp}
        line["bf16_speedup_over_fp32"] = ms_fp / ms_bf
    line["phase_ms_per_step"] = {k: v / len(st_bf) for k, v in tot.items()}
    line["ms_init"] = st_bf[-1]["ms_init"]
    line["ms_final"] = st_bf[-1]["ms_final"]
    line["valid"] = recall >= 0.95
    if not args.no_serving:
        line["serving"] = run_serving(args, torch, knnm, ctx)
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-fp32", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--recall-queries", type=int, default=10000,
                    help="sampled nodes for recall@10 (L1 and chi-square runs use at most 2,000)")
    ap.add_argument("--cpu-rows", type=int, default=20000)
    ap.add_argument("--reference-rows", type=int, default=5000)
    ap.add_argument("--workload", default=WORKLOAD,
                    choices=[WORKLOAD, "jmerge_gmm_2m_d96_k16_cos", "smerge_gist_1m_d960_k20",
                             "hmerge_sift_1m_d128_k20", "hsearch_sift_1m_d128_k20",
                             "smerge_nuswide_260k_d500_k20_chi2",
                             "smerge_kosarak_75k_k20_jaccard", "serve_sift_2m_d128_k16"],
                    help="another merge workload (one JSON line of its own)")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--serve-batches", type=int, default=16)
    ap.add_argument("--serve-slots", type=int, default=3)
    ap.add_argument("--serve-resident", type=int, default=None,
                    help="resident rows of the serving run (profiling only)")
    ap.add_argument("--rows", type=int, default=None,
                    help="run the same workload cut to this many points (profiling only)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("at least 3 warm-up steps")
    w = dict(datagen.WORKLOADS[WORKLOAD])
    if args.rows:
        w["n"] = args.rows
    if args.impl == "reference":
        return run_reference(args, w)
    if args.workload == "hsearch_sift_1m_d128_k20":
        return run_search(args, args.workload)
    if args.workload == "smerge_kosarak_75k_k20_jaccard":
        return run_sets(args, args.workload)
    if args.workload == SERVE:
        return run_serve_workload(args)
    if args.workload != WORKLOAD:
        return run_other(args, args.workload)
    return run_ours(args, w)


if __name__ == "__main__":
    sys.exit(main())

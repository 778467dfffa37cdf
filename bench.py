#!/usr/bin/env python
"""Benchmark of the FLASH hot path on GB300.

Step = one all-points k-NN graph (DOPH + bucket grouping + reservoir selection
+ count-based top-k for every row) over the webspam-like workload: 350,000
rows, D = 16,609,143, ~3,700 non-zeros per row (~1.3e9 in total), K=4, L=64,
R=64, 2^18 buckets per table, k=128.  Inputs are seeded synthetic rows shaped
like the paper's webspam dataset (which is not available here).

Prints ONE JSON line (rank 0).  `value` is device-timed queries/s with the CSR
already resident in HBM (5.2 GB, larger than L2, so no flush is needed);
`e2e` is the same metric through flash_knn_graph_host with pinned host buffers
(host->device CSR copy and device->host result copy inside the timed region).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl flash|reference]

--impl reference times the CPU oracle (a plain single-threaded C program that
follows the paper's algorithms step by step) on a bounded sample of the same
workload on this machine's host cores.  Under torchrun every rank runs an
independent replica with its own data seed (no collective on the data path).
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "k-NN graph queries/sec & DOPH HBM GB/s at 1 GB300; served p50/p99 (bit-exact)"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["flash", "reference"], default="flash")
    ap.add_argument("--workload", default="webspam_like")
    ap.add_argument("--rows", type=int, default=0, help="fewer rows (smoke runs only; the line says so)")
    ap.add_argument("--range-bits", type=int, default=0,
                    help="override the workload's range bits, e.g. to keep the full-size bucket load on fewer "
                         "rows for a profile (the line says so)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="target CPU-baseline duration")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving measurement (url-like index)")
    ap.add_argument("--no-tune", action="store_true", help="skip autotuning of the launch knobs")
    ap.add_argument("--serve-seconds", type=float, default=10.0, help="seconds per serving load point and repeat")
    ap.add_argument("--no-url", action="store_true", help="skip the url-like batch and serving sections")
    ap.add_argument("--no-kdd12", action="store_true", help="skip the kdd12-like graph section")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def replica_max(value: float, dist_mod, device) -> float:
    """The largest of a per-rank value over all replicas (the slowest rank's time): every rank
    calls it with its own value and gets the maximum back."""
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist_mod.all_reduce(t, op=dist_mod.ReduceOp.MAX)
    return float(t.item())


def workload(args, rank):
    from paper_1709_01190_gb300 import synth
    w = synth.WORKLOADS[args.workload]
    if args.rows:
        w = w.scaled(args.rows)
    if getattr(args, "range_bits", 0):
        w = w.__class__(**{**w.__dict__, "params": w.params.__class__(**{**w.params.__dict__,
                                                                          "range_bits": args.range_bits})})
    if rank:
        w = w.__class__(**{**w.__dict__, "data": w.data.replace(seed=w.data.seed + 1000 * rank)})
    return w


def host_data(w, pinned: bool):
    """Generate the CSR straight into (pinned) host buffers."""
    import torch
    from paper_1709_01190_gb300 import synth
    spec = w.data.replace(with_val=False)  # the method is set-based: values are never read
    rp0 = synth.row_lengths(spec)
    nnz = int(rp0[-1])
    rp_t = torch.empty(spec.n_rows + 1, dtype=torch.int64, pin_memory=pinned)
    col_t = torch.empty(max(nnz, 1), dtype=torch.int32, pin_memory=pinned)
    csr = synth.generate(spec, row_ptr_out=rp_t.numpy(), col_out=col_t.numpy())
    return csr, rp_t, col_t


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms while running."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                       "-lms", "200", "-i", str(gpu_index)], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self) -> dict:
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None

        sm = [num(r[1]) for r in rows if num(r[1])]
        mx = [num(r[2]) for r in rows if num(r[2])]
        pw = [num(r[3]) for r in rows if num(r[3])]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        loaded = [s for s in sm if mx and s > 0.5 * max(mx)] or sm
        return {"sm_mhz": statistics.median(loaded) if loaded else None, "sm_max_mhz": max(mx) if mx else None,
                "power_w_max": max(pw) if pw else None, "samples": len(rows), "reasons": reasons,
                "window": "sustained warm-up loop + timed region"}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except OSError:
        return {}


def _oracle_graph(w, csr, n, threaded) -> float:
    """Seconds for the oracle's full k-NN graph over the first n rows of the matrix."""
    import oracle
    p = w.params
    rp = csr.row_ptr[:n + 1]
    col = csr.col[:int(rp[-1])]
    fn = oracle.knn_graph_threaded if threaded else oracle.knn_graph
    t0 = time.perf_counter()
    fn(rp, col, p.K, p.L, p.R, p.range_bits, p.seed, w.k)
    return time.perf_counter() - t0


def _oracle_sample(w, csr, threaded, target):
    """Rows n whose oracle graph takes about target seconds, and that run's time. A small first run
    overstates the per-row cost (fixed per-table costs), so the estimate is refined until the run is
    near the target."""
    n = min(csr.n_rows, 2000)
    t = _oracle_graph(w, csr, n, threaded)
    for _ in range(3):
        if t >= 0.6 * target or n >= csr.n_rows:
            break
        n = min(csr.n_rows, max(n + 1, int(n * target / max(t, 1e-3))))
        t = _oracle_graph(w, csr, n, threaded)
    return n, t


def cpu_baseline(w, csr, target_s: float) -> dict:
    """The oracle on the first n rows of the same matrix: a full k-NN graph over them, on all host
    cores (addresses in row blocks, one Adding phase per table, queries in row blocks; the C
    functions are the single-threaded oracle's), and single-threaded beside it."""
    import oracle
    threads = oracle._workers(None)
    n_mt, t_mt = _oracle_sample(w, csr, True, target_s)
    n_st, t_st = _oracle_sample(w, csr, False, target_s / 3)
    return {"value": n_mt / t_mt, "unit": "queries/s", "cores": threads, "kind": "oracle",
            "sample": f"first {n_mt} rows of the same matrix ({int(csr.row_ptr[n_mt])} nnz): full build + all-points "
                      f"query of those rows, C oracle on {threads} host threads, {t_mt:.1f} s",
            "single_thread": {"value": n_st / t_st, "unit": "queries/s", "cores": 1,
                              "sample": f"first {n_st} rows, single-threaded C oracle, {t_st:.1f} s"}}


def _timed(fn, reps, stream=None):
    """Mean device milliseconds of fn() over reps calls (CUDA events on the launching stream)."""
    import torch
    fn()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        fn()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def _phases(fl, fn, reps):
    """Mean per-phase device milliseconds of fn() (events recorded between the library's phases)."""
    fl.flash_enable_phase_timing(True)
    acc = {}
    try:
        for _ in range(reps):
            fn()
            for name, v in fl.flash_phase_times().items():
                acc[name] = acc.get(name, 0.0) + v / reps
    finally:
        fl.flash_enable_phase_timing(False)
    return acc


def _candidates(fl, ix, keys, R):
    """Sum over queries and tables of min(m_t, R): the reservoir ids the queries gather (for the
    query kernel's algorithmic bytes); keys int32 [L][nq] from flash_keys."""
    import torch
    p = ix.params
    T = 1 << p.range_bits
    tables = torch.empty((p.L, T, p.R), dtype=torch.int32, device="cuda")
    counts = torch.empty((p.L, T), dtype=torch.int32, device="cuda")
    fl.flash_index_export(ix, tables, counts)
    del tables
    total = 0
    for t in range(p.L):
        k = keys[t].long()
        c = counts[t][k.clamp(max=T - 1)].clamp(max=R).long()
        total += int(torch.where(k < T, c, torch.zeros_like(c)).sum())
    del counts
    torch.cuda.empty_cache()
    return total


def _peak(kind="hbm"):
    peaks = measured_peaks()
    v = peaks.get("hbm_gbs")
    return (v, "measured (MEASURED_PEAKS.json hbm_gbs)") if v else (6800.0, "fallback")


def url_section(fl, args, tune: bool) -> tuple[dict, dict]:
    """The url-like index (2.4M rows, L=128, R=128, 2^15 buckets) resident on the device:
    the 1,000,000-query batch (one call: untuned, autotuned, CUDA-graph captured) and the serving loop."""
    import torch
    from paper_1709_01190_gb300 import synth, tuning
    w = synth.WORKLOADS["url_like_batched"]
    p = w.params
    params = fl.FlashParams(p.K, p.L, p.R, p.range_bits, p.seed)
    data = synth.generate(w.data)
    dev_data = fl.DeviceCSR.from_host(data)
    build_ms = _timed(lambda: fl.flash_build(params, dev_data).free(), 3)
    ix = fl.flash_build(params, dev_data)
    torch.cuda.synchronize()
    n_rows, dim = data.n_rows, data.dim
    del dev_data, data
    qc = synth.generate(w.query_data)
    dq = fl.DeviceCSR.from_host(qc)
    k = w.k
    ids = torch.empty((qc.n_rows, k), dtype=torch.int32, device="cuda")
    cnt = torch.empty_like(ids)
    stream = torch.cuda.current_stream()

    def q_call():
        fl.flash_query(ix, dq, k, None, ids, cnt, stream)

    tuning.set_tuning(None)
    plain_ms = _timed(q_call, 3)
    ph = _phases(fl, q_call, 3)
    tuned = None
    tuned_ms = plain_ms
    if tune:
        key = tuning.shape_key("query", params, n_rows, 0, k, q_rows=qc.n_rows)
        best, _ = tuning.autotune(q_call, key=key, reps=2)
        tuned = dataclasses.asdict(best)
        tuned_ms = _timed(q_call, 3)
    g = tuning.GraphedQuery(ix, dq, k, None, ids, cnt)
    graph_ms = _timed(g.replay, 5)
    tuned_ph = _phases(fl, q_call, 3)
    del g
    tuning.set_tuning(None)
    qkeys = fl.row_keys(params, dq)
    m_total = _candidates(fl, ix, qkeys, p.R)
    del qkeys
    nq = qc.n_rows
    qbytes = 4 * p.L * nq + 4 * m_total + 8 * k * nq
    qms = tuned_ph.get("query", ph.get("query"))
    peak, src = _peak()
    c3 = {"workload": w.name, "index_rows": n_rows, "queries": nq, "k": k, "index_build_ms": build_ms,
          "one_call_ms": plain_ms, "one_call_queries_per_s": nq / (plain_ms / 1e3),
          "tuned": tuned, "tuned_ms": tuned_ms, "tuned_queries_per_s": nq / (tuned_ms / 1e3),
          "graph_replay_ms": graph_ms, "graph_replay_queries_per_s": nq / (graph_ms / 1e3),
          "phases_ms_untuned": ph, "phases_ms_tuned": tuned_ph,
          "candidates_per_query": m_total / nq,
          "query_roofline": {"kernel": "query kernels (gather, count, top-k) of the tuned call", "bound": "hbm",
                             "algorithmic_bytes": qbytes,
                             "bytes_formula": "sum over queries of sum_t (4 + 4 min(m_t, R)) + 8k",
                             "duration_ms": qms, "achieved": qbytes / (qms / 1e3) / 1e9, "peak": peak,
                             "unit": "GB/s", "frac": qbytes / (qms / 1e3) / 1e9 / peak, "peak_source": src}}
    del dq, ids, cnt
    torch.cuda.empty_cache()
    served = None
    if not args.no_serve:
        served = serving_measurement(fl, ix, dim, args.serve_seconds)
    ix.free()
    return c3, served


def serving_measurement(fl, ix, dim, seconds_per_load: float = 10.0, repeats: int = 3) -> dict:
    """Served p50/p99 and queries/s on the resident url-like index, requests of U[1, 4096] query rows."""
    import threading
    from paper_1709_01190_gb300 import serve, synth
    w = synth.WORKLOADS["serving_url"]
    qc = synth.generate(w.query_data)
    rng = np.random.default_rng(5)
    reqs, r0 = [], 0
    while True:
        s = int(rng.integers(1, 4097))
        if r0 + s > qc.n_rows:
            break
        sub = qc.slice(r0, r0 + s)
        reqs.append((sub.row_ptr, sub.col))
        r0 += s
    mean_rows = float(np.mean([rp.shape[0] - 1 for rp, _ in reqs]))
    k = w.k
    out = {"workload": w.name, "index_rows": int(ix.n_rows), "k": k, "slots": 4, "mem_budget_bytes": 8 << 30,
           "seconds_per_load": seconds_per_load, "repeats": repeats}

    def server():
        return serve.Server(serve.CudaBackend(ix, k, dim, n_slots=4), mem_budget=8 << 30, max_batch_rows=16384)

    # saturated (closed loop: everything queued at once)
    srv = server()
    for t in [srv.submit(*r) for r in reqs[:8]]:
        t.wait(120)
    srv.close()
    srv = server()
    n_sat = min(len(reqs), 240)
    t0 = time.perf_counter()
    ts = [srv.submit(*r) for r in reqs[:n_sat]]
    for t in ts:
        t.wait(300)
    sat_s = time.perf_counter() - t0
    srv.close()
    sat_rows = sum(r[0].shape[0] - 1 for r in reqs[:n_sat])
    out["saturated_queries_per_s"] = sat_rows / sat_s
    out["saturated_batches"] = srv.stats()["batches"]

    # plain path: one request at a time, one stream, copy in / query / copy out / wait
    n_plain = min(len(reqs), 200)
    serve.plain_serve(ix, k, reqs[:2], dim)
    t0 = time.perf_counter()
    serve.plain_serve(ix, k, reqs[:n_plain], dim)
    plain_s = time.perf_counter() - t0
    out["plain_queries_per_s"] = sum(r[0].shape[0] - 1 for r in reqs[:n_plain]) / plain_s
    out["plain_requests"] = n_plain

    # open loop: Poisson arrivals at fractions of the saturated rate, several repeats per load
    loads = {}
    pos = n_sat
    for load in (0.25, 0.5, 0.8, 1.0):
        rate = load * out["saturated_queries_per_s"] / mean_rows  # requests per second
        reps = []
        for rep in range(repeats):
            srv = server()
            stop = time.perf_counter() + seconds_per_load
            arng = np.random.default_rng(int(load * 100) + 1000 * rep)
            sent = []

            def gen():
                nonlocal pos
                t_next = time.perf_counter()
                while time.perf_counter() < stop:
                    t_next += arng.exponential(1.0 / rate)
                    dt = t_next - time.perf_counter()
                    if dt > 0:
                        time.sleep(dt)
                    if pos >= len(reqs):
                        pos = n_sat
                    sent.append(srv.submit(*reqs[pos]))
                    pos += 1

            th = threading.Thread(target=gen)
            t0 = time.perf_counter()
            th.start()
            th.join()
            for t in sent:
                t.wait(300)
            wall = time.perf_counter() - t0
            srv.close()
            st = srv.stats()
            reps.append({"served_queries_per_s": st["rows"] / wall, "p50_ms": st.get("p50_ms"),
                         "p99_ms": st.get("p99_ms"), "requests": st["requests"], "batches": st["batches"]})
        p99s = [r["p99_ms"] for r in reps if r["p99_ms"] is not None]
        loads[str(load)] = {"offered_queries_per_s": load * out["saturated_queries_per_s"],
                            "served_queries_per_s": float(np.median([r["served_queries_per_s"] for r in reps])),
                            "p50_ms": float(np.median([r["p50_ms"] for r in reps if r["p50_ms"] is not None])),
                            "p99_ms": float(np.median(p99s)) if p99s else None,
                            "p99_ms_range": [min(p99s), max(p99s)] if p99s else None,
                            "requests": sum(r["requests"] for r in reps), "repeats": reps}
    out["poisson"] = loads
    out["mean_request_rows"] = mean_rows
    return out


def kdd12_section(fl, args) -> dict:
    """The kdd12-like all-points k-NN graph (10M rows, L=256, R=32, 2^20 buckets, k=32): per-phase
    times with their rooflines, and the plain unbatched path beside it."""
    import torch
    from paper_1709_01190_gb300 import synth
    w = synth.WORKLOADS["kdd12_like"]
    p = w.params
    params = fl.FlashParams(p.K, p.L, p.R, p.range_bits, p.seed)
    c = synth.generate(w.data)
    dev = fl.DeviceCSR.from_host(c)
    n, nnz, k = c.n_rows, c.nnz, w.k
    del c
    ids = torch.empty((n, k), dtype=torch.int32, device="cuda")
    cnt = torch.empty_like(ids)
    stream = torch.cuda.current_stream()

    def step():
        fl.flash_knn_graph(params, dev, k, ids, cnt, stream)

    ms = _timed(step, 3)
    ph = _phases(fl, step, 2)
    qual_q = torch.from_numpy(synth.sample_rows(n, 1000, seed=41).astype(np.int32)).cuda()
    qual = fl.quality(dev, qual_q, ids[qual_q.long()].contiguous())
    plain_ms = _timed(lambda: fl.flash_knn_graph_plain(params, dev, k, ids, cnt, stream), 1)
    plain_ph = _phases(fl, lambda: fl.flash_knn_graph_plain(params, dev, k, ids, cnt, stream), 1)
    torch.cuda.synchronize()
    hashes = torch.empty((n, p.K * p.L), dtype=torch.int32, device="cuda")
    hash_ms = _timed(lambda: fl.flash_hash(params, dev, hashes, stream), 3)
    del hashes
    keys = fl.row_keys(params, dev)
    keys_ms = _timed(lambda: fl.flash_keys(params, dev, keys, stream), 3)
    ix = fl.flash_build(params, dev)
    m_total = _candidates(fl, ix, keys, p.R)
    index_bytes = ix.info()["bytes"]
    ix.free()
    del keys
    torch.cuda.empty_cache()
    # reservoir sharing (Section 3.5): one pool of F * L * 2^rb reservoirs for all tables
    T = 1 << p.range_bits
    share = {}
    for F in (0.3,):
        P = int(round(F * p.L * T))
        ps = fl.FlashParams(p.K, p.L, p.R, p.range_bits, p.seed, share_pool=P)
        s_ms = _timed(lambda: fl.flash_knn_graph(ps, dev, k, ids, cnt, stream), 2)
        s_qual = fl.quality(dev, qual_q, ids[qual_q.long()].contiguous())
        ixs = fl.flash_build(ps, dev)
        s_bytes = ixs.info()["bytes"]
        ixs.free()
        share[str(F)] = {"pool_reservoirs": P, "graph_ms": s_ms, "queries_per_s": n / (s_ms / 1e3),
                         "R@k": s_qual["R@k"], "S@k": s_qual["S@k"], "index_bytes": s_bytes,
                         "dense_table_bytes": 4 * P * (p.R + 1)}
    share["1.0 (no sharing)"] = {"graph_ms": ms, "R@k": qual["R@k"], "S@k": qual["S@k"], "index_bytes": index_bytes,
                                 "dense_table_bytes": 4 * p.L * T * (p.R + 1)}
    del ids, cnt, dev
    torch.cuda.empty_cache()
    peak, src = _peak()
    T = 1 << p.range_bits
    b_keys = 8 * (n + 1) + 4 * nnz + 4 * p.L * n
    b_hash = 8 * (n + 1) + 4 * nnz + 4 * p.K * p.L * n
    b_sort = 4 * p.L * n + 4 * p.L * n + 4 * p.L * (T + 1)
    b_query = 4 * p.L * n + 4 * m_total + 8 * k * n

    def roof(bytes_, ms_):
        return {"algorithmic_bytes": bytes_, "duration_ms": ms_, "achieved_GB/s": bytes_ / (ms_ / 1e3) / 1e9,
                "frac": bytes_ / (ms_ / 1e3) / 1e9 / peak}

    return {"workload": w.name, "n_rows": n, "nnz": nnz, "graph_ms": ms, "queries_per_s": n / (ms / 1e3),
            "phases_ms": ph, "plain_graph_ms": plain_ms, "plain_queries_per_s": n / (plain_ms / 1e3),
            "plain_phases_ms": plain_ph, "speedup_vs_plain": plain_ms / ms,
            "candidates_per_query": m_total / n, "peak_GB/s": peak, "peak_source": src,
            "quality": {"queries": int(qual_q.numel()), "k": k, "R@k": qual["R@k"], "S@k": qual["S@k"],
                        "gold_standard": "cosine of column sets over all rows (flash_eval_quality)"},
            "reservoir_sharing": share,
            "rooflines": {
                "hash_phase (keys, 8(N+1)+4nnz+4LN)": roof(b_keys, ph.get("hash", keys_ms)),
                "sort+reservoir (4LN keys read + 4LN ids + 4L(T+1) starts written)":
                    roof(b_sort, ph.get("sort", 0.0) + ph.get("reservoir", 0.0)),
                "query (sum_t (4 + 4 min(m_t,R)) + 8k per query)": roof(b_query, ph.get("query", ms))},
            "flash_hash": {"ms": hash_ms, "bytes": b_hash, "bytes_formula": "8(N+1) + 4 nnz + 4 K L N",
                           "GB/s": b_hash / (hash_ms / 1e3) / 1e9, "frac": b_hash / (hash_ms / 1e3) / 1e9 / peak},
            "flash_keys": {"ms": keys_ms, "bytes": b_keys, "bytes_formula": "8(N+1) + 4 nnz + 4 L N",
                           "GB/s": b_keys / (keys_ms / 1e3) / 1e9, "frac": b_keys / (keys_ms / 1e3) / 1e9 / peak}}


def pinned_copy_ceiling(nbytes: int = 4 << 30) -> dict:
    """Host->device and device->host bandwidth of one large copy from / to pinned memory (the ceiling
    of the end-to-end number, whose inputs cross the host link every step)."""
    import torch
    h = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
    d = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    h2d = _timed(lambda: d.copy_(h, non_blocking=True), 3)
    d2h = _timed(lambda: h.copy_(d, non_blocking=True), 3)
    del h, d
    torch.cuda.empty_cache()
    return {"bytes": nbytes, "h2d_GB/s": nbytes / (h2d / 1e3) / 1e9, "d2h_GB/s": nbytes / (d2h / 1e3) / 1e9}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    w = workload(args, 0)
    csr, _, _ = host_data(w, pinned=False)
    import oracle
    p = w.params
    # bounded sample per step, sized so the whole run takes a few minutes; the oracle runs on all
    # host cores (its C functions in threads over row blocks and tables)
    threads = oracle._workers(None)
    per_step = max(2.0, 120.0 / max(1, args.steps + args.warmup))
    n, _ = _oracle_sample(w, csr, True, per_step)
    rp, col = csr.row_ptr[:n + 1], csr.col[:int(csr.row_ptr[n])]
    times = []
    for i in range(args.warmup + args.steps):
        t = time.perf_counter()
        oracle.knn_graph_threaded(rp, col, p.K, p.L, p.R, p.range_bits, p.seed, w.k)
        if i >= args.warmup:
            times.append(time.perf_counter() - t)
    ms = 1000.0 * sum(times) / len(times)
    value = n / (ms / 1000.0)
    sample = (f"first {n} rows ({int(rp[-1])} nnz) of {w.name.split(':')[0]}: full build + all-points query, "
              f"C oracle on {threads} host threads")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "queries/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": config_of(w, csr),
            "cpu_baseline": {"value": value, "unit": "queries/s", "cores": threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "queries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def config_of(w, csr):
    p = w.params
    return {"workload": w.name, "n_rows": csr.n_rows, "nnz": csr.nnz, "dim": csr.dim, "K": p.K, "L": p.L,
            "R": p.R, "range_bits": p.range_bits, "k": w.k, "seed": p.seed,
            "l2": "inputs larger than L2 (CSR of %.1f GB resident in HBM), no flush" % (
                (8 * (csr.n_rows + 1) + 4 * csr.nnz) / 1e9)}


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    rank, world, local = dist_env()
    import torch
    import torch.distributed as dist
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import paper_1709_01190_gb300 as fl
    fl.build()
    w = workload(args, rank)
    p = w.params
    params = fl.FlashParams(p.K, p.L, p.R, p.range_bits, p.seed)
    csr, rp_pin, col_pin = host_data(w, pinned=True)
    n, nnz, k = csr.n_rows, csr.nnz, w.k
    dev = fl.DeviceCSR(rp_pin.cuda(), col_pin[:nnz].cuda() if nnz else col_pin.cuda(), csr.dim, nnz=nnz)
    ids = torch.empty((n, k), dtype=torch.int32, device="cuda")
    cnt = torch.empty((n, k), dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()

    def step():
        fl.flash_knn_graph(params, dev, k, ids, cnt, stream)

    tuned = None
    if not args.no_tune:
        from paper_1709_01190_gb300 import tuning
        os.environ.setdefault("FLASH_TUNING_CACHE", os.path.join(tempfile.gettempdir(), "flash_tuning_bench.json"))
        key = tuning.shape_key("graph", params, n, nnz, k)
        best, _ = tuning.autotune(step, key=key, reps=2)
        tuned = dataclasses.asdict(best)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    assert fl.flash_device_error(stream) == 0

    sampler = ClockSampler(local) if rank == 0 else None
    t_end = time.perf_counter() + 2.0  # sustained load so the clock samples see the kernels
    while time.perf_counter() < t_end:
        for _ in range(20):
            step()
        torch.cuda.synchronize()

    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ms = e0.elapsed_time(e1) / args.steps
    launches_per_step = fl.flash_last_launch_count()
    clocks = sampler.stop() if sampler else None
    if world > 1:
        ms = replica_max(ms, dist, "cuda")
    value = world * n / (ms / 1000.0)

    # per-phase device times (same kernels, same launches; events on the stream between phases)
    acc = _phases(fl, step, args.steps)

    # DOPH kernels timed alone: the keys epilogue (the graph's hash phase) and the hashes output (DOPH GB/s)
    keys_out = torch.empty((p.L, n), dtype=torch.int32, device="cuda")
    hashes_out = torch.empty((n, p.K * p.L), dtype=torch.int32, device="cuda")

    graph_ms = None
    try:
        from paper_1709_01190_gb300 import tuning as _t
        g = _t.GraphedKnnGraph(params, dev, k, ids, cnt)
        graph_ms = _timed(g.replay, max(args.steps, 5), stream)
        del g
    except Exception as e:  # report, do not fail the bench
        graph_ms = f"capture failed: {e}"

    keys_ms = _timed(lambda: fl.flash_keys(params, dev, keys_out, stream), max(args.steps, 5), stream)
    hash_ms = _timed(lambda: fl.flash_hash(params, dev, hashes_out, stream), max(args.steps, 5), stream)
    in_bytes = 8 * (n + 1) + 4 * nnz
    keys_bytes = in_bytes + 4 * p.L * n           # the fused keys path: one key array
    hash_bytes = in_bytes + 4 * p.K * p.L * n
    peak, peak_src = _peak()
    hash_phase_ms = acc.get("hash", keys_ms)
    achieved = keys_bytes / (hash_phase_ms / 1000.0) / 1e9
    roofline = {"kernel": "doph_kernel<keys> (hash phase of the graph step)", "bound": "hbm",
                "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "peak_source": peak_src + " (torch copy read+write; kernel timed inside the step, burst copy figure)",
                "algorithmic_bytes_per_launch": keys_bytes,
                "bytes_formula": "8(N+1) + 4 nnz + 4 L N (the fused keys path)",
                "overhead_bytes_per_launch": 4 * p.L * n,
                "overhead": "a row-major copy of the keys for the graph's queries (4 L N written), not counted",
                "traffic": None, "duration_ms": hash_phase_ms}
    prof = os.path.join(ROOT, "profiles", "doph_keys_webspam_like_traffic.json")
    if os.path.exists(prof) and not args.rows and not args.range_bits and args.workload == "webspam_like":
        try:
            import hashlib
            with open(prof) as fh:
                rec = json.load(fh)
            fresh = all(hashlib.sha256(open(os.path.join(ROOT, f), "rb").read()).hexdigest() == h
                        for f, h in rec.get("source_sha256", {}).items())
            # counters describe the kernel as it was captured: none once it has changed since
            roofline["traffic"] = rec.get("traffic_bytes_per_launch") if fresh else None
        except (OSError, ValueError):
            pass
    doph = {"GB/s": hash_bytes / (hash_ms / 1000.0) / 1e9, "ms": hash_ms, "bytes": hash_bytes,
            "frac_of_hbm_peak": hash_bytes / (hash_ms / 1000.0) / 1e9 / peak,
            "bytes_formula": "8(N+1) + 4 nnz + 4 K L N", "keys_epilogue_GB/s": keys_bytes / (keys_ms / 1e3) / 1e9,
            "keys_frac_of_hbm_peak": keys_bytes / (keys_ms / 1e3) / 1e9 / peak}

    # Section 4.3's quality measures of the graph on 1000 sampled rows (brute force on the GPU)
    from paper_1709_01190_gb300 import synth as _sy
    qq = torch.from_numpy(_sy.sample_rows(n, min(1000, n), seed=41).astype(np.int32)).cuda()
    step()
    qres = fl.quality(dev, qq, ids[qq.long()].contiguous())
    quality = {"queries": int(qq.numel()), "k": k, "R@k": qres["R@k"], "S@k": qres["S@k"],
               "gold_standard": "cosine of column sets over all rows (flash_eval_quality)"}

    # the plain, unbatched GPU path on the same rows (same results; a baseline)
    plain = None
    if world == 1:
        plain_ms = _timed(lambda: fl.flash_knn_graph_plain(params, dev, k, ids, cnt, stream), 2, stream)
        plain = {"api": "flash_knn_graph_plain", "ms_per_step": plain_ms, "value": n / (plain_ms / 1e3),
                 "unit": "queries/s", "phases_ms": _phases(
                     fl, lambda: fl.flash_knn_graph_plain(params, dev, k, ids, cnt, stream), 1),
                 "speedup_of_optimised": plain_ms / ms}

    # the two densifications (rotation; optimal, [36]) on sparse kdd12-like rows, where most bins are empty
    densify = None
    if not args.rows and not args.range_bits and args.workload == "webspam_like":
        from paper_1709_01190_gb300 import synth as _s
        wk = _s.WORKLOADS["kdd12_like"].scaled(1_000_000)
        ck = _s.generate(wk.data)
        dk = fl.DeviceCSR.from_host(ck)
        pk = wk.params
        kout = torch.empty((pk.L, ck.n_rows), dtype=torch.int32, device="cuda")
        dms = {}
        for mode in (0, 1):
            pm = fl.FlashParams(pk.K, pk.L, pk.R, pk.range_bits, pk.seed, densify=mode)
            dms[mode] = _timed(lambda: fl.flash_keys(pm, dk, kout, stream), 3, stream)
        densify = {"workload": f"kdd12-like rows: {ck.n_rows:,} rows, {ck.nnz:,} non-zeros, K={pk.K} L={pk.L} "
                               f"(B={pk.K * pk.L}), flash_keys",
                   "rotation_ms": dms[0], "optimal_ms": dms[1],
                   "rotation_rows_per_s": ck.n_rows / (dms[0] / 1e3), "optimal_rows_per_s": ck.n_rows / (dms[1] / 1e3)}
        del dk, kout

    e2e = None
    if not args.no_e2e:
        out_i = torch.empty((n, k), dtype=torch.int32, pin_memory=True).numpy()
        out_c = torch.empty((n, k), dtype=torch.int32, pin_memory=True).numpy()
        rp_np, col_np = rp_pin.numpy(), col_pin.numpy()[:max(nnz, 0)]
        fl.flash_knn_graph_host(params, rp_np, col_np, csr.dim, k, out_i, out_c, stream)
        t = time.perf_counter()
        for _ in range(args.steps):
            fl.flash_knn_graph_host(params, rp_np, col_np, csr.dim, k, out_i, out_c, stream)
        e2e_s = (time.perf_counter() - t) / args.steps
        if world > 1:
            e2e_s = replica_max(e2e_s, dist, "cuda")
        link = pinned_copy_ceiling()
        e2e = {"value": world * n / e2e_s, "unit": "queries/s", "ms_per_step": e2e_s * 1000.0,
               "h2d_bytes_per_step": in_bytes, "d2h_bytes_per_step": 8 * n * k,
               "api": "flash_knn_graph_host (pinned host buffers)",
               "link_ceiling": {**link, "ms_per_step_at_ceiling":
                                1e3 * (in_bytes / (link["h2d_GB/s"] * 1e9) + 8 * n * k / (link["d2h_GB/s"] * 1e9)),
                                "frac": (1e3 * (in_bytes / (link["h2d_GB/s"] * 1e9) +
                                                8 * n * k / (link["d2h_GB/s"] * 1e9))) / (e2e_s * 1000.0)}}

    config3 = served = config4 = None
    if rank == 0 and world == 1 and not args.rows and not args.range_bits:
        del dev, keys_out, hashes_out
        torch.cuda.empty_cache()
        if not args.no_url:
            config3, served = url_section(fl, args, tune=not args.no_tune)
        if not args.no_kdd12:
            config4 = kdd12_section(fl, args)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(w, csr, args.cpu_seconds)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "queries/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "u32", "data": "synthetic (seeded, webspam-shaped; see config)",
                "config": config_of(w, csr), "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": launches_per_step * args.steps, "clocks": clocks,
                "phases_ms": acc, "doph": doph, "plain": plain, "densify": densify, "quality": quality,
                "graph_replay_ms_per_step": graph_ms, "tuning": tuned,
                "config3_url_like_batch": config3, "config4_kdd12_like_graph": config4,
                "served": served, "reduced": bool(args.rows or args.range_bits)}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

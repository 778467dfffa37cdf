"""Launch-knob autotuning and CUDA-graph capture for the FLASH hot path.

The knobs (``flash_tuning`` in include/flash.h) change only the schedule of the
CUDA kernels -- never a result -- so the autotuner can pick them by timing
the real workload:
  * query_warp_table   : words of the per-warp count table of the query kernel;
  * doph_rows_per_grab : rows a DOPH warp claims at a time;
  * doph_order         : rows in index order, or longest rows first.
Choices are cached in a JSON file keyed by the workload's shape and the GPU.

``GraphedKnnGraph`` captures one flash_knn_graph call (DOPH -> radix grouping
-> reservoir selection -> query, with its stream-ordered scratch) into a CUDA
graph and replays it.
"""
from __future__ import annotations

import ctypes
import dataclasses
import json
import math
import os
import threading

from ._lib import check, lib

_CACHE_LOCK = threading.Lock()


class _Tuning(ctypes.Structure):
    _fields_ = [("query_warp_table", ctypes.c_uint32), ("doph_rows_per_grab", ctypes.c_uint32),
                ("doph_order", ctypes.c_uint32)]


def _bind():
    L = lib()
    if not getattr(L, "_tuning_bound", False):
        L.flash_set_tuning.argtypes = [ctypes.POINTER(_Tuning)]
        L.flash_set_tuning.restype = ctypes.c_int
        L.flash_get_tuning.argtypes = [ctypes.POINTER(_Tuning)]
        L.flash_get_tuning.restype = ctypes.c_int
        L._tuning_bound = True
    return L


@dataclasses.dataclass(frozen=True)
class Tuning:
    query_warp_table: int = 0
    doph_rows_per_grab: int = 0
    doph_order: int = 0


def set_tuning(t: Tuning | None) -> None:
    L = _bind()
    if t is None:
        check(L.flash_set_tuning(None), "flash_set_tuning")
    else:
        c = _Tuning(t.query_warp_table, t.doph_rows_per_grab, t.doph_order)
        check(L.flash_set_tuning(ctypes.byref(c)), "flash_set_tuning")


def get_tuning() -> Tuning:
    c = _Tuning()
    check(_bind().flash_get_tuning(ctypes.byref(c)), "flash_get_tuning")
    return Tuning(c.query_warp_table, c.doph_rows_per_grab, c.doph_order)


CANDIDATES = {
    "query_warp_table": [256, 512, 1024, 2048],
    "doph_order": [0, 1],
    "doph_rows_per_grab": [0, 1, 4, 16],
}


def _cache_path() -> str:
    return os.environ.get("FLASH_TUNING_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "flash_gb300", "tuning.json"))


def _load_cache() -> dict:
    try:
        with open(_cache_path()) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def _store_cache(key: str, t: Tuning, ms: float) -> None:
    with _CACHE_LOCK:
        data = _load_cache()
        data[key] = {"tuning": dataclasses.asdict(t), "ms": ms}
        path = _cache_path()
        try:
            os.makedirs(os.path.dirname(path), exist_ok=True)
            tmp = path + f".tmp{os.getpid()}"
            with open(tmp, "w") as fh:
                json.dump(data, fh, indent=1, sort_keys=True)
            os.replace(tmp, path)
        except OSError:
            pass


def shape_key(kind: str, params, n_rows: int, nnz: int, k: int, q_rows: int = 0) -> str:
    import torch
    name = torch.cuda.get_device_name() if torch.cuda.is_available() else "cpu"
    avg = nnz / max(n_rows, 1)
    return (f"{kind}|{name}|n~2^{round(math.log2(max(n_rows, 1)))}|q~2^{round(math.log2(max(q_rows, 1)))}"
            f"|nnz/row~2^{round(math.log2(max(avg, 1)))}|K{params.K}L{params.L}R{params.R}rb{params.range_bits}|k{k}")


def _time_ms(fn, reps: int) -> float:
    import torch
    fn()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        fn()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def autotune(fn, key: str | None = None, reps: int = 3, use_cache: bool = True) -> tuple[Tuning, float]:
    """Coordinate search over the knobs timing ``fn()`` (which must launch the workload);
    leaves the best tuning set and returns it with its time (ms)."""
    if use_cache and key:
        hit = _load_cache().get(key)
        if hit:
            t = Tuning(**hit["tuning"])
            set_tuning(t)
            return t, float(hit["ms"])
    best = Tuning()
    set_tuning(best)
    best_ms = _time_ms(fn, reps)
    for knob, values in CANDIDATES.items():
        for v in values:
            cand = dataclasses.replace(best, **{knob: v})
            if cand == best:
                continue
            set_tuning(cand)
            ms = _time_ms(fn, reps)
            if ms < best_ms:
                best, best_ms = cand, ms
    set_tuning(best)
    if key:
        _store_cache(key, best, best_ms)
    return best, best_ms


class GraphedKnnGraph:
    """One flash_knn_graph call captured as a CUDA graph (hash -> group -> reservoir -> query).

    The graph owns its scratch (stream-ordered allocations captured as memory
    nodes); replays must not overlap.  Inputs are read from, and outputs
    written to, the same device buffers at every replay."""

    def __init__(self, params, x, k: int, out_ids=None, out_counts=None):
        import torch
        from . import flash_device_error, flash_knn_graph
        self.ids = out_ids if out_ids is not None else torch.empty((x.n_rows, k), dtype=torch.int32, device="cuda")
        self.counts = out_counts if out_counts is not None else torch.empty_like(self.ids)
        flash_device_error()  # the device error word is allocated before any capture
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            flash_knn_graph(params, x, k, self.ids, self.counts, side)  # warm-up outside the graph
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph, capture_error_mode="thread_local"):
            flash_knn_graph(params, x, k, self.ids, self.counts, torch.cuda.current_stream())

    def replay(self):
        self.graph.replay()
        return self.ids, self.counts


class GraphedQuery:
    """One flash_query call over a fixed batch of query rows captured as a CUDA graph (DOPH of the
    rows -> gather -> count -> top-k, with the call's stream-ordered scratch).  Replays read the
    batch from, and write the results to, the same device buffers; replays must not overlap."""

    def __init__(self, index, q, k: int, exclude_ids=None, out_ids=None, out_counts=None):
        import torch
        from . import flash_device_error, flash_query
        self.ids = out_ids if out_ids is not None else torch.empty((q.n_rows, k), dtype=torch.int32, device="cuda")
        self.counts = out_counts if out_counts is not None else torch.empty_like(self.ids)
        flash_device_error()  # the device error word is allocated before any capture
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            flash_query(index, q, k, exclude_ids, self.ids, self.counts, side)  # warm-up outside the graph
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph, capture_error_mode="thread_local"):
            flash_query(index, q, k, exclude_ids, self.ids, self.counts, torch.cuda.current_stream())

    def replay(self):
        self.graph.replay()
        return self.ids, self.counts

"""FLASH hot path on GB300 (sm_103a): DOPH hashing, reservoir hash tables,
count-based top-k querying and the all-points k-NN graph.

The functions named ``flash_*`` mirror the C ABI of ``include/flash.h`` one
to one; they only marshal arguments (torch tensors give device pointers and
the current CUDA stream) and raise :class:`FlashError` on a non-zero status.
The CUDA library must be built (:func:`build`); without it, or without a
GPU, every call raises -- there is no CPU fallback.

Convenience helpers (:func:`hash_rows`, :func:`knn_graph`, ...) allocate the
outputs and call the same entry points.
"""
from __future__ import annotations

import ctypes
import dataclasses

from ._lib import (DEVERR_COL_RANGE, DEVERR_ROW_PTR, DEVERR_TIMEOUT, FlashError, Params, check, lib,
                   strerror)
from .build import build as _build_lib

__all__ = [
    "FlashError", "FlashParams", "DeviceCSR", "FlashIndex", "build",
    "flash_hash", "flash_keys", "flash_build", "flash_add", "flash_query", "flash_knn_graph", "flash_knn_graph_plain",
    "flash_knn_graph_host", "flash_eval_quality", "quality",
    "flash_index_export", "flash_device_error", "flash_set_scratch_budget", "flash_knn_graph_scratch_bytes",
    "flash_query_scratch_bytes", "flash_strerror", "flash_version",
    "hash_rows", "row_keys", "knn_graph", "DEVERR_COL_RANGE", "DEVERR_ROW_PTR", "DEVERR_TIMEOUT",
]


def build(force: bool = False) -> str:
    """Compile the CUDA library for sm_103a (in-tree) and return its path."""
    return _build_lib(force=force)


@dataclasses.dataclass(frozen=True)
class FlashParams:
    """K hashes per table, L tables (Section 2.2), reservoirs of R ids (Section 3.2),
    2^range_bits buckets per table (Section 4.4.1), the seed of every random choice, the
    densification of empty bins (Section 2.3): 0 rotation, 1 optimal densification ([36]), and
    reservoir sharing (Section 3.5): 0 none, else one pool of share_pool reservoirs for all tables
    (F = share_pool / (L * 2^range_bits))."""
    K: int
    L: int
    R: int
    range_bits: int
    seed: int
    densify: int = 0
    share_pool: int = 0

    def c(self) -> Params:
        return Params(self.K, self.L, self.R, self.range_bits, self.seed & ((1 << 64) - 1), self.densify,
                      self.share_pool)

    @property
    def B(self) -> int:
        return self.K * self.L


@dataclasses.dataclass
class DeviceCSR:
    """CSR rows on the device: row_ptr int64 [n+1], col int32 [nnz], val float32 [nnz] or None."""
    row_ptr: "torch.Tensor"
    col: "torch.Tensor"
    dim: int
    val: "torch.Tensor | None" = None
    nnz: int | None = None

    def __post_init__(self):
        import torch
        assert self.row_ptr.dtype == torch.int64 and self.row_ptr.is_cuda and self.row_ptr.is_contiguous()
        assert self.col.dtype == torch.int32 and self.col.is_cuda and self.col.is_contiguous()
        if self.nnz is None:
            self.nnz = int(self.col.numel())

    @property
    def n_rows(self) -> int:
        return int(self.row_ptr.numel() - 1)

    @classmethod
    def from_host(cls, csr, device="cuda", with_val: bool = False) -> "DeviceCSR":
        import torch
        rp = torch.from_numpy(csr.row_ptr).to(device)
        col = torch.from_numpy(csr.col).to(device)
        val = torch.from_numpy(csr.val).to(device) if (with_val and csr.val is not None) else None
        return cls(rp, col, csr.dim, val, int(csr.row_ptr[-1]))

    def c(self) -> "Csr":
        from ._lib import Csr
        return Csr(self.row_ptr.data_ptr(), self.col.data_ptr() if self.col.numel() else None,
                   self.val.data_ptr() if self.val is not None else None, self.n_rows, int(self.nnz), int(self.dim))


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _check_out(t, shape, dtype_name):
    import torch
    dt = {"int32": torch.int32, "uint32": torch.int32}[dtype_name]
    if t.dtype not in (dt, getattr(torch, "uint32", dt)) or not t.is_cuda or not t.is_contiguous():
        raise FlashError(1, f"output must be a contiguous CUDA {dtype_name} tensor")
    if tuple(t.shape) != tuple(shape) and t.numel() != int(__import__("math").prod(shape)):
        raise FlashError(1, f"output has shape {tuple(t.shape)}, expected {tuple(shape)}")


# ---------------------------------------------------------------- C ABI mirror

def flash_hash(params: FlashParams, x: DeviceCSR, hashes, stream=None) -> None:
    """DOPH hashes into ``hashes`` (uint32 viewed as int32 ok) [n_rows][K*L]."""
    _check_out(hashes, (x.n_rows, params.B), "uint32")
    p, c = params.c(), x.c()
    check(lib().flash_hash(ctypes.byref(p), ctypes.byref(c), _ptr(hashes), _stream(stream)), "flash_hash")


def flash_keys(params: FlashParams, x: DeviceCSR, keys, stream=None) -> None:
    """Bucket addresses of every row into ``keys`` [L][n_rows] (2^range_bits for empty rows)."""
    _check_out(keys, (params.L, x.n_rows), "uint32")
    p, c = params.c(), x.c()
    check(lib().flash_keys(ctypes.byref(p), ctypes.byref(c), _ptr(keys), _stream(stream)), "flash_keys")


class FlashIndex:
    """Library-owned hash tables (Adding phase, Algorithm 2)."""

    def __init__(self, handle: int, params: FlashParams, n_rows: int):
        self._h = ctypes.c_void_p(handle)
        self.params = params
        self.n_rows = n_rows

    @property
    def handle(self):
        return self._h

    def info(self) -> dict:
        from ._lib import IndexInfo
        inf = IndexInfo()
        check(lib().flash_index_get_info(self._h, ctypes.byref(inf)), "flash_index_get_info")
        return {"n_rows": inf.n_rows, "bytes": inf.bytes}

    def free(self) -> None:
        if self._h and self._h.value:
            lib().flash_index_free(self._h)
            self._h = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.free()
        except Exception:  # pragma: no cover - interpreter shutdown
            pass

    def export(self, stream=None):
        """Dense (tables int32 [L][2^rb][R] with -1 = empty, counts uint32-as-int32 [L][2^rb]);
        with reservoir sharing the pool's (tables [P][R], counts [P])."""
        import torch
        p = self.params
        shape = (p.share_pool,) if p.share_pool else (p.L, 1 << p.range_bits)
        tables = torch.empty(shape + (p.R,), dtype=torch.int32, device="cuda")
        counts = torch.empty(shape, dtype=torch.int32, device="cuda")
        flash_index_export(self, tables, counts, stream)
        return tables, counts


def flash_build(params: FlashParams, x: DeviceCSR, stream=None) -> FlashIndex:
    p, c = params.c(), x.c()
    h = ctypes.c_void_p(0)
    check(lib().flash_build(ctypes.byref(p), ctypes.byref(c), ctypes.byref(h), _stream(stream)), "flash_build")
    return FlashIndex(h.value, params, x.n_rows)


def flash_add(index: FlashIndex, x: DeviceCSR, stream=None) -> None:
    """Index the rows of x as new points index.n_rows, index.n_rows + 1, ... (Algorithm 2 continued)."""
    c = x.c()
    check(lib().flash_add(index.handle, ctypes.byref(c), _stream(stream)), "flash_add")
    index.n_rows += x.n_rows


def flash_query(index: FlashIndex, q: DeviceCSR, k: int, exclude_ids, out_ids, out_counts, stream=None) -> None:
    _check_out(out_ids, (q.n_rows, k), "int32")
    _check_out(out_counts, (q.n_rows, k), "int32")
    c = q.c()
    check(lib().flash_query(index.handle, ctypes.byref(c), int(k), _ptr(exclude_ids), _ptr(out_ids),
                            _ptr(out_counts), _stream(stream)), "flash_query")


def flash_knn_graph(params: FlashParams, x: DeviceCSR, k: int, out_ids, out_counts, stream=None) -> None:
    _check_out(out_ids, (x.n_rows, k), "int32")
    _check_out(out_counts, (x.n_rows, k), "int32")
    p, c = params.c(), x.c()
    check(lib().flash_knn_graph(ctypes.byref(p), ctypes.byref(c), int(k), _ptr(out_ids), _ptr(out_counts),
                                _stream(stream)), "flash_knn_graph")


def flash_knn_graph_plain(params: FlashParams, x: DeviceCSR, k: int, out_ids, out_counts, stream=None) -> None:
    """The plain, unbatched GPU path (a baseline): the same graph as flash_knn_graph."""
    _check_out(out_ids, (x.n_rows, k), "int32")
    _check_out(out_counts, (x.n_rows, k), "int32")
    p, c = params.c(), x.c()
    check(lib().flash_knn_graph_plain(ctypes.byref(p), ctypes.byref(c), int(k), _ptr(out_ids), _ptr(out_counts),
                                      _stream(stream)), "flash_knn_graph_plain")


def flash_eval_quality(x: DeviceCSR, queries, reported, nn, nn_sim, sim_at_k, stream=None) -> None:
    """Section 4.3's gold standard by brute force on the GPU (see include/flash.h)."""
    nq, k = int(reported.shape[0]), int(reported.shape[1])
    c = x.c()
    check(lib().flash_eval_quality(ctypes.byref(c), _ptr(queries), nq, _ptr(reported), k, _ptr(nn), _ptr(nn_sim),
                                   _ptr(sim_at_k), _stream(stream)), "flash_eval_quality")


def quality(x: DeviceCSR, queries, reported, stream=None) -> dict:
    """R@k and S@k (Section 4.3) of the reported ids [nq][k] of the query rows `queries` (row ids
    of x), with the per-query nearest neighbours."""
    import torch
    nq = int(queries.numel())
    nn = torch.empty(nq, dtype=torch.int32, device="cuda")
    nn_sim = torch.empty(nq, dtype=torch.float64, device="cuda")
    sim = torch.empty(nq, dtype=torch.float64, device="cuda")
    flash_eval_quality(x, queries, reported, nn, nn_sim, sim, stream)
    hit = (reported == nn[:, None]).any(dim=1)
    return {"R@k": float(hit.double().mean()), "S@k": float(sim.mean()), "nn": nn, "nn_sim": nn_sim,
            "sim_at_k": sim}


def flash_knn_graph_host(params: FlashParams, row_ptr, col, dim: int, k: int, out_ids, out_counts,
                         stream=None) -> None:
    """Host-buffer variant: numpy (ideally pinned) inputs and outputs; synchronizes the stream."""
    import numpy as np
    n = int(row_ptr.shape[0] - 1)
    for a, dt in ((row_ptr, np.int64), (col, np.int32), (out_ids, np.int32), (out_counts, np.int32)):
        if a.dtype != dt or not a.flags["C_CONTIGUOUS"]:
            raise FlashError(1, "flash_knn_graph_host: wrong dtype or non-contiguous array")
    if out_ids.size != n * k or out_counts.size != n * k:
        raise FlashError(1, "flash_knn_graph_host: output size")
    p = params.c()
    check(lib().flash_knn_graph_host(ctypes.byref(p), row_ptr.ctypes.data, col.ctypes.data if col.size else None,
                                     n, int(dim), int(k), out_ids.ctypes.data, out_counts.ctypes.data,
                                     _stream(stream)), "flash_knn_graph_host")


def flash_index_export(index: FlashIndex, tables, counts, stream=None) -> None:
    check(lib().flash_index_export(index.handle, _ptr(tables), _ptr(counts), _stream(stream)), "flash_index_export")


def flash_device_error(stream=None) -> int:
    return int(lib().flash_device_error(_stream(stream)))


def flash_set_scratch_budget(nbytes: int) -> int:
    return int(lib().flash_set_scratch_budget(int(nbytes)))


def flash_knn_graph_scratch_bytes(params: FlashParams, n_rows: int) -> int:
    p = params.c()
    return int(lib().flash_knn_graph_scratch_bytes(ctypes.byref(p), int(n_rows)))


def flash_query_scratch_bytes(params: FlashParams, q_rows: int) -> int:
    p = params.c()
    return int(lib().flash_query_scratch_bytes(ctypes.byref(p), int(q_rows)))


def flash_enable_phase_timing(on: bool) -> bool:
    return bool(lib().flash_enable_phase_timing(1 if on else 0))


def flash_phase_times() -> dict:
    """{phase name: device milliseconds} of this thread's last flash_knn_graph (timing enabled)."""
    ms = (ctypes.c_float * 8)()
    names = (ctypes.c_char_p * 8)()
    n = lib().flash_phase_times(ms, names, 8)
    return {names[i].decode(): float(ms[i]) for i in range(max(n, 0))}


def flash_last_launch_count() -> int:
    return int(lib().flash_last_launch_count())


def flash_strerror(code: int) -> str:
    return strerror(code)


def flash_version() -> str:
    return lib().flash_version().decode()


# ------------------------------------------------------------- conveniences

def hash_rows(params: FlashParams, x: DeviceCSR, stream=None):
    import torch
    out = torch.empty((x.n_rows, params.B), dtype=torch.int32, device="cuda")
    flash_hash(params, x, out, stream)
    return out


def row_keys(params: FlashParams, x: DeviceCSR, stream=None):
    import torch
    out = torch.empty((params.L, x.n_rows), dtype=torch.int32, device="cuda")
    flash_keys(params, x, out, stream)
    return out


def knn_graph(params: FlashParams, x: DeviceCSR, k: int, stream=None):
    import torch
    ids = torch.empty((x.n_rows, k), dtype=torch.int32, device="cuda")
    cnt = torch.empty((x.n_rows, k), dtype=torch.int32, device="cuda")
    flash_knn_graph(params, x, k, ids, cnt, stream)
    return ids, cnt


def knn_graph_plain(params: FlashParams, x: DeviceCSR, k: int, stream=None):
    import torch
    ids = torch.empty((x.n_rows, k), dtype=torch.int32, device="cuda")
    cnt = torch.empty((x.n_rows, k), dtype=torch.int32, device="cuda")
    flash_knn_graph_plain(params, x, k, ids, cnt, stream)
    return ids, cnt


def query(index: FlashIndex, q: DeviceCSR, k: int, exclude_ids=None, stream=None):
    import torch
    ids = torch.empty((q.n_rows, k), dtype=torch.int32, device="cuda")
    cnt = torch.empty((q.n_rows, k), dtype=torch.int32, device="cuda")
    flash_query(index, q, k, exclude_ids, ids, cnt, stream)
    return ids, cnt

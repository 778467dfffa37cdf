"""Seeded synthetic CSR workloads shaped like the paper's datasets.

The paper evaluates on url, webspam and kdd12 (Section 4.2, Table 1), which
are not available here.  The generators below draw rows with the same shapes
(row count, dimensionality, mean non-zeros per row) and stand in for them.
This module holds no arithmetic of the method itself: it only produces inputs
(CSR ``row_ptr`` int64, ``col`` int32, optional ``val`` float32) that both the
CPU oracle and the CUDA path consume.  The native part is ``synth.cpp``.
"""
from __future__ import annotations

import ctypes
import dataclasses
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.cpp")
_OUT_DIR = os.path.join(_HERE, "_build")
_SO = os.path.join(_OUT_DIR, "libflash_synth.so")
_LOCK = threading.Lock()
_LIB = None


class _Spec(ctypes.Structure):
    _fields_ = [
        ("n_rows", ctypes.c_int64),
        ("dim", ctypes.c_int64),
        ("len_kind", ctypes.c_int32),
        ("id_kind", ctypes.c_int32),
        ("len_a", ctypes.c_double),
        ("len_b", ctypes.c_double),
        ("clip_lo", ctypes.c_int64),
        ("clip_hi", ctypes.c_int64),
        ("zipf_s", ctypes.c_double),
        ("n_clusters", ctypes.c_int64),
        ("cluster_size", ctypes.c_int64),
        ("resample_frac", ctypes.c_double),
        ("seed", ctypes.c_uint64),
    ]


def build(force: bool = False) -> str:
    """Compile synth.cpp into an in-tree shared library (host code only)."""
    with _LOCK:
        if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
            return _SO
        os.makedirs(_OUT_DIR, exist_ok=True)
        tmp = _SO + f".tmp{os.getpid()}"
        cmd = ["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-pthread", _SRC, "-o", tmp]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
        return _SO


def _lib():
    global _LIB
    if _LIB is None:
        lib = ctypes.CDLL(build())
        lib.synth_lengths.restype = ctypes.c_int64
        lib.synth_lengths.argtypes = [ctypes.POINTER(_Spec), ctypes.c_void_p, ctypes.c_int]
        lib.synth_fill.restype = ctypes.c_int
        lib.synth_fill.argtypes = [ctypes.POINTER(_Spec), ctypes.c_void_p, ctypes.c_void_p,
                                   ctypes.c_void_p, ctypes.c_int]
        lib.synth_sample_rows.restype = ctypes.c_int
        lib.synth_sample_rows.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_uint64, ctypes.c_void_p]
        _LIB = lib
    return _LIB


@dataclasses.dataclass(frozen=True)
class DataSpec:
    """Distribution of one synthetic sparse matrix."""
    n_rows: int
    dim: int
    len_kind: str            # "uniform" | "lognormal" | "poisson1"
    len_a: float             # uniform: low;  lognormal: mu;     poisson1: lambda
    len_b: float = 0.0       # uniform: high; lognormal: sigma
    clip_lo: int = 1
    clip_hi: int = 1 << 40
    id_kind: str = "uniform"  # "uniform" | "zipf"
    zipf_s: float = 1.1
    n_clusters: int = 0
    cluster_size: int = 0
    resample_frac: float = 0.0
    seed: int = 0
    with_val: bool = False   # positive float32 values, unit L2 norm per row

    def replace(self, **kw) -> "DataSpec":
        return dataclasses.replace(self, **kw)

    def _c(self) -> _Spec:
        return _Spec(self.n_rows, self.dim,
                     {"uniform": 0, "lognormal": 1, "poisson1": 2}[self.len_kind],
                     {"uniform": 0, "zipf": 1}[self.id_kind],
                     float(self.len_a), float(self.len_b), int(self.clip_lo), int(self.clip_hi),
                     float(self.zipf_s), int(self.n_clusters), int(self.cluster_size),
                     float(self.resample_frac), int(self.seed) & ((1 << 64) - 1))


@dataclasses.dataclass
class CSR:
    row_ptr: np.ndarray        # int64 [n_rows + 1]
    col: np.ndarray            # int32 [nnz]
    val: np.ndarray | None     # float32 [nnz] or None (the method ignores values)
    dim: int

    @property
    def n_rows(self) -> int:
        return int(self.row_ptr.shape[0] - 1)

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def slice(self, r0: int, r1: int) -> "CSR":
        """Rows [r0, r1) as a new CSR whose row_ptr starts at 0 (views of the arrays)."""
        a, b = int(self.row_ptr[r0]), int(self.row_ptr[r1])
        val = None if self.val is None else self.val[a:b]
        return CSR(self.row_ptr[r0:r1 + 1] - a, self.col[a:b], val, self.dim)

    def rows(self, ids) -> "CSR":
        """Gather a subset of rows into a new CSR (host)."""
        ids = np.asarray(ids, dtype=np.int64)
        lens = self.row_ptr[ids + 1] - self.row_ptr[ids]
        rp = np.zeros(len(ids) + 1, dtype=np.int64)
        np.cumsum(lens, out=rp[1:])
        col = np.empty(int(rp[-1]), dtype=np.int32)
        val = None if self.val is None else np.empty(int(rp[-1]), dtype=np.float32)
        for i, r in enumerate(ids):
            a, b = self.row_ptr[r], self.row_ptr[r + 1]
            col[rp[i]:rp[i + 1]] = self.col[a:b]
            if val is not None:
                val[rp[i]:rp[i + 1]] = self.val[a:b]
        return CSR(rp, col, val, self.dim)


def _threads(n_threads):
    if n_threads is not None:
        return int(n_threads)
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


def generate(spec: DataSpec, n_threads: int | None = None, row_ptr_out=None, col_out=None) -> CSR:
    """Draw the CSR matrix described by ``spec`` (deterministic in ``spec.seed``).

    ``row_ptr_out`` / ``col_out`` may be caller-provided numpy views (e.g. of
    pinned host memory) of the right dtype; they are filled in place.
    """
    lib = _lib()
    cs = spec._c()
    nt = _threads(n_threads)
    rp = row_ptr_out if row_ptr_out is not None else np.empty(spec.n_rows + 1, dtype=np.int64)
    assert rp.dtype == np.int64 and rp.shape == (spec.n_rows + 1,)
    nnz = lib.synth_lengths(ctypes.byref(cs), rp.ctypes.data, nt)
    if nnz < 0:
        raise ValueError(f"bad synthetic spec: {spec}")
    if col_out is not None:
        assert col_out.dtype == np.int32 and col_out.shape[0] >= nnz
        col = col_out[:nnz]
    else:
        col = np.empty(nnz, dtype=np.int32)
    val = np.empty(nnz, dtype=np.float32) if spec.with_val else None
    rc = lib.synth_fill(ctypes.byref(cs), rp.ctypes.data, col.ctypes.data,
                        None if val is None else val.ctypes.data, nt)
    if rc != 0:
        raise RuntimeError("synth_fill failed")
    return CSR(rp, col, val, spec.dim)


def row_lengths(spec: DataSpec, n_threads: int | None = None) -> np.ndarray:
    """row_ptr only (cheap: no ids drawn)."""
    rp = np.empty(spec.n_rows + 1, dtype=np.int64)
    if _lib().synth_lengths(ctypes.byref(spec._c()), rp.ctypes.data, _threads(n_threads)) < 0:
        raise ValueError(f"bad synthetic spec: {spec}")
    return rp


def sample_rows(m: int, n: int, seed: int) -> np.ndarray:
    """n distinct row ids of [0, m), keyed by seed (sampling without replacement)."""
    out = np.empty(n, dtype=np.int64)
    if _lib().synth_sample_rows(m, n, seed & ((1 << 64) - 1), out.ctypes.data) != 0:
        raise ValueError("n > m")
    return out


# --------------------------------------------------------------------------
# Workloads.  Data seed = 1000 + workload index; method seed = 0x5EEDF1A5 + index.


def _lognormal_mu_for_clipped_mean(target: float, sigma: float, clip_hi: float) -> float:
    """mu such that E[min(exp(mu + sigma Z), clip_hi)] = target (closed form, bisection)."""
    phi = lambda x: 0.5 * (1.0 + math.erf(x / math.sqrt(2.0)))

    def clipped_mean(mu):
        lc = math.log(clip_hi)
        return (math.exp(mu + sigma * sigma / 2) * phi((lc - mu - sigma * sigma) / sigma)
                + clip_hi * (1.0 - phi((lc - mu) / sigma)))

    lo, hi = math.log(target) - 5 * sigma, math.log(target) + 5 * sigma
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if clipped_mean(mid) < target:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


@dataclasses.dataclass(frozen=True)
class MethodParams:
    K: int
    L: int
    R: int
    range_bits: int
    seed: int

    @property
    def B(self) -> int:
        return self.K * self.L


@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    data: DataSpec
    params: MethodParams
    k: int
    mode: str                     # "sampled_queries" | "graph" | "fresh_queries" | "serving"
    n_queries: int = 0
    query_data: DataSpec | None = None

    def scaled(self, n_rows: int, n_queries: int | None = None) -> "Workload":
        """Same distributions and method parameters, fewer rows (parity-test sizes)."""
        nc = self.data.n_clusters
        if nc:
            nc = max(1, min(nc, n_rows // (4 * max(1, self.data.cluster_size))))
        d = self.data.replace(n_rows=n_rows, n_clusters=nc)
        q = self.query_data
        nq = self.n_queries if n_queries is None else n_queries
        if q is not None:
            q = q.replace(n_rows=nq)
        if self.mode == "sampled_queries":
            nq = min(nq, n_rows)
        return dataclasses.replace(self, data=d, query_data=q, n_queries=nq)


def _workloads():
    w = {}
    w["tiny_plain"] = Workload(
        name="tiny_plain: N=10,000 rows, D=100,000, nnz U[20,200], Zipf(1.1) ids, 500x5 planted clusters; "
             "K=4 L=16 R=32 2^15 buckets; 100 sampled queries, k=10",
        data=DataSpec(n_rows=10_000, dim=100_000, len_kind="uniform", len_a=20, len_b=200,
                      id_kind="zipf", zipf_s=1.1, n_clusters=500, cluster_size=5, resample_frac=0.3,
                      seed=1001),
        params=MethodParams(K=4, L=16, R=32, range_bits=15, seed=0x5EEDF1A5 + 1),
        k=10, mode="sampled_queries", n_queries=100)
    w["webspam_like"] = Workload(
        name="webspam-like all-points k-NN graph: N=350,000, D=16,609,143, nnz lognormal mean 3,700 "
             "(sigma 1.0, clip [1,200000]), uniform ids, unit-L2 float32 values; K=4 L=64 R=64 2^18 buckets; k=128",
        data=DataSpec(n_rows=350_000, dim=16_609_143, len_kind="lognormal",
                      len_a=math.log(3700.0) - 0.5, len_b=1.0, clip_lo=1, clip_hi=200_000,
                      id_kind="uniform", seed=1002, with_val=True),
        params=MethodParams(K=4, L=64, R=64, range_bits=18, seed=0x5EEDF1A5 + 2),
        k=128, mode="graph")
    mu3 = _lognormal_mu_for_clipped_mean(116.0, 0.6, 400.0)
    url_rows = DataSpec(n_rows=2_400_000, dim=3_200_000, len_kind="lognormal", len_a=mu3, len_b=0.6,
                        clip_lo=1, clip_hi=400, id_kind="zipf", zipf_s=1.1, seed=1003)
    w["url_like_batched"] = Workload(
        name="url-like batched uneven queries: N=2,400,000, D=3,200,000, nnz lognormal mean 116 (max 400), "
             "Zipf(1.1) ids, binary; K=3 L=128 R=128 2^15 buckets; 1,000,000 fresh queries, k=64",
        data=url_rows,
        params=MethodParams(K=3, L=128, R=128, range_bits=15, seed=0x5EEDF1A5 + 3),
        k=64, mode="fresh_queries", n_queries=1_000_000,
        query_data=url_rows.replace(n_rows=1_000_000, seed=1003 + 1))
    w["kdd12_like"] = Workload(
        name="kdd12-like very sparse k-NN graph: N=10,000,000, D=54,700,000, nnz Poisson(11)+1, Zipf(1.2) ids, "
             "binary; K=4 L=256 R=32 2^20 buckets; k=32",
        data=DataSpec(n_rows=10_000_000, dim=54_700_000, len_kind="poisson1", len_a=11.0,
                      id_kind="zipf", zipf_s=1.2, seed=1004),
        params=MethodParams(K=4, L=256, R=32, range_bits=20, seed=0x5EEDF1A5 + 4),
        k=32, mode="graph")
    w["serving_url"] = Workload(
        name="serving loop on the url-like index: request batches U[1,4096] rows, Poisson arrivals, k=64",
        data=url_rows,
        params=MethodParams(K=3, L=128, R=128, range_bits=15, seed=0x5EEDF1A5 + 3),
        k=64, mode="serving", n_queries=1_000_000,
        query_data=url_rows.replace(n_rows=1_000_000, seed=1005))
    return w


WORKLOADS = _workloads()
WORKLOAD_ORDER = ["tiny_plain", "webspam_like", "url_like_batched", "kdd12_like", "serving_url"]

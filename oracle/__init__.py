"""CPU oracle for FLASH's hot path -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this package.  The product path (``paper_1709_01190_gb300``)
never imports it and shares no code with it.

The arithmetic lives in ``flash_oracle.c`` (plain C, one step per line of
the paper's definitions); this module compiles it with gcc and marshals
numpy arrays into it.  See the C file for the cited passages and readings.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "flash_oracle.c")
_OUT = os.path.join(_HERE, "_build")
_SO = os.path.join(_OUT, "libflash_oracle.so")
_LOCK = threading.Lock()
_LIB = None

_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_U32 = ctypes.c_uint32
_U64 = ctypes.c_uint64
_I32 = ctypes.c_int32


def build(force: bool = False) -> str:
    with _LOCK:
        if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
            return _SO
        os.makedirs(_OUT, exist_ok=True)
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-std=c99", "-Wall", "-shared", "-fPIC", _SRC, "-o", tmp], check=True)
        os.replace(tmp, _SO)
        return _SO


def _lib():
    global _LIB
    if _LIB is None:
        lib = ctypes.CDLL(build())
        lib.oracle_seeds.argtypes = [_U64, _P]
        lib.oracle_hash.argtypes = [_P, _P, _I64, _I64, _U32, _U32, _U64, _U32, _P]
        lib.oracle_keys.argtypes = [_P, _P, _I64, _I64, _U32, _U32, _U32, _U64, _U32, _P, _I64]
        lib.oracle_build.argtypes = [_P, _P, _I64, _U32, _U32, _U32, _U32, _U64, _U32, _P, _P]
        lib.oracle_add.argtypes = [_P, _P, _I64, _I32, _U32, _U32, _U32, _U32, _U64, _U32, _P, _P]
        lib.oracle_bucket.argtypes = [_P, _P, _I64, _U32, _U32, _U32, _U64, _P, _P]
        lib.oracle_kselect.argtypes = [_P, _I64, _I32, _I32, _P, _P]
        lib.oracle_query.argtypes = [_P, _P, _U32, _U32, _U32, _U32, _U64, _U32, _P, _P, _I64, _I32, _P, _P, _P]
        lib.oracle_query_one_streamed.argtypes = [_P, _I64, _P, _I64, _U32, _U32, _U64, _P, ctypes.c_int,
                                                  _I32, _I32, _P, _P]
        lib.oracle_knn_graph.argtypes = [_P, _P, _I64, _U32, _U32, _U32, _U32, _U64, _U32, _I32, _P, _P]
        lib.oracle_address.argtypes = [_P, _U32, _U32, _U32, _U32, _U64]
        lib.oracle_build_tables_from_keys.argtypes = [_P, _I64, _P, _I64, _U32, _U32, _U32, _U32, _U64, _P, _P]
        lib.oracle_address.restype = ctypes.c_uint32
        lib.oracle_pool_index.argtypes = [_U32, _U32, _U32, _U64]
        lib.oracle_pool_index.restype = ctypes.c_uint32
        lib.oracle_build_shared.argtypes = [_P, _P, _I64, _U32, _U32, _U32, _U32, _U64, _U32, _U32, _P, _P]
        lib.oracle_build_shared.restype = ctypes.c_int
        lib.oracle_query_shared.argtypes = [_P, _P, _U32, _U32, _U32, _U32, _U64, _U32, _U32, _P, _P, _I64, _I32,
                                            _P, _P, _P]
        lib.oracle_query_shared.restype = ctypes.c_int
        for f in ("oracle_hash", "oracle_keys", "oracle_build", "oracle_bucket", "oracle_kselect",
                  "oracle_query", "oracle_query_one_streamed", "oracle_knn_graph", "oracle_build_tables_from_keys"):
            getattr(lib, f).restype = ctypes.c_int
        _LIB = lib
    return _LIB


def _c(a, dtype):
    a = np.ascontiguousarray(a, dtype=dtype)
    return a, a.ctypes.data


def _check(rc):
    if rc != 0:
        raise MemoryError("oracle allocation failed")


def _workers(n_threads):
    if n_threads:
        return n_threads
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


def seeds(seed: int) -> dict:
    out = np.zeros(5, dtype=np.uint64)
    _lib().oracle_seeds(seed & ((1 << 64) - 1), out.ctypes.data)
    return dict(zip(("a1", "b1", "a2", "b2", "r"), (int(x) for x in out)))


def doph(row_ptr, col, K: int, L: int, seed: int, rows=None, n_threads=None, densify: int = 0) -> np.ndarray:
    """DOPH hashes, uint32 [n_rows][K*L] (Section 2.3 on Eq. 1); densify 0 = rotation, 1 = optimal."""
    rp, prp = _c(row_ptr, np.int64)
    cl, pcl = _c(col, np.int32)
    n = rp.shape[0] - 1
    B = K * L
    if rows is not None:
        rows = np.asarray(rows, dtype=np.int64)
        out = np.empty((len(rows), B), dtype=np.uint32)
        for i, r in enumerate(rows):
            _check(_lib().oracle_hash(prp, pcl, int(r), int(r) + 1, K, L, seed, densify, out[i].ctypes.data))
        return out
    out = np.empty((n, B), dtype=np.uint32)
    chunks = _chunks(n, _workers(n_threads))
    lib = _lib()

    def run(ab):
        a, b = ab
        _check(lib.oracle_hash(prp, pcl, a, b, K, L, seed, densify, out[a:b].ctypes.data if b > a else None))

    _pmap(run, chunks)
    return out


def keys(row_ptr, col, K: int, L: int, range_bits: int, seed: int, n_threads=None, densify: int = 0) -> np.ndarray:
    """Table addresses, uint32 [L][n_rows] (MapKHashesToAddress per table)."""
    rp, prp = _c(row_ptr, np.int64)
    cl, pcl = _c(col, np.int32)
    n = rp.shape[0] - 1
    out = np.empty((L, n), dtype=np.uint32)
    lib = _lib()

    def run(ab):
        a, b = ab
        if b > a:
            _check(lib.oracle_keys(prp, pcl, a, b, K, L, range_bits, seed, densify, out[:, a:].ctypes.data, n))

    _pmap(run, _chunks(n, _workers(n_threads)))
    return out


def address(h, t: int, K: int, L: int, range_bits: int, seed: int) -> int:
    """MapKHashesToAddress of table t for a given hash array h (uint32 [K*L])."""
    hh, ph = _c(h, np.uint32)
    assert hh.shape[0] == K * L
    return int(_lib().oracle_address(ph, t, K, L, range_bits, seed))


def build_tables(row_ptr, col, K, L, R, range_bits, seed, densify=0):
    """Adding phase (Algorithm 2).  Returns (tables int32 [L][2^rb][R], counts uint32 [L][2^rb])."""
    rp, prp = _c(row_ptr, np.int64)
    cl, pcl = _c(col, np.int32)
    n = rp.shape[0] - 1
    T = 1 << range_bits
    tables = np.empty((L, T, R), dtype=np.int32)
    counts = np.empty((L, T), dtype=np.uint32)
    _check(_lib().oracle_build(prp, pcl, n, K, L, R, range_bits, seed, densify, tables.ctypes.data,
                               counts.ctypes.data))
    return tables, counts


def add_rows(tables, counts, row_ptr, col, id0, K, L, R, range_bits, seed, densify=0):
    """Algorithm 2 continued: ADD rows [0, n) of (row_ptr, col) as points id0 + row into the
    given tables / counts (int32 [L][2^rb][R], uint32 [L][2^rb]), in place."""
    rp, prp = _c(row_ptr, np.int64)
    cl, pcl = _c(col, np.int32)
    assert tables.dtype == np.int32 and counts.dtype == np.uint32
    assert tables.flags.c_contiguous and counts.flags.c_contiguous
    _check(_lib().oracle_add(prp, pcl if cl.size else None, rp.shape[0] - 1, id0, K, L, R, range_bits, seed, densify,
                             tables.ctypes.data, counts.ctypes.data))


def bucket(keys_t, row_ptr, t, key, R, seed):
    """Reservoir of one bucket (Algorithm 1 on its arrival stream). Returns (slots int32[R], count)."""
    kt, pkt = _c(keys_t, np.uint32)
    rp, prp = _c(row_ptr, np.int64)
    res = np.empty(R, dtype=np.int32)
    cnt = np.zeros(1, dtype=np.uint32)
    _check(_lib().oracle_bucket(pkt, prp, kt.shape[0], t, int(key), R, seed, res.ctypes.data, cnt.ctypes.data))
    return res, int(cnt[0])


def kselect(A, k: int, exclude: int = -1):
    """KSELECT of Algorithm 3 on one candidate array."""
    a = np.array(A, dtype=np.int32, copy=True)
    ids = np.empty(k, dtype=np.int32)
    cnt = np.empty(k, dtype=np.int32)
    _check(_lib().oracle_kselect(a.ctypes.data if a.size else None, a.size, exclude, k, ids.ctypes.data,
                                 cnt.ctypes.data))
    return ids, cnt


def query(tables, counts, K, L, R, range_bits, seed, q_row_ptr, q_col, k, exclude=None, densify=0):
    """Querying phase (Algorithm 3).  Returns (ids int32 [nq][k], counts int32 [nq][k])."""
    tb, ptb = _c(tables, np.int32)
    ct, pct = _c(counts, np.uint32)
    rp, prp = _c(q_row_ptr, np.int64)
    cl, pcl = _c(q_col, np.int32)
    nq = rp.shape[0] - 1
    ids = np.empty((nq, k), dtype=np.int32)
    cnt = np.empty((nq, k), dtype=np.int32)
    ex = None
    if exclude is not None:
        ex, pex = _c(exclude, np.int32)
    _check(_lib().oracle_query(ptb, pct, K, L, R, range_bits, seed, densify, prp, pcl if cl.size else None, nq, k,
                               None if ex is None else pex, ids.ctypes.data, cnt.ctypes.data))
    return ids, cnt


def query_streamed(keys_all, row_ptr, L, R, seed, q_keys, q_empty, k, exclude=-1):
    """Algorithm 3 for one query with its buckets rebuilt from the arrival streams (large workloads)."""
    ka, pka = _c(keys_all, np.uint32)
    rp, prp = _c(row_ptr, np.int64)
    qk, pqk = _c(q_keys, np.uint32)
    ids = np.empty(k, dtype=np.int32)
    cnt = np.empty(k, dtype=np.int32)
    _check(_lib().oracle_query_one_streamed(pka, ka.shape[1], prp, ka.shape[1], L, R, seed, pqk, int(bool(q_empty)),
                                            k, exclude, ids.ctypes.data, cnt.ctypes.data))
    return ids, cnt


def knn_graph(row_ptr, col, K, L, R, range_bits, seed, k, densify=0):
    """All-points k-NN graph: build on all rows, query every row excluding itself."""
    rp, prp = _c(row_ptr, np.int64)
    cl, pcl = _c(col, np.int32)
    n = rp.shape[0] - 1
    ids = np.empty((n, k), dtype=np.int32)
    cnt = np.empty((n, k), dtype=np.int32)
    _check(_lib().oracle_knn_graph(prp, pcl if cl.size else None, n, K, L, R, range_bits, seed, densify, k,
                                   ids.ctypes.data, cnt.ctypes.data))
    return ids, cnt


def build_tables_threaded(row_ptr, col, K, L, R, range_bits, seed, n_threads=None, densify=0):
    """build_tables with the addresses computed on several threads (row blocks) and the tables
    built on several threads (each table is an independent Adding phase, Section 3.4); the
    result equals build_tables."""
    rp, prp = _c(row_ptr, np.int64)
    n = rp.shape[0] - 1
    T = 1 << range_bits
    ks = keys(row_ptr, col, K, L, range_bits, seed, n_threads, densify)
    tables = np.empty((L, T, R), dtype=np.int32)
    counts = np.empty((L, T), dtype=np.uint32)
    lib = _lib()

    def run(t):
        _check(lib.oracle_build_tables_from_keys(ks.ctypes.data, n, prp, n, t, t + 1, R, range_bits, seed,
                                                 tables.ctypes.data, counts.ctypes.data))

    _pmap(run, range(L))
    return tables, counts


def knn_graph_threaded(row_ptr, col, K, L, R, range_bits, seed, k, n_threads=None, densify=0):
    """knn_graph on several threads: build_tables_threaded, then the queries in row blocks; the
    result equals knn_graph."""
    rp, _ = _c(row_ptr, np.int64)
    cl, _ = _c(col, np.int32)
    n = rp.shape[0] - 1
    tables, counts = build_tables_threaded(rp, cl, K, L, R, range_bits, seed, n_threads, densify)
    ids = np.empty((n, k), dtype=np.int32)
    cnt = np.empty((n, k), dtype=np.int32)

    def run(ab):
        a, b = ab
        if b > a:
            sub_rp = rp[a:b + 1] - rp[a]
            i, c = query(tables, counts, K, L, R, range_bits, seed, sub_rp, cl[rp[a]:rp[b]], k,
                         exclude=np.arange(a, b, dtype=np.int32), densify=densify)
            ids[a:b] = i
            cnt[a:b] = c

    _pmap(run, _chunks(n, _workers(n_threads)))
    return ids, cnt


def _chunks(n, w):
    step = max(1, -(-n // (4 * w)))
    return [(a, min(n, a + step)) for a in range(0, n, step)] or [(0, 0)]


def _pmap(fn, items):
    items = list(items)
    if len(items) <= 1:
        for it in items:
            fn(it)
        return
    with ThreadPoolExecutor(max_workers=_workers(None)) as ex:
        list(ex.map(fn, items))


# ------------------------------------------------ reservoir sharing (Section 3.5)

def pool_index(t: int, b: int, P: int, seed: int) -> int:
    """The reservoir of the shared pool that bucket b of table t points to."""
    return int(_lib().oracle_pool_index(t, b, P, seed))


def build_tables_shared(row_ptr, col, K, L, R, range_bits, seed, P, densify=0):
    """Adding phase with reservoir sharing: (tables int32 [P][R], counts uint32 [P])."""
    rp, prp = _c(row_ptr, np.int64)
    cl, pcl = _c(col, np.int32)
    n = rp.shape[0] - 1
    tables = np.empty((P, R), dtype=np.int32)
    counts = np.empty(P, dtype=np.uint32)
    _check(_lib().oracle_build_shared(prp, pcl if cl.size else None, n, K, L, R, range_bits, seed, densify, P,
                                      tables.ctypes.data, counts.ctypes.data))
    return tables, counts


def query_shared(tables, counts, K, L, R, range_bits, seed, P, q_row_ptr, q_col, k, exclude=None, densify=0):
    """Querying phase with reservoir sharing.  Returns (ids int32 [nq][k], counts int32 [nq][k])."""
    tb, ptb = _c(tables, np.int32)
    ct, pct = _c(counts, np.uint32)
    rp, prp = _c(q_row_ptr, np.int64)
    cl, pcl = _c(q_col, np.int32)
    nq = rp.shape[0] - 1
    ids = np.empty((nq, k), dtype=np.int32)
    cnt = np.empty((nq, k), dtype=np.int32)
    ex = None
    if exclude is not None:
        ex, pex = _c(exclude, np.int32)
    _check(_lib().oracle_query_shared(ptb, pct, K, L, R, range_bits, seed, densify, P, prp,
                                      pcl if cl.size else None, nq, k, None if ex is None else pex,
                                      ids.ctypes.data, cnt.ctypes.data))
    return ids, cnt


def knn_graph_shared(row_ptr, col, K, L, R, range_bits, seed, k, P, densify=0):
    """All-points k-NN graph over an index with reservoir sharing."""
    rp, _ = _c(row_ptr, np.int64)
    cl, _ = _c(col, np.int32)
    n = rp.shape[0] - 1
    tables, counts = build_tables_shared(rp, cl, K, L, R, range_bits, seed, P, densify)
    return query_shared(tables, counts, K, L, R, range_bits, seed, P, rp, cl, k,
                        exclude=np.arange(n, dtype=np.int32), densify=densify)

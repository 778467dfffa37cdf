"""Continuous-batching query server over a resident FLASH index.

Requests are batches of query rows (CSR on the host) that arrive at any time.
A scheduler thread admits waiting requests in arrival order whenever a stream
slot is free and their device memory fits the budget, coalescing consecutive
waiting requests into one device batch (up to ``max_batch_rows``).  Each batch
runs on its own CUDA stream -- host->device copy of the rows, flash_query
(DOPH of the rows, gather, count, top-k), device->host copy of the results --
so batches admitted while others are still on the GPU overlap with them.  A
completion thread hands every request its own rows of the batch result and
frees the slot and the memory.

A query row's result depends only on the index and the row, never on the
rows it is batched with, so every request gets exactly the result it would
get alone (``tests/test_gpu_serving.py`` checks this).

The scheduling core (``Server``) does not touch CUDA; ``CudaBackend`` is the
GPU implementation and tests may substitute a host backend.
"""
from __future__ import annotations

import collections
import dataclasses
import threading
import time

import numpy as np


@dataclasses.dataclass
class Request:
    row_ptr: np.ndarray   # int64 [rows + 1]
    col: np.ndarray       # int32 [nnz]
    ticket: "Ticket"

    @property
    def rows(self) -> int:
        return int(self.row_ptr.shape[0] - 1)

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])


class Ticket:
    """Handle of one request: wait() returns (ids, counts), each int32 [rows][k]."""

    def __init__(self, rid: int, rows: int):
        self.rid = rid
        self.rows = rows
        self.t_submit = time.perf_counter()
        self.t_admit = None
        self.t_done = None
        self.batch_id = None
        self.ids = None
        self.counts = None
        self.error = None
        self._ev = threading.Event()

    def _finish(self, ids=None, counts=None, error=None):
        self.ids, self.counts, self.error = ids, counts, error
        self.t_done = time.perf_counter()
        self._ev.set()

    def done(self) -> bool:
        return self._ev.is_set()

    def wait(self, timeout: float | None = None):
        if not self._ev.wait(timeout):
            raise TimeoutError(f"request {self.rid} not finished after {timeout} s")
        if self.error is not None:
            raise self.error
        return self.ids, self.counts

    @property
    def latency(self) -> float | None:
        return None if self.t_done is None else self.t_done - self.t_submit


@dataclasses.dataclass
class Batch:
    bid: int
    requests: list
    rows: int
    nnz: int
    nbytes: int
    slot: int = -1
    handle: object = None


class Server:
    """Continuous-batching scheduler.

    backend must provide: ``n_slots``, ``k``, ``batch_bytes(rows, nnz)``,
    ``launch(slot, batch) -> handle`` (asynchronous), ``poll(handle) -> bool``,
    ``wait(handle)`` (block until done) and ``results(handle)`` returning
    (ids, counts) for the whole batch in request order.
    """

    def __init__(self, backend, mem_budget: int = 8 << 30, max_batch_rows: int = 8192, coalesce: bool = True):
        self.backend = backend
        self.mem_budget = int(mem_budget)
        self.max_batch_rows = int(max_batch_rows)
        self.coalesce = coalesce
        self._pending = collections.deque()
        self._inflight = collections.deque()
        self._free_slots = list(range(backend.n_slots))
        self._budget_used = 0
        self._peak_budget = 0
        self._lock = threading.Lock()
        self._cv = threading.Condition(self._lock)
        self._stop = False
        self._next_rid = 0
        self._next_bid = 0
        self.tickets = []
        self.batches_launched = 0
        self.max_concurrent = 0
        self._sched = threading.Thread(target=self._schedule_loop, name="flash-serve-sched", daemon=True)
        self._compl = threading.Thread(target=self._complete_loop, name="flash-serve-done", daemon=True)
        self._sched.start()
        self._compl.start()

    # ------------------------------------------------------------- client API
    def submit(self, row_ptr: np.ndarray, col: np.ndarray) -> Ticket:
        """Queue a request of rows (CSR on the host); returns at once."""
        row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
        col = np.ascontiguousarray(col[int(row_ptr[0]):int(row_ptr[-1])], dtype=np.int32)
        row_ptr = row_ptr - row_ptr[0]
        with self._cv:
            if self._stop:
                raise RuntimeError("server is closed")
            t = Ticket(self._next_rid, int(row_ptr.shape[0] - 1))
            self._next_rid += 1
            self.tickets.append(t)
            req = Request(row_ptr, col, t)
            if self.backend.batch_bytes(req.rows, req.nnz) > self.mem_budget:
                from ._lib import FlashError
                t._finish(error=FlashError(2, f"request {t.rid} needs more device memory than the serving budget"))
                return t
            self._pending.append(req)
            self._cv.notify_all()
        return t

    def close(self, drain: bool = True, timeout: float = 60.0) -> None:
        if drain:
            deadline = time.perf_counter() + timeout
            with self._cv:
                while (self._pending or self._inflight) and time.perf_counter() < deadline:
                    self._cv.wait(0.05)
        with self._cv:
            self._stop = True
            self._cv.notify_all()
        self._sched.join(timeout)
        self._compl.join(timeout)

    def stats(self) -> dict:
        lat = np.array([t.latency for t in self.tickets if t.latency is not None and t.error is None])
        rows = sum(t.rows for t in self.tickets if t.done() and t.error is None)
        out = {"requests": len(lat), "rows": rows, "batches": self.batches_launched,
               "max_concurrent_batches": self.max_concurrent, "peak_budget_bytes": self._peak_budget}
        if len(lat):
            out.update(p50_ms=float(np.percentile(lat, 50) * 1e3), p99_ms=float(np.percentile(lat, 99) * 1e3),
                       mean_ms=float(lat.mean() * 1e3))
        return out

    # ------------------------------------------------------------- scheduling
    def _take_batch(self) -> Batch | None:
        """Called with the lock held: the longest admissible prefix of the queue."""
        if not self._pending or not self._free_slots:
            return None
        first = self._pending[0]
        rows, nnz = first.rows, first.nnz
        nbytes = self.backend.batch_bytes(rows, nnz)
        if self._budget_used + nbytes > self.mem_budget:
            return None
        reqs = [self._pending.popleft()]
        while self.coalesce and self._pending:
            nxt = self._pending[0]
            r2, z2 = rows + nxt.rows, nnz + nxt.nnz
            b2 = self.backend.batch_bytes(r2, z2)
            if r2 > self.max_batch_rows or self._budget_used + b2 > self.mem_budget:
                break
            reqs.append(self._pending.popleft())
            rows, nnz, nbytes = r2, z2, b2
        b = Batch(self._next_bid, reqs, rows, nnz, nbytes)
        self._next_bid += 1
        b.slot = self._free_slots.pop()
        self._budget_used += nbytes
        self._peak_budget = max(self._peak_budget, self._budget_used)
        return b

    def _schedule_loop(self):
        while True:
            with self._cv:
                b = None
                while not self._stop:
                    b = self._take_batch()
                    if b is not None:
                        break
                    self._cv.wait(0.05)
                if b is None:
                    return
            now = time.perf_counter()
            for r in b.requests:
                r.ticket.t_admit = now
                r.ticket.batch_id = b.bid
            try:
                b.handle = self.backend.launch(b.slot, b)
            except Exception as e:  # launch failed: fail its requests, free its resources
                for r in b.requests:
                    r.ticket._finish(error=e)
                with self._cv:
                    self._free_slots.append(b.slot)
                    self._budget_used -= b.nbytes
                    self._cv.notify_all()
                continue
            with self._cv:
                self._inflight.append(b)
                self.batches_launched += 1
                self.max_concurrent = max(self.max_concurrent, len(self._inflight))
                self._cv.notify_all()

    def _complete_loop(self):
        while True:
            with self._cv:
                while not self._stop and not self._inflight:
                    self._cv.wait(0.05)
                if self._stop and not self._inflight:
                    return
                batches = list(self._inflight)
            done = [b for b in batches if self.backend.poll(b.handle)]
            if not done:
                self.backend.wait(batches[0].handle)  # oldest batch first; frees the GIL while waiting
                done = [batches[0]]
            for b in done:
                try:
                    ids, counts = self.backend.results(b.handle)
                    off = 0
                    for r in b.requests:
                        r.ticket._finish(ids[off:off + r.rows].copy(), counts[off:off + r.rows].copy())
                        off += r.rows
                except Exception as e:
                    for r in b.requests:
                        if not r.ticket.done():
                            r.ticket._finish(error=e)
                with self._cv:
                    self._inflight.remove(b)
                    self._free_slots.append(b.slot)
                    self._budget_used -= b.nbytes
                    self._cv.notify_all()


def concat_requests(requests) -> tuple[np.ndarray, np.ndarray]:
    """One CSR holding the rows of the requests in order (each request's row_ptr starts at 0)."""
    rows = sum(r.rows for r in requests)
    rp = np.empty(rows + 1, dtype=np.int64)
    rp[0] = 0
    o, z = 0, 0
    for r in requests:
        rp[o + 1:o + r.rows + 1] = r.row_ptr[1:] + z
        o += r.rows
        z += r.nnz
    col = np.concatenate([r.col for r in requests]) if requests else np.zeros(0, np.int32)
    return rp, col


class CudaBackend:
    """Runs batches with flash_query on a pool of CUDA streams (one per slot)."""

    def __init__(self, index, k: int, dim: int, n_slots: int = 4, device=None):
        import torch
        from . import flash_query_scratch_bytes
        self.torch = torch
        self.index = index
        self.dim = int(dim)
        self.k = int(k)
        self.n_slots = int(n_slots)
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.streams = [torch.cuda.Stream(device=self.device) for _ in range(self.n_slots)]
        self._scratch = lambda rows: flash_query_scratch_bytes(index.params, rows)
        self._bufs = [None] * self.n_slots

    def batch_bytes(self, rows: int, nnz: int) -> int:
        """Device bytes one batch holds while in flight: its CSR, its results (each rounded to the
        caching allocator's 512-byte blocks) and the library's scratch for it."""
        def blk(nb):
            return (nb + 511) // 512 * 512
        return (blk(8 * (rows + 1)) + blk(4 * max(nnz, 1)) + 2 * blk(4 * rows * self.k) +
                self._scratch(rows))

    def _host_buffers(self, slot: int, rows: int, nnz: int):
        """Pinned host staging of a slot, grown to the largest batch the slot has seen (host memory
        only: the device buffers of a batch live exactly as long as the batch, see launch)."""
        torch = self.torch
        b = self._bufs[slot]
        if b is None or b["rows"] < rows or b["nnz"] < nnz:
            R = max(rows, b["rows"] if b else 0, 256)
            Z = max(nnz, b["nnz"] if b else 0, 4096)
            b = {"rows": R, "nnz": Z,
                 "h_rp": torch.empty(R + 1, dtype=torch.int64, pin_memory=True),
                 "h_col": torch.empty(Z, dtype=torch.int32, pin_memory=True),
                 "h_ids": torch.empty(R * self.k, dtype=torch.int32, pin_memory=True),
                 "h_cnt": torch.empty(R * self.k, dtype=torch.int32, pin_memory=True)}
            self._bufs[slot] = b
        return b

    def launch(self, slot: int, batch: Batch):
        torch = self.torch
        from . import DeviceCSR, flash_query
        rp, col = concat_requests(batch.requests)
        rows, nnz = batch.rows, int(rp[-1])
        b = self._host_buffers(slot, rows, nnz)
        s = self.streams[slot]
        b["h_rp"][:rows + 1].numpy()[:] = rp
        if nnz:
            b["h_col"][:nnz].numpy()[:] = col
        with torch.cuda.stream(s):
            # device buffers sized for this batch (the bytes batch_bytes admitted); they are
            # released when the batch completes, so device memory held by the server is exactly
            # that of the batches in flight (torch's caching allocator reuses the blocks)
            d_rp = torch.empty(rows + 1, dtype=torch.int64, device=self.device)
            d_col = torch.empty(max(nnz, 1), dtype=torch.int32, device=self.device)
            d_ids = torch.empty((rows, self.k), dtype=torch.int32, device=self.device)
            d_cnt = torch.empty((rows, self.k), dtype=torch.int32, device=self.device)
            d_rp.copy_(b["h_rp"][:rows + 1], non_blocking=True)
            if nnz:
                d_col[:nnz].copy_(b["h_col"][:nnz], non_blocking=True)
            x = DeviceCSR(d_rp, d_col, self.dim, nnz=nnz)
            flash_query(self.index, x, self.k, None, d_ids, d_cnt, s)
            b["h_ids"][:rows * self.k].copy_(d_ids.view(-1), non_blocking=True)
            b["h_cnt"][:rows * self.k].copy_(d_cnt.view(-1), non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(s)
        return {"ev": ev, "slot": slot, "rows": rows, "dev": (d_rp, d_col, d_ids, d_cnt)}

    def poll(self, h) -> bool:
        return h["ev"].query()

    def wait(self, h) -> None:
        h["ev"].synchronize()

    def results(self, h):
        h["ev"].synchronize()
        h["dev"] = None  # the batch is complete: its device buffers go back to the allocator
        b = self._bufs[h["slot"]]
        rows = h["rows"]
        ids = b["h_ids"][:rows * self.k].numpy().reshape(rows, self.k)
        cnt = b["h_cnt"][:rows * self.k].numpy().reshape(rows, self.k)
        return ids, cnt


def plain_serve(index, k: int, requests, dim: int, stream=None):
    """The unbatched baseline: one request at a time on one stream (copy in, query, copy out, wait)."""
    import torch
    from . import DeviceCSR, flash_query
    out = []
    for rp, col in requests:
        rows = rp.shape[0] - 1
        x = DeviceCSR(torch.from_numpy(rp).cuda(non_blocking=True), torch.from_numpy(col).cuda(non_blocking=True),
                      dim, nnz=int(rp[-1]))
        ids = torch.empty((rows, k), dtype=torch.int32, device="cuda")
        cnt = torch.empty((rows, k), dtype=torch.int32, device="cuda")
        flash_query(index, x, k, None, ids, cnt, stream)
        out.append((ids.cpu().numpy(), cnt.cpu().numpy()))
    return out

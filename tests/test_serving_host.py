"""Host-side logic of the continuous-batching server (no GPU): coalescing,
admission by memory budget and free slots, FIFO order, per-request results,
rejection of oversize requests, draining on close.  A host backend stands in
for CUDA: it "computes" a deterministic per-row result after a delay."""
import threading
import time

import numpy as np
import pytest

from paper_1709_01190_gb300.serve import Server, concat_requests


class HostBackend:
    def __init__(self, n_slots=3, k=4, delay=0.01):
        self.n_slots, self.k, self.delay = n_slots, k, delay
        self.launched = []
        self.live = 0
        self.max_live = 0
        self.lock = threading.Lock()

    def batch_bytes(self, rows, nnz):
        return 100 * rows + 4 * nnz

    def launch(self, slot, batch):
        rp, col = concat_requests(batch.requests)
        with self.lock:
            self.launched.append((slot, [r.ticket.rid for r in batch.requests], batch.nbytes))
            self.live += 1
            self.max_live = max(self.max_live, self.live)
        h = {"t": time.perf_counter() + self.delay, "rp": rp, "col": col}
        return h

    def poll(self, h):
        return time.perf_counter() >= h["t"]

    def wait(self, h):
        while not self.poll(h):
            time.sleep(0.001)

    def results(self, h):
        with self.lock:
            self.live -= 1
        rp, col = h["rp"], h["col"]
        rows = rp.shape[0] - 1
        ids = np.zeros((rows, self.k), np.int32)
        cnt = np.zeros((rows, self.k), np.int32)
        for i in range(rows):
            seg = col[rp[i]:rp[i + 1]]
            ids[i, 0] = int(seg.sum()) if seg.size else -1
            cnt[i, 0] = seg.size
        return ids, cnt


def make_request(rng, rows):
    lens = rng.integers(0, 6, rows)
    rp = np.zeros(rows + 1, np.int64)
    rp[1:] = np.cumsum(lens)
    col = rng.integers(0, 1000, int(rp[-1])).astype(np.int32)
    return rp, col


def expected(rp, col, k):
    rows = rp.shape[0] - 1
    ids = np.zeros((rows, k), np.int32)
    cnt = np.zeros((rows, k), np.int32)
    for i in range(rows):
        seg = col[rp[i]:rp[i + 1]]
        ids[i, 0] = int(seg.sum()) if seg.size else -1
        cnt[i, 0] = seg.size
    return ids, cnt


def test_every_request_gets_its_own_rows_and_batches_coalesce():
    rng = np.random.default_rng(0)
    be = HostBackend(n_slots=2, delay=0.02)
    srv = Server(be, mem_budget=10 ** 9, max_batch_rows=64)
    reqs = [make_request(rng, int(rng.integers(1, 20))) for _ in range(60)]
    tickets = [srv.submit(rp, col) for rp, col in reqs]
    for (rp, col), t in zip(reqs, tickets):
        ids, cnt = t.wait(10)
        ei, ec = expected(rp, col, be.k)
        assert np.array_equal(ids, ei) and np.array_equal(cnt, ec)
    srv.close()
    st = srv.stats()
    assert st["requests"] == 60
    assert st["batches"] < 60                       # waiting requests were coalesced
    assert be.max_live <= 2 and st["max_concurrent_batches"] >= 2
    admitted = [rid for _, rids, _ in be.launched for rid in rids]
    assert admitted == sorted(admitted)             # FIFO


def test_budget_is_never_exceeded_and_oversize_is_rejected():
    rng = np.random.default_rng(1)
    be = HostBackend(n_slots=4, delay=0.01)
    budget = 3000
    srv = Server(be, mem_budget=budget, max_batch_rows=1000)
    reqs = [make_request(rng, int(rng.integers(1, 12))) for _ in range(40)]
    tickets = [srv.submit(rp, col) for rp, col in reqs]
    big = make_request(rng, 40)                      # 100 * 40 > budget
    tb = srv.submit(*big)
    for t in tickets:
        t.wait(10)
    with pytest.raises(Exception):
        tb.wait(1)
    srv.close()
    assert srv.stats()["peak_budget_bytes"] <= budget
    live_bytes_ok = all(nb <= budget for _, _, nb in be.launched)
    assert live_bytes_ok


def test_requests_arriving_while_others_run_are_admitted():
    rng = np.random.default_rng(2)
    be = HostBackend(n_slots=2, delay=0.05)
    srv = Server(be, mem_budget=10 ** 9, max_batch_rows=8, coalesce=True)
    first = [srv.submit(*make_request(rng, 8)) for _ in range(2)]   # fill both slots
    time.sleep(0.01)
    late = [srv.submit(*make_request(rng, 3)) for _ in range(4)]     # arrive while those run
    for t in first + late:
        t.wait(10)
    srv.close()
    assert all(t.t_admit >= first[0].t_admit for t in late)
    assert len({t.batch_id for t in late}) < len(late)               # late arrivals share a batch


def test_close_drains_the_queue():
    rng = np.random.default_rng(3)
    be = HostBackend(n_slots=1, delay=0.005)
    srv = Server(be, mem_budget=10 ** 9, max_batch_rows=4)
    ts = [srv.submit(*make_request(rng, 3)) for _ in range(20)]
    srv.close(drain=True, timeout=30)
    assert all(t.done() for t in ts)
    with pytest.raises(RuntimeError):
        srv.submit(*make_request(rng, 1))

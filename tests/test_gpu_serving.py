"""Serving loop, launch knobs and CUDA-graph capture on the GPU, against the oracle.

* Every request served in a mix (coalesced with others, overlapping on several
  streams) gets exactly the oracle's result for its rows (Algorithm 3 on the
  oracle's tables), the same as it gets alone through flash_query, and the
  plain one-at-a-time path agrees too (integer results: exact).
* Under every launch knob (count-table size, rows per claim, row order) the
  k-NN graph equals the oracle's; the autotuner leaves a valid setting.
* Every CUDA-graph replay of flash_knn_graph equals the oracle's graph.
"""
import numpy as np
import pytest

import oracle
from paper_1709_01190_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1709_01190_gb300 as fl  # noqa: E402
from paper_1709_01190_gb300 import serve, tuning  # noqa: E402


@pytest.fixture(scope="module")
def url_index():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    fl.build()
    w = synth.WORKLOADS["url_like_batched"].scaled(30_000, n_queries=6_000)
    c = synth.generate(w.data)
    p = w.params
    params = fl.FlashParams(p.K, p.L, p.R, 13, p.seed)
    ix = fl.flash_build(params, fl.DeviceCSR.from_host(c))
    q = synth.generate(w.query_data)
    yield ix, q, c.dim, w.k, c
    ix.free()


@pytest.fixture(scope="module")
def url_oracle(url_index):
    """The oracle's answers for every query row of url_index (tables built by Algorithm 2)."""
    ix, q, dim, k, c = url_index
    p = ix.params
    et, ec = oracle.build_tables(c.row_ptr, c.col, p.K, p.L, p.R, p.range_bits, p.seed)
    return oracle.query(et, ec, p.K, p.L, p.R, p.range_bits, p.seed, q.row_ptr, q.col, k)


def _split(q, sizes):
    out, r0 = [], 0
    for s in sizes:
        sub = q.rows(np.arange(r0, r0 + s))
        out.append((sub.row_ptr, sub.col))
        r0 += s
    return out


def test_served_results_equal_oracle_and_alone_results(url_index, url_oracle):
    ix, q, dim, k, _ = url_index
    oi, oc = url_oracle
    rng = np.random.default_rng(0)
    sizes = []
    total = 0
    while total < q.n_rows - 300:
        s = int(rng.integers(1, 300))
        sizes.append(s)
        total += s
    reqs = _split(q, sizes)
    alone = []
    for rp, col in reqs:
        ids, cnt = fl.query(ix, fl.DeviceCSR(torch.from_numpy(rp).cuda(), torch.from_numpy(col).cuda(), dim), k)
        alone.append((ids.cpu().numpy(), cnt.cpu().numpy()))
    be = serve.CudaBackend(ix, k, dim, n_slots=3)
    srv = serve.Server(be, mem_budget=1 << 30, max_batch_rows=1024)
    tickets = [srv.submit(rp, col) for rp, col in reqs]
    r0 = 0
    for t, s, (ai, ac) in zip(tickets, sizes, alone):
        ids, cnt = t.wait(60)
        # the oracle's answer for these rows, element by element
        assert np.array_equal(ids, oi[r0:r0 + s]) and np.array_equal(cnt, oc[r0:r0 + s]), f"request at row {r0}"
        # and the same as the request alone
        assert np.array_equal(ids, ai) and np.array_equal(cnt, ac)
        r0 += s
    srv.close()
    st = srv.stats()
    assert st["batches"] < len(reqs)          # requests were coalesced into shared device batches
    plain = serve.plain_serve(ix, k, reqs[:20], dim)
    r0 = 0
    for (pi, pc), s in zip(plain, sizes[:20]):
        assert np.array_equal(pi, oi[r0:r0 + s]) and np.array_equal(pc, oc[r0:r0 + s])
        r0 += s


def test_tight_memory_budget_still_serves_everything(url_index, url_oracle):
    ix, q, dim, k, _ = url_index
    oi, oc = url_oracle
    reqs = _split(q, [500] * 6)
    be = serve.CudaBackend(ix, k, dim, n_slots=4)
    one = be.batch_bytes(500, int(max(rp[-1] for rp, _ in reqs)))
    srv = serve.Server(be, mem_budget=int(one * 1.5), max_batch_rows=4096)
    tickets = [srv.submit(rp, col) for rp, col in reqs]
    for i, t in enumerate(tickets):
        ids, cnt = t.wait(60)
        assert np.array_equal(ids, oi[500 * i:500 * (i + 1)]) and np.array_equal(cnt, oc[500 * i:500 * (i + 1)])
    srv.close()
    assert srv.stats()["peak_budget_bytes"] <= int(one * 1.5)


KNOBS = [tuning.Tuning(query_warp_table=256), tuning.Tuning(query_warp_table=2048),
         tuning.Tuning(doph_order=1), tuning.Tuning(doph_rows_per_grab=1), tuning.Tuning(doph_rows_per_grab=64),
         tuning.Tuning(query_warp_table=128, doph_order=1, doph_rows_per_grab=3)]


@pytest.mark.parametrize("name,n", [("webspam_like", 1500), ("url_like_batched", 12_000)])
def test_launch_knobs_do_not_change_results(name, n):
    w = synth.WORKLOADS[name].scaled(n)
    c = synth.generate(w.data)
    p = w.params
    params = fl.FlashParams(p.K, p.L, p.R, 12, p.seed)
    dev = fl.DeviceCSR.from_host(c)
    ei, en = oracle.knn_graph(c.row_ptr, c.col, params.K, params.L, params.R, params.range_bits, params.seed, w.k)
    eh = oracle.doph(c.row_ptr, c.col, params.K, params.L, params.seed)
    try:
        for t in [None] + KNOBS:
            tuning.set_tuning(t)
            got = fl.knn_graph(params, dev, w.k)
            assert np.array_equal(got[0].cpu().numpy(), ei) and np.array_equal(got[1].cpu().numpy(), en), t
            assert np.array_equal(fl.hash_rows(params, dev).cpu().numpy().view(np.uint32), eh), t
    finally:
        tuning.set_tuning(None)


def test_autotune_and_graph_replay(tmp_path, monkeypatch):
    monkeypatch.setenv("FLASH_TUNING_CACHE", str(tmp_path / "tuning.json"))
    w = synth.WORKLOADS["tiny_plain"].scaled(6000)
    c = synth.generate(w.data)
    p = w.params
    params = fl.FlashParams(p.K, p.L, p.R, p.range_bits, p.seed)
    dev = fl.DeviceCSR.from_host(c)
    tuning.set_tuning(None)
    ei, en = oracle.knn_graph(c.row_ptr, c.col, p.K, p.L, p.R, p.range_bits, p.seed, w.k)
    key = tuning.shape_key("graph", params, c.n_rows, c.nnz, w.k)
    try:
        best, ms = tuning.autotune(lambda: fl.knn_graph(params, dev, w.k), key=key, reps=2)
        assert ms > 0 and tuning.get_tuning() == best
        again, _ = tuning.autotune(lambda: fl.knn_graph(params, dev, w.k), key=key, reps=2)
        assert again == best                       # cached
        got = fl.knn_graph(params, dev, w.k)  # under the tuned knobs
        assert np.array_equal(got[0].cpu().numpy(), ei) and np.array_equal(got[1].cpu().numpy(), en)
        g = tuning.GraphedKnnGraph(params, dev, w.k)
        for _ in range(3):
            ids, cnt = g.replay()
            torch.cuda.synchronize()
            assert np.array_equal(ids.cpu().numpy(), ei) and np.array_equal(cnt.cpu().numpy(), en)
    finally:
        tuning.set_tuning(None)

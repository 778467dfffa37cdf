"""Parity at the full workload sizes, in the launch configuration the bench uses.

The oracle cannot rebuild these indexes whole in seconds, so it checks sampled
outputs one by one: it hashes every row (threads over row blocks; each row's
hashes depend on that row only), rebuilds the reservoirs of each sampled
query's L buckets from their arrival streams (Algorithm 1 on the points of the
bucket in index order) and runs KSELECT (Algorithm 3).  Every table address of
every row is compared too.  Integer results: exact.
"""
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import oracle
from paper_1709_01190_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]

import paper_1709_01190_gb300 as fl  # noqa: E402
from paper_1709_01190_gb300 import serve  # noqa: E402


def _threads():
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    fl.build()


def _params(w, **over):
    p = w.params
    d = dict(K=p.K, L=p.L, R=p.R, range_bits=p.range_bits, seed=p.seed)
    d.update(over)
    return fl.FlashParams(**d)


def _check_queries(keys_all, row_ptr, p, q_keys, q_empty, k, got_ids, got_cnt, excludes):
    def one(i):
        ei, ec = oracle.query_streamed(keys_all, row_ptr, p.L, p.R, p.seed, q_keys[:, i], q_empty[i], k, excludes[i])
        return i, ei, ec

    with ThreadPoolExecutor(max_workers=_threads()) as ex:
        for i, ei, ec in ex.map(one, range(q_keys.shape[1])):
            assert np.array_equal(got_ids[i], ei), f"query {i}: ids differ"
            assert np.array_equal(got_cnt[i], ec), f"query {i}: counts differ"


def _keys_equal(gpu_keys, exp, row_ptr, rb):
    exp = exp.copy()
    exp[:, np.diff(row_ptr) == 0] = 1 << rb
    assert np.array_equal(gpu_keys, exp)


def test_webspam_like_graph_full_size():
    w = synth.WORKLOADS["webspam_like"]
    c = synth.generate(w.data.replace(with_val=False))
    p = _params(w)
    dev = fl.DeviceCSR.from_host(c)
    ids, cnt = fl.knn_graph(p, dev, w.k)
    gpu_keys = fl.row_keys(p, dev).cpu().numpy().view(np.uint32)
    sample = synth.sample_rows(c.n_rows, 300, seed=11)
    gpu_hash = fl.hash_rows(p, dev)[torch.from_numpy(sample).cuda()].cpu().numpy().view(np.uint32)
    ids, cnt = ids.cpu().numpy(), cnt.cpu().numpy()
    del dev
    torch.cuda.empty_cache()
    assert np.array_equal(gpu_hash, oracle.doph(c.row_ptr, c.col, p.K, p.L, p.seed, rows=sample))
    keys_all = oracle.keys(c.row_ptr, c.col, p.K, p.L, p.range_bits, p.seed)
    _keys_equal(gpu_keys, keys_all, c.row_ptr, p.range_bits)
    qs = sample[:48]
    empty = np.diff(c.row_ptr)[qs] == 0
    _check_queries(keys_all, c.row_ptr, p, keys_all[:, qs], empty, w.k, ids[qs], cnt[qs], qs.astype(np.int32))


def test_url_like_index_and_batched_queries_full_size():
    w = synth.WORKLOADS["url_like_batched"]
    c = synth.generate(w.data)
    qc = synth.generate(w.query_data)
    p = _params(w)
    ix = fl.flash_build(p, fl.DeviceCSR.from_host(c))
    dq = fl.DeviceCSR.from_host(qc)
    ids, cnt = fl.query(ix, dq, w.k)
    ids, cnt = ids.cpu().numpy(), cnt.cpu().numpy()
    gpu_qkeys = fl.row_keys(p, dq).cpu().numpy().view(np.uint32)
    keys_all = oracle.keys(c.row_ptr, c.col, p.K, p.L, p.range_bits, p.seed)
    gpu_keys = fl.row_keys(p, fl.DeviceCSR.from_host(c)).cpu().numpy().view(np.uint32)
    _keys_equal(gpu_keys, keys_all, c.row_ptr, p.range_bits)
    qs = synth.sample_rows(qc.n_rows, 24, seed=12)
    sub = qc.rows(qs)
    qk = oracle.keys(sub.row_ptr, sub.col, p.K, p.L, p.range_bits, p.seed)
    _keys_equal(gpu_qkeys[:, qs], qk, sub.row_ptr, p.range_bits)
    _check_queries(keys_all, c.row_ptr, p, qk, np.diff(sub.row_ptr) == 0, w.k, ids[qs], cnt[qs],
                   np.full(len(qs), -1, np.int32))
    # served requests (several overlapping, coalesced) return the same rows as the batched launch
    be = serve.CudaBackend(ix, w.k, c.dim, n_slots=3)
    srv = serve.Server(be, mem_budget=4 << 30, max_batch_rows=8192)
    starts = [0, 5000, 9000, 9001, 20000, 600000]
    sizes = [4096, 1, 2500, 300, 4000, 1234]
    tickets = []
    for s0, sz in zip(starts, sizes):
        part = qc.slice(s0, s0 + sz)
        tickets.append((s0, sz, srv.submit(part.row_ptr, part.col)))
    served_i, served_c, served_rows = [], [], []
    for s0, sz, t in tickets:
        si, sc = t.wait(120)
        assert np.array_equal(si, ids[s0:s0 + sz]) and np.array_equal(sc, cnt[s0:s0 + sz])
        served_i.append(si)
        served_c.append(sc)
        served_rows.append(np.arange(s0, s0 + sz))
    srv.close()
    ix.free()
    # rows the served requests carried, checked one by one against the oracle (Algorithm 3 on the
    # buckets rebuilt from their arrival streams): a few from every request, 320 in all
    served_i = np.concatenate(served_i)
    served_c = np.concatenate(served_c)
    served_rows = np.concatenate(served_rows)
    rng = np.random.default_rng(21)
    first_rows = np.flatnonzero(np.isin(served_rows, starts))  # the first row of every request
    pick = np.unique(np.concatenate([first_rows, rng.choice(len(served_rows), 320, replace=False)]))
    sub = qc.rows(served_rows[pick])
    qk = oracle.keys(sub.row_ptr, sub.col, p.K, p.L, p.range_bits, p.seed)
    _check_queries(keys_all, c.row_ptr, p, qk, np.diff(sub.row_ptr) == 0, w.k, served_i[pick], served_c[pick],
                   np.full(len(pick), -1, np.int32))


def test_kdd12_like_graph_full_size():
    w = synth.WORKLOADS["kdd12_like"]
    c = synth.generate(w.data)
    p = _params(w)
    dev = fl.DeviceCSR.from_host(c)
    ids, cnt = fl.knn_graph(p, dev, w.k)
    sample = synth.sample_rows(c.n_rows, 32, seed=13)
    sel = torch.from_numpy(sample).cuda()
    ids, cnt = ids[sel].cpu().numpy(), cnt[sel].cpu().numpy()
    gpu_hash = fl.hash_rows(p, fl.DeviceCSR.from_host(c.rows(sample))).cpu().numpy().view(np.uint32)
    del dev
    torch.cuda.empty_cache()
    assert np.array_equal(gpu_hash, oracle.doph(c.row_ptr, c.col, p.K, p.L, p.seed, rows=sample))
    keys_all = oracle.keys(c.row_ptr, c.col, p.K, p.L, p.range_bits, p.seed)
    empty = np.diff(c.row_ptr)[sample] == 0
    _check_queries(keys_all, c.row_ptr, p, keys_all[:, sample], empty, w.k, ids, cnt, sample.astype(np.int32))

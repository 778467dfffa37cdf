"""The threaded oracle drivers (addresses in row blocks, one Adding phase per table, queries in
row blocks) give exactly the single-threaded oracle's tables and graph.  CPU only."""
import numpy as np
import pytest

import oracle
from paper_1709_01190_gb300 import synth


@pytest.mark.parametrize("name,n,over", [("tiny_plain", 3_000, dict(range_bits=7, R=8)),
                                         ("kdd12_like", 4_000, dict(range_bits=9, L=16, R=4)),
                                         ("url_like_batched", 2_000, dict(range_bits=8, L=8))])
def test_threaded_oracle_equals_single_threaded(name, n, over):
    w = synth.WORKLOADS[name].scaled(n)
    c = synth.generate(w.data)
    p = dict(K=w.params.K, L=w.params.L, R=w.params.R, range_bits=w.params.range_bits, seed=w.params.seed)
    p.update(over)
    et, ec = oracle.build_tables(c.row_ptr, c.col, p["K"], p["L"], p["R"], p["range_bits"], p["seed"])
    tt, tc = oracle.build_tables_threaded(c.row_ptr, c.col, p["K"], p["L"], p["R"], p["range_bits"], p["seed"],
                                          n_threads=4)
    assert np.array_equal(et, tt) and np.array_equal(ec, tc)
    ei, en = oracle.knn_graph(c.row_ptr, c.col, p["K"], p["L"], p["R"], p["range_bits"], p["seed"], w.k)
    ti, tn = oracle.knn_graph_threaded(c.row_ptr, c.col, p["K"], p["L"], p["R"], p["range_bits"], p["seed"], w.k,
                                       n_threads=4)
    assert np.array_equal(ei, ti) and np.array_equal(en, tn)
